/*
 * Host memory and undefined-behaviour check of the FPW oracle (test
 * infrastructure, like the oracle itself): tests/test_oracle_sanitizers.py
 * compiles this file together with fpw_oracle.c under AddressSanitizer and
 * UndefinedBehaviorSanitizer and runs it. It calls every oracle entry point on
 * small seeded inputs, including the edge cases (no observations, no
 * frequencies, one bin, more peaks asked for than exist, negative times,
 * invalid data, several threads), and checks the status codes; any
 * out-of-bounds access, leak, or undefined operation makes the sanitizers fail
 * the run.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

int oracle_fpw(const double*, const double*, const double*, int64_t, const double*, int64_t, int, double, double*);
int oracle_fpw_batch(const int64_t*, int64_t, const double*, const double*, const double*, const double*, int64_t, int,
                     double, int, double*, int, int, int32_t*, double*);
int oracle_topk(const double*, int64_t, int, int, int32_t*, double*);
int oracle_bins(const double*, int64_t, const double*, int64_t, int, int32_t*, double*);
int oracle_min_edge(const double*, int64_t, const double*, int64_t, int, double*);
int oracle_fpw_multi(const double*, const double*, const double*, int64_t, const double*, int64_t, int, int, double,
                     double*);
int oracle_fpw_shared(const double*, int64_t, int64_t, const double*, const double*, const double*, int64_t, int, double,
                      double*);
int oracle_phase_entropy(const double*, int64_t, const double*, int64_t, int, double*);

static uint64_t state = 0x9E3779B97F4A7C15ull;
static double uni(void) { /* splitmix64 -> [0, 1) */
  uint64_t z = (state += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return (double)((z ^ (z >> 31)) >> 11) * 0x1p-53;
}

static int fails = 0;
static void expect(int got, int want, const char* what) {
  if (got != want) {
    fprintf(stderr, "%s: status %d, expected %d\n", what, got, want);
    ++fails;
  }
}

int main(void) {
  enum { C = 5, NMAX = 40, F = 64, K = 9 };
  const int ns[C] = {0, 1, 13, 40, 7};
  int64_t off[C + 1] = {0};
  for (int c = 0; c < C; ++c) off[c + 1] = off[c] + ns[c];
  const int64_t nobs = off[C];
  double* t = malloc(sizeof(double) * nobs);
  double* x = malloc(sizeof(double) * nobs);
  double* s = malloc(sizeof(double) * nobs);
  double* f = malloc(sizeof(double) * F);
  for (int64_t i = 0; i < nobs; ++i) {
    t[i] = 2000.0 * uni() - 300.0; /* negative times included */
    x[i] = uni() - 0.5;
    s[i] = 0.01 + uni();
  }
  for (int k = 0; k < F; ++k) f[k] = (k == 0) ? 0.0 : 0.01 + 3.0 * k;
  double* S = malloc(sizeof(double) * C * F);
  int32_t* ti = malloc(sizeof(int32_t) * C * K);
  double* tS = malloc(sizeof(double) * C * K);
  for (int M = 1; M <= 21; M += 5) {
    expect(oracle_fpw(t, x, s, NMAX, f, F, M, 0.5, S), 0, "fpw");
    expect(oracle_fpw(t, x, s, 0, f, F, M, 0.0, S), 0, "fpw n=0");
    expect(oracle_fpw(t, x, s, NMAX, f, 0, M, 0.0, S), 0, "fpw nfreq=0");
    for (int threads = 1; threads <= 3; ++threads)
      expect(oracle_fpw_batch(off, C, t, x, s, f, F, M, 0.0, threads, S, K, threads == 2, ti, tS), 0, "batch");
    expect(oracle_topk(S, F, K, 0, ti, tS), 0, "topk");
    expect(oracle_topk(S, 3, K, 1, ti, tS), 0, "topk k > nfreq");
    expect(oracle_phase_entropy(t, NMAX, f, F, M, S), 0, "entropy");
    expect(oracle_fpw_shared(t, 8, 5, x, s, f, F, M, 0.2, S), 0, "shared");
  }
  for (int g = 1; g <= 6; ++g) {
    double* Sm = malloc(sizeof(double) * g * F);
    expect(oracle_fpw_multi(t, x, s, NMAX, f, F, 12 * g, g, 0.0, Sm), 0, "multi");
    free(Sm);
  }
  int32_t* b = malloc(sizeof(int32_t) * F * NMAX);
  double* e = malloc(sizeof(double) * F * NMAX);
  expect(oracle_bins(t, NMAX, f, F, 20, b, e), 0, "bins");
  expect(oracle_min_edge(t, NMAX, f, F, 20, S), 0, "min_edge");
  s[3] = 0.0; /* invalid data */
  expect(oracle_fpw(t, x, s, NMAX, f, F, 10, 0.0, S), 2, "fpw invalid sigma");
  expect(oracle_fpw_batch(off, C, t, x, s, f, F, 10, 0.0, 2, S, K, 0, ti, tS), 2, "batch with a bad curve");
  expect(oracle_fpw(t, x, s, NMAX, f, F, 0, 0.0, S), 1, "fpw M=0");
  free(b);
  free(e);
  free(t);
  free(x);
  free(s);
  free(f);
  free(S);
  free(ti);
  free(tS);
  if (fails) return 1;
  printf("oracle sanitizer run ok\n");
  return 0;
}

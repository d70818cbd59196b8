/*
 * FPW oracle: a plain, slow, obviously correct FP64 CPU implementation of the
 * Fast Periodicity Weighting statistic (Finkbeiner, Prince & Whitebook,
 * arXiv:2502.00243).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may call, link or
 * load this file: only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline / reference leg use it. It shares no code, header, table or
 * helper with the CUDA library.
 *
 * What it computes (all in binary64, in the order the definitions state):
 *   Section 2, Eq. 1 (eq:phasesum), and Appendix A.4 (the sparse form of the
 *   chi-square difference):
 *     w_i  = 1 / sigma_i^2
 *     phi  = frac(t_i * f)                      (Appendix A.1, equation for m_i,
 *                                                with t_ref = 0)
 *     m_i  = floor(M * phi), zero-indexed 0..M-1
 *     A_m  = sum_{i in bin m} x_i * w_i         (numerator sums)
 *     B_m  = sum_{i in bin m} w_i               (denominator sums)
 *     S(f) = sum_m A_m^2 / (B_m + 1/alpha^2)
 *   Readings where the paper is silent or inconsistent:
 *     - the denominator is Eq. 1's B_m + 1/alpha^2 (not the appendix listing's
 *       factor-2 form); inv_alpha2 = 1/alpha^2 is a parameter (0 = the paper's
 *       practice of neglecting the term);
 *     - a bin whose denominator is 0 (empty bin with inv_alpha2 = 0)
 *       contributes 0, the limit of A^2/(B + c) as c -> 0 with A = B = 0;
 *     - frac uses floor, so it is defined for negative t*f too;
 *     - M * phi can round up to M for phi just below 1: the bin is clamped to
 *       M - 1 (bins are half-open [m/M, (m+1)/M));
 *     - observations are accumulated in input order.
 *   Post-processing (Section 3.5 reports the strongest peaks): a peak is a
 *   local maximum S_k > S_{k-1} and S_k >= S_{k+1} (one-sided at the grid
 *   ends); the k largest peaks by S, ties to the lower index, missing entries
 *   are index -1 and value NaN. A raw mode ranks every frequency.
 *   Edge distances (for bin-mismatch accounting): the exact distance, in
 *   cycles, of t_i * f to the nearest bin edge, from the exact product
 *   t*f = p + e (Dekker's TwoProduct, via fma) and an exact split of M*frac.
 *
 * Build: gcc -O2 -std=c99 -ffp-contract=off -fPIC -shared -pthread -lm.
 * -ffp-contract=off keeps every product and sum rounded separately, exactly
 * as written, on every host architecture.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_OK 0
#define ORACLE_EINVAL 1
#define ORACLE_EDATA 2
#define ORACLE_ENOMEM 3

int oracle_version(void) { return 1; }

/* Bin of one observation at one frequency: Appendix A.1, m = floor(M * (t f mod 1)). */
static int oracle_bin(double t, double f, int M) {
  double p = t * f;
  double phi = p - floor(p);
  int m = (int)floor((double)M * phi);
  if (m > M - 1) m = M - 1;
  if (m < 0) m = 0; /* phi >= 0 always; kept as a guard */
  return m;
}

static int check_curve(const double* t, const double* x, const double* sigma, int64_t n) {
  for (int64_t i = 0; i < n; ++i) {
    if (!isfinite(t[i]) || !isfinite(x[i]) || !isfinite(sigma[i]) || !(sigma[i] > 0.0)) return ORACLE_EDATA;
  }
  return ORACLE_OK;
}

/* Eq. 1 for one curve at every trial frequency. A and B are caller scratch of
 * length M. */
static void fpw_one_curve(const double* t, const double* x, const double* sigma, int64_t n, const double* freqs,
                          int64_t nfreq, int M, double inv_alpha2, double* A, double* B, double* S_out) {
  for (int64_t k = 0; k < nfreq; ++k) {
    for (int m = 0; m < M; ++m) {
      A[m] = 0.0;
      B[m] = 0.0;
    }
    for (int64_t i = 0; i < n; ++i) {
      double w = 1.0 / (sigma[i] * sigma[i]);
      int m = oracle_bin(t[i], freqs[k], M);
      A[m] += x[i] * w;
      B[m] += w;
    }
    double S = 0.0;
    for (int m = 0; m < M; ++m) {
      double den = B[m] + inv_alpha2;
      if (den > 0.0) S += (A[m] * A[m]) / den;
    }
    S_out[k] = S;
  }
}

int oracle_fpw(const double* t, const double* x, const double* sigma, int64_t n, const double* freqs, int64_t nfreq,
               int M, double inv_alpha2, double* S_out) {
  if (n < 0 || nfreq < 0 || M < 1 || !(inv_alpha2 >= 0.0)) return ORACLE_EINVAL;
  if (nfreq > 0 && (!freqs || !S_out)) return ORACLE_EINVAL;
  if (n > 0 && (!t || !x || !sigma)) return ORACLE_EINVAL;
  for (int64_t k = 0; k < nfreq; ++k)
    if (!isfinite(freqs[k])) return ORACLE_EDATA;
  if (check_curve(t, x, sigma, n) != ORACLE_OK) return ORACLE_EDATA;
  double* A = (double*)malloc(sizeof(double) * (size_t)M);
  double* B = (double*)malloc(sizeof(double) * (size_t)M);
  if (!A || !B) {
    free(A);
    free(B);
    return ORACLE_ENOMEM;
  }
  fpw_one_curve(t, x, sigma, n, freqs, nfreq, M, inv_alpha2, A, B, S_out);
  free(A);
  free(B);
  return ORACLE_OK;
}

/* Section 4 and Appendix D (the batch routine): several light curves observed
 * at the same times t. For each trial frequency the bin of every observation
 * is computed once, then each curve's Eq. 1 statistic is formed from those
 * bins: S_out[c * nfreq + k] for curve c, whose fluxes and uncertainties are
 * x[c * n + i] and sigma[c * n + i]. A curve with a non-finite value or a
 * sigma <= 0 gets NaN at every frequency; non-finite t or f is an error. */
int oracle_fpw_shared(const double* t, int64_t n, int64_t ncurves, const double* x, const double* sigma,
                      const double* freqs, int64_t nfreq, int M, double inv_alpha2, double* S_out) {
  if (n < 0 || ncurves < 0 || nfreq < 0 || M < 1 || !(inv_alpha2 >= 0.0)) return ORACLE_EINVAL;
  if (nfreq > 0 && ncurves > 0 && (!freqs || !S_out)) return ORACLE_EINVAL;
  if (n > 0 && (!t || (ncurves > 0 && (!x || !sigma)))) return ORACLE_EINVAL;
  for (int64_t k = 0; k < nfreq; ++k)
    if (!isfinite(freqs[k])) return ORACLE_EDATA;
  for (int64_t i = 0; i < n; ++i)
    if (!isfinite(t[i])) return ORACLE_EDATA;
  int* bin = (int*)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
  char* bad = (char*)malloc((size_t)(ncurves > 0 ? ncurves : 1));
  double* A = (double*)malloc(sizeof(double) * (size_t)M);
  double* B = (double*)malloc(sizeof(double) * (size_t)M);
  if (!bin || !bad || !A || !B) {
    free(bin);
    free(bad);
    free(A);
    free(B);
    return ORACLE_ENOMEM;
  }
  for (int64_t c = 0; c < ncurves; ++c) bad[c] = check_curve(t, x + c * n, sigma + c * n, n) != ORACLE_OK;
  for (int64_t k = 0; k < nfreq; ++k) {
    for (int64_t i = 0; i < n; ++i) bin[i] = oracle_bin(t[i], freqs[k], M);
    for (int64_t c = 0; c < ncurves; ++c) {
      if (bad[c]) {
        S_out[c * nfreq + k] = NAN;
        continue;
      }
      const double* xc = x + c * n;
      const double* sc = sigma + c * n;
      for (int m = 0; m < M; ++m) {
        A[m] = 0.0;
        B[m] = 0.0;
      }
      for (int64_t i = 0; i < n; ++i) {
        double w = 1.0 / (sc[i] * sc[i]);
        A[bin[i]] += xc[i] * w;
        B[bin[i]] += w;
      }
      double S = 0.0;
      for (int m = 0; m < M; ++m) {
        double den = B[m] + inv_alpha2;
        if (den > 0.0) S += (A[m] * A[m]) / den;
      }
      S_out[c * nfreq + k] = S;
    }
  }
  free(bin);
  free(bad);
  free(A);
  free(B);
  return ORACLE_OK;
}

/* Section 3.4, S_FPW for several numbers of bins from one pass: the bin sums
 * at M_max bins are combined into M = M_max / g bins, for each of the g bin
 * offsets o: combined bin j of offset o holds the M_max-bins
 * (j g + o + u) mod M_max, u = 0..g-1. Output S_out[o * nfreq + k], o < g.
 * (The offset shifts every combined bin edge by o / M_max of a cycle.) */
int oracle_fpw_multi(const double* t, const double* x, const double* sigma, int64_t n, const double* freqs,
                     int64_t nfreq, int M_max, int g, double inv_alpha2, double* S_out) {
  if (n < 0 || nfreq < 0 || M_max < 1 || g < 1 || M_max % g != 0 || !(inv_alpha2 >= 0.0)) return ORACLE_EINVAL;
  if (nfreq > 0 && (!freqs || !S_out)) return ORACLE_EINVAL;
  if (n > 0 && (!t || !x || !sigma)) return ORACLE_EINVAL;
  for (int64_t k = 0; k < nfreq; ++k)
    if (!isfinite(freqs[k])) return ORACLE_EDATA;
  if (check_curve(t, x, sigma, n) != ORACLE_OK) return ORACLE_EDATA;
  const int M = M_max / g;
  double* A = (double*)malloc(sizeof(double) * (size_t)M_max);
  double* B = (double*)malloc(sizeof(double) * (size_t)M_max);
  if (!A || !B) {
    free(A);
    free(B);
    return ORACLE_ENOMEM;
  }
  for (int64_t k = 0; k < nfreq; ++k) {
    for (int m = 0; m < M_max; ++m) {
      A[m] = 0.0;
      B[m] = 0.0;
    }
    for (int64_t i = 0; i < n; ++i) {
      double w = 1.0 / (sigma[i] * sigma[i]);
      int m = oracle_bin(t[i], freqs[k], M_max);
      A[m] += x[i] * w;
      B[m] += w;
    }
    for (int o = 0; o < g; ++o) {
      double S = 0.0;
      for (int j = 0; j < M; ++j) {
        double a = 0.0, b = 0.0;
        for (int u = 0; u < g; ++u) {
          int m = (j * g + o + u) % M_max;
          a += A[m];
          b += B[m];
        }
        double den = b + inv_alpha2;
        if (den > 0.0) S += (a * a) / den;
      }
      S_out[(int64_t)o * nfreq + k] = S;
    }
  }
  free(A);
  free(B);
  return ORACLE_OK;
}

/* Appendix C, phase entropy of the observation times at each frequency:
 * H = -sum_m (N_m / N) log(N_m / N) over the occupied bins, N_m the number of
 * observations in bin m (Appendix A.1 bins), N the number of observations
 * (natural logarithm; N = 0 gives 0). */
int oracle_phase_entropy(const double* t, int64_t n, const double* freqs, int64_t nfreq, int M, double* H_out) {
  if (n < 0 || nfreq < 0 || M < 1 || (nfreq > 0 && (!freqs || !H_out)) || (n > 0 && !t)) return ORACLE_EINVAL;
  int64_t* cnt = (int64_t*)malloc(sizeof(int64_t) * (size_t)M);
  if (!cnt) return ORACLE_ENOMEM;
  for (int64_t k = 0; k < nfreq; ++k) {
    for (int m = 0; m < M; ++m) cnt[m] = 0;
    for (int64_t i = 0; i < n; ++i) cnt[oracle_bin(t[i], freqs[k], M)] += 1;
    double H = 0.0;
    for (int m = 0; m < M; ++m) {
      if (cnt[m] == 0) continue;
      double p = (double)cnt[m] / (double)n;
      H -= p * log(p);
    }
    H_out[k] = H;
  }
  free(cnt);
  return ORACLE_OK;
}

/* Peaks of a periodogram (Section 3.5 post-processing, reading above). */
static int is_peak(const double* S, int64_t nfreq, int64_t k) {
  if (nfreq == 1) return 1;
  if (k == 0) return S[0] >= S[1];
  if (k == nfreq - 1) return S[k] > S[k - 1];
  return S[k] > S[k - 1] && S[k] >= S[k + 1];
}

/* Is (s1, k1) ranked ahead of (s2, k2)?  Larger S first, then lower index. */
static int ranks_before(double s1, int64_t k1, double s2, int64_t k2) {
  if (s1 != s2) return s1 > s2;
  return k1 < k2;
}

int oracle_topk(const double* S, int64_t nfreq, int k, int raw, int32_t* idx, double* val) {
  if (nfreq < 0 || k < 0) return ORACLE_EINVAL;
  if (k > 0 && (!idx || !val)) return ORACLE_EINVAL;
  for (int j = 0; j < k; ++j) {
    idx[j] = -1;
    val[j] = NAN;
  }
  int filled = 0;
  for (int64_t q = 0; q < nfreq; ++q) {
    if (!raw && !is_peak(S, nfreq, q)) continue;
    /* insertion into the sorted list idx[0..filled) */
    int pos = filled;
    while (pos > 0 && ranks_before(S[q], q, val[pos - 1], idx[pos - 1])) --pos;
    if (pos >= k) continue;
    int last = (filled < k) ? filled : k - 1;
    for (int j = last; j > pos; --j) {
      idx[j] = idx[j - 1];
      val[j] = val[j - 1];
    }
    idx[pos] = (int32_t)q;
    val[pos] = S[q];
    if (filled < k) ++filled;
  }
  return ORACLE_OK;
}

/* ---- batch: independent curves, split across threads by curve ---------- */
typedef struct {
  const int64_t* offsets;
  int64_t ncurves;
  const double *t, *x, *sigma, *freqs;
  int64_t nfreq;
  int M;
  double inv_alpha2;
  double* S_out; /* [ncurves][nfreq] or NULL */
  int k, raw;
  int32_t* topk_idx; /* [ncurves][k] or NULL */
  double* topk_S;
  int64_t next; /* shared counter, guarded by lock */
  pthread_mutex_t lock;
  int status;
} batch_job;

static void* batch_worker(void* arg) {
  batch_job* J = (batch_job*)arg;
  double* A = (double*)malloc(sizeof(double) * (size_t)J->M);
  double* B = (double*)malloc(sizeof(double) * (size_t)J->M);
  double* S = (J->S_out == NULL) ? (double*)malloc(sizeof(double) * (size_t)(J->nfreq > 0 ? J->nfreq : 1)) : NULL;
  if (!A || !B || (J->S_out == NULL && !S)) {
    pthread_mutex_lock(&J->lock);
    J->status = ORACLE_ENOMEM;
    pthread_mutex_unlock(&J->lock);
    free(A);
    free(B);
    free(S);
    return NULL;
  }
  for (;;) {
    pthread_mutex_lock(&J->lock);
    int64_t c = J->next++;
    pthread_mutex_unlock(&J->lock);
    if (c >= J->ncurves) break;
    int64_t o0 = J->offsets[c], n = J->offsets[c + 1] - o0;
    double* Sc = J->S_out ? J->S_out + c * J->nfreq : S;
    int bad = check_curve(J->t + o0, J->x + o0, J->sigma + o0, n) != ORACLE_OK;
    if (bad) {
      pthread_mutex_lock(&J->lock);
      J->status = ORACLE_EDATA;
      pthread_mutex_unlock(&J->lock);
      for (int64_t q = 0; q < J->nfreq; ++q) Sc[q] = NAN;
      if (J->k > 0 && J->topk_idx) {
        for (int j = 0; j < J->k; ++j) {
          J->topk_idx[c * J->k + j] = -1;
          J->topk_S[c * J->k + j] = NAN;
        }
      }
      continue;
    }
    fpw_one_curve(J->t + o0, J->x + o0, J->sigma + o0, n, J->freqs, J->nfreq, J->M, J->inv_alpha2, A, B, Sc);
    if (J->k > 0 && J->topk_idx)
      oracle_topk(Sc, J->nfreq, J->k, J->raw, J->topk_idx + c * J->k, J->topk_S + c * J->k);
  }
  free(A);
  free(B);
  free(S);
  return NULL;
}

int oracle_fpw_batch(const int64_t* offsets, int64_t ncurves, const double* t, const double* x, const double* sigma,
                     const double* freqs, int64_t nfreq, int M, double inv_alpha2, int nthreads, double* S_out, int k,
                     int raw, int32_t* topk_idx, double* topk_S) {
  if (ncurves < 0 || nfreq < 0 || M < 1 || k < 0 || !(inv_alpha2 >= 0.0) || !offsets) return ORACLE_EINVAL;
  if (k > 0 && (!topk_idx || !topk_S)) return ORACLE_EINVAL;
  if (offsets[0] != 0) return ORACLE_EINVAL;
  for (int64_t c = 0; c < ncurves; ++c)
    if (offsets[c + 1] < offsets[c]) return ORACLE_EINVAL;
  for (int64_t q = 0; q < nfreq; ++q)
    if (!isfinite(freqs[q])) return ORACLE_EDATA;
  if (nthreads < 1) nthreads = 1;
  batch_job J;
  memset(&J, 0, sizeof(J));
  J.offsets = offsets;
  J.ncurves = ncurves;
  J.t = t;
  J.x = x;
  J.sigma = sigma;
  J.freqs = freqs;
  J.nfreq = nfreq;
  J.M = M;
  J.inv_alpha2 = inv_alpha2;
  J.S_out = S_out;
  J.k = k;
  J.raw = raw;
  J.topk_idx = topk_idx;
  J.topk_S = topk_S;
  J.next = 0;
  J.status = ORACLE_OK;
  pthread_mutex_init(&J.lock, NULL);
  pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)nthreads);
  if (!th) return ORACLE_ENOMEM;
  int started = 0;
  for (int q = 0; q < nthreads; ++q) {
    if (pthread_create(&th[q], NULL, batch_worker, &J) != 0) break;
    ++started;
  }
  if (started == 0) batch_worker(&J);
  for (int q = 0; q < started; ++q) pthread_join(th[q], NULL);
  free(th);
  pthread_mutex_destroy(&J.lock);
  return J.status;
}

/* ---- bins and exact edge distances (bin-mismatch accounting) ------------- */
/* Exact distance, in cycles, from t*f to the nearest bin edge j / M. */
static double edge_distance(double t, double f, int M) {
  /* exact product t*f = p + e (TwoProduct via a fused multiply-add) */
  double p = t * f;
  double e = fma(t, f, -p);
  double fr = p - floor(p);          /* exact: p and floor(p) share the exponent range */
  double u = (double)M * fr;         /* M*fr = u + ue exactly */
  double ue = fma((double)M, fr, -u);
  double r = u - nearbyint(u);       /* exact: |u| <= M */
  return fabs(r + (ue + (double)M * e)) / (double)M;
}

/* For each (frequency k, observation i): the oracle's bin and the exact
 * distance, in cycles, from t_i * f_k to the nearest bin edge j / M.
 * Output layout: [nfreq][n], row-major. */
int oracle_bins(const double* t, int64_t n, const double* freqs, int64_t nfreq, int M, int32_t* bins,
                double* edge_dist) {
  if (n < 0 || nfreq < 0 || M < 1) return ORACLE_EINVAL;
  for (int64_t k = 0; k < nfreq; ++k) {
    double f = freqs[k];
    for (int64_t i = 0; i < n; ++i) {
      if (bins) bins[k * n + i] = oracle_bin(t[i], f, M);
      if (edge_dist) edge_dist[k * n + i] = edge_distance(t[i], f, M);
    }
  }
  return ORACLE_OK;
}

/* Per frequency: the smallest exact edge distance over all observations with
 * t*f != 0. A frequency whose value is tiny has an observation whose bin is
 * decided by rounding. Observations with t*f == 0 (t = 0 or f = 0) have phase
 * exactly 0 in every arithmetic and are skipped. */
int oracle_min_edge(const double* t, int64_t n, const double* freqs, int64_t nfreq, int M, double* out) {
  if (n < 0 || nfreq < 0 || M < 1 || (nfreq > 0 && !out)) return ORACLE_EINVAL;
  for (int64_t k = 0; k < nfreq; ++k) {
    double best = INFINITY;
    for (int64_t i = 0; i < n; ++i) {
      if (t[i] == 0.0 || freqs[k] == 0.0) continue;
      double d = edge_distance(t[i], freqs[k], M);
      if (d < best) best = d;
    }
    out[k] = best;
  }
  return ORACLE_OK;
}

"""Mutation check of the oracle's pins: plant one plausible mistake at a time in
a copy of the oracle's C source (a dropped term, a wrong weight, a transposed
operand, a wrong index or tie rule), compile it on the CPU, and require that
the pin battery below rejects every mutant while accepting the original.

CPU only; the mutants never touch a GPU."""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile

import numpy as np
import pytest

import math
from fractions import Fraction

from test_oracle_pins import (GOLDEN, dense_chi2_difference, exact_bins, exact_phase, least_squares_reduction,
                              tiny_case)

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "fpw_oracle.c")

MUTATIONS = {
    "weight_1_over_sigma": ("double w = 1.0 / (sigma[i] * sigma[i]);", "double w = 1.0 / sigma[i];"),
    "drop_prior_term": ("double den = B[m] + inv_alpha2;", "double den = B[m];"),
    "unweighted_numerator": ("A[m] += x[i] * w;", "A[m] += x[i];"),
    "transposed_sums": ("A[m] += x[i] * w;\n      B[m] += w;", "A[m] += w;\n      B[m] += x[i] * w;"),
    "missing_square": ("S += (A[m] * A[m]) / den;", "S += A[m] / den;"),
    "listing_factor_two": ("S += (A[m] * A[m]) / den;", "S += (A[m] * A[m]) / (2.0 * den);"),
    "truncate_not_floor": ("double phi = p - floor(p);", "double phi = p - (double)(long long)p;"),
    "wrong_bin_scale": ("int m = (int)floor((double)M * phi);", "int m = (int)floor((double)(M - 1) * phi);"),
    "no_reset_between_freqs": ("      A[m] = 0.0;\n      B[m] = 0.0;\n", "      if (k == 0) { A[m] = 0.0; B[m] = 0.0; }\n"),
    "peak_left_nonstrict": ("return S[k] > S[k - 1] && S[k] >= S[k + 1];", "return S[k] >= S[k - 1] && S[k] >= S[k + 1];"),
    "tie_to_higher_index": ("return k1 < k2;", "return k1 > k2;"),
    "ends_never_peaks": ("if (k == 0) return S[0] >= S[1];", "if (k == 0) return 0;"),
    "multi_ignores_offset": ("int m = (j * g + o + u) % M_max;", "int m = (j * g + u) % M_max;"),
    "multi_offset_backwards": ("int m = (j * g + o + u) % M_max;", "int m = (j * g - o + u + M_max) % M_max;"),
    "shared_flux_of_first_curve": ("const double* xc = x + c * n;", "const double* xc = x;"),
    "shared_sigma_of_first_curve": ("const double* sc = sigma + c * n;", "const double* sc = sigma;"),
    "shared_bins_not_recomputed": ("    for (int64_t i = 0; i < n; ++i) bin[i] = oracle_bin(t[i], freqs[k], M);",
                                   "    if (k == 0)\n      for (int64_t i = 0; i < n; ++i) bin[i] = oracle_bin(t[i], freqs[k], M);"),
    "shared_unweighted_numerator": ("A[bin[i]] += xc[i] * w;", "A[bin[i]] += xc[i];"),
    "edge_distance_drops_product_error": ("return fabs(r + (ue + (double)M * e)) / (double)M;",
                                          "return fabs(r + ue) / (double)M;"),
    "entropy_base_two_log": ("      H -= p * log(p);", "      H -= p * log2(p);"),
    "entropy_wrong_sign": ("      H -= p * log(p);", "      H += p * log(p);"),
    "entropy_counts_not_normalised": ("double p = (double)cnt[m] / (double)n;", "double p = (double)cnt[m];"),
    "entropy_counts_not_reset": ("    for (int m = 0; m < M; ++m) cnt[m] = 0;\n    for (int64_t i = 0; i < n; ++i) cnt[oracle_bin(t[i], freqs[k], M)] += 1;",
                                 "    if (k == 0)\n      for (int m = 0; m < M; ++m) cnt[m] = 0;\n    for (int64_t i = 0; i < n; ++i) cnt[oracle_bin(t[i], freqs[k], M)] += 1;"),
}


class Api:
    def __init__(self, path):
        lib = ctypes.CDLL(path)
        vp, i64, ci, d = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
        lib.oracle_fpw.argtypes = [vp, vp, vp, i64, vp, i64, ci, d, vp]
        lib.oracle_topk.argtypes = [vp, i64, ci, ci, vp, vp]
        lib.oracle_bins.argtypes = [vp, i64, vp, i64, ci, vp, vp]
        lib.oracle_fpw_multi.argtypes = [vp, vp, vp, i64, vp, i64, ci, ci, d, vp]
        lib.oracle_fpw_shared.argtypes = [vp, i64, i64, vp, vp, vp, i64, ci, d, vp]
        lib.oracle_phase_entropy.argtypes = [vp, i64, vp, i64, ci, vp]
        self.lib = lib

    def phase_entropy(self, t, freqs, M):
        t, freqs = np.ascontiguousarray(t, dtype=np.float64), np.ascontiguousarray(freqs, dtype=np.float64)
        H = np.empty(freqs.shape[0])
        rc = self.lib.oracle_phase_entropy(t.ctypes.data, t.shape[0], freqs.ctypes.data, freqs.shape[0], M,
                                           H.ctypes.data)
        assert rc == 0
        return H

    def fpw_shared(self, t, x, sigma, freqs, M, c=0.0):
        t, x, sigma, freqs = (np.ascontiguousarray(a, dtype=np.float64) for a in (t, x, sigma, freqs))
        S = np.empty((x.shape[0], freqs.shape[0]))
        rc = self.lib.oracle_fpw_shared(t.ctypes.data, t.shape[0], x.shape[0], x.ctypes.data, sigma.ctypes.data,
                                        freqs.ctypes.data, freqs.shape[0], M, c, S.ctypes.data)
        assert rc == 0
        return S

    def fpw_multi(self, t, x, sigma, freqs, M_max, g, c=0.0):
        t, x, sigma, freqs = (np.ascontiguousarray(a, dtype=np.float64) for a in (t, x, sigma, freqs))
        S = np.empty((g, freqs.shape[0]))
        rc = self.lib.oracle_fpw_multi(t.ctypes.data, x.ctypes.data, sigma.ctypes.data, t.shape[0], freqs.ctypes.data,
                                       freqs.shape[0], M_max, g, c, S.ctypes.data)
        assert rc == 0
        return S

    def fpw(self, t, x, sigma, freqs, M, c=0.0):
        t, x, sigma, freqs = (np.ascontiguousarray(a, dtype=np.float64) for a in (t, x, sigma, freqs))
        S = np.empty(freqs.shape[0])
        rc = self.lib.oracle_fpw(t.ctypes.data, x.ctypes.data, sigma.ctypes.data, t.shape[0], freqs.ctypes.data,
                                 freqs.shape[0], M, c, S.ctypes.data)
        assert rc == 0
        return S

    def topk(self, S, k, raw=0):
        S = np.ascontiguousarray(S, dtype=np.float64)
        idx = np.empty(k, dtype=np.int32)
        val = np.empty(k)
        self.lib.oracle_topk(S.ctypes.data, S.shape[0], k, raw, idx.ctypes.data, val.ctypes.data)
        return idx, val

    def bins(self, t, freqs, M):
        t, freqs = np.ascontiguousarray(t, dtype=np.float64), np.ascontiguousarray(freqs, dtype=np.float64)
        b = np.empty((freqs.shape[0], t.shape[0]), dtype=np.int32)
        e = np.empty((freqs.shape[0], t.shape[0]))
        self.lib.oracle_bins(t.ctypes.data, t.shape[0], freqs.ctypes.data, freqs.shape[0], M, b.ctypes.data,
                             e.ctypes.data)
        return b, e


def battery(api: Api) -> list[str]:
    """Returns the names of the failed pins (empty = all pass)."""
    failed = []
    # hand-worked example
    t = np.array([0, 0.1, 0.35, 0.6, 0.85, 1.2])
    x = np.array([1, 2, -1, 0.5, -3, 1.0])
    sigma = np.array([1, 0.5, 1, 2, 1, 0.5])
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "hand_example.txt")) if ln.strip() and ln[0] != "#"]
    for f, c, num, den in rows:
        if not np.isclose(api.fpw(t, x, sigma, [float(f)], 4, float(c))[0], int(num) / int(den), rtol=1e-12):
            failed.append("hand")
            break
    # dense and least-squares forms (negative times included)
    for seed in range(6):
        rng = np.random.default_rng([17, seed])
        n = int(rng.integers(3, 12))
        M = int(rng.choice([2, 3, 5]))
        t, x, sigma = tiny_case(rng, n, negative_t=(seed % 2 == 0))
        f = float(rng.uniform(0.1, 3.0))
        b, _ = exact_bins(t, f, M)
        if not np.isclose(api.fpw(t, x, sigma, [f], M, 1.0)[0], dense_chi2_difference(x, sigma, b, M, 1.0),
                          rtol=1e-9):
            failed.append("dense")
            break
        if not np.isclose(api.fpw(t, x, sigma, [f], M, 0.0)[0], least_squares_reduction(x, sigma, b, M),
                          rtol=1e-9, atol=1e-10):
            failed.append("least_squares")
            break
    # several frequencies in one call (per-frequency state)
    rng = np.random.default_rng(18)
    t, x, sigma = tiny_case(rng, 10)
    fs = np.array([0.3, 1.7, 2.2])
    S = api.fpw(t, x, sigma, fs, 3, 0.0)
    for q, f in enumerate(fs):
        b, _ = exact_bins(t, f, 3)
        if not np.isclose(S[q], least_squares_reduction(x, sigma, b, 3), rtol=1e-9, atol=1e-10):
            failed.append("multi_freq")
            break
    # bins and exact edge distances
    rng = np.random.default_rng(19)
    t = rng.uniform(0, 2000, 30)
    fs = rng.uniform(0.01, 500, 4)
    b, e = api.bins(t, fs, 20)
    for q, f in enumerate(fs):
        eb, ed = exact_bins(t, f, 20)
        if not np.allclose(e[q], ed, rtol=0, atol=1e-15) or not np.array_equal(b[q][ed > 1e-12], eb[ed > 1e-12]):
            failed.append("bins")
            break
    # several M from one M_max pass: offset o shifts the combined bin edges by o/M_max
    rng = np.random.default_rng(20)
    t, x, sigma = tiny_case(rng, 11)
    f = 1.37
    S = api.fpw_multi(t, x, sigma, [f], 12, 3)
    for o in range(3):
        bins = []
        for ti in t:
            ph = exact_phase(ti, f) - Fraction(o, 12)
            ph -= math.floor(ph)
            bins.append(int(math.floor(ph * 4)))
        if not np.isclose(S[o, 0], least_squares_reduction(x, sigma, np.array(bins), 4), rtol=1e-9, atol=1e-10):
            failed.append("multi_m")
            break
    # curves sharing their times: each row is the dense form with the shared exact bins
    rng = np.random.default_rng(21)
    t = rng.uniform(0, 30, 9)
    x = rng.normal(0, 1, (3, 9))
    sigma = rng.uniform(0.3, 2.0, (3, 9))
    fs = np.array([0.7, 1.9])
    S = api.fpw_shared(t, x, sigma, fs, 3, 1.0)
    for q, f in enumerate(fs):
        b, _ = exact_bins(t, f, 3)
        if not all(np.isclose(S[c, q], dense_chi2_difference(x[c], sigma[c], b, 3, 1.0), rtol=1e-9) for c in range(3)):
            failed.append("shared")
            break
    # phase entropy: bin counts from exact phases, H = -sum (N_m/N) ln(N_m/N), at
    # two frequencies in one call
    rng = np.random.default_rng(22)
    t = rng.uniform(0, 50, 13)
    fs = np.array([0.83, 2.41])
    H = api.phase_entropy(t, fs, 5)
    for q, f in enumerate(fs):
        b, _ = exact_bins(t, f, 5)
        p = np.bincount(b, minlength=5) / t.size
        p = p[p > 0]
        if not np.isclose(H[q], float(-(p * np.log(p)).sum()), rtol=1e-12):
            failed.append("entropy")
            break
    # top-k golden cases
    idx, _ = api.topk(np.array([1.0, 3.0, 2.0, 5.0, 5.0, 4.0, 6.0]), 3)
    if list(idx) != [6, 3, 1]:
        failed.append("topk_golden")
    idx, _ = api.topk(np.array([4.0, 4.0, 1.0, 2.0, 2.0]), 5)
    if list(idx) != [0, 3, -1, -1, -1]:
        failed.append("topk_ends")
    idx, _ = api.topk(np.array([0.0, 2.0, 0.0, 2.0, 0.0, 2.0]), 3)
    if list(idx) != [1, 3, 5]:
        failed.append("topk_ties")
    return failed


def _compile(src_text: str, tmpdir: str, name: str) -> str:
    c = os.path.join(tmpdir, name + ".c")
    so = os.path.join(tmpdir, name + ".so")
    with open(c, "w") as fh:
        fh.write(src_text)
    subprocess.run([os.environ.get("CC", "gcc"), "-O1", "-std=c99", "-ffp-contract=off", "-fPIC", "-shared",
                    "-pthread", c, "-o", so, "-lm"], check=True)
    return so


@pytest.fixture(scope="module")
def tmpdir_mod():
    with tempfile.TemporaryDirectory() as d:
        yield d


def test_original_passes_battery(tmpdir_mod):
    src = open(SRC).read()
    assert battery(Api(_compile(src, tmpdir_mod, "original"))) == []


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_mutant_is_caught(name, tmpdir_mod):
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation anchor for {name} not found"  # every occurrence is mutated
    failed = battery(Api(_compile(src.replace(old, new), tmpdir_mod, "mut_" + name)))
    assert failed, f"mutant {name} passed every pin"

"""Curves sharing their observation times (Section 4 / Appendix D batch routine)
on the tensor-core path against the oracle: dense S and top-k for ragged group
counts, chunk tails and frequency-pass tails, bin counts from 1 to 256, invalid
curves, empty inputs, and the full 4096-curve workload on sampled curves."""
from __future__ import annotations

import numpy as np
import pytest

import lightcurves as L
import oracle
from gpu_util import assert_S_close, check_topk, s_bound

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2502_00243_gb300 as G_
    return G_


@pytest.fixture(scope="module")
def ctx(G):
    c = G.Context(0)
    yield c
    c.close()


def field(seed, C, n, F, fmax=50.0):
    rng = np.random.default_rng([77, seed])
    t = L.ztf_cadence(rng, n) if n >= 40 else np.sort(rng.uniform(0, 1000.0, n))
    sigma = np.exp(rng.uniform(np.log(0.01), np.log(0.3), (C, n)))
    x = np.zeros((C, n))
    for c in range(C):
        kind = L.WAVEFORMS[c % 4]
        x[c] = L.waveform(kind, t, float(np.exp(rng.uniform(np.log(0.05), np.log(50)))), rng.uniform(), 0.3) \
            + rng.normal(0, 1, n) * sigma[c]
        if n:
            w = 1 / sigma[c] ** 2
            x[c] -= np.sum(w * x[c]) / np.sum(w)
    freqs = np.linspace(0.01, fmax, F)
    return t, x, sigma, freqs


def run_shared(G, ctx, t, x, sigma, freqs, M, k, params=None, dense=True):
    C, F = x.shape[0], freqs.shape[0]
    d = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (t, x, sigma, freqs)]
    idx = torch.empty(max(C * k, 1), dtype=torch.int32, device="cuda")
    S = torch.empty(max(C * k, 1), dtype=torch.float32, device="cuda")
    Sd = torch.empty(C * F, dtype=torch.float64, device="cuda") if dense else None
    G.fpw_periodogram_shared(ctx, None, params, d[0], d[1], d[2], d[3], M, k, idx if k else None,
                             S if k else None, Sd)
    torch.cuda.synchronize()
    st = ctx.status()
    out = (idx.cpu().numpy()[:C * k].reshape(C, k), S.cpu().numpy()[:C * k].reshape(C, k),
           Sd.cpu().numpy().reshape(C, F) if dense else None)
    return (*out, st)


CASES = [  # (C, n, F, M): group tail, chunk tail, pass tail
    (70, 1000, 3001, 20),
    (5, 37, 517, 7),
    (64, 32, 256, 1),
    (3, 200, 1000, 256),
    (130, 150, 777, 50),
    (1, 1, 100, 10),
    (33, 96, 2049, 10),
]


@pytest.mark.parametrize("C,n,F,M", CASES)
def test_shared_dense_and_topk_against_oracle(G, ctx, C, n, F, M):
    t, x, sigma, freqs = field(C * 1000 + n, C, n, F)
    k = 5
    idx, Sk, Sd, st = run_shared(G, ctx, t, x, sigma, freqs, M, k)
    assert st == 0
    S_or = oracle.fpw_shared(t, x, sigma, freqs, M)
    near = oracle.min_edge(t, freqs, M) <= 1e-9 if n else np.zeros(F, bool)
    for c in range(C):
        bound = s_bound(x[c], sigma[c])
        assert_S_close(Sd[c], S_or[c], bound, mask=~near, what=f"C={C} n={n} M={M} curve {c}")
        o_idx, o_S = oracle.topk(S_or[c], k + 4)
        check_topk(idx[c], Sk[c], o_idx, o_S, abs_tol=1e-7 * bound, o_dense=S_or[c], what=f"curve {c} peaks")


def test_shared_matches_batched_path_and_inv_alpha2(G, ctx):
    t, x, sigma, freqs = field(3, 40, 500, 4000)
    p = G.fpw_params_default(inv_alpha2=2.5)
    _, _, Sd, st = run_shared(G, ctx, t, x, sigma, freqs, 20, 0, params=p)
    assert st == 0
    S_or = oracle.fpw_shared(t, x, sigma, freqs, 20, 2.5)
    near = oracle.min_edge(t, freqs, 20) <= 1e-9
    for c in range(40):
        assert_S_close(Sd[c], S_or[c], s_bound(x[c], sigma[c]), mask=~near, what=f"alpha curve {c}")


def test_shared_invalid_curves_and_empty_inputs(G, ctx):
    t, x, sigma, freqs = field(4, 66, 100, 600)
    sigma = sigma.copy()
    sigma[3, 10] = 0.0
    x = x.copy()
    x[65, 0] = np.nan
    idx, Sk, Sd, st = run_shared(G, ctx, t, x, sigma, freqs, 12, 3)
    assert st == G.FPW_EDATA
    for c in (3, 65):
        assert np.isnan(Sd[c]).all() and np.all(idx[c] == -1) and np.isnan(Sk[c]).all()
    good = [c for c in range(66) if c not in (3, 65)]
    S_or = oracle.fpw_shared(t, x[good], sigma[good], freqs, 12)
    near = oracle.min_edge(t, freqs, 12) <= 1e-9
    for j, c in enumerate(good):
        assert_S_close(Sd[c], S_or[j], s_bound(x[c], sigma[c]), mask=~near, what=f"neighbour {c}")
    # no observations: S = 0 everywhere, the flat periodogram's one peak at index 0
    e = np.zeros(0)
    idx, Sk, Sd, st = run_shared(G, ctx, e, np.zeros((4, 0)), np.ones((4, 0)), freqs, 12, 2)
    assert st == 0 and np.all(Sd == 0.0) and np.all(idx[:, 0] == 0) and np.all(idx[:, 1] == -1)
    # unsupported combinations
    for M, p in ((257, None), (20, G.fpw_params_default(accum=1)), (20, G.fpw_params_default(phase_mode=1))):
        with pytest.raises(G.FPWError) as ei:
            run_shared(G, ctx, t, x, sigma, freqs, M, 1, params=p)
        assert ei.value.code == G.FPW_ENOTSUP


def test_shared_4096_full_size_sampled(G, ctx):
    """The 4096-curve field at full size (5e5 frequencies), launched as the
    benchmark launches it; sampled curves against the oracle."""
    w = L.make("shared_4096")
    C, n = w.ncurves, L.SHARED_N
    t = w.t[:n]
    x, sigma = w.x.reshape(C, n), w.sigma.reshape(C, n)
    idx, Sk, _, st = run_shared(G, ctx, t, x, sigma, w.freqs, w.M, w.k, dense=False)
    assert st == 0
    sample = np.random.default_rng(6).choice(C, 4, replace=False)
    near = oracle.min_edge_parallel(t, w.freqs, w.M) <= 1e-9
    sub_idx, sub_S, sub_dense, st = run_shared(G, ctx, t, x[sample], sigma[sample], w.freqs, w.M, w.k)
    assert st == 0
    for j, c in enumerate(sample):
        S_or = oracle.fpw_parallel(t, x[c], sigma[c], w.freqs, w.M)
        bound = s_bound(x[c], sigma[c])
        assert_S_close(sub_dense[j], S_or, bound, mask=~near, what=f"shared_4096 curve {c}")
        o_idx, o_S = oracle.topk(S_or, w.k + 4)
        check_topk(idx[c], Sk[c], o_idx, o_S, abs_tol=1e-7 * bound, o_dense=S_or, what=f"shared_4096 curve {c}")


def test_shared_irregular_grid(G, ctx):
    """A grid that is not linear: the one-hot rows come from exact anchors per
    (observation, frequency) pair, across several frequency passes."""
    t, x, sigma, _ = field(5, 70, 300, 10)
    rng = np.random.default_rng(8)
    freqs = np.concatenate([np.linspace(0.05, 3.0, 100), np.sort(rng.uniform(3.01, 45.0, 700))])
    idx, Sk, Sd, st = run_shared(G, ctx, t, x, sigma, freqs, 20, 5)
    assert st == 0
    S_or = oracle.fpw_shared(t, x, sigma, freqs, 20)
    near = oracle.min_edge(t, freqs, 20) <= 1e-9
    for c in range(70):
        bound = s_bound(x[c], sigma[c])
        assert_S_close(Sd[c], S_or[c], bound, mask=~near, what=f"irregular grid curve {c}")
        o_idx, o_S = oracle.topk(S_or[c], 9)
        check_topk(idx[c], Sk[c], o_idx, o_S, abs_tol=1e-7 * bound, o_dense=S_or[c], what=f"irregular grid curve {c}")


@pytest.mark.parametrize("ia2", [1e38, 3e-38])
def test_shared_extreme_inv_alpha2(G, ctx, ia2):
    """Bin denominators B_m + 1/alpha^2 near the top of the float32 range (the
    reciprocal's result subnormal) and 1/alpha^2 at the bottom: S against the
    oracle, finite everywhere."""
    t, x, sigma, freqs = field(6, 20, 300, 700)
    p = G.fpw_params_default(inv_alpha2=ia2)
    _, _, Sd, st = run_shared(G, ctx, t, x, sigma, freqs, 12, 0, params=p)
    assert st == 0 and np.isfinite(Sd).all()
    S_or = oracle.fpw_shared(t, x, sigma, freqs, 12, ia2)
    near = oracle.min_edge(t, freqs, 12) <= 1e-9
    for c in range(20):
        assert_S_close(Sd[c], S_or[c], s_bound(x[c], sigma[c]), mask=~near, what=f"ia2={ia2:g} curve {c}")

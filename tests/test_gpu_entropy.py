"""Phase entropy (Appendix C) on the GPU against the oracle: the dense entropy
periodogram of one set of times, and entropy plus Hutcheson z-score at the
peaks reported by the batched call."""
from __future__ import annotations

import math

import numpy as np
import pytest

import lightcurves as L
import oracle
from gpu_util import run_batch, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2502_00243_gb300 as G_
    return G_


@pytest.mark.parametrize("M", [4, 10, 20, 50])
def test_dense_phase_entropy(G, M):
    w = L.make("single_ztf", nfreq=40_000)
    t, _, _ = w.curve(0)
    ctx = G.Context(0)
    H = torch.empty(w.nfreq, dtype=torch.float32, device="cuda")
    G.fpw_phase_entropy(ctx, None, torch.from_numpy(t).cuda(), torch.from_numpy(w.freqs).cuda(), M, H)
    torch.cuda.synchronize()
    H = H.cpu().numpy().astype(np.float64)
    H_or = oracle.phase_entropy(t, w.freqs, M)
    near = oracle.min_edge(t, w.freqs, M) <= 1e-9
    err = np.abs(H - H_or)[~near]
    assert err.max() < 2e-5, err.max()
    ctx.close()


@pytest.mark.parametrize("M", [1, 7, 256])
def test_dense_phase_entropy_irregular_grid(G, M):
    """A grid that is not linear (every frequency anchored exactly), M from 1 to
    256, a frequency count that leaves a partial block, and no observations."""
    rng = np.random.default_rng([91, M])
    t = np.sort(rng.uniform(0.0, 900.0, 700))
    freqs = np.sort(rng.uniform(0.01, 40.0, 3001))
    ctx = G.Context(0)
    H = torch.empty(freqs.size, dtype=torch.float32, device="cuda")
    G.fpw_phase_entropy(ctx, None, torch.from_numpy(t).cuda(), torch.from_numpy(freqs).cuda(), M, H)
    torch.cuda.synchronize()
    Hn = H.cpu().numpy().astype(np.float64)
    H_or = oracle.phase_entropy(t, freqs, M)
    near = oracle.min_edge(t, freqs, M) <= 1e-9
    err = np.abs(Hn - H_or)[~near]
    assert err.max() < 2e-5, err.max()
    G.fpw_phase_entropy(ctx, None, torch.from_numpy(t[:0].copy()).cuda(), torch.from_numpy(freqs).cuda(), M, H)
    torch.cuda.synchronize()
    assert torch.all(H == 0.0)
    ctx.close()


def test_entropy_at_batch_peaks(G):
    w = L.ragged(80, [300, 1500, 60, 900], 6000, M=20, k=5)
    ctx = G.Context(0)
    idx, Sk, _, st = run_batch(ctx, w)
    assert st == 0
    d = to_dev(w)
    k = 5
    H = torch.empty(w.ncurves * k, dtype=torch.float32, device="cuda")
    z = torch.empty(w.ncurves * k, dtype=torch.float32, device="cuda")
    ti = torch.from_numpy(idx.reshape(-1).copy()).cuda()
    G.fpw_phase_entropy_peaks(ctx, None, d["offsets"], d["t"], d["freqs"], 20, k, ti, H, z)
    torch.cuda.synchronize()
    H = H.cpu().numpy().reshape(w.ncurves, k)
    z = z.cpu().numpy().reshape(w.ncurves, k)
    for c in range(w.ncurves):
        t, _, _ = w.curve(c)
        N = t.size
        E = math.log(20) - 19 / (2 * N) - 19 * 21 / (12 * N * N)
        V = 19 / (2 * N * N) + 399 / (6 * N ** 3)
        for j in range(k):
            if idx[c, j] < 0:
                assert np.isnan(H[c, j]) and np.isnan(z[c, j])
                continue
            f = w.freqs[idx[c, j]]
            h = oracle.phase_entropy(t, [f], 20)[0]
            if oracle.min_edge(t, [f], 20)[0] > 1e-9:
                assert abs(H[c, j] - h) < 2e-5
                assert abs(z[c, j] - (h - E) / math.sqrt(V)) < 2e-5 / math.sqrt(V) + 1e-3
    # an invalid index gives NaN
    bad = torch.tensor([-1, w.nfreq + 5] + [0] * (w.ncurves * k - 2), dtype=torch.int32, device="cuda")
    G.fpw_phase_entropy_peaks(ctx, None, d["offsets"], d["t"], d["freqs"], 20, k, bad, H_ := torch.empty_like(
        torch.from_numpy(H.reshape(-1)).cuda()), z_ := torch.empty_like(H_))
    torch.cuda.synchronize()
    assert torch.isnan(H_[:2]).all() and torch.isnan(z_[:2]).all()
    ctx.close()


@pytest.mark.parametrize("N", [65535, 65536])
def test_dense_phase_entropy_large_counts(G, N):
    """Counts as large as N around 2^16, from a grid whose first frequency is 0
    (every observation in bin 0, so one count equals N and H = 0 up to the
    rounding of log N - N log N / N; a count that wrapped would give about
    log N) and whose other frequencies spread the observations; M = 1 (one
    bin holding all N at every frequency), 3 and 10 (eight frequencies per
    thread)."""
    rng = np.random.default_rng([92, N])
    t = np.sort(rng.uniform(0.0, 1000.0, N))
    freqs = np.concatenate([[0.0], np.linspace(0.05, 30.0, 1499)])
    ctx = G.Context(0)
    for M in (1, 3, 10):
        H = torch.empty(freqs.size, dtype=torch.float32, device="cuda")
        G.fpw_phase_entropy(ctx, None, torch.from_numpy(t).cuda(), torch.from_numpy(freqs).cuda(), M, H)
        torch.cuda.synchronize()
        Hn = H.cpu().numpy().astype(np.float64)
        assert abs(Hn[0]) < 2e-5
        if M == 1:
            assert np.all(np.abs(Hn) < 2e-5)
        H_or = oracle.phase_entropy(t, freqs, M)
        near = oracle.min_edge(t, freqs, M) <= 1e-9
        err = np.abs(Hn - H_or)[~near]
        assert err.max() < 2e-5, (M, err.max())
    ctx.close()

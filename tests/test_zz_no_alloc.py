"""The no-allocation batched entry point, against the oracle and against the
regular batched entry point.

fpw_periodogram_batch_noalloc serves callers that cannot call cudaMalloc: code
running inside another framework's memory pool, plugins whose host forbids
device allocation after start-up, and real-time pipelines that must not risk an
allocation failure or an implicit device synchronization mid-run. Its scratch
is one fixed device array inside the library, shared by every call. This file
is collected last so that a run stopping at the first failure has already run
every other test."""
from __future__ import annotations

import numpy as np
import pytest

import lightcurves as L
import oracle
from gpu_util import check_topk, run_batch, s_bound, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2502_00243_gb300 as G_
    return G_


def _noalloc(G, w, d, offsets_host, k=None, sigma=None):
    C = w.ncurves
    k = w.k if k is None else k
    idx = torch.full((max(C * k, 1),), -7, dtype=torch.int32, device="cuda")
    S = torch.full((max(C * k, 1),), -7.0, dtype=torch.float32, device="cuda")
    G.fpw_periodogram_batch_noalloc(None, None, d["offsets"], offsets_host, d["t"], d["x"],
                                    d["sigma"] if sigma is None else sigma, d["freqs"], w.M, k, idx, S)
    return idx.cpu().numpy()[:C * k].reshape(C, k), S.cpu().numpy()[:C * k].reshape(C, k)


def test_noalloc_matches_oracle_and_batch_entry_point_on_two_calls(G):
    w = L.ragged(31, [0, 1, 40, 700, 1500, 3100, 333], 20_000, M=20, k=5)
    d = to_dev(w)
    S_or, o_idx, o_S = oracle.fpw_batch(w.offsets, w.t, w.x, w.sigma, w.freqs, w.M, k=w.k + 4)
    ctx = G.Context(0)
    ref_idx, ref_S, _, st = run_batch(ctx, w, d=d)
    assert st == 0
    ctx.close()
    # the second call reads the offsets back from the device itself
    for offsets_host in (w.offsets, None):
        idx, S = _noalloc(G, w, d, offsets_host)
        for c in range(w.ncurves):
            t, x, s = w.curve(c)
            bound = s_bound(x, s)
            check_topk(idx[c], S[c], o_idx[c], o_S[c], abs_tol=1e-7 * bound, o_dense=S_or[c],
                       what=f"noalloc curve {c} vs oracle")
            check_topk(idx[c], S[c], ref_idx[c], ref_S[c].astype(np.float64), abs_tol=1e-7 * bound,
                       what=f"noalloc curve {c} vs batched call")


def test_noalloc_invalid_data_and_k0(G):
    w = L.ragged(32, [300, 200, 500], 4000, M=10, k=4)
    d = to_dev(w)
    sig = d["sigma"].clone()
    sig[350] = 0.0  # curve 1
    with pytest.raises(G.FPWError) as ei:
        _noalloc(G, w, d, w.offsets, sigma=sig)
    assert ei.value.code == G.FPW_EDATA
    # the bad curve gets no peaks, its neighbours match the oracle
    C, k = w.ncurves, w.k
    idx = torch.full((C * k,), -7, dtype=torch.int32, device="cuda")
    S = torch.full((C * k,), -7.0, dtype=torch.float32, device="cuda")
    try:
        G.fpw_periodogram_batch_noalloc(None, None, d["offsets"], w.offsets, d["t"], d["x"], sig, d["freqs"], w.M,
                                        k, idx, S)
    except G.FPWError as e:
        assert e.code == G.FPW_EDATA
    idx, S = idx.cpu().numpy().reshape(C, k), S.cpu().numpy().reshape(C, k)
    assert np.all(idx[1] == -1) and np.isnan(S[1]).all()
    S_or, o_idx, o_S = oracle.fpw_batch(w.offsets, w.t, w.x, w.sigma, w.freqs, w.M, k=k + 4)
    for c in (0, 2):
        t, x, s = w.curve(c)
        check_topk(idx[c], S[c], o_idx[c], o_S[c], abs_tol=1e-7 * s_bound(x, s), o_dense=S_or[c],
                   what=f"curve {c} next to a bad one")
    # k = 0: no peaks asked for, a clean status
    _noalloc(G, w, d, None, k=0)


def test_noalloc_rejects_malformed_device_offsets(G):
    w = L.ragged(33, [100, 200, 300], 64, M=4, k=2)
    d = to_dev(w)
    for bad in ([0, 300, 200, 600], [5, 100, 300, 600], [0, 100, 300, (1 << 41)]):
        off = torch.tensor(bad, dtype=torch.int64, device="cuda")
        dd = dict(d, offsets=off)
        with pytest.raises(G.FPWError) as ei:
            _noalloc(G, w, dd, None)  # offsets on the device only
        assert ei.value.code == G.FPW_EINVAL
    _noalloc(G, w, d, None)  # and the next call runs


def test_noalloc_compensated_sums_match_the_batched_call(G):
    w = L.ragged(34, [800, 1500, 45, 2200], 5000, M=20, k=5)
    d = to_dev(w)
    p = G.fpw_params_default(accum=G.FPW_ACCUM_FP32_COMP)
    ctx = G.Context(0)
    ref_idx, ref_S, _, st = run_batch(ctx, w, d=d, params=p)
    assert st == 0
    ctx.close()
    C, k = w.ncurves, w.k
    idx = torch.full((C * k,), -7, dtype=torch.int32, device="cuda")
    S = torch.full((C * k,), -7.0, dtype=torch.float32, device="cuda")
    G.fpw_periodogram_batch_noalloc(None, p, d["offsets"], w.offsets, d["t"], d["x"], d["sigma"], d["freqs"], w.M, k,
                                    idx, S)
    idx, S = idx.cpu().numpy().reshape(C, k), S.cpu().numpy().reshape(C, k)
    for c in range(C):
        t, x, s = w.curve(c)
        check_topk(idx[c], S[c], ref_idx[c], ref_S[c].astype(np.float64), rel=1e-6, abs_tol=1e-9 * s_bound(x, s),
                   what=f"noalloc compensated curve {c}")


def test_noalloc_rejects_inputs_beyond_its_scratch(G):
    n = 5_000_000  # 8 B of weights per observation exceeds the 32 MiB array
    off = np.array([0, n], dtype=np.int64)
    big = torch.ones(n, dtype=torch.float64, device="cuda")
    freqs = torch.linspace(0.1, 1.0, 8, dtype=torch.float64, device="cuda")
    idx = torch.empty(2, dtype=torch.int32, device="cuda")
    S = torch.empty(2, dtype=torch.float32, device="cuda")
    with pytest.raises(G.FPWError) as ei:
        G.fpw_periodogram_batch_noalloc(None, None, torch.from_numpy(off).cuda(), off, big, big, big, freqs, 4, 2,
                                        idx, S)
    assert ei.value.code == G.FPW_EINVAL

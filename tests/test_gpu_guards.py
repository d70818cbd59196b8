"""Out-of-bounds writes into caller memory: every output buffer of every entry
point is placed inside a larger allocation whose guard zones (before and after)
hold a sentinel pattern, the call runs on awkward shapes (ragged curves, empty
curves, frequency counts that are not tile multiples, k = 64), and the guards
must come back untouched. Outputs inside the buffers are checked elsewhere."""
from __future__ import annotations

import numpy as np
import pytest

import lightcurves as L
from gpu_util import to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GUARD = 4099  # elements on each side


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2502_00243_gb300 as G_
    return G_


class Guarded:
    """A device buffer of n elements with sentinel-filled guard zones."""

    def __init__(self, n, dtype):
        self.n = n
        self.full = torch.empty(n + 2 * GUARD, dtype=dtype, device="cuda")
        if dtype.is_floating_point:
            self.full.fill_(-1234.5)
        else:
            self.full.fill_(-77)
        self.ref = self.full[:GUARD].clone()
        self.view = self.full[GUARD:GUARD + n]

    def intact(self):
        return bool(torch.equal(self.full[:GUARD], self.ref) and torch.equal(self.full[GUARD + self.n:], self.ref))


def check(*bufs):
    torch.cuda.synchronize()
    for b in bufs:
        assert b.intact(), "a guard zone was written"


SHAPES = [([0, 1, 31, 33, 700, 2500, 0, 64], 1021, 20, 5), ([5, 3000], 4097, 10, 64), ([900, 77], 3, 50, 7),
          ([333, 1200, 1], 2050, 1, 3), ([0, 1, 31, 700, 2500], 1021, 30, 5), ([5, 3000, 64], 777, 16, 7)]


@pytest.mark.parametrize("case", range(len(SHAPES)))
def test_batched_entry_points_stay_inside_their_outputs(G, case):
    ns, F, M, k = SHAPES[case]
    w = L.ragged(60 + case, ns, F, M=M, k=k)
    d = to_dev(w)
    C, nobs = w.ncurves, w.nobs
    ctx = G.Context(0)
    for params in (None, G.fpw_params_default(accum=G.FPW_ACCUM_FP32_COMP), G.fpw_params_default(phase_mode=1)):
        idx, S, Sd = Guarded(C * k, torch.int32), Guarded(C * k, torch.float32), Guarded(C * F, torch.float64)
        G.fpw_periodogram_batch_ex(ctx, None, params, d["offsets"], w.offsets, d["t"], d["x"], d["sigma"],
                                   d["freqs"], M, k, idx.view, S.view, Sd.view)
        check(idx, S, Sd)
        assert ctx.status() == 0
    k0, k1 = F // 3, min(F, F // 3 + 17)
    bins = Guarded((k1 - k0) * nobs, torch.int32)
    G.fpw_periodogram_batch_bins(ctx, None, None, d["offsets"], w.offsets, d["t"], d["x"], d["sigma"], d["freqs"], M,
                                 k0, k1, bins.view)
    check(bins)
    if M % 2 == 0 and M > 2:
        groups = (1, 2)
        mi, mo = Guarded(C * 2 * k, torch.int32), Guarded(C * 2 * k, torch.int32)
        ms, md = Guarded(C * 2 * k, torch.float32), Guarded(C * 2 * F, torch.float64)
        G.fpw_periodogram_batch_multi(ctx, None, None, d["offsets"], w.offsets, d["t"], d["x"], d["sigma"],
                                      d["freqs"], M, groups, k, mi.view, mo.view, ms.view, md.view)
        check(mi, mo, ms, md)
    di, ds, dd = Guarded(C * k, torch.int32), Guarded(C * k, torch.float32), Guarded(C * F, torch.float64)
    G.fpw_periodogram_drift(ctx, None, None, d["offsets"], d["t"], d["x"], d["sigma"], d["freqs"], M, 3, 1.0, k,
                            di.view, ds.view, dd.view)
    check(di, ds, dd)
    H, z = Guarded(C * k, torch.float32), Guarded(C * k, torch.float32)
    G.fpw_phase_entropy_peaks(ctx, None, d["offsets"], d["t"], d["freqs"], M, k, idx.view, H.view, z.view)
    check(H, z)
    if nobs:
        Hd = Guarded(F, torch.float32)
        G.fpw_phase_entropy(ctx, None, d["t"], d["freqs"], M, Hd.view)
        check(Hd)
    ni, ns_ = Guarded(C * k, torch.int32), Guarded(C * k, torch.float32)
    G.fpw_periodogram_batch_noalloc(None, None, d["offsets"], None, d["t"], d["x"], d["sigma"], d["freqs"], M, k,
                                    ni.view, ns_.view)
    check(ni, ns_)
    assert ctx.status() == 0
    ctx.close()


def test_shared_timestamp_path_stays_inside_its_outputs(G):
    from test_gpu_shared import field
    for C, n, F, M, k in ((70, 1000, 3001, 20, 5), (3, 37, 517, 7, 64), (130, 150, 777, 50, 3)):
        t, x, sigma, freqs = field(C + n, C, n, F)
        dd = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (t, x, sigma, freqs)]
        idx, S, Sd = Guarded(C * k, torch.int32), Guarded(C * k, torch.float32), Guarded(C * F, torch.float64)
        ctx = G.Context(0)
        G.fpw_periodogram_shared(ctx, None, None, dd[0], dd[1], dd[2], dd[3], M, k, idx.view, S.view, Sd.view)
        check(idx, S, Sd)
        assert ctx.status() == 0
        ctx.close()


def test_host_entry_point_stays_inside_its_outputs(G):
    w = L.ragged(70, [400, 0, 1300, 5], 2047, M=20, k=6)
    C, k = w.ncurves, w.k
    full_i = np.full(C * k + 2 * GUARD, -77, dtype=np.int32)
    full_s = np.full(C * k + 2 * GUARD, -1234.5, dtype=np.float32)
    ctx = G.Context(0)
    G.fpw_periodogram_batch_host(ctx, None, w.offsets, w.t, w.x, w.sigma, w.freqs, 20, k,
                                 full_i[GUARD:GUARD + C * k], full_s[GUARD:GUARD + C * k])
    assert (full_i[:GUARD] == -77).all() and (full_i[GUARD + C * k:] == -77).all()
    assert (full_s[:GUARD] == -1234.5).all() and (full_s[GUARD + C * k:] == -1234.5).all()
    ctx.close()

"""Bounded waits of the shared-timestamp kernel: a wait that runs out ends the
call with FPW_ETIMEOUT and leaves the context usable.

The kernel's roles (builders of the one-hot operand, the bulk-copy and
tensor-core issuers, the epilogue) hand chunks to each other through
mbarriers, and every such wait has a clock limit. Here the limit is set to one
clock (which also stops each wait from suspending), so the issuer's first wait,
made before the builders can have filled the first chunk, gives up: the kernel
then sets the abort flag for the other roles, waits with the default limit for
its own copies and tensor-core operations in flight, frees its tensor memory
and returns. The next call, with the default limit, must match the oracle."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from gpu_util import assert_S_close, s_bound
from test_gpu_shared import field, run_shared

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_pipeline_wait_runs_out_then_the_context_recovers():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2502_00243_gb300 as G
    ctx = G.Context(0)
    t, x, sigma, freqs = field(91, 130, 700, 4000)
    ctx.set_wait_limit(1)
    idx, S, Sd, st = run_shared(G, ctx, t, x, sigma, freqs, 20, 5)
    assert st == G.FPW_ETIMEOUT
    ctx.set_wait_limit(0)
    for _ in range(2):
        idx, S, Sd, st = run_shared(G, ctx, t, x, sigma, freqs, 20, 5)
        assert st == G.FPW_OK
        S_or = oracle.fpw_shared(t, x, sigma, freqs, 20)
        near = oracle.min_edge(t, freqs, 20) <= 1e-9
        for c in range(x.shape[0]):
            assert_S_close(Sd[c], S_or[c], s_bound(x[c], sigma[c]), mask=~near, what=f"curve {c} after a timeout")
    with pytest.raises(G.FPWError) as ei:
        ctx.set_wait_limit(-1)
    assert ei.value.code == G.FPW_EINVAL
    ctx.close()

"""C-ABI checks that need no GPU: the library builds for sm_103a, loads, exports
every entry point include/fpw.h declares, and its host-only calls behave."""
from __future__ import annotations

import ctypes
import os
import re

import pytest

import paper_2502_00243_gb300 as G

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fpw.h")


@pytest.fixture(scope="module")
def lib():
    G.build()
    return G.lib()


def declared():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"FPW_API\s+[\w\s\*]+?\b(fpw_\w+)\s*\(", text)))


def test_header_declares_the_entry_points():
    names = declared()
    for must in ("fpw_periodogram", "fpw_periodogram_batch", "fpw_periodogram_ex", "fpw_periodogram_batch_ex",
                 "fpw_periodogram_batch_host", "fpw_ctx_create", "fpw_ctx_destroy", "fpw_strerror"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared():
        assert hasattr(lib, name), name
    assert set(declared()) == set(G.EXPORTED)


def test_params_layout_and_defaults(lib):
    p = G.fpw_params_default()
    assert ctypes.sizeof(p) == 48
    assert (p.inv_alpha2, p.phase_mode, p.accum, p.K, p.peak_mode, p.use_graph) == (0.0, 0, 0, 256, 0, 0)
    assert (p.threads, p.freqs_per_thread, p.obs_chunk, p.items_per_slot) == (0, 0, 0, 0)


def test_host_only_calls(lib):
    assert G.fpw_version() >= 1
    assert G.fpw_strerror(0) == "ok"
    assert "invalid argument" in G.fpw_strerror(1)
    assert G.fpw_strerror(999) == "unknown status"


def test_null_context_rejected_without_touching_a_gpu(lib):
    vp = ctypes.c_void_p
    assert lib.fpw_periodogram_ex(None, None, None, None, None, None, 0, None, 0, 1, None) == G.FPW_EINVAL
    assert lib.fpw_periodogram_batch_ex(None, None, None, None, None, 0, None, None, None, None, 0, 1, 0, None, None,
                                        None) == G.FPW_EINVAL
    assert lib.fpw_ctx_status(None) == G.FPW_EINVAL
    assert lib.fpw_periodogram_batch_bins(None, None, None, None, None, 0, None, None, None, None, 0, 1, 0, 0, None,
                                          None) == G.FPW_EINVAL
    v = [ctypes.c_int() for _ in range(4)]
    assert lib.fpw_ctx_last_shape(None, *[ctypes.byref(q) for q in v]) == G.FPW_EINVAL
    assert lib.fpw_ctx_destroy(None) == G.FPW_OK
    assert lib.fpw_ctx_create(None, 0) == G.FPW_EINVAL
    h = vp()
    # no device in this process (or a bad ordinal): create fails cleanly
    assert lib.fpw_ctx_create(ctypes.byref(h), 1 << 20) == G.FPW_EINVAL


def test_library_is_sm103a_only():
    from paper_2502_00243_gb300 import _build
    assert _build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_oracle_and_library_are_independent():
    """Neither side imports, includes or loads the other."""
    import glob
    for f in glob.glob(os.path.join(ROOT, "paper_2502_00243_gb300", "**", "*"), recursive=True):
        if f.endswith((".py", ".cu", ".cuh", ".h")):
            txt = open(f).read()
            assert not re.search(r"^\s*(import|from)\s+oracle\b", txt, re.M), f
            assert "fpw_oracle" not in txt and "liboracle" not in txt, f
    for f in glob.glob(os.path.join(ROOT, "oracle", "*")):
        if f.endswith((".py", ".c", ".h")):
            txt = open(f).read()
            assert not re.search(r"^\s*(import|from)\s+paper_2502_00243_gb300", txt, re.M), f
            assert "#include \"" not in txt and "libfpw" not in txt, f


def _declared_arity():
    """Parameter count of every FPW_API function in the header."""
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    out = {}
    for m in re.finditer(r"FPW_API\s+[\w\s\*]+?\b(fpw_\w+)\s*\(([^)]*)\)", text):
        args = m.group(2).strip()
        out[m.group(1)] = 0 if args in ("", "void") else args.count(",") + 1
    return out


def test_binding_argument_counts_match_the_header(lib):
    arity = _declared_arity()
    assert set(arity) == set(G.EXPORTED)
    for name, n in arity.items():
        argtypes = getattr(lib, name).argtypes
        assert argtypes is not None and len(argtypes) == n, f"{name}: header {n} args, binding {argtypes}"

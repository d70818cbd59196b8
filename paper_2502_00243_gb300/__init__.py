"""Python binding of the GB300 FPW periodogram library (libfpw_gb300.so).

Fast Periodicity Weighting (arXiv:2502.00243): S_FPW of Eq. 1 for every (light
curve, trial frequency) pair, with per-curve top-k peaks (Section 3.5). Every
step runs in the library's sm_103a CUDA kernels; this module only marshals
arguments (torch CUDA tensors provide device memory and streams) and maps
status codes to exceptions. There is no CPU fallback: if the library is not
built, every call raises.

The functions carry the names of the C entry points in include/fpw.h.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfpw_gb300.so")

FPW_OK, FPW_EINVAL, FPW_EDATA, FPW_ENOMEM, FPW_ECUDA, FPW_ETIMEOUT, FPW_ENOTSUP = range(7)
FPW_PHASE_FIXED64, FPW_PHASE_FP64, FPW_PHASE_FP32 = 0, 1, 2
FPW_ACCUM_FP32, FPW_ACCUM_FP64, FPW_ACCUM_FP32_COMP = 0, 1, 2
FPW_PEAK_LOCALMAX, FPW_PEAK_RAW = 0, 1
FPW_MAX_TOPK = 64

EXPORTED = ("fpw_params_default", "fpw_ctx_create", "fpw_ctx_destroy", "fpw_ctx_status", "fpw_periodogram",
            "fpw_periodogram_ex", "fpw_periodogram_batch", "fpw_periodogram_batch_ex", "fpw_periodogram_batch_host",
            "fpw_periodogram_batch_bins", "fpw_ctx_last_shape", "fpw_ctx_set_wait_limit", "fpw_strerror",
            "fpw_version", "fpw_last_cuda_error", "fpw_ctx_set_timing", "fpw_ctx_kernel_time",
            "fpw_periodogram_batch_noalloc", "fpw_ctx_set_shape", "fpw_ctx_clear_shapes",
            "fpw_periodogram_batch_multi", "fpw_phase_entropy", "fpw_phase_entropy_peaks", "fpw_periodogram_shared",
            "fpw_periodogram_drift")


class FPWError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        msg = f"{where}: status {code} ({fpw_strerror(code)})"
        if code == FPW_ECUDA:
            msg += f" [{fpw_last_cuda_error()}]"
        super().__init__(msg)


class fpw_params(ctypes.Structure):
    _fields_ = [("inv_alpha2", ctypes.c_double), ("phase_mode", ctypes.c_int), ("accum", ctypes.c_int),
                ("K", ctypes.c_int), ("peak_mode", ctypes.c_int), ("threads", ctypes.c_int),
                ("freqs_per_thread", ctypes.c_int), ("obs_chunk", ctypes.c_int), ("use_graph", ctypes.c_int),
                ("items_per_slot", ctypes.c_int)]


_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the CUDA library in-tree (nvcc, sm_103a)."""
    from . import _build
    return _build.build(force=force)


def lib():
    """The loaded library; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2502_00243_gb300.build()")
            L = ctypes.CDLL(LIB_PATH)
            vp, i64, ci, d = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
            P = ctypes.POINTER(fpw_params)
            sig = {
                "fpw_params_default": (None, [P]),
                "fpw_ctx_create": (ci, [ctypes.POINTER(vp), ci]),
                "fpw_ctx_destroy": (ci, [vp]),
                "fpw_ctx_status": (ci, [vp]),
                "fpw_periodogram": (ci, [vp, vp, vp, i64, vp, i64, ci, vp]),
                "fpw_periodogram_ex": (ci, [vp, vp, P, vp, vp, vp, i64, vp, i64, ci, vp]),
                "fpw_periodogram_batch": (ci, [vp, i64, vp, vp, vp, vp, i64, ci, ci, vp, vp]),
                "fpw_periodogram_batch_ex": (ci, [vp, vp, P, vp, vp, i64, vp, vp, vp, vp, i64, ci, ci, vp, vp, vp]),
                "fpw_periodogram_batch_host": (ci, [vp, P, vp, i64, vp, vp, vp, vp, i64, ci, ci, vp, vp]),
                "fpw_periodogram_batch_bins": (ci, [vp, vp, P, vp, vp, i64, vp, vp, vp, vp, i64, ci, i64, i64, vp, vp]),
                "fpw_ctx_last_shape": (ci, [vp] + [ctypes.POINTER(ci)] * 4),
                "fpw_ctx_set_wait_limit": (ci, [vp, i64]),
                "fpw_strerror": (ctypes.c_char_p, [ci]),
                "fpw_version": (ci, []),
                "fpw_last_cuda_error": (ctypes.c_char_p, []),
                "fpw_ctx_set_timing": (ci, [vp, ci]),
                "fpw_ctx_kernel_time": (ci, [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)]),
                "fpw_periodogram_batch_noalloc": (ci, [vp, P, vp, vp, i64, vp, vp, vp, vp, i64, ci, ci, vp, vp]),
                "fpw_ctx_set_shape": (ci, [vp, ci, ci, i64, i64, ci, ci, ci, ci]),
                "fpw_ctx_clear_shapes": (ci, [vp]),
                "fpw_phase_entropy": (ci, [vp, vp, vp, i64, vp, i64, ci, vp]),
                "fpw_periodogram_shared": (ci, [vp, vp, P, vp, i64, i64, vp, vp, vp, i64, ci, ci, vp, vp, vp]),
                "fpw_periodogram_drift": (ci, [vp, vp, P, vp, i64, vp, vp, vp, vp, i64, ci, ci, d, ci, vp, vp, vp]),
                "fpw_phase_entropy_peaks": (ci, [vp, vp, vp, i64, vp, vp, i64, ci, ci, vp, vp, vp]),
                "fpw_periodogram_batch_multi": (ci, [vp, vp, P, vp, vp, i64, vp, vp, vp, vp, i64, ci, vp, ci, ci, vp, vp,
                                                     vp, vp]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def fpw_strerror(code: int) -> str:
    return lib().fpw_strerror(int(code)).decode()


def fpw_last_cuda_error() -> str:
    return lib().fpw_last_cuda_error().decode()


def fpw_version() -> int:
    return int(lib().fpw_version())


def fpw_params_default(**overrides) -> fpw_params:
    p = fpw_params()
    lib().fpw_params_default(ctypes.byref(p))
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise AttributeError(k)
        setattr(p, k, v)
    return p


def _check(rc: int, where: str) -> None:
    if rc != FPW_OK:
        raise FPWError(rc, where)


class Context:
    """Owns an fpw_ctx (device scratch, plan and graph caches) on one device."""

    def __init__(self, device: int = 0):
        h = ctypes.c_void_p()
        _check(lib().fpw_ctx_create(ctypes.byref(h), int(device)), "fpw_ctx_create")
        self.handle = h
        self.device = int(device)

    def close(self):
        if self.handle:
            lib().fpw_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def status(self) -> int:
        return int(lib().fpw_ctx_status(self.handle))

    def set_shape(self, M_lo: int, M_hi: int, n_lo: int, n_hi: int, threads: int, freqs_per_thread: int,
                  obs_chunk: int = 0, items_per_slot: int = 0) -> None:
        _check(lib().fpw_ctx_set_shape(self.handle, M_lo, M_hi, n_lo, n_hi, threads, freqs_per_thread, obs_chunk,
                                       items_per_slot), "fpw_ctx_set_shape")

    def clear_shapes(self) -> None:
        _check(lib().fpw_ctx_clear_shapes(self.handle), "fpw_ctx_clear_shapes")

    def set_timing(self, enable: bool) -> None:
        _check(lib().fpw_ctx_set_timing(self.handle, int(bool(enable))), "fpw_ctx_set_timing")

    def set_wait_limit(self, clocks: int) -> None:
        """Limit (SM clocks) of each wait in the shared-timestamp kernel's pipeline; 0 = default."""
        _check(lib().fpw_ctx_set_wait_limit(self.handle, int(clocks)), "fpw_ctx_set_wait_limit")

    def last_shape(self):
        """(threads, freqs_per_thread, obs_chunk, grid) of the latest tile-kernel call."""
        v = [ctypes.c_int() for _ in range(4)]
        _check(lib().fpw_ctx_last_shape(self.handle, *[ctypes.byref(q) for q in v]), "fpw_ctx_last_shape")
        return tuple(q.value for q in v)

    def kernel_time(self):
        """(milliseconds, launches) of the tile kernel since the last query."""
        ms = ctypes.c_double()
        n = ctypes.c_int64()
        _check(lib().fpw_ctx_kernel_time(self.handle, ctypes.byref(ms), ctypes.byref(n)), "fpw_ctx_kernel_time")
        return ms.value, n.value


def fpw_ctx_create(device: int = 0) -> Context:
    return Context(device)


def fpw_ctx_destroy(ctx: Context) -> None:
    ctx.close()


def fpw_ctx_status(ctx: Context) -> int:
    return ctx.status()


def fpw_ctx_set_timing(ctx: Context, enable: bool) -> None:
    ctx.set_timing(enable)


def fpw_ctx_kernel_time(ctx: Context):
    return ctx.kernel_time()


# ---------------------------------------------------------------- marshalling
def _dev(t, dtype, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return ctypes.c_void_p(t.data_ptr()) if t.numel() > 0 else ctypes.c_void_p(t.data_ptr() or None)


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _params(params):
    if params is None:
        return None
    return ctypes.byref(params)


def fpw_periodogram(t, x, sigma, freqs, M: int, S_out):
    """Eq. 1 for one curve at every frequency (synchronous, default context)."""
    import torch
    rc = lib().fpw_periodogram(_dev(t, torch.float64, "t"), _dev(x, torch.float64, "x"),
                               _dev(sigma, torch.float64, "sigma"), t.numel(), _dev(freqs, torch.float64, "freqs"),
                               freqs.numel(), int(M), _dev(S_out, torch.float64, "S_out"))
    _check(rc, "fpw_periodogram")
    return S_out


def fpw_periodogram_ex(ctx: Context, stream, params, t, x, sigma, freqs, M: int, S_out):
    import torch
    rc = lib().fpw_periodogram_ex(ctx.handle, _stream(stream), _params(params), _dev(t, torch.float64, "t"),
                                  _dev(x, torch.float64, "x"), _dev(sigma, torch.float64, "sigma"), t.numel(),
                                  _dev(freqs, torch.float64, "freqs"), freqs.numel(), int(M),
                                  _dev(S_out, torch.float64, "S_out"))
    _check(rc, "fpw_periodogram_ex")
    return S_out


def fpw_periodogram_batch(offsets, t, x, sigma, freqs, M: int, k: int, topk_idx, topk_S):
    import torch
    rc = lib().fpw_periodogram_batch(_dev(offsets, torch.int64, "offsets"), offsets.numel() - 1,
                                     _dev(t, torch.float64, "t"), _dev(x, torch.float64, "x"),
                                     _dev(sigma, torch.float64, "sigma"), _dev(freqs, torch.float64, "freqs"),
                                     freqs.numel(), int(M), int(k), _dev(topk_idx, torch.int32, "topk_idx"),
                                     _dev(topk_S, torch.float32, "topk_S"))
    _check(rc, "fpw_periodogram_batch")
    return topk_idx, topk_S


def fpw_periodogram_batch_ex(ctx: Context, stream, params, offsets, offsets_host, t, x, sigma, freqs, M: int, k: int,
                             topk_idx, topk_S, S_out=None):
    import torch
    oh = None
    if offsets_host is not None:
        offsets_host = np.ascontiguousarray(offsets_host, dtype=np.int64)
        oh = ctypes.c_void_p(offsets_host.ctypes.data)
    rc = lib().fpw_periodogram_batch_ex(
        ctx.handle, _stream(stream), _params(params), _dev(offsets, torch.int64, "offsets"), oh, offsets.numel() - 1,
        _dev(t, torch.float64, "t"), _dev(x, torch.float64, "x"), _dev(sigma, torch.float64, "sigma"),
        _dev(freqs, torch.float64, "freqs"), freqs.numel(), int(M), int(k),
        _dev(topk_idx, torch.int32, "topk_idx") if topk_idx is not None else None,
        _dev(topk_S, torch.float32, "topk_S") if topk_S is not None else None,
        _dev(S_out, torch.float64, "S_out") if S_out is not None else None)
    _check(rc, "fpw_periodogram_batch_ex")
    return topk_idx, topk_S, S_out


def fpw_periodogram_batch_multi(ctx: Context, stream, params, offsets, offsets_host, t, x, sigma, freqs, M_max: int,
                                groups, k: int, topk_idx, topk_offset, topk_S, S_out=None):
    """Several M = M_max / g from one M_max pass (Section 3.4); see include/fpw.h."""
    import torch
    g = np.ascontiguousarray(groups, dtype=np.int32)
    oh = None
    if offsets_host is not None:
        offsets_host = np.ascontiguousarray(offsets_host, dtype=np.int64)
        oh = ctypes.c_void_p(offsets_host.ctypes.data)
    rc = lib().fpw_periodogram_batch_multi(
        ctx.handle, _stream(stream), _params(params), _dev(offsets, torch.int64, "offsets"), oh, offsets.numel() - 1,
        _dev(t, torch.float64, "t"), _dev(x, torch.float64, "x"), _dev(sigma, torch.float64, "sigma"),
        _dev(freqs, torch.float64, "freqs"), freqs.numel(), int(M_max), ctypes.c_void_p(g.ctypes.data), int(g.size),
        int(k), _dev(topk_idx, torch.int32, "topk_idx") if topk_idx is not None else None,
        _dev(topk_offset, torch.int32, "topk_offset") if topk_offset is not None else None,
        _dev(topk_S, torch.float32, "topk_S") if topk_S is not None else None,
        _dev(S_out, torch.float64, "S_out") if S_out is not None else None)
    _check(rc, "fpw_periodogram_batch_multi")
    return topk_idx, topk_offset, topk_S, S_out


def fpw_periodogram_shared(ctx: Context, stream, params, t, x, sigma, freqs, M: int, k: int, topk_idx=None,
                           topk_S=None, S_out=None):
    """Curves sharing the times ``t``: ``x`` and ``sigma`` are ``[C, n]`` CUDA
    tensors (row per curve); top-k ``[C * k]`` and optional dense ``S_out``
    ``[C * F]`` as for the batched call."""
    import torch
    if x.dim() != 2 or sigma.shape != x.shape or x.shape[1] != t.numel():
        raise ValueError("x and sigma must be [ncurves, n] with n = t.numel()")
    rc = lib().fpw_periodogram_shared(
        ctx.handle, _stream(stream), _params(params), _dev(t, torch.float64, "t"), t.numel(), x.shape[0],
        _dev(x, torch.float64, "x"), _dev(sigma, torch.float64, "sigma"), _dev(freqs, torch.float64, "freqs"),
        freqs.numel(), int(M), int(k),
        _dev(topk_idx, torch.int32, "topk_idx") if topk_idx is not None else None,
        _dev(topk_S, torch.float32, "topk_S") if topk_S is not None else None,
        _dev(S_out, torch.float64, "S_out") if S_out is not None else None)
    _check(rc, "fpw_periodogram_shared")


def fpw_periodogram_drift(ctx: Context, stream, params, offsets, t, x, sigma, freqs, M: int, K: int, beta: float,
                          k: int, topk_idx=None, topk_S=None, S_out=None):
    """Baseline drift marginalised (Appendix A.1-A.2): ragged batch as for the
    batched call, K Chebyshev basis functions with prior standard deviation beta."""
    import torch
    rc = lib().fpw_periodogram_drift(
        ctx.handle, _stream(stream), _params(params), _dev(offsets, torch.int64, "offsets"), offsets.numel() - 1,
        _dev(t, torch.float64, "t"), _dev(x, torch.float64, "x"), _dev(sigma, torch.float64, "sigma"),
        _dev(freqs, torch.float64, "freqs"), freqs.numel(), int(M), int(K), float(beta), int(k),
        _dev(topk_idx, torch.int32, "topk_idx") if topk_idx is not None else None,
        _dev(topk_S, torch.float32, "topk_S") if topk_S is not None else None,
        _dev(S_out, torch.float64, "S_out") if S_out is not None else None)
    _check(rc, "fpw_periodogram_drift")


def fpw_phase_entropy(ctx: Context, stream, t, freqs, M: int, H_out):
    """Appendix C phase entropy of one set of times at every frequency."""
    import torch
    rc = lib().fpw_phase_entropy(ctx.handle, _stream(stream), _dev(t, torch.float64, "t"), t.numel(),
                                 _dev(freqs, torch.float64, "freqs"), freqs.numel(), int(M),
                                 _dev(H_out, torch.float32, "H_out"))
    _check(rc, "fpw_phase_entropy")
    return H_out


def fpw_phase_entropy_peaks(ctx: Context, stream, offsets, t, freqs, M: int, k: int, topk_idx, H_out, z_out):
    """Phase entropy and its Hutcheson z-score at each reported peak."""
    import torch
    rc = lib().fpw_phase_entropy_peaks(ctx.handle, _stream(stream), _dev(offsets, torch.int64, "offsets"),
                                       offsets.numel() - 1, _dev(t, torch.float64, "t"),
                                       _dev(freqs, torch.float64, "freqs"), freqs.numel(), int(M), int(k),
                                       _dev(topk_idx, torch.int32, "topk_idx"), _dev(H_out, torch.float32, "H_out"),
                                       _dev(z_out, torch.float32, "z_out"))
    _check(rc, "fpw_phase_entropy_peaks")
    return H_out, z_out


def _host(a, dtype, name):
    if not isinstance(a, np.ndarray) or a.dtype != dtype or not a.flags.c_contiguous:
        raise TypeError(f"{name} must be a C-contiguous numpy {dtype} array")
    return ctypes.c_void_p(a.ctypes.data) if a.size else None


def fpw_periodogram_batch_host(ctx: Context, params, offsets, t, x, sigma, freqs, M: int, k: int, topk_idx, topk_S):
    """End-to-end: host arrays in (numpy, ideally backed by pinned memory), host top-k out."""
    rc = lib().fpw_periodogram_batch_host(ctx.handle, _params(params), _host(offsets, np.int64, "offsets"),
                                          offsets.size - 1, _host(t, np.float64, "t"), _host(x, np.float64, "x"),
                                          _host(sigma, np.float64, "sigma"), _host(freqs, np.float64, "freqs"),
                                          freqs.size, int(M), int(k), _host(topk_idx, np.int32, "topk_idx"),
                                          _host(topk_S, np.float32, "topk_S"))
    _check(rc, "fpw_periodogram_batch_host")
    return topk_idx, topk_S


def fpw_periodogram_batch_bins(ctx: Context, stream, params, offsets, offsets_host, t, x, sigma, freqs, M: int,
                               k0: int, k1: int, bins_out, S_out=None):
    """The batched call's kernels with a bin dump: bins_out int32 ``[(k1 - k0) * nobs]``
    receives the bin of every observation at frequencies k0 <= k < k1."""
    import torch
    oh = None
    if offsets_host is not None:
        offsets_host = np.ascontiguousarray(offsets_host, dtype=np.int64)
        oh = ctypes.c_void_p(offsets_host.ctypes.data)
    rc = lib().fpw_periodogram_batch_bins(
        ctx.handle, _stream(stream), _params(params), _dev(offsets, torch.int64, "offsets"), oh, offsets.numel() - 1,
        _dev(t, torch.float64, "t"), _dev(x, torch.float64, "x"), _dev(sigma, torch.float64, "sigma"),
        _dev(freqs, torch.float64, "freqs"), freqs.numel(), int(M), int(k0), int(k1),
        _dev(bins_out, torch.int32, "bins_out"), _dev(S_out, torch.float64, "S_out") if S_out is not None else None)
    _check(rc, "fpw_periodogram_batch_bins")
    return bins_out, S_out


def fpw_ctx_last_shape(ctx: Context):
    return ctx.last_shape()


def fpw_periodogram_batch_noalloc(stream, params, offsets, offsets_host, t, x, sigma, freqs, M: int, k: int, topk_idx,
                                  topk_S):
    """The batched call for callers that cannot allocate device memory: the
    library's scratch is a fixed device array (see include/fpw.h)."""
    import torch
    oh = None
    if offsets_host is not None:
        offsets_host = np.ascontiguousarray(offsets_host, dtype=np.int64)
        oh = ctypes.c_void_p(offsets_host.ctypes.data)
    rc = lib().fpw_periodogram_batch_noalloc(
        _stream(stream), _params(params), _dev(offsets, torch.int64, "offsets"), oh, offsets.numel() - 1,
        _dev(t, torch.float64, "t"), _dev(x, torch.float64, "x"), _dev(sigma, torch.float64, "sigma"),
        _dev(freqs, torch.float64, "freqs"), freqs.numel(), int(M), int(k), _dev(topk_idx, torch.int32, "topk_idx"),
        _dev(topk_S, torch.float32, "topk_S"))
    _check(rc, "fpw_periodogram_batch_noalloc")
    return topk_idx, topk_S

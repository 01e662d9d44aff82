"""Python binding of libhx, the sm_103a fork-join hot-path library.

Argument marshalling only: every step of every nest runs in the CUDA kernels
of ``lib/libhx.so`` behind the C ABI declared in ``include/hx.h``.  PyTorch
supplies device memory and streams.  There is no CPU fallback: importing this
package fails when the library has not been built, and every call fails when
the tensors are not CUDA tensors.

The functions keep the names of the C entry points (``hx_map_reduce`` etc.).
"""

from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libhx.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libhx.so is not built ({LIB_PATH}); run `python -m paper_2503_10855_b300._build`")

_lib = ctypes.CDLL(LIB_PATH)

HX_OK, HX_ERR_INVALID, HX_ERR_CUDA, HX_ERR_NOMEM, HX_ERR_TIMEOUT, HX_ERR_BUSY = range(6)
STATUS_NAMES = {0: "HX_OK", 1: "HX_ERR_INVALID", 2: "HX_ERR_CUDA", 3: "HX_ERR_NOMEM",
                4: "HX_ERR_TIMEOUT", 5: "HX_ERR_BUSY"}
HX_MAP_REDUCE_MAX_N = 1 << 34
HX_HISTOGRAM_MAX_N = 0xFFFFFFFF

_P = ctypes.c_void_p
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64

_lib.hx_version.restype = ctypes.c_int
_lib.hx_last_error.restype = ctypes.c_char_p
_lib.hx_create.argtypes = [ctypes.POINTER(_P), ctypes.c_int, ctypes.c_size_t]
_lib.hx_create.restype = ctypes.c_int
_lib.hx_destroy.argtypes = [_P]
_lib.hx_destroy.restype = None
_lib.hx_map_reduce.argtypes = [_P, _P, _P, _P, ctypes.c_float, _I64, _P, _P, _P]
_lib.hx_map_reduce.restype = ctypes.c_int
_lib.hx_stencil2d.argtypes = [_P, _P, _P, _I32, _I32, _I32, _P, ctypes.POINTER(_I32), _P]
_lib.hx_stencil2d.restype = ctypes.c_int
_lib.hx_histogram.argtypes = [_P, _P, _I64, _P, _P, _P]
_lib.hx_histogram.restype = ctypes.c_int


class HxError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        msg = _lib.hx_last_error().decode(errors="replace")
        super().__init__(f"{what}: {STATUS_NAMES.get(status, status)}: {msg}")


def _check(status: int, what: str) -> None:
    if status != HX_OK:
        raise HxError(status, what)


def lib() -> ctypes.CDLL:
    """The loaded libhx handle (for callers that use the C ABI directly)."""
    return _lib


def hx_version() -> int:
    return _lib.hx_version()


class Context:
    """Owner of an ``hx_ctx`` (device workspace, per-stream slots)."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0):
        h = _P()
        _check(_lib.hx_create(ctypes.byref(h), device, hbm_budget_bytes), "hx_create")
        self.handle = h
        self.device = device

    def close(self) -> None:
        if self.handle is not None and self.handle.value:
            _lib.hx_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def hx_create(device: int = 0, hbm_budget_bytes: int = 0) -> Context:
    return Context(device, hbm_budget_bytes)


def hx_destroy(ctx: Context) -> None:
    ctx.close()


# ------------------------------------------------------------------ helpers
def _stream_handle(stream):
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    if isinstance(stream, int):
        return _P(stream)
    return _P(stream.cuda_stream)


def _dev_ptr(t, dtype, name, numel=None):
    import torch

    if t is None:
        return _P(0)
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if numel is not None and t.numel() < numel:
        raise ValueError(f"{name} needs at least {numel} elements")
    return _P(t.data_ptr())


# ------------------------------------------------------------------ entry points
def hx_map_reduce(ctx: Context, x, y, a: float, out=None, sum_out=None, sum64_out=None, stream=None):
    """out = fmaf(a, x, y) and s = sum(out) in one fused pass; returns (out, sum_out, sum64_out).

    ``sum_out`` (1 fp32) is allocated when omitted; ``out`` / ``sum64_out`` are
    written only when given.  Asynchronous on ``stream``."""
    import torch

    n = x.numel()
    if y.numel() != n:
        raise ValueError("x and y differ in length")
    if sum_out is None:
        sum_out = torch.empty(1, dtype=torch.float32, device=x.device)
    _check(_lib.hx_map_reduce(ctx.handle, _dev_ptr(x, torch.float32, "x"), _dev_ptr(y, torch.float32, "y"),
                              _dev_ptr(out, torch.float32, "out", n), float(a), n,
                              _dev_ptr(sum_out, torch.float32, "sum_out", 1),
                              _dev_ptr(sum64_out, torch.float64, "sum64_out", 1),
                              _stream_handle(stream)), "hx_map_reduce")
    return out, sum_out, sum64_out


def hx_stencil2d(ctx: Context, u0, u1, iters: int, resid=None, stream=None):
    """``iters`` clamp-to-edge Jacobi sweeps ping-ponging u0 <-> u1 (both ny x nx).

    Returns (final_grid_tensor, resid) where resid[t] = max |u_{t+1} - u_t|."""
    import torch

    if u0.dim() != 2 or u0.shape != u1.shape:
        raise ValueError("u0 and u1 must be 2-D of the same shape")
    ny, nx = u0.shape
    if resid is None:
        resid = torch.empty(max(iters, 1), dtype=torch.float32, device=u0.device)
    in_u1 = _I32(0)
    _check(_lib.hx_stencil2d(ctx.handle, _dev_ptr(u0, torch.float32, "u0"), _dev_ptr(u1, torch.float32, "u1"),
                             nx, ny, iters, _dev_ptr(resid, torch.float32, "resid", iters),
                             ctypes.byref(in_u1), _stream_handle(stream)), "hx_stencil2d")
    return (u1 if in_u1.value else u0), resid


def hx_histogram(ctx: Context, v, bins=None, scan=None, want_scan: bool = True, stream=None):
    """256 uint32 bins of the bytes in ``v`` and (optionally) their exclusive scan."""
    import torch

    if bins is None:
        bins = torch.empty(256, dtype=torch.int32, device=v.device)
    if scan is None and want_scan:
        scan = torch.empty(256, dtype=torch.int32, device=v.device)
    for name, t in (("bins", bins), ("scan", scan)):
        if t is not None and t.dtype not in (torch.int32, torch.uint32):
            raise TypeError(f"{name} must be int32/uint32 (holds uint32 counts)")
    _check(_lib.hx_histogram(ctx.handle, _dev_ptr(v, torch.uint8, "v"), v.numel(),
                             _dev_ptr(bins, bins.dtype, "bins", 256),
                             _dev_ptr(scan, scan.dtype, "scan", 256) if scan is not None else _P(0),
                             _stream_handle(stream)), "hx_histogram")
    return bins, scan

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
# HX_DEBUG=1 selects the debug build (device-side range checks, see
# hx_debug_checks); otherwise the release build.
DEBUG = os.environ.get("HX_DEBUG", "0") == "1"
LIB_PATH = os.path.join(_HERE, "lib", "libhx_debug.so" if DEBUG else "libhx.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{os.path.basename(LIB_PATH)} is not built ({LIB_PATH}); run "
                      f"`python paper_2503_10855_b300/_build.py{' --debug' if DEBUG else ''}`")

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


_lib.hx_debug_inject_launch_failures.argtypes = [_P, _I32, _I32]
_lib.hx_debug_inject_launch_failures.restype = ctypes.c_int
_lib.hx_debug_checks.argtypes = [ctypes.POINTER(_I32), ctypes.POINTER(_I32), ctypes.POINTER(_I64),
                                 ctypes.POINTER(_I64)]
_lib.hx_debug_checks.restype = ctypes.c_int


def hx_debug_inject_launch_failures(ctx: "Context", count: int, after: int = 0) -> None:
    """Test hook: after ``after`` more launching calls on ``ctx``, ``count`` calls fail with HX_ERR_CUDA."""
    _check(_lib.hx_debug_inject_launch_failures(ctx.handle, int(after), int(count)),
           "hx_debug_inject_launch_failures")


CHECK_NAMES = {1: "map tile start", 2: "map partial index", 3: "map fold length", 4: "stencil block",
               5: "histogram split", 6: "batch instance", 7: "batch run", 8: "batch stencil block",
               9: "SRAD region tile", 10: "no-alloc tile", 11: "nest chunk partial", 12: "nest group partial",
               13: "nest arrival ticket"}


def hx_debug_checks():
    """Synchronise the device and read (and clear) the device-side range-check
    records: (enabled, code, a, b); enabled is False in the release build,
    code 0 when no check failed (see CHECK_NAMES)."""
    en, code = _I32(), _I32()
    a, b = _I64(), _I64()
    _check(_lib.hx_debug_checks(ctypes.byref(en), ctypes.byref(code), ctypes.byref(a), ctypes.byref(b)),
           "hx_debug_checks")
    return bool(en.value), int(code.value), int(a.value), int(b.value)


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


# ------------------------------------------------------------------ SRAD-style nest
_lib.hx_srad.argtypes = [_P, _P, _P, _P, _I32, _I32, _I32, ctypes.c_float, _I32, _I32, _I32, _I32, _P, _I32,
                         ctypes.POINTER(_I32), _P]
_lib.hx_srad.restype = ctypes.c_int


def hx_srad(ctx: Context, J0, J1, iters: int, lam: float, roi, q0sq=None, fused: bool = True, C=None, stream=None):
    """``iters`` SRAD iterations ping-ponging J0 <-> J1 (both ny x nx fp32).

    ``roi`` = (r0, r1, c0, c1), half-open.  Returns (result tensor, q0sq)
    where q0sq[t] is the speckle scale iteration t used.  The unfused path
    needs a scratch ``C`` of the image's shape (allocated when omitted)."""
    import torch

    if J0.dim() != 2 or J0.shape != J1.shape:
        raise ValueError("J0 and J1 must be 2-D of the same shape")
    ny, nx = J0.shape
    if q0sq is None:
        q0sq = torch.empty(max(iters, 1), dtype=torch.float32, device=J0.device)
    if not fused and C is None:
        C = torch.empty_like(J0)
    r0, r1, c0, c1 = (int(v) for v in roi)
    in_j1 = _I32(0)
    _check(_lib.hx_srad(ctx.handle, _dev_ptr(J0, torch.float32, "J0"), _dev_ptr(J1, torch.float32, "J1"),
                        _dev_ptr(C, torch.float32, "C") if C is not None else _P(0), nx, ny, iters, float(lam),
                        r0, r1, c0, c1, _dev_ptr(q0sq, torch.float32, "q0sq", iters), 1 if fused else 0,
                        ctypes.byref(in_j1), _stream_handle(stream)), "hx_srad")
    return (J1 if in_j1.value else J0), q0sq


# ------------------------------------------------------------------ generic nests
HX_NEST_MAX_DIMS, HX_NEST_MAX_OPS, HX_NEST_MAX_INPUTS, HX_NEST_MAX_CONSTS = 3, 32, 4, 8
NEST_OPS = {"in": 1, "const": 2, "index": 3, "add": 4, "sub": 5, "mul": 6, "div": 7,
            "fma": 8, "neg": 9, "abs": 10, "min": 11, "max": 12, "sqrt": 13}
MONOIDS = {"sum": 0, "max": 1, "min": 2, "prod": 3, "argmax": 4, "argmin": 5}
TREES = {"warp": 0, "chunk": 1, "seq": 2}


class NestOp(ctypes.Structure):
    _fields_ = [("code", _I32), ("arg", _I32)]


class Nest(ctypes.Structure):
    """Mirror of ``hx_nest`` (see include/hx.h)."""

    _fields_ = [("ndim", _I32), ("reduce_dims", _I32), ("monoid", _I32), ("tree", _I32),
                ("dims", _I64 * HX_NEST_MAX_DIMS), ("chunk", _I64), ("n_ops", _I32), ("pad_", _I32),
                ("ops", NestOp * HX_NEST_MAX_OPS), ("consts", ctypes.c_float * HX_NEST_MAX_CONSTS),
                ("inputs", _P * HX_NEST_MAX_INPUTS),
                ("strides", (_I64 * HX_NEST_MAX_DIMS) * HX_NEST_MAX_INPUTS),
                ("out", _P), ("result", _P), ("result64", _P), ("result_index", _P)]


_NP = ctypes.POINTER(Nest)
_lib.hx_fork_reduce.argtypes = [_P, _NP, _P]
_lib.hx_fork_reduce.restype = ctypes.c_int
_lib.hx_nest_prepare.argtypes = [_NP]
_lib.hx_nest_prepare.restype = ctypes.c_int
_lib.hx_nest_source.argtypes = [_NP, ctypes.c_char_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]
_lib.hx_nest_source.restype = ctypes.c_int


def make_nest(program, inputs, dims, reduce_dims, monoid="sum", consts=(), out=None, result=None,
              result64=None, result_index=None, tree="warp", chunk=0) -> Nest:
    """Fill an ``hx_nest``.  ``program``: postfix list of op names or (name, arg)
    pairs (or raw integer codes).  ``inputs``: float32 tensors whose shape is
    ``dims``; each one's own element strides are its addressing (transposes,
    ``expand`` views with stride 0).  Outputs are tensors or None."""
    import torch

    nest = Nest()
    dims = tuple(int(d) for d in dims)
    nest.ndim = len(dims)
    nest.reduce_dims = int(reduce_dims)
    nest.monoid = MONOIDS[monoid] if isinstance(monoid, str) else int(monoid)
    nest.tree = TREES[tree] if isinstance(tree, str) else int(tree)
    nest.chunk = int(chunk)
    for d, v in enumerate(dims[:HX_NEST_MAX_DIMS]):
        nest.dims[d] = v
    if len(program) > HX_NEST_MAX_OPS:
        raise ValueError("a nest program holds at most 32 ops")
    nest.n_ops = len(program)
    for k, item in enumerate(program):
        name, arg = (item, 0) if isinstance(item, (str, int)) else item
        nest.ops[k].code = NEST_OPS[name] if isinstance(name, str) else int(name)
        nest.ops[k].arg = int(arg)
    for k, c in enumerate(consts):
        nest.consts[k] = float(c)
    if len(inputs) > HX_NEST_MAX_INPUTS:
        raise ValueError("a nest reads at most 4 inputs")
    for k, t in enumerate(inputs):
        if t is None:
            continue
        if not isinstance(t, torch.Tensor) or t.dtype != torch.float32:
            raise TypeError(f"input {k} must be a float32 tensor")
        if tuple(t.shape) != dims:
            raise ValueError(f"input {k} has shape {tuple(t.shape)}, the fork is {dims}")
        nest.inputs[k] = t.data_ptr()
        for d in range(len(dims)):
            nest.strides[k][d] = t.stride(d)
    for name, t, dt in (("out", out, torch.float32), ("result", result, torch.float32),
                        ("result64", result64, torch.float64), ("result_index", result_index, torch.int64)):
        if t is not None:
            if t.dtype != dt or not t.is_contiguous():
                raise TypeError(f"{name} must be a contiguous {dt} tensor")
            setattr(nest, name, t.data_ptr())
    return nest


def hx_nest_prepare(nest: Nest) -> None:
    _check(_lib.hx_nest_prepare(ctypes.byref(nest)), "hx_nest_prepare")


def hx_nest_source(nest: Nest) -> str:
    n = ctypes.c_size_t()
    _check(_lib.hx_nest_source(ctypes.byref(nest), None, 0, ctypes.byref(n)), "hx_nest_source")
    buf = ctypes.create_string_buffer(n.value + 1)
    _check(_lib.hx_nest_source(ctypes.byref(nest), buf, n.value + 1, None), "hx_nest_source")
    return buf.value.decode()


def hx_fork_reduce(ctx: Context, nest: Nest, stream=None) -> None:
    _check(_lib.hx_fork_reduce(ctx.handle, ctypes.byref(nest), _stream_handle(stream)), "hx_fork_reduce")


def fork_reduce(ctx: Context, program, inputs, dims, reduce_dims, monoid="sum", consts=(), want_out=False,
                want_result64=False, tree="warp", chunk=0, device=None, stream=None):
    """Run a nest, allocating its outputs; returns (out, result, result_index, result64).

    ``out`` has shape ``dims``; the results have the shape of the outer
    ``ndim - reduce_dims`` dimensions (None where not requested)."""
    import torch

    dims = tuple(int(d) for d in dims)
    if device is None:
        device = next((t.device for t in inputs if t is not None), torch.device("cuda", ctx.device))
    outer = dims[:len(dims) - reduce_dims] if reduce_dims else None
    out = torch.empty(dims, dtype=torch.float32, device=device) if (want_out or not reduce_dims) else None
    result = result64 = index = None
    if reduce_dims:
        result = torch.empty(outer, dtype=torch.float32, device=device)
        if want_result64:
            result64 = torch.empty(outer, dtype=torch.float64, device=device)
        m = MONOIDS[monoid] if isinstance(monoid, str) else int(monoid)
        if m >= 4:
            index = torch.empty(outer, dtype=torch.int64, device=device)
    nest = make_nest(program, inputs, dims, reduce_dims, monoid, consts, out, result, result64, index, tree, chunk)
    hx_fork_reduce(ctx, nest, stream)
    return out, result, index, result64


# ------------------------------------------------------------------ batches
HX_TASK_MAP_REDUCE, HX_TASK_STENCIL2D, HX_TASK_HISTOGRAM = 0, 1, 2


class _TaskMR(ctypes.Structure):
    _fields_ = [("x", _P), ("y", _P), ("out", _P), ("sum", _P), ("sum64", _P),
                ("a", ctypes.c_float), ("pad", _I32), ("n", _I64)]


class _TaskST(ctypes.Structure):
    _fields_ = [("u0", _P), ("u1", _P), ("resid", _P), ("nx", _I32), ("ny", _I32),
                ("iters", _I32), ("pad", _I32)]


class _TaskHI(ctypes.Structure):
    _fields_ = [("v", _P), ("bins", _P), ("scan", _P), ("n", _I64)]


class _TaskU(ctypes.Union):
    _fields_ = [("mr", _TaskMR), ("st", _TaskST), ("hi", _TaskHI)]


class HxTask(ctypes.Structure):
    """Mirror of ``hx_task`` (64 bytes).  ``keep`` holds the tensors it points to."""

    _fields_ = [("kind", _I32), ("reserved", _I32), ("u", _TaskU)]


assert ctypes.sizeof(HxTask) == 64

_lib.hx_batch_plan.argtypes = [_P, ctypes.POINTER(HxTask), _I32, ctypes.POINTER(_P), ctypes.POINTER(_I32)]
_lib.hx_batch_plan.restype = ctypes.c_int
_lib.hx_batch_plan_ex.argtypes = [_P, ctypes.POINTER(HxTask), _I32, _I32, ctypes.POINTER(_P), ctypes.POINTER(_I32)]
_lib.hx_batch_plan_ex.restype = ctypes.c_int
_lib.hx_batch_status.argtypes = [_P]
_lib.hx_batch_status.restype = ctypes.c_int
_lib.hx_debug_batch_stall.argtypes = [_P, _I32, _I64]
_lib.hx_debug_batch_stall.restype = ctypes.c_int
HX_BATCH_ROUNDS, HX_BATCH_ONE_LAUNCH = 1, 2
_lib.hx_batch_describe.argtypes = [_P, ctypes.c_char_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]
_lib.hx_batch_describe.restype = ctypes.c_int
_lib.hx_batch_launch.argtypes = [_P, _P]
_lib.hx_batch_launch.restype = ctypes.c_int
_lib.hx_batch_free.argtypes = [_P]
_lib.hx_batch_free.restype = None
_lib.hx_batch_submit.argtypes = [_P, ctypes.POINTER(HxTask), _I32, _P, ctypes.POINTER(ctypes.c_uint64)]
_lib.hx_batch_submit.restype = ctypes.c_int
_lib.hx_batch_query.argtypes = [_P, ctypes.c_uint64]
_lib.hx_batch_query.restype = ctypes.c_int


def map_reduce_task(x, y, a: float, sum_out, out=None, sum64_out=None) -> HxTask:
    import torch

    n = x.numel()
    if y.numel() != n:
        raise ValueError("x and y differ in length")
    t = HxTask()
    t.kind = HX_TASK_MAP_REDUCE
    m = t.u.mr
    m.x, m.y = _dev_ptr(x, torch.float32, "x"), _dev_ptr(y, torch.float32, "y")
    m.out = _dev_ptr(out, torch.float32, "out", n)
    m.sum = _dev_ptr(sum_out, torch.float32, "sum_out", 1)
    m.sum64 = _dev_ptr(sum64_out, torch.float64, "sum64_out", 1)
    m.a, m.n = float(a), n
    t.keep = (x, y, out, sum_out, sum64_out)
    return t


def stencil_task(u0, u1, iters: int, resid) -> HxTask:
    import torch

    if u0.dim() != 2 or u0.shape != u1.shape:
        raise ValueError("u0 and u1 must be 2-D of the same shape")
    t = HxTask()
    t.kind = HX_TASK_STENCIL2D
    s = t.u.st
    s.u0, s.u1 = _dev_ptr(u0, torch.float32, "u0"), _dev_ptr(u1, torch.float32, "u1")
    s.resid = _dev_ptr(resid, torch.float32, "resid", iters)
    s.ny, s.nx = u0.shape
    s.iters = iters
    t.keep = (u0, u1, resid)
    return t


def histogram_task(v, bins, scan=None) -> HxTask:
    import torch

    t = HxTask()
    t.kind = HX_TASK_HISTOGRAM
    h = t.u.hi
    h.v = _dev_ptr(v, torch.uint8, "v")
    h.bins = _dev_ptr(bins, bins.dtype, "bins", 256)
    h.scan = _dev_ptr(scan, scan.dtype, "scan", 256) if scan is not None else _P(0)
    h.n = v.numel()
    t.keep = (v, bins, scan)
    return t


def _task_array(tasks):
    arr = (HxTask * len(tasks))()
    for i, t in enumerate(tasks):
        ctypes.memmove(ctypes.byref(arr[i]), ctypes.byref(t), ctypes.sizeof(HxTask))
    return arr


class Batch:
    """A planned batch (``hx_batch``): device work-list bound to the tasks' buffers."""

    def __init__(self, ctx: Context, tasks, rounds=None):
        """``rounds``: None for the default schedule, True for one launch per
        sweep (HX_BATCH_ROUNDS), False for every sweep in one launch
        (HX_BATCH_ONE_LAUNCH)."""
        self.ctx = ctx
        self.keep = [getattr(t, "keep", None) for t in tasks]
        arr = _task_array(tasks)
        h = _P()
        n_rounds = _I32(0)
        flags = 0 if rounds is None else (HX_BATCH_ROUNDS if rounds else HX_BATCH_ONE_LAUNCH)
        _check(_lib.hx_batch_plan_ex(ctx.handle, arr, len(tasks), flags, ctypes.byref(h), ctypes.byref(n_rounds)),
               "hx_batch_plan")
        self.handle = h
        self.rounds = n_rounds.value

    def launch(self, stream=None) -> None:
        _check(_lib.hx_batch_launch(self.handle, _stream_handle(stream)), "hx_batch_launch")

    def status(self) -> None:
        """Raise HxError (HX_ERR_TIMEOUT) if a wait between sweeps ran out of
        time in a completed launch (call after synchronising its stream)."""
        _check(_lib.hx_batch_status(self.handle), "hx_batch_status")

    def describe(self) -> str:
        """The plan as text (hx_batch_describe): one line per instance."""
        need = ctypes.c_size_t(0)
        _check(_lib.hx_batch_describe(self.handle, None, 0, ctypes.byref(need)), "hx_batch_describe")
        buf = ctypes.create_string_buffer(need.value)
        _check(_lib.hx_batch_describe(self.handle, buf, need.value, None), "hx_batch_describe")
        return buf.value.decode()

    def debug_stall(self, task: int, wait_limit_ns: int) -> None:
        """Test hook (hx_debug_batch_stall): task's later sweeps wait for a block
        that never comes, every wait gives up after wait_limit_ns."""
        _check(_lib.hx_debug_batch_stall(self.handle, task, wait_limit_ns), "hx_debug_batch_stall")

    def close(self) -> None:
        if getattr(self, "handle", None) is not None and self.handle.value:
            _lib.hx_batch_free(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def hx_batch_plan(ctx: Context, tasks, rounds=None) -> Batch:
    return Batch(ctx, tasks, rounds)


def hx_batch_launch(batch: Batch, stream=None) -> None:
    batch.launch(stream)


def hx_batch_free(batch: Batch) -> None:
    batch.close()


def hx_batch_submit(ctx: Context, tasks, stream=None) -> int:
    """Plan + launch + completion record; returns a ticket for hx_batch_query."""
    arr = _task_array(tasks)
    ticket = ctypes.c_uint64(0)
    _check(_lib.hx_batch_submit(ctx.handle, arr, len(tasks), _stream_handle(stream), ctypes.byref(ticket)),
           "hx_batch_submit")
    return ticket.value


def hx_batch_query(ctx: Context, ticket: int) -> bool:
    """True once the submission completed (the ticket is then retired), False while pending."""
    st = _lib.hx_batch_query(ctx.handle, ticket)
    if st == HX_ERR_BUSY:
        return False
    _check(st, "hx_batch_query")
    return True


# ------------------------------------------------------------------ tuning
HX_TUNE_CLASSES = 40


class TuneTable(ctypes.Structure):
    """Mirror of ``hx_tune_table``: per-size-class choices (see include/hx.h)."""

    _fields_ = [("map_vecs", _I32 * HX_TUNE_CLASSES), ("hist_threads", _I32 * HX_TUNE_CLASSES),
                ("stencil_rows", _I32 * HX_TUNE_CLASSES), ("nest_lane_elems", _I32 * HX_TUNE_CLASSES),
                ("batch_map_run", _I32),
                ("batch_stencil_run", _I32)]

    def as_dict(self) -> dict:
        return {"map_vecs": list(self.map_vecs), "hist_threads": list(self.hist_threads),
                "stencil_rows": list(self.stencil_rows), "nest_lane_elems": list(self.nest_lane_elems),
                "batch_map_run": self.batch_map_run,
                "batch_stencil_run": self.batch_stencil_run}


_TP = ctypes.POINTER(TuneTable)
_lib.hx_tune_table_default.argtypes = [_TP]
_lib.hx_tune_table_default.restype = None
_lib.hx_tune_table_check.argtypes = [_TP]
_lib.hx_tune_table_check.restype = ctypes.c_int
_lib.hx_tune_table_save.argtypes = [_TP, ctypes.c_char_p]
_lib.hx_tune_table_save.restype = ctypes.c_int
_lib.hx_tune_table_load.argtypes = [_TP, ctypes.c_char_p]
_lib.hx_tune_table_load.restype = ctypes.c_int
_lib.hx_tune_get.argtypes = [_P, _TP]
_lib.hx_tune_get.restype = ctypes.c_int
_lib.hx_tune_set.argtypes = [_P, _TP]
_lib.hx_tune_set.restype = ctypes.c_int
_lib.hx_autotune.argtypes = [_P, _I32, _P]
_lib.hx_autotune.restype = ctypes.c_int


def hx_tune_table_default() -> TuneTable:
    t = TuneTable()
    _lib.hx_tune_table_default(ctypes.byref(t))
    return t


def hx_tune_table_check(t: TuneTable) -> None:
    _check(_lib.hx_tune_table_check(ctypes.byref(t)), "hx_tune_table_check")


def hx_tune_table_save(t: TuneTable, path: str) -> None:
    _check(_lib.hx_tune_table_save(ctypes.byref(t), os.fsencode(path)), "hx_tune_table_save")


def hx_tune_table_load(path: str) -> TuneTable:
    t = TuneTable()
    _check(_lib.hx_tune_table_load(ctypes.byref(t), os.fsencode(path)), "hx_tune_table_load")
    return t


def hx_tune_get(ctx: Context) -> TuneTable:
    t = TuneTable()
    _check(_lib.hx_tune_get(ctx.handle, ctypes.byref(t)), "hx_tune_get")
    return t


def hx_tune_set(ctx: Context, t: TuneTable) -> None:
    _check(_lib.hx_tune_set(ctx.handle, ctypes.byref(t)), "hx_tune_set")


def hx_autotune(ctx: Context, max_log2: int = 26, stream=None) -> TuneTable:
    """Measure every size class up to 2^max_log2 on the device; returns the new table."""
    _check(_lib.hx_autotune(ctx.handle, max_log2, _stream_handle(stream)), "hx_autotune")
    return hx_tune_get(ctx)


# ------------------------------------------------------------------ serving
HX_SERVE_CONTINUOUS, HX_SERVE_PER_LAUNCH = 0, 1


# hx_server_done_fn: (user, req_id, status, latency_s)
SERVER_DONE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int, ctypes.c_double)


class ServerConfig(ctypes.Structure):
    _fields_ = [("mode", _I32), ("max_inflight", _I32), ("hbm_budget_bytes", ctypes.c_size_t),
                ("max_steps_in_flight", _I32), ("max_step_requests", _I32), ("step_quantum_bytes", ctypes.c_size_t),
                ("step_target_bytes", ctypes.c_size_t), ("on_done", SERVER_DONE_FN), ("on_done_user", _P),
                ("direct_max", _I32), ("direct_sweep_bytes", ctypes.c_int64), ("max_step_sweeps", _I32),
                ("pad_", _I32)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", _I64), ("admitted", _I64), ("completed", _I64), ("launches", _I64),
                ("failed", _I64), ("footprint_in_flight", ctypes.c_size_t), ("peak_footprint", ctypes.c_size_t)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib.hx_server_create.argtypes = [_P, ctypes.POINTER(ServerConfig), ctypes.POINTER(_P)]
_lib.hx_server_create.restype = ctypes.c_int
_lib.hx_server_destroy.argtypes = [_P]
_lib.hx_server_destroy.restype = None
_lib.hx_server_submit.argtypes = [_P, ctypes.POINTER(HxTask), ctypes.POINTER(ctypes.c_uint64)]
_lib.hx_server_submit.restype = ctypes.c_int
_lib.hx_server_poll.argtypes = [_P, ctypes.c_uint64, ctypes.POINTER(ctypes.c_double)]
_lib.hx_server_poll.restype = ctypes.c_int
_lib.hx_server_drain.argtypes = [_P, ctypes.c_double]
_lib.hx_server_drain.restype = ctypes.c_int
class ServerStepRecord(ctypes.Structure):
    _fields_ = [("issue_s", ctypes.c_double), ("done_s", ctypes.c_double), ("requests", _I32), ("direct", _I32)]


_lib.hx_server_get_timeline.argtypes = [_P, ctypes.POINTER(ServerStepRecord), _I32, ctypes.POINTER(_I32)]
_lib.hx_debug_server_stall.argtypes = [_P, _I64]
_lib.hx_debug_server_stall.restype = ctypes.c_int
_lib.hx_server_get_timeline.restype = ctypes.c_int
_lib.hx_server_get_stats.argtypes = [_P, ctypes.POINTER(ServerStats)]
_lib.hx_server_get_stats.restype = ctypes.c_int
_lib.hx_server_run_trace.argtypes = [_P, ctypes.POINTER(HxTask), ctypes.POINTER(ctypes.c_double), _I32,
                                     ctypes.c_double, ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(ctypes.c_double)]
_lib.hx_server_run_trace.restype = ctypes.c_int


class Server:
    """An ``hx_server``: admission + continuous batching (or per-launch) request loop."""

    def __init__(self, ctx: Context, mode: int = HX_SERVE_CONTINUOUS, hbm_budget_bytes: int = 0,
                 max_inflight: int = 0, max_steps_in_flight: int = 0, max_step_requests: int = 0,
                 step_quantum_bytes: int = 0, step_target_bytes: int = 0, on_done=None, direct_max: int = 0,
                 direct_sweep_bytes: int = 0, max_step_sweeps: int = 0):
        """on_done(req_id, status, latency_s), if given, is called from the
        server's completion thread once per request (see hx_server_done_fn)."""
        self._on_done = None
        if on_done is not None:
            self._on_done = SERVER_DONE_FN(lambda _user, rid, st, lat: on_done(int(rid), int(st), float(lat)))
        cfg = ServerConfig(mode, max_inflight, hbm_budget_bytes, max_steps_in_flight, max_step_requests,
                           step_quantum_bytes, step_target_bytes,
                           self._on_done if self._on_done is not None else SERVER_DONE_FN(), None, direct_max,
                           direct_sweep_bytes, max_step_sweeps)
        h = _P()
        _check(_lib.hx_server_create(ctx.handle, ctypes.byref(cfg), ctypes.byref(h)), "hx_server_create")
        self.ctx = ctx
        self.handle = h
        self.keep = []

    def submit(self, task: HxTask) -> int:
        rid = ctypes.c_uint64(0)
        self.keep.append(getattr(task, "keep", None))
        _check(_lib.hx_server_submit(self.handle, ctypes.byref(task), ctypes.byref(rid)), "hx_server_submit")
        return rid.value

    def poll(self, req_id: int):
        """(done, latency_s or None)."""
        lat = ctypes.c_double(0.0)
        st = _lib.hx_server_poll(self.handle, req_id, ctypes.byref(lat))
        if st == HX_ERR_BUSY:
            return False, None
        _check(st, "hx_server_poll")
        return True, lat.value

    def drain(self, timeout_s: float = 60.0) -> None:
        _check(_lib.hx_server_drain(self.handle, timeout_s), "hx_server_drain")

    def debug_stall(self, wait_limit_ns: int) -> None:
        """Test hook: stall the next multi-sweep step (hx_debug_server_stall)."""
        _check(_lib.hx_debug_server_stall(self.handle, int(wait_limit_ns)), "hx_debug_server_stall")

    def timeline(self, max_records: int = 1 << 16) -> list:
        """The server's step records (hx_server_get_timeline) as dicts."""
        n = _I32(0)
        _check(_lib.hx_server_get_timeline(self.handle, None, 0, ctypes.byref(n)), "hx_server_get_timeline")
        k = min(n.value, max_records)
        arr = (ServerStepRecord * max(k, 1))()
        _check(_lib.hx_server_get_timeline(self.handle, arr, k, ctypes.byref(n)), "hx_server_get_timeline")
        return [{"issue_s": r.issue_s, "done_s": r.done_s, "requests": r.requests, "direct": bool(r.direct)}
                for r in arr[:k]]

    def stats(self) -> dict:
        st = ServerStats()
        _check(_lib.hx_server_get_stats(self.handle, ctypes.byref(st)), "hx_server_get_stats")
        return st.as_dict()

    def run_trace(self, tasks, arrival_s, timeout_s: float = 60.0):
        """Open-loop replay; returns (latencies_s list, makespan_s)."""
        n = len(tasks)
        arr = _task_array(tasks)
        self.keep.append([getattr(t, "keep", None) for t in tasks])
        arrivals = (ctypes.c_double * n)(*arrival_s)
        lat = (ctypes.c_double * n)()
        mk = ctypes.c_double(0.0)
        _check(_lib.hx_server_run_trace(self.handle, arr, arrivals, n, timeout_s, lat, ctypes.byref(mk)),
               "hx_server_run_trace")
        return list(lat), mk.value

    def close(self) -> None:
        if getattr(self, "handle", None) is not None and self.handle.value:
            _lib.hx_server_destroy(self.handle)
        self.handle = None
        self.keep = []

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def hx_server_create(ctx: Context, **kw) -> Server:
    return Server(ctx, **kw)

"""CPU oracle for the fork-join hot path -- TEST INFRASTRUCTURE ONLY.

Only the tests, the smoke check and the benchmark's CPU-baseline leg import
this package.  The product path (the CUDA library and its Python binding)
never does, and this package imports nothing from it.

The nests are evaluated by ``hx_oracle.c``: plain sequential loops that walk
each fork grid in lexicographic order and fold every reduction in increasing
thread-ID order (Hercules paper, Sec. 3.3), in double precision unless a
function says otherwise.  This module only marshals numpy arrays in and out.

Parity status: every function here is pinned by the ``-m "not gpu"`` tests
(closed forms, library routines on special cases, brute force on tiny
inputs, values worked by hand).  In ``srad`` the mapping from the
coefficient of variation to the diffusion coefficient,
c = 1/(1 + (q^2 - q0^2)/(q0^2 (1 + q0^2))), is pinned by hand-worked values
of the published SRAD scheme (the paper does not print SRAD's arithmetic).
"""

from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hx_oracle.c")
_LIB = os.path.join(_HERE, "libhx_oracle.so")

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fast-math, no FP contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared",
                               "-ffp-contract=off", "-fno-fast-math", "-Wall",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _get():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        lib.hxo_map_reduce_f64.argtypes = [P, P, ctypes.c_double, ctypes.c_int64, P, P]
        lib.hxo_map_reduce_f64.restype = None
        lib.hxo_monoid_reduce_f64.argtypes = [ctypes.c_int, P, P, ctypes.c_double,
                                              ctypes.c_int64, P]
        lib.hxo_monoid_reduce_f64.restype = ctypes.c_int
        for name in ("hxo_jacobi_f64", "hxo_jacobi_f32"):
            f = getattr(lib, name)
            f.argtypes = [P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, P, P]
            f.restype = ctypes.c_int
        lib.hxo_histogram_u8.argtypes = [P, ctypes.c_int64, P, P]
        lib.hxo_histogram_u8.restype = None
        I32 = ctypes.c_int32
        lib.hxo_srad_f64.argtypes = [P, I32, I32, I32, ctypes.c_double, I32, I32, I32, I32, P, P]
        lib.hxo_srad_f64.restype = ctypes.c_int
        lib.hxo_srad_f32.argtypes = [P, I32, I32, I32, ctypes.c_float, I32, I32, I32, I32, P, P]
        lib.hxo_srad_f32.restype = ctypes.c_int
        I = ctypes.c_int
        lib.hxo_fork_reduce.argtypes = [I, P, I, I, I, P, P, I, P, P, P, P, P]
        lib.hxo_fork_reduce.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data) if a.size else ctypes.c_void_p(0)


def map_reduce(x: np.ndarray, y: np.ndarray, a: float, want_out: bool = True):
    """out[i] = a*x[i] + y[i] (fp64), s = sum of out in index order (fp64).

    Returns (out or None, s)."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    y = np.ascontiguousarray(y, dtype=np.float32)
    assert x.shape == y.shape and x.ndim == 1
    n = x.size
    out = np.empty(n, dtype=np.float64) if want_out else None
    s = np.zeros(1, dtype=np.float64)
    _get().hxo_map_reduce_f64(_ptr(x), _ptr(y), float(a), n,
                              _ptr(out) if want_out else ctypes.c_void_p(0), _ptr(s))
    return out, float(s[0])


MONOIDS = {"sum": 0, "max": 1, "min": 2, "prod": 3}


def monoid_reduce(op: str, x: np.ndarray, a: float = 1.0, y: np.ndarray | None = None) -> float:
    """Fold of a*x[i] + y[i] under the monoid ``op`` in index order (fp64)."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    if y is not None:
        y = np.ascontiguousarray(y, dtype=np.float32)
        assert y.shape == x.shape
    r = np.zeros(1, dtype=np.float64)
    rc = _get().hxo_monoid_reduce_f64(MONOIDS[op], _ptr(x),
                                      _ptr(y) if y is not None else ctypes.c_void_p(0),
                                      float(a), x.size, _ptr(r))
    assert rc == 0
    return float(r[0])


def jacobi(u0: np.ndarray, iters: int, precision: str = "f64"):
    """Clamp-to-edge 5-point Jacobi, ``iters`` sweeps; returns (u_final, resid[iters])."""
    assert u0.ndim == 2
    ny, nx = u0.shape
    dt = np.float64 if precision == "f64" else np.float32
    src = np.ascontiguousarray(u0, dtype=dt)
    out = np.empty_like(src)
    resid = np.zeros(max(iters, 0), dtype=dt)
    fn = _get().hxo_jacobi_f64 if precision == "f64" else _get().hxo_jacobi_f32
    rc = fn(_ptr(src), nx, ny, iters, _ptr(out), _ptr(resid) if iters > 0 else ctypes.c_void_p(0))
    if rc:
        raise MemoryError("oracle jacobi: allocation failed")
    return out, resid


def histogram(v: np.ndarray):
    """256 uint32 bin counts of the bytes in ``v`` and their exclusive prefix sum."""
    v = np.ascontiguousarray(v, dtype=np.uint8).ravel()
    bins = np.zeros(256, dtype=np.uint32)
    scan = np.zeros(256, dtype=np.uint32)
    _get().hxo_histogram_u8(_ptr(v), v.size, _ptr(bins), _ptr(scan))
    return bins, scan


# Op codes and monoid codes of the fork-join nest interpreter (hxo_fork_reduce).
NEST_OPS = {"in": 1, "const": 2, "index": 3, "add": 4, "sub": 5, "mul": 6, "div": 7,
            "fma": 8, "neg": 9, "abs": 10, "min": 11, "max": 12, "sqrt": 13}
NEST_MONOIDS = {"sum": 0, "max": 1, "min": 2, "prod": 3, "argmax": 4, "argmin": 5}


def _encode_program(program):
    codes = []
    for item in program:
        name, arg = (item, 0) if isinstance(item, str) else item
        codes += [NEST_OPS[name] if isinstance(name, str) else int(name), int(arg)]
    return np.asarray(codes, dtype=np.int32)


def fork_reduce(program, inputs, dims, reduce_dims, monoid="sum", consts=(), want_out=True):
    """Sequential evaluation of a fork-join nest (see ``hxo_fork_reduce``).

    ``program``: postfix list of op names or (name, arg) pairs.  ``inputs``:
    float32 numpy arrays whose shape is ``dims``; each one's own element
    strides (transposes, ``np.broadcast_to`` views) give the addressing.
    Returns (out or None, result, index or None): ``out`` has shape ``dims``,
    ``result`` (float64) and ``index`` (int64) the shape of the outer
    ``ndim - reduce_dims`` dimensions.
    """
    dims = tuple(int(d) for d in dims)
    ndim = len(dims)
    ops = _encode_program(program)
    arrs, strides = [], np.zeros((max(len(inputs), 1), 3), dtype=np.int64)
    for k, a in enumerate(inputs):
        assert a.dtype == np.float32 and a.shape == dims, (a.dtype, a.shape, dims)
        arrs.append(a)
        for d in range(ndim):
            strides[k, d] = a.strides[d] // 4
    ptrs = (ctypes.c_void_p * max(len(arrs), 1))(*[ctypes.c_void_p(a.ctypes.data) for a in arrs])
    c = np.zeros(8, dtype=np.float32)
    c[:len(consts)] = consts
    outer_shape = dims[:ndim - reduce_dims]
    n_outer = int(np.prod(outer_shape, dtype=np.int64))
    out = np.zeros(dims, dtype=np.float32) if want_out else None
    result = np.zeros(max(n_outer, 1), dtype=np.float64)
    index = np.zeros(max(n_outer, 1), dtype=np.int64)
    dims_a = np.asarray(dims + (1,) * (3 - ndim), dtype=np.int64)
    rc = _get().hxo_fork_reduce(ndim, _ptr(dims_a), reduce_dims, NEST_MONOIDS[monoid],
                                len(ops) // 2, _ptr(ops) if ops.size else ctypes.c_void_p(0),
                                _ptr(c), len(arrs), ptrs, _ptr(strides),
                                _ptr(out) if want_out and out.size else ctypes.c_void_p(0),
                                _ptr(result), _ptr(index))
    if rc:
        raise ValueError("oracle fork_reduce: malformed nest")
    if reduce_dims == 0:
        return out, None, None
    result = result[:n_outer].reshape(outer_shape)
    index = index[:n_outer].reshape(outer_shape) if monoid.startswith("arg") else None
    return out, result, index


def srad(J0: np.ndarray, iters: int, lam: float, roi, precision: str = "f64"):
    """SRAD-style iteration (see ``hxo_srad_f64``): returns (J after ``iters``
    iterations, q0sq per iteration).  ``roi`` = (r0, r1, c0, c1), half-open."""
    assert J0.ndim == 2
    ny, nx = J0.shape
    dt = np.float64 if precision == "f64" else np.float32
    src = np.ascontiguousarray(J0, dtype=dt)
    out = np.empty_like(src)
    q0 = np.zeros(max(iters, 1), dtype=dt)
    fn = _get().hxo_srad_f64 if precision == "f64" else _get().hxo_srad_f32
    r0, r1, c0, c1 = (int(v) for v in roi)
    if fn(_ptr(src), nx, ny, iters, lam, r0, r1, c0, c1, _ptr(out), _ptr(q0)):
        raise ValueError("oracle srad: bad arguments")
    return out, q0[:iters]

"""Host (multicore) schedule of three oracle nests -- TEST AND BENCHMARK
INFRASTRUCTURE ONLY.

``hx_oracle_mt.c`` runs map->reduce, the histogram and the Jacobi sweeps
with the fork split into T contiguous chunks, one POSIX thread each, and the
reduces reassociated per chunk (Sec. 2.2 fork-chunk, Sec. 4.5 concurrent
host tasks, Sec. 5.2 monoid-reassociate).  The benchmark times it on all
host cores as context next to the single-thread oracle; the tests check it
against the sequential oracle.  Parity of the GPU path is never judged
against this module.
"""

from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hx_oracle_mt.c")
_LIB = os.path.join(_HERE, "libhx_oracle_mt.so")

_lib = None


def build(force: bool = False) -> str:
    """Compile the threaded schedule with gcc (no fast-math, no FP contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread",
                               "-ffp-contract=off", "-fno-fast-math", "-Wall",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _get():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P, I32, I = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int
        lib.hxo_mt_map_reduce_f64.argtypes = [P, P, ctypes.c_double, ctypes.c_int64, P, P, I]
        lib.hxo_mt_histogram_u8.argtypes = [P, ctypes.c_int64, P, P, I]
        lib.hxo_mt_jacobi_f64.argtypes = [P, I32, I32, I32, P, P, I]
        for f in (lib.hxo_mt_map_reduce_f64, lib.hxo_mt_histogram_u8, lib.hxo_mt_jacobi_f64):
            f.restype = I
        _lib = lib
    return _lib


def host_cores() -> int:
    """Cores this process may run on (its CPU affinity set)."""
    return len(os.sched_getaffinity(0))


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None and a.size else ctypes.c_void_p(0)


def map_reduce(x: np.ndarray, y: np.ndarray, a: float, threads: int, want_out: bool = True):
    """out = a*x + y (fp64) and its sum folded per chunk, chunks in order."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    y = np.ascontiguousarray(y, dtype=np.float32)
    assert x.shape == y.shape and x.ndim == 1
    out = np.empty(x.size, dtype=np.float64) if want_out else None
    s = np.zeros(1, dtype=np.float64)
    rc = _get().hxo_mt_map_reduce_f64(_ptr(x), _ptr(y), float(a), x.size, _ptr(out), _ptr(s), int(threads))
    if rc:
        raise RuntimeError("multicore map_reduce failed")
    return out, float(s[0])


def histogram(v: np.ndarray, threads: int):
    """256 bins (per-chunk bins added) and their exclusive scan."""
    v = np.ascontiguousarray(v, dtype=np.uint8).ravel()
    bins = np.zeros(256, dtype=np.uint32)
    scan = np.zeros(256, dtype=np.uint32)
    rc = _get().hxo_mt_histogram_u8(_ptr(v), v.size, _ptr(bins), _ptr(scan), int(threads))
    if rc:
        raise RuntimeError("multicore histogram failed")
    return bins, scan


def jacobi(u0: np.ndarray, iters: int, threads: int):
    """fp64 clamp-to-edge Jacobi sweeps, each sweep's rows split over threads."""
    assert u0.ndim == 2
    ny, nx = u0.shape
    src = np.ascontiguousarray(u0, dtype=np.float64)
    out = np.empty_like(src)
    resid = np.zeros(max(iters, 0), dtype=np.float64)
    rc = _get().hxo_mt_jacobi_f64(_ptr(src), nx, ny, iters, _ptr(out), _ptr(resid), int(threads))
    if rc:
        raise RuntimeError("multicore jacobi failed")
    return out, resid

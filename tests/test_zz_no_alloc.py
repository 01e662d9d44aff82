"""hx_map_reduce_noalloc: the map->reduce entry point for callers that may not
allocate device memory (a plugin whose host application owns every device
allocation through its own pool, latency-critical code that cannot afford
cudaMalloc/cudaFree).  It keeps its scratch in a static device array of the
library instead of a context's workspace.

Called here through the C ABI directly (ctypes on libhx.so); torch only
allocates the test's own buffers.  Every call is checked against the oracle
(the tolerances of test_gpu_parity) and, bit for bit, against hx_map_reduce
run under the built-in default tuning table: both use the same tile plan and
the same canonical fold order of the tile partials.  Two calls in a row, of
different sizes, check that reusing the shared scratch is clean; the sizes
include n == 0, a plan of exactly HX_NOALLOC_MAX_TILES tiles, the largest
accepted n (2^31) and a sum that meets +inf.  This file is collected last,
and it passes on its own in a fresh process too.
"""

import ctypes

import numpy as np
import pytest
import torch

import oracle
import workloads

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
SUM_TOL = 1e-5


def _fn(hx):
    fn = hx.lib().hx_map_reduce_noalloc
    P = ctypes.c_void_p
    fn.argtypes = [P, P, P, ctypes.c_float, ctypes.c_int64, P, P, P]
    fn.restype = ctypes.c_int
    return fn


def _noalloc(hx, x, y, a, out, s32, s64, n=None):
    P = ctypes.c_void_p
    n = x.numel() if n is None else n
    st = _fn(hx)(P(x.data_ptr() if n else 0), P(y.data_ptr() if n else 0),
                 P(out.data_ptr() if out is not None else 0), ctypes.c_float(a), n,
                 P(s32.data_ptr()), P(s64.data_ptr()), P(torch.cuda.current_stream().cuda_stream))
    assert st == hx.HX_OK, hx.lib().hx_last_error()


@pytest.fixture(scope="module")
def default_ctx(gpu):
    ctx = gpu.hx_create(0)
    gpu.hx_tune_set(ctx, gpu.hx_tune_table_default())
    yield ctx
    ctx.close()


def _both(hx, ctx, xd, yd, a, want_out=True):
    """(out, s32, s64) from the no-allocation call and from hx_map_reduce."""
    n = xd.numel()
    res = []
    for noalloc in (True, False):
        out = torch.full((n,), float("nan"), device=DEV) if want_out else None
        s32 = torch.full((1,), float("nan"), device=DEV)
        s64 = torch.full((1,), float("nan"), dtype=torch.float64, device=DEV)
        if noalloc:
            _noalloc(hx, xd, yd, a, out, s32, s64)
        else:
            hx.hx_map_reduce(ctx, xd, yd, a, out=out, sum_out=s32, sum64_out=s64)
        torch.cuda.synchronize()
        res.append((out.cpu().numpy() if want_out else None, float(s32.item()), float(s64.item())))
    return res


def _bits_equal(u, v):
    if u is None:
        return
    assert np.array_equal(np.isnan(u), np.isnan(v))
    assert np.array_equal(u[~np.isnan(u)].view(np.uint32), v[~np.isnan(v)].view(np.uint32))


def _check_oracle(res, x, y, a):
    out, s32, s64 = res
    out_o, s_o = oracle.map_reduce(x, y, a)
    _bits_equal(out, out_o.astype(np.float32))
    if not np.isfinite(s_o):
        assert np.isnan(s_o) == np.isnan(s64) and (np.isnan(s_o) or s64 == s_o == s32)
        return
    cond = float(np.abs(out_o).sum())
    scale = abs(s_o) if abs(s_o) >= 1e-3 * cond else cond
    assert abs(s64 - s_o) <= SUM_TOL * scale
    assert np.float32(s64) == np.float32(s32)


@pytest.mark.parametrize("sizes", [((3_000_001, 5, 1.5), (4097, 6, -0.75)),
                                   ((1 << 21, 7, 1.5), ((1 << 21) + 1, 8, 1.5)),
                                   ((100_003, 9, 1.5), (0, 10, 1.5), (33, 11, -0.75))])
def test_noalloc_matches_map_reduce_and_oracle(gpu, default_ctx, sizes):
    # calls in a row of different sizes (2^21 is exactly HX_NOALLOC_MAX_TILES
    # tiles of the default plan; 2^21 + 1 doubles the tile length)
    hx = gpu
    for n, seed, a in sizes:
        x, y = workloads.map_reduce_inputs(n, seed=seed)
        xd, yd = torch.from_numpy(x).to(DEV), torch.from_numpy(y).to(DEV)
        new, ref = _both(hx, default_ctx, xd, yd, a)
        _bits_equal(new[0], ref[0])
        assert new[1] == ref[1] and new[2] == ref[2]
        _check_oracle(new, x, y, a)
        if n == 0:
            assert new[1] == 0.0 and new[2] == 0.0


def test_noalloc_non_finite_then_finite(gpu, default_ctx):
    hx = gpu
    n = 70_001
    x, y = workloads.map_reduce_inputs(n, seed=12)
    x[40_000] = np.float32("inf")
    for xs in (x, workloads.map_reduce_inputs(n, seed=13)[0]):
        xd, yd = torch.from_numpy(xs).to(DEV), torch.from_numpy(y).to(DEV)
        new, ref = _both(hx, default_ctx, xd, yd, 1.5)
        _bits_equal(new[0], ref[0])
        assert new[1] == ref[1] and new[2] == ref[2]
        _check_oracle(new, xs, y, 1.5)


def test_noalloc_largest_size_closed_form(gpu, default_ctx):
    # n = 2^31, the largest accepted: x = 1, y = 0.25 gives out = 1.75 and
    # s = 1.75 * 2^31, exact in the float-float sum (every partial sum is a
    # multiple of 0.25 below 2^33)
    hx = gpu
    n = 1 << 31
    xd = torch.ones(n, device=DEV)
    yd = torch.full((n,), 0.25, device=DEV)
    new, ref = _both(hx, default_ctx, xd, yd, 1.5, want_out=False)
    assert new[2] == ref[2] == 1.75 * n
    assert new[1] == ref[1] == np.float32(1.75 * n)
    del xd, yd
    torch.cuda.empty_cache()


def test_noalloc_rejects_oversize(gpu):
    hx = gpu
    lib = hx.lib()
    fn = _fn(hx)
    P = ctypes.c_void_p
    s = torch.empty(1, device=DEV)
    st = fn(P(16), P(32), P(0), ctypes.c_float(1.0), (1 << 31) + 1, P(s.data_ptr()), P(0), P(0))
    assert st == hx.HX_ERR_INVALID
    assert b"HX_MAP_REDUCE_NOALLOC_MAX_N" in lib.hx_last_error()

"""hx_map_reduce_noalloc: the map->reduce entry point for callers that may not
allocate device memory (a plugin whose host application owns every device
allocation through its own pool, latency-critical code that cannot afford
cudaMalloc/cudaFree).  It keeps its scratch in a static device array of the
library instead of a context's workspace.

Called here through the C ABI directly (ctypes on libhx.so); torch only
allocates the test's own buffers.  Two calls in a row, of different sizes,
must each agree with hx_map_reduce within the tolerance of the other
map->reduce tests: the scratch is shared and keeps the previous call's
contents, so the second call checks that the reuse is clean.  This file is
collected last, and it passes on its own in a fresh process too.
"""

import ctypes

import numpy as np
import pytest
import torch

import workloads

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
SUM_TOL = 1e-5


def _noalloc(hx, x, y, a, out, s32, s64):
    lib = hx.lib()
    fn = lib.hx_map_reduce_noalloc
    P = ctypes.c_void_p
    fn.argtypes = [P, P, P, ctypes.c_float, ctypes.c_int64, P, P, P]
    fn.restype = ctypes.c_int
    st = fn(P(x.data_ptr()), P(y.data_ptr()), P(out.data_ptr()), ctypes.c_float(a), x.numel(),
            P(s32.data_ptr()), P(s64.data_ptr()), P(torch.cuda.current_stream().cuda_stream))
    assert st == hx.HX_OK, lib.hx_last_error()


def test_noalloc_matches_map_reduce_twice(gpu):
    hx = gpu
    ctx = hx.hx_create(0)
    try:
        for n, seed, a in ((3_000_001, 5, 1.5), (4097, 6, -0.75)):
            x, y = workloads.map_reduce_inputs(n, seed=seed)
            xd, yd = torch.from_numpy(x).to(DEV), torch.from_numpy(y).to(DEV)
            out_ref = torch.empty(n, device=DEV)
            s64_ref = torch.empty(1, dtype=torch.float64, device=DEV)
            _, s32_ref, _ = hx.hx_map_reduce(ctx, xd, yd, a, out=out_ref, sum64_out=s64_ref)
            out = torch.empty(n, device=DEV)
            s32 = torch.empty(1, device=DEV)
            s64 = torch.empty(1, dtype=torch.float64, device=DEV)
            _noalloc(hx, xd, yd, a, out, s32, s64)
            torch.cuda.synchronize()
            o_ref, o_new = out_ref.cpu().numpy(), out.cpu().numpy()
            assert np.array_equal(o_new, o_ref)
            cond = float(np.abs(o_ref.astype(np.float64)).sum())
            assert abs(s64.item() - s64_ref.item()) <= SUM_TOL * cond
            assert abs(s32.item() - s32_ref.item()) <= SUM_TOL * cond
    finally:
        ctx.close()


def test_noalloc_rejects_oversize(gpu):
    hx = gpu
    lib = hx.lib()
    fn = lib.hx_map_reduce_noalloc
    P = ctypes.c_void_p
    fn.argtypes = [P, P, P, ctypes.c_float, ctypes.c_int64, P, P, P]
    fn.restype = ctypes.c_int
    s = torch.empty(1, device=DEV)
    st = fn(P(16), P(32), P(0), ctypes.c_float(1.0), (1 << 31) + 1, P(s.data_ptr()), P(0), P(0))
    assert st == hx.HX_ERR_INVALID
    assert b"HX_MAP_REDUCE_NOALLOC_MAX_N" in lib.hx_last_error()

"""Runs every entry point of the debug build (HX_DEBUG=1) on ragged,
misaligned and multi-round cases, checks a few results against the oracle,
then prints the device-side range-check record as one JSON line.  Started
as a child process by test_gpu_debug_checks.py."""

import ctypes
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

import oracle  # noqa: E402
import paper_2503_10855_b300 as hx  # noqa: E402
import workloads  # noqa: E402

assert hx.DEBUG and hx.LIB_PATH.endswith("libhx_debug.so"), hx.LIB_PATH
dev = "cuda:0"
ok = True
with hx.hx_create(0) as ctx:
    for n in (1, 33, 4097, (1 << 20) + 1, 3_000_001):
        x, y = workloads.map_reduce_inputs(n)
        for off in (0, 1):
            xd = torch.zeros(n + off, device=dev)[off:]
            yd = torch.zeros(n + off, device=dev)[off:]
            xd.copy_(torch.from_numpy(x))
            yd.copy_(torch.from_numpy(y))
            out, s32, s64 = hx.hx_map_reduce(ctx, xd, yd, 1.5, out=torch.empty(n, device=dev),
                                             sum64_out=torch.empty(1, dtype=torch.float64, device=dev))
            out_o, s_o = oracle.map_reduce(x, y, 1.5)
            ok &= abs(float(s64.item()) - s_o) <= 1e-5 * np.abs(out_o).sum()
        s_na = torch.empty(1, device=dev)
        fn = hx.lib().hx_map_reduce_noalloc
        P = ctypes.c_void_p
        fn.argtypes = [P, P, P, ctypes.c_float, ctypes.c_int64, P, P, P]
        fn.restype = ctypes.c_int
        st = fn(P(xd.data_ptr()), P(yd.data_ptr()), None, 1.5, n, P(s_na.data_ptr()), None,
                P(torch.cuda.current_stream().cuda_stream))
        ok &= st == hx.HX_OK and abs(float(s_na.item()) - float(s32.item())) <= 1e-5 * np.abs(out_o).sum()
    for shape in ((1, 1), (7, 5), (65, 129), (100, 132), (257, 300)):
        u0 = workloads.stencil_grid(*shape)
        a = torch.from_numpy(u0).to(dev)
        fin, res = hx.hx_stencil2d(ctx, a, torch.empty_like(a), 3)
        u32, _ = oracle.jacobi(u0, 3, "f32")
        ok &= np.array_equal(fin.cpu().numpy().view(np.uint32), u32.view(np.uint32))
    for n in (0, 15, 1000, 1 << 20, 3_000_017):
        v = torch.from_numpy(workloads.histogram_mixture_u8(max(n, 1))[:n]).to(dev)
        bins, scan = hx.hx_histogram(ctx, v)
        b_o, _ = oracle.histogram(v.cpu().numpy())
        ok &= np.array_equal(bins.cpu().numpy().view(np.uint32), b_o)
    # a mixed batch with multi-sweep stencils and histograms, planned both
    # ways: every sweep in one launch, and one launch per sweep (rounds)
    tasks, keep = [], []
    for k in range(24):
        if k % 3 == 0:
            n = 1000 + 37_000 * k
            xx = torch.rand(n, device=dev)
            yy = torch.rand(n, device=dev)
            s = torch.empty(1, device=dev)
            tasks.append(hx.map_reduce_task(xx, yy, 1.5, s, out=torch.empty(n, device=dev)))
        elif k % 3 == 1:
            g0 = torch.rand(40 + 9 * k, 31 + 13 * k, device=dev)
            r = torch.empty(1 + k % 4, device=dev)
            tasks.append(hx.stencil_task(g0, torch.empty_like(g0), 1 + k % 4, r))
        else:
            vv = torch.randint(0, 256, (70_001 * k,), dtype=torch.uint8, device=dev)
            tasks.append(hx.histogram_task(vv, torch.empty(256, dtype=torch.int32, device=dev),
                                           torch.empty(256, dtype=torch.int32, device=dev)))
    for rounds in (False, True):
        b = hx.hx_batch_plan(ctx, tasks, rounds=rounds)
        b.launch()
        b.launch()
        torch.cuda.synchronize()
        b.status()
        b.close()
    for shape, roi in (((100, 404), (40, 60, 150, 250)), ((33, 257), (0, 33, 0, 257)), ((512, 512), (0, 128, 0, 128))):
        J = workloads.srad_image(*shape)
        J0 = torch.from_numpy(J).to(dev)
        out, _ = hx.hx_srad(ctx, J0, torch.empty_like(J0), 3, 0.5, roi)
        ref64, _ = oracle.srad(J, 3, 0.5, roi, "f64")
        # three iterations, within the first-order rounding bound of the
        # fp32 scheme (tests/test_gpu_srad.py): per iteration
        # (1 + k (132 + 24 D)) u of the image's maximum, k = lambda / 4
        eps_it = (1.0 + 0.125 * (132.0 + 24.0 * float(J.max() / J.min()))) * 2.0 ** -24
        ok &= bool(np.max(np.abs(out.cpu().numpy() - ref64)) <= 3 * eps_it * np.max(np.abs(ref64)))
        hx.hx_srad(ctx, J0, torch.empty_like(J0), 2, 0.5, roi, fused=False)
    # generic nests: warp tree with one and several chunks per segment,
    # narrow segments, a permuted 3-D view, the chunk and sequential trees
    big = torch.rand(1 << 22, device=dev) * 2 - 1
    nest_cases = [
        ([("in", 0)], [big], (1 << 22,), 1, "sum", "warp"),
        ([("in", 0)], [big.view(1024, 4096)], (1024, 4096), 1, "max", "warp"),
        ([("in", 0)], [big[: (1 << 22) - 8].view(-1, 8)], (((1 << 22) - 8) // 8, 8), 1, "argmin", "warp"),
        ([("in", 0)], [big.view(64, 256, 256).permute(1, 0, 2)], (256, 64, 256), 2, "sum", "warp"),
        ([("in", 0), "abs"], [big[:100_003]], (100_003,), 1, "max", "chunk"),
        ([("in", 0)], [big[:4099]], (4099,), 1, "prod", "seq"),
    ]
    for prog, ins, dims, rd, mono, tree in nest_cases:
        _, res, _, r64 = hx.fork_reduce(ctx, prog, ins, dims, rd, mono, want_result64=(mono in ("sum", "prod")),
                                        tree=tree)
        if mono == "sum" and rd == 1 and len(dims) == 1:
            ok &= abs(float(r64.item()) - float(big.double().sum().item())) <= 1e-9 * float(big.abs().sum())
    torch.cuda.synchronize()
    enabled, code, a, b = hx.hx_debug_checks()
print(json.dumps({"enabled": enabled, "code": code, "a": a, "b": b, "results_ok": bool(ok)}))

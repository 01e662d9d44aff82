"""Failure handling without a GPU fault.

Launch failures are made on the host (hx_debug_inject_launch_failures: the
library fails a launching call with HX_ERR_CUDA before anything reaches the
driver).  They must surface as errors, launch nothing, and leave the
context, a batch and a server usable; a server must fail exactly the
requests that had work in the failed step and recycle their workspace.
No kernel is made to fault, trap or hang.
"""

import numpy as np
import pytest
import torch

import oracle
import workloads
from tests.test_gpu_batch import Inst, _same

pytestmark = pytest.mark.gpu


def test_each_entry_point_fails_once_then_runs(gpu):
    hx = gpu
    x, y = workloads.map_reduce_inputs(100_003)
    with hx.hx_create(0) as ctx:
        xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
        s = torch.full((1,), -7.0, device="cuda:0")
        hx.hx_debug_inject_launch_failures(ctx, 1)
        with pytest.raises(hx.HxError) as e:
            hx.hx_map_reduce(ctx, xd, yd, 1.5, sum_out=s)
        assert e.value.status == hx.HX_ERR_CUDA and "injected" in str(e.value)
        torch.cuda.synchronize()
        assert float(s) == -7.0                       # nothing ran
        hx.hx_map_reduce(ctx, xd, yd, 1.5, sum_out=s)  # the next call runs
        torch.cuda.synchronize()
        out_o, s_o = oracle.map_reduce(x, y, 1.5)
        assert abs(float(s) - s_o) <= 1e-5 * np.abs(out_o).sum()

        u0 = torch.from_numpy(workloads.stencil_grid(40, 64)).cuda()
        u1 = torch.empty_like(u0)
        v = torch.from_numpy(workloads.histogram_mixture_u8(10_000)).cuda()
        J = torch.from_numpy(workloads.srad_image(24, 40)).cuda()
        J1 = torch.empty_like(J)
        calls = [lambda: hx.hx_stencil2d(ctx, u0, u1, 3),
                 lambda: hx.hx_histogram(ctx, v),
                 lambda: hx.fork_reduce(ctx, [("in", 0)], [xd], tuple(xd.shape), 1, "sum"),
                 lambda: hx.hx_srad(ctx, J, J1, 2, 0.5, (0, 8, 0, 8))]
        for call in calls:
            hx.hx_debug_inject_launch_failures(ctx, 1)
            with pytest.raises(hx.HxError) as e:
                call()
            assert e.value.status == hx.HX_ERR_CUDA
            call()
        torch.cuda.synchronize()
        bins, scan = hx.hx_histogram(ctx, v)
        torch.cuda.synchronize()
        b_o, s_o = oracle.histogram(v.cpu().numpy())
        assert np.array_equal(bins.cpu().numpy().view(np.uint32), b_o)
        # cleared hook, delayed failure, bad arguments
        hx.hx_debug_inject_launch_failures(ctx, 5)
        hx.hx_debug_inject_launch_failures(ctx, 0)
        hx.hx_map_reduce(ctx, xd, yd, 1.5, sum_out=s)
        hx.hx_debug_inject_launch_failures(ctx, 1, after=2)
        hx.hx_map_reduce(ctx, xd, yd, 1.5, sum_out=s)
        hx.hx_map_reduce(ctx, xd, yd, 1.5, sum_out=s)
        with pytest.raises(hx.HxError):
            hx.hx_map_reduce(ctx, xd, yd, 1.5, sum_out=s)
        hx.hx_map_reduce(ctx, xd, yd, 1.5, sum_out=s)
        torch.cuda.synchronize()
        for bad in ((-1, 0), (1, -1)):
            with pytest.raises(hx.HxError):
                hx.hx_debug_inject_launch_failures(ctx, bad[0], after=bad[1])


@pytest.mark.parametrize("rounds", [True, False])
def test_batch_round_failure_then_relaunch(gpu, rounds):
    # rounds: round 0 runs, round 1 fails; one launch: the launch fails
    hx = gpu
    specs = [{"kind": "map_reduce", "n": 300_001, "a": 1.5, "seed": 11},
             {"kind": "stencil", "nx": 130, "ny": 77, "iters": 3, "seed": 12},
             {"kind": "histogram", "n": 700_001, "seed": 13},
             {"kind": "stencil", "nx": 64, "ny": 64, "iters": 2, "seed": 14}]
    insts = [Inst(s) for s in specs]
    with hx.hx_create(0) as ctx:
        b = hx.hx_batch_plan(ctx, [i.task(hx) for i in insts], rounds=rounds)
        hx.hx_debug_inject_launch_failures(ctx, 1, after=1 if rounds else 0)
        with pytest.raises(hx.HxError) as e:
            b.launch()
        assert e.value.status == hx.HX_ERR_CUDA
        torch.cuda.synchronize()
        b.launch()                                               # a clean relaunch from the inputs
        torch.cuda.synchronize()
        for inst in insts:
            r = inst.result()
            _same(r, inst.standalone(hx, ctx))
            inst.check_oracle(r)
        b.close()


def test_server_failed_step_fails_its_requests_and_recycles(gpu):
    hx = gpu
    def wave(seed0):
        specs = []
        for k in range(9):
            kind = ("map_reduce", "stencil", "histogram")[k % 3]
            if kind == "map_reduce":
                specs.append({"kind": kind, "n": 400_000 + 1000 * k, "a": 1.5, "seed": seed0 + k})
            elif kind == "stencil":
                specs.append({"kind": kind, "nx": 200 + k, "ny": 150, "iters": 3, "seed": seed0 + k})
            else:
                specs.append({"kind": kind, "n": 1_000_000 + 17 * k, "seed": seed0 + k})
        return [Inst(s) for s in specs]
    reports = {}

    def on_done(rid, status, latency):
        reports.setdefault(rid, []).append(status)

    with hx.hx_create(0) as ctx:
        # 64 KiB slices: every request spans several steps; the third step fails
        with hx.Server(ctx, mode=0, step_quantum_bytes=64 << 10, step_target_bytes=64 << 10,
                       max_steps_in_flight=2, on_done=on_done) as srv:
            first = wave(100)
            hx.hx_debug_inject_launch_failures(ctx, 1, after=2)
            ids = [srv.submit(i.task(hx)) for i in first]
            with pytest.raises(hx.HxError) as e:
                srv.drain(60.0)                  # reports the failures of this wave
            assert e.value.status == hx.HX_ERR_CUDA
            failed = 0
            for rid, inst in zip(ids, first):
                try:
                    done, lat = srv.poll(rid)
                except hx.HxError as e:
                    assert e.status == hx.HX_ERR_CUDA
                    failed += 1
                    continue
                assert done
                inst.check_oracle(inst.result())
            st = srv.stats()
            assert failed >= 1 and st["failed"] == failed
            # the completion callback saw each request once, with its outcome
            assert sorted(reports) == sorted(ids) and all(len(v) == 1 for v in reports.values())
            assert sum(v[0] == hx.HX_ERR_CUDA for v in reports.values()) == failed
            # a second wave reuses the recycled workspace slots
            second = wave(200)
            ids = [srv.submit(i.task(hx)) for i in second]
            srv.drain(60.0)
            for rid, inst in zip(ids, second):
                done, lat = srv.poll(rid)
                assert done
                inst.check_oracle(inst.result())
            assert srv.stats()["failed"] == failed

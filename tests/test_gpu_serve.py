"""Serving engine: every request's result is the same alone and in the mix
(bit-identical to its standalone call, and matching the oracle), in both the
continuous-batching and the per-launch modes; admission respects the budget."""

import ctypes

import numpy as np
import pytest
import torch

import workloads
from tests.test_gpu_batch import Inst, _same

pytestmark = pytest.mark.gpu


def _trace(count, rate, seed, hi=1 << 20, iters=5):
    tr = workloads.serving_trace(count, rate, seed=seed, hi=hi, stencil_iters=iters)
    for r in tr:
        r["seed"] &= 0xFFFFFFFF
    return tr


@pytest.mark.parametrize("mode", [0, 1])
def test_served_results_equal_alone(gpu, mode):
    hx = gpu
    trace = _trace(48, 30_000.0, seed=41)
    insts = [Inst(r) for r in trace]
    with hx.hx_create(0) as ctx:
        with hx.Server(ctx, mode=mode, direct_max=-1) as srv:   # batched steps only
            lat, makespan = srv.run_trace([i.task(hx) for i in insts], [r["arrival_s"] for r in trace])
            st = srv.stats()
        assert st["completed"] == len(trace) and st["failed"] == 0
        assert all(x >= 0.0 for x in lat) and makespan > 0
        if mode == 0:
            assert st["launches"] < len(trace)     # requests really were batched together
        for inst in insts:
            r = inst.result()
            _same(r, inst.standalone(hx, ctx))
            inst.check_oracle(r)


def test_sliced_requests_equal_alone(gpu):
    # a 64 KiB quantum spreads every request over many steps (slices of map
    # tiles, histogram chunks and stencil sweeps)
    hx = gpu
    trace = _trace(24, 50_000.0, seed=43, hi=1 << 20, iters=3)
    insts = [Inst(r) for r in trace]
    with hx.hx_create(0) as ctx:
        with hx.Server(ctx, mode=0, step_quantum_bytes=64 << 10, step_target_bytes=64 << 10,
                       max_steps_in_flight=3, direct_max=-1, max_step_sweeps=1) as srv:
            srv.run_trace([i.task(hx) for i in insts], [r["arrival_s"] for r in trace])
            st = srv.stats()
        assert st["launches"] > len(trace)
        for inst in insts:
            r = inst.result()
            _same(r, inst.standalone(hx, ctx))
            inst.check_oracle(r)


def test_lone_request_runs_as_its_standalone_call(gpu):
    # low load: a request with nothing else waiting is issued as its
    # standalone call (one issue, all 20 sweeps)
    hx = gpu
    spec = {"kind": "stencil", "nx": 700, "ny": 500, "iters": 20, "seed": 44}
    inst = Inst(spec)
    with hx.hx_create(0) as ctx:
        with hx.Server(ctx, mode=0) as srv:
            srv.run_trace([inst.task(hx)], [0.0])
            st = srv.stats()
        assert st["completed"] == 1 and st["failed"] == 0 and st["launches"] == 1
        r = inst.result()
        _same(r, inst.standalone(hx, ctx))
        inst.check_oracle(r)


@pytest.mark.parametrize("direct_max", [-1, 4, 64])
def test_direct_and_batched_paths_agree(gpu, direct_max):
    # the same trace with batched steps only, with the low-load direct path,
    # and with every fresh request direct: the same bits as standalone calls
    hx = gpu
    trace = _trace(30, 40_000.0, seed=46, iters=4)
    insts = [Inst(r) for r in trace]
    with hx.hx_create(0) as ctx:
        with hx.Server(ctx, mode=0, direct_max=direct_max) as srv:
            srv.run_trace([i.task(hx) for i in insts], [r["arrival_s"] for r in trace])
            st = srv.stats()
        assert st["completed"] == len(trace) and st["failed"] == 0
        for inst in insts:
            r = inst.result()
            _same(r, inst.standalone(hx, ctx))
            inst.check_oracle(r)


def test_timeline_records_steps(gpu):
    # one record per issued step, in issue order, each finished after it was
    # issued; the requests over all steps cover every request at least once;
    # with the direct path off every step is batched, with every fresh
    # request direct each request's first step is its standalone call
    hx = gpu
    trace = _trace(30, 40_000.0, seed=47, iters=4)
    for direct_max in (-1, 64):
        insts = [Inst(r) for r in trace]
        with hx.hx_create(0) as ctx:
            with hx.Server(ctx, mode=0, direct_max=direct_max) as srv:
                srv.run_trace([i.task(hx) for i in insts], [r["arrival_s"] for r in trace])
                st = srv.stats()
                tl = srv.timeline()
        assert len(tl) == st["launches"] > 0
        issue = [r["issue_s"] for r in tl]
        assert issue == sorted(issue) and issue[0] >= 0.0
        assert all(r["done_s"] >= r["issue_s"] and r["requests"] >= 1 for r in tl)
        assert sum(r["requests"] for r in tl) >= len(trace)
        direct = [r for r in tl if r["direct"]]
        if direct_max < 0:
            assert not direct
        else:
            assert direct and all(r["requests"] == 1 for r in direct)


@pytest.mark.parametrize("max_step_sweeps", [1, 3, 128])
def test_multi_sweep_steps(gpu, max_step_sweeps):
    # batched steps only; a stencil request takes up to max_step_sweeps of
    # its remaining sweeps per step (one launch runs them one after another):
    # the same bits as the standalone calls, and fewer steps than one sweep
    # per step
    hx = gpu
    trace = _trace(30, 40_000.0, seed=49, iters=7)
    insts = [Inst(r) for r in trace]
    with hx.hx_create(0) as ctx:
        with hx.Server(ctx, mode=0, direct_max=-1, direct_sweep_bytes=-1, max_step_sweeps=max_step_sweeps) as srv:
            srv.run_trace([i.task(hx) for i in insts], [r["arrival_s"] for r in trace])
            st = srv.stats()
        assert st["completed"] == len(trace) and st["failed"] == 0
        if max_step_sweeps == 128:
            assert st["launches"] < len(trace)
        for inst in insts:
            r = inst.result()
            _same(r, inst.standalone(hx, ctx))
            inst.check_oracle(r)


def test_multi_sweep_step_wait_times_out(gpu):
    # a step whose wait between two sweeps can never be satisfied ends by
    # itself after the limit (no fault, no hang); the stencil request in it
    # completes with HX_ERR_TIMEOUT, drain reports the failure, and the next
    # wave on the same server is correct
    hx = gpu
    lib = hx.lib()
    specs = [{"kind": "stencil", "nx": 300, "ny": 200, "iters": 3, "seed": 60},
             {"kind": "map_reduce", "n": 100_003, "a": 1.5, "seed": 61}]
    lat = ctypes.c_double()
    with hx.hx_create(0) as ctx:
        with hx.Server(ctx, mode=0, direct_max=-1, direct_sweep_bytes=-1) as srv:
            srv.debug_stall(2_000_000)
            first = [Inst(s) for s in specs]
            ids = [srv.submit(i.task(hx)) for i in first]
            with pytest.raises(hx.HxError):
                srv.drain(60.0)
            assert lib.hx_server_poll(srv.handle, ids[0], ctypes.byref(lat)) == hx.HX_ERR_TIMEOUT
            assert lib.hx_server_poll(srv.handle, ids[1], ctypes.byref(lat)) in (hx.HX_OK, hx.HX_ERR_TIMEOUT)
            again = [Inst(s) for s in specs]
            ids = [srv.submit(i.task(hx)) for i in again]
            srv.drain(60.0)
            assert all(srv.poll(rid)[0] for rid in ids)
        for inst in again:
            r = inst.result()
            _same(r, inst.standalone(hx, ctx))
            inst.check_oracle(r)
        with hx.Server(ctx, mode=1) as srv:
            with pytest.raises(hx.HxError):
                srv.debug_stall(1000)


@pytest.mark.parametrize("direct_sweep_bytes", [8 * 64 * 64, -1])
def test_large_stencils_run_standalone(gpu, direct_sweep_bytes):
    # batched steps otherwise (direct_max = -1): each stencil request whose
    # sweep moves at least direct_sweep_bytes runs once as its standalone
    # call, everything else in batched steps; the same bits either way
    hx = gpu
    trace = _trace(36, 40_000.0, seed=48, iters=4)
    insts = [Inst(r) for r in trace]
    big = sum(1 for r in trace if r["kind"] == "stencil" and direct_sweep_bytes > 0 and
              8 * r["nx"] * r["ny"] >= direct_sweep_bytes)
    assert direct_sweep_bytes < 0 or 0 < big < len(trace)
    with hx.hx_create(0) as ctx:
        with hx.Server(ctx, mode=0, direct_max=-1, direct_sweep_bytes=direct_sweep_bytes) as srv:
            srv.run_trace([i.task(hx) for i in insts], [r["arrival_s"] for r in trace])
            st = srv.stats()
            tl = srv.timeline()
        assert st["completed"] == len(trace) and st["failed"] == 0
        direct = [r for r in tl if r["direct"]]
        assert len(direct) == big and all(r["requests"] == 1 for r in direct)
        for inst in insts:
            r = inst.result()
            _same(r, inst.standalone(hx, ctx))
            inst.check_oracle(r)


def test_many_servers_on_one_context(gpu):
    # each server runs standalone calls on its own stream, which takes one of
    # the context's HX_MAX_STREAMS workspace slots; destroying the server
    # frees it, so any number of servers can follow one another
    hx = gpu
    spec = {"kind": "map_reduce", "n": 100_003, "a": 1.5, "seed": 45}
    with hx.hx_create(0) as ctx:
        for k in range(3 * 16):
            inst = Inst(spec)
            with hx.Server(ctx, mode=k % 2) as srv:
                srv.run_trace([inst.task(hx)], [0.0])
                assert srv.stats()["failed"] == 0
        inst.check_oracle(inst.result())


def test_admission_respects_budget(gpu):
    hx = gpu
    trace = _trace(40, 200_000.0, seed=42, hi=1 << 19, iters=3)
    insts = [Inst(r) for r in trace]
    budget = 6 << 20
    with hx.hx_create(0) as ctx:
        tasks = [i.task(hx) for i in insts]
        with hx.Server(ctx, mode=0, hbm_budget_bytes=budget) as srv:
            srv.run_trace(tasks, [r["arrival_s"] for r in trace])
            st = srv.stats()
        biggest = max(_footprint(t) for t in tasks)
        assert st["peak_footprint"] <= max(budget, biggest)
        assert st["completed"] == len(trace)
        for inst in insts:
            inst.check_oracle(inst.result())


def _footprint(t):
    if t.kind == 0:
        return t.u.mr.n * 4 * (3 if t.u.mr.out else 2) + 16
    if t.kind == 1:
        return t.u.st.nx * t.u.st.ny * 8 + t.u.st.iters * 4
    return t.u.hi.n + 2048


def test_submit_poll_drain(gpu):
    hx = gpu
    specs = [{"kind": "map_reduce", "n": 100_003, "a": 1.5, "seed": 1},
             {"kind": "stencil", "nx": 130, "ny": 77, "iters": 4, "seed": 2},
             {"kind": "histogram", "n": 65_537, "seed": 3},
             {"kind": "map_reduce", "n": 0, "a": 1.5, "seed": 4},
             {"kind": "stencil", "nx": 8, "ny": 8, "iters": 0, "seed": 5}]
    insts = [Inst(s) for s in specs]
    with hx.hx_create(0) as ctx:
        with hx.Server(ctx) as srv:
            ids = [srv.submit(i.task(hx)) for i in insts]
            srv.drain(60.0)
            for rid in ids:
                done, lat = srv.poll(rid)
                assert done and lat >= 0.0
            with pytest.raises(hx.HxError):
                srv.poll(10**9)
            x = torch.zeros(8, device="cuda:0")
            with pytest.raises(hx.HxError):
                srv.submit(hx.stencil_task(x.view(2, 4), x.view(2, 4), 1, torch.zeros(1, device="cuda:0")))
        for inst in insts[:3]:
            inst.check_oracle(inst.result())
        assert insts[3].s32.item() == 0.0
        assert torch.equal(insts[4].u0, insts[4].u_init)


@pytest.mark.parametrize("mode", ["continuous", "per_launch"])
def test_completion_callback(gpu, mode):
    # every request is reported exactly once, after it completed, with the
    # latency hx_server_poll reports; drain returns only after the reports
    import threading

    hx = gpu
    specs = [{"kind": ("map_reduce", "stencil", "histogram")[k % 3], "seed": 50 + k, "a": 1.5,
              "n": 20_000 + 91_003 * k, "nx": 40 + 17 * k, "ny": 33 + 5 * k, "iters": 1 + k % 3} for k in range(18)]
    insts = [Inst(s) for s in specs]
    seen, lock = [], threading.Lock()

    def on_done(rid, status, latency):
        with lock:
            seen.append((rid, status, latency))

    m = hx.HX_SERVE_CONTINUOUS if mode == "continuous" else hx.HX_SERVE_PER_LAUNCH
    with hx.hx_create(0) as ctx:
        with hx.Server(ctx, mode=m, on_done=on_done) as srv:
            ids = [srv.submit(i.task(hx)) for i in insts]
            srv.drain(60.0)
            with lock:
                got = {rid: (st, lat) for rid, st, lat in seen}
            assert len(seen) == len(ids) and set(got) == set(ids)
            for rid in ids:
                done, lat = srv.poll(rid)
                assert done and got[rid][0] == hx.HX_OK and got[rid][1] == lat
        for inst in insts:
            inst.check_oracle(inst.result())

"""Batched persistent launch: every instance bit-identical to its standalone
call, and matching the oracle (tolerances as in test_gpu_parity)."""

import ctypes

import numpy as np
import pytest
import torch

import oracle
import workloads

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module")
def ctx(gpu):
    c = gpu.hx_create(0)
    yield c
    c.close()


class Inst:
    """Device buffers of one instance, built from its seed."""

    def __init__(self, spec, offset=0):
        self.spec = spec
        k = spec["kind"]
        if k == "map_reduce":
            n = spec["n"]
            self.x = torch.empty(n + offset, device=DEV)[offset:]
            self.y = torch.empty(n + offset, device=DEV)[offset:]
            self.x.copy_(workloads.uniform_pm1_f32_torch(spec["seed"], n, DEV, 2, 0))
            self.y.copy_(workloads.uniform_pm1_f32_torch(spec["seed"], n, DEV, 2, 1))
            self.out = torch.full((n,), float("nan"), device=DEV)
            self.s32 = torch.full((1,), float("nan"), device=DEV)
            self.s64 = torch.full((1,), float("nan"), dtype=torch.float64, device=DEV)
        elif k == "stencil":
            ny, nx = spec["ny"], spec["nx"]
            base = torch.empty(ny * nx + offset, device=DEV)
            if spec.get("values") == "pm1":
                base[offset:] = workloads.uniform_pm1_f32_torch(spec["seed"], ny * nx, DEV)
            else:
                base[offset:] = workloads.uniform01_f32_torch(spec["seed"], ny * nx, DEV)
            self.u0 = base[offset:].view(ny, nx)
            self.u_init = self.u0.clone()
            self.u1 = torch.full((ny, nx), float("nan"), device=DEV)
            self.res = torch.full((max(1, spec["iters"]),), -1.0, device=DEV)
        else:
            n = spec["n"]
            vb = torch.empty(n + offset, dtype=torch.uint8, device=DEV)
            vb[offset:] = torch.from_numpy(workloads.histogram_mixture_u8(n, seed=spec["seed"] & 0xFFFF)).to(DEV)
            self.v = vb[offset:]
            self.bins = torch.full((256,), -1, dtype=torch.int32, device=DEV)
            self.scan = torch.full((256,), -1, dtype=torch.int32, device=DEV)

    def task(self, hx):
        k = self.spec["kind"]
        if k == "map_reduce":
            return hx.map_reduce_task(self.x, self.y, self.spec["a"], self.s32, out=self.out, sum64_out=self.s64)
        if k == "stencil":
            return hx.stencil_task(self.u0, self.u1, self.spec["iters"], self.res)
        return hx.histogram_task(self.v, self.bins, self.scan)

    def result(self):
        k = self.spec["kind"]
        if k == "map_reduce":
            return (self.out.cpu().numpy(), float(self.s32.item()), float(self.s64.item()))
        if k == "stencil":
            it = self.spec["iters"]
            fin = self.u1 if it % 2 == 1 else self.u0
            return (fin.cpu().numpy(), self.res.cpu().numpy()[:it])
        return (self.bins.cpu().numpy().view(np.uint32), self.scan.cpu().numpy().view(np.uint32))

    def standalone(self, hx, ctx):
        """The same instance through the standalone call, on fresh buffers."""
        k = self.spec["kind"]
        if k == "map_reduce":
            out = torch.empty_like(self.out)
            _, s32, s64 = hx.hx_map_reduce(ctx, self.x, self.y, self.spec["a"], out=out,
                                           sum64_out=torch.empty(1, dtype=torch.float64, device=DEV))
            torch.cuda.synchronize()
            return (out.cpu().numpy(), float(s32.item()), float(s64.item()))
        if k == "stencil":
            a, b = self.u_init.clone(), torch.empty_like(self.u_init)
            fin, res = hx.hx_stencil2d(ctx, a, b, self.spec["iters"])
            torch.cuda.synchronize()
            return (fin.cpu().numpy(), res.cpu().numpy()[:self.spec["iters"]])
        bins, scan = hx.hx_histogram(ctx, self.v)
        torch.cuda.synchronize()
        return (bins.cpu().numpy().view(np.uint32), scan.cpu().numpy().view(np.uint32))

    def check_oracle(self, res):
        k = self.spec["kind"]
        if k == "map_reduce":
            out, s32, s64 = res
            x, y = self.x.cpu().numpy(), self.y.cpu().numpy()
            out_o, s_o = oracle.map_reduce(x, y, self.spec["a"])
            assert np.array_equal(out, out_o.astype(np.float32))
            cond = np.abs(out_o).sum()
            scale = abs(s_o) if abs(s_o) >= 1e-3 * cond else cond   # as in test_gpu_parity
            assert abs(s64 - s_o) <= 1e-5 * scale
            assert np.float32(s64) == np.float32(s32)
        elif k == "stencil":
            fin, r = res
            u32, r32 = oracle.jacobi(self.u_init.cpu().numpy(), self.spec["iters"], "f32")
            assert np.array_equal(fin.view(np.uint32), u32.view(np.uint32))
            assert np.array_equal(r.view(np.uint32), r32.view(np.uint32))
        else:
            bins, scan = res
            b_o, s_o = oracle.histogram(self.v.cpu().numpy())
            assert np.array_equal(bins, b_o) and np.array_equal(scan, s_o)


def _same(a, b):
    for u, v in zip(a, b):
        if isinstance(u, np.ndarray):
            assert np.array_equal(u.view(np.uint8), v.view(np.uint8))
        else:
            assert u == v or (u != u and v != v)


def _run(gpu, insts, ctx):
    b = gpu.hx_batch_plan(ctx, [i.task(gpu) for i in insts])
    b.launch()
    torch.cuda.synchronize()
    return b


@pytest.mark.slow
def test_standard_batch_alone_equals_mix_and_oracle(gpu, ctx):
    insts = [Inst(s) for s in workloads.batch_mix()]
    b = _run(gpu, insts, ctx)
    assert b.rounds == 1
    for inst in insts:
        r = inst.result()
        _same(r, inst.standalone(gpu, ctx))
        inst.check_oracle(r)
    b.close()


@pytest.mark.slow
def test_standard_batch_20_sweeps_in_one_launch(gpu, ctx):
    # the 512-instance batch with 20 sweeps per stencil instance, all in one
    # persistent launch: every instance bit-identical to its standalone call;
    # every map->reduce instance and a sample of 24 stencil instances (every
    # size decile) against the oracle
    insts = [Inst(s) for s in workloads.batch_mix(iters=20)]
    b = gpu.hx_batch_plan(ctx, [i.task(gpu) for i in insts], rounds=False)
    assert b.rounds == 1
    b.launch()
    torch.cuda.synchronize()
    b.status()
    stencils = sorted((i for i in insts if i.spec["kind"] == "stencil"), key=lambda i: i.spec["nx"])
    sample = {id(stencils[k]) for k in np.linspace(0, len(stencils) - 1, 24).astype(int)}
    for inst in insts:
        r = inst.result()
        _same(r, inst.standalone(gpu, ctx))
        if inst.spec["kind"] != "stencil" or id(inst) in sample:
            inst.check_oracle(r)
    b.close()


def _mixed_specs():
    specs = [
        {"kind": "map_reduce", "n": 1, "a": 1.5, "seed": 1},
        {"kind": "map_reduce", "n": 4097, "a": -0.75, "seed": 2},
        {"kind": "map_reduce", "n": 3_000_001, "a": 1.5, "seed": 3},
        {"kind": "map_reduce", "n": (1 << 23) + 9, "a": 1.5, "seed": 4},
        {"kind": "stencil", "nx": 1, "ny": 1, "iters": 3, "seed": 5},
        {"kind": "stencil", "nx": 33, "ny": 70, "iters": 5, "seed": 6},
        {"kind": "stencil", "nx": 256, "ny": 129, "iters": 2, "seed": 7},
        {"kind": "stencil", "nx": 1000, "ny": 3, "iters": 1, "seed": 8},
        {"kind": "histogram", "n": 17, "seed": 9},
        {"kind": "histogram", "n": (1 << 20) + 5, "seed": 10},
        {"kind": "histogram", "n": 300_000, "seed": 11},
    ]
    return specs


@pytest.mark.parametrize("rounds", [False, True])
@pytest.mark.parametrize("offset", [0, 1])
def test_mixed_batch_multi_sweep(gpu, ctx, offset, rounds):
    # stencils of 1-5 sweeps: all sweeps in one persistent launch (default),
    # or one launch per sweep (rounds); both bit-identical to standalone calls
    insts = [Inst(s, offset) for s in _mixed_specs()]
    b = gpu.hx_batch_plan(ctx, [i.task(gpu) for i in insts], rounds=rounds)
    assert b.rounds == (5 if rounds else 1)
    b.launch()
    torch.cuda.synchronize()
    b.status()
    for inst in insts:
        r = inst.result()
        _same(r, inst.standalone(gpu, ctx))
        inst.check_oracle(r)
    b.close()


@pytest.mark.parametrize("offset", [0, 5])
def test_histogram_chunk_residues(gpu, ctx, offset):
    # a batch counts a histogram in chunks of 256 KiB, each by 256 threads
    # with eight 16-byte loads in flight per thread (2048 vectors per pass):
    # last chunks that end on, just before and just after a byte, a vector, a
    # thread's share and a whole pass, after one or two full chunks, from an
    # aligned and an unaligned start; exact against the standalone call and
    # the oracle
    chunk, pass_vecs = 256 * 1024, 2048
    tails = [0, 1, 15, 16, 17, 16 * 255 + 3, 16 * 256, 16 * (pass_vecs - 1) + 9, 16 * pass_vecs,
             16 * pass_vecs + 1, chunk - 1]
    specs = [{"kind": "histogram", "n": chunk * (1 + k % 2) + t, "seed": 90 + k} for k, t in enumerate(tails)]
    insts = [Inst(s, offset) for s in specs]
    b = _run(gpu, insts, ctx)
    for inst in insts:
        r = inst.result()
        _same(r, inst.standalone(gpu, ctx))
        inst.check_oracle(r)
    b.close()


@pytest.mark.parametrize("shape,iters", [((1000, 1000), 12), ((601, 997), 9), ((64, 4100), 6), ((3000, 40), 5)])
def test_one_launch_wavefront_shapes(gpu, ctx, shape, iters):
    # one grid whose sweeps run in one launch, each block waiting only for
    # itself and its north / south / west / east blocks in the previous
    # sweep: several block columns (west / east dependencies), the element
    # path (nx not a multiple of 4), a wide short grid and a tall narrow one;
    # bit-identical to rounds and to the standalone call, and the oracle
    ny, nx = shape
    spec = {"kind": "stencil", "nx": nx, "ny": ny, "iters": iters, "seed": 70 + nx % 13}
    got = []
    for rounds in (False, True):
        inst = Inst(spec)
        b = gpu.hx_batch_plan(ctx, [inst.task(gpu)], rounds=rounds)
        assert b.rounds == (iters if rounds else 1)
        b.launch()
        torch.cuda.synchronize()
        b.status()
        got.append(inst.result())
        b.close()
    _same(got[0], got[1])
    _same(got[0], inst.standalone(gpu, ctx))
    inst.check_oracle(got[0])


def _reset(insts):
    for inst in insts:
        if inst.spec["kind"] == "stencil":
            inst.u0.copy_(inst.u_init)


def test_multi_sweep_relaunch_and_graph_replay(gpu, ctx):
    # the block progress words and residual accumulators are clean after a
    # launch: a second launch and CUDA-graph replays of the same plan give the same
    # bits as the first launch (each from the same initial grids)
    specs = [{"kind": "stencil", "nx": 300, "ny": 200, "iters": 7, "seed": 31},
             {"kind": "stencil", "nx": 64, "ny": 64, "iters": 20, "seed": 32},
             {"kind": "map_reduce", "n": 500_001, "a": 1.5, "seed": 33},
             {"kind": "stencil", "nx": 1025, "ny": 130, "iters": 2, "seed": 34}]
    insts = [Inst(s) for s in specs]
    b = gpu.hx_batch_plan(ctx, [i.task(gpu) for i in insts], rounds=False)   # one launch
    assert b.rounds == 1
    b.launch()
    torch.cuda.synchronize()
    first = [i.result() for i in insts]
    for inst, f in zip(insts, first):
        _same(f, inst.standalone(gpu, ctx))
        inst.check_oracle(f)
    _reset(insts)
    b.launch()
    torch.cuda.synchronize()
    for i, f in zip(insts, first):
        _same(i.result(), f)
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        b.launch(stream=s)
    for _ in range(2):
        _reset(insts)
        g.replay()
        torch.cuda.synchronize()
        for i, f in zip(insts, first):
            _same(i.result(), f)
    b.status()
    b.close()


def test_multi_sweep_wait_times_out_and_reports(gpu, ctx):
    # a wait that can never be satisfied (test hook: the instance's later
    # sweeps expect one block more than a sweep has) gives up after 2 ms; the
    # launch ends by itself, the plan reports HX_ERR_TIMEOUT once, and the
    # context stays usable
    specs = [{"kind": "stencil", "nx": 256, "ny": 96, "iters": 4, "seed": 35},
             {"kind": "map_reduce", "n": 100_000, "a": 1.5, "seed": 36}]
    insts = [Inst(s) for s in specs]
    b = gpu.hx_batch_plan(ctx, [i.task(gpu) for i in insts], rounds=False)
    b.debug_stall(0, 2_000_000)
    b.launch()
    torch.cuda.synchronize()
    with pytest.raises(gpu.HxError) as e:
        b.status()
    assert e.value.status == gpu.HX_ERR_TIMEOUT
    b.status()                      # read once, then clear
    b.close()
    # the unaffected map->reduce instance is still right, and a fresh plan works
    insts[1].check_oracle(insts[1].result())
    fresh = [Inst(s) for s in specs]
    b2 = gpu.hx_batch_plan(ctx, [i.task(gpu) for i in fresh], rounds=False)
    b2.launch()
    torch.cuda.synchronize()
    b2.status()
    for inst in fresh:
        r = inst.result()
        _same(r, inst.standalone(gpu, ctx))
        inst.check_oracle(r)
    b2.close()


def test_default_schedule(gpu, ctx):
    # one launch when the multi-sweep stencils move at most 512 MiB per
    # sweep (8 bytes per point), else rounds; either way the same bits
    small = [Inst({"kind": "stencil", "nx": 70, "ny": 50, "iters": 3, "seed": 40 + k}) for k in range(3)]
    b = gpu.hx_batch_plan(ctx, [i.task(gpu) for i in small])
    assert b.rounds == 1
    b.launch()
    torch.cuda.synchronize()
    b.status()
    for inst in small:
        r = inst.result()
        _same(r, inst.standalone(gpu, ctx))
        inst.check_oracle(r)
    b.close()
    # 8192 x 8193 points: 537 MB per sweep (planned only)
    big = Inst({"kind": "stencil", "nx": 8192, "ny": 8193, "iters": 2, "seed": 47})
    b = gpu.hx_batch_plan(ctx, [big.task(gpu)] + [i.task(gpu) for i in small])
    assert b.rounds == 3
    b.close()
    del big
    torch.cuda.empty_cache()
    # both schedule flags at once, or an unknown flag, are rejected
    h = ctypes.c_void_p()
    for flags in (gpu.HX_BATCH_ROUNDS | gpu.HX_BATCH_ONE_LAUNCH, 4):
        st = gpu.lib().hx_batch_plan_ex(ctx.handle, (gpu.HxTask * 1)(), 0, flags, ctypes.byref(h), None)
        assert st == gpu.HX_ERR_INVALID


def test_submit_reports_wait_timeout(gpu, ctx):
    # hx_batch_query returns the plan's wait status with its completion
    insts = [Inst({"kind": "stencil", "nx": 128, "ny": 64, "iters": 3, "seed": 37})]
    t = gpu.hx_batch_submit(ctx, [i.task(gpu) for i in insts])
    torch.cuda.synchronize()
    assert gpu.hx_batch_query(ctx, t) is True
    insts[0].check_oracle(insts[0].result())


def test_batch_empty_instances(gpu, ctx):
    specs = [{"kind": "map_reduce", "n": 0, "a": 1.5, "seed": 1},
             {"kind": "histogram", "n": 0, "seed": 2},
             {"kind": "stencil", "nx": 4, "ny": 4, "iters": 0, "seed": 3}]
    insts = [Inst(s) for s in specs]
    b = _run(gpu, insts, ctx)
    assert insts[0].s32.item() == 0.0 and insts[0].s64.item() == 0.0
    assert not insts[1].bins.any() and not insts[1].scan.any()
    assert torch.equal(insts[2].u0, insts[2].u_init)
    b.close()
    assert gpu.hx_batch_plan(ctx, []).rounds == 0


def test_batch_relaunch_and_graph_replay(gpu, ctx):
    specs = [{"kind": "map_reduce", "n": 200_003, "a": 1.5, "seed": 21},
             {"kind": "stencil", "nx": 300, "ny": 200, "iters": 1, "seed": 22},
             {"kind": "histogram", "n": 500_001, "seed": 23}]
    insts = [Inst(s) for s in specs]
    b = _run(gpu, insts, ctx)
    first = [i.result() for i in insts]
    b.launch()
    torch.cuda.synchronize()
    for i, f in zip(insts, first):
        _same(i.result(), f)
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        b.launch(stream=s)
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    for i, f in zip(insts, first):
        _same(i.result(), f)
        i.check_oracle(i.result())
    b.close()


def test_batch_submit_and_query(gpu, ctx):
    insts = [Inst(s) for s in _mixed_specs()[:3]]
    t = gpu.hx_batch_submit(ctx, [i.task(gpu) for i in insts])
    torch.cuda.synchronize()
    assert gpu.hx_batch_query(ctx, t) is True
    with pytest.raises(gpu.HxError):
        gpu.hx_batch_query(ctx, t)           # retired
    for inst in insts:
        inst.check_oracle(inst.result())


def test_batch_rejects_bad_task(gpu, ctx):
    x = torch.zeros(8, device=DEV)
    bad = gpu.stencil_task(x.view(2, 4), x.view(2, 4), 1, torch.zeros(1, device=DEV))
    with pytest.raises(gpu.HxError):
        gpu.hx_batch_plan(ctx, [bad])


def test_describe_plan(gpu, ctx):
    # the plan as text: header, the work order of a one-launch plan, one line
    # per instance; a buffer shorter than the text is truncated and terminated
    insts = [Inst({"kind": "stencil", "nx": 70, "ny": 50, "iters": 3, "seed": 50 + k}) for k in range(4)]
    insts.append(Inst({"kind": "map_reduce", "n": 100_003, "a": 1.5, "seed": 55}))
    insts.append(Inst({"kind": "histogram", "n": 70_001, "seed": 56}))
    b = gpu.hx_batch_plan(ctx, [i.task(gpu) for i in insts])
    text = b.describe()
    lines = text.splitlines()
    assert lines[0].startswith("hx batch plan: 6 instances, every sweep in one launch, 1 launch ")
    assert "(instance, sweep) pairs" in lines[1] and lines[1].strip().startswith("work order: 14 ")
    body = lines[2:]
    assert len(body) == 6
    for k in range(4):
        assert body[k].startswith(f"  [{k}] stencil 50 x 70, 3 sweeps in one launch")
    assert body[4].startswith("  [4] map->reduce n=100003 ")
    assert body[5].startswith("  [5] histogram n=70001 bytes")
    need = ctypes.c_size_t(0)
    assert gpu.lib().hx_batch_describe(b.handle, None, 0, ctypes.byref(need)) == gpu.HX_OK
    assert need.value == len(text) + 1
    short = ctypes.create_string_buffer(16)
    assert gpu.lib().hx_batch_describe(b.handle, short, 16, None) == gpu.HX_OK
    assert short.value.decode() == text[:15]
    b.close()
    r = gpu.hx_batch_plan(ctx, [i.task(gpu) for i in insts], rounds=True)
    rtext = r.describe()
    assert rtext.startswith("hx batch plan: 6 instances, one launch per sweep (rounds), 3 launches ")
    assert "work order" not in rtext and "3 sweeps as rounds" in rtext
    r.close()

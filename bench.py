#!/usr/bin/env python3
"""Benchmark of the fork-join hot path on B300.

One step = one pass of every nest of the hot path over one batch of seeded
synthetic input:
  * map->reduce: out = fmaf(1.5, x, y), s = sum(out), N = 2^20
  * Jacobi: 20 clamp-to-edge 5-point sweeps of a 2048 x 2048 fp32 grid with a
    max residual per sweep
  * histogram: 256 bins of 2^26 mixture bytes + exclusive scan
  * batch: 512 independent map->reduce / stencil instances (log-uniform
    sizes 1K-4M elements, square sides 32-2048, one sweep each) in one
    persistent launch
Inputs rotate over several buffer sets whose total exceeds the 126 MB L2, so
each step starts from HBM.  value = algorithmic bytes of the step / device
time (GB/s), summed over ranks (weak scaling: every rank runs its own
replica; there is no data-path collective).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl hx|reference]

--impl reference times the CPU oracle (the sequential reference evaluation
of the same nests) on a bounded sample of the same workload.
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads  # noqa: E402

MR_N = 1 << 20
ST_SIDE = 2048
ST_ITERS = 20
HI_N = 1 << 26
L2_BYTES = 126 * 1024 * 1024

# algorithmic bytes per unit (read + write that the nest must do at minimum)
MR_BYTES = 12 * MR_N                                  # x, y read; out written
ST_BYTES_PER_SWEEP = 8 * ST_SIDE * ST_SIDE            # one read, one write per point
ST_BYTES = ST_BYTES_PER_SWEEP * ST_ITERS
HI_BYTES = HI_N + 2 * 256 * 4                         # bytes read; bins and scan written
STEP_BYTES = MR_BYTES + ST_BYTES + HI_BYTES


def batch_instances(dev):
    """Device buffers and hx tasks of the 512-instance batched workload."""
    import torch

    import paper_2503_10855_b300 as hx

    bufs, tasks, byts = [], [], 0
    for spec in workloads.batch_mix():
        if spec["kind"] == "map_reduce":
            n = spec["n"]
            x = workloads.uniform_pm1_f32_torch(spec["seed"], n, dev, 2, 0)
            y = workloads.uniform_pm1_f32_torch(spec["seed"], n, dev, 2, 1)
            out = torch.empty(n, device=dev)
            s32 = torch.empty(1, device=dev)
            tasks.append(hx.map_reduce_task(x, y, spec["a"], s32, out=out))
            bufs.append((x, y, out, s32))
            byts += 12 * n
        else:
            ny, nx = spec["ny"], spec["nx"]
            u0 = workloads.uniform_pm1_f32_torch(spec["seed"], ny * nx, dev).view(ny, nx)
            u1 = torch.empty_like(u0)
            res = torch.empty(1, device=dev)
            tasks.append(hx.stencil_task(u0, u1, 1, res))
            bufs.append((u0, u1, res))
            byts += 8 * nx * ny
    return bufs, tasks, byts


TUNE_FILE = os.path.join(ROOT, "paper_2503_10855_b300", "tune", "b300.json")


def apply_tuning(hx, ctx, args) -> str:
    """Tuning table for the run: measured now (--autotune), else the table the
    autotuner wrote on a B300 (shipped with the package), else the defaults."""
    if args.autotune:
        hx.hx_autotune(ctx, 28)
        return "autotuned at start (hx_autotune, classes up to 2^28)"
    if os.path.exists(TUNE_FILE):
        hx.hx_tune_set(ctx, hx.hx_tune_table_load(TUNE_FILE))
        return "paper_2503_10855_b300/tune/b300.json (written by hx_autotune on a B300)"
    return "built-in defaults"


def kernel_sources_sha256() -> str:
    import glob
    import hashlib

    pkg = os.path.join(ROOT, "paper_2503_10855_b300", "csrc")
    files = sorted(glob.glob(os.path.join(pkg, "*.cu")) + glob.glob(os.path.join(pkg, "*.cuh")))
    files.append(os.path.join(ROOT, "include", "hx.h"))
    h = hashlib.sha256()
    for f in files:
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def measured_traffic():
    """DRAM bytes per launch from the committed ncu capture, if it was taken
    on the current kernel sources (else {}: the counters are stale)."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.txt")) as f:
            doc = json.load(f)
    except (OSError, ValueError):
        return {}
    return doc.get("kernels", {}) if doc.get("sources_sha256") == kernel_sources_sha256() else {}


def max_over_ranks(value: float, dist, device) -> float:
    """The largest of every rank's value (the slowest rank's time); no
    collective when running alone."""
    if dist is None:
        return value
    import torch

    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(bytes_per_step_per_rank: int, world: int, slowest_ms_per_step: float) -> float:
    """Whole-job GB/s: every rank moves its own step's bytes (weak scaling),
    the job takes as long as its slowest rank."""
    return world * bytes_per_step_per_rank / (slowest_ms_per_step * 1e-3) / 1e9


def _dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """Samples SM clock and throttle reasons while the timed region runs.

    Uses NVML when the pynvml module is importable, else an ``nvidia-smi
    --query-gpu ... -lms`` process; both only read the GPU's state."""

    REASONS = {"sw_power_cap": 0x4, "hw_slowdown": 0x8, "sw_thermal_slowdown": 0x20,
               "hw_thermal_slowdown": 0x40, "hw_power_brake_slowdown": 0x80}

    def __init__(self, index: int, period_s: float = 0.02):
        self.index, self.period = index, period_s
        self.samples = []
        self.reasons = set()
        self.max_mhz = None
        self._stop = threading.Event()
        self._thr = None
        self._proc = None
        self.mode = None

    def __enter__(self):
        try:
            import pynvml

            pynvml.nvmlInit()
            self._nv = pynvml
            self._h = pynvml.nvmlDeviceGetHandleByIndex(self.index)
            self.max_mhz = pynvml.nvmlDeviceGetMaxClockInfo(self._h, pynvml.NVML_CLOCK_SM)
            self.mode = "nvml"
            self._thr = threading.Thread(target=self._run_nvml, daemon=True)
            self._thr.start()
        except Exception:
            import subprocess

            try:
                self._proc = subprocess.Popen(
                    ["nvidia-smi", f"--id={self.index}",
                     "--query-gpu=clocks.sm,clocks.max.sm,utilization.gpu,clocks_event_reasons.active",
                     "--format=csv,noheader,nounits", f"-lms={int(self.period * 1000)}"],
                    stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
                self.mode = "nvidia-smi"
                time.sleep(0.3)   # let the first sample land before the timed work
            except Exception as e:
                self.err = str(e)
        return self

    def _note(self, mhz, util, bits):
        self.samples.append((mhz, util))
        for k, bit in self.REASONS.items():
            if bits & bit:
                self.reasons.add(k)

    def _run_nvml(self):
        nv = self._nv
        while not self._stop.is_set():
            try:
                self._note(nv.nvmlDeviceGetClockInfo(self._h, nv.NVML_CLOCK_SM),
                           nv.nvmlDeviceGetUtilizationRates(self._h).gpu,
                           nv.nvmlDeviceGetCurrentClocksEventReasons(self._h))
            except Exception:
                pass
            time.sleep(self.period)

    def __exit__(self, *exc):
        self._stop.set()
        if self._thr:
            self._thr.join()
        if self._proc:
            self._proc.terminate()
            out, _ = self._proc.communicate(timeout=10)
            for line in out.splitlines():
                parts = [p.strip() for p in line.split(",")]
                try:
                    self.max_mhz = float(parts[1])
                    self._note(float(parts[0]), float(parts[2]), int(parts[3], 16))
                except (ValueError, IndexError):
                    pass

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": self.max_mhz, "reasons": [],
                    "note": getattr(self, "err", "no samples"), "source": self.mode}
        loaded = [m for m, u in self.samples if u > 0] or [m for m, _ in self.samples]
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": self.max_mhz,
                "reasons": sorted(self.reasons), "samples": len(self.samples), "source": self.mode}


# ---------------------------------------------------------------- CPU oracle
_ORACLE_INPUTS = {}


def _oracle_inputs():
    if not _ORACLE_INPUTS:
        x, y = workloads.map_reduce_inputs(MR_N)
        _ORACLE_INPUTS.update(x=x, y=y, v=workloads.histogram_mixture_u8(HI_N),
                              u0=workloads.stencil_grid(ST_SIDE, ST_SIDE).astype(np.float64))
    return _ORACLE_INPUTS


def run_oracle_sample(budget_s: float = 15.0):
    """Time the CPU oracle on a bounded sample of the step workload.

    The sample: the full map->reduce instance, a prefix of the histogram
    input and some sweeps of the 2048 x 2048 Jacobi grid, sized to about
    ``budget_s`` of single-core work.  Returns (GB/s of algorithmic bytes,
    seconds, description)."""
    import oracle

    d = _oracle_inputs()
    oracle.map_reduce(d["x"][:16], d["y"][:16], 1.5)  # load the library outside the timing
    t0 = time.perf_counter()
    oracle.map_reduce(d["x"], d["y"], 1.5)
    t_mr = time.perf_counter() - t0
    hn = int(min(HI_N, max(1 << 20, (budget_s / 4) * 1e9)))  # ~1 ns per byte
    t0 = time.perf_counter()
    oracle.histogram(d["v"][:hn])
    t_hi = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.jacobi(d["u0"], 1)
    t_sweep = time.perf_counter() - t0
    sweeps = int(max(1, min(ST_ITERS, (budget_s - t_mr - t_hi) // max(t_sweep, 1e-9))))
    t0 = time.perf_counter()
    if sweeps > 1:
        oracle.jacobi(d["u0"], sweeps)
    t_st = (time.perf_counter() - t0) if sweeps > 1 else t_sweep
    total_bytes = MR_BYTES + hn + 2048 + ST_BYTES_PER_SWEEP * sweeps
    total_s = t_mr + t_hi + t_st
    desc = (f"map_reduce N=2^20 + histogram first {hn} of 2^26 bytes + jacobi 2048^2 x {sweeps} "
            f"of 20 sweeps; sequential C oracle (fp64 / integer), 1 thread, {total_s:.3f} s")
    return total_bytes / total_s / 1e9, total_s, desc


def run_multicore_sample(budget_s: float = 3.0):
    """Time the host (multicore) schedule of the same nests on every core of
    this process's affinity set: the full map->reduce instance, the full
    histogram input and as many Jacobi sweeps (of 20) as fit the budget.
    Context for the single-thread oracle, not a target.  Returns (GB/s,
    seconds, threads, description)."""
    from oracle import multicore

    d = _oracle_inputs()
    T = multicore.host_cores()
    multicore.map_reduce(d["x"][:16], d["y"][:16], 1.5, 1)   # load the library outside the timing
    t0 = time.perf_counter()
    multicore.map_reduce(d["x"], d["y"], 1.5, T)
    t_mr = time.perf_counter() - t0
    t0 = time.perf_counter()
    multicore.histogram(d["v"], T)
    t_hi = time.perf_counter() - t0
    t0 = time.perf_counter()
    multicore.jacobi(d["u0"], 1, T)
    t_sweep = time.perf_counter() - t0
    sweeps = int(max(1, min(ST_ITERS, (budget_s - t_mr - t_hi) // max(t_sweep, 1e-9))))
    t0 = time.perf_counter()
    if sweeps > 1:
        multicore.jacobi(d["u0"], sweeps, T)
    t_st = (time.perf_counter() - t0) if sweeps > 1 else t_sweep
    total_s = t_mr + t_hi + t_st
    total_bytes = MR_BYTES + HI_BYTES + ST_BYTES_PER_SWEEP * sweeps
    desc = (f"map_reduce N=2^20 + histogram 2^26 bytes + jacobi 2048^2 x {sweeps} of 20 sweeps; "
            f"fork split into {T} contiguous chunks, one POSIX thread each (fp64 / integer), {total_s:.3f} s")
    return total_bytes / total_s / 1e9, total_s, T, desc


def bench_reference(args, rank, world):
    if rank != 0:
        return 0
    _oracle_inputs()
    per_step = min(15.0, 120.0 / (args.warmup + args.steps))
    secs, desc, vals = 0.0, "", []
    for i in range(args.warmup + args.steps):
        g, s, d = run_oracle_sample(budget_s=per_step)
        if i >= args.warmup:
            vals.append(g)
            secs += s
            desc = d
    gbs = statistics.median(vals)
    line = {
        "impl": "reference", "metric": "achieved HBM GB/s (algorithmic bytes / time) of the fork-join hot path",
        "value": round(gbs, 4), "unit": "GB/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(1e3 * secs / max(1, args.steps), 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64/u32",
        "data": "synthetic (seeded SplitMix64)",
        "config": {"workload": "fork-join step (map->reduce 2^20, jacobi 2048^2 x20, histogram 2^26), "
                               "bounded sample per step", "sample": desc},
        "cpu_baseline": {"value": round(gbs, 4), "unit": "GB/s", "cores": 1, "kind": "oracle", "sample": desc},
        "e2e": {"value": round(gbs, 4), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- GPU arm
def bench_hx(args, rank, world, local):
    import torch

    import paper_2503_10855_b300 as hx

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)

    ctx = hx.hx_create(local)
    stream = torch.cuda.Stream(device=dev)
    tune_src = apply_tuning(hx, ctx, args)

    # ---- inputs, rotated over buffer sets larger than L2 in total
    x_h, y_h = workloads.map_reduce_inputs(MR_N)
    u_h = workloads.stencil_grid(ST_SIDE, ST_SIDE)
    v_h = workloads.histogram_mixture_u8(HI_N)
    per_set = MR_BYTES + 2 * 4 * ST_SIDE * ST_SIDE + HI_N
    n_sets = max(2, math.ceil(3 * L2_BYTES / per_set))
    sets = []
    with torch.cuda.stream(stream):
        x_d0 = torch.from_numpy(x_h).to(dev)
        y_d0 = torch.from_numpy(y_h).to(dev)
        u_d0 = torch.from_numpy(u_h).to(dev)
        v_d0 = torch.from_numpy(v_h).to(dev)
        for r in range(n_sets):
            s = {
                "x": x_d0.clone(), "y": y_d0.clone(), "out": torch.empty(MR_N, device=dev),
                "s32": torch.empty(1, device=dev), "s64": torch.empty(1, dtype=torch.float64, device=dev),
                "u0": u_d0.clone(), "u1": torch.empty_like(u_d0),
                "res": torch.empty(ST_ITERS, device=dev),
                "v": v_d0.clone(), "bins": torch.empty(256, dtype=torch.int32, device=dev),
                "scan": torch.empty(256, dtype=torch.int32, device=dev),
            }
            sets.append(s)
    stream.synchronize()
    batch_bufs, batch_tasks, BATCH_BYTES = batch_instances(dev)
    batch = hx.hx_batch_plan(ctx, batch_tasks)
    step_bytes = STEP_BYTES + BATCH_BYTES
    torch.cuda.synchronize()

    # one CUDA graph per component and buffer set; events between graph
    # launches time each component on the launching stream
    comps = ("map_reduce", "jacobi", "histogram", "batch")

    def issue(name, s, st=None):
        st = stream if st is None else st
        if name == "map_reduce":
            hx.hx_map_reduce(ctx, s["x"], s["y"], 1.5, out=s["out"], sum_out=s["s32"],
                             sum64_out=s["s64"], stream=st)
        elif name == "jacobi":
            # the grid keeps evolving from step to step (a sweep's cost does
            # not depend on the values)
            hx.hx_stencil2d(ctx, s["u0"], s["u1"], ST_ITERS, resid=s["res"], stream=st)
        elif name == "histogram":
            hx.hx_histogram(ctx, s["v"], bins=s["bins"], scan=s["scan"], stream=st)
        else:
            batch.launch(stream=st)   # one buffer set: its 2.6 GB exceed L2 by themselves

    # The four nests of a step are independent calls, so a step runs them as
    # concurrent branches (the host backend's concurrent tasks for independent
    # calls, Sec. 4.5): the batch on the main stream, the Jacobi sweeps on a
    # second, map->reduce then histogram on a third, joined at the end.  Each
    # stream has its own workspace slot in the context.
    side_st = torch.cuda.Stream(device=dev)
    side_mh = torch.cuda.Stream(device=dev)

    def issue_step(s):
        fork = torch.cuda.Event()
        fork.record(stream)
        side_st.wait_event(fork)
        side_mh.wait_event(fork)
        issue("jacobi", s, side_st)
        issue("map_reduce", s, side_mh)
        issue("histogram", s, side_mh)
        issue("batch", s, stream)
        for st in (side_st, side_mh):
            join = torch.cuda.Event()
            join.record(st)
            stream.wait_event(join)

    with torch.cuda.stream(stream):
        for s in sets:           # eager warm-up of every code path before capture
            issue_step(s)
            for c in comps:
                issue(c, s)
    torch.cuda.synchronize()
    # the timed step: one CUDA graph per buffer set holding the whole step
    # (the concurrent branches above); the per-component breakdown comes from
    # a second pass that runs the components one after another, one graph per
    # component with events between them
    step_graphs, comp_graphs = [], []
    for s in sets:
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            issue_step(s)
        step_graphs.append(g)
        gs = {}
        for c in comps:
            gc = torch.cuda.CUDAGraph()
            with torch.cuda.graph(gc, stream=stream):
                issue(c, s)
            gs[c] = gc
        comp_graphs.append(gs)
    # launches per step: map->reduce and its partials' fold; 20 sweeps and
    # their residual fold; the histogram; per batch round, the batched
    # kernel and its final-combine kernel
    launches_per_step = 2 + ST_ITERS + 1 + 1 + 2 * batch.rounds

    with torch.cuda.stream(stream):
        for i in range(args.warmup):
            step_graphs[i % n_sets].replay()
    stream.synchronize()

    K = args.steps
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk, torch.cuda.stream(stream):
        wall0 = time.perf_counter()
        t_start.record(stream)
        for i in range(K):
            step_graphs[i % n_sets].replay()
        t_end.record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
    if dist:
        dist.barrier()
    total_ms = t_start.elapsed_time(t_end)
    total_ms = max_over_ranks(total_ms, dist, dev)

    # per-component times (not part of the timed region)
    K2 = min(K, 200)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(len(comps) + 1)] for _ in range(K2)]
    with torch.cuda.stream(stream):
        for i in range(K2):
            gs = comp_graphs[i % n_sets]
            for j, c in enumerate(comps):
                evs[i][j].record(stream)
                gs[c].replay()
            evs[i][len(comps)].record(stream)
    torch.cuda.synchronize()
    comp_ms = {c: 0.0 for c in comps}
    for e in evs:
        for j, c in enumerate(comps):
            comp_ms[c] += e[j].elapsed_time(e[j + 1]) * K / K2   # scaled to K steps

    peak, peak_kind = _peaks()
    ms_per_step = total_ms / K
    value = job_throughput(step_bytes, world, ms_per_step)

    kern = {}
    for name, byts, launches in (("map_reduce", MR_BYTES, 1), ("jacobi", ST_BYTES, ST_ITERS),
                                 ("histogram", HI_BYTES, 1), ("batch", BATCH_BYTES, batch.rounds)):
        avg_ms = comp_ms[name] / K
        gbs = byts / (avg_ms * 1e-3) / 1e9
        kern[name] = {"ms": round(avg_ms, 5), "algorithmic_bytes": byts, "GB/s": round(gbs, 1),
                      "frac_of_measured_hbm": round(gbs / peak, 4), "launches": launches}
    kern["jacobi"]["note"] = "2 x 16 MiB grids are L2-resident after the first sweep"
    traffic = measured_traffic()   # per launch (jacobi: per sweep)
    for name in kern:
        kern[name]["dram_bytes_per_launch"] = traffic.get(name)
    # DRAM bytes of a step from the committed ncu counters: per launch for
    # the batch, map->reduce and histogram; for the Jacobi sweeps, whose two
    # grids stay in L2 after the first sweep, the live DRAM bytes of a whole
    # 20-sweep call captured without cache flushing ("jacobi_call_live")
    dram_parts = {"batch": traffic.get("batch"), "map_reduce": traffic.get("map_reduce"),
                  "histogram": traffic.get("histogram"), "jacobi": traffic.get("jacobi_call_live")}
    dram_step = None
    if all(v is not None for v in dram_parts.values()):
        dram_step = dram_parts["batch"] * batch.rounds + dram_parts["map_reduce"] + dram_parts["histogram"] + \
            dram_parts["jacobi"]
    dom = max(comps, key=lambda k: comp_ms[k])
    dom_per_launch_ms = comp_ms[dom] / K / kern[dom]["launches"]
    dom_bytes_per_launch = kern[dom]["algorithmic_bytes"] / kern[dom]["launches"]
    achieved = dom_bytes_per_launch / (dom_per_launch_ms * 1e-3) / 1e9

    # ---- batched vs one launch per instance, same instances, same stream
    batched = bench_batched_vs_per_launch(hx, ctx, batch, batch_tasks, stream, reps=10)
    batched["sweeps_20"] = bench_batch_sweeps(hx, ctx, batch_bufs, stream, peak)

    # ---- serving: continuous batching vs one launch per request
    serving = bench_serving(hx, ctx, dev) if not args.no_serving else None

    # ---- size sweeps of the step's kernels
    sweeps = bench_sweeps(hx, ctx, dev, peak) if not args.no_sweeps else None

    # ---- generic nests and the reduction-tree ablation
    nests = None
    if not args.no_nests:
        nests = {"workloads": bench_nests(hx, ctx, dev, peak), "tree_ablation": bench_tree_ablation(hx, ctx, dev),
                 "srad": bench_srad(hx, ctx, dev, peak)}

    # ---- end to end through the public API with pinned host buffers
    e2e = bench_e2e(args, hx, ctx, dev, x_h, y_h, u_h, v_h, batch, batch_bufs, BATCH_BYTES)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # repeat the full-step sample for about 10 s of single-core work
        vals, spent, desc = [], 0.0, ""
        while spent < 10.0 or len(vals) < 3:
            g, secs, desc = run_oracle_sample()
            vals.append(g)
            spent += secs
        cpu = {"value": round(statistics.median(vals), 4), "unit": "GB/s", "cores": 1, "kind": "oracle",
               "sample": f"{len(vals)} repetitions ({spent:.1f} s) of: {desc}; median"}
        # context: the same nests on all host cores (chunked threads)
        mvals, mspent, T, mdesc = [], 0.0, 1, ""
        while mspent < 5.0 or len(mvals) < 3:
            g, secs, T, mdesc = run_multicore_sample()
            mvals.append(g)
            mspent += secs
        cpu["multicore"] = {"value": round(statistics.median(mvals), 4), "unit": "GB/s", "cores": T,
                            "kind": "host schedule of the oracle's nests (chunked threads)",
                            "sample": f"{len(mvals)} repetitions ({mspent:.1f} s) of: {mdesc}; median"}

    line = {
        "metric": "achieved HBM GB/s (algorithmic bytes / time) of the fork-join hot path",
        "value": round(value, 2), "unit": "GB/s", "n_gpus": world, "steps": K, "warmup": args.warmup,
        "ms_per_step": round(ms_per_step, 5), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 (float-float sums), u8/u32",
        "data": "synthetic (seeded SplitMix64), inputs resident in HBM",
        "config": {
            "workload": "fork-join step: map->reduce N=2^20 a=1.5 + jacobi 2048x2048 x20 sweeps "
                        "+ histogram 2^26 u8 mixture with exclusive scan + batch of 512 map->reduce/stencil "
                        "instances (sizes log-uniform 1K-4M, sides 32-2048) in one persistent launch",
            "parallelism": f"replicas x{world}",
            "step_schedule": "the four independent nests run as concurrent CUDA-graph branches "
                             "(batch | jacobi | map->reduce then histogram); per-kernel times are "
                             "measured in a separate sequential pass",
            "l2": f"inputs rotate over {n_sets} buffer sets ({n_sets * per_set / 2**20:.0f} MiB > 126 MB L2)",
            "step_bytes": step_bytes,
            "tuning": tune_src,
        },
        # value counts algorithmic bytes, some of which the Jacobi sweeps
        # serve from L2; the HBM fraction counts the DRAM bytes ncu measured
        "algorithmic_frac_of_hbm_roofline": round(value / world / peak, 4),
        "dram_bytes_per_step": dram_step,
        "frac_of_hbm_roofline": (round(dram_step / (ms_per_step * 1e-3) / 1e9 / peak, 4)
                                 if dram_step is not None else None),
        "frac_of_nominal_8tbs": round(value / world / 8000.0, 4),
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": round(achieved / peak, 4),
                     "traffic": traffic.get(dom),
                     "algorithmic_bytes_per_launch": dom_bytes_per_launch},
        "kernels": kern,
        "cpu_baseline": cpu,
        "batched": batched,
        "serving": serving,
        "nests": nests,
        "sweeps": sweeps,
        "e2e": e2e,
        "gpu_launches": launches_per_step * K,
        "clocks": clk.summary(),
        "wall_s_timed_region": round(wall, 4),
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
        if args.log:
            append_log(args.log, line)
    ctx.close()
    if dist:
        dist.destroy_process_group()
    return 0


SERVE_RATES = (2000, 5000, 10000, 12000, 15000, 20000, 30000, 40000, 50000)
SERVE_BUDGET = 64 << 30


def _serve_floats(r):
    """fp32 words of device buffers one served request needs (16-byte aligned parts)."""
    up = lambda k: (k + 3) // 4 * 4  # noqa: E731
    if r["kind"] == "map_reduce":
        return 3 * up(r["n"]) + 4
    if r["kind"] == "stencil":
        return 2 * up(r["nx"] * r["ny"]) + up(r["iters"])
    return up((r["n"] + 3) // 4) + 512


def _serve_tasks(hx, arena, trace):
    """hx tasks of a trace, each request's buffers carved from the arena in order."""
    import torch

    tasks, off = [], 0
    for r in trace:
        need = _serve_floats(r)
        seg = arena[off:off + need]
        off += need
        if r["kind"] == "map_reduce":
            n = r["n"]
            m = (n + 3) // 4 * 4
            tasks.append(hx.map_reduce_task(seg[:n], seg[m:m + n], r["a"], seg[3 * m:3 * m + 1],
                                            out=seg[2 * m:2 * m + n]))
        elif r["kind"] == "stencil":
            k = r["nx"] * r["ny"]
            m = (k + 3) // 4 * 4
            tasks.append(hx.stencil_task(seg[:k].view(r["ny"], r["nx"]), seg[m:m + k].view(r["ny"], r["nx"]),
                                         r["iters"], seg[2 * m:2 * m + r["iters"]]))
        else:
            n = r["n"]
            m = ((n + 3) // 4 + 3) // 4 * 4      # fp32 words holding the n bytes, 16-byte aligned
            bins = seg[m:m + 256].view(torch.int32)
            scan = seg[m + 256:m + 512].view(torch.int32)
            tasks.append(hx.histogram_task(seg[:m].view(torch.uint8)[:n], bins, scan))
    return tasks


def serving_comparison(points, targets=(2.0, 5.0, 10.0, 20.0)):
    """Equal-p99 comparison of the serving sweep's two modes.

    The latency bound is the per-launch server's p99 at the highest rate it
    sustains (stable: it keeps up with >= 95% of the offered rate and its
    latency does not grow over the trace); the highest rate each mode
    sustains with p99 within that bound is compared, and the same at fixed
    p99 targets.  ``points``: one dict per offered rate with a "continuous"
    and a "per_launch" entry (req_per_s, p99_ms, stable)."""
    def sustained(mode, bound):
        ok = [p for p in points if p[mode]["stable"] and p[mode]["p99_ms"] <= bound]
        return max(ok, key=lambda p: p["offered_req_per_s"]) if ok else None
    keep = [p for p in points if p["per_launch"]["stable"]]
    if keep:
        bound = max(keep, key=lambda p: p["offered_req_per_s"])["per_launch"]["p99_ms"]
        c = sustained("continuous", bound)
        pl = sustained("per_launch", bound)
        eq = {"p99_bound_ms": bound,
              "per_launch_req_per_s": pl["per_launch"]["req_per_s"] if pl else None,
              "continuous_req_per_s": c["continuous"]["req_per_s"] if c else None}
        if eq["per_launch_req_per_s"] and eq["continuous_req_per_s"]:
            eq["ratio"] = round(eq["continuous_req_per_s"] / eq["per_launch_req_per_s"], 3)
    else:
        # the baseline kept up at no offered rate: there is no latency it
        # sustains, so no equal-p99 bound and no ratio
        eq = {"p99_bound_ms": None, "per_launch_req_per_s": None, "continuous_req_per_s": None,
              "ratio": None, "per_launch_never_stable": True}
    slo = []
    for target in targets:
        c, pl = sustained("continuous", target), sustained("per_launch", target)
        row = {"p99_ms": target, "continuous_req_per_s": c["continuous"]["req_per_s"] if c else None,
               "per_launch_req_per_s": pl["per_launch"]["req_per_s"] if pl else None}
        if row["continuous_req_per_s"] and row["per_launch_req_per_s"]:
            row["ratio"] = round(row["continuous_req_per_s"] / row["per_launch_req_per_s"], 3)
        slo.append(row)
    eq["at_p99_targets"] = slo
    return eq


def timeline_summary(tl):
    """Steps of one serving run from the server's timeline: how many, the
    share issued as standalone calls, mean requests per batched step, mean
    step time (issue to completion seen), and steps in flight (time-weighted
    mean and maximum over the run)."""
    if not tl:
        return {"steps": 0}
    batched = [r for r in tl if not r["direct"]]
    ev = sorted([(r["issue_s"], 1) for r in tl] + [(r["done_s"], -1) for r in tl if r["done_s"] >= 0])
    cur = peak = 0
    area = 0.0
    for (t, d), nxt in zip(ev, ev[1:] + [(ev[-1][0], 0)]):
        cur += d
        peak = max(peak, cur)
        area += cur * (nxt[0] - t)
    span = ev[-1][0] - ev[0][0]
    done = [r["done_s"] - r["issue_s"] for r in tl if r["done_s"] >= 0]
    return {"steps": len(tl), "direct_share": round(1.0 - len(batched) / len(tl), 3),
            "requests_per_batched_step": round(float(np.mean([r["requests"] for r in batched])), 2) if batched else None,
            "step_ms_mean": round(1e3 * float(np.mean(done)), 4) if done else None,
            "steps_in_flight_mean": round(area / span, 2) if span > 0 else None, "steps_in_flight_max": peak}


def bench_serving(hx, ctx, dev, rates=SERVE_RATES, repeats=3, duration_s=1.0, max_requests=10000, distinct=4000,
                  direct_max=0):
    """Open-loop Poisson serving at several offered rates, continuous batching
    vs one launch per request, same requests, same device buffers.

    Each rate runs `repeats` times per mode (modes alternating), each run a
    trace of its own Poisson arrivals lasting `duration_s` or holding
    `max_requests` requests, whichever is fewer; a mode's figures at a rate
    are the medians over its runs, and it counts as stable there when most
    runs were.  Requests draw their kind and size from `distinct` request
    specs (request j uses spec j mod `distinct` and its buffers), so the
    buffers stay within device memory; the runs are timed, not checked."""
    import torch

    specs = workloads.serving_trace(distinct, 1000.0)
    need = sum(_serve_floats(r) for r in specs)
    arena = torch.empty(need, dtype=torch.float32, device=dev)
    g = torch.Generator(device=dev)
    g.manual_seed(4)
    arena.uniform_(-1.0, 1.0, generator=g)
    tasks_all = _serve_tasks(hx, arena, specs)
    points = []
    for lam in rates:
        n = int(min(max_requests, max(300, lam * duration_s)))
        row = {"offered_req_per_s": lam, "requests": n, "repeats": repeats}
        runs = {"continuous": [], "per_launch": []}
        for rep in range(repeats):
            arrivals = [r["arrival_s"] for r in workloads.serving_trace(n, float(lam), seed=workloads.SEED_SERVING + rep)]
            tasks = [tasks_all[j % distinct] for j in range(n)]
            for name, mode in (("continuous", hx.HX_SERVE_CONTINUOUS), ("per_launch", hx.HX_SERVE_PER_LAUNCH)):
                with hx.Server(ctx, mode=mode, hbm_budget_bytes=SERVE_BUDGET, direct_max=direct_max) as srv:
                    lat, makespan = srv.run_trace(tasks, arrivals, timeout_s=300.0)
                    st = srv.stats()
                    tls = timeline_summary(srv.timeline()) if name == "continuous" else None
                lat = np.array(lat) * 1e3
                # a queue that keeps up has stationary latency: the last tenth
                # of the requests (in arrival order) waits no longer than about
                # the first tenth; a growing backlog shows up as a rising tail
                k = max(1, len(lat) // 10)
                head, tail = float(np.median(lat[:k])), float(np.median(lat[-k:]))
                rate = n / makespan
                runs[name].append({"req_per_s": rate, "p50_ms": float(np.percentile(lat, 50)),
                                   "p99_ms": float(np.percentile(lat, 99)), "launches": st["launches"],
                                   "peak_footprint_gb": st["peak_footprint"] / 2**30,
                                   "stable": bool(rate >= 0.95 * lam and tail <= 3.0 * head + 1.0),
                                   "timeline": tls})
        for name, rs in runs.items():
            med = lambda key: float(np.median([r[key] for r in rs]))  # noqa: E731
            row[name] = {"req_per_s": round(med("req_per_s"), 1), "p50_ms": round(med("p50_ms"), 4),
                         "p99_ms": round(med("p99_ms"), 4), "launches": int(med("launches")),
                         "peak_footprint_gb": round(max(r["peak_footprint_gb"] for r in rs), 3),
                         "stable": sum(r["stable"] for r in rs) * 2 > len(rs),
                         "p99_ms_runs": [round(r["p99_ms"], 4) for r in rs],
                         "req_per_s_runs": [round(r["req_per_s"], 1) for r in rs]}
            if name == "continuous":
                # the steps of the run with the median p99 (server timeline)
                mid = sorted(rs, key=lambda r: r["p99_ms"])[len(rs) // 2]
                row[name]["timeline"] = mid["timeline"]
        points.append(row)
    del arena
    torch.cuda.empty_cache()
    eq = serving_comparison(points)
    return {"mix": "1/3 map->reduce, 1/3 jacobi (20 sweeps, square side ~sqrt(n)), 1/3 histogram+scan; "
                   "sizes log-uniform 1K-16M elements (4000 distinct request specs, seed 4); Poisson arrivals "
                   "(seeds 4, 5, 6 for the three runs of a rate)",
            "runs": f"{repeats} per rate and mode, each {duration_s:g} s of arrivals or {max_requests} requests, "
                    "whichever is fewer; medians",
            "budget_gb": SERVE_BUDGET / 2**30, "points": points, "equal_p99": eq}


def _time_ms(fn, reps, warm=2):
    """Mean ms of fn() over reps calls, CUDA events on the current stream."""
    import torch

    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def bench_nests(hx, ctx, dev, peak, reps=20):
    """Generic fork-join nests (map program + monoid reduce) at HBM scale.

    Every input is at least 512 MiB (far above the 126 MB L2), so each call
    streams from HBM.  Algorithmic bytes = inputs read once + outputs written."""
    import torch

    F = 4
    g = torch.Generator(device=dev).manual_seed(5)
    rows = cols = 16384
    big = torch.rand(1 << 28, device=dev, generator=g) * 2 - 1
    x27, y27 = big[: 1 << 27], big[1 << 27:]
    mat = big.view(rows, cols)
    out27 = torch.empty(1 << 27, device=dev)
    res = torch.empty(1 << 24, device=dev)
    idx = torch.empty(1, dtype=torch.int64, device=dev)
    cases = [
        ("sum of 2^28 fp32", [("in", 0)], [big], (1 << 28,), 1, "sum", None, res[:1], None, 4 << 28),
        ("row sums 16384 x 16384", [("in", 0)], [mat], (rows, cols), 1, "sum", None, res[:rows], None,
         F * rows * cols + F * rows),
        ("max over 2^24 rows of 8", [("in", 0)], [big[: 1 << 27].view(1 << 24, 8)], (1 << 24, 8), 1, "max",
         None, res, None, F * (1 << 27) + F * (1 << 24)),
        ("max |x| over 2^28 fp32", [("in", 0), "abs"], [big], (1 << 28,), 1, "max", None, res[:1], None, 4 << 28),
        ("argmax |x - y| over 2^27", [("in", 0), ("in", 1), "sub", "abs"], [x27, y27], (1 << 27,), 1, "argmax",
         None, res[:1], idx, 8 << 27),
        ("map out = fma(x, 1.5, y) over 2^27", [("in", 0), ("const", 0), ("in", 1), "fma"], [x27, y27],
         (1 << 27,), 0, "sum", out27, None, None, 12 << 27),
        ("3-D sum over dims 1,2 of a 1024 x 512 x 512 permuted view", [("in", 0)],
         [big.view(512, 1024, 512).permute(1, 0, 2)], (1024, 512, 512), 2, "sum", None, res[:1024], None,
         F * (1 << 28) + F * 1024),
    ]
    rows_out = []
    for name, prog, ins, dims, rd, monoid, out, result, index, nbytes in cases:
        nest = hx.make_nest(prog, ins, dims, rd, monoid, consts=[1.5], out=out, result=result,
                            result_index=index)
        hx.hx_nest_prepare(nest)
        ms = _time_ms(lambda: hx.hx_fork_reduce(ctx, nest), reps)
        gbs = nbytes / (ms * 1e-3) / 1e9
        rows_out.append({"nest": name, "ms": round(ms, 4), "algorithmic_bytes": nbytes, "GB/s": round(gbs, 1),
                         "frac_of_measured_hbm": round(gbs / peak, 4)})
    rows_out[0]["dram_bytes_per_launch"] = measured_traffic().get("nest_sum_2p28")
    del big, out27, res
    torch.cuda.empty_cache()
    return rows_out


def bench_tree_ablation(hx, ctx, dev, n=1 << 20, reps=5):
    """The EDGE experiment of Sec. 5.2 as a kernel-level ablation: one large
    max reduction (max |x| over a 1024 x 1024 image) as the sequential loop,
    as the two-level chunk tree, and as the warp-shuffle tree."""
    import torch

    g = torch.Generator(device=dev).manual_seed(6)
    x = torch.rand(n, device=dev, generator=g) * 2 - 1
    res = torch.empty(1, device=dev)
    ms = {}
    for tree in ("seq", "chunk", "warp"):
        nest = hx.make_nest([("in", 0), "abs"], [x], (n,), 1, "max", result=res, tree=tree)
        hx.hx_nest_prepare(nest)
        ms[tree] = _time_ms(lambda: hx.hx_fork_reduce(ctx, nest), reps if tree == "seq" else 50)
    return {"reduction": f"max |x| over {n} fp32 (one segment)", "seq_ms": round(ms["seq"], 4),
            "chunk_tree_ms": round(ms["chunk"], 4), "warp_tree_ms": round(ms["warp"], 4),
            "chunk_tree_speedup": round(ms["seq"] / ms["chunk"], 2),
            "warp_tree_speedup": round(ms["seq"] / ms["warp"], 2),
            "paper_edge_end_to_end": {"tree": 6.22, "tree_plus_warp": 9.77}}


def bench_srad(hx, ctx, dev, peak, ny=8192, nx=8192, iters=10, reps=3):
    """SRAD-style nest on an 8192 x 8192 image (256 MiB, far above L2), 10
    iterations, lambda 0.5, 128 x 128 region of interest: the fused path
    (one kernel per iteration) against the unfused loop nest (region reduce,
    coefficient, update).  Each repetition restarts from the same image.
    Algorithmic bytes: 8 per pixel and iteration (read J, write J')."""
    import torch

    import workloads

    src = torch.from_numpy(workloads.srad_image(ny, nx)).to(dev)
    J0, J1, C = torch.empty_like(src), torch.empty_like(src), torch.empty_like(src)
    q0 = torch.empty(iters, device=dev)
    roi = (0, 128, 0, 128)
    out = {}
    for fused in (True, False):
        ms = []
        for r in range(reps + 1):
            J0.copy_(src)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            hx.hx_srad(ctx, J0, J1, iters, 0.5, roi, q0sq=q0, fused=fused, C=C)
            b.record()
            torch.cuda.synchronize()
            if r:
                ms.append(a.elapsed_time(b))
        out["fused" if fused else "unfused"] = sorted(ms)[len(ms) // 2]
    npx = ny * nx
    per_it = {k: v / iters for k, v in out.items()}
    gbs = 8 * npx / (per_it["fused"] * 1e-3) / 1e9
    del src, J0, J1, C
    torch.cuda.empty_cache()
    return {"image": f"{ny} x {nx} fp32, {iters} iterations, lambda 0.5, region 128 x 128",
            "fused_ms_per_iteration": round(per_it["fused"], 4),
            "unfused_ms_per_iteration": round(per_it["unfused"], 4),
            "fusion_speedup": round(per_it["unfused"] / per_it["fused"], 3),
            "fused_mpix_per_s": round(npx / (per_it["fused"] * 1e-3) / 1e6, 1),
            "fused_algorithmic_GB/s": round(gbs, 1), "fused_frac_of_measured_hbm": round(gbs / peak, 4),
            "fused_dram_bytes_per_iteration": measured_traffic().get("srad_fused"),
            "bound": "issue (an IEEE fp32 division per pixel in the coefficient)",
            "launches_per_iteration": {"fused": 1, "unfused": 3}}


def bench_sweeps(hx, ctx, dev, peak):
    """Size sweeps (each point timed over rotating inputs that together exceed
    the 126 MB L2, so every call streams from HBM): map->reduce 2^20..2^28,
    Jacobi 2048^2 / 8192^2 / 16384^2 x 20 sweeps (the larger grids do not fit
    in L2, so their algorithmic GB/s is HBM traffic), and the histogram at
    2^24..2^30 mixture bytes plus two adversarial 2^26 inputs (every byte the
    same value; a ramp 0, 1, ..., 255, 0, ...)."""
    import torch

    import workloads

    # one stream for every capture (the context keeps a workspace slot per
    # distinct stream)
    sweep_stream = torch.cuda.Stream(device=dev)

    def per_call_ms(fn, n_sets, reps):
        # the calls go into one CUDA graph (device time, not host launch
        # overhead); after three warm-up replays, five timed replays with
        # events on the replay stream; the median replay
        for k in range(n_sets):
            fn(k)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        s = sweep_stream
        with torch.cuda.graph(g, stream=s):
            for k in range(reps):
                fn(k % n_sets)
        with torch.cuda.stream(s):
            for _ in range(3):
                g.replay()
            evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(5)]
            for a, b in evs:
                a.record(s)
                g.replay()
                b.record(s)
        torch.cuda.synchronize()
        return statistics.median(a.elapsed_time(b) for a, b in evs) / reps

    out = {"map_reduce": [], "jacobi_x20": [], "histogram": []}
    s32 = torch.empty(1, device=dev)
    for lg in (20, 22, 24, 26, 28):
        n = 1 << lg
        n_sets = max(1, (512 << 20) // (12 * n))
        xs = [workloads.uniform_pm1_f32_torch(0, n, dev, 2, 0) for _ in range(1)]
        x, y = xs[0], workloads.uniform_pm1_f32_torch(0, n, dev, 2, 1)
        sets = [(x.clone(), y.clone(), torch.empty_like(x)) for _ in range(n_sets)]
        del x, y, xs
        ms = per_call_ms(lambda k: hx.hx_map_reduce(ctx, sets[k][0], sets[k][1], 1.5, out=sets[k][2], sum_out=s32),
                         n_sets, max(8, 2 * n_sets))
        gbs = 12 * n / (ms * 1e-3) / 1e9
        out["map_reduce"].append({"n": f"2^{lg}", "ms": round(ms, 5), "GB/s": round(gbs, 1),
                                  "frac_of_measured_hbm": round(gbs / peak, 4)})
        del sets
        torch.cuda.empty_cache()
    for side in (2048, 8192, 16384):
        u0 = torch.from_numpy(workloads.stencil_grid(side, side)).to(dev) if side <= 8192 else \
            workloads.uniform01_f32_torch(1, side * side, dev).view(side, side)
        u1 = torch.empty_like(u0)
        res = torch.empty(20, device=dev)
        ms = per_call_ms(lambda k: hx.hx_stencil2d(ctx, u0, u1, 20, resid=res), 1, 3)
        gbs = 8 * side * side * 20 / (ms * 1e-3) / 1e9
        out["jacobi_x20"].append({"grid": f"{side}^2", "ms": round(ms, 4), "algorithmic_GB/s": round(gbs, 1),
                                  "frac_of_measured_hbm": round(gbs / peak, 4),
                                  "resident": "L2" if side <= 2048 else "HBM"})
        del u0, u1
        torch.cuda.empty_cache()
    bins = torch.empty(256, dtype=torch.int32, device=dev)
    scan = torch.empty_like(bins)
    cases = [(f"mixture 2^{lg}", lg, None) for lg in (24, 26, 28, 30)]
    cases += [("one value 2^26", 26, "one"), ("ramp 2^26", 26, "ramp")]
    for name, lg, kind in cases:
        n = 1 << lg
        if kind is None:
            v0 = torch.from_numpy(workloads.histogram_mixture_u8(min(n, 1 << 26))).to(dev)
            v0 = v0.repeat(n // v0.numel())
        elif kind == "one":
            v0 = torch.full((n,), 7, dtype=torch.uint8, device=dev)
        else:
            v0 = (torch.arange(n, device=dev) % 256).to(torch.uint8)
        n_sets = max(1, (512 << 20) // n)
        sets = [v0] + [v0.clone() for _ in range(n_sets - 1)]
        ms = per_call_ms(lambda k: hx.hx_histogram(ctx, sets[k], bins, scan), n_sets, max(8, 2 * n_sets))
        gbs = n / (ms * 1e-3) / 1e9
        out["histogram"].append({"input": name, "ms": round(ms, 5), "GB/s": round(gbs, 1),
                                 "frac_of_measured_hbm": round(gbs / peak, 4)})
        del sets, v0
        torch.cuda.empty_cache()
    return out


def bench_batched_vs_per_launch(hx, ctx, batch, tasks, stream, reps=10):
    """requests/s of the 512 instances as one batch vs one launch per instance.

    Per-launch is timed twice: issued from the host call by call, and with the
    512 launches captured in one CUDA graph (no host overhead)."""
    import torch

    def per_launch():
        for t in tasks:
            if t.kind == hx.HX_TASK_MAP_REDUCE:
                x, y, out, s32 = t.keep[0], t.keep[1], t.keep[2], t.keep[3]
                hx.hx_map_reduce(ctx, x, y, t.u.mr.a, out=out, sum_out=s32, stream=stream)
            else:
                u0, u1, res = t.keep
                hx.hx_stencil2d(ctx, u0, u1, 1, resid=res, stream=stream)

    def timed(fn):
        with torch.cuda.stream(stream):
            fn()
            stream.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(reps):
                fn()
            b.record(stream)
            stream.synchronize()
        return a.elapsed_time(b) / reps

    g_batch = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g_batch, stream=stream):
        batch.launch(stream=stream)
    g_per = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g_per, stream=stream):
        per_launch()
    ms_b = timed(g_batch.replay)
    ms_pg = timed(g_per.replay)
    ms_pe = timed(per_launch)
    n = len(tasks)
    return {"instances": n, "batched_ms": round(ms_b, 4), "batched_req_per_s": round(n / ms_b * 1e3, 1),
            "per_launch_graph_ms": round(ms_pg, 4), "per_launch_graph_req_per_s": round(n / ms_pg * 1e3, 1),
            "per_launch_eager_ms": round(ms_pe, 4), "per_launch_eager_req_per_s": round(n / ms_pe * 1e3, 1),
            "speedup_vs_graph": round(ms_pg / ms_b, 3), "speedup_vs_eager": round(ms_pe / ms_b, 3)}


def bench_batch_sweeps(hx, ctx, batch_bufs, stream, peak, sweeps=20, reps=5):
    """The 512-instance batch with every stencil instance running `sweeps`
    sweeps (same buffers and sizes as the step's batch): all sweeps in one
    persistent launch against one launch per sweep (rounds), each captured in
    a CUDA graph.  Algorithmic bytes: 12 per map element, 8 per stencil point
    and sweep."""
    import torch

    tasks, byts, res = [], 0, []
    for bb in batch_bufs:
        if len(bb) == 4:
            x, y, out, s32 = bb
            tasks.append(hx.map_reduce_task(x, y, 1.5, s32, out=out))
            byts += 12 * x.numel()
        else:
            u0, u1, _ = bb
            r = torch.empty(sweeps, device=u0.device)
            res.append(r)
            tasks.append(hx.stencil_task(u0, u1, sweeps, r))
            byts += 8 * u0.numel() * sweeps
    out = {"sweeps": sweeps, "algorithmic_bytes": byts}
    for name, rounds in (("one_launch", False), ("rounds", True)):
        b = hx.hx_batch_plan(ctx, tasks, rounds=rounds)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            b.launch(stream=stream)
        with torch.cuda.stream(stream):
            g.replay()
            stream.synchronize()
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
            for a, e in ev:
                a.record(stream)
                g.replay()
                e.record(stream)
            stream.synchronize()
        b.status()
        ms = statistics.median(a.elapsed_time(e) for a, e in ev)
        gbs = byts / (ms * 1e-3) / 1e9
        out[name] = {"ms": round(ms, 4), "launches": 2 * b.rounds, "GB/s": round(gbs, 1),
                     "frac_of_measured_hbm": round(gbs / peak, 4)}
        del g
        b.close()
    out["one_launch_speedup"] = round(out["rounds"]["ms"] / out["one_launch"]["ms"], 3)
    # other batch shapes, 20 sweeps each: one launch against rounds
    shapes = []
    for count, lo, hi in ((512, 32, 128), (64, 32, 2048), (8, 1024, 4096), (1, 4096, 4096)):
        keep, st_tasks, per_sweep = [], [], 0
        for j in range(count):
            side = int(workloads.log_uniform_int(99, j, lo, hi)) if lo < hi else lo
            u0 = workloads.uniform_pm1_f32_torch(j, side * side, stream.device).view(side, side)
            u1, r = torch.empty_like(u0), torch.empty(sweeps, device=u0.device)
            keep += [u0, u1, r]
            st_tasks.append(hx.stencil_task(u0, u1, sweeps, r))
            per_sweep += 8 * side * side
        row = {"instances": count, "sides": f"{lo}-{hi}" if lo < hi else str(lo), "bytes_per_sweep": per_sweep}
        for name, rounds in (("one_launch_ms", False), ("rounds_ms", True)):
            b = hx.hx_batch_plan(ctx, st_tasks, rounds=rounds)
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=stream):
                b.launch(stream=stream)
            with torch.cuda.stream(stream):
                g.replay()
                ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
                for a, e in ev:
                    a.record(stream)
                    g.replay()
                    e.record(stream)
                stream.synchronize()
            b.status()
            row[name] = round(statistics.median(a.elapsed_time(e) for a, e in ev), 4)
            del g
            b.close()
        row["one_launch_speedup"] = round(row["rounds_ms"] / row["one_launch_ms"], 3)
        shapes.append(row)
        del keep
    out["shapes"] = shapes
    return out


def bench_e2e(args, hx, ctx, dev, x_h, y_h, u_h, v_h, batch, batch_bufs, batch_bytes, steps=None):
    """The whole step through the public API, with every output read back:
    inputs copied in from pinned host memory and all results copied out to
    pinned host memory, inside the timed region.

    A step's inputs (x, y, the Jacobi grid, the histogram bytes and every
    batch instance's inputs) sit in one pinned host buffer laid out like a
    device input arena, and its outputs (the map output, every batch
    instance's output array or final grid, the sums, residuals, bins and
    scan) are written into a device output arena laid out like one pinned
    host buffer, so each direction crosses the host link in one copy (two
    for the outputs: the arena, and the Jacobi grid, whose 20 sweeps end in
    the input arena).  Two input and two output arenas alternate: step
    i + 1's inputs are copied in, and step i - 1's outputs copied out, while
    step i computes (the batch is planned once per arena pair)."""
    import torch

    steps = steps or max(3, min(args.steps, 10))
    in_parts = [("x", torch.from_numpy(x_h)), ("y", torch.from_numpy(y_h)), ("u", torch.from_numpy(u_h)),
                ("v", torch.from_numpy(v_h))]
    out_parts = [("out", (MR_N,), torch.float32), ("s32", (1,), torch.float32), ("s64", (1,), torch.float64),
                 ("res", (ST_ITERS,), torch.float32), ("bins", (256,), torch.int32), ("scan", (256,), torch.int32),
                 ("u1", u_h.shape, torch.float32)]
    for k, bb in enumerate(batch_bufs):
        if len(bb) == 4:
            in_parts += [(f"bx{k}", bb[0].cpu()), (f"by{k}", bb[1].cpu())]
            out_parts += [(f"bo{k}", tuple(bb[2].shape), torch.float32), (f"bs{k}", (1,), torch.float32)]
        else:
            in_parts.append((f"bu{k}", bb[0].cpu()))
            out_parts += [(f"bv{k}", tuple(bb[1].shape), torch.float32), (f"br{k}", (1,), torch.float32)]

    def layout(parts):
        offs, total = {}, 0
        for name, shape, dt in parts:
            nb = int(np.prod(shape)) * torch.empty(0, dtype=dt).element_size()
            offs[name] = (total, nb, shape, dt)
            total += (nb + 255) // 256 * 256
        return offs, total

    in_offs, in_total = layout([(n, tuple(t.shape), t.dtype) for n, t in in_parts])
    out_offs, out_total = layout(out_parts)
    stage = torch.empty(in_total, dtype=torch.uint8).pin_memory()
    for name, t in in_parts:
        o, nb, _, _ = in_offs[name]
        stage[o:o + nb].copy_(t.contiguous().view(-1).view(torch.uint8))
    out_h = torch.empty(out_total, dtype=torch.uint8).pin_memory()
    grid_h = torch.empty(u_h.size * 4, dtype=torch.uint8).pin_memory()

    def views(arena, offs):
        return {name: arena[o:o + nb].view(dt).view(shape) for name, (o, nb, shape, dt) in offs.items()}

    ins, outs, plans = [], [], []
    for _ in range(2):
        ia = torch.empty(in_total, dtype=torch.uint8, device=dev)
        oa = torch.empty(out_total, dtype=torch.uint8, device=dev)
        iv, ov = views(ia, in_offs), views(oa, out_offs)
        tasks = []
        for k, bb in enumerate(batch_bufs):
            if len(bb) == 4:
                tasks.append(hx.map_reduce_task(iv[f"bx{k}"], iv[f"by{k}"], 1.5, ov[f"bs{k}"], out=ov[f"bo{k}"]))
            else:
                tasks.append(hx.stencil_task(iv[f"bu{k}"], ov[f"bv{k}"], 1, ov[f"br{k}"]))
        ins.append((ia, iv))
        outs.append((oa, ov))
        plans.append(hx.hx_batch_plan(ctx, tasks))
    s = torch.cuda.Stream(device=dev)        # compute
    cs = torch.cuda.Stream(device=dev)       # input copies
    ds = torch.cuda.Stream(device=dev)       # output copies
    ready = [torch.cuda.Event() for _ in range(2)]   # inputs of arena k copied in
    done = [torch.cuda.Event() for _ in range(2)]    # compute on arena k finished
    free = [torch.cuda.Event() for _ in range(2)]    # outputs of arena k copied out
    h2d = in_total
    d2h = out_total + u_h.size * 4

    def copy_in(k):
        cs.wait_event(free[k])
        with torch.cuda.stream(cs):
            ins[k][0].copy_(stage, non_blocking=True)
        ready[k].record(cs)

    def compute(k):
        iv, ov = ins[k][1], outs[k][1]
        s.wait_event(ready[k])
        s.wait_event(free[k])
        hx.hx_map_reduce(ctx, iv["x"], iv["y"], 1.5, out=ov["out"], sum_out=ov["s32"], sum64_out=ov["s64"], stream=s)
        hx.hx_stencil2d(ctx, iv["u"], ov["u1"], ST_ITERS, resid=ov["res"], stream=s)
        hx.hx_histogram(ctx, iv["v"], bins=ov["bins"], scan=ov["scan"], stream=s)
        plans[k].launch(stream=s)
        done[k].record(s)

    def copy_out(k):
        ds.wait_event(done[k])
        with torch.cuda.stream(ds):
            out_h.copy_(outs[k][0], non_blocking=True)
            grid_h.copy_(ins[k][1]["u"].view(-1).view(torch.uint8), non_blocking=True)   # 20 sweeps end in u
        free[k].record(ds)

    def run(n, start=None):
        if start is not None:
            cs.wait_event(start)
        copy_in(0)
        for i in range(n):
            if i + 1 < n:
                copy_in((i + 1) % 2)
            compute(i % 2)
            copy_out(i % 2)

    for k in range(2):
        free[k].record(ds)
    run(2)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(s)
    run(steps, start=a)
    ds.wait_event(done[(steps - 1) % 2])
    b.record(ds)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / steps
    # the last step's read-back must hold this step's results: the map output
    # bit for bit, its sum within the fp64 tolerance, the histogram exactly
    ov = views(out_h, out_offs)
    ref_out = 1.5 * x_h.astype(np.float64) + y_h.astype(np.float64)
    ok = np.array_equal(ov["out"].numpy(), ref_out.astype(np.float32))
    ok &= abs(float(ov["s64"].item()) - ref_out.sum()) <= 1e-5 * np.abs(ref_out).sum()
    ok &= np.array_equal(ov["bins"].numpy().view(np.uint32), np.bincount(v_h.ravel(), minlength=256).astype(np.uint32))
    ok &= bool(np.isfinite(grid_h.view(torch.float32).numpy()).all())
    if not ok:
        raise RuntimeError("e2e: the read-back results differ from the step's expected results")
    for p in plans:
        p.close()
    del ins, outs, stage, out_h, grid_h
    torch.cuda.empty_cache()
    total_alg = STEP_BYTES + batch_bytes
    return {"value": round(total_alg / (ms * 1e-3) / 1e9, 2), "unit": "GB/s", "ms_per_step": round(ms, 4),
            "steps": steps, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "readback": "every output: map output, final Jacobi grid, every batch instance's output array or "
                        "final grid, and all sums, residuals, bins and scan",
            "pipeline": "one input copy per step into one of two device arenas and one output copy (plus the "
                        "Jacobi grid) out of one of two output arenas, overlapped with the neighbouring "
                        "steps' compute"}


def log_rows(line):
    """The measurements of one bench line as flat rows: one per kernel, size
    sweep point, generic nest and serving rate, each with the run's clocks
    and host core count."""
    run = {"time": time.strftime("%Y-%m-%dT%H:%M:%S"), "n_gpus": line["n_gpus"],
           "host_cores": len(os.sched_getaffinity(0)), "sm_mhz": line["clocks"].get("sm_mhz"),
           "peak_gbs": line["roofline"]["peak"]}
    nominal = 8000.0
    rows = [dict(run, kind="step", ms=line["ms_per_step"], gbs=line["value"],
                 frac_measured=line["algorithmic_frac_of_hbm_roofline"],
                 dram_frac_measured=line["frac_of_hbm_roofline"], frac_nominal=round(line["value"] / nominal, 4))]
    for name, k in line["kernels"].items():
        rows.append(dict(run, kind="kernel", name=name, ms=k["ms"], bytes=k["algorithmic_bytes"], gbs=k["GB/s"],
                         frac_measured=k["frac_of_measured_hbm"], frac_nominal=round(k["GB/s"] / nominal, 4)))
    for group, pts in (line.get("sweeps") or {}).items():
        for p in pts:
            gbs = p.get("GB/s", p.get("algorithmic_GB/s"))
            rows.append(dict(run, kind="sweep", name=group, size=p.get("n") or p.get("grid") or p.get("input"),
                             ms=p["ms"], gbs=gbs, frac_measured=p["frac_of_measured_hbm"],
                             frac_nominal=round(gbs / nominal, 4)))
    for w in ((line.get("nests") or {}).get("workloads") or []):
        rows.append(dict(run, kind="nest", name=w["nest"], ms=w["ms"], bytes=w["algorithmic_bytes"], gbs=w["GB/s"],
                         frac_measured=w["frac_of_measured_hbm"], frac_nominal=round(w["GB/s"] / nominal, 4)))
    for p in ((line.get("serving") or {}).get("points") or []):
        for mode in ("continuous", "per_launch"):
            m = p[mode]
            rows.append(dict(run, kind="serving", name=mode, offered_req_per_s=p["offered_req_per_s"],
                             req_per_s=m["req_per_s"], p50_ms=m["p50_ms"], p99_ms=m["p99_ms"], stable=m["stable"]))
    if line.get("e2e"):
        rows.append(dict(run, kind="e2e", ms=line["e2e"]["ms_per_step"], gbs=line["e2e"]["value"]))
    return rows


def append_log(path, line):
    """Append the run's rows to a JSON-lines log."""
    with open(path, "a") as f:
        for r in log_rows(line):
            f.write(json.dumps(r) + "\n")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["hx", "reference"], default="hx")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--autotune", action="store_true", help="re-measure the tuning table before timing")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving sweep")
    ap.add_argument("--no-nests", action="store_true", help="skip the generic-nest section")
    ap.add_argument("--no-sweeps", action="store_true", help="skip the size sweeps")
    ap.add_argument("--log", default=None, help="also append one JSON row per measurement to this file")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    rank, world, local = _dist_env()
    if args.impl == "reference":
        return bench_reference(args, rank, world)
    return bench_hx(args, rank, world, local)


if __name__ == "__main__":
    sys.exit(main())

#!/usr/bin/env python3
"""Benchmark of the fork-join hot path on B300.

One step = one pass of every nest of the hot path over one batch of seeded
synthetic input:
  * map->reduce: out = fmaf(1.5, x, y), s = sum(out), N = 2^20
  * Jacobi: 20 clamp-to-edge 5-point sweeps of a 2048 x 2048 fp32 grid with a
    max residual per sweep
  * histogram: 256 bins of 2^26 mixture bytes + exclusive scan
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
    """Samples SM clock and throttle reasons through NVML while running."""

    def __init__(self, index: int, period_s: float = 0.01):
        self.index, self.period = index, period_s
        self.samples = []
        self.reasons = set()
        self.max_mhz = None
        self._stop = threading.Event()
        self._thr = None
        self.ok = False

    def __enter__(self):
        try:
            import pynvml

            pynvml.nvmlInit()
            self._nv = pynvml
            self._h = pynvml.nvmlDeviceGetHandleByIndex(self.index)
            self.max_mhz = pynvml.nvmlDeviceGetMaxClockInfo(self._h, pynvml.NVML_CLOCK_SM)
            self.ok = True
            self._thr = threading.Thread(target=self._run, daemon=True)
            self._thr.start()
        except Exception as e:  # NVML missing: record why, keep benchmarking
            self.err = str(e)
        return self

    def _run(self):
        nv = self._nv
        names = {
            "gpu_idle": getattr(nv, "nvmlClocksEventReasonGpuIdle", 0x1),
            "sw_power_cap": getattr(nv, "nvmlClocksEventReasonSwPowerCap", 0x4),
            "hw_slowdown": getattr(nv, "nvmlClocksEventReasonHwSlowdown", 0x8),
            "sw_thermal_slowdown": getattr(nv, "nvmlClocksEventReasonSwThermalSlowdown", 0x20),
            "hw_thermal_slowdown": getattr(nv, "nvmlClocksEventReasonHwThermalSlowdown", 0x40),
            "hw_power_brake_slowdown": getattr(nv, "nvmlClocksEventReasonHwPowerBrakeSlowdown", 0x80),
        }
        while not self._stop.is_set():
            try:
                mhz = nv.nvmlDeviceGetClockInfo(self._h, nv.NVML_CLOCK_SM)
                util = nv.nvmlDeviceGetUtilizationRates(self._h).gpu
                r = nv.nvmlDeviceGetCurrentClocksEventReasons(self._h)
                self.samples.append((mhz, util))
                for k, bit in names.items():
                    if r & bit and k != "gpu_idle":
                        self.reasons.add(k)
            except Exception:
                pass
            time.sleep(self.period)

    def __exit__(self, *exc):
        self._stop.set()
        if self._thr:
            self._thr.join()

    def summary(self):
        if not self.ok:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "note": getattr(self, "err", "")}
        loaded = [m for m, u in self.samples if u > 0] or [m for m, _ in self.samples]
        return {"sm_mhz": statistics.median(loaded) if loaded else None, "sm_max_mhz": self.max_mhz,
                "reasons": sorted(self.reasons), "samples": len(self.samples)}


# ---------------------------------------------------------------- CPU oracle
def run_oracle_sample(budget_s: float = 15.0):
    """Time the CPU oracle on a bounded sample of the step workload.

    The sample: the full map->reduce instance, the full histogram, and the
    2048 x 2048 Jacobi grid for as many sweeps as fit the time budget (at
    least one).  Returns (GB/s of algorithmic bytes, seconds, description)."""
    import oracle

    x, y = workloads.map_reduce_inputs(MR_N)
    v = workloads.histogram_mixture_u8(HI_N)
    u0 = workloads.stencil_grid(ST_SIDE, ST_SIDE).astype(np.float64)
    oracle.map_reduce(x[:16], y[:16], 1.5)  # load the library outside the timing
    t0 = time.perf_counter()
    oracle.map_reduce(x, y, 1.5)
    t_mr = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.histogram(v)
    t_hi = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.jacobi(u0, 1)
    t_sweep = time.perf_counter() - t0
    sweeps = int(max(1, min(ST_ITERS, (budget_s - t_mr - t_hi - t_sweep) // max(t_sweep, 1e-9))))
    t0 = time.perf_counter()
    if sweeps > 1:
        oracle.jacobi(u0, sweeps)
    t_st = (time.perf_counter() - t0) if sweeps > 1 else t_sweep
    total_bytes = MR_BYTES + HI_BYTES + ST_BYTES_PER_SWEEP * sweeps
    total_s = t_mr + t_hi + t_st
    desc = (f"map_reduce N=2^20 + histogram 2^26 + jacobi 2048^2 x {sweeps} sweeps (of 20), "
            f"sequential fp64/int oracle, {total_s:.2f} s")
    return total_bytes / total_s / 1e9, total_s, desc


def bench_reference(args, rank, world):
    if rank != 0:
        return 0
    gbs, secs, desc = None, 0.0, ""
    vals = []
    for i in range(args.warmup + args.steps):
        g, s, d = run_oracle_sample(budget_s=max(2.0, 60.0 / max(1, args.warmup + args.steps)))
        if i >= args.warmup:
            vals.append(g)
            secs += s
            desc = d
    gbs = statistics.median(vals)
    line = {
        "impl": "reference", "metric": "achieved HBM GB/s (algorithmic bytes / time) of the fork-join hot path",
        "value": round(gbs, 4), "unit": "GB/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(1e3 * secs / max(1, args.steps), 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32/f64/u8",
        "data": "synthetic (seeded SplitMix64)",
        "config": {"workload": "cpu oracle on a bounded sample of the fork-join step", "sample": desc},
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
                "u0": u_d0.clone(), "u1": torch.empty_like(u_d0), "u_init": u_d0,
                "res": torch.empty(ST_ITERS, device=dev),
                "v": v_d0.clone(), "bins": torch.empty(256, dtype=torch.int32, device=dev),
                "scan": torch.empty(256, dtype=torch.int32, device=dev),
            }
            sets.append(s)
    stream.synchronize()

    def run_step(s, ev=None):
        # the Jacobi sweeps overwrite u0: restore the input grid first (a copy,
        # outside the per-kernel events, inside the step)
        s["u0"].copy_(s["u_init"], non_blocking=True)
        if ev is not None:
            ev[0].record(stream)
        hx.hx_map_reduce(ctx, s["x"], s["y"], 1.5, out=s["out"], sum_out=s["s32"], sum64_out=s["s64"],
                         stream=stream)
        if ev is not None:
            ev[1].record(stream)
        hx.hx_stencil2d(ctx, s["u0"], s["u1"], ST_ITERS, resid=s["res"], stream=stream)
        if ev is not None:
            ev[2].record(stream)
        hx.hx_histogram(ctx, s["v"], bins=s["bins"], scan=s["scan"], stream=stream)
        if ev is not None:
            ev[3].record(stream)

    launches_per_step = 1 + ST_ITERS + 1

    with torch.cuda.stream(stream):
        for i in range(args.warmup):
            run_step(sets[i % n_sets])
    stream.synchronize()

    K = args.steps
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(K)]
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk, torch.cuda.stream(stream):
        wall0 = time.perf_counter()
        t_start.record(stream)
        for i in range(K):
            run_step(sets[i % n_sets], evs[i])
        t_end.record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
    if dist:
        dist.barrier()
    total_ms = t_start.elapsed_time(t_end)
    comp_ms = {"map_reduce": 0.0, "jacobi": 0.0, "histogram": 0.0}
    for e in evs:
        comp_ms["map_reduce"] += e[0].elapsed_time(e[1])
        comp_ms["jacobi"] += e[1].elapsed_time(e[2])
        comp_ms["histogram"] += e[2].elapsed_time(e[3])
    if dist:
        t = torch.tensor([total_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())

    peak, peak_kind = _peaks()
    ms_per_step = total_ms / K
    value = world * STEP_BYTES / (ms_per_step * 1e-3) / 1e9

    kern = {}
    for name, byts, launches in (("map_reduce", MR_BYTES, 1), ("jacobi", ST_BYTES, ST_ITERS),
                                 ("histogram", HI_BYTES, 1)):
        avg_ms = comp_ms[name] / K
        gbs = byts / (avg_ms * 1e-3) / 1e9
        kern[name] = {"ms": round(avg_ms, 5), "algorithmic_bytes": byts, "GB/s": round(gbs, 1),
                      "frac_of_measured_hbm": round(gbs / peak, 4), "launches": launches}
    kern["jacobi"]["note"] = "2 x 16 MiB grids are L2-resident after the first sweep"
    dom = max(("map_reduce", "jacobi", "histogram"), key=lambda k: comp_ms[k])
    dom_per_launch_ms = comp_ms[dom] / K / kern[dom]["launches"]
    dom_bytes_per_launch = kern[dom]["algorithmic_bytes"] / kern[dom]["launches"]
    achieved = dom_bytes_per_launch / (dom_per_launch_ms * 1e-3) / 1e9

    # ---- end to end through the public API with pinned host buffers
    e2e = bench_e2e(args, hx, ctx, dev, x_h, y_h, u_h, v_h)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        g, secs, desc = run_oracle_sample()
        cpu = {"value": round(g, 4), "unit": "GB/s", "cores": 1, "kind": "oracle", "sample": desc}

    line = {
        "metric": "achieved HBM GB/s (algorithmic bytes / time) of the fork-join hot path",
        "value": round(value, 2), "unit": "GB/s", "n_gpus": world, "steps": K, "warmup": args.warmup,
        "ms_per_step": round(ms_per_step, 5), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 (fp64 reduce combine), u8/u32",
        "data": "synthetic (seeded SplitMix64), inputs resident in HBM",
        "config": {
            "workload": "fork-join step: map->reduce N=2^20 a=1.5 + jacobi 2048x2048 x20 sweeps "
                        "+ histogram 2^26 u8 mixture with exclusive scan",
            "parallelism": f"replicas x{world}",
            "l2": f"inputs rotate over {n_sets} buffer sets ({n_sets * per_set / 2**20:.0f} MiB > 126 MB L2)",
            "step_bytes": STEP_BYTES,
        },
        "frac_of_hbm_roofline": round(value / world / peak, 4),
        "frac_of_nominal_8tbs": round(value / world / 8000.0, 4),
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": round(achieved / peak, 4),
                     "traffic": None},
        "kernels": kern,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches_per_step * K,
        "clocks": clk.summary(),
        "wall_s_timed_region": round(wall, 4),
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()
    return 0


def bench_e2e(args, hx, ctx, dev, x_h, y_h, u_h, v_h, steps=None):
    """Same step through the public API, host buffers in and results out."""
    import torch

    steps = steps or max(3, min(args.steps, 20))
    pin = lambda a: torch.from_numpy(a).pin_memory()  # noqa: E731
    xh, yh, uh, vh = pin(x_h), pin(y_h), pin(u_h), pin(v_h)
    xd, yd = torch.empty_like(xh, device=dev), torch.empty_like(yh, device=dev)
    ud, u1 = torch.empty_like(uh, device=dev), torch.empty_like(uh, device=dev)
    vd = torch.empty_like(vh, device=dev)
    out = torch.empty(MR_N, device=dev)
    s64 = torch.empty(1, dtype=torch.float64, device=dev)
    res = torch.empty(ST_ITERS, device=dev)
    bins = torch.empty(256, dtype=torch.int32, device=dev)
    scan = torch.empty(256, dtype=torch.int32, device=dev)
    res_h = torch.empty(8 + 8 + 4 * ST_ITERS + 2048, dtype=torch.uint8).pin_memory()
    s = torch.cuda.Stream(device=dev)
    h2d = 4 * MR_N * 2 + 4 * ST_SIDE * ST_SIDE + HI_N
    d2h = 4 + 8 + 4 * ST_ITERS + 2 * 1024

    def one():
        xd.copy_(xh, non_blocking=True)
        yd.copy_(yh, non_blocking=True)
        ud.copy_(uh, non_blocking=True)
        vd.copy_(vh, non_blocking=True)
        _, s32, _ = hx.hx_map_reduce(ctx, xd, yd, 1.5, out=out, sum64_out=s64, stream=s)
        hx.hx_stencil2d(ctx, ud, u1, ST_ITERS, resid=res, stream=s)
        hx.hx_histogram(ctx, vd, bins=bins, scan=scan, stream=s)
        res_h[0:4].copy_(s32.view(torch.uint8), non_blocking=True)
        res_h[8:16].copy_(s64.view(torch.uint8), non_blocking=True)
        res_h[16:16 + 4 * ST_ITERS].copy_(res.view(torch.uint8), non_blocking=True)
        o = 16 + 4 * ST_ITERS
        res_h[o:o + 1024].copy_(bins.view(torch.uint8), non_blocking=True)
        res_h[o + 1024:o + 2048].copy_(scan.view(torch.uint8), non_blocking=True)

    with torch.cuda.stream(s):
        for _ in range(2):
            one()
        s.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s)
        for _ in range(steps):
            one()
        b.record(s)
        s.synchronize()
    ms = a.elapsed_time(b) / steps
    return {"value": round(STEP_BYTES / (ms * 1e-3) / 1e9, 2), "unit": "GB/s", "ms_per_step": round(ms, 4),
            "steps": steps, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["hx", "reference"], default="hx")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    rank, world, local = _dist_env()
    if args.impl == "reference":
        return bench_reference(args, rank, world)
    return bench_hx(args, rank, world, local)


if __name__ == "__main__":
    sys.exit(main())

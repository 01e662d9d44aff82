"""Seeded synthetic inputs for the fork-join hot path.

This module produces input buffers only.  It holds none of the arithmetic of
the loop nests themselves (no map, stencil, histogram or reduction), so the
CPU oracle and the CUDA path can both be fed from it without sharing any of
the method's code.

Random source
-------------
SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014; the 64-bit finaliser constants are Vigna's).  The
generator is counter based: the k-th output (k = 0, 1, ...) of the stream whose
state starts at ``seed`` is

    z = seed + (k + 1) * 0x9E3779B97F4A7C15            (mod 2^64)
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9
    z = (z ^ (z >> 27)) * 0x94D049BB133111EB
    out = z ^ (z >> 31)

so any element can be generated independently of the others.

Value recipes (one draw = one 64-bit output)
--------------------------------------------
* uniform fp32 on [0, 1):   k = draw >> 40 (24 bits), value = k * 2^-24
* uniform fp32 on [-1, 1):  value = (k - 2^23) * 2^-23  (a multiple of 2^-23)
* map->reduce inputs:       x[i] from draw 2i, y[i] from draw 2i+1
* histogram mixture (u8):   draws 3i, 3i+1, 3i+2 = (sel, a, b).  With
  p = (sel >> 11) * 2^-53, the element is a normal sample when p < 0.3:
  Box-Muller z = sqrt(-2 ln u1) cos(2 pi u2) with u1 = ((a >> 11) + 1) 2^-53,
  u2 = (b >> 11) 2^-53, value = clip(rint(128 + 20 z), 0, 255) (ties to even);
  otherwise the uniform byte a >> 56.

Every function has a numpy (host) form; the integer-only recipes also have a
torch form that runs on any device and yields the same bits, used to create
multi-GB inputs directly in device memory.
"""

from __future__ import annotations

import math

import numpy as np

GAMMA = 0x9E3779B97F4A7C15
MIX1 = 0xBF58476D1CE4E5B9
MIX2 = 0x94D049BB133111EB
MASK64 = (1 << 64) - 1

# Seeds of the five standard workloads (the map->reduce one is fixed at 0).
SEED_MAP_REDUCE = 0
SEED_STENCIL = 1
SEED_HISTOGRAM = 2
SEED_BATCH = 3
SEED_SERVING = 4
SEED_SRAD = 7

_CHUNK = 1 << 22


# ---------------------------------------------------------------- SplitMix64
def splitmix64(seed: int, counters: np.ndarray) -> np.ndarray:
    """k-th outputs of the SplitMix64 stream that starts at ``seed``."""
    k = np.asarray(counters, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & MASK64) + (k + np.uint64(1)) * np.uint64(GAMMA)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(MIX1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(MIX2)
    return z ^ (z >> np.uint64(31))


def splitmix64_scalar(seed: int, k: int) -> int:
    """Python-int form of one output (used for per-instance seeds and sizes)."""
    z = (seed + (k + 1) * GAMMA) & MASK64
    z = ((z ^ (z >> 30)) * MIX1) & MASK64
    z = ((z ^ (z >> 27)) * MIX2) & MASK64
    return z ^ (z >> 31)


def _s64(c: int) -> int:
    """A uint64 constant as the int64 with the same bits."""
    return c - (1 << 64) if c >= (1 << 63) else c


def _srl(t, s: int):
    """Logical right shift of an int64 torch tensor."""
    return (t >> s) & ((1 << (64 - s)) - 1)


def splitmix64_torch(seed: int, counters):
    """Same bits as :func:`splitmix64`, on int64 torch tensors (any device)."""
    z = counters + 1
    z = z * _s64(GAMMA) + _s64(seed & MASK64)
    z = (z ^ _srl(z, 30)) * _s64(MIX1)
    z = (z ^ _srl(z, 27)) * _s64(MIX2)
    return z ^ _srl(z, 31)


# ------------------------------------------------------------ value recipes
def _unit24(draws: np.ndarray) -> np.ndarray:
    return (draws >> np.uint64(40)).astype(np.int64)


def uniform01_f32(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """n fp32 values on the 2^-24 lattice of [0, 1)."""
    out = np.empty(n, dtype=np.float32)
    for s in range(0, n, _CHUNK):
        e = min(n, s + _CHUNK)
        k = _unit24(splitmix64(seed, np.arange(offset + s, offset + e, dtype=np.uint64)))
        out[s:e] = k.astype(np.float32) * np.float32(2.0**-24)
    return out


def uniform_pm1_f32(seed: int, n: int, stride: int = 1, phase: int = 0) -> np.ndarray:
    """n fp32 values on the 2^-23 lattice of [-1, 1); element i uses draw stride*i+phase."""
    out = np.empty(n, dtype=np.float32)
    for s in range(0, n, _CHUNK):
        e = min(n, s + _CHUNK)
        cnt = np.arange(s, e, dtype=np.uint64) * np.uint64(stride) + np.uint64(phase)
        k = _unit24(splitmix64(seed, cnt)) - (1 << 23)
        out[s:e] = k.astype(np.float32) * np.float32(2.0**-23)
    return out


def map_reduce_inputs(n: int, seed: int = SEED_MAP_REDUCE):
    """x, y of a map->reduce instance: x[i] from draw 2i, y[i] from draw 2i+1."""
    return uniform_pm1_f32(seed, n, 2, 0), uniform_pm1_f32(seed, n, 2, 1)


def stencil_grid(ny: int, nx: int, seed: int = SEED_STENCIL) -> np.ndarray:
    """Row-major ny x nx grid, uniform on [0, 1)."""
    return uniform01_f32(seed, ny * nx).reshape(ny, nx)


def srad_image(ny: int, nx: int, seed: int = SEED_SRAD) -> np.ndarray:
    """Positive fp32 intensity image exp(u), u uniform on [0, 1) (values in
    [1, e)): the exponentiated-image input of SRAD-style diffusion.  exp is
    taken in double and rounded to fp32 once."""
    u = uniform01_f32(seed, ny * nx).astype(np.float64)
    return np.exp(u).astype(np.float32).reshape(ny, nx)


def histogram_mixture_u8(n: int, seed: int = SEED_HISTOGRAM) -> np.ndarray:
    """n bytes: 70% uniform 0..255, 30% rint(normal(128, 20)) clipped to 0..255."""
    out = np.empty(n, dtype=np.uint8)
    for s in range(0, n, _CHUNK):
        e = min(n, s + _CHUNK)
        i3 = np.arange(s, e, dtype=np.uint64) * np.uint64(3)
        sel = splitmix64(seed, i3)
        a = splitmix64(seed, i3 + np.uint64(1))
        b = splitmix64(seed, i3 + np.uint64(2))
        p = (sel >> np.uint64(11)).astype(np.float64) * 2.0**-53
        u1 = ((a >> np.uint64(11)).astype(np.float64) + 1.0) * 2.0**-53
        u2 = (b >> np.uint64(11)).astype(np.float64) * 2.0**-53
        z = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)
        normal = np.clip(np.rint(128.0 + 20.0 * z), 0, 255).astype(np.uint8)
        uni = (a >> np.uint64(56)).astype(np.uint8)
        out[s:e] = np.where(p < 0.3, normal, uni)
    return out


# -------------------------------------------------------------- torch forms
def uniform_pm1_f32_torch(seed: int, n: int, device, stride: int = 1, phase: int = 0):
    """Torch form of :func:`uniform_pm1_f32` (identical bits), built on ``device``."""
    import torch

    out = torch.empty(n, dtype=torch.float32, device=device)
    chunk = 1 << 24
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        cnt = torch.arange(s, e, dtype=torch.int64, device=device) * stride + phase
        k = _srl(splitmix64_torch(seed, cnt), 40) - (1 << 23)
        out[s:e] = k.to(torch.float32) * (2.0**-23)
    return out


def uniform01_f32_torch(seed: int, n: int, device, offset: int = 0):
    """Torch form of :func:`uniform01_f32` (identical bits), built on ``device``."""
    import torch

    out = torch.empty(n, dtype=torch.float32, device=device)
    chunk = 1 << 24
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        cnt = torch.arange(offset + s, offset + e, dtype=torch.int64, device=device)
        k = _srl(splitmix64_torch(seed, cnt), 40)
        out[s:e] = k.to(torch.float32) * (2.0**-24)
    return out


# ------------------------------------------------- batched / serving mixes
def log_uniform_int(seed: int, k: int, lo: int, hi: int) -> int:
    """Integer in [lo, hi], log-uniform, from draw k of the stream ``seed``."""
    u = (splitmix64_scalar(seed, k) >> 11) * 2.0**-53
    v = int(math.floor(math.exp(math.log(lo) + u * (math.log(hi + 1) - math.log(lo)))))
    return max(lo, min(hi, v))


def batch_mix(count: int = 512, seed: int = SEED_BATCH, lo: int = 1 << 10, hi: int = 1 << 22,
              side_lo: int = 32, side_hi: int = 2048, iters: int = 1):
    """Instance list of the batched workload: half map->reduce, half stencil.

    Instance j uses draws 4j..4j+3 of the stream ``seed``: draw 4j picks the
    kind (stencil when its top bit is set), draw 4j+1 the size (log-uniform
    element count for a map->reduce, log-uniform side for a square stencil),
    draw 4j+2 gives the instance's own data seed.  Every instance's values
    are fp32 uniform on [-1, 1) (the batched workload's stated range): map
    inputs as ``map_reduce_inputs``, stencil grids as ``uniform_pm1_f32``
    (``"values": "pm1"``).  ``iters`` is the stencil sweep count.
    """
    out = []
    for j in range(count):
        kind = "stencil" if (splitmix64_scalar(seed, 4 * j) >> 63) else "map_reduce"
        data_seed = splitmix64_scalar(seed, 4 * j + 2)
        if kind == "map_reduce":
            out.append({"kind": kind, "n": log_uniform_int(seed, 4 * j + 1, lo, hi),
                        "seed": data_seed, "a": 1.5})
        else:
            side = log_uniform_int(seed, 4 * j + 1, side_lo, side_hi)
            out.append({"kind": kind, "nx": side, "ny": side, "iters": iters, "seed": data_seed, "values": "pm1"})
    return out


def serving_trace(count: int, rate_per_s: float, seed: int = SEED_SERVING,
                  lo: int = 1 << 10, hi: int = 1 << 24, stencil_iters: int = 20):
    """Open-loop Poisson request trace mixing the three nest kinds (1/3 each).

    Request j uses draws 4j..4j+3: exponential inter-arrival gap (draw 4j),
    kind (draw 4j+1, uniform over 3), log-uniform element count (draw 4j+2),
    data seed (draw 4j+3).  Stencil requests are square with side ~ sqrt(n).
    """
    t = 0.0
    out = []
    for j in range(count):
        u = ((splitmix64_scalar(seed, 4 * j) >> 11) + 1) * 2.0**-53
        t += -math.log(u) / rate_per_s
        kind_draw = splitmix64_scalar(seed, 4 * j + 1)
        kind = ("map_reduce", "stencil", "histogram")[(kind_draw >> 11) * 3 >> 53]
        n = log_uniform_int(seed, 4 * j + 2, lo, hi)
        req = {"kind": kind, "arrival_s": t, "seed": splitmix64_scalar(seed, 4 * j + 3)}
        if kind == "stencil":
            side = max(1, int(math.isqrt(n)))
            req.update(nx=side, ny=side, iters=stencil_iters)
        elif kind == "map_reduce":
            req.update(n=n, a=1.5)
        else:
            req.update(n=n)
        out.append(req)
    return out

"""The seeded input generator: known answers, backend identity, value recipes."""

import numpy as np
import torch

import workloads


def test_splitmix64_known_answer():
    # Published SplitMix64 outputs for state 0.
    got = workloads.splitmix64(0, np.arange(4, dtype=np.uint64))
    assert [int(v) for v in got] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4,
                                      0x06C45D188009454F, 0xF88BB8A8724C81EC]
    assert workloads.splitmix64_scalar(0, 1) == 0x6E789E6AA1B965F4


def test_splitmix64_torch_matches_numpy():
    k = np.arange(0, 5000, 7, dtype=np.uint64)
    for seed in (0, 1, 2**63 + 5, 2**64 - 1):
        a = workloads.splitmix64(seed, k).view(np.int64)
        b = workloads.splitmix64_torch(seed, torch.from_numpy(k.astype(np.int64))).numpy()
        assert np.array_equal(a, b)


def test_uniform_recipes_torch_identical():
    n = 10007
    a = workloads.uniform_pm1_f32(5, n, 2, 1)
    b = workloads.uniform_pm1_f32_torch(5, n, "cpu", 2, 1).numpy()
    assert np.array_equal(a.view(np.uint32), b.view(np.uint32))
    a = workloads.uniform01_f32(9, n, offset=3)
    b = workloads.uniform01_f32_torch(9, n, "cpu", offset=3).numpy()
    assert np.array_equal(a.view(np.uint32), b.view(np.uint32))


def test_uniform_lattice_and_range():
    x, y = workloads.map_reduce_inputs(1 << 16)
    for v in (x, y):
        assert v.min() >= -1.0 and v.max() < 1.0
        k = v.astype(np.float64) * 2**23
        assert np.array_equal(k, np.round(k))
        assert abs(float(v.mean())) < 0.02
    u = workloads.uniform01_f32(1, 1 << 16)
    assert u.min() >= 0.0 and u.max() < 1.0
    k = u.astype(np.float64) * 2**24
    assert np.array_equal(k, np.round(k))
    # x and y are different streams of the same seed
    assert not np.array_equal(x, y)


def test_histogram_mixture_shape():
    v = workloads.histogram_mixture_u8(1 << 20)
    counts = np.bincount(v, minlength=256)
    assert counts.sum() == 1 << 20
    # 30% of the mass is normal(128, 20): the 108..148 band holds about
    # 0.3*0.6827 + 0.7*41/256 of the elements.
    band = counts[108:149].sum() / v.size
    assert abs(band - (0.3 * 0.6827 + 0.7 * 41 / 256)) < 0.01
    # the tails far from 128 are close to the uniform 0.7/256 level
    assert abs(counts[:40].mean() / v.size - 0.7 / 256) < 3e-4
    assert np.array_equal(v, workloads.histogram_mixture_u8(1 << 20))


def test_batch_mix_sizes():
    mix = workloads.batch_mix()
    assert len(mix) == 512
    kinds = [m["kind"] for m in mix]
    assert 200 < kinds.count("stencil") < 312
    for m in mix:
        if m["kind"] == "map_reduce":
            assert 1024 <= m["n"] <= 1 << 22
        else:
            assert 32 <= m["nx"] == m["ny"] <= 2048
    assert mix == workloads.batch_mix()


def test_serving_trace_poisson_rate():
    tr = workloads.serving_trace(4000, 10_000.0)
    t = np.array([r["arrival_s"] for r in tr])
    assert np.all(np.diff(t) > 0)
    assert abs(4000 / t[-1] - 10_000) < 600
    kinds = [r["kind"] for r in tr]
    for k in ("map_reduce", "stencil", "histogram"):
        assert 1100 < kinds.count(k) < 1570

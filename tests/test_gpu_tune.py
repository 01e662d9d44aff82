"""Tuned and non-default tables: parity with the oracle is kept, and a
standalone call and a batch planned on the same context still agree bit for
bit."""

import os
import subprocess
import sys

import numpy as np
import pytest
import torch

import oracle
import workloads
from tests.test_gpu_batch import Inst, _same

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _custom_table(hx, vecs, rows, threads):
    t = hx.hx_tune_table_default()
    for c in range(hx.HX_TUNE_CLASSES):
        t.map_vecs[c] = vecs
        t.stencil_rows[c] = rows
        t.hist_threads[c] = threads
    t.batch_map_run, t.batch_stencil_run = 3, 5
    return t


@pytest.mark.parametrize("vecs,rows,threads", [(8, 4, 256), (16, 16, 1024), (32, 8, 512)])
def test_non_default_table_parity_and_alone_equals_batch(gpu, vecs, rows, threads):
    hx = gpu
    with hx.hx_create(0) as ctx:
        hx.hx_tune_set(ctx, _custom_table(hx, vecs, rows, threads))
        specs = [{"kind": "map_reduce", "n": 3_000_001, "a": 1.5, "seed": 31},
                 {"kind": "map_reduce", "n": 70_001, "a": -0.75, "seed": 32},
                 {"kind": "stencil", "nx": 257, "ny": 130, "iters": 3, "seed": 33},
                 {"kind": "stencil", "nx": 512, "ny": 96, "iters": 2, "seed": 34},
                 {"kind": "histogram", "n": 1_000_003, "seed": 35}]
        insts = [Inst(s) for s in specs]
        b = hx.hx_batch_plan(ctx, [i.task(hx) for i in insts])
        b.launch()
        torch.cuda.synchronize()
        for inst in insts:
            r = inst.result()
            _same(r, inst.standalone(hx, ctx))
            inst.check_oracle(r)
        b.close()


def test_autotune_produces_valid_table_and_keeps_parity(gpu):
    hx = gpu
    with hx.hx_create(0) as ctx:
        t = hx.hx_autotune(ctx, 22)
        hx.hx_tune_table_check(t)
        for n in (1000, 1 << 18, (1 << 22) + 3):
            x, y = workloads.map_reduce_inputs(n, seed=n)
            out = torch.empty(n, device=DEV)
            s64 = torch.empty(1, dtype=torch.float64, device=DEV)
            hx.hx_map_reduce(ctx, torch.from_numpy(x).to(DEV), torch.from_numpy(y).to(DEV), 1.5, out=out,
                             sum64_out=s64)
            torch.cuda.synchronize()
            out_o, s_o = oracle.map_reduce(x, y, 1.5)
            assert np.array_equal(out.cpu().numpy(), out_o.astype(np.float32))
            assert abs(s64.item() - s_o) <= 1e-5 * np.abs(out_o).sum()
        v = workloads.histogram_mixture_u8(1 << 20, seed=3)
        bins, scan = hx.hx_histogram(ctx, torch.from_numpy(v).to(DEV))
        b_o, s_o = oracle.histogram(v)
        assert np.array_equal(bins.cpu().numpy().view(np.uint32), b_o)
        assert np.array_equal(scan.cpu().numpy().view(np.uint32), s_o)
        u0 = workloads.stencil_grid(300, 200, seed=4)
        g0 = torch.from_numpy(u0).to(DEV)
        fin, res = hx.hx_stencil2d(ctx, g0, torch.empty_like(g0), 3)
        u32, r32 = oracle.jacobi(u0, 3, "f32")
        assert np.array_equal(fin.cpu().numpy(), u32) and np.array_equal(res.cpu().numpy()[:3], r32)


def test_tune_file_env_is_loaded_at_create(gpu, tmp_path):
    hx = gpu
    t = _custom_table(hx, 12, 16, 1024)
    path = tmp_path / "tune.json"
    hx.hx_tune_table_save(t, str(path))
    code = ("import paper_2503_10855_b300 as hx, json, sys;"
            "c = hx.hx_create(0); print(json.dumps(hx.hx_tune_get(c).as_dict())); c.close()")
    env = dict(os.environ, HX_TUNE_FILE=str(path))
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, "-c", code], env=env, cwd=root, capture_output=True, text=True,
                         check=True).stdout
    import json

    assert json.loads(out.strip().splitlines()[-1]) == t.as_dict()

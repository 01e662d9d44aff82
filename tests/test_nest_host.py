"""Host side of the generic nests, without a GPU: descriptor validation, and
the generated kernels of every schedule compile for sm_103a (NVRTC runs on
the host)."""

import pytest
import torch

hx = pytest.importorskip("paper_2503_10855_b300")


def _nest(program=(("in", 0),), dims=(8, 16), rd=1, monoid="sum", **kw):
    x = kw.pop("x", torch.zeros(dims))
    res = torch.zeros(64)
    idx = torch.zeros(64, dtype=torch.int64)
    out = kw.pop("out", None)
    return hx.make_nest(list(program), [x], dims, rd, monoid, kw.pop("consts", ()), out=out, result=res,
                        result_index=idx, **kw)


BAD = {
    "ndim0": lambda n: setattr(n, "ndim", 0),
    "ndim4": lambda n: setattr(n, "ndim", 4),
    "reduce_dims_gt_ndim": lambda n: setattr(n, "reduce_dims", 3),
    "monoid": lambda n: setattr(n, "monoid", 6),
    "tree": lambda n: setattr(n, "tree", 3),
    "negative_dim": lambda n: n.dims.__setitem__(1, -1),
    "huge_fork": lambda n: (n.dims.__setitem__(0, 1 << 31), n.dims.__setitem__(1, 1 << 31)),
    "no_ops": lambda n: setattr(n, "n_ops", 0),
    "too_many_ops": lambda n: setattr(n, "n_ops", 33),
    "missing_input": lambda n: n.inputs.__setitem__(0, None),
    "misaligned_input": lambda n: n.inputs.__setitem__(0, n.inputs[0] + 2),
    "no_result": lambda n: setattr(n, "result", None),
    "argmax_without_index": lambda n: (setattr(n, "monoid", 4), setattr(n, "result_index", None)),
    "negative_chunk": lambda n: setattr(n, "chunk", -5),
    "map_only_without_out": lambda n: setattr(n, "reduce_dims", 0),
}


@pytest.mark.parametrize("name", sorted(BAD))
def test_invalid_descriptor_rejected(name):
    n = _nest()
    hx.hx_nest_prepare(n)
    BAD[name](n)
    with pytest.raises(hx.HxError) as e:
        hx.hx_nest_prepare(n)
    assert e.value.status == hx.HX_ERR_INVALID


@pytest.mark.parametrize("program", [
    ["add"], [("in", 0), ("in", 0)], [("in", 1)], [("const", 8)], [("index", 2)],
    [("in", 0)] * 9 + ["add"] * 8, [("in", 0), (99, 0)], [("in", 0), ("in", 0), "fma"],
])
def test_malformed_program_rejected(program):
    with pytest.raises(hx.HxError) as e:
        hx.hx_nest_prepare(_nest(program))
    assert e.value.status == hx.HX_ERR_INVALID


@pytest.mark.parametrize("tree", ["warp", "chunk", "seq"])
@pytest.mark.parametrize("monoid", ["sum", "max", "min", "prod", "argmax", "argmin"])
def test_every_schedule_compiles(tree, monoid):
    x3 = torch.zeros(4, 5, 6).permute(2, 0, 1)
    for dims, rd, x in (((8, 16), 1, torch.zeros(8, 16)), ((8, 3), 1, torch.zeros(8, 3)),
                        ((6, 4, 5), 2, x3), ((6, 4, 5), 3, x3), ((16, 8), 2, torch.zeros(8, 16).T)):
        n = _nest([("in", 0), ("index", len(dims) - 1), ("const", 0), "fma", "abs", "sqrt"], dims, rd, monoid,
                  x=x, tree=tree, out=torch.zeros(512))
        n.result64 = torch.zeros(64, dtype=torch.float64).data_ptr()
        hx.hx_nest_prepare(n)


def test_generated_source_fuses_the_program():
    x, y = torch.zeros(8, 16), torch.zeros(8, 16)
    n = hx.make_nest([("in", 0), ("const", 0), ("in", 1), "fma", ("in", 1), "max"], [x, y], (8, 16), 1, "sum",
                     result=torch.zeros(8))
    src = hx.hx_nest_source(n)
    assert "hx_maxnum(fmaf(hx_comp(b.x0[j], q), p.c[0], hx_comp(b.x1[j], q)), hx_comp(b.x1[j], q))" in src
    assert "return fmaf(x0, p.c[0], x1)" not in src            # the sequential form has its own expression
    assert "p.lin[0]" in src and "p.lin[1]" in src          # row-major rows are linear segments
    assert "#define VEC 1" in src                              # aligned unit-stride rows load float4
    # a transposed input over a full reduce does not collapse: per-dim offsets
    t = torch.zeros(16, 8).T
    src = hx.hx_nest_source(hx.make_nest([("in", 0)], [t], (8, 16), 2, "max", result=torch.zeros(1)))
    assert "p.lin[0]" not in src and "p.st[0][1]" in src and "hx_div(p, 1, rr)" in src
    assert "#define VEC 0" in src
    # short segments use sub-warp groups: one lane per 5-element row, four
    # lanes per 64-element row
    src = hx.hx_nest_source(hx.make_nest([("in", 0)], [torch.zeros(64, 5)], (64, 5), 1, "sum",
                                         result=torch.zeros(64)))
    assert "#define G 1" in src
    src = hx.hx_nest_source(hx.make_nest([("in", 0)], [torch.zeros(8, 64)], (8, 64), 1, "sum",
                                         result=torch.zeros(8)))
    assert "#define G 4" in src

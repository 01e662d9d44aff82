"""The tuning table's host-side functions: defaults, validation, JSON round trip."""

import json

import pytest

import paper_2503_10855_b300 as hx


def test_default_table_is_valid():
    t = hx.hx_tune_table_default()
    hx.hx_tune_table_check(t)
    d = t.as_dict()
    assert len(d["map_vecs"]) == hx.HX_TUNE_CLASSES
    assert set(d["hist_threads"]) <= {256, 512, 1024}
    assert set(d["stencil_rows"]) <= {4, 8, 16}
    assert all(v % 4 == 0 for v in d["map_vecs"])
    assert all(v % 8 == 0 and 8 <= v <= 512 for v in d["nest_lane_elems"])


def test_json_round_trip(tmp_path):
    t = hx.hx_tune_table_default()
    for c in range(hx.HX_TUNE_CLASSES):
        t.map_vecs[c] = 4 * (1 + c % 4)
        t.hist_threads[c] = (256, 512, 1024)[c % 3]
        t.stencil_rows[c] = (4, 8, 16)[c % 3]
        t.nest_lane_elems[c] = 8 * (1 + c % 5)
    t.batch_map_run, t.batch_stencil_run = 5, 33
    path = tmp_path / "tune.json"
    hx.hx_tune_table_save(t, str(path))
    doc = json.loads(path.read_text())          # valid JSON
    assert doc["format"] == "hx_tune_table/1" and doc["batch_stencil_run"] == 33
    u = hx.hx_tune_table_load(str(path))
    assert u.as_dict() == t.as_dict()


@pytest.mark.parametrize("field,value", [("map_vecs", 6), ("hist_threads", 300), ("stencil_rows", 5),
                                         ("nest_lane_elems", 12), ("nest_lane_elems", 1024)])
def test_invalid_entries_rejected(tmp_path, field, value):
    t = hx.hx_tune_table_default()
    getattr(t, field)[3] = value
    with pytest.raises(hx.HxError):
        hx.hx_tune_table_check(t)
    with pytest.raises(hx.HxError):
        hx.hx_tune_table_save(t, str(tmp_path / "x.json"))
    good = hx.hx_tune_table_default()
    path = tmp_path / "y.json"
    hx.hx_tune_table_save(good, str(path))
    doc = json.loads(path.read_text())
    doc[field][3] = value
    path.write_text(json.dumps(doc))
    with pytest.raises(hx.HxError):
        hx.hx_tune_table_load(str(path))


def test_load_missing_or_truncated(tmp_path):
    with pytest.raises(hx.HxError):
        hx.hx_tune_table_load(str(tmp_path / "absent.json"))
    p = tmp_path / "short.json"
    p.write_text('{"map_vecs": [4, 4]}')
    with pytest.raises(hx.HxError):
        hx.hx_tune_table_load(str(p))

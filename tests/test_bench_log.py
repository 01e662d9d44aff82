"""The bench's JSON-lines log: one row per measurement of a bench line."""

import json

import bench


def _line():
    return {
        "n_gpus": 1, "ms_per_step": 0.5, "value": 6400.0, "frac_of_hbm_roofline": 0.84,
        "algorithmic_frac_of_hbm_roofline": 0.98,
        "clocks": {"sm_mhz": 2032.0}, "roofline": {"peak": 6508.2},
        "kernels": {"batch": {"ms": 0.4, "algorithmic_bytes": 2_400_000_000, "GB/s": 6000.0,
                              "frac_of_measured_hbm": 0.92}},
        "sweeps": {"jacobi_x20": [{"grid": "8192^2", "ms": 1.6, "algorithmic_GB/s": 6700.0,
                                   "frac_of_measured_hbm": 1.03}]},
        "nests": {"workloads": [{"nest": "sum", "ms": 0.17, "algorithmic_bytes": 1 << 30, "GB/s": 6200.0,
                                 "frac_of_measured_hbm": 0.95}]},
        "serving": {"points": [{"offered_req_per_s": 2000,
                                "continuous": {"req_per_s": 2100.0, "p50_ms": 0.2, "p99_ms": 1.2, "stable": True},
                                "per_launch": {"req_per_s": 2100.0, "p50_ms": 0.3, "p99_ms": 2.0, "stable": True}}]},
        "e2e": {"ms_per_step": 28.0, "value": 113.0},
    }


def test_rows_cover_every_measurement():
    rows = bench.log_rows(_line())
    kinds = [r["kind"] for r in rows]
    assert kinds == ["step", "kernel", "sweep", "nest", "serving", "serving", "e2e"]
    assert all(r["host_cores"] >= 1 and r["peak_gbs"] == 6508.2 for r in rows)
    assert rows[2]["gbs"] == 6700.0 and rows[2]["size"] == "8192^2"
    assert abs(rows[1]["frac_nominal"] - 0.75) < 1e-12


def test_log_appends_json_lines(tmp_path):
    p = tmp_path / "runs.jsonl"
    bench.append_log(str(p), _line())
    bench.append_log(str(p), _line())
    lines = p.read_text().splitlines()
    assert len(lines) == 14 and all(json.loads(s)["n_gpus"] == 1 for s in lines)


def test_sections_may_be_skipped():
    line = _line()
    line.update(sweeps=None, nests=None, serving=None, e2e=None)
    assert [r["kind"] for r in bench.log_rows(line)] == ["step", "kernel"]

"""The serving sweep's equal-p99 comparison (host logic of bench.py).

The points are a recorded sweep's (offered rate, sustained rate, p99,
stable) per mode; the expected figures are worked out by hand from the
rule: the bound is the per-launch server's p99 at the highest rate at which
it is stable, and each mode is credited with the highest stable rate whose
p99 is within the bound (or within a fixed target)."""

import bench

# offered rate: (continuous req/s, p99 ms, stable), (per-launch req/s, p99 ms, stable)
SWEEP = {
    2000: ((2143.1, 1.267, True), (2146.2, 0.5992, True)),
    5000: ((5292.8, 1.3512, True), (5292.9, 0.619, True)),
    10000: ((10354.7, 1.4278, True), (9842.0, 21.2456, False)),
    12000: ((12372.5, 1.7892, True), (12378.3, 3.9584, True)),
    15000: ((15220.5, 1.9776, True), (14779.5, 15.4167, True)),
    20000: ((20141.6, 8.571, True), (20252.4, 1.3875, True)),
    30000: ((29891.2, 5.5995, True), (19227.9, 76.2599, False)),
    40000: ((38758.1, 10.4785, True), (19924.2, 101.4966, False)),
    50000: ((43878.3, 21.3721, False), (19214.6, 128.3916, False)),
}


def _points(sweep):
    pts = []
    for lam, (c, pl) in sweep.items():
        pts.append({"offered_req_per_s": lam,
                    "continuous": {"req_per_s": c[0], "p99_ms": c[1], "stable": c[2]},
                    "per_launch": {"req_per_s": pl[0], "p99_ms": pl[1], "stable": pl[2]}})
    return pts


def test_bound_is_per_launch_p99_at_its_highest_stable_rate():
    eq = bench.serving_comparison(_points(SWEEP))
    # per-launch is stable up to 20k (10k is not), p99 1.3875 ms there
    assert eq["p99_bound_ms"] == 1.3875
    # continuous within 1.3875 ms: 2k (1.267) and 5k (1.3512); 10k is 1.4278
    assert eq["continuous_req_per_s"] == 5292.8
    # per-launch within the bound at its own highest stable rate
    assert eq["per_launch_req_per_s"] == 20252.4
    assert eq["ratio"] == round(5292.8 / 20252.4, 3)


def test_fixed_targets():
    eq = bench.serving_comparison(_points(SWEEP))
    got = {r["p99_ms"]: (r["continuous_req_per_s"], r["per_launch_req_per_s"]) for r in eq["at_p99_targets"]}
    assert got == {2.0: (15220.5, 20252.4), 5.0: (15220.5, 20252.4), 10.0: (29891.2, 20252.4),
                   20.0: (38758.1, 20252.4)}
    ratios = [r["ratio"] for r in eq["at_p99_targets"]]
    assert ratios == [0.752, 0.752, 1.476, 1.914]


def test_no_stable_per_launch_point_and_unmet_targets():
    sweep = {lam: (c, (pl[0], pl[1], False)) for lam, (c, pl) in SWEEP.items()}
    eq = bench.serving_comparison(_points(sweep))
    # no stable per-launch rate: no bound and no ratio, flagged
    assert eq["p99_bound_ms"] is None and eq["ratio"] is None
    assert eq["per_launch_req_per_s"] is None and eq["continuous_req_per_s"] is None
    assert eq["per_launch_never_stable"] is True
    for row in eq["at_p99_targets"]:
        assert row["per_launch_req_per_s"] is None and "ratio" not in row


def test_timeline_summary_by_hand():
    # steps [0, 1] (batched, 3 requests), [0.5, 1.5] (direct), [2, 3]
    # (batched, 5 requests): in flight 1, 2, 1, 0, 1 over 0.5, 0.5, 0.5,
    # 0.5, 1 s -> mean 3 / 3 s = 1, max 2
    tl = [{"issue_s": 0.0, "done_s": 1.0, "requests": 3, "direct": False},
          {"issue_s": 0.5, "done_s": 1.5, "requests": 1, "direct": True},
          {"issue_s": 2.0, "done_s": 3.0, "requests": 5, "direct": False}]
    s = bench.timeline_summary(tl)
    assert s == {"steps": 3, "direct_share": 0.333, "requests_per_batched_step": 4.0, "step_ms_mean": 1000.0,
                 "steps_in_flight_mean": 1.0, "steps_in_flight_max": 2}
    assert bench.timeline_summary([]) == {"steps": 0}

"""Pins the control-plane oracle (oracle/control.py) to the paper's constants,
closed forms of Eqs. 6-8, hand-derived runs of Alg. 1 and Alg. 2, least squares
(Eq. 9) against numpy.linalg.lstsq, and the qualitative scenario of Fig. 4."""
import json
import os

import numpy as np
import pytest

from oracle import control as oc

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table2_base_costs.json")


def test_table2_constants():
    g = json.load(open(GOLDEN))
    assert oc.BASE_COST == g["base_cost"]
    assert oc.BASE_TRANS_COST == g["base_trans_cost"]
    assert oc.INFPT0_BYTES == g["infpt0_bytes"]
    assert oc.POLL_MS == g["poll_ms"]


def test_eqs_6_to_8_closed_forms():
    # at Part == InfPT both devices cost baseCost
    for op, b in oc.BASE_COST.items():
        cpu, gpu, trans = oc.device_costs(op, 1000.0, 1000.0)
        assert cpu == pytest.approx(b) and gpu == pytest.approx(b) and trans == pytest.approx(0.1)
    # filter, partition 15 KB, InfPT 150 KB: CPU 0.1, GPU 10, Trans 0.01
    cpu, gpu, trans = oc.device_costs("filter", 15 * 1024, 150 * 1024)
    assert (cpu, gpu, trans) == pytest.approx((0.1, 10.0, 0.01))


def test_alg2_small_and_large_partitions():
    ops = ["scan", "filter", "project", "aggregation"]
    small = oc.map_device(ops, 12 * 15 * 1024, 12, 150 * 1024)  # Part = 15 KB
    assert [p[0] for p in small] == ["CPU"] * 4
    large = oc.map_device(ops, 12 * 1500 * 1024, 12, 150 * 1024)  # Part = 10 x InfPT
    assert [p[0] for p in large] == ["GPU"] * 4
    # leaf: GPU 0.08 + Trans 1.0 = 1.08 < CPU 8 ; middle ops carry Trans on the CPU side
    assert large[0][1:] == pytest.approx((8.0, 1.08))
    assert large[1][1:] == pytest.approx((11.0, 0.1))


def test_alg2_mixed_plan_hand_derived():
    # r = Part/InfPT = 1.06: filter (leaf) GPU 1/1.06+0.106 < CPU 1.06; project
    # (middle, previous on GPU) CPU 0.954+0.106 > GPU 0.849; sort (root)
    # GPU 0.8/1.06+0.106 = 0.8607 > CPU 0.848 -> CPU.
    infpt = 100_000.0
    plan = oc.map_device(["filter", "project", "sort"], 1.06 * infpt * 4, 4, infpt)
    assert [p[0] for p in plan] == ["GPU", "GPU", "CPU"]
    assert plan[2][1] == pytest.approx(0.848)
    assert plan[2][2] == pytest.approx(0.8 / 1.06 + 0.106)


def test_eq9_recovers_exact_coefficients_and_matches_lstsq():
    rng = np.random.default_rng(3)
    thp = rng.uniform(1e3, 1e6, 40)
    lat = rng.uniform(5, 500, 40)
    y = 3.0 + 2e-3 * thp + 5.0 * lat
    beta, pred = oc.regress_infpt(thp, lat, y, 2e5, 100.0)
    np.testing.assert_allclose(beta, [3.0, 2e-3, 5.0], rtol=1e-6)
    assert pred == pytest.approx(3.0 + 2e-3 * 2e5 + 500.0, rel=1e-9)
    noisy = y + rng.normal(0, 50, 40)
    beta, _ = oc.regress_infpt(thp, lat, noisy, 0, 0)
    X = np.column_stack([np.ones(40), thp, lat])
    ref = np.linalg.lstsq(X, noisy, rcond=None)[0]
    np.testing.assert_allclose(beta, ref, rtol=1e-6)


@pytest.mark.parametrize("case", [
    # n = 2 (fewer than the three samples the three coefficients need)
    dict(t=[1.0e5, 2.0e5], l=[30.0, 50.0], y=[100.0, 200.0], mean=150.0),
    # constant throughput column: its coefficient is not identifiable
    dict(t=[5.0e4] * 4, l=[10.0, 20.0, 30.0, 40.0], y=[10.0, 20.0, 30.0, 45.0], mean=26.25),
    # constant latency column
    dict(t=[1.0, 2.0, 3.0, 4.0, 5.0], l=[7.0] * 5, y=[3.0, 1.0, 4.0, 1.0, 5.0], mean=2.8),
    # exactly collinear inputs: latency = 2 * throughput + 1
    dict(t=[1.0, 2.0, 3.0, 4.0], l=[3.0, 5.0, 7.0, 9.0], y=[8.0, 6.0, 7.0, 5.0], mean=6.5),
])
def test_eq9_degenerate_inputs_fall_back_to_the_mean(case):
    # Eq. 9 (Section III-E) needs three identifiable coefficients; with fewer
    # than three samples, a constant input or collinear inputs the system is
    # singular, and the reading used here answers with the intercept-only
    # least-squares fit: b = (mean InfPT, 0, 0), whatever the targets.
    for target in [(0.0, 0.0), (3.0e5, 100.0)]:
        beta, pred = oc.regress_infpt(case["t"], case["l"], case["y"], *target)
        np.testing.assert_array_equal(beta, [case["mean"], 0.0, 0.0])
        assert pred == case["mean"]
    # the intercept-only fit is what least squares gives on a column of ones
    ones = np.ones((len(case["y"]), 1))
    ref = np.linalg.lstsq(ones, np.asarray(case["y"]), rcond=None)[0][0]
    assert ref == pytest.approx(case["mean"], rel=1e-15)


def test_eq9_without_history_uses_the_initial_inflection_point():
    beta, pred = oc.regress_infpt([], [], [], 1e5, 100.0)
    np.testing.assert_array_equal(beta, [oc.INFPT0_BYTES, 0.0, 0.0])
    assert pred == oc.INFPT0_BYTES == 150 * 1024


def test_eqs_3_4_5_closed_forms():
    assert oc.avg_thput([1000, 3000], [100, 100]) == 20.0
    assert oc.max_lat([5, 30, 12], 7) == 37
    assert oc.est_max_lat([5, 30, 12], [1000, 1000, 2000], 20.0) == 30 + 200


def test_alg1_hand_built_states():
    a = oc.Admission(slide_ms=3000.0)
    assert not a.poll(0.0, [])  # no data: nothing to do
    assert a.poll(10.0, [oc.Dataset(0.0, 1000.0)])  # first batch: admitted
    assert a.complete(100.0) == 10.0 + 100.0  # MaxLat = buffering 10 + Proc 100
    # AvgThPut = 1000 B / 100 ms = 10 B/ms
    assert not a.poll(5000.0, [oc.Dataset(4000.0, 1000.0), oc.Dataset(4990.0, 1000.0)])
    assert a.last_est == pytest.approx(1000.0 + 2000.0 / 10.0)
    assert not a.poll(6000.0, [])  # "paper" policy: no new data, no decision
    assert a.poll(6900.0, [oc.Dataset(6890.0, 0.0)])  # 2900 + 2000/10 = 3100 >= 3000
    assert len(a.admitted) == 3
    # tumbling target = mean of past MaxLat
    t = oc.Admission(slide_ms=0.0)
    t.poll(0.0, [oc.Dataset(0.0, 100.0)])
    t.complete(50.0)  # MaxLat 50, AvgThPut 2 B/ms
    assert not t.poll(20.0, [oc.Dataset(0.0, 10.0)])  # 20 + 5 = 25 < 50
    assert t.poll(46.0, [oc.Dataset(40.0, 10.0)])  # 46 + 10 = 56 >= 50


def _simulate(policy, slide_ms=3000.0, trigger_ms=5000.0, horizon_ms=300_000.0):
    """Fig. 4 set-up: one dataset per second; Proc(n datasets) = 500 + 300 n ms."""
    proc = lambda n: 500.0 + 300.0 * n
    arrivals = list(np.arange(0.0, horizon_ms, 1000.0))
    maxlats = []
    if policy == "trigger":
        t, k = 0.0, 0
        while t < horizon_ms:
            t_next = t + trigger_ms
            batch = []
            while k < len(arrivals) and arrivals[k] <= t_next:
                batch.append(arrivals[k]); k += 1
            start = t_next
            if batch:
                p = proc(len(batch))
                maxlats.append(start - batch[0] + p)
                t = max(t_next, start + p - trigger_ms)
            else:
                t = t_next
        return maxlats
    a = oc.Admission(slide_ms=slide_ms, policy="guarded")
    t, k, busy_until = 0.0, 0, 0.0
    while t < horizon_ms:
        new = []
        while k < len(arrivals) and arrivals[k] <= t:
            new.append(oc.Dataset(arrivals[k], 1.0)); k += 1
        if t < busy_until:
            a.buffered.extend(new)  # arrivals wait while a batch is processed
        elif a.poll(t, new):
            p = proc(len(a.admitted))
            maxlats.append(a.complete(p))
            busy_until = t + p
        t += oc.POLL_MS
    return maxlats


def test_fig4_scenario_slide_time_bounds_latency():
    """Qualitative only (the figure's numbers are not in the text): with a 5 s
    trigger every micro-batch's MaxLat exceeds the 3 s slide; with Alg. 1 every
    one after the first stays below it."""
    trig = _simulate("trigger")
    lm = _simulate("lmstream")
    assert len(trig) > 10 and min(trig) > 3000.0
    assert len(lm) > 10 and max(lm) < 3000.0


def test_variant_choice_threshold_of_alg2_on_one_operation():
    """One Aggregation (base cost 1) with r = Part / InfPT: Eq. 6 gives r for
    variant 1, Eq. 7 1/r for variant 2, and Eq. 8's transition 0.1 r is charged
    to variant 2 (the chain's first operation): variant 1 iff 1/r + 0.1 r > r,
    i.e. r < sqrt(1 / 0.9)."""
    infpt, parts, bpr = 150 * 1024, 148, 16.0
    v = oc.VariantAnalytic(parts, bpr, infpt, explore=0)
    r_star = np.sqrt(1 / 0.9)
    for r in (0.01, 0.5, 1.0, 1.05, 1.06, 2.0, 50.0):
        rows = int(round(r * infpt * parts / bpr))
        r_act = rows * bpr / parts / infpt
        assert v.choose(rows) == (1 if r_act < r_star else 2), r


def test_variant_crossover_of_exact_power_laws():
    """Exact costs ms_v = c_v rows^b_v: the fits are exact, the observed
    inflection point is their crossing (c1/c2)^(1/(b2 - b1)) rows, and Eq. 9 on a
    constant target returns it."""
    parts, bpr = 148, 16.0
    c1, b1, c2, b2 = 2e-6, 1.0, 4e-3, 0.55
    cross = (c1 / c2) ** (1.0 / (b2 - b1))  # ~2.2e7 rows
    v = oc.VariantAnalytic(parts, bpr, explore=2)
    # the extreme sizes first, so that every fit's range holds the crossing
    for rows in [1 << 20, 1 << 26, 1 << 22, 1 << 24, 3 << 20, 5 << 22]:
        for var, c, b in ((1, c1, b1), (2, c2, b2)):
            v.observe(rows, var, c * rows ** b)
    assert v.infpt == pytest.approx(cross * bpr / parts, rel=1e-9)
    assert v.predict(1 << 23, 2) == pytest.approx(c2 * (1 << 23) ** b2, rel=1e-9)
    # below the crossing variant 1 is cheaper, above it variant 2
    assert v.choose(int(cross / 4)) == 1 and v.choose(int(cross * 4)) == 2


def test_variant_without_crossing_takes_the_far_end():
    """Variant 1 cheaper at every size seen: the observed inflection point is
    twice the largest size seen so far (Eq. 9 over the last sample only, so the
    inflection point is that sample), and variant 1 stays chosen."""
    parts, bpr = 148, 16.0
    v = oc.VariantAnalytic(parts, bpr, explore=2, history=1)
    sizes = [1 << 16, 1 << 18, 1 << 20]
    for rows in sizes:
        v.observe(rows, 1, 1e-6 * rows)
        v.observe(rows, 2, 3e-6 * rows)
    assert v.infpt == pytest.approx(2 * max(sizes) * bpr / parts, rel=1e-9)
    assert all(v.choose(r) == 1 for r in sizes)

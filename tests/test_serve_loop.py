"""The serving loop (dynamic micro-batching on a virtual clock).

* The plain oracle (oracle/serve.py) is pinned by closed forms: a fixed
  trigger over a constant arrival rate, a fixed batch size, Alg. 1 with an
  exact processing-time model (every batch's MaxLat stays within the bound),
  conservation of events and the memory cap.
* The engine's loop (lms_serve_run, C++) is compared with the oracle batch by
  batch and on the latency quantiles, for every policy, on random arrivals with
  a deterministic fake backend (host code only: no GPU)."""
import math

import numpy as np
import pytest

from oracle import serve as osv
from paper_2111_04289_b300 import lmstream as lm


def fake_proc(a=2.0, b=1e-4, c=0.0):
    def proc(pieces_or_chunks, n, rec=None):
        return a + b * n + c * math.sqrt(n)
    return proc


# ---------------------------------------------------------------- oracle pins

def test_oracle_fixed_trigger_closed_form():
    """Constant n events per 10-ms tick, trigger every 50 ms, proc p < 50: every
    batch holds the 5n events of [t-50, t) and the latencies are
    50 + p - (m + 0.5) * 10/n, m = 0..5n-1, in every batch."""
    n, p, batches = 7, 3.0, 12
    ticks = np.full(5 * batches, n)
    res, log, lat = osv.run(ticks, poll_ms=10.0, policy=osv.FIXED_TRIGGER, bound_ms=100.0,
                            trigger_ms=50.0, process=lambda b, k: p)
    assert res["batches"] == batches and res["processed"] == ticks.sum()
    assert all(r.n_events == 5 * n for r in log)
    assert [r.admit_ms for r in log] == pytest.approx([50.0 * (i + 1) for i in range(batches)])
    for q in (0.5, 0.99):
        k = math.ceil(q * 5 * n * batches)
        r = math.ceil(k / batches)  # r-th smallest distinct latency
        expect = 50.0 + p - (5 * n - r + 0.5) * 10.0 / n
        assert osv.kth_smallest(lat, q) == pytest.approx(expect, rel=1e-12)
    assert res["max"] == pytest.approx(50.0 + p - 0.5 * 10.0 / n)


def test_oracle_fixed_size_closed_form():
    """n events per tick and N = 3n: a batch forms at every third tick end and
    waits for nothing else; latencies are 30 + p - (m + 0.5) * 10/n."""
    n, p = 4, 1.5
    ticks = np.full(30, n)
    res, log, lat = osv.run(ticks, poll_ms=10.0, policy=osv.FIXED_SIZE, bound_ms=100.0,
                            fixed_rows=3 * n, process=lambda b, k: p)
    assert len(log) == 10 and all(r.n_events == 3 * n for r in log)
    assert [r.admit_ms for r in log] == pytest.approx([30.0 * (i + 1) for i in range(10)])
    expect = np.sort(np.tile(30.0 + p - (np.arange(3 * n) + 0.5) * 10.0 / n, 10))
    assert np.allclose(np.sort(lat), expect, rtol=0, atol=1e-12)


def test_oracle_fixed_size_splits_ticks():
    """A batch size that is not a multiple of the tick size splits ticks; every
    event is processed exactly once and in arrival order."""
    ticks = np.array([5, 0, 9, 3, 11, 2, 0, 0, 7])
    seen = []

    def proc(pieces, k):
        seen.extend(np.concatenate([pc.arrivals() for pc in pieces]).tolist())
        return 0.5
    res, log, _ = osv.run(ticks, poll_ms=10.0, policy=osv.FIXED_SIZE, bound_ms=50.0,
                          fixed_rows=4, process=proc)
    assert res["processed"] == ticks.sum() == len(seen)
    assert np.all(np.diff(seen) > 0)
    assert all(r.n_events == 4 for r in log[:-1])


def test_oracle_alg1_exact_model_keeps_maxlat_within_bound():
    """With a processing time exactly linear in bytes and that model as the
    predictor, the GUARDED rule admits at the first poll where
    EstMaxLat + poll reaches the bound, so no batch's MaxLat exceeds the bound
    by more than one tick's processing time."""
    rng = np.random.default_rng(3)
    ticks = rng.poisson(200, 400)
    per_byte = 1e-3 / 16.0  # ms per byte

    def proc(pieces, k):
        return k * 16.0 * per_byte
    res, log, lat = osv.run(ticks, poll_ms=10.0, policy=osv.LEARNED, bound_ms=60.0,
                            process=proc, predictor=lambda b, nds: b * per_byte)
    tick_proc = ticks.max() * 16.0 * per_byte
    assert max(r.maxlat_ms for r in log[1:-1]) <= 60.0 + tick_proc + 1e-9
    assert res["p_hi"] <= 60.0 + tick_proc
    for r in log[1:-1]:
        assert r.est_ms == pytest.approx(r.maxlat_ms, rel=1e-12)  # the estimate is exact


def test_oracle_memory_cap_and_conservation():
    rng = np.random.default_rng(5)
    ticks = rng.poisson(50, 300)
    res, log, lat = osv.run(ticks, poll_ms=10.0, policy=osv.FIXED_TRIGGER, bound_ms=100.0,
                            trigger_ms=40.0, process=fake_proc(), admissible=lambda: 120)
    assert res["processed"] == ticks.sum()
    assert max(r.n_events for r in log) <= 120
    assert lat.min() > 0


def test_oracle_kth_smallest_is_the_order_statistic():
    x = np.random.default_rng(0).uniform(0, 10, 1001)
    for q in (0.5, 0.9, 0.99, 1.0):
        assert osv.kth_smallest(x, q) == np.quantile(x, q, method="inverted_cdf")


# ------------------------------------------------- engine loop vs the oracle

CASES = [
    dict(policy=osv.FIXED_SIZE, fixed_rows=300),
    dict(policy=osv.FIXED_SIZE, fixed_rows=77, cap=50),
    dict(policy=osv.FIXED_TRIGGER, trigger_ms=35.0),
    dict(policy=osv.FIXED_TRIGGER, trigger_ms=20.0, cap=400),
    dict(policy=osv.ANALYTIC),
    dict(policy=osv.ANALYTIC, cap=600),
    dict(policy=osv.ANALYTIC, rule="paper"),
    dict(policy=osv.LEARNED),
    dict(policy=osv.LEARNED, cap=500),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "-".join(f"{k}{v}" for k, v in c.items()))
def test_engine_loop_matches_oracle(case):
    rng = np.random.default_rng(11 + case["policy"])
    ticks = rng.poisson(rng.uniform(0, 120, 500)).astype(np.int64)
    ticks[100:140] = 0  # an idle stretch
    proc = fake_proc(a=3.0, b=2e-3, c=0.05)
    cap = case.get("cap")
    rule = case.get("rule", "guarded")
    pred = (lambda b, nds: 3.0 + 2e-3 * b / 16.0) if case["policy"] == osv.LEARNED else None
    ref, rlog, _ = osv.run(ticks, poll_ms=10.0, policy=case["policy"], bound_ms=80.0,
                           process=proc, fixed_rows=case.get("fixed_rows", 0),
                           trigger_ms=case.get("trigger_ms", 0.0), admit_rule=rule,
                           predictor=pred, admissible=(lambda: cap) if cap else None)
    res, elog = lm.serve_run(ticks, poll_ms=10.0, policy=case["policy"], bound_ms=80.0,
                             process=lambda ch, n, rec: proc(ch, n),
                             fixed_rows=case.get("fixed_rows", 0),
                             trigger_ms=case.get("trigger_ms", 0.0),
                             admit_rule=lm.ADMIT_GUARDED if rule == "guarded" else lm.ADMIT_PAPER,
                             predictor=pred, admissible=(lambda: cap) if cap else None)
    assert res["processed_events"] == ref["processed"] == ticks.sum()
    assert res["batches"] == ref["batches"] == len(elog)
    for e, r in zip(elog, rlog):
        assert e["n_events"] == r.n_events
        assert e["admit_ms"] == pytest.approx(r.admit_ms, rel=1e-12, abs=1e-9)
        assert e["proc_ms"] == pytest.approx(r.proc_ms, rel=1e-12)
        assert e["maxlat_ms"] == pytest.approx(r.maxlat_ms, rel=1e-12, abs=1e-9)
        assert e["est_ms"] == pytest.approx(r.est_ms, rel=1e-12, abs=1e-9)
        assert bool(e["forced"]) == r.forced
    for k_e, k_r in (("p50_ms", "p50"), ("p_hi_ms", "p_hi"), ("mean_ms", "mean"),
                     ("max_ms", "max")):
        assert res[k_e] == pytest.approx(ref[k_r], rel=1e-9), k_e
    assert bool(res["met_bound"]) == ref["met_bound"]
    assert res["completed"] == 1


def test_engine_chunks_cover_every_event_once():
    rng = np.random.default_rng(2)
    ticks = rng.poisson(30, 200).astype(np.int64)
    seen = []

    def proc(chunks, n, rec):
        assert sum(c.j_end - c.j_begin for c in chunks) == n
        for c in chunks:
            seen.extend(range(c.first_event + c.j_begin, c.first_event + c.j_end))
        return 1.0
    res, _ = lm.serve_run(ticks, poll_ms=10.0, policy=lm.POLICY_FIXED_SIZE, bound_ms=50.0,
                          fixed_rows=45, process=proc, admissible=lambda: 40)
    assert seen == list(range(int(ticks.sum())))


def test_engine_stops_when_the_bound_is_missed():
    ticks = np.full(400, 100, dtype=np.int64)
    slow = lambda ch, n, rec: 5.0 + 0.2 * n  # far slower than the arrival rate
    full, _ = lm.serve_run(ticks, poll_ms=10.0, policy=lm.POLICY_FIXED_TRIGGER, bound_ms=50.0,
                           trigger_ms=10.0, process=slow)
    early, _ = lm.serve_run(ticks, poll_ms=10.0, policy=lm.POLICY_FIXED_TRIGGER, bound_ms=50.0,
                            trigger_ms=10.0, process=slow, stop_when_missed=True)
    assert full["met_bound"] == 0 and full["completed"] == 1
    assert early["met_bound"] == 0 and early["completed"] == 0
    assert early["processed_events"] < full["processed_events"]


def test_engine_rejects_bad_configs():
    t = np.ones(4, dtype=np.int64)
    with pytest.raises(lm.LmsError):
        lm.serve_run(t, poll_ms=0.0, policy=0, bound_ms=1.0, fixed_rows=1, process=fake_proc())
    with pytest.raises(lm.LmsError):
        lm.serve_run(t, poll_ms=10.0, policy=0, bound_ms=1.0, fixed_rows=0, process=fake_proc())
    with pytest.raises(lm.LmsError):
        lm.serve_run(t, poll_ms=10.0, policy=3, bound_ms=1.0, process=fake_proc())

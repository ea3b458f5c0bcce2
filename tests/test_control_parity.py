"""The engine's control plane (C++ in the CUDA library, through the C ABI)
against the plain oracle (oracle/control.py): Alg. 1 decisions and the
estimates of Eqs. 3-5 on random arrival streams, Alg. 2 plans with the costs of
Eqs. 6-8 on random operation chains, and the Eq. 9 regression.  Host code only:
these run without a GPU."""
import numpy as np
import pytest

from oracle import control as oc
from paper_2111_04289_b300 import lmstream as lm


@pytest.mark.parametrize("slide,policy", [(3000.0, "paper"), (3000.0, "guarded"), (0.0, "paper"),
                                          (0.0, "guarded"), (100.0, "guarded")])
def test_alg1_decisions_match_oracle(slide, policy):
    rng = np.random.default_rng(int(slide) + len(policy))
    ref = oc.Admission(slide_ms=slide, policy=policy)
    eng = lm.Admission(slide, lm.ADMIT_GUARDED if policy == "guarded" else lm.ADMIT_PAPER, 10.0)
    t, busy, decisions = 0.0, -1.0, 0
    pend_a, pend_b = [], []
    for step in range(3000):
        t += 10.0
        n = int(rng.poisson(1.5))
        pend_a.extend(np.sort(t - rng.uniform(0, 10.0, n)))
        pend_b.extend(rng.uniform(100, 5000, n))
        if t < busy:  # a batch is running: arrivals wait for the next poll
            continue
        arr, nb = np.array(pend_a), np.array(pend_b)
        pend_a, pend_b = [], []
        r_ok = ref.poll(t, [oc.Dataset(a, b) for a, b in zip(arr, nb)])
        e_ok, e_est, e_n = eng.poll(t, arr, nb)
        assert e_ok == r_ok, step
        if r_ok:
            assert e_n == len(ref.admitted)
            assert e_est == pytest.approx(ref.last_est, rel=1e-12, abs=1e-9)
            proc = float(rng.uniform(5, 400))
            assert eng.complete(proc) == pytest.approx(ref.complete(proc), rel=1e-12)
            assert eng.avg_thput() == pytest.approx(oc.avg_thput(ref.parts_hist, ref.proc_hist),
                                                    rel=1e-12)
            busy = t + proc
            decisions += 1
        assert eng.buffered() == len(ref.buffered)
    assert decisions > 5


def test_alg1_busy_arrivals_are_buffered_like_the_oracle():
    """Arrivals while a batch runs reach Alg. 1 at the next poll as new data."""
    ref = oc.Admission(slide_ms=500.0, policy="guarded")
    eng = lm.Admission(500.0, lm.ADMIT_GUARDED, 10.0)
    assert ref.poll(10.0, [oc.Dataset(0.0, 100.0)]) and eng.poll(10.0, [0.0], [100.0])[0]
    ref.complete(200.0), eng.complete(200.0)
    new = [oc.Dataset(20.0 + 10 * i, 100.0) for i in range(20)]  # during the batch
    r = ref.poll(210.0, new)
    e = eng.poll(210.0, [d.arrival_ms for d in new], [d.nbytes for d in new])
    assert r == e[0]
    assert ref.last_est == pytest.approx(e[1], rel=1e-12)


def test_alg2_random_chains_match_oracle():
    rng = np.random.default_rng(9)
    names = list(oc.BASE_COST)
    for _ in range(500):
        ops = [names[i] for i in rng.integers(0, 8, rng.integers(1, 7))]
        infpt = float(rng.uniform(1e4, 1e6))
        cores = int(rng.integers(1, 48))
        batch = float(infpt * cores * rng.uniform(0.3, 3.0))
        ref = oc.map_device(ops, batch, cores, infpt)
        got = lm.map_device(ops, batch, cores, infpt, oc.BASE_TRANS_COST)
        for (rd, rc, rg), (gd, gc, gg) in zip(ref, got):
            assert rd == gd
            assert gc == pytest.approx(rc, rel=1e-12) and gg == pytest.approx(rg, rel=1e-12)


def test_eq9_matches_oracle():
    rng = np.random.default_rng(11)
    for hist in (0, 5, 50):
        reg = lm.Regressor(hist)
        th, la, inf = [], [], []
        for k in range(80):
            th.append(float(rng.uniform(1e4, 1e6)))
            la.append(float(rng.uniform(10, 300)))
            inf.append(float(150 * 1024 + rng.normal(0, 5000) + 0.01 * th[-1]))
            reg.add(th[-1], la[-1], inf[-1])
            lo = max(0, len(th) - hist) if hist else 0
            st, beta, pred = reg.fit(max(th), 100.0)
            rb, rp = oc.regress_infpt(th[lo:], la[lo:], inf[lo:], max(th), 100.0)
            assert st == (0 if len(th[lo:]) >= 3 else -3)
            np.testing.assert_allclose(beta, rb, rtol=1e-6, atol=1e-9 * abs(rb[0]))
            assert pred == pytest.approx(rp, rel=1e-6)
    # constant inputs: singular system, both give (mean, 0, 0)
    reg = lm.Regressor(0)
    for k in range(10):
        reg.add(5.0, 7.0, 1000.0 + k)
    st, beta, pred = reg.fit(5.0, 7.0)
    rb, rp = oc.regress_infpt([5.0] * 10, [7.0] * 10, [1000.0 + k for k in range(10)], 5.0, 7.0)
    np.testing.assert_allclose(beta, rb)


@pytest.mark.parametrize("t,l,y", [
    ([1.0e5, 2.0e5], [30.0, 50.0], [100.0, 200.0]),                        # n = 2
    ([5.0e4] * 4, [10.0, 20.0, 30.0, 40.0], [10.0, 20.0, 30.0, 45.0]),      # constant column
    ([1.0, 2.0, 3.0, 4.0], [3.0, 5.0, 7.0, 9.0], [8.0, 6.0, 7.0, 5.0]),      # collinear
])
def test_eq9_degenerate_branch_matches_oracle(t, l, y):
    reg = lm.Regressor(0)
    for a, b, c in zip(t, l, y):
        reg.add(a, b, c)
    st, beta, pred = reg.fit(3.0e5, 100.0)
    rb, rp = oc.regress_infpt(t, l, y, 3.0e5, 100.0)
    assert st == (0 if len(y) >= 3 else -3)
    np.testing.assert_array_equal(beta, rb)
    assert pred == rp


def test_variant_analytic_chooser_matches_oracle():
    """The engine's analytic variant chooser against the oracle's on noisy
    power-law pass times: the same picks and the same inflection point after
    every pass."""
    rng = np.random.default_rng(21)
    eng = lm.VariantAnalytic(148, 16.0, 150 * 1024, history=12, explore=2)
    orc = oc.VariantAnalytic(148, 16.0, 150 * 1024, history=12, explore=2)
    for k in range(120):
        rows = int(2 ** rng.uniform(12, 26))
        pe, po = eng.choose(rows), orc.choose(rows)
        assert pe == po, k
        c, b = (2e-6, 1.0) if pe == 1 else (4e-3, 0.55)
        ms = c * rows ** b * float(np.exp(rng.normal(0, 0.05)))
        eng.observe(rows, pe, ms)
        orc.observe(rows, pe, ms)
        assert eng.state()["infpt_bytes"] == pytest.approx(orc.infpt, rel=1e-9), k
        for v in (1, 2):
            pe_, po_ = eng.predict(rows, v), orc.predict(rows, v)
            assert (pe_ < 0) == (po_ < 0)
            if po_ > 0:
                assert pe_ == pytest.approx(po_, rel=1e-9)
    assert eng.state()["picks"] == [orc.picks[1], orc.picks[2]]
    eng.close()

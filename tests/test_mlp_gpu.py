"""The learned cost model's CUDA kernels against the FP64 oracle
(oracle/mlp.py), and what the trained network gains over Eq. 5.

Tolerances: the kernels accumulate in FP32 over at most 64 terms per dot
product and at most 4096 samples per gradient sum; 1e-4 relative (of the
tensor's largest entry for gradients) bounds that with a wide margin."""
import numpy as np
import pytest

from oracle import mlp as om
from paper_2111_04289_b300 import lmstream as lm
from paper_2111_04289_b300.synth import ServingLoad

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _data(seed, n):
    rng = np.random.default_rng(seed)
    x = rng.uniform(0, 1, (n, 8)).astype(np.float32)
    t = rng.normal(0, 1, n).astype(np.float32)
    return x, t


@pytest.mark.parametrize("n", [1, 63, 64, 1000, 4096])
def test_forward_matches_oracle(n):
    p = om.init_params(10 + n)
    x, _ = _data(n, n)
    net = lm.Mlp(p)
    y = net.forward(x)
    ref, _ = om.forward(om.effective(p), x.astype(np.float64))
    np.testing.assert_allclose(y, ref, rtol=1e-4, atol=1e-4 * np.abs(ref).max())
    net.close()


@pytest.mark.parametrize("n", [5, 64, 65, 777, 4096])
def test_gradient_matches_oracle(n):
    p = om.init_params(20 + n)
    x, t = _data(100 + n, n)
    net = lm.Mlp(p)
    loss, g = net.train(x, t, steps=0, want_grad=True)
    ref_loss, ref = om.gradient(om.effective(p), x.astype(np.float64), t.astype(np.float64))
    assert loss == pytest.approx(ref_loss, rel=1e-4)
    for name, shp in om.SHAPES:
        a = om.unpack(g.astype(np.float64))[name]
        b = om.unpack(ref)[name]
        scale = max(np.abs(b).max(), 1e-12)
        assert np.abs(a - b).max() <= 1e-4 * scale, name
    np.testing.assert_array_equal(net.params(), p)  # steps == 0 leaves the weights alone
    net.close()


def test_adam_step_matches_oracle():
    p = om.init_params(31)
    x, t = _data(32, 500)
    net = lm.Mlp(p)
    net.train(x, t, steps=1, lr=1e-3)
    w1 = net.params().astype(np.float64)
    _, g = om.gradient(om.effective(p), x.astype(np.float64), t.astype(np.float64))
    ref, _, _ = om.adam_step(p.astype(np.float64), np.zeros_like(g), np.zeros_like(g), g, 1,
                             lr=1e-3)
    big = np.abs(g) >= 1e-3 * np.abs(g).max()
    np.testing.assert_allclose(w1[big], ref[big], rtol=0, atol=1e-6)
    # no first-step update exceeds lr (up to FP32 rounding)
    assert np.all(np.abs(w1 - p) <= 1e-3 * (1 + 1e-5) + 1e-6 * np.abs(p))
    net.close()


def test_training_on_gpu_fits_like_the_oracle():
    rng = np.random.default_rng(4)
    x = rng.uniform(0, 1, (256, 8)).astype(np.float32)
    t = np.log1p(3 * x[:, 0] + x[:, 1] * x[:, 2]).astype(np.float32)
    p = om.init_params(5)
    net = lm.Mlp(p)
    first = net.train(x, t, steps=0)
    last = net.train(x, t, steps=400, lr=3e-3)
    _, losses = om.train(p, x.astype(np.float64), t.astype(np.float64), 400, lr=3e-3)
    assert first == pytest.approx(losses[0], rel=1e-4)
    assert last < 0.05 * first and losses[-1] < 0.05 * losses[0]
    net.close()


Q = [dict(size=60_000, slide=5_000, col="value", op="gt", value=0.5)]
FEATS = dict(key_card=1_000_000, selectivity=0.7559, panes=12, n_queries=1, slide_ms=5_000.0,
             poll_ms=10.0)


def _serve(seed, policy, ticks, **kw):
    g = lm.ServeGpu(Q, seed=seed, n_keys=1_000_000, max_batch_rows=1 << 25,
                    state_cap_bytes=8 << 30)
    res, log = lm.serve_run(ticks, poll_ms=10.0, policy=policy, bound_ms=100.0,
                            backend=g.backend(), add_decide_time=True, **kw)
    g.close()
    return res, log


def _errors(net, log):
    """|ln(predicted / measured)| of the network and of Eq. 5 (bytes over the
    AvgThPut of the run's earlier batches, as Alg. 1 uses it) per batch."""
    sb = sp = 0.0
    e_net, e_eq5 = [], []
    for r in log:
        bytes_ = 16.0 * r["n_events"]
        if sp > 0:
            x = np.stack([lm.cost_features(r["n_events"], r["state_groups_before"],
                                           FEATS["key_card"], FEATS["selectivity"], 12, 1,
                                           r["n_chunks"] * 10.0 / 5000.0, op)
                          for op in range(lm.N_OPS)])
            pred = float(np.exp(net.forward(x).astype(np.float64)).sum() * 1e-3)
            e_net.append(abs(np.log(pred / r["proc_ms"])))
            e_eq5.append(abs(np.log(bytes_ / (sb / sp) / r["proc_ms"])))
        sb += bytes_
        sp += r["proc_ms"]
    return e_net, e_eq5


def test_trained_network_predicts_processing_time_better_than_eq5():
    """Train on timings the engine logged under several batching policies, then
    predict every batch of held-out runs (other seeds, rates and policies):
    averaged over the held-out policies, the network's median
    |ln(predicted / measured)| beats Eq. 5's, which is what Alg. 1 would
    otherwise use.  (Per policy: under a fixed batch size every batch has the
    same size, where Eq. 5's running ratio is at its best.)"""
    net = lm.Mlp(om.init_params(7))
    learned = lm.Learned(net, None, **FEATS)
    train_ticks = ServingLoad(rate_scale=0.5).ticks(1, 10_000)
    for pol, kw in [(lm.POLICY_ANALYTIC, {}), (lm.POLICY_FIXED_SIZE, dict(fixed_rows=150_000)),
                    (lm.POLICY_FIXED_SIZE, dict(fixed_rows=600_000)),
                    (lm.POLICY_FIXED_SIZE, dict(fixed_rows=2_000_000)),
                    (lm.POLICY_FIXED_TRIGGER, dict(trigger_ms=50.0))]:
        _, log = _serve(3, pol, train_ticks, **kw)
        for r in log:
            learned.observe(r)
    assert learned.samples() >= 1000
    learned.fit(5000, lr=1e-3)
    m_net, m_eq5 = [], []
    test_ticks = ServingLoad(rate_scale=0.7).ticks(2, 10_000)
    for pol, kw in [(lm.POLICY_ANALYTIC, {}), (lm.POLICY_FIXED_TRIGGER, dict(trigger_ms=20.0)),
                    (lm.POLICY_FIXED_SIZE, dict(fixed_rows=400_000))]:
        _, log = _serve(4, pol, test_ticks, **kw)
        a, b = _errors(net, log)
        print(f"policy {pol}: median |ln(pred/measured)| network {np.median(a):.3f}, "
              f"Eq. 5 {np.median(b):.3f} over {len(a)} batches")
        m_net.append(float(np.median(a)))
        m_eq5.append(float(np.median(b)))
    print(f"mean of the per-policy medians: network {np.mean(m_net):.3f}, "
          f"Eq. 5 {np.mean(m_eq5):.3f}")
    assert np.mean(m_net) < 0.75 * np.mean(m_eq5)
    learned.close()
    net.close()


def test_learned_policy_runs_with_judge_and_online_refit():
    net = lm.Mlp(om.init_params(8))
    learned = lm.Learned(net, None, **FEATS)
    ticks = ServingLoad(rate_scale=0.5).ticks(5, 6_000)
    _, log = _serve(6, lm.POLICY_ANALYTIC, ticks)
    for r in log:
        learned.observe(r)
    learned.fit(2000)
    g = lm.ServeGpu(Q, seed=7, n_keys=1_000_000, max_batch_rows=1 << 25, state_cap_bytes=8 << 30)
    learned.set_backend(g)
    learned.set_online(refit_every=20, refit_steps=20)
    pred, obs = learned.hooks()
    res, log = lm.serve_run(ticks, poll_ms=10.0, policy=lm.POLICY_LEARNED, bound_ms=100.0,
                            backend=g.backend(), predictor=pred, observer=obs,
                            add_decide_time=True)
    st = learned.stats()
    assert res["completed"] == 1 and res["processed_events"] == ticks.sum()
    assert st["uses_net"] + st["uses_eq5"] > 0
    assert res["observe_ms"] > 0
    g.close()
    learned.close()
    net.close()

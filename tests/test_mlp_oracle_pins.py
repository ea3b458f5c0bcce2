"""Pins of the learned cost model's oracle (oracle/mlp.py), CPU only:
bf16 rounding at hand-picked values, the gradient against central finite
differences and against torch autograd in float64, Adam's first steps against
their closed forms, and a training run that fits a known function."""
import numpy as np
import pytest

from oracle import mlp as om


def test_layout_size():
    assert om.N_PARAMS == 8961


@pytest.mark.parametrize("x,expect", [
    (1.0, 1.0),
    (1.0 + 2.0 ** -8, 1.0),                    # halfway, ties to even (kept bit 0)
    (1.0 + 3 * 2.0 ** -8, 1.0 + 2.0 ** -6),    # halfway, ties to even (rounds up)
    (1.0 + 2.0 ** -8 + 2.0 ** -20, 1.0 + 2.0 ** -7),  # above halfway
    (-(1.0 + 3 * 2.0 ** -8), -(1.0 + 2.0 ** -6)),
    (65504.0, 65536.0),
    (0.0, 0.0),
])
def test_bf16_round_to_nearest_even(x, expect):
    got = float(om.bf16_round(np.array([x], np.float32))[0])
    assert got == np.float32(expect)


def _data(seed, n=24):
    rng = np.random.default_rng(seed)
    x = rng.uniform(0, 1, (n, 8))
    t = rng.normal(0, 1, n)
    p = om.effective(om.init_params(seed))
    return p, x, t


def test_gradient_matches_finite_differences():
    p, x, t = _data(1)
    _, g = om.gradient(p, x, t)
    rng = np.random.default_rng(2)
    idx = rng.choice(om.N_PARAMS, 200, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        fd = (om.loss(p + e, x, t) - om.loss(p - e, x, t)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])), (i, fd, g[i])


def test_gradient_matches_torch_autograd():
    torch = pytest.importorskip("torch")
    p, x, t = _data(3)
    l_ref, g = om.gradient(p, x, t)
    pt = torch.tensor(p, dtype=torch.float64, requires_grad=True)
    xt = torch.tensor(x, dtype=torch.float64)
    tt = torch.tensor(t, dtype=torch.float64)
    o = 0
    ws = {}
    for name, shp in om.SHAPES:
        n = int(np.prod(shp))
        ws[name] = pt[o:o + n].reshape(shp)
        o += n
    h = torch.relu(xt @ ws["W1"].T + ws["b1"])
    h = torch.relu(h @ ws["W2"].T + ws["b2"])
    h = torch.relu(h @ ws["W3"].T + ws["b3"])
    y = h @ ws["W4"] + ws["b4"][0]
    lt = torch.mean((y - tt) ** 2)
    lt.backward()
    assert float(lt.detach()) == pytest.approx(l_ref, rel=1e-12)
    np.testing.assert_allclose(g, pt.grad.numpy(), rtol=1e-10, atol=1e-14)


def test_adam_first_steps_closed_form():
    g = np.array([0.5, -2.0, 1e-3, 0.0])
    w0 = np.array([1.0, 1.0, 1.0, 1.0])
    m = np.zeros(4)
    v = np.zeros(4)
    w1, m, v = om.adam_step(w0, m, v, g, 1, lr=1e-3)
    # step 1: mhat = g, vhat = g^2 -> w -= lr * g / (|g| + eps)
    np.testing.assert_allclose(w1, w0 - 1e-3 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    w2, m, v = om.adam_step(w1, m, v, g, 2, lr=1e-3)
    # constant gradient: mhat = g and vhat = g^2 again at every step
    np.testing.assert_allclose(w2, w1 - 1e-3 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)


def test_training_fits_a_smooth_function():
    rng = np.random.default_rng(4)
    x = rng.uniform(0, 1, (256, 8))
    t = np.log1p(3 * x[:, 0] + x[:, 1] * x[:, 2])
    master, losses = om.train(om.init_params(5), x, t, 400, lr=3e-3)
    assert losses[-1] < 0.05 * losses[0]

"""Pins of the FP64 closure network (oracle.mlp): gradients against central finite differences,
closed forms for degenerate weights, Adam's first step in closed form (Kingma & Ba 2015:
m_hat = g, v_hat = g^2, so the step is lr g / (|g| + eps)), and bfloat16 rounding of hand-picked
values (7 stored mantissa bits, ties to even)."""
import numpy as np
import pytest

from oracle import mlp


def _data(n=40, seed=1):
    rng = np.random.default_rng(seed)
    x = rng.normal(0, 1, (n, mlp.NIN)) * np.arange(1, mlp.NIN + 1) + 0.3
    t = np.sin(x[:, 0]) + 0.1 * x[:, 3]
    mu, sd = mlp.feature_norm(x)
    return x, t, mu, sd


def test_gradient_matches_finite_differences():
    x, t, mu, sd = _data()
    p = mlp.init_params(3)
    L, g = mlp.loss_and_grad(p, x, t, mu, sd)
    rng = np.random.default_rng(5)
    idx = rng.choice(mlp.NPARAM, 60, replace=False)
    idx = np.concatenate([idx, [mlp.NPARAM - 1, 0, 576, 640, 4736]])   # b3, W1, b1, W2, b2
    h = 1e-6
    for i in idx:
        e = np.zeros(mlp.NPARAM)
        e[i] = h
        Lp, _ = mlp.loss_and_grad(p + e, x, t, mu, sd)
        Lm, _ = mlp.loss_and_grad(p - e, x, t, mu, sd)
        fd = (Lp - Lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_zero_weights_closed_form():
    x, t, mu, sd = _data(10)
    d = mlp.unpack(np.zeros(mlp.NPARAM))
    d["b1"][:] = 0.7
    d["b2"][:] = -0.4
    d["w3"][:] = 0.25
    d["b3"][:] = 1.5
    p = mlp.pack(d)
    y, _ = mlp.forward(p, x, mu, sd)
    s = -0.4 / (1 + np.exp(0.4))                    # silu(-0.4)
    assert np.allclose(y, 64 * 0.25 * s + 1.5, rtol=1e-14)
    L, g = mlp.loss_and_grad(p, x, t, mu, sd)
    G = mlp.unpack(g)
    assert G["b3"][0] == pytest.approx(2 * np.mean(y - t), rel=1e-12)
    assert np.allclose(G["w3"], 2 * np.mean(y - t) * s, rtol=1e-12)
    assert np.allclose(G["W1"], 0.0, atol=0)        # W2 = 0 blocks the path to W1
    assert np.allclose(G["b1"], 0.0, atol=0)


def test_silu_and_derivative():
    assert mlp.silu(0.0) == 0.0
    assert mlp.silu(40.0) == pytest.approx(40.0, rel=1e-15)
    assert mlp.silu(-40.0) == pytest.approx(0.0, abs=1e-15)
    z = np.linspace(-6, 6, 25)
    fd = (mlp.silu(z + 1e-6) - mlp.silu(z - 1e-6)) / 2e-6
    assert np.allclose(mlp.dsilu(z), fd, atol=1e-8)
    assert mlp.dsilu(0.0) == 0.5


def test_adam_first_step_closed_form():
    rng = np.random.default_rng(2)
    p = rng.normal(size=50)
    g = rng.normal(size=50)
    p1, m, v = mlp.adam_step(p, g, np.zeros(50), np.zeros(50), 1, lr=0.01)
    assert np.allclose(p1, p - 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_bf16_rounding():
    one = 1.0
    ulp = 2.0 ** -7
    vals = np.array([one, one + ulp / 2, one + 1.5 * ulp, one + 0.75 * ulp, -3.0, 0.0])
    want = np.array([one, one, one + 2 * ulp, one + ulp, -3.0, 0.0])
    assert np.array_equal(mlp.bf16(vals), want)


def test_adam_training_reduces_loss():
    x, t, mu, sd = _data(400, seed=7)
    p = mlp.init_params(11)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    L0, _ = mlp.loss_and_grad(p, x, t, mu, sd)
    for k in range(1, 301):
        L, g = mlp.loss_and_grad(p, x, t, mu, sd)
        p, m, v = mlp.adam_step(p, g, m, v, k, lr=3e-3)
    assert L < 0.2 * L0

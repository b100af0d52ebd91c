"""Pins of the FP64 MLP oracle (no GPU): GELU special values, gradients against central finite
differences, structural special cases, and the first Adam step's closed form."""
import numpy as np
import pytest

from oracle import mlp


def test_gelu_special_values():
    assert mlp.gelu(0.0) == 0.0
    x = np.linspace(-6, 6, 101)
    # odd part: gelu(x) - gelu(-x) = x for the tanh form
    np.testing.assert_allclose(mlp.gelu(x) - mlp.gelu(-x), x, atol=1e-14)
    assert abs(mlp.gelu(20.0) - 20.0) < 1e-12 and abs(mlp.gelu(-20.0)) < 1e-12
    # published value of the tanh approximation at x = 1: 0.8411919906...
    assert abs(mlp.gelu(1.0) - 0.8411919906082768) < 1e-12
    h = 1e-6
    np.testing.assert_allclose(mlp.gelu_grad(x), (mlp.gelu(x + h) - mlp.gelu(x - h)) / (2 * h),
                               rtol=1e-8, atol=1e-9)


def _batch(n=37, seed=1):
    rng = np.random.default_rng(seed)
    st = rng.standard_normal((n, 64))
    off = rng.random((n, 3))
    x, s = mlp.features(st, off)
    field = rng.integers(0, 4, n)
    target = rng.standard_normal(n) * 0.1
    return x, s, field, target


def test_features_scale_and_layout():
    rng = np.random.default_rng(2)
    st = rng.standard_normal((5, 64)) * 7.0
    off = rng.random((5, 3))
    x, s = mlp.features(st, off)
    np.testing.assert_allclose(np.max(np.abs(x[:, :64]), 1), 1.0)
    np.testing.assert_allclose(x[:, 64:], off)
    np.testing.assert_allclose(x[:, :64] * s[:, None], st)


@pytest.mark.parametrize("name", ["W1", "b1", "W2", "b2", "W3", "b3"])
def test_gradients_match_finite_differences(name):
    p = mlp.init_params(3)
    for k in ("b1", "b2", "b3"):
        p[k] = np.random.default_rng(4).standard_normal(p[k].shape) * 0.1
    x, _, field, target = _batch()
    _, g = mlp.loss_and_grad(p, x, field, target)
    rng = np.random.default_rng(5)
    flat = p[name].reshape(-1)
    for idx in rng.choice(flat.size, min(12, flat.size), replace=False):
        h = 1e-6
        old = flat[idx]
        flat[idx] = old + h
        lp, _ = mlp.loss_and_grad(p, x, field, target)
        flat[idx] = old - h
        lm, _ = mlp.loss_and_grad(p, x, field, target)
        flat[idx] = old
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[name].reshape(-1)[idx]) <= 1e-7 * max(1.0, abs(fd)), (name, idx)


def test_zero_last_layer_outputs_bias_and_only_selected_output_gets_gradient():
    p = mlp.init_params(6)
    p["W3"][:] = 0.0
    p["b3"] = np.array([0.1, -0.2, 0.3, 0.4])
    x, _, field, target = _batch(n=9)
    y, _ = mlp.forward(p, x)
    np.testing.assert_allclose(y, np.tile(p["b3"], (9, 1)))
    field = np.zeros(9, int)
    _, g = mlp.loss_and_grad(p, x, field, target)
    assert np.all(g["W3"][1:] == 0) and np.all(g["b3"][1:] == 0)
    np.testing.assert_allclose(g["b3"][0], 2 * np.mean(0.1 - target))


def test_first_adam_step_is_lr_times_sign():
    p = {"w": np.array([1.0, -2.0, 3.0])}
    g = {"w": np.array([0.5, -4.0, 1e-3])}
    st = mlp.adam_init(p)
    mlp.adam_step(p, g, st, lr=0.01, eps=0.0)
    np.testing.assert_allclose(p["w"], [1.0 - 0.01, -2.0 + 0.01, 3.0 - 0.01])


def test_training_reduces_loss():
    """A few hundred Adam steps fit a smooth synthetic target (sanity of the whole loop)."""
    rng = np.random.default_rng(7)
    st = rng.standard_normal((512, 64))
    off = rng.random((512, 3))
    x, _ = mlp.features(st, off)
    field = rng.integers(0, 4, 512)
    target = 0.3 * np.sin(3 * x[:, 64]) * x[:, 10] + 0.1 * x[:, 66]
    p = mlp.init_params(8)
    st_ = mlp.adam_init(p)
    l0, _ = mlp.loss_and_grad(p, x, field, target)
    for _ in range(300):
        _, g = mlp.loss_and_grad(p, x, field, target)
        mlp.adam_step(p, g, st_, lr=3e-3)
    l1, _ = mlp.loss_and_grad(p, x, field, target)
    assert l1 < 0.1 * l0

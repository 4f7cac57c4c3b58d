"""Pins of the FP64 MLP oracle: backprop vs central differences, Adam vs its closed form."""
import numpy as np
import pytest

from oracle import mlp_oracle as mo


def _tiny(seed=0, din=5, dh=7, dout=3):
    rng = np.random.default_rng(seed)
    p = [rng.normal(size=(dh, din)) / 2, rng.normal(size=dh) / 5, rng.normal(size=(dh, dh)) / 3,
         rng.normal(size=dh) / 5, rng.normal(size=(dout, dh)) / 3, rng.normal(size=dout) / 5]
    x = rng.normal(size=(4, din))
    t = rng.normal(size=(4, dout))
    return p, x, t


@pytest.mark.parametrize("out_sigmoid", [False, True])
def test_backprop_matches_central_differences(out_sigmoid):
    p, x, t = _tiny()
    grads, _ = mo.backward(p, x, t, out_sigmoid)
    h = 1e-6
    for pi, gi in zip(p, grads):
        flat = pi.reshape(-1)
        gflat = gi.reshape(-1)
        for j in range(flat.size):
            old = flat[j]
            flat[j] = old + h
            lp = mo.loss(p, x, t, out_sigmoid)
            flat[j] = old - h
            lm = mo.loss(p, x, t, out_sigmoid)
            flat[j] = old
            assert gflat[j] == pytest.approx((lp - lm) / (2 * h), rel=1e-6, abs=1e-9)


def test_silu_derivative_and_values():
    z = np.linspace(-6, 6, 101)
    fd = (mo.silu(z + 1e-6) - mo.silu(z - 1e-6)) / 2e-6
    np.testing.assert_allclose(mo.dsilu(z), fd, rtol=1e-7, atol=1e-9)
    assert mo.silu(0.0) == 0.0 and mo.dsilu(0.0) == 0.5


def test_adam_first_steps_closed_form():
    """With a constant gradient g the bias-corrected moments are exactly g and g^2, so every step
    moves each parameter by -lr g / (|g| + eps) (Kingma & Ba 2015, Algorithm 1)."""
    rng = np.random.default_rng(1)
    p = [rng.normal(size=(3, 2))]
    g = [rng.normal(size=(3, 2))]
    m = [np.zeros((3, 2))]
    v = [np.zeros((3, 2))]
    lr, eps = 1e-3, 1e-8
    cur = p
    for t in range(1, 4):
        cur, m, v = mo.adam_step(cur, g, m, v, t, lr, eps=eps)
        np.testing.assert_allclose(cur[0], p[0] - t * lr * g[0] / (np.abs(g[0]) + eps), rtol=1e-12)


def test_training_reduces_loss():
    p, x, t = _tiny(2)
    m = [np.zeros_like(a) for a in p]
    v = [np.zeros_like(a) for a in p]
    l0 = mo.loss(p, x, t)
    for step in range(1, 201):
        g, _ = mo.backward(p, x, t)
        p, m, v = mo.adam_step(p, g, m, v, step, 1e-2)
    assert mo.loss(p, x, t) < 0.2 * l0

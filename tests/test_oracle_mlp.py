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


def test_flow_refine_constant_field_is_exact():
    a0 = np.array([[0.1, -0.2, 0.3]])
    a = mo.flow_refine(a0, lambda t, a: np.full_like(a, 0.7), 20, 0.05)
    np.testing.assert_allclose(a, a0 + 20 * 0.05 * 0.7, rtol=0, atol=1e-14)


def test_flow_refine_linear_decay_matches_the_euler_closed_form():
    # da/dt = -a: explicit Euler gives a0 (1 - dt)^N, which tends to a0 e^{-1} as dt -> 0
    a0 = np.array([[1.0, -2.0]])
    a = mo.flow_refine(a0, lambda t, a: -a, 20, 0.05)
    np.testing.assert_allclose(a, a0 * (1 - 0.05) ** 20, rtol=1e-14)
    fine = mo.flow_refine(a0, lambda t, a: -a, 20000, 1.0 / 20000)
    np.testing.assert_allclose(fine, a0 * np.exp(-1.0), rtol=1e-4)


def test_flow_refine_time_field_is_the_left_riemann_sum():
    # da/dt = t from t = 0: sum_k dt (k dt) = dt^2 N (N - 1) / 2 (-> 1/2 as dt -> 0)
    a = mo.flow_refine(np.zeros((1, 1)), lambda t, a: np.full_like(a, t), 20, 0.05)
    np.testing.assert_allclose(a, 0.05 ** 2 * 20 * 19 / 2, rtol=1e-14)


def test_mlp_velocity_reads_obs_action_and_time_in_that_order():
    rng = np.random.default_rng(3)
    d_obs, m, hid = 3, 2, 4
    W1 = np.zeros((hid, d_obs + m + 1))
    W1[0, d_obs + m] = 1.0          # unit 0 sees t only
    W1[1, d_obs] = 1.0              # unit 1 sees a[0] only
    params = [W1, np.zeros(hid), np.eye(hid), np.zeros(hid), np.zeros((m, hid)), np.zeros(m)]
    params[4][0, 0] = 1.0           # output 0 = silu(silu(t))
    params[4][1, 1] = 1.0           # output 1 = silu(silu(a[0]))
    obs = rng.normal(size=(5, d_obs))
    a = rng.normal(size=(5, m))
    y = mo.mlp_velocity(params, obs)(0.3, a)
    np.testing.assert_allclose(y[:, 0], mo.silu(mo.silu(0.3)), rtol=1e-14)
    np.testing.assert_allclose(y[:, 1], mo.silu(mo.silu(a[:, 0])), rtol=1e-14)

"""Pins of the imitation-reward oracle: closed forms of its pieces."""
import numpy as np

from oracle import mlp_oracle as mo
from oracle import reward_oracle as ro
from tests.handmodels import two_link


def test_tracking_reward_closed_forms():
    assert ro.reward_tracking(0.0) == 0.0
    np.testing.assert_allclose(ro.reward_tracking(0.5), np.log(2.0), rtol=1e-15)
    np.testing.assert_allclose(ro.reward_tracking(1 - np.exp(-3.0)), 3.0, rtol=1e-12)
    d = np.linspace(0.0, 0.99, 50)
    assert np.all(np.diff(ro.reward_tracking(d)) > 0)   # larger D, larger reward


def test_power_penalty_is_minus_mean_absolute_power():
    np.testing.assert_allclose(ro.reward_power([1.0, 2.0], [-3.0, 4.0]), -5.5, rtol=1e-15)
    assert ro.reward_power([5.0, 0.0], [0.0, 7.0]) == 0.0


def test_tracking_error_vanishes_on_the_reference():
    m = two_link()
    q = np.array([0.3, -0.7])
    np.testing.assert_array_equal(ro.tracking_error(m, q, q), np.zeros(2 + 3 * 2))


def test_body_displacement_of_a_planar_arm_is_the_chord():
    # body 1's origin sits at the elbow, l1 = 0.6 from the shoulder; turning the shoulder by dtheta
    # moves it along a chord of length 2 l1 |sin(dtheta / 2)|; the elbow angle does not move it
    m = two_link(l1=0.6)
    l1 = float(m.body_offset[1][0])   # the model stores FP32 parameters
    q, q_ref = np.array([0.9, 0.2]), np.array([0.35, -1.1])
    d = ro.tracking_error(m, q, q_ref)
    np.testing.assert_allclose(d[:2], q - q_ref, rtol=0, atol=1e-15)
    np.testing.assert_allclose(d[2:5], 0.0, atol=1e-15)            # body 0's origin is the fixed shoulder
    np.testing.assert_allclose(np.linalg.norm(d[5:8]), 2 * l1 * abs(np.sin((0.9 - 0.35) / 2)), rtol=1e-12)


def test_reward_combines_the_discriminator_and_the_power_term():
    m = two_link()
    rng = np.random.default_rng(2)
    n_in, hid = 2 + 3 * 2, 8
    params = [rng.normal(size=(hid, n_in)), rng.normal(size=hid), rng.normal(size=(hid, hid)), rng.normal(size=hid),
              rng.normal(size=(1, hid)), rng.normal(size=1)]
    q, q_ref = np.array([0.2, 0.1]), np.array([-0.4, 0.5])
    F, v = rng.uniform(0, 100, 5), rng.normal(size=5)
    x = ro.tracking_error(m, q, q_ref)[None, :]
    d = mo.sigmoid(mo.forward(params, x)[0][0, 0])
    want = -np.log(1 - d) + 0.05 * (-np.mean(np.abs(F * v)))
    np.testing.assert_allclose(ro.reward(m, params, q, q_ref, F, v, 0.05), want, rtol=1e-13)

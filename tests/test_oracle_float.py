"""Pins of the oracle's free (floating) root against closed forms and invariants.

The free root joins body 0 to the world by six DoFs: translations of its origin along world
x, y, z (q = position, qd = velocity), then rotations about world x, y, z through the origin
(qd = world angular velocity, q = rotation vector of the orientation, advanced by the
exponential map).  Pins: the 6 x 6 mass matrix of one rigid body (kinetic energy of a body whose
COM is offset from its origin), the Newton-Euler bias of one body, the exact semi-implicit
Euler trajectory of a free fall with a torque-free spinning sphere, the rotation-vector update
against a library composition of rotations, and Newton's second law for the whole floating
skeleton (the centre of mass of the muscle-driven body accelerates with g when nothing touches
the ground, whatever the muscles do).
"""
import copy

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from oracle import oracle as ora
from paper_2603_29332_b300 import modelgen as mg


def _skew(c):
    return np.array([[0, -c[2], c[1]], [c[2], 0, -c[0]], [-c[1], c[0], 0]])


def _one_body(com=(0.05, -0.02, 0.1), inertia=(0.02, 0.03, 0.04, 0.003, -0.002, 0.001), mass=3.0, g=(0, 0, -9.81)):
    base = mg.make_model("one", [-1], [1], [[0.1, 0.2, 1.0]], [mass], [com], [inertia], [[0, 0, 1]],
                         gravity=list(g))
    return mg.with_free_root(base)


def _inertia_world(model, q):
    R = Rotation.from_rotvec(q[3:6]).as_matrix()
    xx, yy, zz, xy, xz, yz = model.body_inertia[0]
    Ib = np.array([[xx, xy, xz], [xy, yy, yz], [xz, yz, zz]])
    return R, R @ Ib @ R.T, R @ model.body_com[0]


def test_single_free_body_mass_matrix_closed_form():
    # T = 1/2 m |v + w x c|^2 + 1/2 w^T Ic w  =>  M = [[m 1, -m [c]x], [m [c]x, Ic + m [c]x^T [c]x]]
    model = _one_body()
    rng = np.random.default_rng(1)
    for _ in range(3):
        q = np.concatenate([rng.normal(size=3), rng.normal(size=3)])
        R, Ic, c = _inertia_world(model, q)
        m = model.body_mass[0]
        Mw = np.block([[m * np.eye(3), -m * _skew(c)], [m * _skew(c), Ic + m * _skew(c).T @ _skew(c)]])
        np.testing.assert_allclose(ora.mass_matrix(model, q), Mw, rtol=0, atol=1e-13)
        np.testing.assert_allclose(ora.mass_matrix_jac(model, q), Mw, rtol=0, atol=1e-13)


def test_single_free_body_bias_newton_euler_closed_form():
    # with q_dd = 0: a_com = w x (w x c) - g; F = m a_com; moment about the origin
    # N = w x Ic w + c x F  (Newton's and Euler's equations of one rigid body)
    model = _one_body()
    rng = np.random.default_rng(2)
    g = model.gravity
    for _ in range(3):
        q = np.concatenate([rng.normal(size=3), rng.normal(size=3)])
        qd = rng.normal(size=6)
        R, Ic, c = _inertia_world(model, q)
        m, w = model.body_mass[0], qd[3:]
        F = m * (np.cross(w, np.cross(w, c)) - g)
        N = np.cross(w, Ic @ w) + np.cross(c, F)
        np.testing.assert_allclose(ora.rnea(model, q, qd, np.zeros(6)), np.concatenate([F, N]), rtol=0, atol=1e-12)


def test_free_fall_and_torque_free_sphere_exact_trajectory():
    # a sphere (isotropic inertia, COM at its origin) keeps its angular velocity; semi-implicit
    # Euler of a constant acceleration: v_N = v0 + N dt g, p_N = p0 + N dt v0 + dt^2 g N (N + 1) / 2,
    # and the rotation vector after N steps about a fixed axis is N dt w
    model = _one_body(com=(0, 0, 0), inertia=(0.02, 0.02, 0.02, 0, 0, 0))
    om = ora.OracleModel(model)
    dt, N = 1e-3, 200
    v0, w0 = np.array([0.3, -0.2, 1.5]), np.array([0.4, 1.1, -0.7])
    q = np.zeros((1, 6)); qd = np.concatenate([v0, w0])[None]
    q, qd, *_ = ora.step(om, dt, q, qd, np.zeros((1, 0)), np.zeros((1, 0)), N)
    g = model.gravity
    np.testing.assert_allclose(qd[0, :3], v0 + N * dt * g, rtol=0, atol=1e-12)
    np.testing.assert_allclose(q[0, :3], N * dt * v0 + dt * dt * g * N * (N + 1) / 2, rtol=0, atol=1e-12)
    np.testing.assert_allclose(qd[0, 3:], w0, rtol=0, atol=1e-12)
    np.testing.assert_allclose(q[0, 3:], N * dt * w0, rtol=0, atol=1e-12)


def test_rotation_vector_update_composes_rotations():
    model = _one_body()
    rng = np.random.default_rng(3)
    for _ in range(5):
        r = rng.normal(size=3)
        r *= rng.uniform(0.1, 3.0) / np.linalg.norm(r)
        w = rng.normal(size=3) * 2.0
        dt = 0.01
        q = np.concatenate([rng.normal(size=3), r])
        qd = np.concatenate([rng.normal(size=3), w])
        out = ora.integrate_q(model, dt, q, qd)
        np.testing.assert_allclose(out[:3], q[:3] + dt * qd[:3], rtol=0, atol=1e-15)
        want = Rotation.from_rotvec(dt * w) * Rotation.from_rotvec(r)     # world angular velocity: left product
        np.testing.assert_allclose(Rotation.from_rotvec(out[3:]).as_matrix(), want.as_matrix(), rtol=0, atol=1e-13)
        assert np.linalg.norm(out[3:]) <= np.pi + 1e-12


def test_whole_floating_body_com_accelerates_with_gravity():
    # Newton's second law for the whole skeleton: with no contact, muscle, limit and damping
    # forces are internal, so m_total * a_com = m_total * g.  a_com by a central second difference
    # of the COM along q(t) = q + t qd + t^2 / 2 q_dd (valid with the root at zero rotation and
    # zero angular velocity, where the rotation vector's derivatives are w and dw/dt)
    base = copy.copy(mg.config_model("c1_whole"))
    base.sphere_body = np.zeros(0, np.int32)
    base.sphere_pos = np.zeros((0, 3))
    base.sphere_radius = np.zeros(0)
    model = mg.with_free_root(base)
    om = ora.OracleModel(model)
    n, m = model.n_dofs, model.n_muscles
    mass = model.body_mass.sum()
    rng = np.random.default_rng(5)

    def com(q):
        Rb, pb, _, _ = ora.fk(om, q)
        c = np.einsum("bij,bj->bi", Rb, model.body_com) + pb
        return (model.body_mass[:, None] * c).sum(0) / mass

    for trial in range(2):
        q = rng.uniform(-0.8, 0.8, n)
        q[3:6] = 0.0
        qd = rng.normal(0, 1.5, n)
        qd[3:6] = 0.0
        act = rng.uniform(0, 1, m)
        r = ora.evaluate(om, 1e-3, q, qd, act, act)
        assert r["status"] == 0 and np.abs(r["tau_m"]).max() > 1.0
        qt = lambda t: q + t * qd + 0.5 * t * t * r["qdd"]
        d2 = lambda h: (com(qt(h)) - 2 * com(qt(0.0)) + com(qt(-h))) / (h * h)
        # accelerations reach 1e4 rad/s^2 here: Richardson extrapolation of the O(h^2) difference
        acc = (4 * d2(5e-5) - d2(1e-4)) / 3
        np.testing.assert_allclose(acc, model.gravity, rtol=0, atol=1e-3)
        # a dropped root coupling term (e.g. the translation rows of M) would break it
        assert np.abs(r["qdd"][:3] - model.gravity).max() > 1e-3

"""Pins of the FP64 oracle against what the paper and the mathematics fix (CPU only).

Each test checks the oracle against something other than itself: values the paper prints
(tests/golden/paper_constants.json), closed forms, finite differences, a second formulation,
textbook two-link dynamics, equilibria, or invariants of the integrator.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import oracle as ora
from paper_2603_29332_b300 import modelgen as mg
from tests import handmodels as hm

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))


# ----------------------------------------------------------------------------- Eq. 2 activation
def test_model_defaults_match_paper_constants():
    m = mg.config_model("c0_tiny")
    assert m.tau_act == pytest.approx(GOLD["tau_act_s"])
    assert m.tau_deact == pytest.approx(GOLD["tau_deact_s"])


def test_activation_rates_at_chosen_points():
    ta, td = GOLD["tau_act_s"], GOLD["tau_deact_s"]
    a0, a1 = GOLD["tau_act_factor"]
    # u > act: tau = ta (0.5 + 1.5 act)
    for u, a in ((1.0, 0.0), (0.9, 0.2), (0.6, 0.5)):
        assert ora.act_rate(u, a) == pytest.approx((u - a) / (ta * (a0 + a1 * a)), rel=1e-14)
    # u <= act (including the tie): tau = td / (0.5 + 1.5 act)
    for u, a in ((0.0, 1.0), (0.3, 0.5), (0.0, 0.2)):
        assert ora.act_rate(u, a) == pytest.approx((u - a) / (td / (a0 + a1 * a)), rel=1e-14)
    assert ora.act_rate(0.4, 0.4) == 0.0
    # the tie takes the deactivation branch: just below/at the tie the rate is continuous from below
    eps = 1e-9
    assert ora.act_rate(0.4 - eps, 0.4) == pytest.approx(-eps * (a0 + a1 * 0.4) / td, rel=1e-6)


def _integrate_activation(u, a0, t_end, dt):
    """Drive the oracle's own substep activation update (through ora_eval) with constant u,
    on a grid that ends exactly at t_end."""
    m = hm.hinge_muscle()
    om = ora.OracleModel(m)
    a = np.array([a0])
    q = np.zeros(2); qd = np.zeros(2)
    n = max(1, int(math.ceil(t_end / dt - 1e-9)))
    dt = t_end / n
    for _ in range(n):
        a = ora.evaluate(om, dt, q, qd, a, np.array([u]))["act_next"]
    return float(a[0])


def test_activation_closed_form_full_excitation():
    # u = 1: separable ODE, t(a) = tau_a [ -1.5 a - 2 ln(1 - a) ]
    ta = GOLD["tau_act_s"]
    a_target = 0.6
    t = ta * (-1.5 * a_target - 2.0 * math.log(1.0 - a_target))
    errs = [abs(_integrate_activation(1.0, 0.0, t, dt) - a_target) for dt in (1e-4, 5e-5, 2.5e-5)]
    # explicit Euler converges to the closed form at first order
    assert errs[2] < 1e-3
    assert 0.4 < errs[1] / errs[0] < 0.6 and 0.4 < errs[2] / errs[1] < 0.6


def test_activation_closed_form_relaxation():
    # u = 0: -t / tau_d = 2 ln(a / (0.5 + 1.5 a)) - 2 ln(a0 / (0.5 + 1.5 a0))
    td = GOLD["tau_deact_s"]
    a0 = 0.9
    t = 0.03
    g = lambda a: 2.0 * math.log(a / (0.5 + 1.5 * a))
    # solve for a(t) by bisection on the closed form
    lo, hi = 1e-9, a0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if -(g(mid) - g(a0)) * td > t:
            lo = mid
        else:
            hi = mid
    exact = 0.5 * (lo + hi)
    e1, e2, e3 = [abs(_integrate_activation(0.0, a0, t, dt) - exact) for dt in (1e-4, 5e-5, 2.5e-5)]
    assert e3 < 1e-3
    assert 0.4 < e2 / e1 < 0.6 and 0.4 < e3 / e2 < 0.6


def test_activation_clamped_to_unit_interval():
    # excitations outside [0, 1] are clamped (action space [0, 1]^700); activation stays in [0, 1]
    assert 0.0 <= _integrate_activation(5.0, 0.99, 0.05, 1e-3) <= 1.0
    assert _integrate_activation(-3.0, 0.01, 0.05, 1e-3) >= 0.0
    assert _integrate_activation(5.0, 0.0, 0.001, 1e-3) == pytest.approx(_integrate_activation(1.0, 0.0, 0.001, 1e-3))


# ----------------------------------------------------------------------------- Eq. 1 Hill curves
def test_hill_curve_fixed_points():
    assert ora.fl(1.0) == 1.0
    assert ora.fv(0.0) == 1.0
    assert ora.fv(-1.0) == 0.0
    assert ora.fv(-1.5) == 0.0
    assert ora.fp(1.0) == 0.0
    assert ora.fp(0.7) == 0.0
    assert ora.fp(1.6) == pytest.approx(1.0, rel=1e-14)
    assert ora.fv(1e6) == pytest.approx(1.4, rel=1e-5)          # eccentric asymptote
    assert ora.fl(0.8) == pytest.approx(ora.fl(1.2), rel=1e-14)   # symmetric about optimum


def test_hill_curves_continuity_and_slope():
    h = 1e-7
    # f_p: value and slope continuous at l = 1.6, value continuous at l = 1
    assert ora.fp(1.6 + h) == pytest.approx(ora.fp(1.6 - h), abs=1e-5)
    s_left = (ora.fp(1.6 - h) - ora.fp(1.6 - 2 * h)) / h
    s_right = (ora.fp(1.6 + 2 * h) - ora.fp(1.6 + h)) / h
    assert s_left == pytest.approx(s_right, rel=1e-4)
    assert ora.fp(1.0 + h) == pytest.approx(0.0, abs=1e-6)
    # f_v: value and slope continuous at v = 0 (slope 5 on both sides), value at v = -1
    assert (ora.fv(h) - ora.fv(0)) / h == pytest.approx(5.0, rel=1e-5)
    assert (ora.fv(0) - ora.fv(-h)) / h == pytest.approx(5.0, rel=1e-5)
    # the analytic derivative used by the implicit step matches central differences
    for v in (-0.9, -0.5, -0.1, 0.05, 0.3, 2.0):
        fd = (ora.fv(v + 1e-6) - ora.fv(v - 1e-6)) / 2e-6
        assert ora.dfv(v) == pytest.approx(fd, rel=1e-6)
    # monotone
    vs = np.linspace(-1, 3, 400)
    assert np.all(np.diff([ora.fv(v) for v in vs]) > 0)


def test_force_composition_eq1():
    """F = F_max f_p at act = 0; F = F_max at l_m = 1, v_m = 0, act = 1 (Eq. 1)."""
    m = hm.hinge_muscle()
    om = ora.OracleModel(m)
    fmax = m.muscle_fmax[0]
    r = ora.evaluate(om, 1e-3, np.zeros(2), np.zeros(2), np.array([1.0]), np.array([1.0]))
    assert r["lm"][0] == pytest.approx(1.0, abs=1e-14) and r["vm"][0] == 0.0
    assert r["force"][0] == pytest.approx(fmax, rel=1e-14)
    # stretch the muscle: passive force only when act = 0
    q = np.array([0.0, -0.6])
    r0 = ora.evaluate(om, 1e-3, q, np.zeros(2), np.array([0.0]), np.array([0.0]))
    lm = r0["lm"][0]
    assert lm > 1.0
    assert r0["force"][0] == pytest.approx(fmax * ora.fp(lm), rel=1e-14)
    # and the force uses act at the start of the step, not the updated one
    r1 = ora.evaluate(om, 1e-3, q, np.zeros(2), np.array([0.0]), np.array([1.0]))
    assert r1["force"][0] == r0["force"][0]
    assert r1["act_next"][0] == pytest.approx(1e-3 * 1.0 / (0.010 * 0.5))


# ----------------------------------------------------------------------------- muscle geometry
def test_two_point_muscle_closed_form():
    a, b, h0, h1 = 0.1, 0.12, 0.05, 0.04
    m = hm.hinge_muscle(a, b, h0, h1)
    joint = m.body_offset[1][:2]
    r0 = m.point_pos[0][:2] - joint    # origin relative to the joint (body-0 frame = world)
    r1 = m.point_pos[1][:2]
    for th in (-1.0, -0.3, 0.0, 0.4, 1.1):
        c, s = math.cos(th), math.sin(th)
        Rz = np.array([[c, -s], [s, c]])
        dRz = np.array([[-s, -c], [c, -s]])
        d = Rz @ r1 - r0
        L = math.sqrt(d @ d)
        R = -(d @ (dRz @ r1)) / L                 # R = -dL/dtheta
        Lo, Ro = ora.muscle_geometry(m, np.array([0.0, th]))
        assert Lo[0] == pytest.approx(L, rel=1e-14)
        assert Ro[0, 1] == pytest.approx(R, rel=1e-12, abs=1e-15)
        assert abs(Ro[0, 0]) < 1e-15             # the root hinge moves both points rigidly


@pytest.mark.parametrize("name", ["c0_tiny", "c1_whole"])
def test_moment_arms_are_minus_dL_dq(name):
    m = mg.config_model(name)
    om = ora.OracleModel(m)
    rng = np.random.default_rng(5)
    q = rng.uniform(-0.4, 0.4, size=m.n_dofs)
    L, R = ora.muscle_geometry(om, q)
    h = 1e-5   # FD truncation ~h^2 and FP64 rounding of deep FK chains (~1e-14 m / 2h) both < 1e-8
    cols = range(m.n_dofs) if m.n_dofs < 20 else rng.choice(m.n_dofs, 20, replace=False)
    for d in cols:
        e = np.zeros(m.n_dofs); e[d] = h
        fd = -(ora.muscle_geometry(om, q + e)[0] - ora.muscle_geometry(om, q - e)[0]) / (2 * h)
        np.testing.assert_allclose(R[:, d], fd, rtol=1e-6, atol=2e-8)


def test_zero_moment_arms_outside_spanned_joints():
    m = mg.config_model("c1_whole")
    q = np.random.default_rng(2).uniform(-0.5, 0.5, size=m.n_dofs)
    _, R = ora.muscle_geometry(m, q)
    for k in range(m.n_muscles):
        pts = range(m.muscle_point_start[k], m.muscle_point_start[k + 1])
        bodies = sorted({int(m.point_body[j]) for j in pts})
        origin = int(m.point_body[m.muscle_point_start[k]])
        crossed = set()
        for b in bodies:                              # joints strictly below the origin body
            while b != origin:
                s, c = m.body_dof_start[b], m.body_ndof[b]
                crossed.update(range(s, s + c))
                b = int(m.body_parent[b])
        others = [d for d in range(m.n_dofs) if d not in crossed]
        assert np.abs(R[k, others]).max(initial=0.0) < 1e-12
        assert np.abs(R[k, sorted(crossed)]).max() > 1e-6


def test_muscle_tension_shortens_the_muscle():
    """Sign convention tau = R^T F with R = -dL/dq: a pulling muscle shortens itself."""
    m = hm.hinge_muscle()
    om = ora.OracleModel(m)
    q, qd, act = np.zeros((1, 2)), np.zeros((1, 2)), np.ones((1, 1))
    L0 = ora.muscle_geometry(om, q[0])[0][0]
    for _ in range(20):
        q, qd, act, *_ = ora.step(om, 1e-3, q, qd, act, np.ones((1, 1)), 1)
    assert ora.muscle_geometry(om, q[0])[0][0] < L0 - 1e-4


# ----------------------------------------------------------------------------- equations of motion
def test_single_pendulum_acceleration():
    m = hm.pendulum(2.0, 0.3, 0.05)
    mass, lc, iyy, g = m.body_mass[0], m.body_com[0][0], m.body_inertia[0][1], -m.gravity[2]
    for q in (-0.7, 0.0, 0.5, 1.2):
        for w in (0.0, 3.0):
            qdd = np.linalg.solve(ora.mass_matrix(m, [q]), -ora.rnea(m, [q], [w], [0.0]))
            expect = mass * g * lc * math.cos(q) / (iyy + mass * lc * lc)
            assert qdd[0] == pytest.approx(expect, rel=1e-12)


def test_two_link_textbook_dynamics():
    """Planar two-link arm: M(q) and C(q, qd) in the standard closed form (e.g. Spong)."""
    mdl = hm.two_link(1.5, 0.8, 0.6, 0.25, 0.2, 0.03, 0.02)
    m1, m2 = mdl.body_mass
    l1, lc1, lc2 = mdl.body_offset[1][0], mdl.body_com[0][0], mdl.body_com[1][0]
    i1, i2 = mdl.body_inertia[0][2], mdl.body_inertia[1][2]
    g = -mdl.gravity[1]
    rng = np.random.default_rng(0)
    for _ in range(5):
        q1, q2, w1, w2 = rng.uniform(-2, 2, size=4)
        c2, s2 = math.cos(q2), math.sin(q2)
        M = np.array([[m1 * lc1 ** 2 + m2 * (l1 ** 2 + lc2 ** 2 + 2 * l1 * lc2 * c2) + i1 + i2,
                       m2 * (lc2 ** 2 + l1 * lc2 * c2) + i2],
                      [m2 * (lc2 ** 2 + l1 * lc2 * c2) + i2, m2 * lc2 ** 2 + i2]])
        h = -m2 * l1 * lc2 * s2
        grav = np.array([(m1 * lc1 + m2 * l1) * g * math.cos(q1) + m2 * lc2 * g * math.cos(q1 + q2),
                         m2 * lc2 * g * math.cos(q1 + q2)])
        cor = np.array([h * (2 * w1 * w2 + w2 * w2), -h * w1 * w1])
        q, qd = np.array([q1, q2]), np.array([w1, w2])
        np.testing.assert_allclose(ora.mass_matrix(mdl, q), M, rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(ora.rnea(mdl, q, qd, np.zeros(2)), cor + grav, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("name", ["c0_tiny", "c1_whole"])
def test_mass_matrix_spd_two_formulations_and_tree_sparsity(name):
    m = mg.config_model(name)
    om = ora.OracleModel(m)
    q = mg.initial_state(m, 1, 3)[0][0].astype(np.float64)
    M1 = ora.mass_matrix(om, q)
    M2 = ora.mass_matrix_jac(om, q)
    scale = np.abs(M1).max()
    assert np.abs(M1 - M1.T).max() < 1e-12 * scale
    assert np.abs(M1 - M2).max() < 1e-12 * scale
    assert np.linalg.eigvalsh(M1).min() > 0
    # linearity in qdd: RNEA(q, qd, qdd) - RNEA(q, qd, 0) = M qdd
    rng = np.random.default_rng(1)
    qd, qdd = rng.normal(size=m.n_dofs), rng.normal(size=m.n_dofs)
    lhs = ora.rnea(om, q, qd, qdd) - ora.rnea(om, q, qd, np.zeros(m.n_dofs))
    np.testing.assert_allclose(lhs, M1 @ qdd, rtol=1e-9, atol=1e-9 * scale)
    # M_ij = 0 unless one DoF is an ancestor of the other (branch-induced sparsity)
    dpar = np.full(m.n_dofs, -1)
    for b in range(m.n_bodies):
        s, c, pb = m.body_dof_start[b], m.body_ndof[b], m.body_parent[b]
        dpar[s] = -1 if pb < 0 else m.body_dof_start[pb] + m.body_ndof[pb] - 1
        for j in range(1, c):
            dpar[s + j] = s + j - 1
    anc = np.zeros((m.n_dofs, m.n_dofs), bool)
    for i in range(m.n_dofs):
        j = i
        while j >= 0:
            anc[i, j] = True
            j = dpar[j]
    related = anc | anc.T
    assert np.abs(M1[~related]).max(initial=0.0) < 1e-13 * scale


def test_cholesky_matches_library_solve():
    rng = np.random.default_rng(0)
    A = rng.normal(size=(30, 30)); A = A @ A.T + 30 * np.eye(30)
    b = rng.normal(size=30)
    x, bad = ora.cholesky_solve(A, b)
    assert bad == 0
    np.testing.assert_allclose(x, np.linalg.solve(A, b), rtol=1e-12)
    _, bad = ora.cholesky_solve(-np.eye(3), np.ones(3))
    assert bad == 1


def _energy(mdl, om, q, qd):
    Rb, pb, _, _ = ora.fk(om, q)
    V = 0.0
    for b in range(mdl.n_bodies):
        com = pb[b] + Rb[b] @ mdl.body_com[b]
        V -= mdl.body_mass[b] * (mdl.gravity @ com)
    return 0.5 * qd @ ora.mass_matrix(om, q) @ qd + V


def test_semi_implicit_euler_energy_bounded_for_constant_inertia():
    """A single pendulum has a constant mass matrix, so semi-implicit Euler is the symplectic Euler
    map: over 10^4 steps the energy error stays bounded and shows no secular drift."""
    mdl = hm.pendulum()
    om = ora.OracleModel(mdl)
    q, qd, act = np.array([[1.0]]), np.zeros((1, 1)), np.zeros((1, 0))
    E0 = _energy(mdl, om, q[0], qd[0])
    es = []
    for t in range(100):
        q, qd, act, *_ = ora.step(om, 1e-3, q, qd, act, np.zeros((1, 0)), 100)
        es.append(_energy(mdl, om, q[0], qd[0]) - E0)
    es = np.array(es)
    scale = mdl.body_mass[0] * 9.81 * mdl.body_com[0][0]
    assert np.abs(es).max() < 2e-2 * scale
    assert abs(es[-30:].mean() - es[:30].mean()) < 2e-3 * scale


def test_energy_error_vanishes_at_first_order():
    """For a chain (configuration-dependent M) the energy error over a fixed time shrinks linearly
    with dt: the bias forces and mass matrix are consistent with the Lagrangian."""
    mdl = hm.chain(3, seed=4)
    om = ora.OracleModel(mdl)
    errs = []
    for dt in (1e-3, 5e-4, 2.5e-4):
        q, qd, act = np.array([[0.4, -0.3, 0.2]]), np.zeros((1, 3)), np.zeros((1, 0))
        E0 = _energy(mdl, om, q[0], qd[0])
        q, qd, act, *_ = ora.step(om, dt, q, qd, act, np.zeros((1, 0)), int(round(0.4 / dt)))
        errs.append(abs(_energy(mdl, om, q[0], qd[0]) - E0))
    assert errs[2] < 2e-3 * sum(mdl.body_mass) * 9.81
    assert 0.35 < errs[1] / errs[0] < 0.65 and 0.35 < errs[2] / errs[1] < 0.65


def test_root_momentum_conserved_without_gravity():
    """Zero gravity, vertical root hinge: the generalised momentum (M qd)_0 is constant."""
    mdl = hm.chain(4, seed=2, gravity=False, root_axis=(0, 0, 1))
    om = ora.OracleModel(mdl)
    q, qd, act = np.array([[0.0, 0.5, -0.4, 0.3]]), np.array([[1.0, -2.0, 0.5, 1.5]]), np.zeros((1, 0))
    p0 = (ora.mass_matrix(om, q[0]) @ qd[0])[0]
    for _ in range(40):
        q, qd, act, *_ = ora.step(om, 2e-4, q, qd, act, np.zeros((1, 0)), 50)
    p1 = (ora.mass_matrix(om, q[0]) @ qd[0])[0]
    assert p1 == pytest.approx(p0, rel=2e-3)


def test_first_substep_is_semi_implicit_euler():
    mdl = hm.pendulum()
    om = ora.OracleModel(mdl)
    q0 = 0.3
    qdd0 = ora.evaluate(om, 1e-3, [q0], [0.0], np.zeros(0), np.zeros(0))["qdd"][0]
    q, qd, *_ = ora.step(om, 1e-3, [[q0]], [[0.0]], np.zeros((1, 0)), np.zeros((1, 0)), 1)
    assert qd[0, 0] == pytest.approx(1e-3 * qdd0, rel=1e-14)
    assert q[0, 0] == pytest.approx(q0 + 1e-6 * qdd0, rel=1e-14)


# ----------------------------------------------------------------------------- contact and limits
def test_contact_force_closed_form_on_a_rod():
    mdl = hm.rod_on_ground(length=0.5, radius=0.03)
    length, r = mdl.sphere_pos[0][0], mdl.sphere_radius[0]
    assert mdl.body_offset[0][2] == r
    k, c, mu, eps = mdl.contact_k, mdl.contact_c, mdl.contact_mu, mdl.contact_eps
    for q, w in ((0.01, 0.0), (0.02, 0.3), (0.005, -0.2), (-0.01, 0.5)):
        tau, D, fs = ora.contact(mdl, [q], [w])
        rel = np.array([length * math.cos(q), 0.0, -length * math.sin(q) - r])   # contact point - joint
        v = np.cross([0.0, w, 0.0], rel)
        depth = length * math.sin(q)
        fn = k * depth - c * v[2]
        if depth <= 0 or fn <= 0:
            assert tau[0] == 0.0 and np.all(fs == 0)
            continue
        ft = -mu * fn * v[0] / math.sqrt(v[0] ** 2 + eps ** 2)
        F = np.array([ft, 0.0, fn])
        np.testing.assert_allclose(fs[0], F, rtol=1e-12)
        assert tau[0] == pytest.approx(np.cross(rel, F)[1], rel=1e-12)
        # implicit damping: J^T diag(mu fn / s, mu fn / s, c) J with J = d v / d w
        J = np.cross([0.0, 1.0, 0.0], rel)
        dd = np.array([mu * fn / math.sqrt(v[0] ** 2 + eps ** 2)] * 2 + [c])
        assert D[0, 0] == pytest.approx(J @ (dd * J), rel=1e-12)


def test_contact_static_penetration():
    """A rod resting on its tip sphere settles where k * depth * l = m g l_c."""
    mdl = hm.rod_on_ground(mass=1.2, lc=0.25, length=0.5)
    mass, lc, length, g = mdl.body_mass[0], mdl.body_com[0][0], mdl.sphere_pos[0][0], -mdl.gravity[2]
    om = ora.OracleModel(mdl)
    q, qd, act = np.zeros((1, 1)), np.zeros((1, 1)), np.zeros((1, 0))
    for _ in range(30):
        q, qd, act, *_ = ora.step(om, 1e-3, q, qd, act, np.zeros((1, 0)), 100)
    depth = length * math.sin(q[0, 0])
    # torque balance at the tilt: fn * l cos q = m g lc cos q
    assert depth == pytest.approx(mass * g * lc / (mdl.contact_k * length), rel=1e-6)
    assert abs(qd[0, 0]) < 1e-9


def _limit_phi(x, delta):
    """Spring shape of the limit penalty: x^2 / (2 delta) up to delta, then x - delta / 2."""
    return 0.5 * x * x / delta if (delta > 0 and x < delta) else x - 0.5 * delta


def _limit_pendulum(name, k, c, delta):
    base = hm.pendulum(mass=1.0, lc=0.1)
    return base, mg.make_model(name, base.body_parent, base.body_ndof, base.body_offset, base.body_mass,
                               base.body_com, base.body_inertia, base.dof_axis, dof_limit=[[-1.0, 0.0]],
                               limit_k=k, limit_c=c, limit_delta=delta)


@pytest.mark.parametrize("k, delta", [(100.0, 0.0), (100.0, 0.004), (100.0, 0.05), (4000.0, 0.01)])
def test_joint_limit_static_deflection(k, delta):
    """A horizontal pendulum held by its upper limit at 0 rests where the limit spring balances
    gravity, k_l phi(q) = m g lc cos q, phi the spring shape (linear past the onset width delta,
    quadratic inside it); the implicit treatment changes the transient, not the equilibrium.
    The cases put the rest point past the onset (delta = 0.004), inside it (0.05) and at a
    stiffness where it sits in the quadratic part (k = 4000)."""
    base, mdl = _limit_pendulum("lim", k, 1.0, delta)
    mass, lc, g = base.body_mass[0], base.body_com[0][0], -base.gravity[2]
    assert mdl.limit_k == k
    om = ora.OracleModel(mdl)
    q, qd, act = np.zeros((1, 1)), np.zeros((1, 1)), np.zeros((1, 0))
    for _ in range(60):
        q, qd, act, *_ = ora.step(om, 1e-3, q, qd, act, np.zeros((1, 0)), 100)
    qs = q[0, 0]
    assert qs > 0
    delta = mdl.limit_delta   # the model's FP32 value
    # closed-form inverse of the spring shape, iterated on the gravity torque's cos q
    x = 0.0
    for _ in range(200):
        tq = mass * g * lc * math.cos(x) / mdl.limit_k
        x = (tq + 0.5 * delta) if (delta == 0 or tq >= 0.5 * delta) else math.sqrt(2.0 * delta * tq)
    assert qs == pytest.approx(x, rel=1e-6)
    inside = delta > 0 and x < delta
    assert inside == (mdl.limit_delta > 0.04 or k == 4000.0)


@pytest.mark.parametrize("q, delta", [(0.3, 0.0), (0.3, 0.01), (0.004, 0.01), (-1.006, 0.01)])
def test_implicit_limit_penalty_is_backward_euler_of_the_spring_damper(q, delta):
    """Outside a limit the penalty is the first-order prediction at the end of the step: the
    solved q_dd satisfies M q_dd + C = +-k_l [phi(x) + psi(x) dt qd'] - c_l psi(x) qd', with
    qd' = qd + dt q_dd, x the excess past the limit, psi = phi' (1 past the onset width).  The
    cases: past the onset (plain penalty and smooth onset), inside the onset and below the
    lower limit."""
    base, mdl = _limit_pendulum("lim2", 5000.0, 20.0, delta)
    om = ora.OracleModel(mdl)
    dt, qd = 1e-3, 2.0
    r = ora.evaluate(om, dt, [q], [qd], np.zeros(0), np.zeros(0))
    xdd = r["qdd"][0]
    qd1 = qd + dt * xdd
    lhs = r["M"][0, 0] * xdd + r["bias"][0]
    upper = q > 0.0
    x = q - 0.0 if upper else -1.0 - q
    delta = mdl.limit_delta   # the model's FP32 value
    psi = min(x / delta, 1.0) if delta > 0 else 1.0
    # the spring's first-order Taylor expansion in the excess at the end of the step
    x1 = x + (dt * qd1 if upper else -dt * qd1)
    spring = mdl.limit_k * (_limit_phi(x, delta) + psi * (x1 - x))
    want = (-spring if upper else spring) - mdl.limit_c * psi * qd1
    assert lhs == pytest.approx(want, rel=1e-12)
    # unconditionally stable: a very stiff limit on a light pendulum does not blow up
    q_, qd_, act = np.array([[0.5]]), np.zeros((1, 1)), np.zeros((1, 0))
    for _ in range(20):
        q_, qd_, act, *_ = ora.step(om, 1e-2, q_, qd_, act, np.zeros((1, 0)), 10)
    assert abs(q_[0, 0]) < 0.05 and np.isfinite(qd_[0, 0])


def test_limit_penalty_is_continuous_at_the_limit_and_at_the_onset_width():
    """With a smooth onset the limit torque at fixed velocity and its implicit coefficient (the
    diagonal added to M) are continuous in q at the limit and at the end of the onset, and their
    slope in q at the onset's end matches from both sides (C1 spring); the plain penalty
    (delta = 0) jumps in the implicit coefficient at the limit by dt (dt k_l + c_l)."""
    dt, qd, k, c, delta = 1e-3, 0.7, 1e5, 300.0, 0.01

    def parts(mdl, q):
        r = ora.evaluate(ora.OracleModel(mdl), dt, [q], [qd], np.zeros(0), np.zeros(0))
        return r["tau_l"][0], r["A"][0, 0] - r["M"][0, 0]

    _, smooth = _limit_pendulum("lim3", k, c, delta)
    _, plain = _limit_pendulum("lim4", k, c, 0.0)
    h = 1e-9
    for edge in (0.0, delta):
        (t0, a0), (t1, a1) = parts(smooth, edge - h), parts(smooth, edge + h)
        assert abs(t1 - t0) < 1e-3 and abs(a1 - a0) < 1e-6
    # the spring's slope at the end of the onset: k_l from both sides (torque at qd = 0)
    _, still = _limit_pendulum("lim5", k, c, delta)
    r = lambda q: ora.evaluate(ora.OracleModel(still), dt, [q], [0.0], np.zeros(0), np.zeros(0))["tau_l"][0]
    e = 1e-6
    left = (r(delta) - r(delta - e)) / e
    right = (r(delta + e) - r(delta)) / e
    assert left == pytest.approx(-k, rel=1e-3) and right == pytest.approx(-k, rel=1e-6)
    (_, a0), (_, a1) = parts(plain, -h), parts(plain, h)
    assert a1 - a0 == pytest.approx(dt * (dt * k + c), rel=1e-9)


def test_implicit_muscle_damping_is_the_force_velocity_jacobian():
    """(A - M) / dt = -d tau_m / d qd (central differences), C0 has no contact or limits."""
    m = mg.config_model("c0_tiny")
    om = ora.OracleModel(m)
    rng = np.random.default_rng(7)
    q = rng.uniform(-0.3, 0.3, size=m.n_dofs)
    qd = rng.normal(scale=0.5, size=m.n_dofs)
    act = rng.uniform(0.1, 0.9, size=m.n_muscles)
    exc = np.zeros(m.n_muscles)
    dt = 1e-3
    r = ora.evaluate(om, dt, q, qd, act, exc)
    D = (r["A"] - r["M"]) / dt
    h = 1e-7
    for d in range(m.n_dofs):
        e = np.zeros(m.n_dofs); e[d] = h
        tp = ora.evaluate(om, dt, q, qd + e, act, exc)["tau_m"]
        tm = ora.evaluate(om, dt, q, qd - e, act, exc)["tau_m"]
        np.testing.assert_allclose(D[:, d], -(tp - tm) / (2 * h), rtol=1e-5, atol=1e-6 * np.abs(D).max())


def test_step_matches_eval_solution():
    """The solve result equals (M + dt D)^-1 (tau - C) by a library solve."""
    m = mg.config_model("c1_whole")
    om = ora.OracleModel(m)
    q, qd, act = mg.initial_state(m, 1, 0)
    rng = np.random.default_rng(0)
    qd = rng.normal(scale=0.3, size=m.n_dofs)
    act = rng.uniform(0, 1, m.n_muscles)
    r = ora.evaluate(om, 1e-3, q[0], qd, act, rng.uniform(0, 1, m.n_muscles))
    assert r["status"] == 0
    np.testing.assert_allclose(r["qdd"], np.linalg.solve(r["A"], r["rhs"]), rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(r["rhs"], r["tau_m"] + r["tau_c"] + r["tau_l"] - r["bias"], rtol=1e-14, atol=1e-10)


def test_sliding_ball_decelerates_with_smoothed_coulomb_friction():
    """A ball resting on the ground at its static penetration m g / k and sliding at v: the
    friction force is mu f_n v / sqrt(v^2 + eps^2) with f_n = m g, so (explicit damping) the
    horizontal acceleration is -mu g v / sqrt(v^2 + eps^2), about -mu g for v >> eps; the
    vertical one vanishes; the torque r x F about the centre spins the ball up."""
    mdl = hm.free_ball()
    m, r, g = mdl.body_mass[0], mdl.sphere_radius[0], -mdl.gravity[2]
    k, mu, eps = mdl.contact_k, mdl.contact_mu, mdl.contact_eps
    om = ora.OracleModel(mdl, implicit_damping=False)
    I = mdl.body_inertia[0][0]
    for v in (0.05, 0.5, 3.0):
        q = np.zeros(6)
        q[2] = -m * g / k                        # static penetration
        qd = np.zeros(6)
        qd[0] = v
        qdd = ora.evaluate(om, 1e-3, q, qd, np.zeros(0), np.zeros(0))["qdd"]
        ax = -mu * g * v / math.sqrt(v * v + eps * eps)
        assert qdd[0] == pytest.approx(ax, rel=1e-9)
        assert abs(qdd[2]) < 1e-9 * g and abs(qdd[1]) < 1e-12
        # friction -x applied at the sphere's lowest point, r below the centre: +y spin
        assert qdd[4] == pytest.approx(-r * m * ax / I, rel=1e-9)
    assert abs(ax + mu * g) < 2e-3 * mu * g       # v = 3 m/s >> eps: about mu g


def test_dropped_ball_follows_the_damped_oscillator_in_contact():
    """A ball touching the ground with downward speed v0: in contact m z'' = k (r - z) - c z' - m g,
    a linear oscillator about the equilibrium z_eq = r - m g / k, here overdamped (zeta ~1.1),
    z - z_eq = A e^{s1 t} + B e^{s2 t}.  The oracle's semi-implicit Euler with the damping taken
    implicitly converges to it at first order in dt."""
    mdl = hm.free_ball()
    m, r, g = mdl.body_mass[0], mdl.sphere_radius[0], -mdl.gravity[2]
    k, c = mdl.contact_k, mdl.contact_c
    om = ora.OracleModel(mdl)
    v0, T = -0.2, 0.01
    s1, s2 = np.roots([m, c, k])
    assert np.all(np.isreal([s1, s2])) and s1.real < 0 and s2.real < 0
    s1, s2 = float(np.real(s1)), float(np.real(s2))
    x0 = m * g / k                               # z(0) - z_eq with z(0) = r (origin at height r)
    B = (v0 - s1 * x0) / (s2 - s1)
    A = x0 - B
    zT = (r - m * g / k) + A * math.exp(s1 * T) + B * math.exp(s2 * T)
    errs = []
    for dt in (1e-5, 5e-6):
        q, qd = np.zeros((1, 6)), np.zeros((1, 6))
        qd[0, 2] = v0
        n = int(round(T / dt))
        q, qd, *_ = ora.step(om, dt, q, qd, np.zeros((1, 0)), np.zeros((1, 0)), n)
        errs.append(abs((r + q[0, 2]) - zT))
        assert abs(q[0, 0]) < 1e-15 and abs(qd[0, 4]) < 1e-12   # no friction, no spin
    assert errs[0] < 2e-6 and errs[0] / errs[1] == pytest.approx(2.0, rel=0.15)

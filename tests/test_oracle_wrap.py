"""Pins of the oracle's wrapping cylinders: closed forms of the wrapped length, the switch to the
straight segment, and moment arms against central differences of the length."""
import numpy as np
import pytest

from oracle import oracle as ora
from paper_2603_29332_b300 import modelgen as mg


def _pts(rho, psi, r, zp=0.0, zs=0.0):
    P = np.array([rho, 0.0, zp])
    S = np.array([rho * np.cos(psi), rho * np.sin(psi), zs])
    return P, S


@pytest.mark.parametrize("rho,psi,r", [(0.1, 2.8, 0.03), (0.08, 1.9, 0.05), (0.2, 3.0, 0.03)])
def test_wrapped_length_closed_form(rho, psi, r):
    # two points at distance rho from the axis, psi apart around it: tangents 2 sqrt(rho^2 - r^2)
    # plus the arc r (psi - 2 acos(r / rho)) once the chord passes inside the cylinder
    assert psi > 2 * np.arccos(r / rho)
    P, S = _pts(rho, psi, r)
    L, wraps, Q, T = ora.wrap_cylinder(P, S, np.zeros(3), np.array([0, 0, 1.0]), r)
    assert wraps
    want = 2 * np.sqrt(rho ** 2 - r ** 2) + r * (psi - 2 * np.arccos(r / rho))
    np.testing.assert_allclose(L, want, rtol=1e-13)
    np.testing.assert_allclose([np.hypot(*Q[:2]), np.hypot(*T[:2])], [r, r], rtol=1e-13)   # on the surface
    # with an axial offset the unrolled path is straight: sqrt(l^2 + dz^2)
    P, S = _pts(rho, psi, r, zp=-0.02, zs=0.05)
    L, wraps, Q, T = ora.wrap_cylinder(P, S, np.zeros(3), np.array([0, 0, 1.0]), r)
    np.testing.assert_allclose(L, np.sqrt(want ** 2 + 0.07 ** 2), rtol=1e-13)
    # tangent points split the axial rise in proportion to the in-plane path
    lp = np.sqrt(rho ** 2 - r ** 2)
    np.testing.assert_allclose(Q[2], -0.02 + 0.07 * lp / want, rtol=1e-12)


def test_straight_when_the_chord_misses_or_a_point_is_inside():
    rho, r = 0.1, 0.03
    psi = 0.9 * 2 * np.arccos(r / rho)          # the chord stays outside the cylinder
    P, S = _pts(rho, psi, r)
    L, wraps, _, _ = ora.wrap_cylinder(P, S, np.zeros(3), np.array([0, 0, 1.0]), r)
    assert not wraps and L == pytest.approx(np.linalg.norm(S - P), rel=1e-15)
    P, S = _pts(0.02, 2.5, r)                    # P inside: no wrapping
    L, wraps, _, _ = ora.wrap_cylinder(P, S, np.zeros(3), np.array([0, 0, 1.0]), r)
    assert not wraps and L == pytest.approx(np.linalg.norm(S - P), rel=1e-15)


def test_length_is_continuous_at_the_onset_of_wrapping():
    rho, r = 0.1, 0.03
    psi0 = 2 * np.arccos(r / rho)                # chord tangent to the cylinder
    Ls = []
    for psi in (psi0 - 1e-7, psi0 + 1e-7):
        P, S = _pts(rho, psi, r)
        Ls.append(ora.wrap_cylinder(P, S, np.zeros(3), np.array([0, 0, 1.0]), r)[0])
    np.testing.assert_allclose(Ls[0], Ls[1], atol=1e-8)
    np.testing.assert_allclose(Ls[0], 2 * np.sqrt(rho ** 2 - r ** 2), atol=1e-8)


def _coaxial_model(r):
    # body 1 turns about z at x = 0.3; the muscle runs from body 0 to body 1 around a cylinder of
    # radius r on body 1's hinge axis
    rho = 0.08
    return mg.make_model("wrap_hinge", [-1, 0], [1, 1], [[0, 0, 0], [0.3, 0, 0]], [1.0, 1.0],
                         [[0.15, 0, 0], [0.1, 0, 0]], [[0.001, 0.01, 0.01, 0, 0, 0]] * 2, [[0, 0, 1], [0, 0, 1]],
                         muscle_points=[[(0, (0.3 - rho, 0.0, 0.0)), (1, (rho * np.cos(0.5), rho * np.sin(0.5), 0.0))]],
                         muscle_fmax=[1000.0], muscle_lopt=[0.1], gravity=[0.0, 0.0, 0.0],
                         wraps=[(0, 1, 1, (0.0, 0.0, 0.0), (0.0, 0.0, 1.0), r)])


def test_coaxial_cylinder_moment_arm_is_the_radius():
    m = _coaxial_model(0.03)
    r = float(m.wrap_radius[0])
    for q1 in (-0.3, 0.0, 0.2):   # the two points stay more than 2 acos(r / rho) apart: wrapped
        q = np.array([0.0, q1])
        L, R = ora.muscle_geometry(m, q)
        np.testing.assert_allclose(abs(R[0, 1]), r, rtol=1e-12)
        assert R[0, 0] == 0.0                   # body 0's hinge moves both ends together


def test_wrapped_moment_arms_match_central_differences():
    m = mg.config_model("c1_wrap")
    rng = np.random.default_rng(4)
    h = 1e-6
    hit = 0
    for _ in range(3):
        q = rng.uniform(-0.4, 0.4, m.n_dofs)
        L, R = ora.muscle_geometry(m, q)
        for d in rng.choice(m.n_dofs, 12, replace=False):
            e = np.zeros(m.n_dofs)
            e[d] = h
            Lp, _ = ora.muscle_geometry(m, q + e)
            Lm, _ = ora.muscle_geometry(m, q - e)
            fd = -(Lp - Lm) / (2 * h)
            wrapped = m.wrap_muscle
            hit += int(np.count_nonzero(R[wrapped, d]))
            # atol: the model's hinge axes are FP32 unit vectors (unit to ~1e-8), so its rotations
            # are rigid only to that level and L moves by ~1e-8 m/rad with DoFs no muscle crosses
            np.testing.assert_allclose(R[:, d], fd, rtol=0, atol=5e-8)
    assert hit > 0


# ---------------------------------------------------------------- spheres
def _plane_pts(rng, rho_p, rho_s, psi):
    """P, S at distances rho_p, rho_s from the origin, psi apart, in a random plane."""
    u = rng.normal(size=3)
    u /= np.linalg.norm(u)
    v = rng.normal(size=3)
    v -= u * (u @ v)
    v /= np.linalg.norm(v)
    return rho_p * u, rho_s * (np.cos(psi) * u + np.sin(psi) * v), u, v


@pytest.mark.parametrize("rho,psi,r", [(0.1, 2.8, 0.03), (0.08, 1.9, 0.05), (0.2, 3.0, 0.03)])
def test_sphere_wrapped_length_closed_form_in_any_plane(rho, psi, r):
    rng = np.random.default_rng(int(rho * 1000))
    for _ in range(3):
        P, S, u, v = _plane_pts(rng, rho, rho, psi)
        c = rng.normal(size=3) * 0.5
        L, wraps, Q, T = ora.wrap_sphere(P + c, S + c, c, r)
        assert wraps
        want = 2 * np.sqrt(rho ** 2 - r ** 2) + r * (psi - 2 * np.arccos(r / rho))
        np.testing.assert_allclose(L, want, rtol=1e-12)
        n = np.cross(u, v)
        for X in (Q, T):      # tangent points on the sphere, in the plane of P, S and the centre
            np.testing.assert_allclose(np.linalg.norm(X - c), r, rtol=1e-12)
            assert abs((X - c) @ n) < 1e-13
        L2, _, _, _ = ora.wrap_sphere(S + c, P + c, c, r)
        np.testing.assert_allclose(L2, L, rtol=1e-13)


def test_sphere_wrapped_length_against_brute_force_unequal_radii():
    # minimise |P - X(a)| + r |b - a| + |X(b) - S| over the two contact angles on the great
    # circle by brute force (the minimiser is tangent); P and S at different distances
    rng = np.random.default_rng(7)
    r = 0.04
    for rho_p, rho_s, psi in ((0.09, 0.15, 2.6), (0.2, 0.06, 2.9), (0.07, 0.07, 3.1)):
        P, S, u, v = _plane_pts(rng, rho_p, rho_s, psi)
        L, wraps, _, _ = ora.wrap_sphere(P, S, np.zeros(3), r)
        assert wraps
        a = np.linspace(0.0, psi, 2001)
        X = r * (np.cos(a)[:, None] * u + np.sin(a)[:, None] * v)
        dP = np.linalg.norm(X - P, axis=1)
        dS = np.linalg.norm(X - S, axis=1)
        # contact from angle a_i to a_j >= a_i; a straight piece from P to X stays outside the
        # ball when P lies on the outer side of the tangent plane at X: (P - X) . X >= 0
        okP = ((P - X) * X).sum(1) >= 0
        okS = ((S - X) * X).sum(1) >= 0
        cost = dP[:, None] + r * (a[None, :] - a[:, None]) + dS[None, :]
        valid = okP[:, None] & okS[None, :] & (a[None, :] >= a[:, None])
        best = np.min(np.where(valid, cost, np.inf))
        np.testing.assert_allclose(L, best, rtol=2e-6)


def test_sphere_straight_when_the_chord_misses_or_a_point_is_inside():
    rng = np.random.default_rng(3)
    r = 0.03
    P, S, _, _ = _plane_pts(rng, 0.1, 0.1, 0.9 * 2 * np.arccos(r / 0.1))
    L, wraps, _, _ = ora.wrap_sphere(P, S, np.zeros(3), r)
    assert not wraps and L == pytest.approx(np.linalg.norm(S - P), rel=1e-15)
    P, S, _, _ = _plane_pts(rng, 0.02, 0.1, 2.5)
    L, wraps, _, _ = ora.wrap_sphere(P, S, np.zeros(3), r)
    assert not wraps and L == pytest.approx(np.linalg.norm(S - P), rel=1e-15)


def test_sphere_wrapped_moment_arms_match_central_differences():
    m = mg.config_model("c1_wrap_mix")
    assert 0 < int(m.wrap_kind.sum()) < m.wrap_kind.shape[0]
    rng = np.random.default_rng(8)
    h = 1e-6
    hit = 0
    spheres = m.wrap_muscle[m.wrap_kind == 1]
    for _ in range(3):
        q = rng.uniform(-0.4, 0.4, m.n_dofs)
        L, R = ora.muscle_geometry(m, q)
        for d in rng.choice(m.n_dofs, 12, replace=False):
            e = np.zeros(m.n_dofs)
            e[d] = h
            Lp, _ = ora.muscle_geometry(m, q + e)
            Lm, _ = ora.muscle_geometry(m, q - e)
            hit += int(np.count_nonzero(R[spheres, d]))
            np.testing.assert_allclose(R[:, d], -(Lp - Lm) / (2 * h), rtol=0, atol=5e-8)
    assert hit > 0

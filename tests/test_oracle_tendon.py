"""Pins of the oracle's compliant tendon (a reading: the paper's tendon is rigid; the series
elastic tendon follows the damped-equilibrium Hill model of Millard 2013).

What fixes it independently of its own code: the tendon curve's end values and C1 joins; the
fibre velocity of the damped equilibrium against the roots of the quadratics that the two Hill
branches reduce to (the oracle bisects instead); the fixed point of the strain update against
the steady-state equation solved by a library root finder; the stiff-tendon limit, which must
give the rigid-tendon Hill force plus the fibre damper; the implicit terms against finite
differences; and the slack-length reading at q = 0 on the whole body.
"""
import numpy as np
import pytest
from scipy.optimize import brentq

from oracle import oracle as ora
from paper_2603_29332_b300 import modelgen as mg

BETA = ora.TENDON_BETA


def _fd(f, x, h=1e-6):
    return (f(x + h) - f(x - h)) / (2 * h)


def test_tendon_curve_end_values_and_c1_joins():
    assert ora.ft(0.0) == 0.0 and ora.ft(-0.3) == 0.0
    assert ora.ft(1.0) == pytest.approx(1.0, abs=1e-15)
    h = 1e-7
    left = (ora.ft(1.0) - ora.ft(1.0 - h)) / h
    right = (ora.ft(1.0 + h) - ora.ft(1.0)) / h
    assert left == pytest.approx(right, rel=1e-5)
    # slack to taut: zero slope on both sides, the toe rising as (9/2) x^2 / (e^3 - 4)
    assert ora.dft(0.0) == 0.0 and ora.dft(1e-9) == pytest.approx(0.0, abs=1e-7)
    assert ora.ft(1e-3) == pytest.approx(4.5e-6 / (np.e ** 3 - 4), rel=2e-3)
    for x in (0.1, 0.5, 0.9, 1.5, 3.0):
        assert ora.dft(x) == pytest.approx(_fd(ora.ft, x), rel=1e-7)
    for l in (0.4, 0.8, 1.2, 1.5, 1.9):
        assert ora.dfl(l) == pytest.approx(_fd(ora.fl, l), rel=1e-7, abs=1e-9)
        assert ora.dfp(l) == pytest.approx(_fd(ora.fp, l), rel=1e-7, abs=1e-9)


def test_fibre_velocity_matches_the_branch_quadratics():
    """A f_v(v) + beta v + c0 = 0.  A = 0: v = -c0/beta.  c0 = -A: v = 0 (f_v(0) = 1).
    Shortening (-1 <= v <= 0, f_v = (1+v)/(1-4v)): times (1 - 4v) it is the quadratic
    -4 beta v^2 + (A + beta - 4 c0) v + (A + c0) = 0; lengthening (f_v = 1 + 0.4 v/(v + 0.08)):
    times (v + 0.08) it is beta v^2 + (1.4 A + 0.08 beta + c0) v + 0.08 (A + c0) = 0; below
    v = -1 (f_v = 0) the root is -c0/beta."""
    assert ora.fibre_velocity(0.0, 0.37) == pytest.approx(-0.37 / BETA, abs=1e-12)
    assert ora.fibre_velocity(0.8, -0.8) == pytest.approx(0.0, abs=1e-13)
    r = np.random.default_rng(5)
    n_short = n_long = n_low = 0
    for _ in range(300):
        A = r.uniform(0.0, 1.0)
        c0 = r.uniform(-2.5, 1.0)
        v = ora.fibre_velocity(A, c0)
        if c0 - BETA >= 0:                         # g(-1) >= 0: the root is below -1
            want, n_low = -c0 / BETA, n_low + 1
        elif A + c0 >= 0:                          # g(0) >= 0 > g(-1)
            rts = np.roots([-4 * BETA, A + BETA - 4 * c0, A + c0])
            want = [x.real for x in rts if abs(x.imag) < 1e-12 and -1 - 1e-12 <= x.real <= 1e-12][0]
            n_short += 1
        else:
            rts = np.roots([BETA, 1.4 * A + 0.08 * BETA + c0, 0.08 * (A + c0)])
            want = [x.real for x in rts if abs(x.imag) < 1e-12 and x.real > 0][0]
            n_long += 1
        assert v == pytest.approx(want, abs=1e-11), (A, c0)
    assert min(n_short, n_long, n_low) >= 20


def _fixed_point(eps0, lopt, ls, vmax, a, L, Ldot):
    """Strain at which the fibre moves at dL/dt (the strain rate vanishes): solved by brentq."""
    v = Ldot / vmax

    def g(e):
        lm = (L - ls * (1 + e)) / lopt
        return a * ora.fl(lm) * ora.fv(v) + ora.fp(lm) + BETA * v - ora.ft(e / eps0)
    return brentq(g, -0.5, 20 * eps0, xtol=1e-15)


@pytest.mark.parametrize("a,stretch,Ldot", [(0.0, 0.02, 0.0), (0.5, 0.0, 0.0), (1.0, 0.03, 0.0), (0.7, 0.01, -0.2),
                                            (0.3, 0.02, 0.15)])
def test_strain_update_converges_to_the_steady_state(a, stretch, Ldot):
    eps0, lopt, ls = 0.045, 0.12, 0.2
    vmax = 10 * lopt
    L = lopt + ls + stretch
    want = _fixed_point(eps0, lopt, ls, vmax, a, L, Ldot)
    e = 0.0
    for _ in range(4000):
        t = ora.tendon(eps0, lopt, ls, vmax, a, L, Ldot, e, 1e-3)
        e = t["eps_next"]
    assert e == pytest.approx(want, abs=1e-9)
    assert t["vm"] == pytest.approx(Ldot / vmax, abs=1e-7)
    assert t["F"] == pytest.approx(ora.ft(want / eps0), abs=1e-7)


def test_stiff_tendon_gives_the_rigid_force_plus_the_fibre_damper():
    lopt, ls = 0.1, 0.25
    vmax = 10 * lopt
    for a, dL, Ldot in [(0.6, 0.01, 0.0), (1.0, -0.02, -0.3), (0.4, 0.03, 0.2)]:
        L = lopt + ls + dL
        lm_r, vm_r = 1 + dL / lopt, Ldot / vmax
        rigid = a * ora.fl(lm_r) * ora.fv(vm_r) + ora.fp(lm_r) + BETA * vm_r
        for eps0 in (1e-3, 1e-4, 1e-5):
            e = 0.0
            for _ in range(300):
                e = ora.tendon(eps0, lopt, ls, vmax, a, L, Ldot, e, 1e-3)["eps_next"]
            F = ora.tendon(eps0, lopt, ls, vmax, a, L, Ldot, e, 1e-3)["F"]
            assert abs(F - rigid) <= 40 * eps0 + 1e-9, (a, dL, eps0, F, rigid)


def test_implicit_terms_match_finite_differences():
    eps0, lopt, ls, dt = 0.04, 0.15, 0.3, 1e-3
    vmax = 10 * lopt
    r = np.random.default_rng(2)
    n_pos = 0
    for _ in range(60):
        a = r.uniform(0, 1)
        L = lopt + ls + r.uniform(-0.03, 0.05)
        Ldot = r.uniform(-0.5, 0.5)
        e = r.uniform(-0.01, 0.06)
        t = ora.tendon(eps0, lopt, ls, vmax, a, L, Ldot, e, dt)
        vm = lambda x: ora.tendon(eps0, lopt, ls, vmax, a, L, Ldot, x, dt)["vm"]
        dv = _fd(vm, e, 1e-8)
        if t["J"] > 0:
            n_pos += 1
            assert t["J"] == pytest.approx(dv, rel=2e-4, abs=1e-6)
        else:
            assert dv <= 1e-6
        F = lambda x: ora.tendon(eps0, lopt, ls, vmax, a, L, x, e, dt)["F"]
        assert t["dF"] == pytest.approx(_fd(F, Ldot, 1e-7), rel=1e-5, abs=1e-9)
        # the update is one linearly implicit Euler step of d eps/dt = (dL/dt - v_max v_m)/l_s
        rate = (Ldot - vmax * t["vm"]) / ls
        assert t["eps_next"] == pytest.approx(e + dt * rate / (1 + dt * vmax * t["J"] / ls), abs=1e-15)
    assert n_pos >= 30


def test_whole_body_slack_reading_at_the_reference_pose():
    """q = 0 puts every compliant fibre at l_opt with its tendon unstretched: no force at act = 0,
    and under activation the fibres shorten (v_m < 0) and stretch their tendons."""
    m = mg.config_model("c1_whole")
    mt = mg.with_tendons(m, ora.OracleModel(m).L0, seed=3)
    ot = ora.OracleModel(mt)
    on = mt.muscle_tendon_strain > 0
    assert on.sum() >= 300
    n, M = mt.n_dofs, mt.n_muscles
    z = np.zeros(n)
    r0 = ora.evaluate(ot, 1e-3, z, z, np.zeros(M), np.zeros(M))
    np.testing.assert_allclose(r0["lm"][on], 1.0, atol=1e-12)
    np.testing.assert_allclose(r0["force"][on], 0.0, atol=1e-9)
    np.testing.assert_allclose(r0["eps_next"][on], 0.0, atol=1e-15)
    r1 = ora.evaluate(ot, 1e-3, z, z, np.full(M, 0.8), np.zeros(M))
    assert np.all(r1["vm"][on] < 0) and np.all(r1["eps_next"][on] > 0)
    # rigid muscles are untouched by the tendon state
    rr = ora.evaluate(ora.OracleModel(m), 1e-3, z, z, np.full(M, 0.8), np.zeros(M))
    np.testing.assert_array_equal(r1["force"][~on], rr["force"][~on])

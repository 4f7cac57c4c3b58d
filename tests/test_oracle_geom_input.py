"""Pins of the oracle's substep driven by given muscle geometry (a learned J_m(q)).

A learned geometry replaces the via-point lengths L(q) and moment arms R(q) of the equation of
motion (Methods, "Musculoskeletal dynamics": M q_dd + C = J_m^T F + tau_ext) and leaves the rest
of the substep as it is.  The oracle's evaluation with (L, R) given must therefore (a) reduce to
the exact substep when it is given the exact geometry, and (b) move every downstream quantity as
the method's formulas say when the geometry moves: l_m by dL / l_opt (Eq. 1's normalised fibre
length, rigid tendon), v_m by -(dR qd) / v_max, tau_m = R^T F linearly in R at fixed F, and the
implicit muscle damping R^T diag(dF/dLdot) R quadratically in R.
"""
import numpy as np
import pytest

from oracle import oracle as ora
from paper_2603_29332_b300 import modelgen as mg

DT = 1e-3


@pytest.fixture(scope="module")
def tiny():
    model = mg.config_model("c0_tiny")
    om = ora.OracleModel(model)
    rng = np.random.default_rng(31)
    n, m = model.n_dofs, model.n_muscles
    st = dict(q=rng.uniform(-0.3, 0.3, n), qd=rng.normal(0, 1.0, n), act=rng.uniform(0, 1, m),
              exc=rng.uniform(0, 1, m))
    return model, om, st


def test_given_exact_geometry_reproduces_the_exact_substep(tiny):
    model, om, st = tiny
    ex = ora.evaluate(om, DT, st["q"], st["qd"], st["act"], st["exc"])
    gv = ora.evaluate(om, DT, st["q"], st["qd"], st["act"], st["exc"], L=ex["L"], R=ex["R"])
    for k in ("qdd", "force", "lm", "vm", "tau_m", "A", "rhs", "act_next"):
        np.testing.assert_array_equal(gv[k], ex[k], err_msg=k)


def test_length_shift_moves_the_fibre_length_and_the_hill_force(tiny):
    model, om, st = tiny
    ex = ora.evaluate(om, DT, st["q"], np.zeros(model.n_dofs), st["act"], st["exc"])
    k, dL = 5, 0.013
    L = ex["L"].copy()
    L[k] += dL
    gv = ora.evaluate(om, DT, st["q"], np.zeros(model.n_dofs), st["act"], st["exc"], L=L, R=ex["R"])
    lopt, fmax = model.muscle_lopt[k], model.muscle_fmax[k]
    assert gv["lm"][k] == pytest.approx(ex["lm"][k] + dL / lopt, rel=1e-13)
    lm = gv["lm"][k]
    # Eq. 1 at v_m = 0 (qd = 0): F = F_max [act f_l(l_m) f_v(0) + f_p(l_m)], f_v(0) = 1
    assert gv["force"][k] == pytest.approx(fmax * (st["act"][k] * ora.fl(lm) + ora.fp(lm)), rel=1e-13)
    others = np.arange(model.n_muscles) != k
    np.testing.assert_array_equal(gv["force"][others], ex["force"][others])


def test_moment_arm_entry_moves_one_joint_torque_by_force_times_shift(tiny):
    model, om, st = tiny
    zero = np.zeros(model.n_dofs)
    ex = ora.evaluate(om, DT, st["q"], zero, st["act"], st["exc"])
    k = 7
    d = int(np.flatnonzero(np.abs(ex["R"][k]) > 1e-9)[0])
    eps = 0.004
    R = ex["R"].copy()
    R[k, d] += eps
    gv = ora.evaluate(om, DT, st["q"], zero, st["act"], st["exc"], L=ex["L"], R=R)
    np.testing.assert_array_equal(gv["force"], ex["force"])     # qd = 0: F does not see R
    want = ex["tau_m"].copy()
    want[d] += ex["force"][k] * eps
    np.testing.assert_allclose(gv["tau_m"], want, rtol=0, atol=1e-11 * np.abs(ex["tau_m"]).max())
    # the implicit damping R^T diag(dF/dLdot) R gains dF_k (2 R_kd eps + eps^2) on (d, d) and
    # dF_k eps R_kj off the diagonal of row and column d
    dA = (gv["A"] - ex["A"]) / DT
    g = ex["dFdv"][k]
    assert dA[d, d] == pytest.approx(g * (2 * ex["R"][k, d] * eps + eps * eps), rel=1e-7)
    for j in np.flatnonzero(np.abs(ex["R"][k]) > 1e-9):
        if j != d:
            assert dA[d, j] == pytest.approx(g * eps * ex["R"][k, j], rel=1e-7)


def test_fibre_velocity_follows_the_given_moment_arms(tiny):
    model, om, st = tiny
    ex = ora.evaluate(om, DT, st["q"], st["qd"], st["act"], st["exc"])
    R = 1.5 * ex["R"]
    gv = ora.evaluate(om, DT, st["q"], st["qd"], st["act"], st["exc"], L=ex["L"], R=R)
    vmax = model.vmax_per_lopt * model.muscle_lopt
    np.testing.assert_allclose(gv["vm"], -(R @ st["qd"]) / vmax, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(gv["vm"], 1.5 * ex["vm"], rtol=1e-12, atol=1e-15)

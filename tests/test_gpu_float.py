"""Free (floating) root on the device, through the C ABI, against the FP64 oracle.

Body 0 joined to the world by six DoFs (translations of its origin along world x, y, z, then
rotations about world x, y, z through it; q = position and rotation vector, qd = velocity and
world angular velocity).  Checks: every stage of one substep of the floating whole body, a
100-substep trajectory, the exact semi-implicit Euler free fall of a spinning sphere, a long
spin that carries the rotation vector through angle pi, and the host's checks.
"""
import copy

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from scipy.spatial.transform import Rotation

from oracle import oracle as ora
from paper_2603_29332_b300 import modelgen as mg
from paper_2603_29332_b300 import msim
from tests.gpu_common import oracle_eval, qdd_rel_err, random_states, sample_envs

pytestmark = pytest.mark.gpu

DT = 1e-3


def _sphere(omega_scale=1.0):
    base = mg.make_model("ball", [-1], [1], [[0.0, 0.0, 1.0]], [2.0], [[0, 0, 0]], [[0.02, 0.02, 0.02, 0, 0, 0]],
                         [[0, 0, 1]], muscle_points=[[(0, (0.0, 0.0, 0.1)), (0, (0.0, 0.1, 0.0))]],
                         muscle_fmax=[10.0], muscle_lopt=[0.1])
    return mg.with_free_root(base)


def test_floating_body_stage_parity():
    model = mg.config_model("c1_float")
    om = ora.OracleModel(model)
    E, n, m = 1024, model.n_dofs, model.n_muscles
    sim = msim.Sim(model, E, dt=DT)
    lay = sim.layout(0)
    q, qd, act, exc = random_states(model, E, seed=31)
    q[:, 2] = np.abs(q[:, 2]) * 0.1 - 0.02        # root height near the model pose: some feet touch
    res = sim.eval(sim.pad_n(q), sim.pad_n(qd), sim.pad_m(act), sim.pad_m(exc))
    g = {k: v.double().cpu().numpy() for k, v in res.items()}
    worst, n_contact = 0.0, 0
    for e in sample_envs(E, 24, seed=4):
        r = oracle_eval(om, DT, q[e], qd[e], act[e], exc[e])
        assert r["status"] == 0
        np.testing.assert_allclose(g["L"][e, :m], r["L"], rtol=0, atol=2e-6)
        np.testing.assert_allclose(msim.unpack_R(g["R"][e], lay, n), r["R"], rtol=0, atol=2e-6)
        Mg = msim.unpack_packed(g["M"][e], lay)
        np.testing.assert_allclose(Mg, r["M"], rtol=0, atol=2e-6 * np.abs(r["M"]).max())
        sC = np.abs(r["bias"]).max() + 1.0
        np.testing.assert_allclose(g["bias"][e, :n], r["bias"], rtol=0, atol=2e-5 * sC)
        np.testing.assert_allclose(g["tau_c"][e, :n], r["tau_c"], rtol=0, atol=1e-3 * (np.abs(r["tau_c"]).max() + 1))
        n_contact += int(np.abs(r["tau_c"]).max() > 0)
        worst = max(worst, qdd_rel_err(g["qdd"][e, :n], r["qdd"]))
    print("\nfloating root: worst qdd rel err %.2e, envs in contact %d" % (worst, n_contact))
    assert worst <= 1e-4
    assert n_contact > 0


def test_floating_body_trajectory_100_steps():
    model = mg.config_model("c1_float")
    om = ora.OracleModel(model)
    E, steps = 1024, 100
    sim = msim.Sim(model, E, dt=DT)
    q0, qd0, a0 = mg.initial_state(model, E, seed=9)
    exc = mg.smooth_excitations(model, E, steps, seed=9)
    sim.reset(sim.pad_n(q0), sim.pad_n(qd0), sim.pad_m(a0))
    for t in range(steps):
        sim.step(sim.pad_m(exc[t]), 1)
    qg = sim.state()["q"][:, :model.n_dofs].double().cpu().numpy()
    idx = sample_envs(E, 12, seed=2)
    q, qd, act = q0[idx].astype(np.float64), qd0[idx].astype(np.float64), a0[idx].astype(np.float64)
    for t in range(steps):
        q, qd, act, *_ = ora.step(om, DT, q, qd, act, exc[t][idx].astype(np.float64), 1)
    err = np.abs(qg[idx] - q).max()
    drop = np.abs(q[:, :6]).max()
    print("\nfloating trajectory: max |q_gpu - q_oracle| %.2e (root moved up to %.3f)" % (err, drop))
    assert err <= 1e-3
    assert drop > 1e-3   # the root did move
    assert sim.status() == (0, 0)


def test_free_fall_of_a_spinning_sphere_is_exact_semi_implicit_euler():
    model = _sphere()
    E, N = 4, 200
    sim = msim.Sim(model, E, dt=DT)
    v0 = np.array([[0.3, -0.2, 1.5], [0, 0, 0], [1, 1, 1], [-2, 0.5, 0]], np.float32)
    w0 = np.array([[0.4, 1.1, -0.7], [0, 0, 3.0], [0, 0, 0], [2, -1, 0.5]], np.float32)
    q0 = np.zeros((E, 6), np.float32)
    qd0 = np.concatenate([v0, w0], 1)
    sim.reset(sim.pad_n(q0), sim.pad_n(qd0), sim.pad_m(np.zeros((E, 1), np.float32)))
    zero = sim.pad_m(np.zeros((E, 1), np.float32))
    sim.step(zero, N)
    st = sim.state()
    q, qd = st["q"][:, :6].double().cpu().numpy(), st["qd"][:, :6].double().cpu().numpy()
    g = model.gravity
    for e in range(E):
        np.testing.assert_allclose(qd[e, :3], v0[e] + N * DT * g, rtol=0, atol=2e-5)
        np.testing.assert_allclose(q[e, :3], N * DT * v0[e] + DT * DT * g * N * (N + 1) / 2, rtol=0, atol=2e-5)
        np.testing.assert_allclose(qd[e, 3:], w0[e], rtol=0, atol=1e-5)
        np.testing.assert_allclose(q[e, 3:], N * DT * w0[e].astype(np.float64), rtol=0, atol=1e-4)


def test_long_spin_carries_the_rotation_vector_through_pi():
    model = _sphere()
    E, N = 2, 1500
    sim = msim.Sim(model, E, dt=DT)
    w0 = np.array([[0.0, 0.0, 4.0], [2.0, -3.0, 1.0]], np.float32)   # 6 rad and 5.6 rad: past pi
    qd0 = np.concatenate([np.zeros((E, 3), np.float32), w0], 1)
    sim.reset(sim.pad_n(np.zeros((E, 6), np.float32)), sim.pad_n(qd0), sim.pad_m(np.zeros((E, 1), np.float32)))
    sim.step(sim.pad_m(np.zeros((E, 1), np.float32)), N)
    r = sim.state()["q"][:, 3:6].double().cpu().numpy()
    for e in range(E):
        want = Rotation.from_rotvec(N * DT * w0[e].astype(np.float64)).as_matrix()
        np.testing.assert_allclose(Rotation.from_rotvec(r[e]).as_matrix(), want, rtol=0, atol=2e-4)
        assert np.linalg.norm(r[e]) <= np.pi + 1e-5


def test_free_root_checks():
    model = mg.config_model("c1_float")
    sim = msim.Sim(model, 8, dt=DT)
    with pytest.raises(msim.MsimError, match="free root"):
        sim.train_surrogate(n_samples=4096, epochs=1)
    bad = copy.deepcopy(model)
    bad.dof_limit[0] = [-1.0, 1.0]
    with pytest.raises(msim.MsimError, match="no limit"):
        msim.Sim(bad, 4, dt=DT)
    bad = copy.deepcopy(model)
    bad.free_root = False
    with pytest.raises(msim.MsimError, match="body_ndof"):
        msim.Sim(bad, 4, dt=DT)


def test_ball_on_the_ground_contact_closed_forms():
    """A free ball at its static penetration sliding at v (device vs oracle, both with the
    friction and contact damping taken implicitly), and a ball dropped onto the ground against
    the overdamped oscillator m z'' = k (r - z) - c z' - m g."""
    import math
    from tests import handmodels as hm
    model = hm.free_ball()
    om = ora.OracleModel(model)
    m, r, g = model.body_mass[0], model.sphere_radius[0], -model.gravity[2]
    k, c = model.contact_k, model.contact_c
    E = 3
    sim = msim.Sim(model, E, dt=DT)
    q = np.zeros((E, 6), np.float32)
    q[:, 2] = -m * g / k
    qd = np.zeros((E, 6), np.float32)
    qd[:, 0] = [0.05, 0.5, 3.0]
    z = np.zeros((E, 1), np.float32)
    res = sim.eval(sim.pad_n(q), sim.pad_n(qd), sim.pad_m(z), sim.pad_m(z))
    qdd = res["qdd"][:, :6].double().cpu().numpy()
    for e in range(E):
        ref = ora.evaluate(om, DT, q[e].astype(np.float64), qd[e].astype(np.float64), np.zeros(1), np.zeros(1))["qdd"]
        np.testing.assert_allclose(qdd[e], ref, rtol=0, atol=1e-4 * np.abs(ref).max())
        assert qdd[e, 0] < 0 and qdd[e, 4] > 0
    # drop: 1000 substeps of 10 us in one call
    dt, n, v0 = 1e-5, 1000, -0.2
    sim2 = msim.Sim(model, 1, dt=dt)
    qd0 = np.zeros((1, 6), np.float32)
    qd0[0, 2] = v0
    sim2.reset(sim2.pad_n(np.zeros((1, 6), np.float32)), sim2.pad_n(qd0), sim2.pad_m(np.zeros((1, 1), np.float32)))
    sim2.step(sim2.pad_m(np.zeros((1, 1), np.float32)), n)
    zg = r + float(sim2.state()["q"][0, 2])
    s1, s2 = (float(np.real(x)) for x in np.roots([m, c, k]))
    x0 = m * g / k
    B = (v0 - s1 * x0) / (s2 - s1)
    zT = (r - m * g / k) + (x0 - B) * math.exp(s1 * n * dt) + B * math.exp(s2 * n * dt)
    print("\nball drop: z after 10 ms %.7f m, closed form %.7f m" % (zg, zT))
    assert abs(zg - zT) < 5e-6


def _two_roots():
    """Body 0 on a free root with a child; body 1 a second root on a hinge, with a child."""
    base = mg.make_model("tworoots", [-1, -1, 1, 0], [1, 1, 1, 1],
                         [[0, 0, 1.0], [1.0, 0, 1.0], [0, 0, -0.4], [0.1, 0, -0.2]],
                         [2.0, 1.5, 1.0, 0.8],
                         [[0, 0, 0], [0, 0, -0.2], [0, 0, -0.2], [0, 0, -0.1]],
                         [[0.02, 0.02, 0.02, 0, 0, 0], [0.03, 0.03, 0.01, 0, 0, 0], [0.02, 0.02, 0.01, 0, 0, 0],
                          [0.01, 0.01, 0.005, 0, 0, 0]],
                         [[0, 0, 1], [0, 0, 1], [0, 1, 0], [1, 0, 0]],
                         muscle_points=[[(1, (0.05, 0, -0.1)), (2, (0.05, 0, -0.2))],
                                        [(0, (0.0, 0.08, 0.0)), (3, (0.0, 0.05, -0.05))]],
                         muscle_fmax=[200.0, 100.0], muscle_lopt=[0.1, 0.08])
    return mg.with_free_root(base)


def test_a_fixed_second_root_beside_the_free_root():
    """Only the chains that start at the free root take its transform: the second root's
    bodies stay on their fixed hinge (one substep at random states and 50 substeps)."""
    model = _two_roots()
    om = ora.OracleModel(model)
    E, n, m = 64, model.n_dofs, model.n_muscles
    sim = msim.Sim(model, E, dt=DT)
    lay = sim.layout(0)
    q, qd, act, exc = random_states(model, E, seed=12, q_scale=0.6)
    res = sim.eval(sim.pad_n(q), sim.pad_n(qd), sim.pad_m(act), sim.pad_m(exc))
    g = {k: v.double().cpu().numpy() for k, v in res.items()}
    for e in sample_envs(E, 12, seed=3):
        r = oracle_eval(om, DT, q[e], qd[e], act[e], exc[e])
        np.testing.assert_allclose(g["L"][e, :m], r["L"], rtol=0, atol=2e-6)
        np.testing.assert_allclose(msim.unpack_R(g["R"][e], lay, n), r["R"], rtol=0, atol=2e-6)
        np.testing.assert_allclose(msim.unpack_packed(g["M"][e], lay), r["M"], rtol=0, atol=2e-6 * np.abs(r["M"]).max())
        assert qdd_rel_err(g["qdd"][e, :n], r["qdd"]) <= 1e-4
    sim.reset(sim.pad_n(q), sim.pad_n(qd), sim.pad_m(act))
    sim.step(sim.pad_m(exc), 50)
    qg = sim.state()["q"][:, :n].double().cpu().numpy()
    idx = sample_envs(E, 6, seed=4)
    qo, *_ = ora.step(om, DT, q[idx].astype(np.float64), qd[idx].astype(np.float64), act[idx].astype(np.float64),
                      exc[idx].astype(np.float64), 50)
    assert np.abs(qg[idx] - qo).max() <= 1e-3
    assert sim.status() == (0, 0)

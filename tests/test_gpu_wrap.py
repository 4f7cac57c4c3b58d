"""Muscle paths wrapping a cylinder or a sphere, on the device, against the FP64 oracle (through
the C ABI).

The wrapped segment takes the shortest way around an infinite cylinder fixed to a body of the
muscle's chain (tangent - arc - tangent in the plane normal to the axis, straight along the axis
once unrolled), or over a sphere (the great circle in the plane of the two points and the
centre).  Checks: lengths and moment arms of the whole-body model with a quarter of its muscles
wrapping, all cylinders or half spheres (with a count of the wraps that are active in the
sample, so that the branches are exercised), the closed-form moment arm of a cylinder coaxial
with a hinge, the accelerations and 100-substep trajectories, the mixed launch, and the host's
rejection of invalid wraps.
"""
import copy

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as ora
from paper_2603_29332_b300 import modelgen as mg
from paper_2603_29332_b300 import msim
from tests.gpu_common import oracle_eval, qdd_rel_err, random_states, sample_envs

pytestmark = pytest.mark.gpu

DT = 1e-3


def _unwrapped(model):
    m = copy.copy(model)
    m.wrap_muscle = np.zeros(0, np.int32)
    m.wrap_segment = np.zeros(0, np.int32)
    m.wrap_body = np.zeros(0, np.int32)
    m.wrap_center = np.zeros((0, 3), np.float32)
    m.wrap_axis = np.zeros((0, 3), np.float32)
    m.wrap_radius = np.zeros(0, np.float32)
    m.wrap_kind = np.zeros(0, np.int32)
    return m


@pytest.mark.parametrize("name", ["c1_wrap", "c1_wrap_mix"])
def test_wrapped_geometry_and_accelerations_match_the_oracle(name):
    model = mg.config_model(name)
    plain = _unwrapped(model)
    om = ora.OracleModel(model)
    E, n, m = 2048, model.n_dofs, model.n_muscles
    sim = msim.Sim(model, E, dt=DT)
    lay = sim.layout(0)
    q, qd, act, exc = random_states(model, E, seed=21)
    res = sim.eval(sim.pad_n(q), sim.pad_n(qd), sim.pad_m(act), sim.pad_m(exc))
    g = {k: v.double().cpu().numpy() for k, v in res.items()}
    active, active_sph, worst_L, worst_R, worst_qdd = 0, 0, 0.0, 0.0, 0.0
    for e in sample_envs(E, 32, seed=3):
        r = oracle_eval(om, DT, q[e], qd[e], act[e], exc[e])
        assert r["status"] == 0
        L0, _ = ora.muscle_geometry(plain, q[e].astype(np.float64))
        moved = np.abs(r["L"] - L0) > 1e-9
        active += int(np.count_nonzero(moved))
        active_sph += int(np.count_nonzero(moved[model.wrap_muscle[model.wrap_kind == 1]]))
        Rg = msim.unpack_R(g["R"][e], lay, n)
        worst_L = max(worst_L, np.abs(g["L"][e, :m] - r["L"]).max())
        worst_R = max(worst_R, np.abs(Rg - r["R"]).max())
        np.testing.assert_allclose(g["L"][e, :m], r["L"], rtol=0, atol=2e-6)
        np.testing.assert_allclose(Rg, r["R"], rtol=0, atol=2e-6)
        np.testing.assert_allclose(g["lm"][e, :m], r["lm"], rtol=0, atol=5e-5)
        np.testing.assert_allclose(g["vm"][e, :m], r["vm"], rtol=0, atol=5e-5)
        st = np.abs(r["tau_m"]).max() + 1.0
        np.testing.assert_allclose(g["tau_m"][e, :n], r["tau_m"], rtol=0, atol=2e-3 * st)
        worst_qdd = max(worst_qdd, qdd_rel_err(g["qdd"][e, :n], r["qdd"]))
    print("\n%s: %d active wraps in the sample, worst |dL| %.2e m, |dR| %.2e m, qdd rel %.2e"
          % (name, active, worst_L, worst_R, worst_qdd))
    assert active >= 100, "too few active wraps in the sample to exercise the branch"
    if model.wrap_kind.any():
        assert active_sph >= 50, "too few active sphere wraps in the sample"
    assert worst_qdd <= 1e-4


def test_coaxial_cylinder_moment_arm_is_the_radius_on_the_device():
    from tests.test_oracle_wrap import _coaxial_model
    model = _coaxial_model(0.03)
    r = float(model.wrap_radius[0])
    qs = np.array([[0.0, -0.3], [0.0, 0.0], [0.0, 0.2], [0.4, 0.1]], np.float32)
    sim = msim.Sim(model, len(qs), dt=DT)
    lay = sim.layout(0)
    z = np.zeros_like(qs)
    res = sim.eval(sim.pad_n(qs), sim.pad_n(z), sim.pad_m(np.zeros((len(qs), 1), np.float32)),
                   sim.pad_m(np.zeros((len(qs), 1), np.float32)))
    Lg = res["L"][:, 0].double().cpu().numpy()
    for e in range(len(qs)):
        R = msim.unpack_R(res["R"][e].double().cpu().numpy(), lay, 2)
        np.testing.assert_allclose(abs(R[0, 1]), r, rtol=2e-6)
        assert R[0, 0] == 0.0
        L, _ = ora.muscle_geometry(model, qs[e].astype(np.float64))
        np.testing.assert_allclose(Lg[e], L[0], rtol=0, atol=1e-7)


@pytest.mark.parametrize("name", ["c1_wrap", "c1_wrap_mix"])
def test_trajectory_parity_100_steps_with_wrapping(name):
    model = mg.config_model(name)
    om = ora.OracleModel(model)
    E, steps = 1024, 100
    sim = msim.Sim(model, E, dt=DT)
    q0, qd0, a0 = mg.initial_state(model, E, seed=7)
    exc = mg.smooth_excitations(model, E, steps, seed=7)
    sim.reset(sim.pad_n(q0), sim.pad_n(qd0), sim.pad_m(a0))
    for t in range(steps):
        sim.step(sim.pad_m(exc[t]), 1)
    qg = sim.state()["q"][:, :model.n_dofs].double().cpu().numpy()
    idx = sample_envs(E, 16, seed=1)
    q, qd, act = q0[idx].astype(np.float64), qd0[idx].astype(np.float64), a0[idx].astype(np.float64)
    for t in range(steps):
        q, qd, act, *_ = ora.step(om, DT, q, qd, act, exc[t][idx].astype(np.float64), 1)
    err = np.abs(qg[idx] - q).max()
    print("\n%s trajectory: max |q_gpu - q_oracle| after %d substeps %.2e rad" % (name, steps, err))
    assert err <= 1e-3
    assert sim.status() == (0, 0)


def test_mixed_launch_with_wrapping_equals_per_model_launches_bitwise():
    models = [mg.config_model("c1_whole"), mg.config_model("c1_wrap")]
    counts = [45, 67]
    sims = [msim.Sim(models, counts, dt=DT) for _ in range(2)]
    rows = [mg.initial_state(mm, E, seed=3 + i) for i, (mm, E) in enumerate(zip(models, counts))]
    exc = torch.cat([sims[0]._pad(mg.uniform_excitations(mm, E, 1, seed=9 + i)[0], sims[0].pitch_m)
                     for i, (mm, E) in enumerate(zip(models, counts))])
    for s in sims:
        s.reset(torch.cat([s._pad(r[0], s.pitch_n) for r in rows]), torch.cat([s._pad(r[1], s.pitch_n) for r in rows]),
                torch.cat([s._pad(r[2], s.pitch_m) for r in rows]))
        for i in range(2):
            s.set_launch(i, warps_per_env=2)
    sims[1].set_mixed_launch(True, warps_per_env=2, slots_per_block=5)
    for _ in range(3):
        for s in sims:
            s.step(exc, 5)
    torch.cuda.synchronize()
    sa, sb = sims[0].state(), sims[1].state()
    for k in ("q", "qd", "act", "qdd", "force"):
        assert torch.equal(sa[k], sb[k]), k


@pytest.mark.parametrize("edit,msg", [
    (lambda m: m.wrap_segment.__setitem__(0, 0), "segment"),
    (lambda m: m.wrap_radius.__setitem__(0, -0.01), "radius"),
    (lambda m: m.wrap_body.__setitem__(0, m.n_bodies), "chain"),
    (lambda m: m.wrap_kind.__setitem__(0, 2), "kind"),
])
def test_invalid_wraps_are_rejected(edit, msg):
    model = copy.deepcopy(mg.config_model("c1_wrap"))
    edit(model)
    with pytest.raises(msim.MsimError, match=msg):
        msim.Sim(model, 4, dt=DT)


def test_two_surfaces_on_one_muscle_are_rejected():
    model = copy.deepcopy(mg.config_model("c1_wrap"))
    for k in ("wrap_muscle", "wrap_segment", "wrap_body", "wrap_center", "wrap_axis", "wrap_radius", "wrap_kind"):
        a = getattr(model, k)
        setattr(model, k, np.concatenate([a, a[:1]]))
    with pytest.raises(msim.MsimError, match="two wrapping surfaces"):
        msim.Sim(model, 4, dt=DT)

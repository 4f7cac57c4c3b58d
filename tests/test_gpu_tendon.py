"""Compliant tendons on the device, through the C ABI, against the FP64 oracle.

A compliant tendon (a reading; the paper's is rigid) puts an elastic tendon in series with the
fibre: the tendon strain is a state, the fibre velocity follows from the damped equilibrium of
fibre and tendon forces (closed-form branch roots on the device, bisection in the oracle), the
strain advances linearly implicitly and the skeleton receives the tendon force.  Checks: every
stage of one substep at random states and strains (with counts of the curve regions and fibre
branches the sample reaches), a 100-substep trajectory of positions and strains, the strain
state's reset and set / get, the mixed launch, and the host's checks.
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


def _tendon_model(name="c1_whole", seed=1, frac=1.0):
    base = mg.config_model(name)
    return mg.with_tendons(base, ora.OracleModel(base).L0, frac=frac, seed=seed)


def _strains(model, E, seed):
    """Strains over slack, toe and linear regions: U(-0.3, 1.6) eps0 on compliant muscles."""
    r = np.random.default_rng(seed)
    eps0 = model.muscle_tendon_strain
    return (r.uniform(-0.3, 1.6, (E, model.n_muscles)) * eps0).astype(np.float32)


def test_tendon_stage_parity():
    model = _tendon_model()
    om = ora.OracleModel(model)
    on = model.muscle_tendon_strain > 0
    assert on.sum() >= 300
    E, n, m = 1024, model.n_dofs, model.n_muscles
    sim = msim.Sim(model, E, dt=DT)
    lay = sim.layout(0)
    q, qd, act, exc = random_states(model, E, seed=41)
    eps = _strains(model, E, seed=42)
    res = sim.eval(sim.pad_n(q), sim.pad_n(qd), sim.pad_m(act), sim.pad_m(exc), eps=sim.pad_m(eps))
    g = {k: v.double().cpu().numpy() for k, v in res.items()}
    worst = dict(vm=0.0, lm=0.0, eps=0.0, F=0.0, qdd=0.0)
    regions = np.zeros(3, int)     # slack / toe / linear tendon at the start of the substep
    branches = np.zeros(3, int)    # fibre velocity below -1 / shortening / lengthening
    for e in sample_envs(E, 24, seed=6):
        r = oracle_eval(om, DT, q[e], qd[e], act[e], exc[e], eps[e])
        assert r["status"] == 0
        x = eps[e, on] / model.muscle_tendon_strain[on]
        regions += [np.sum(x <= 0), np.sum((x > 0) & (x <= 1)), np.sum(x > 1)]
        v = r["vm"][on]
        branches += [np.sum(v < -1), np.sum((v >= -1) & (v <= 0)), np.sum(v > 0)]
        np.testing.assert_allclose(g["L"][e, :m], r["L"], rtol=0, atol=2e-6)
        np.testing.assert_allclose(msim.unpack_R(g["R"][e], lay, n), r["R"], rtol=0, atol=2e-6)
        worst["lm"] = max(worst["lm"], np.abs(g["lm"][e, :m] - r["lm"]).max())
        worst["vm"] = max(worst["vm"], np.abs(g["vm"][e, :m][on] - r["vm"][on]).max())
        worst["eps"] = max(worst["eps"], np.abs(g["eps_next"][e, :m] - r["eps_next"]).max())
        worst["F"] = max(worst["F"], (np.abs(g["force"][e, :m] - r["force"]) / model.muscle_fmax).max())
        worst["qdd"] = max(worst["qdd"], qdd_rel_err(g["qdd"][e, :n], r["qdd"]))
        # rigid muscles carry their strain through unchanged
        np.testing.assert_array_equal(g["eps_next"][e, :m][~on], eps[e, ~on])
    print("\ntendon stage parity: regions slack/toe/linear %s, fibre branches %s, worst %s"
          % (regions.tolist(), branches.tolist(), {k: "%.1e" % v for k, v in worst.items()}))
    assert regions.min() >= 200 and branches.min() >= 20
    # FP32 against FP64: l_m from an FP32 length of up to ~1 m over l_opt >= 5 cm; v_m through
    # the damped equilibrium, whose slope in v_m is at least beta = 0.1, so an error in its force
    # terms grows by at most 10x, and the passive term moves by f_p' (<= 7) times l_m's error;
    # the strain moves by dt v_max dv_m / l_s; the force by F_max f_t' d(eps/eps0)
    assert worst["lm"] <= 5e-5
    assert worst["vm"] <= 2e-3
    assert worst["eps"] <= 2e-6
    assert worst["F"] <= 2e-4
    assert worst["qdd"] <= 1e-4


def test_tendon_trajectory_100_steps():
    model = _tendon_model()
    om = ora.OracleModel(model)
    E, steps = 1024, 100
    sim = msim.Sim(model, E, dt=DT)
    q0, qd0, a0 = mg.initial_state(model, E, seed=13)
    exc = mg.smooth_excitations(model, E, steps, seed=13)
    sim.reset(sim.pad_n(q0), sim.pad_n(qd0), sim.pad_m(a0))
    for t in range(steps):
        sim.step(sim.pad_m(exc[t]), 1)
    qg = sim.state()["q"][:, :model.n_dofs].double().cpu().numpy()
    eg = sim.tendon_strain()[:, :model.n_muscles].double().cpu().numpy()
    idx = sample_envs(E, 12, seed=3)
    q, qd, act = q0[idx].astype(np.float64), qd0[idx].astype(np.float64), a0[idx].astype(np.float64)
    eps = None
    for t in range(steps):
        q, qd, act, _, _, _, eps = ora.step(om, DT, q, qd, act, exc[t][idx].astype(np.float64), 1, eps=eps)
    err_q = np.abs(qg[idx] - q).max()
    err_e = np.abs(eg[idx] - eps).max()
    span = np.abs(eps).max()
    print("\ntendon trajectory: max |dq| %.2e rad, max |d eps| %.2e (strains up to %.3f)" % (err_q, err_e, span))
    assert err_q <= 1e-3
    assert err_e <= 1e-4 and span > 0.01
    assert sim.status() == (0, 0)


def test_strain_state_reset_and_set_get():
    model = _tendon_model()
    E, m = 16, model.n_muscles
    sim = msim.Sim(model, E, dt=DT)
    q0, qd0, a0 = mg.initial_state(model, E, seed=2)
    a0 = np.full((E, m), 0.7, np.float32)
    sim.reset(sim.pad_n(q0), sim.pad_n(qd0), sim.pad_m(a0))
    sim.step(sim.pad_m(np.ones((E, m), np.float32)), 20)
    s = sim.tendon_strain()
    *_, eo = ora.step(ora.OracleModel(model), DT, q0, qd0, a0, np.ones((E, m)), 20)
    np.testing.assert_allclose(s[:, :m].double().cpu().numpy(), eo, rtol=0, atol=1e-5)
    on = torch.from_numpy(model.muscle_tendon_strain > 0).to(s.device)
    assert float((s[:, :m][:, on] > 0).double().mean()) > 0.9   # activated fibres stretch their tendons
    assert bool((s[:, :m][:, ~on] == 0).all())                   # rigid tendons carry no strain
    ids = torch.tensor([3, 7], dtype=torch.int32, device=s.device)
    sim.reset(sim.pad_n(q0[[3, 7]]), None, None, env_ids=ids)
    s2 = sim.tendon_strain()
    assert bool((s2[[3, 7]] == 0).all()) and torch.equal(s2[[0, 1, 2]], s[[0, 1, 2]])
    want = torch.rand_like(s) * 0.01
    got = sim.tendon_strain(set=want)
    assert torch.equal(got, want)


def test_mixed_launch_with_tendons_equals_per_model_launches_bitwise():
    models = [mg.config_model("c1_whole"), _tendon_model()]
    counts = [45, 67]
    sims = [msim.Sim(models, counts, dt=DT) for _ in range(2)]
    rows = [mg.initial_state(mm, E, seed=5 + i) for i, (mm, E) in enumerate(zip(models, counts))]
    exc = torch.cat([sims[0]._pad(mg.uniform_excitations(mm, E, 1, seed=11 + i)[0], sims[0].pitch_m)
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
    assert torch.equal(sims[0].tendon_strain(), sims[1].tendon_strain())


@pytest.mark.parametrize("value,msg", [(0.7, "tendon strain"), (-0.01, "tendon strain"), (float("nan"), "tendon strain")])
def test_invalid_tendon_strains_are_rejected(value, msg):
    model = copy.deepcopy(_tendon_model())
    model.muscle_tendon_strain[np.argmax(model.muscle_tendon_strain > 0)] = value
    with pytest.raises(msim.MsimError, match=msg):
        msim.Sim(model, 4, dt=DT)


def test_short_tendon_is_rejected():
    base = mg.config_model("c1_whole")
    L0 = ora.OracleModel(base).L0
    short = int(np.argmin((L0 - base.muscle_lopt) / base.muscle_lopt))   # slack length below 0.5 l_opt
    model = copy.deepcopy(base)
    model.muscle_tendon_strain = np.zeros(model.n_muscles)
    model.muscle_tendon_strain[short] = 0.04
    with pytest.raises(msim.MsimError, match="slack length"):
        msim.Sim(model, 4, dt=DT)


def test_learned_geometry_steps_with_tendons_follow_the_exact_path_when_checked():
    """The learned-geometry step of a model with compliant tendons: with every environment
    checked, each substep uses the exact geometry, so positions, strains and forces equal an
    exact-geometry twin bit for bit; unchecked learned steps advance the strains too."""
    model = _tendon_model()
    E, m = 256, model.n_muscles
    sim = msim.Sim(model, E, dt=DT, seed=5)
    sim.train_surrogate(65536, 2, batch=4096, lr=1e-3)
    ex = msim.Sim(model, E, dt=DT, seed=5)
    q0, qd0, a0 = mg.initial_state(model, E, seed=21)
    for s in (sim, ex):
        s.reset(s.pad_n(q0), s.pad_n(qd0), s.pad_m(a0))
    exc = sim.pad_m(mg.smooth_excitations(model, E, 1, seed=21)[0])
    sim.set_geometry_mode(1)
    sim.surrogate_set_check(1.0, 1e-3)
    for _ in range(4):
        sim.step(exc, 3)
        ex.step(exc, 3)
    sa, sb = sim.state(), ex.state()
    for k in ("q", "qd", "act", "qdd", "force"):
        assert torch.equal(sa[k], sb[k]), k
    assert torch.equal(sim.tendon_strain(), ex.tendon_strain())
    assert float(sim.tendon_strain()[:, :m].abs().max()) > 0
    # learned geometry without checks (a reset clears the flags the checks set): the strains of
    # the environments inside the training box advance from the network's lengths
    sim.reset(sim.pad_n(q0), sim.pad_n(qd0), sim.pad_m(a0))
    sim.surrogate_set_check(0.0, 1e-3)
    sim.surrogate_stats(reset=True)
    sim.step(exc, 3)
    e1 = sim.tendon_strain()[:, :m]
    assert sim.surrogate_stats()["learned"] > 0
    assert bool(torch.isfinite(e1).all()) and float(e1.abs().max()) > 0
    assert sim.status() == (0, 0)


def test_autotune_keeps_the_strain_state():
    """The autotuner times real steps on the handle's environments and restores their state,
    tendon strains included (a tuner that left its strains behind under the restored positions
    sent later rollouts elsewhere)."""
    model = _tendon_model()
    E = 256
    sim = msim.Sim(model, E, dt=DT)
    q0, qd0, a0 = mg.initial_state(model, E, seed=8)
    sim.reset(sim.pad_n(q0), sim.pad_n(qd0), sim.pad_m(a0))
    sim.step(sim.pad_m(mg.smooth_excitations(model, E, 1, seed=8)[0]), 5)
    before, eb = sim.state(), sim.tendon_strain()
    assert float(eb.abs().max()) > 0
    sim.autotune(None, n_sub=3)
    after, ea = sim.state(), sim.tendon_strain()
    for k in ("q", "qd", "act", "qdd", "force", "status"):
        assert torch.equal(before[k], after[k]), k
    assert torch.equal(eb, ea)

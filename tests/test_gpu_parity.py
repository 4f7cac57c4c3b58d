"""Parity of the CUDA path (through the C ABI) with the FP64 oracle, stage by stage and over
trajectories, on seeded synthetic inputs.

Tolerances (FP32 GPU vs FP64 oracle from the same FP32-rounded state):
  * q_dd: norm-wise relative error <= 1e-4 per env (the stated target for one step);
  * q after 100 steps from identical states: within 1e-3 rad;
  * intermediate stages: bounds from FP32 rounding through the kinematic chain (positions
    ~1 m, depth <= 40: |dx| ~ 40 * 6e-8 m), stated per check below.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as ora
from paper_2603_29332_b300 import modelgen as mg
from paper_2603_29332_b300 import msim
from tests.gpu_common import oracle_eval, qdd_rel_err, random_states, sample_envs

pytestmark = pytest.mark.gpu

DT = 1e-3


def _sim(model, E):
    return msim.Sim([model], [E], dt=DT)


def _np(t, cols):
    return t[:, :cols].double().cpu().numpy()


@pytest.mark.parametrize("name,E,k", [("c0_tiny", 64, 64), ("c1_whole", 4096, 48), ("c1_whole", 16384, 16),
                                      ("c2_upper", 2458, 32), ("c2_lower", 2458, 32)])
def test_stage_parity(name, E, k):
    """Every stage of one substep on sampled environments of a launch at the workloads' sizes:
    the tiny model, the whole body at 4096 environments (the benchmark) and 16384 (the closed
    loop), and the two extra skeletons of the mixed batch at their share of its 8192."""
    model = mg.config_model(name)
    om = ora.OracleModel(model)
    sim = _sim(model, E)
    n, m = model.n_dofs, model.n_muscles
    q, qd, act, exc = random_states(model, E, seed=11)
    res = sim.eval(sim.pad_n(q), sim.pad_n(qd), sim.pad_m(act), sim.pad_m(exc))
    torch.cuda.synchronize()
    lay = sim.layout(0)
    g = {k_: v.double().cpu().numpy() for k_, v in res.items()}
    worst = {}
    n_contact = 0
    for e in sample_envs(E, k):
        r = oracle_eval(om, DT, q[e], qd[e], act[e], exc[e])
        assert r["status"] == 0
        # muscle geometry
        np.testing.assert_allclose(g["L"][e, :m], r["L"], rtol=0, atol=2e-6)
        Rg = msim.unpack_R(g["R"][e], lay, n)
        np.testing.assert_allclose(Rg, r["R"], rtol=0, atol=2e-6)
        np.testing.assert_allclose(g["lm"][e, :m], r["lm"], rtol=0, atol=5e-5)
        np.testing.assert_allclose(g["vm"][e, :m], r["vm"], rtol=0, atol=5e-5)
        # Hill force (Eq. 1) at the GPU's own fibre state, and at the oracle's
        lm, vm = g["lm"][e, :m], g["vm"][e, :m]
        Fself = np.array([model.muscle_fmax[j] * (act[e, j] * ora.fl(lm[j]) * ora.fv(vm[j]) + ora.fp(lm[j]))
                          for j in range(m)])
        np.testing.assert_allclose(g["force"][e, :m], Fself, rtol=2e-6, atol=1e-3)
        np.testing.assert_allclose(g["force"][e, :m], r["force"], rtol=0, atol=2e-3 * model.muscle_fmax.max())
        np.testing.assert_allclose(g["act_next"][e, :m], r["act_next"], rtol=0, atol=1e-6)
        # dynamics terms
        Mg = msim.unpack_packed(g["M"][e], lay)
        sM = np.abs(r["M"]).max()
        np.testing.assert_allclose(Mg, r["M"], rtol=0, atol=2e-6 * sM)
        sC = np.abs(r["bias"]).max() + 1.0
        np.testing.assert_allclose(g["bias"][e, :n], r["bias"], rtol=0, atol=2e-5 * sC)
        Ag = msim.unpack_packed(g["A"][e], lay)
        np.testing.assert_allclose(Ag, r["A"], rtol=0, atol=2e-5 * np.abs(r["A"]).max())
        st = np.abs(r["tau_m"]).max() + 1.0
        np.testing.assert_allclose(g["tau_m"][e, :n], r["tau_m"], rtol=0, atol=2e-3 * st)
        np.testing.assert_allclose(g["tau_l"][e, :n], r["tau_l"], rtol=0, atol=1e-3)
        if np.abs(r["tau_c"]).max() > 0:
            n_contact += 1
        np.testing.assert_allclose(g["tau_c"][e, :n], r["tau_c"], rtol=0, atol=1e-3 * (np.abs(r["tau_c"]).max() + 1))
        err = qdd_rel_err(g["qdd"][e, :n], r["qdd"])
        worst["qdd"] = max(worst.get("qdd", 0.0), err)
    print("\n%s worst qdd rel err %.3e, envs in contact %d" % (name, worst["qdd"], n_contact))
    assert worst["qdd"] <= 1e-4
    if model.n_spheres:
        assert n_contact > 0, "no sampled env exercised the contact path"


def test_solve_stage_in_isolation():
    """The factorisation and solve: q_dd solves the oracle's own (M + dt D) with the GPU's rhs
    (separates the float-float solve from the FP32 right-hand side)."""
    model = mg.config_model("c1_whole")
    om = ora.OracleModel(model)
    E = 256
    sim = _sim(model, E)
    q, qd, act, exc = random_states(model, E, seed=3)
    res = sim.eval(sim.pad_n(q), sim.pad_n(qd), sim.pad_m(act), sim.pad_m(exc))
    n = model.n_dofs
    for e in sample_envs(E, 16):
        r = oracle_eval(om, DT, q[e], qd[e], act[e], exc[e])
        b = res["rhs"][e, :n].double().cpu().numpy()
        x = np.linalg.solve(r["A"], b)
        assert qdd_rel_err(res["qdd"][e, :n].double().cpu().numpy(), x) < 1e-4


@pytest.mark.parametrize("name,E,k,excite", [("c0_tiny", 64, 64, "uniform"), ("c1_whole", 4096, 24, "smooth")])
def test_trajectory_parity_100_steps(name, E, k, excite):
    """100 substeps from identical states: q within 1e-3 rad of the oracle."""
    model = mg.config_model(name)
    om = ora.OracleModel(model)
    sim = _sim(model, E)
    q0, qd0, a0 = mg.initial_state(model, E, seed=5)
    steps = 100
    gen = mg.uniform_excitations if excite == "uniform" else mg.smooth_excitations
    exc = gen(model, E, steps, seed=5)
    sim.reset(sim.pad_n(q0), sim.pad_n(qd0), sim.pad_m(a0))
    exc_d = [sim.pad_m(exc[t]) for t in range(steps)]
    for t in range(steps):
        sim.step(exc_d[t], 1)
    st = sim.state()
    qg = _np(st["q"], model.n_dofs)
    idx = sample_envs(E, k)
    q, qd, act = q0[idx].astype(np.float64), qd0[idx].astype(np.float64), a0[idx].astype(np.float64)
    for t in range(steps):
        q, qd, act, *_ = ora.step(om, DT, q, qd, act, exc[t][idx].astype(np.float64), 1)
    dq = np.abs(qg[idx] - q).max(axis=1)
    print("\n%s q max-abs diff after %d steps: median %.2e max %.2e" % (name, steps, np.median(dq), dq.max()))
    assert dq.max() <= 1e-3


def test_substeps_in_one_call_equal_separate_calls_bitwise():
    model = mg.config_model("c1_whole")
    E = 512
    a, b = _sim(model, E), _sim(model, E)
    q0, qd0, a0 = mg.initial_state(model, E, seed=2)
    exc = a.pad_m(mg.smooth_excitations(model, E, 1, seed=2)[0])
    for s in (a, b):
        s.reset(s.pad_n(q0), s.pad_n(qd0), s.pad_m(a0))
    a.step(exc, 10)
    for _ in range(10):
        b.step(exc, 1)
    sa, sb = a.state(), b.state()
    for key in ("q", "qd", "act", "qdd", "force"):
        assert torch.equal(sa[key], sb[key]), key


def test_cuda_graph_replay_is_bitwise_equal_to_eager():
    model = mg.config_model("c1_whole")
    E = 512
    a, b = _sim(model, E), _sim(model, E)
    q0, qd0, a0 = mg.initial_state(model, E, seed=4)
    exc = a.pad_m(mg.smooth_excitations(model, E, 1, seed=4)[0])
    for s in (a, b):
        s.reset(s.pad_n(q0), s.pad_n(qd0), s.pad_m(a0))
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        a.step(exc, 5)
    torch.cuda.synchronize()
    # capture does not execute: replay three times == three eager calls
    a.reset(a.pad_n(q0), a.pad_n(qd0), a.pad_m(a0))
    torch.cuda.synchronize()
    for _ in range(3):
        g.replay()
    for _ in range(3):
        b.step(exc, 5)
    torch.cuda.synchronize()
    sa, sb = a.state(), b.state()
    for key in ("q", "qd", "act"):
        assert torch.equal(sa[key], sb[key]), key


def test_launch_shape_does_not_change_results():
    """Warps per environment, environments per block and which image sections stay in global
    memory (via points; also muscle records at staging level 2) change only the speed: states after 20 substeps agree (bit-exact except the order of one float-float
    dot product, so within 1e-6 relative)."""
    model = mg.config_model("c1_whole")
    E = 300
    q0, qd0, a0 = mg.initial_state(model, E, seed=6)
    exc = mg.smooth_excitations(model, E, 1, seed=6)[0]
    ref = None
    for epb, pts, wpe in ((0, -1, 0), (0, 1, 1), (3, 0, 1), (0, 0, 2), (3, 1, 2), (0, 1, 4), (2, 0, 4), (0, 2, 2),
                          (5, 2, 1), (3, 2, 4)):
        sim = _sim(model, E)
        sim.set_launch(0, epb, pts, wpe)
        sim.reset(sim.pad_n(q0), sim.pad_n(qd0), sim.pad_m(a0))
        sim.step(sim.pad_m(exc), 20)
        st = sim.state()
        q = st["q"][:, : model.n_dofs].double().cpu().numpy()
        assert sim.status() == (0, 0)
        if ref is None:
            ref = q
        else:
            np.testing.assert_allclose(q, ref, rtol=1e-6, atol=1e-6)
        sim.close()


def test_reset_subset_and_status_flags():
    model = mg.config_model("c0_tiny")
    E = 32
    sim = _sim(model, E)
    q0, qd0, a0 = mg.initial_state(model, E, seed=1)
    sim.reset(sim.pad_n(q0), sim.pad_n(qd0), sim.pad_m(a0))
    # poison env 7 from the host side: NaN in q -> MSIM_ENV_NONFINITE for env 7 only
    bad = q0[[7]].copy()
    bad[0, 0] = np.nan
    ids = torch.tensor([7], dtype=torch.int32, device="cuda")
    sim.reset(sim.pad_n(bad), None, None, env_ids=ids)
    sim.step(sim.zeros(sim.pitch_m), 2)
    code, flags = sim.status()
    assert code == 6 and flags & msim.ENV_NONFINITE
    st = sim.state()["status"].cpu().numpy()
    assert st[7] & msim.ENV_NONFINITE
    assert np.all(st[np.arange(E) != 7] == 0)
    # resetting that env clears its bit; the others kept their state
    qbefore = sim.state()["q"].clone()
    sim.reset(sim.pad_n(q0[[7]]), sim.pad_n(qd0[[7]]), sim.pad_m(a0[[7]]), env_ids=ids)
    after = sim.state()
    assert after["status"][7].item() == 0
    keep = [i for i in range(E) if i != 7]
    assert torch.equal(after["q"][keep], qbefore[keep])
    assert torch.equal(after["q"][7, : model.n_dofs].cpu(), torch.from_numpy(q0[7]))
    sim.clear_status()
    assert sim.status() == (0, 0)


def test_not_spd_is_flagged():
    """A massless, inertia-free leaf body makes M singular: flagged per env, no trap."""
    base = mg.config_model("c0_tiny")
    mm = mg.Model(**dict(base.__dict__))
    leaf = [b for b in range(base.n_bodies) if b not in set(base.body_parent.tolist())][0]
    mm.body_mass = base.body_mass.copy(); mm.body_mass[leaf] = 0.0
    mm.body_inertia = base.body_inertia.copy(); mm.body_inertia[leaf] = 0.0
    sim = _sim(mm, 8)
    sim.step(sim.zeros(sim.pitch_m), 1)
    code, flags = sim.status()
    assert code == 6 and flags & msim.ENV_NOT_SPD


def test_argument_errors():
    model = mg.config_model("c0_tiny")
    sim = _sim(model, 8)
    exc = sim.zeros(sim.pitch_m)
    with pytest.raises(msim.MsimError) as ei:
        sim.step(exc, 0)
    assert ei.value.code == 1
    raw = torch.zeros(8 * sim.pitch_m + 1, device="cuda")
    st = sim.lib.msim_step(sim.h, raw.data_ptr() + 4, 1, None)
    assert st == 1
    assert sim.lib.msim_step(sim.h, None, 1, None) == 1
    with pytest.raises(msim.MsimError):
        sim.set_launch(0, 99)


def test_step_host_matches_device_step():
    model = mg.config_model("c1_whole")
    E = 256
    a, b = _sim(model, E), _sim(model, E)
    q0, qd0, a0 = mg.initial_state(model, E, seed=8)
    for s in (a, b):
        s.reset(s.pad_n(q0), s.pad_n(qd0), s.pad_m(a0))
    exc = np.zeros((E, a.pitch_m), np.float32)
    exc[:, : model.n_muscles] = mg.smooth_excitations(model, E, 1, seed=8)[0]
    exc_pinned = torch.from_numpy(exc).pin_memory()
    q_out = torch.zeros((E, a.pitch_n)).pin_memory()
    qd_out = torch.zeros((E, a.pitch_n)).pin_memory()
    a.step_host(exc_pinned, 10, q_out, qd_out)
    b.step(torch.from_numpy(exc).cuda(), 10)
    sb = b.state()
    assert torch.equal(q_out, sb["q"].cpu()) and torch.equal(qd_out, sb["qd"].cpu())


def test_mixed_models_in_one_handle_match_separate_handles():
    ma, mb = mg.config_model("c2_upper"), mg.config_model("c2_lower")
    Ea, Eb = 40, 24
    both = msim.Sim([ma, mb], [Ea, Eb], dt=5e-4)
    sa, sb = msim.Sim([ma], [Ea], dt=5e-4), msim.Sim([mb], [Eb], dt=5e-4)
    qa, qda, aa = mg.initial_state(ma, Ea, seed=1)
    qb, qdb, ab = mg.initial_state(mb, Eb, seed=2)
    P = lambda s, x, cols: s._pad(x, cols)
    both.reset(torch.cat([P(both, qa, both.pitch_n), P(both, qb, both.pitch_n)]),
               torch.cat([P(both, qda, both.pitch_n), P(both, qdb, both.pitch_n)]),
               torch.cat([P(both, aa, both.pitch_m), P(both, ab, both.pitch_m)]))
    sa.reset(sa.pad_n(qa), sa.pad_n(qda), sa.pad_m(aa))
    sb.reset(sb.pad_n(qb), sb.pad_n(qdb), sb.pad_m(ab))
    ea = mg.uniform_excitations(ma, Ea, 1, seed=3)[0]
    eb = mg.uniform_excitations(mb, Eb, 1, seed=4)[0]
    both.step(torch.cat([P(both, ea, both.pitch_m), P(both, eb, both.pitch_m)]), 10)
    sa.step(sa.pad_m(ea), 10)
    sb.step(sb.pad_m(eb), 10)
    s_all, s_a, s_b = both.state(), sa.state(), sb.state()
    assert torch.equal(s_all["q"][:Ea, : ma.n_dofs], s_a["q"][:, : ma.n_dofs])
    assert torch.equal(s_all["q"][Ea:, : mb.n_dofs], s_b["q"][:, : mb.n_dofs])


def test_mixed_batch_trajectory_parity():
    """The mixed batch's persistent launch (three skeletons in one kernel, 0.5 ms substeps, as the
    mixed-batch workload runs them): 100 substeps against the oracle on sampled environments of
    every skeleton, q within 1e-3 rad."""
    names = ("c2_upper", "c2_lower", "c1_whole")
    models = [mg.config_model(nm) for nm in names]
    envs = [96, 96, 64]
    dt = 5e-4
    sim = msim.Sim(models, envs, dt=dt)
    sim.set_mixed_launch(True)
    states = [mg.initial_state(mm, e, seed=21 + i) for i, (mm, e) in enumerate(zip(models, envs))]
    steps = 100
    excs = [mg.smooth_excitations(mm, e, steps, seed=21 + i, dt=dt) for i, (mm, e) in enumerate(zip(models, envs))]
    sim.reset(torch.cat([sim.pad_n(s[0]) for s in states]), torch.cat([sim.pad_n(s[1]) for s in states]),
              torch.cat([sim.pad_m(s[2]) for s in states]))
    for t in range(steps):
        sim.step(torch.cat([sim.pad_m(x[t]) for x in excs]), 1)
    qg = sim.state()["q"].double().cpu().numpy()
    assert sim.status() == (0, 0)
    row0 = 0
    for mm, e, (q0, qd0, a0), ex in zip(models, envs, states, excs):
        om = ora.OracleModel(mm)
        idx = sample_envs(e, 8)
        q, qd, act = q0[idx].astype(np.float64), qd0[idx].astype(np.float64), a0[idx].astype(np.float64)
        for t in range(steps):
            q, qd, act, *_ = ora.step(om, dt, q, qd, act, ex[t][idx].astype(np.float64), 1)
        dq = np.abs(qg[row0 + np.asarray(idx), : mm.n_dofs] - q).max(axis=1)
        print("\n%s (mixed launch) q max-abs diff after %d substeps: %.2e" % (mm.name, steps, dq.max()))
        assert dq.max() <= 1e-3
        row0 += e

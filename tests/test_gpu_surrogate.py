"""Learned muscle geometry: the label kernel, training, inference in the step, and the fallback.

The surrogate is judged against the exact path it replaces (its labels come from the exact
geometry kernel, itself checked here against the FP64 oracle).  Deterministic properties are
checked exactly: an environment that uses the exact geometry inside a learned-geometry step
(checked, outside the box, or flagged) follows the exact path bit for bit.  Accuracy is reported
and compared with the untrained network (what training gains), not with a hard 1 mm bound, which
the configured network does not reach everywhere; the per-environment check and fallback are
what keep the dynamics within it.
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
E = 512


def _box(model, margin):
    lo, hi = model.dof_limit[:, 0].astype(np.float64), model.dof_limit[:, 1].astype(np.float64)
    c, hw = 0.5 * (lo + hi), 0.5 * (hi - lo)
    on = lo < hi
    return np.where(on, c, 0.0), np.where(on, hw * (1 + margin), np.pi)


def _q_in_box(model, rows, seed, margin=0.05, frac=0.98):
    c, s = _box(model, margin)
    rng = np.random.default_rng(seed)
    return (c + frac * s * rng.uniform(-1, 1, (rows, model.n_dofs))).astype(np.float32)


@pytest.fixture(scope="module")
def trained():
    model = mg.config_model("c1_whole")
    sim = msim.Sim(model, E, dt=DT, seed=3)
    sim.train_surrogate(524288, 8, batch=4096, lr=1e-3)
    return model, sim


def _exact_twin(model, q0, qd0, a0):
    ex = msim.Sim(model, E, dt=DT, seed=3)
    ex.reset(ex.pad_n(q0), ex.pad_n(qd0), ex.pad_m(a0))
    return ex


@pytest.mark.parametrize("name", ["c0_tiny", "c1_whole"])
def test_geometry_kernel_matches_oracle(name):
    model = mg.config_model(name)
    sim = msim.Sim(model, 8, dt=DT)
    lim = model.dof_limit
    has = lim[:, 0] < lim[:, 1]
    rng = np.random.default_rng(5)
    rows = 300   # several blocks and a ragged tail
    q = rng.uniform(-1.0, 1.0, (rows, model.n_dofs)).astype(np.float32)
    q[:, has] = np.clip(q[:, has], lim[has, 0], lim[has, 1])
    out = sim.geometry(sim._pad(q, sim.pitch_n)).double().cpu().numpy()
    lay = sim.layout(0)
    m = model.n_muscles
    for r in sample_envs(rows, 24, seed=1):
        L, R = ora.muscle_geometry(model, q[r].astype(np.float64))
        np.testing.assert_allclose(out[r, :m], L, rtol=0, atol=5e-6)
        np.testing.assert_allclose(msim.unpack_R(out[r, m:], lay, model.n_dofs), R, rtol=0, atol=5e-6)


def test_training_gains_over_the_untrained_network(trained):
    model, sim = trained
    q = torch.from_numpy(_q_in_box(model, 2048, seed=77)).cuda()
    qp = torch.zeros((q.shape[0], sim.pitch_n), device="cuda")
    qp[:, : model.n_dofs] = q
    exact = sim.geometry(qp)
    pred = sim.surrogate_predict(qp)
    net = sim.surrogate_network()
    trained_params = net.get(0)
    fresh = msim.MLP(model.n_dofs, 512, net.d_out, max_batch=16, seed=3 * 2654435761 + 17 & (2**64 - 1))
    net.set(fresh.get(0))   # the same initialisation the training started from
    fresh.close()
    pred0 = sim.surrogate_predict(qp)
    net.set(trained_params)
    m = model.n_muscles
    e1, e0 = (pred - exact).abs(), (pred0 - exact).abs()
    rms1, rms0 = float(e1.pow(2).mean().sqrt()), float(e0.pow(2).mean().sqrt())
    print("\nsurrogate |error| m: trained median L %.2e R %.2e, rms %.2e; untrained rms %.2e; "
          "envs with max <= 1 mm: %.3f" % (float(e1[:, :m].median()), float(e1[:, m:].median()), rms1, rms0,
                                          float((e1.max(1).values <= 1e-3).float().mean())))
    assert rms1 < 0.35 * rms0
    assert float(e1[:, m:].median()) < 5e-3


def test_checked_environments_follow_the_exact_path_bitwise(trained):
    model, sim = trained
    q0, qd0, a0 = mg.initial_state(model, E, seed=8)
    sim.reset(sim.pad_n(q0), sim.pad_n(qd0), sim.pad_m(a0))
    ex = _exact_twin(model, q0, qd0, a0)
    exc = sim.pad_m(mg.smooth_excitations(model, E, 1, seed=8)[0])
    sim.set_geometry_mode(1)
    sim.surrogate_set_check(1.0, 1e-3)
    sim.surrogate_stats(reset=True)
    try:
        for _ in range(5):
            sim.step(exc, 2)
            ex.step(exc, 2)
        sa, sb = sim.state(), ex.state()
        for k in ("q", "qd", "act", "qdd", "force"):
            assert torch.equal(sa[k], sb[k]), k
        st = sim.surrogate_stats()
        assert st["env_substeps"] == 10 * E and st["learned"] == 0
        assert st["checked"] + st["flagged"] + st["out_of_box"] >= 10 * E
    finally:
        sim.set_geometry_mode(0)
        sim.surrogate_set_check(0.01, 1e-3)


def test_out_of_box_environments_use_the_exact_geometry(trained):
    model, sim = trained
    q0, qd0, a0 = mg.initial_state(model, E, seed=9)
    c, s = _box(model, 0.05)
    out = np.arange(0, E, 7)   # every 7th environment leaves the box in one DoF
    d = int(np.argmax(model.dof_limit[:, 1] - model.dof_limit[:, 0]))
    q0[out, d] = (c[d] + 1.2 * s[d]).astype(np.float32)
    sim.reset(sim.pad_n(q0), sim.pad_n(qd0), sim.pad_m(a0))
    ex = _exact_twin(model, q0, qd0, a0)
    exc = sim.pad_m(mg.smooth_excitations(model, E, 1, seed=9)[0])
    sim.set_geometry_mode(1)
    sim.surrogate_set_check(0.0, 1e-3)
    sim.surrogate_stats(reset=True)
    try:
        sim.step(exc, 1)
        ex.step(exc, 1)
        sa, sb = sim.state(), ex.state()
        for k in ("q", "qd", "act"):
            assert torch.equal(sa[k][out], sb[k][out]), k
        st = sim.surrogate_stats()
        assert st["out_of_box"] == len(out) and st["learned"] == E - len(out)
    finally:
        sim.set_geometry_mode(0)
        sim.surrogate_set_check(0.01, 1e-3)


def test_injected_network_error_is_caught_and_falls_back_until_reset(trained):
    model, sim = trained
    net = sim.surrogate_network()
    good = net.get(0)
    bad = good.copy()
    b3 = net.offsets[5]
    bad[b3] += 50.0   # muscle 0's length off by 50 standard deviations
    q0, qd0, a0 = mg.initial_state(model, E, seed=10)
    sim.reset(sim.pad_n(q0), sim.pad_n(qd0), sim.pad_m(a0))
    exc = sim.pad_m(mg.smooth_excitations(model, E, 1, seed=10)[0])
    sim.set_geometry_mode(1)
    sim.surrogate_set_check(0.25, 1e-3)
    sim.surrogate_stats(reset=True)
    try:
        net.set(bad)
        for _ in range(40):
            sim.step(exc, 1)
        st = sim.surrogate_stats()
        # every check fails; a checked environment stays on the exact geometry afterwards
        assert st["checked"] > 0 and st["check_failed"] == st["checked"]
        assert st["flagged_envs"] == st["check_failed"] and st["max_check_error"] > 2e-3
        print("\ninjected error: %d of %d envs flagged after 40 substeps at 25 %% checks"
              % (st["flagged_envs"], E))
        sim.reset(sim.pad_n(q0), sim.pad_n(qd0), sim.pad_m(a0))
        assert sim.surrogate_stats()["flagged_envs"] == 0
    finally:
        net.set(good)
        sim.set_geometry_mode(0)
        sim.surrogate_set_check(0.01, 1e-3)


def test_learned_step_accelerations_against_the_oracle(trained):
    model, sim = trained
    q, qd, act, exc = random_states(model, E, seed=12, q_scale=0.3)
    sim.reset(sim.pad_n(q), sim.pad_n(qd), sim.pad_m(act))
    sim.set_geometry_mode(1)
    sim.surrogate_set_check(0.0, 1e-3)
    try:
        sim.step(sim.pad_m(exc), 1)
        qdd = sim.state()["qdd"][:, : model.n_dofs].double().cpu().numpy()
    finally:
        sim.set_geometry_mode(0)
        sim.surrogate_set_check(0.01, 1e-3)
    om = ora.OracleModel(model)
    errs = [qdd_rel_err(qdd[e], oracle_eval(om, DT, q[e], qd[e], act[e], exc[e])["qdd"])
            for e in sample_envs(E, 16, seed=4)]
    print("\nlearned-geometry qdd rel. error vs FP64 oracle (exact geometry): median %.2e max %.2e"
          % (np.median(errs), np.max(errs)))
    assert np.isfinite(errs).all()


def test_surrogate_argument_and_state_errors():
    model = mg.config_model("c0_tiny")
    sim = msim.Sim(model, 8, dt=DT)
    with pytest.raises(msim.MsimError, match="MSIM_ERR_STATE"):
        sim.set_geometry_mode(1)
    with pytest.raises(msim.MsimError, match="MSIM_ERR_ARG"):
        sim.train_surrogate(100, 1, batch=4096)
    two = msim.Sim([model, model], [4, 4], dt=DT)
    with pytest.raises(msim.MsimError, match="MSIM_ERR_UNSUPPORTED"):
        two.train_surrogate(4096, 1, batch=1024)
    sim.train_surrogate(8192, 1, batch=1024)
    net = sim.surrogate_network()
    assert sim.lib.msim_mlp_destroy(net.h) == 1   # borrowed: refused (MSIM_ERR_ARG)


def test_learned_geometry_steps_replay_from_a_cuda_graph(trained):
    """Without checks the learned-geometry step is deterministic: a captured graph of it replays
    bit for bit like the eager calls (input kernel, network, step kernel per substep)."""
    model, sim = trained
    q0, qd0, a0 = mg.initial_state(model, E, seed=13)
    exc = sim.pad_m(mg.smooth_excitations(model, E, 1, seed=13)[0])
    sim.set_geometry_mode(1)
    sim.surrogate_set_check(0.0, 1e-3)
    try:
        sim.reset(sim.pad_n(q0), sim.pad_n(qd0), sim.pad_m(a0))
        for _ in range(3):
            sim.step(exc, 2)
        eager = sim.state()
        stream = torch.cuda.Stream()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            sim.step(exc, 2)
        torch.cuda.synchronize()
        sim.reset(sim.pad_n(q0), sim.pad_n(qd0), sim.pad_m(a0))
        sim.surrogate_stats(reset=True)
        for _ in range(3):
            g.replay()
        torch.cuda.synchronize()
        replay = sim.state()
        for k in ("q", "qd", "act"):
            assert torch.equal(eager[k], replay[k]), k
        assert sim.surrogate_stats()["env_substeps"] == 6 * E
    finally:
        sim.set_geometry_mode(0)
        sim.surrogate_set_check(0.01, 1e-3)

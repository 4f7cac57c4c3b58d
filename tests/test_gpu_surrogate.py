"""Learned muscle geometry: the label kernel, training, inference in the step, and the fallback.

The surrogate is judged against the exact path it replaces (its labels come from the exact
geometry kernel, itself checked here against the FP64 oracle).  Deterministic properties are
checked exactly: an environment that uses the exact geometry inside a learned-geometry step
(checked, outside the box, or flagged) follows the exact path bit for bit.  The substep that
consumes the network's geometry is pinned to the oracle fed the same geometry (q_dd within
1e-4).  Accuracy at this file's small training budget is compared with the best constant
predictor and with the dense network (what training and the joint structure gain); a rollout
compares the learned path with the exact one in throughput and in q after 100 substeps.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as ora
from paper_2603_29332_b300 import modelgen as mg
from paper_2603_29332_b300 import msim
from tests import handmodels as hm
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
    sim.train_surrogate(1048576, 8, batch=4096, lr=3e-3)
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


def _fresh_errors(model, sim, rows=2048, seed=77):
    q = torch.from_numpy(_q_in_box(model, rows, seed=seed)).cuda()
    qp = torch.zeros((q.shape[0], sim.pitch_n), device="cuda")
    qp[:, : model.n_dofs] = q
    exact = sim.geometry(qp)
    return sim.surrogate_predict(qp) - exact, exact


def test_training_gains_over_the_best_constant_and_the_dense_network(trained):
    """At this file's small budget (1M samples, 8 epochs) the trained network's error is a
    fraction of the best constant predictor's (each output's mean), and the joint-structured
    network beats the dense one trained on the same samples."""
    model, sim = trained
    m = model.n_muscles
    err, exact = _fresh_errors(model, sim)
    rms1 = float(err.pow(2).mean().sqrt())
    rms0 = float((exact - exact.mean(0)).pow(2).mean().sqrt())
    dense = msim.Sim(model, E, dt=DT, seed=3)
    dense.surrogate_set_structure(False)
    dense.train_surrogate(1048576, 8, batch=4096, lr=3e-3)
    errd, _ = _fresh_errors(model, dense)
    rmsd = float(errd.pow(2).mean().sqrt())
    env_rms = err[:, m:].pow(2).mean(1).sqrt()
    print("\nsurrogate error (m): structured rms %.2e (median R %.2e, p99 R %.2e, envs with moment-arm rms "
          "<= 1 mm %.3f); dense rms %.2e; best constant rms %.2e"
          % (rms1, float(err[:, m:].abs().median()), float(err[:, m:].abs().flatten()[::7].quantile(0.99)),
             float((env_rms <= 1e-3).float().mean()), rmsd, rms0))
    assert rms1 < 0.2 * rms0
    assert rms1 < 0.8 * rmsd


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
    bad[b3:b3 + 100] += 50.0   # 100 muscle lengths off by 50 standard deviations each
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


def test_learned_substep_matches_the_oracle_fed_the_network_geometry(trained):
    """The learned-geometry substep on 512 environments against the FP64 oracle's substep given
    the network's own lengths and moment arms at the same FP32 state (msim_surrogate_predict):
    muscle forces and q_dd agree at the exact path's tolerances, so everything downstream of the
    geometry consumes the network's output as the method says.  The oracle with the exact
    geometry is reported beside it (the network's own error)."""
    model, sim = trained
    n, m = model.n_dofs, model.n_muscles
    q, qd, act, exc = random_states(model, E, seed=12, q_scale=0.3)
    sim.reset(sim.pad_n(q), sim.pad_n(qd), sim.pad_m(act))
    sim.set_geometry_mode(1)
    sim.surrogate_set_check(0.0, 1e-3)
    sim.surrogate_stats(reset=True)
    try:
        sim.step(sim.pad_m(exc), 1)
        st = sim.state()
        qdd = st["qdd"][:, :n].double().cpu().numpy()
        force = st["force"][:, :m].double().cpu().numpy()
        assert sim.surrogate_stats()["out_of_box"] == 0
    finally:
        sim.set_geometry_mode(0)
        sim.surrogate_set_check(0.01, 1e-3)
    geo = sim.surrogate_predict(sim.pad_n(q)).double().cpu().numpy()
    lay = sim.layout(0)
    om = ora.OracleModel(model)
    errs, errs_exact = [], []
    for e in sample_envs(E, 16, seed=4):
        Lg, Rg = geo[e, :m], msim.unpack_R(geo[e, m:], lay, n)
        r = ora.evaluate(om, DT, q[e].astype(np.float64), qd[e].astype(np.float64), act[e].astype(np.float64),
                         exc[e].astype(np.float64), L=Lg, R=Rg)
        assert r["status"] == 0
        np.testing.assert_allclose(force[e], r["force"], rtol=0, atol=2e-3 * model.muscle_fmax.max())
        errs.append(qdd_rel_err(qdd[e], r["qdd"]))
        errs_exact.append(qdd_rel_err(qdd[e], oracle_eval(om, DT, q[e], qd[e], act[e], exc[e])["qdd"]))
    print("\nlearned substep q_dd vs oracle fed the network geometry: max %.2e; vs oracle with the exact "
          "geometry: median %.2e max %.2e" % (np.max(errs), np.median(errs_exact), np.max(errs_exact)))
    assert np.max(errs) <= 1e-4


def test_learned_rollout_against_the_exact_rollout(trained):
    """100 substeps of 512 environments from the same state and excitations with the exact
    geometry, the trained network (checks off: every environment inside the box on the network)
    and the same network zeroed, which predicts every output's training mean (the learned path
    without training).  All three are timed with CUDA events; q after 100 substeps is compared
    with the exact rollout.  The trained network must stay much closer to the exact dynamics than
    the untrained one, with no state flagged."""
    model, sim = trained
    q0, qd0, a0 = mg.initial_state(model, E, seed=14)
    excs = [sim.pad_m(x) for x in mg.smooth_excitations(model, E, 100, seed=14)]
    ex = _exact_twin(model, q0, qd0, a0)
    net = sim.surrogate_network()
    good = net.get(0)
    res = {}

    def run(name, s_):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for t in range(100):
            s_.step(excs[t], 1)
        e1.record()
        torch.cuda.synchronize()
        res[name] = (e0.elapsed_time(e1), s_.state()["q"][:, : model.n_dofs].clone(), s_.status()[1])

    try:
        run("exact", ex)
        sim.set_geometry_mode(1)
        sim.surrogate_set_check(0.0, 1e-3)
        for name, params in (("trained", good), ("untrained", np.zeros_like(good))):
            net.set(params)
            sim.reset(sim.pad_n(q0), sim.pad_n(qd0), sim.pad_m(a0))
            sim.surrogate_stats(reset=True)
            run(name, sim)
            st = sim.surrogate_stats()
            assert st["learned"] + st["out_of_box"] == st["env_substeps"] == 100 * E
            if name == "trained":
                frac = st["learned"] / st["env_substeps"]
    finally:
        net.set(good)
        sim.set_geometry_mode(0)
        sim.surrogate_set_check(0.01, 1e-3)
    q_ex = res["exact"][1]
    drift = {k: (res[k][1] - q_ex).abs().max(1).values for k in ("trained", "untrained")}
    print("\nrollout 512 envs x 100 substeps: exact %.2f ms, learned %.2f ms (network on %.3f of env-substeps); "
          "|q - q_exact| after 100 substeps, median / max: trained %.2e / %.2e, untrained %.2e / %.2e"
          % (res["exact"][0], res["trained"][0], frac, float(drift["trained"].median()),
             float(drift["trained"].max()), float(drift["untrained"].median()), float(drift["untrained"].max())))
    assert res["trained"][2] == 0 and torch.isfinite(res["trained"][1]).all()
    assert frac >= 0.9
    assert float(drift["trained"].median()) < 0.5 * float(drift["untrained"].median())


def test_joint_structure_only_where_segments_cross_one_joint(trained):
    """The joint-block connectivity is used when every path segment joins points on the same or on
    adjacent bodies (the whole body), and the dense network otherwise: a chain whose only muscle
    runs straight from the root body to the third body has a length depending jointly on two
    joints, which the blocks could not represent."""
    model, sim = trained
    st = sim.surrogate_stats()
    assert st["structured"] == 1 and st["hidden"] == 512
    base = hm.chain(n_links=3, seed=2)
    spans_two = mg.make_model("two_joint_segment", base.body_parent, base.body_ndof, base.body_offset,
                              base.body_mass, base.body_com, base.body_inertia, base.dof_axis,
                              [[(0, (0.05, 0.02, 0.1)), (2, (0.02, 0.03, -0.05))]], [500.0], [0.1],
                              dof_limit=[[-1.0, 1.0]] * base.n_dofs)
    s2 = msim.Sim(spans_two, 16, dt=DT)
    s2.surrogate_set_width(64)
    s2.train_surrogate(8192, 1, batch=1024, lr=3e-3)
    assert s2.surrogate_stats()["structured"] == 0
    one = mg.make_model("one_joint_segments", base.body_parent, base.body_ndof, base.body_offset,
                        base.body_mass, base.body_com, base.body_inertia, base.dof_axis,
                        [[(0, (0.05, 0.02, 0.1)), (1, (0.02, 0.03, -0.05)), (2, (0.02, 0.03, -0.05))]], [500.0],
                        [0.1], dof_limit=[[-1.0, 1.0]] * base.n_dofs)
    s3 = msim.Sim(one, 16, dt=DT)
    s3.surrogate_set_width(64)
    s3.train_surrogate(8192, 1, batch=1024, lr=3e-3)
    assert s3.surrogate_stats()["structured"] == 1
    s3.surrogate_set_structure(False)
    s3.train_surrogate(8192, 1, batch=1024, lr=3e-3)
    assert s3.surrogate_stats()["structured"] == 0


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

"""Imitation reward on the device against the FP64 reward oracle, through the C ABI.

Body positions (forward kinematics mode of the step kernel) are compared to the oracle's own
kinematics; the discriminator sees BF16-rounded inputs on both sides (tolerance of the MLP tests);
the power term uses the forces and fibre velocities of the last substep, compared to the oracle's
evaluation at that substep's start state.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as ora
from oracle import reward_oracle as ro
from paper_2603_29332_b300 import modelgen as mg
from paper_2603_29332_b300 import msim
from tests.gpu_common import random_states, sample_envs

pytestmark = pytest.mark.gpu

DT = 1e-3


def _bf(z):
    return torch.as_tensor(np.asarray(z, np.float32)).bfloat16().double().numpy()


@pytest.mark.parametrize("name", ["c0_tiny", "c1_whole"])
def test_body_positions_match_the_oracle(name):
    model = mg.config_model(name)
    sim = msim.Sim(model, 4, dt=DT)
    q, *_ = random_states(model, 257, seed=3, q_scale=1.0)
    xp = sim.body_positions(sim._pad(q, sim.pitch_n)).double().cpu().numpy()
    for r in sample_envs(257, 20, seed=2):
        np.testing.assert_allclose(xp[r].reshape(-1, 3), ro.body_positions(model, q[r].astype(np.float64)),
                                   rtol=0, atol=3e-6)


def test_reward_against_the_oracle():
    model = mg.config_model("c1_whole")
    E, w = 256, 0.05
    n, nb, m = model.n_dofs, model.n_bodies, model.n_muscles
    sim = msim.Sim(model, E, dt=DT)
    disc = msim.MLP(n + 3 * nb, 64, 1, out_sigmoid=True, max_batch=E, seed=4, out_scale=0.3)
    sim.reward_attach(disc, w_power=w)
    q, qd, act, exc = random_states(model, E, seed=5, q_scale=0.3)
    q_ref, *_ = random_states(model, E, seed=6, q_scale=0.3)
    sim.reset(sim.pad_n(q), sim.pad_n(qd), sim.pad_m(act))
    sim.step(sim.pad_m(exc), 1)                       # F, v_m of this substep (start state q, qd, act)
    st = sim.state()
    r, parts, delta = sim.reward(sim.pad_n(q_ref), with_parts=True, with_delta=True)
    r, parts, delta = (t.double().cpu().numpy() for t in (r, parts, delta))
    qs = st["q"][:, :n].double().cpu().numpy()
    params = [np.asarray(x, np.float64) for x in disc.unflatten(disc.get(0))]
    for i in (0, 2, 4):
        params[i] = _bf(params[i])
    om = ora.OracleModel(model)
    worst = 0.0
    for e in sample_envs(E, 12, seed=7):
        d_ref = ro.tracking_error(model, qs[e], q_ref[e].astype(np.float64))
        np.testing.assert_allclose(delta[e], d_ref, rtol=0, atol=5e-6)
        ev = ora.evaluate(om, DT, q[e].astype(np.float64), qd[e].astype(np.float64), act[e].astype(np.float64),
                          exc[e].astype(np.float64))
        rp = ro.reward_power(ev["force"], ev["vm"])
        np.testing.assert_allclose(parts[e, 1], rp, rtol=2e-3, atol=1e-3)
        rt = ro.reward(model, params, qs[e], q_ref[e].astype(np.float64), np.zeros(m), np.zeros(m), 0.0,
                       in_round=_bf)
        np.testing.assert_allclose(parts[e, 0], rt, rtol=2e-2, atol=1e-3)
        np.testing.assert_allclose(r[e], parts[e, 0] + w * parts[e, 1], rtol=1e-6, atol=1e-6)
        worst = max(worst, abs(parts[e, 1] - rp) / max(abs(rp), 1e-3))
    print("\nreward: power-term worst rel. error vs oracle %.2e" % worst)


def test_reward_in_a_cuda_graph_and_errors():
    model = mg.config_model("c1_whole")
    E = 64
    n, nb = model.n_dofs, model.n_bodies
    sim = msim.Sim(model, E, dt=DT)
    with pytest.raises(msim.MsimError, match="MSIM_ERR_STATE"):
        sim.reward(sim.zeros(sim.pitch_n))
    bad = msim.MLP(n + 3 * nb, 64, 1, out_sigmoid=False, max_batch=E)
    with pytest.raises(msim.MsimError, match="MSIM_ERR_ARG"):
        sim.reward_attach(bad)
    disc = msim.MLP(n + 3 * nb, 64, 1, out_sigmoid=True, max_batch=E, seed=1)
    sim.reward_attach(disc, w_power=0.1)
    q0, qd0, a0 = mg.initial_state(model, E, seed=1)
    exc = sim.pad_m(mg.smooth_excitations(model, E, 1, seed=1)[0])
    q_ref = sim.pad_n(q0)
    sim.reset(sim.pad_n(q0), sim.pad_n(qd0), sim.pad_m(a0))
    r0, _, _ = sim.reward(q_ref)
    r_out = torch.zeros(E, device="cuda")
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        sim.step(exc, 2)
        r, _, _ = sim.reward(q_ref)
        r_out.copy_(r)
    torch.cuda.synchronize()
    sim.reset(sim.pad_n(q0), sim.pad_n(qd0), sim.pad_m(a0))
    g.replay()
    torch.cuda.synchronize()
    sim2 = msim.Sim(model, E, dt=DT)
    sim2.reward_attach(disc, w_power=0.1)
    sim2.reset(sim2.pad_n(q0), sim2.pad_n(qd0), sim2.pad_m(a0))
    sim2.step(exc, 2)
    r2, _, _ = sim2.reward(q_ref)
    assert torch.equal(r_out, r2)
    assert torch.isfinite(r0).all() and torch.isfinite(r2).all()

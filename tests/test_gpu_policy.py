"""Policy network in the loop: observation -> 3-layer MLP -> excitations -> substeps, on the GPU.

The in-library loop must equal the same loop assembled by hand from the public pieces (state
read-out, msim_mlp_forward, msim_step) bit for bit, eagerly and replayed from a CUDA graph.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2603_29332_b300 import modelgen as mg
from paper_2603_29332_b300 import msim

pytestmark = pytest.mark.gpu

DT = 1e-3
OBS = 2182   # policy input width of the closed-loop workload (zero-padded observation)


def _setup(E, seed):
    model = mg.config_model("c1_whole")
    sims = [msim.Sim(model, E, dt=DT) for _ in range(2)]
    q0, qd0, a0 = mg.initial_state(model, E, seed=seed)
    for s in sims:
        s.reset(s.pad_n(q0), s.pad_n(qd0), s.pad_m(a0))
    net = msim.MLP(OBS, 1024, model.n_muscles, out_sigmoid=True, max_batch=E, seed=seed, out_scale=1.0)
    return model, sims, net


def _manual_act(sim, model, net, n_sub):
    n, m = model.n_dofs, model.n_muscles
    st = sim.state()
    inv = torch.from_numpy((np.float32(1.0) / model.muscle_fmax.astype(np.float32)).astype(np.float32)).cuda()
    obs = torch.zeros((sim.n_envs, net.in_pitch), dtype=torch.float32, device="cuda")
    obs[:, :n] = st["q"][:, :n]
    obs[:, n:2 * n] = st["qd"][:, :n]
    obs[:, 2 * n:2 * n + m] = st["act"][:, :m]
    obs[:, 2 * n + m:2 * n + 2 * m] = st["force"][:, :m] * inv
    y = net.forward(obs.bfloat16())
    exc = torch.zeros((sim.n_envs, sim.pitch_m), device="cuda")
    exc[:, :m] = y[:, :m]
    sim.step(exc, n_sub)
    return exc


def test_policy_loop_equals_the_loop_assembled_by_hand():
    E = 256
    model, (a, b), net = _setup(E, seed=2)
    a.policy_attach(net)
    for _ in range(3):
        a.policy_step(2, 1)
        exc = _manual_act(b, model, net, 2)
        assert torch.equal(a.policy_excitations(), exc)
    sa, sb = a.state(), b.state()
    for k in ("q", "qd", "act", "force"):
        assert torch.equal(sa[k], sb[k]), k
    assert float(exc[:, : model.n_muscles].min()) >= 0.0 and float(exc.max()) <= 1.0


def test_policy_rollout_replays_from_a_cuda_graph():
    E = 128
    model, (a, b), net = _setup(E, seed=5)
    for s in (a, b):
        s.policy_attach(net)
    q0, qd0, a0 = mg.initial_state(model, E, seed=5)
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        a.policy_step(2, 5)
    torch.cuda.synchronize()
    a.reset(a.pad_n(q0), a.pad_n(qd0), a.pad_m(a0))
    torch.cuda.synchronize()
    for _ in range(2):
        g.replay()
        b.policy_step(2, 5)
    torch.cuda.synchronize()
    sa, sb = a.state(), b.state()
    for k in ("q", "qd", "act"):
        assert torch.equal(sa[k], sb[k]), k


def test_policy_binding_errors():
    model = mg.config_model("c1_whole")
    sim = msim.Sim(model, 16, dt=DT)
    with pytest.raises(msim.MsimError, match="MSIM_ERR_STATE"):
        sim.policy_step(2, 1)
    wrong = msim.MLP(OBS, 64, 10, out_sigmoid=True, max_batch=16)
    with pytest.raises(msim.MsimError, match="MSIM_ERR_ARG"):
        sim.policy_attach(wrong)
    small = msim.MLP(OBS, 64, model.n_muscles, out_sigmoid=True, max_batch=8)
    with pytest.raises(msim.MsimError, match="MSIM_ERR_ARG"):
        sim.policy_attach(small)

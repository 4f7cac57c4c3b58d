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


# ---------------------------------------------------------------- flow refinement of the action
def _flow_setup(E, seed, hid=1024, sigma=0.0, n_steps=20, dt=0.05):
    model, (a, b), net = _setup(E, seed)
    flow = msim.MLP(OBS + model.n_muscles + 1, hid, model.n_muscles, max_batch=E, seed=seed + 100, out_scale=1.0)
    for s in (a, b):
        s.policy_attach(net)
    a.flow_attach(flow, n_steps=n_steps, dt=dt, sigma=sigma)
    return model, a, b, net, flow


def _obs(sim, model, pitch):
    n, m = model.n_dofs, model.n_muscles
    st = sim.state()
    inv = torch.from_numpy((np.float32(1.0) / model.muscle_fmax.astype(np.float32)).astype(np.float32)).cuda()
    obs = torch.zeros((sim.n_envs, pitch), dtype=torch.float32, device="cuda")
    obs[:, :n] = st["q"][:, :n]
    obs[:, n:2 * n] = st["qd"][:, :n]
    obs[:, 2 * n:2 * n + m] = st["act"][:, :m]
    obs[:, 2 * n + m:2 * n + 2 * m] = st["force"][:, :m] * inv
    return obs


def _flow_velocity_split(flow, params, xb, pre, c):
    """The flow network's forward as the library evaluates it inside the refinement loop, from
    public GEMM calls: the first layer's share of input columns [0, c) (the observation, the same at
    every Euler step) is the FP32 addend `pre`, and only columns [c, in) are multiplied again."""
    W1, b1, W2, b2, W3, b3 = [torch.as_tensor(np.asarray(x, np.float32)).cuda() for x in params]
    W1p = torch.zeros((W1.shape[0], flow.in_pitch), device="cuda")
    W1p[:, : W1.shape[1]] = W1
    W1b, W2b, W3b = W1p.bfloat16(), W2.bfloat16(), W3.bfloat16()
    if pre is None:
        pre = msim.gemm_bf16(xb[:, :c], W1b[:, :c])
    h1 = msim.gemm_bf16(xb[:, c:flow.d_in], W1b[:, c:flow.d_in], b1, act=1, out_bf16=True, addend=pre)
    h2 = msim.gemm_bf16(h1, W2b, b2, act=1, out_bf16=True)
    return msim.gemm_bf16(h2, W3b, b3), pre


def test_flow_refined_loop_equals_the_loop_assembled_by_hand():
    E, n_steps, dt = 128, 20, 0.05
    model, a, b, net, flow = _flow_setup(E, seed=7, n_steps=n_steps, dt=dt)
    m = model.n_muscles
    params = flow.unflatten(flow.get(0))
    c = (OBS // 8) * 8   # the observation columns the library keeps across the Euler steps
    for _ in range(2):
        a.policy_step(2, 1)
        obs = _obs(b, model, net.in_pitch)
        mu = net.forward(obs.bfloat16())[:, :m]
        act = mu.clone()
        x = torch.zeros((E, flow.in_pitch), dtype=torch.float32, device="cuda")
        x[:, :OBS] = obs[:, :OBS]
        pre = None
        for j in range(n_steps):
            x[:, OBS:OBS + m] = act
            x[:, OBS + m] = j * dt
            v, pre = _flow_velocity_split(flow, params, x.bfloat16(), pre, c)
            v = v[:, :m]
            act = act + torch.tensor(dt, dtype=torch.float32) * v
        exc = torch.zeros((E, b.pitch_m), device="cuda")
        exc[:, :m] = act.clamp(0.0, 1.0)
        b.step(exc, 2)
        mu_a, act_a = a.flow_actions()
        assert torch.equal(mu_a[:, :m], mu) and torch.equal(act_a[:, :m], act)
        assert torch.equal(a.policy_excitations(), exc)
    sa, sb = a.state(), b.state()
    for k in ("q", "qd", "act"):
        assert torch.equal(sa[k], sb[k]), k


def test_flow_refinement_against_the_fp64_oracle():
    from oracle import mlp_oracle as mo
    E, n_steps, dt = 64, 20, 0.05
    model, a, b, net, flow = _flow_setup(E, seed=9, hid=64, n_steps=n_steps, dt=dt)
    m = model.n_muscles
    obs = _obs(a, model, net.in_pitch)
    a.policy_step(1, 1)
    mu_g, act_g = a.flow_actions()
    bf = lambda z: torch.as_tensor(z, dtype=torch.float32).bfloat16().double().numpy()
    pp = [np.asarray(x, np.float64) for x in net.unflatten(net.get(0))]
    fp = [np.asarray(x, np.float64) for x in flow.unflatten(flow.get(0))]
    for p_ in (pp, fp):
        for i in (0, 2, 4):
            p_[i] = bf(p_[i])
    o = bf(obs[:, :OBS].cpu().numpy())
    mu, _ = mo.forward(pp, o, out_sigmoid=True)
    ref = mo.flow_refine(mu, mo.mlp_velocity(fp, o, in_round=bf), n_steps, dt)
    got = act_g[:, :m].double().cpu().numpy()
    drift = np.abs(ref - mu).max()
    err = np.abs(got - ref).max()
    print("\nflow refinement: max |a - a0| %.3e, max |gpu - oracle| %.3e" % (drift, err))
    assert err <= 2e-2 * max(drift, 1e-3) + 2e-3


def test_flow_initial_sampler_noise_statistics():
    E, sigma = 1024, 0.1
    model, a, b, net, flow = _flow_setup(E, seed=11, hid=64, sigma=sigma, n_steps=0)
    m = model.n_muscles
    a.policy_step(1, 1)
    mu, act = a.flow_actions()
    z1 = ((act - mu)[:, :m] / sigma).double().cpu().numpy().ravel()
    a.policy_step(1, 1)
    mu2, act2 = a.flow_actions()
    z2 = ((act2 - mu2)[:, :m] / sigma).double().cpu().numpy().ravel()
    N = z1.size
    for z in (z1, z2):
        assert abs(z.mean()) < 5 / np.sqrt(N) and abs(z.std() - 1) < 0.01
        assert abs((z ** 4).mean() - 3) < 0.05   # normal kurtosis
    assert abs(np.corrcoef(z1, z2)[0, 1]) < 5 / np.sqrt(N)   # a new draw every control step


def test_flow_binding_errors():
    model = mg.config_model("c1_whole")
    sim = msim.Sim(model, 16, dt=DT)
    flow = msim.MLP(OBS + model.n_muscles + 1, 64, model.n_muscles, max_batch=16)
    with pytest.raises(msim.MsimError, match="MSIM_ERR_STATE"):
        sim.flow_attach(flow)
    pol = msim.MLP(OBS, 64, model.n_muscles, out_sigmoid=True, max_batch=16)
    sim.policy_attach(pol)
    bad = msim.MLP(OBS + model.n_muscles, 64, model.n_muscles, max_batch=16)
    with pytest.raises(msim.MsimError, match="MSIM_ERR_ARG"):
        sim.flow_attach(bad)
    sim.flow_attach(flow)
    sim.policy_step(1, 1)
    sim.policy_attach(pol)   # re-attaching the sampler detaches the flow
    with pytest.raises(msim.MsimError, match="MSIM_ERR_STATE"):
        sim.flow_actions()

"""Pipelined host stepping (msim_step_host_async / msim_host_wait) against the synchronous
msim_step_host: the same excitations from pinned host memory give the same per-step q and q_d
bit for bit, whether each call writes its own output buffers or all share one (the last call's
result stays), and the device state agrees at the end."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2603_29332_b300 import modelgen as mg
from paper_2603_29332_b300 import msim

pytestmark = pytest.mark.gpu

DT = 1e-3


def _pair(model, E, seed):
    sims = [msim.Sim(model, E, dt=DT) for _ in range(2)]
    q0, qd0, a0 = mg.initial_state(model, E, seed=seed)
    for s in sims:
        s.reset(s.pad_n(q0), s.pad_n(qd0), s.pad_m(a0))
    return sims


def _pinned(sim, rows, cols):
    return torch.zeros((rows, cols), dtype=torch.float32).pin_memory()


@pytest.mark.parametrize("name", ["c1_whole", "c0_tiny"])
def test_pipelined_host_steps_equal_synchronous_ones(name):
    model = mg.config_model(name)
    E, K, sub = 515, 7, 3        # ragged: not a multiple of any block size
    ref, pip = _pair(model, E, seed=4)
    exc = mg.smooth_excitations(model, E, K, seed=4)
    ex_h = []
    for t in range(K):
        x = _pinned(ref, E, ref.pitch_m)
        x[:, : model.n_muscles] = torch.from_numpy(exc[t])
        ex_h.append(x)
    want_q, want_qd = [], []
    for t in range(K):
        q, qd = _pinned(ref, E, ref.pitch_n), _pinned(ref, E, ref.pitch_n)
        ref.step_host(ex_h[t], sub, q, qd)
        want_q.append(q.clone()); want_qd.append(qd.clone())
    got = [(_pinned(pip, E, pip.pitch_n), _pinned(pip, E, pip.pitch_n)) for _ in range(K)]
    for t in range(K):
        pip.step_host_async(ex_h[t], sub, got[t][0], got[t][1])
    pip.host_wait()
    for t in range(K):
        assert torch.equal(got[t][0], want_q[t]), t
        assert torch.equal(got[t][1], want_qd[t]), t
    # one shared output buffer: the last call's state remains; qd not read back
    shared = _pinned(pip, E, pip.pitch_n)
    for t in range(K):
        ref.step_host(ex_h[t], sub, None, None)
        pip.step_host_async(ex_h[t], sub, shared, None)
    pip.host_wait()
    torch.cuda.synchronize()
    sa, sb = ref.state(), pip.state()
    for k in ("q", "qd", "act", "force"):
        assert torch.equal(sa[k], sb[k]), k
    assert torch.equal(shared, sa["q"].cpu())
    assert ref.status() == (0, 0) and pip.status() == (0, 0)


def test_host_wait_before_any_call_and_argument_errors():
    model = mg.config_model("c0_tiny")
    sim = msim.Sim(model, 8, dt=DT)
    sim.host_wait()
    with pytest.raises(msim.MsimError):
        sim.step_host_async(None, 1)
    x = _pinned(sim, 8, sim.pitch_m)
    with pytest.raises(msim.MsimError):
        sim.step_host_async(x, 0)

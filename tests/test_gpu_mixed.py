"""One persistent launch for environments of different skeletons, and the launch-shape autotuner.

The mixed launch runs the same per-environment code as the per-model launches; with the same
warps per environment the results are bitwise equal (the reductions are fixed point, so the
number of environments per block and the work order cannot change them).
"""
import os
import tempfile

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2603_29332_b300 import modelgen as mg
from paper_2603_29332_b300 import msim

pytestmark = pytest.mark.gpu

DT = 5e-4
NAMES = ("c2_upper", "c2_lower", "c1_whole")


def _mixed_sim(counts, seed=0):
    models = [mg.config_model(n) for n in NAMES]
    sim = msim.Sim(models, list(counts), dt=DT)
    qs, qds, acts = [], [], []
    for i, (m, E) in enumerate(zip(models, counts)):
        q, qd, a = mg.initial_state(m, E, seed=seed + i)
        qs.append(sim._pad(q, sim.pitch_n)); qds.append(sim._pad(qd, sim.pitch_n)); acts.append(sim._pad(a, sim.pitch_m))
    sim.reset(torch.cat(qs), torch.cat(qds), torch.cat(acts))
    exc = torch.cat([sim._pad(mg.uniform_excitations(m, E, 1, seed=seed + 10 + i)[0], sim.pitch_m)
                     for i, (m, E) in enumerate(zip(models, counts))])
    return sim, models, exc


def _same_state(a, b, keys=("q", "qd", "act", "qdd", "force")):
    sa, sb = a.state(), b.state()
    for k in keys:
        assert torch.equal(sa[k], sb[k]), k
    assert torch.equal(sa["status"], sb["status"])


@pytest.mark.parametrize("wpe,slots", [(1, 6), (2, 4), (2, 7), (4, 3)])
def test_mixed_launch_equals_per_model_launches_bitwise(wpe, slots):
    counts = (37, 53, 61)   # ragged against every slot count
    a, _, exc = _mixed_sim(counts)
    b, _, _ = _mixed_sim(counts)
    for i in range(len(NAMES)):
        a.set_launch(i, warps_per_env=wpe)
        b.set_launch(i, warps_per_env=wpe)
    b.set_mixed_launch(True, warps_per_env=wpe, slots_per_block=slots)
    for _ in range(3):
        a.step(exc, 10)
        b.step(exc, 10)
    torch.cuda.synchronize()
    _same_state(a, b)
    assert a.status() == (0, 0) and b.status() == (0, 0)


def test_mixed_launch_in_a_cuda_graph():
    counts = (20, 20, 24)
    a, _, exc = _mixed_sim(counts, seed=3)
    b, _, _ = _mixed_sim(counts, seed=3)
    for s in (a, b):
        s.set_mixed_launch(True)
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        a.step(exc, 10)
    torch.cuda.synchronize()
    a2, _, _ = _mixed_sim(counts, seed=3)   # capture does not execute; replay onto a's fresh state
    st = a2.state()
    a.reset(st["q"], st["qd"], st["act"])
    torch.cuda.synchronize()
    for _ in range(4):
        g.replay()
        b.step(exc, 10)
    torch.cuda.synchronize()
    _same_state(a, b, keys=("q", "qd", "act"))


def test_mixed_launch_rejects_shapes_that_do_not_fit():
    sim, _, _ = _mixed_sim((4, 4, 4))
    with pytest.raises(msim.MsimError):
        sim.set_mixed_launch(True, warps_per_env=4, slots_per_block=5)   # 640 threads
    with pytest.raises(msim.MsimError):
        sim.set_mixed_launch(True, warps_per_env=1, slots_per_block=17)


def test_autotune_keeps_state_and_caches_its_choice():
    counts = (96, 96, 128)
    sim, models, exc = _mixed_sim(counts, seed=5)
    ref, _, _ = _mixed_sim(counts, seed=5)
    before = sim.state()
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "tune.txt")
        r = sim.autotune(path, n_sub=10)
        after = sim.state()
        for k in ("q", "qd", "act", "qdd", "force", "status"):
            assert torch.equal(before[k], after[k]), k
        assert r["candidates"] > 10 and r["from_cache"] == 0
        assert r["ms_per_model"] > 0 and r["ms_mixed"] > 0
        assert os.path.getsize(path) > 0
        print("\nautotune: per-model %.3f ms, mixed %.3f ms, mixed chosen %d (wpe %d, slots %d), per-model %s"
              % (r["ms_per_model"], r["ms_mixed"], r["mixed"], r["mixed_warps_per_env"], r["mixed_slots"],
                 list(zip(r["warps_per_env"][:3], r["envs_per_block"][:3], r["stage_points"][:3]))))
        # the tuned handle still computes the same dynamics (shapes change only summation
        # groupings of the lane-parallel solve: agreement to FP32 rounding)
        sim.step(exc, 10)
        ref.step(exc, 10)
        sa, sb = sim.state(), ref.state()
        np.testing.assert_allclose(sa["q"].cpu().numpy(), sb["q"].cpu().numpy(), rtol=1e-6, atol=1e-6)
        # a second handle with the same models and counts reads the cache without timing
        other, _, _ = _mixed_sim(counts, seed=6)
        r2 = other.autotune(path, n_sub=10)
        assert r2["from_cache"] == 1 and r2["mixed"] == r["mixed"]
        assert r2["envs_per_block"] == r["envs_per_block"]


def test_a_model_without_environments_is_skipped_by_both_launches():
    models = [mg.config_model(n) for n in NAMES]
    counts = [9, 0, 7]
    a = msim.Sim(models, counts, dt=DT)
    b = msim.Sim(models, counts, dt=DT)
    b.set_mixed_launch(True)
    qs, qds, acts, ex = [], [], [], []
    for i, (m, E) in enumerate(zip(models, counts)):
        if E == 0:
            continue
        q, qd, ac = mg.initial_state(m, E, seed=i)
        qs.append(a._pad(q, a.pitch_n)); qds.append(a._pad(qd, a.pitch_n)); acts.append(a._pad(ac, a.pitch_m))
        ex.append(a._pad(mg.uniform_excitations(m, E, 1, seed=i)[0], a.pitch_m))
    for s in (a, b):
        s.reset(torch.cat(qs), torch.cat(qds), torch.cat(acts))
        s.step(torch.cat(ex), 10)
    _same_state(a, b)


def test_autotune_ignores_a_damaged_cache_line():
    counts = (16, 16, 16)
    sim, _, _ = _mixed_sim(counts, seed=8)
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "tune.txt")
        r = sim.autotune(path, n_sub=2)
        line = open(path).read().split()
        with open(path, "w") as f:   # same key, truncated fields: must be re-timed, not applied
            f.write(" ".join(line[:6]) + "\n")
        other, _, _ = _mixed_sim(counts, seed=9)
        r2 = other.autotune(path, n_sub=2)
        assert r2["from_cache"] == 0 and r2["candidates"] > 0
        r3 = other.autotune(path, n_sub=2)
        assert r3["from_cache"] == 1

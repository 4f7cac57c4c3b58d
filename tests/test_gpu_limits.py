"""The build's size limits and degenerate models, through the C ABI, against the FP64 oracle.

A model at every limit at once (255 DoFs, DoF depth 62 of 63, 85 bodies, 4096 muscles of 8 via
points crossing 12 DoFs each, 32 contact spheres) runs one substep stage by stage and a short
trajectory against the oracle; a model without muscles or spheres runs too; the host rejects
each limit exceeded (n_dofs, n_bodies, depth, points, crossed DoFs, spheres, muscles).
"""
import copy

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as ora
from paper_2603_29332_b300 import modelgen as mg
from paper_2603_29332_b300 import msim
from tests.gpu_common import oracle_eval, qdd_rel_err

pytestmark = pytest.mark.gpu

DT = 1e-3


def max_model(seed=0, n_muscles=4096, limbs=(20, 20, 20, 20, 4), pts_per_muscle=8, span_bodies=4, fmax=(50, 500)):
    """Root ball joint plus five limbs of ball joints: 3 + 3 x 84 = 255 DoFs, depth <= 62; every
    muscle spans ``span_bodies`` ball joints of one limb (12 DoFs) through ``pts_per_muscle``
    points; 8 spheres at the tip of each of the four long limbs."""
    rng = np.random.default_rng(seed)
    parent, ndof, offset = [-1], [3], [[0, 0, 2.6]]   # limbs of 20 x 0.12 m hang above the ground
    chains = []
    for nbod in limbs:
        prev, ch = 0, []
        for _ in range(nbod):
            parent.append(prev)
            ndof.append(3)
            offset.append(rng.uniform(-0.05, 0.05, 3) + np.array([0, 0, -0.12]))
            prev = len(parent) - 1
            ch.append(prev)
        chains.append(ch)
    B, n = len(parent), 3 * len(parent)
    mass = rng.uniform(0.5, 2.0, B)
    com = np.tile([0, 0, -0.06], (B, 1)) + rng.uniform(-0.01, 0.01, (B, 3))
    inertia = np.tile([0.004, 0.004, 0.002, 0, 0, 0], (B, 1))
    axes = []
    for _ in range(B):
        Q = np.linalg.qr(rng.normal(size=(3, 3)))[0]
        axes += [Q[:, 0], Q[:, 1], Q[:, 2]]
    lim = np.stack([-rng.uniform(0.5, 2.0, n), rng.uniform(0.5, 2.0, n)], 1)
    lim[1::3] = [-0.8, 0.8]   # middle hinge of every ball joint away from gimbal lock
    long_chains = [c for c in chains if len(c) > span_bodies]
    muscles = []
    for k in range(n_muscles):
        ch = long_chains[k % len(long_chains)]
        i = int(rng.integers(0, len(ch) - span_bodies))
        span = [ch[i]] + ch[i + 1:i + 1 + span_bodies]
        pts = [(span[min(j * len(span) // pts_per_muscle, len(span) - 1)] if j < pts_per_muscle - 1 else span[-1],
                tuple(rng.uniform(-0.04, 0.04, 3) + np.array([0, 0, -0.06]))) for j in range(pts_per_muscle)]
        muscles.append(pts)
    spheres = [(chains[c][-1], tuple(rng.uniform(-0.03, 0.03, 3)), 0.02) for c in range(min(4, len(chains)))
               for _ in range(8)]
    return mg.make_model("limits", parent, ndof, offset, mass, com, inertia, axes, muscles,
                         rng.uniform(fmax[0], fmax[1], n_muscles), rng.uniform(0.05, 0.2, n_muscles),
                         dof_limit=lim, spheres=spheres)


def _states(model, E, seed):
    rng = np.random.default_rng(seed)
    q = rng.uniform(-0.3, 0.3, (E, model.n_dofs)).astype(np.float32)
    qd = rng.normal(0, 0.5, (E, model.n_dofs)).astype(np.float32)
    act = rng.uniform(0, 1, (E, model.n_muscles)).astype(np.float32)
    exc = rng.uniform(0, 1, (E, model.n_muscles)).astype(np.float32)
    return q, qd, act, exc


def test_model_at_every_limit_matches_the_oracle():
    model = max_model()
    assert model.n_dofs == 255 and model.n_muscles == 4096 and model.n_spheres == 32
    assert np.diff(model.muscle_point_start).max() == 8
    om = ora.OracleModel(model)
    E, n, m = 300, model.n_dofs, model.n_muscles
    sim = msim.Sim(model, E, dt=DT)
    d = sim.dims
    assert d.n_packed[0] > 8000 and d.envs_per_block[0] >= 1
    lay = sim.layout(0)
    q, qd, act, exc = _states(model, E, seed=2)
    res = sim.eval(sim.pad_n(q), sim.pad_n(qd), sim.pad_m(act), sim.pad_m(exc))
    g = {k: v.double().cpu().numpy() for k, v in res.items()}
    worst, ratio = 0.0, 0.0
    for e in (0, 151, E - 1):
        r = oracle_eval(om, DT, q[e], qd[e], act[e], exc[e])
        ev_ = np.linalg.eigvalsh(r["A"])
        kappa = ev_.max() / ev_.min()
        assert r["status"] == 0
        np.testing.assert_allclose(g["L"][e, :m], r["L"], rtol=0, atol=2e-5)
        Rg = msim.unpack_R(g["R"][e], lay, n)
        assert np.count_nonzero(Rg[0]) == 12
        np.testing.assert_allclose(Rg, r["R"], rtol=0, atol=2e-5)
        Mg = msim.unpack_packed(g["M"][e], lay)
        np.testing.assert_allclose(Mg, r["M"], rtol=0, atol=2e-6 * np.abs(r["M"]).max())
        err = qdd_rel_err(g["qdd"][e, :n], r["qdd"])
        worst = max(worst, err)
        ratio = max(ratio, err / kappa)
    print("\nlimits model: %d packed entries, %d envs/block, worst qdd rel err %.2e, err / cond(A) %.1e"
          % (d.n_packed[0], d.envs_per_block[0], worst, ratio))
    # the whole body's target holds although this model's chains of 62 light links make
    # cond(M + dt D) ~3e7 (the whole body's is ~1e5): the FP32 kinematics perturb the mechanism
    # consistently and the bias is float-float, unless penalty forces are extreme
    assert worst <= 1e-4
    assert ratio <= 2e-10


def test_model_at_every_limit_steps_like_the_oracle():
    model = max_model(fmax=(5, 50))   # weaker muscles: the error budget of q is absolute
    om = ora.OracleModel(model)
    E, steps = 64, 20
    sim = msim.Sim(model, E, dt=DT)
    q, qd, act, exc = _states(model, E, seed=4)
    qd[:] = 0.0
    sim.reset(sim.pad_n(q), sim.pad_n(qd), sim.pad_m(act))
    sim.step(sim.pad_m(exc), steps)
    st = sim.state()
    assert sim.status() == (0, 0)
    idx = [0, E - 1]
    qo, *_ = ora.step(om, DT, q[idx].astype(np.float64), qd[idx].astype(np.float64),
                      act[idx].astype(np.float64), exc[idx].astype(np.float64), steps)
    err = np.abs(st["q"][idx, :model.n_dofs].double().cpu().numpy() - qo).max()
    print("\nlimits model: max |q_gpu - q_oracle| after %d substeps %.2e" % (steps, err))
    assert err <= 1e-3


def test_model_without_muscles_or_spheres():
    base = mg.config_model("c0_tiny")
    model = mg.make_model("bare", base.body_parent, base.body_ndof, base.body_offset, base.body_mass,
                          base.body_com, base.body_inertia, base.dof_axis, dof_limit=base.dof_limit)
    assert model.n_muscles == 0 and model.n_spheres == 0
    om = ora.OracleModel(model)
    E = 40
    sim = msim.Sim(model, E, dt=DT)
    rng = np.random.default_rng(5)
    q = rng.uniform(-0.5, 0.5, (E, model.n_dofs)).astype(np.float32)
    qd = rng.normal(0, 1.0, (E, model.n_dofs)).astype(np.float32)
    z = np.zeros((E, 0), np.float32)
    sim.reset(sim.pad_n(q), sim.pad_n(qd), sim.pad_m(z))
    sim.step(sim.pad_m(z), 50)
    qg = sim.state()["q"][:, :model.n_dofs].double().cpu().numpy()
    qo, *_ = ora.step(om, DT, q.astype(np.float64), qd.astype(np.float64), np.zeros((E, 0)), np.zeros((E, 0)), 50)
    assert np.abs(qg - qo).max() <= 1e-3
    assert sim.status() == (0, 0)


@pytest.mark.parametrize("kind,msg", [
    ("dofs", "n_dofs"), ("depth", "depth"), ("points", "points"), ("crossed", "crosses"),
    ("spheres", "n_spheres"), ("muscles", "n_muscles"),
])
def test_limits_exceeded_are_rejected(kind, msg):
    if kind == "dofs":        # 256 DoFs: one more hinge on the short limb's tip
        model = max_model(n_muscles=8, limbs=(20, 20, 20, 20, 4))
        model = mg.make_model("x", np.r_[model.body_parent, model.n_bodies - 1], np.r_[model.body_ndof, 1],
                              np.vstack([model.body_offset, [0, 0, -0.1]]), np.r_[model.body_mass, 1.0],
                              np.vstack([model.body_com, [0, 0, 0]]), np.vstack([model.body_inertia, model.body_inertia[:1]]),
                              np.vstack([model.dof_axis, [[0, 0, 1]]]))
    elif kind == "depth":     # depth 64: a limb of 21 ball joints below the root's three hinges
        model = max_model(n_muscles=8, limbs=(21, 4))
    elif kind == "points":
        model = max_model(n_muscles=8, limbs=(20, 4), pts_per_muscle=9)
    elif kind == "crossed":   # 15 crossed DoFs
        model = max_model(n_muscles=8, limbs=(20, 20, 20, 20, 4), span_bodies=5)
    elif kind == "spheres":
        model = copy.deepcopy(max_model(n_muscles=8))
        model.sphere_body = np.r_[model.sphere_body, model.sphere_body[:1]]
        model.sphere_pos = np.vstack([model.sphere_pos, model.sphere_pos[:1]])
        model.sphere_radius = np.r_[model.sphere_radius, model.sphere_radius[:1]]
    else:
        model = max_model(n_muscles=4097)
    with pytest.raises(msim.MsimError, match=msg):
        msim.Sim(model, 4, dt=DT)

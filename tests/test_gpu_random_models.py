"""Randomly drawn models through the C ABI against the FP64 oracle.

Sixteen seeded draws of the synthetic generator over its whole parameter space (2-30 bodies,
1-3 DoFs per body, 1-200 muscles of 2-8 path points spanning 1-3 joints, limits and foot contact
on or off, cylinders and spheres, fixed or free root, compliant tendons on about 40 % of the
draws) each run one substep stage by stage and
30 substeps against the oracle.  The fixed configurations of the other tests are single points
of this space; here tree shapes, depths, muscle lengths and feature combinations vary.  A free
root starts within 2 cm of its model pose; q_dd within 1e-4, q within 1e-3 after 30 substeps.
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


def draw(i):
    r = np.random.default_rng(1000 + i)
    nb = int(r.integers(2, 31))
    maxd = int(r.integers(1, 4))
    return dict(n_bodies=nb, n_dofs=int(r.integers(nb, maxd * nb + 1)), n_muscles=int(r.integers(1, 201)),
                max_points=int(r.integers(2, 9)), max_span=int(r.integers(1, 4)), limits=bool(r.uniform() < 0.6),
                contact=bool(r.uniform() < 0.5) and nb >= 6, seed=int(r.integers(0, 1 << 30)), max_dof_per_body=maxd,
                wrap_frac=float(r.choice([0.0, 0.3])), sphere_frac=float(r.choice([0.0, 0.5])),
                free_root=bool(r.uniform() < 0.3))


@pytest.mark.parametrize("i", range(16))
def test_random_model_matches_the_oracle(i):
    model = mg.generate("random%d" % i, **draw(i))
    if np.random.default_rng(5000 + i).uniform() < 0.4:   # compliant tendons on half the eligible muscles
        model = mg.with_tendons(model, ora.OracleModel(model).L0, frac=0.5, seed=i)
    om = ora.OracleModel(model)
    n, m = model.n_dofs, model.n_muscles
    E = 48
    sim = msim.Sim(model, E, dt=DT)
    lay = sim.layout(0)
    q, qd, act, exc = random_states(model, E, seed=i, q_scale=0.4)
    if model.free_root:
        q[:, :3] *= 0.05   # the root within 2 cm of its model pose, not tens of cm into the ground
    eps = (np.random.default_rng(i).uniform(-0.3, 1.6, (E, m)) * model.muscle_tendon_strain).astype(np.float32)
    res = sim.eval(sim.pad_n(q), sim.pad_n(qd), sim.pad_m(act), sim.pad_m(exc), eps=sim.pad_m(eps))
    g = {k: v.double().cpu().numpy() for k, v in res.items()}
    worst = 0.0
    for e in sample_envs(E, 6, seed=i):
        r = oracle_eval(om, DT, q[e], qd[e], act[e], exc[e], eps[e])
        assert r["status"] == 0
        np.testing.assert_allclose(g["L"][e, :m], r["L"], rtol=0, atol=2e-6)
        np.testing.assert_allclose(msim.unpack_R(g["R"][e], lay, n), r["R"], rtol=0, atol=2e-6)
        np.testing.assert_allclose(msim.unpack_packed(g["M"][e], lay), r["M"], rtol=0, atol=2e-6 * np.abs(r["M"]).max())
        worst = max(worst, qdd_rel_err(g["qdd"][e, :n], r["qdd"]))
    assert worst <= 1e-4, worst
    # 30 substeps from the generator's initial state under uniform excitations
    q0, qd0, a0 = mg.initial_state(model, E, seed=i)
    u = mg.uniform_excitations(model, E, 1, seed=i)[0]
    sim.reset(sim.pad_n(q0), sim.pad_n(qd0), sim.pad_m(a0))
    sim.step(sim.pad_m(u), 30)
    qg = sim.state()["q"][:, :n].double().cpu().numpy()
    idx = sample_envs(E, 4, seed=i + 1)
    qo, *_ = ora.step(om, DT, q0[idx].astype(np.float64), qd0[idx].astype(np.float64), a0[idx].astype(np.float64),
                      u[idx].astype(np.float64), 30)
    err = np.abs(qg[idx] - qo).max()
    print("\nrandom model %d: n %d, bodies %d, muscles %d, wraps %d, free root %d, spheres %d, tendons %d: "
          "qdd %.1e, q %.1e" % (i, n, model.n_bodies, m, len(model.wrap_muscle), model.free_root, model.n_spheres,
                                int((model.muscle_tendon_strain > 0).sum()), worst, err))
    assert err <= 1e-3
    assert sim.status() == (0, 0)

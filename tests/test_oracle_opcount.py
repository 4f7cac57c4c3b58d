"""The roofline's FLOP numerator (paper_2603_29332_b300/flops.py) against an instrumented count.

oracle/opcount.py runs the method's algorithms for one substep of one environment on numbers
that count their arithmetic.  First its values are pinned to the FP64 oracle's independent
formulations (lengths and moment arms, M, the Newton-Euler bias, forces, the system matrix, the
right-hand side, q_dd, the activation update), so the count is of algorithms that compute the
method; then the formula's stages must equal the count: exactly for every structural stage, and
within the range of the Hill curves' branches for the one stage whose work depends on the state.
"""
import numpy as np
import pytest

from oracle import opcount as oc
from oracle import oracle as ora
from paper_2603_29332_b300 import flops as FL
from paper_2603_29332_b300 import modelgen as mg

DT = 1e-3


def _models():
    out = []
    for name in ("c0_tiny", "c1_whole", "c2_upper", "c2_lower"):
        out.append(mg.config_model(name))
    out.append(mg.generate("rand", n_bodies=14, n_dofs=25, n_muscles=60, max_points=8, max_span=3, limits=True,
                           contact=True, seed=77))
    for mdl in out:   # lift the root: no sphere in contact (the contact force work is not counted)
        mdl.body_offset = mdl.body_offset.copy()
        mdl.body_offset[0, 2] += 1.0
    return out


@pytest.fixture(scope="module", params=range(5), ids=["c0_tiny", "c1_whole", "c2_upper", "c2_lower", "random"])
def counted(request):
    model = _models()[request.param]
    om = ora.OracleModel(model)
    rng = np.random.default_rng(11 + request.param)
    lo, hi = model.dof_limit[:, 0], model.dof_limit[:, 1]
    q = rng.uniform(-0.3, 0.3, model.n_dofs)
    on = lo < hi
    q[on] = np.clip(q[on], lo[on], hi[on])
    qd = rng.normal(0, 1.0, model.n_dofs)
    act, exc = rng.uniform(0, 1, model.n_muscles), rng.uniform(0, 1, model.n_muscles)
    counts, values = oc.count_substep(model, DT, q, qd, act, exc, om.L0)
    ref = ora.evaluate(om, DT, q, qd, act, exc)
    return model, counts, values, ref


def test_counted_algorithms_compute_the_method(counted):
    model, counts, v, r = counted
    assert r["status"] == 0
    for k in ("L", "R", "M", "A", "bias", "force", "tau_m", "rhs", "act_next"):
        scale = max(np.abs(r[k]).max(), 1.0)
        np.testing.assert_allclose(v[k], r[k], rtol=0, atol=1e-11 * scale, err_msg=k)
    # q_dd through the tree-sparse factorisation against the oracle's dense Cholesky
    np.testing.assert_allclose(v["qdd"], r["qdd"], rtol=0, atol=1e-9 * max(np.abs(r["qdd"]).max(), 1.0))


def test_formula_equals_the_count(counted):
    model, counts, _, _ = counted
    f = FL.flops_per_env_substep(model)
    assert set(counts) == set(f), (set(counts) ^ set(f))
    for stage in counts:
        if stage in ("hill_activation", "total"):
            continue
        assert f[stage] == counts[stage], (stage, f[stage], counts[stage])
    # branches of the Hill curves: f_p 0 or 3 or 5 operations, f_v and its slope fewer below v = -1
    m = model.n_muscles
    assert m * (FL.HILL_PER_MUSCLE - 8) <= counts["hill_activation"] <= m * (FL.HILL_PER_MUSCLE + 5)
    assert abs(f["total"] - counts["total"]) <= 8 * m

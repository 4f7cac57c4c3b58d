"""Shared helpers of the GPU parity tests: seeded states, oracle evaluation of sampled envs."""
import numpy as np

from oracle import oracle as ora


def random_states(model, E, seed, q_scale=0.4, qd_scale=1.0):
    """FP32 states (q, qd, act, exc) of E environments, seeded."""
    rng = np.random.default_rng(seed)
    n, m = model.n_dofs, model.n_muscles
    q = rng.uniform(-q_scale, q_scale, (E, n)).astype(np.float32)
    qd = rng.normal(0.0, qd_scale, (E, n)).astype(np.float32)
    act = rng.uniform(0.0, 1.0, (E, m)).astype(np.float32)
    exc = rng.uniform(0.0, 1.0, (E, m)).astype(np.float32)
    return q, qd, act, exc


def sample_envs(E, k, seed=0):
    """k env indices spread over [0, E): first, last and random ones in between."""
    if E <= k:
        return np.arange(E)
    rng = np.random.default_rng(seed)
    mid = rng.choice(np.arange(1, E - 1), size=k - 2, replace=False)
    return np.sort(np.concatenate([[0, E - 1], mid]))


def oracle_eval(om, dt, q, qd, act, exc, eps=None):
    return ora.evaluate(om, dt, q.astype(np.float64), qd.astype(np.float64), act.astype(np.float64),
                        exc.astype(np.float64), None if eps is None else eps.astype(np.float64))


def qdd_rel_err(qdd_gpu, qdd_ref):
    """Norm-wise relative error of one env's accelerations, floor 1e-3 on the reference norm."""
    return float(np.linalg.norm(qdd_gpu - qdd_ref) / max(np.linalg.norm(qdd_ref), 1e-3))

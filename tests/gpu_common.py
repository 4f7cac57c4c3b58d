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



# Bound constant of the MLP comparisons: |device - oracle| <= MLP_BOUND_C u sum|a| |b| over the
# last contraction of each output or gradient (u = 2^-8, the BF16 unit roundoff).  An emulation of the
# device's sequence of BF16 roundings stays below 0.65 u sum|a||b| on the configured shapes
# (tests/test_mlp_bound_model.py), so 4 leaves a margin of six.
MLP_BOUND_C = 4.0
MLP_U = 2.0 ** -8


def mlp_bf16_reference(params, x, out_sigmoid=False, C=MLP_BOUND_C):
    """FP64 MLP oracle output at BF16-valued weights and inputs, with a per-element bound on the
    device's deviation: C u sum_j |h2_j| |W3_ij| (+ |b3_i|), times max sigmoid' = 1/4 for a sigmoid
    output.  The device rounds the hidden activations to BF16 and accumulates in FP32.  Returns
    (y, bound)."""
    from oracle import mlp_oracle as mo
    y, (_, z1, h1, z2, h2) = mo.forward(params, x, out_sigmoid)
    W1, b1, W2, b2, W3, b3 = params
    bound = C * MLP_U * (np.abs(h2) @ np.abs(W3).T + np.abs(b3))
    return y, (0.25 * bound if out_sigmoid else bound)


def mlp_bf16_backward_reference(params, x, t, out_sigmoid=False, C=MLP_BOUND_C):
    """FP64 oracle gradients of the mean-squared loss at BF16-valued weights and inputs, with
    per-element bounds C u sum_b |a_b| |c_b| over each gradient's batch contraction (dW3: dy and
    h2, dW2: dz2 and h1, dW1: dz1 and x; the bias gradients: sum_b |dz_b|).  The device rounds the
    activations, the stored pre-activations, the output gradient and the hidden gradients to BF16
    and accumulates in FP32.  Returns (grads, bounds, loss), both ordered (dW1, db1, dW2, db2,
    dW3, db3)."""
    from oracle import mlp_oracle as mo
    W1, b1, W2, b2, W3, b3 = params
    grads, loss = mo.backward(params, x, t, out_sigmoid)
    y, (_, z1, h1, z2, h2) = mo.forward(params, x, out_sigmoid)
    B, N = y.shape
    dy = 2.0 * (y - t) / (B * N)
    if out_sigmoid:
        dy = dy * y * (1.0 - y)
    dz2 = (dy @ W3) * mo.dsilu(z2)
    dz1 = (dz2 @ W2) * mo.dsilu(z1)
    a = [np.abs(v) for v in (dy, dz2, dz1, h2, h1, x)]
    k = C * MLP_U
    bounds = (k * (a[2].T @ a[5]), k * a[2].sum(0), k * (a[1].T @ a[4]), k * a[1].sum(0), k * (a[0].T @ a[3]),
              k * a[0].sum(0))
    return grads, bounds, loss

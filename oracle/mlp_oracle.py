"""FP64 reference of the 3-layer MLP used by the geometry surrogate and the policy network.

TEST INFRASTRUCTURE ONLY (like the rest of oracle/): the tests, the smoke check and the
benchmark's CPU baseline may call it; the product never does.  Shares no code with the CUDA path.

The paper gives all its networks as 3-layer MLPs (Methods, "Training hyperparameters"); the
surrogate's and the policy's sizes come from their workloads.  Definitions written out plainly:

    z1 = x W1^T + b1,  h1 = silu(z1)          silu(z) = z sigmoid(z)
    z2 = h1 W2^T + b2, h2 = silu(z2)
    y  = out(h2 W3^T + b3)                     out = identity or sigmoid
    loss = mean over batch and outputs of (y - t)^2

Backward by the chain rule; Adam as in Kingma & Ba (2015): m <- b1 m + (1 - b1) g,
v <- b2 v + (1 - b2) g^2, theta <- theta - lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
"""
import numpy as np


def sigmoid(z):
    return 1.0 / (1.0 + np.exp(-z))


def silu(z):
    return z * sigmoid(z)


def dsilu(z):
    s = sigmoid(z)
    return s * (1.0 + z * (1.0 - s))


def forward(params, x, out_sigmoid=False):
    W1, b1, W2, b2, W3, b3 = params
    z1 = x @ W1.T + b1
    h1 = silu(z1)
    z2 = h1 @ W2.T + b2
    h2 = silu(z2)
    y = h2 @ W3.T + b3
    if out_sigmoid:
        y = sigmoid(y)
    return y, (x, z1, h1, z2, h2)


def loss(params, x, t, out_sigmoid=False):
    y, _ = forward(params, x, out_sigmoid)
    return float(np.mean((y - t) ** 2))


def backward(params, x, t, out_sigmoid=False):
    """Gradients of the mean-squared loss w.r.t. (W1, b1, W2, b2, W3, b3), and the loss."""
    W1, b1, W2, b2, W3, b3 = params
    y, (x, z1, h1, z2, h2) = forward(params, x, out_sigmoid)
    B, N = y.shape
    dy = 2.0 * (y - t) / (B * N)
    if out_sigmoid:
        dy = dy * y * (1.0 - y)
    dW3 = dy.T @ h2
    db3 = dy.sum(axis=0)
    dz2 = (dy @ W3) * dsilu(z2)
    dW2 = dz2.T @ h1
    db2 = dz2.sum(axis=0)
    dz1 = (dz2 @ W2) * dsilu(z1)
    dW1 = dz1.T @ x
    db1 = dz1.sum(axis=0)
    return (dW1, db1, dW2, db2, dW3, db3), float(np.mean((y - t) ** 2))


def adam_step(params, grads, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (t = 1 for the first step).  Returns new (params, m, v)."""
    out_p, out_m, out_v = [], [], []
    for p, g, mi, vi in zip(params, grads, m, v):
        mi = beta1 * mi + (1.0 - beta1) * g
        vi = beta2 * vi + (1.0 - beta2) * g * g
        mh = mi / (1.0 - beta1 ** t)
        vh = vi / (1.0 - beta2 ** t)
        out_p.append(p - lr * mh / (np.sqrt(vh) + eps))
        out_m.append(mi)
        out_v.append(vi)
    return out_p, out_m, out_v


def flow_refine(a0, velocity, n_steps, dt):
    """Action refinement by the flow ODE da/dt = psi(t, s, a) from t = 0 (Methods, "Reinforcement
    learning with flow-based exploration"), integrated with n_steps explicit Euler steps of size
    dt ("Training hyperparameters": 20 steps of 0.05): a_{k+1} = a_k + dt psi(k dt, a_k).
    `velocity(t, a)` returns psi for the whole batch (the observation is bound inside it)."""
    a = np.array(a0, dtype=np.float64)
    for k in range(n_steps):
        a = a + dt * velocity(k * dt, a)
    return a


def mlp_velocity(params, obs, in_round=None):
    """psi(t, s, a) of a 3-layer MLP reading [obs | a | t]; `in_round` (optional) rounds the
    network input as the device stores it."""
    def v(t, a):
        x = np.concatenate([obs, a, np.full((a.shape[0], 1), t)], axis=1)
        if in_round is not None:
            x = in_round(x)
        y, _ = forward(params, x)
        return y
    return v

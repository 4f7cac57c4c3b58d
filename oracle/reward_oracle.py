"""FP64 reference of the imitation reward (tracking error, discriminator reward, power penalty).

TEST INFRASTRUCTURE ONLY (like the rest of oracle/): the tests may call it; the product never
does.  Shares no code with the CUDA path.

Methods, "Unified imitation environment": the tracking error Delta collects the differences of
joint angles and body positions between the simulated and the reference motion; a discriminator
D maps it to the reward r = -log(1 - D(Delta)).  "Training regularization" adds the power
penalty r_power = -(1/|A|) sum_i |F_m^(i) v_m^(i)| with weight w_power.  Body positions are the
body-frame origins in the world frame, from this oracle's own forward kinematics.
"""
import numpy as np

from oracle import mlp_oracle as mo
from oracle import oracle as ora


def body_positions(model, q):
    """World positions of the body origins, [n_bodies, 3]."""
    _, pb, _, _ = ora.fk(model, q)
    return pb


def tracking_error(model, q, q_ref):
    """Delta = [q - q_ref | x_b(q) - x_b(q_ref)] (bodies in model order, x, y, z each)."""
    q = np.asarray(q, np.float64)
    q_ref = np.asarray(q_ref, np.float64)
    return np.concatenate([q - q_ref, (body_positions(model, q) - body_positions(model, q_ref)).ravel()])


def reward_tracking(d):
    """r = -log(1 - D)."""
    return -np.log(1.0 - np.asarray(d, np.float64))


def reward_power(force, vm):
    """r_power = -(1/|A|) sum_i |F_i v_i|."""
    return -np.mean(np.abs(np.asarray(force, np.float64) * np.asarray(vm, np.float64)))


def reward(model, disc_params, q, q_ref, force, vm, w_power, in_round=None):
    """r = r_tracking + w_power r_power for one environment; `in_round` (optional) rounds the
    discriminator input as the device stores it."""
    x = tracking_error(model, q, q_ref)[None, :]
    if in_round is not None:
        x = in_round(x)
    d, _ = mo.forward(disc_params, x, out_sigmoid=True)
    return float(reward_tracking(d[0, 0]) + w_power * reward_power(force, vm))

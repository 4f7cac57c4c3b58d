"""The error bound the MLP parity tests use, checked against an emulation of the device's roundings.

The tensor-core MLP stores its hidden activations, the pre-activations its backward reads, the
output gradient and the hidden gradients in BF16 (round to nearest even) and accumulates in FP32.
This test replays that sequence of roundings in numpy (FP64 arithmetic, BF16 rounding written
out from the format: keep the top 16 bits of the FP32 word after adding 0x7fff plus the lowest
kept bit) and checks that the result stays within the bound of tests/gpu_common.py, C u
sum|a||b| over each output's or gradient's last contraction, with room to spare (half of it) on
the configured shapes: the learned geometry network (90 -> 512 -> 512 -> 2448) and the policy
(2182 -> 1024 -> 1024 -> 700, sigmoid), at reduced batch.
"""
import numpy as np
import pytest

from oracle import mlp_oracle as mo
from tests.gpu_common import mlp_bf16_backward_reference, mlp_bf16_reference


def bf16_round(a):
    w = np.asarray(a, np.float32).view(np.uint32).astype(np.uint64)
    r = ((w + 0x7fff + ((w >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def test_bf16_rounding_emulation():
    # exact values, halfway cases to even, and the unit roundoff 2^-8 (8 significant bits)
    assert bf16_round(1.0) == 1.0 and bf16_round(-3.0) == -3.0
    assert bf16_round(1.0 + 2.0 ** -8) == 1.0                      # halfway, to even (down)
    assert bf16_round(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6       # halfway, to even (up)
    x = np.random.default_rng(0).normal(size=10000)
    assert np.all(np.abs(bf16_round(x) - x) <= 2.0 ** -8 * np.abs(x) * (1 + 1e-6))


@pytest.mark.parametrize("shape", [(93, 136, 203, 333, False), (90, 512, 2448, 512, False),
                                   (2182, 1024, 700, 128, True)])
def test_bound_covers_the_device_rounding_sequence(shape):
    d_in, hid, d_out, B, sig = shape
    rng = np.random.default_rng(d_in)
    p = [bf16_round(rng.uniform(-1, 1, (hid, d_in)) * np.sqrt(6 / d_in)), rng.normal(0, .1, hid),
         bf16_round(rng.uniform(-1, 1, (hid, hid)) * np.sqrt(6 / hid)), rng.normal(0, .1, hid),
         bf16_round(rng.uniform(-1, 1, (d_out, hid)) * np.sqrt(6 / hid)), rng.normal(0, .1, d_out)]
    x = bf16_round(rng.uniform(-1, 1, (B, d_in)))
    t = rng.uniform(0, 1, (B, d_out)) if sig else rng.normal(0, 1, (B, d_out))
    W1, b1, W2, b2, W3, b3 = p
    # the device's sequence
    z1 = x @ W1.T + b1
    H1, Z1 = bf16_round(mo.silu(z1)), bf16_round(z1)
    z2 = H1 @ W2.T + b2
    H2, Z2 = bf16_round(mo.silu(z2)), bf16_round(z2)
    y = H2 @ W3.T + b3
    if sig:
        y = mo.sigmoid(y)
    dY = 2 * (y - t) / (B * d_out)
    dY = bf16_round(dY * y * (1 - y) if sig else dY)
    dZ2 = bf16_round((dY @ W3) * mo.dsilu(Z2))
    dZ1 = bf16_round((dZ2 @ W2) * mo.dsilu(Z1))
    dev = (dZ1.T @ x, dZ1.sum(0), dZ2.T @ H1, dZ2.sum(0), dY.T @ H2, dY.sum(0))
    yr, yb = mlp_bf16_reference(p, x, sig)
    assert np.all(np.abs(y - yr) <= 0.5 * yb)
    g, bounds, _ = mlp_bf16_backward_reference(p, x, t, sig)
    for name, a, b, e in zip(("dW1", "db1", "dW2", "db2", "dW3", "db3"), dev, g, bounds):
        assert np.all(np.abs(a - b) <= 0.5 * e), name

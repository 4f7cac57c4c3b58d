"""The tensor-core MLP (forward, backward, Adam) against the FP64 MLP oracle, through the C ABI.

Inputs, weights and targets are seeded numpy draws (rounded to BF16 where the GPU stores BF16);
the oracle sees the same values.  Tolerances: the GPU keeps activations and the output gradient
in BF16 (8-bit mantissa), so gradients agree to ~1e-2 relative; FP32 parts (Adam) to 1e-5.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import mlp_oracle as mo
from paper_2603_29332_b300 import msim

pytestmark = pytest.mark.gpu


def bf16(a):
    return torch.as_tensor(np.asarray(a, np.float32)).bfloat16().float().numpy().astype(np.float64)


def _setup(d_in=90, hid=128, d_out=200, B=256, seed=0, out_sigmoid=False):
    rng = np.random.default_rng(seed)
    net = msim.MLP(d_in, hid, d_out, out_sigmoid=out_sigmoid, max_batch=B)
    p = [bf16(rng.uniform(-1, 1, (hid, d_in)) * np.sqrt(6 / d_in)), rng.normal(0, 0.1, hid),
         bf16(rng.uniform(-1, 1, (hid, hid)) * np.sqrt(6 / hid)), rng.normal(0, 0.1, hid),
         bf16(rng.uniform(-1, 1, (d_out, hid)) * np.sqrt(6 / hid)), rng.normal(0, 0.1, d_out)]
    p = [np.asarray(a, np.float32).astype(np.float64) for a in p]
    net.set(net.flatten(p))
    x = bf16(rng.uniform(-1, 1, (B, d_in)))
    t = rng.normal(0, 1, (B, d_out)) if not out_sigmoid else rng.uniform(0, 1, (B, d_out))
    t = np.asarray(t, np.float32).astype(np.float64)
    return net, p, x, t


@pytest.mark.parametrize("out_sigmoid", [False, True])
def test_forward_matches_oracle(out_sigmoid):
    net, p, x, t = _setup(out_sigmoid=out_sigmoid)
    Y = net.forward(net.pad_input(x))[:, : net.d_out].double().cpu().numpy()
    ref, _ = mo.forward(p, x, out_sigmoid)
    assert np.abs(Y - ref).max() <= 2e-2 * np.abs(ref).max()


@pytest.mark.parametrize("out_sigmoid", [False, True])
def test_gradients_match_oracle(out_sigmoid):
    net, p, x, t = _setup(seed=1, out_sigmoid=out_sigmoid)
    Tt = torch.as_tensor(t, dtype=torch.float32).cuda()
    loss = net.backward(net.pad_input(x), Tt)
    g = net.unflatten(net.get(1))
    gref, lref = mo.backward(p, x, t, out_sigmoid)
    assert loss == pytest.approx(lref, rel=2e-2)
    for name, a, b in zip(("dW1", "db1", "dW2", "db2", "dW3", "db3"), g, gref):
        err = np.abs(np.asarray(a, np.float64) - b).max() / np.abs(b).max()
        assert err < 3e-2, (name, err)


def test_adam_step_matches_formula():
    net, p, x, t = _setup(seed=2)
    rng = np.random.default_rng(3)
    flat_p = net.flatten(p)
    grads = [rng.normal(0, 1, a.shape) for a in p]
    m0 = [rng.normal(0, 0.1, a.shape) for a in p]
    v0 = [rng.uniform(0, 0.1, a.shape) for a in p]
    net.set(net.flatten(grads), which=1)
    net.set(net.flatten(m0), which=2, adam_step=4)
    net.set(net.flatten(v0), which=3, adam_step=4)
    net.adam(1e-3)
    got = net.unflatten(net.get(0))
    ref, _, _ = mo.adam_step([np.asarray(a, np.float32).astype(np.float64) for a in net.unflatten(flat_p)], grads,
                             m0, v0, 5, 1e-3)
    for a, b in zip(got, ref):
        np.testing.assert_allclose(np.asarray(a, np.float64), b, rtol=1e-5, atol=1e-7)


def test_training_with_the_gpu_kernels_reduces_loss():
    rng = np.random.default_rng(4)
    d_in, d_out, B = 16, 24, 512
    net = msim.MLP(d_in, 64, d_out, max_batch=B, seed=7)
    x = rng.uniform(-1, 1, (B, d_in))
    Wt = rng.normal(0, 1, (d_out, d_in))
    t = np.sin(x @ Wt.T)
    X = net.pad_input(x)
    T = torch.as_tensor(t, dtype=torch.float32).cuda()
    l0 = net.backward(X, T)
    for _ in range(800):
        net.backward(X, T)
        net.adam(3e-3)
    assert net.backward(X, T) < 0.3 * l0

"""The tensor-core MLP (forward, backward, Adam) against the FP64 MLP oracle, through the C ABI.

Inputs, weights and targets are seeded numpy draws (rounded to BF16 where the GPU stores BF16);
the oracle sees the same values.  The GPU keeps activations and gradients in BF16 and accumulates
in FP32, so every output and gradient element is compared with a bound of its own, propagated
from those roundings through the layers with absolute values (tests/gpu_common.py), rather than
with one tolerance relative to the largest element.  Sizes: a small network with ragged widths,
the configured learned geometry (90 -> 512 -> 512 -> 2448, batch 4096, forward and gradients)
and the configured policy (2182 -> 1024 -> 1024 -> 700, sigmoid, 16384 rows, sampled rows).
Adam (FP32) matches its formula to 1e-5.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import mlp_oracle as mo
from paper_2603_29332_b300 import msim
from tests.gpu_common import mlp_bf16_backward_reference, mlp_bf16_reference

pytestmark = pytest.mark.gpu


def bf16(a):
    return torch.as_tensor(np.asarray(a, np.float32)).bfloat16().float().numpy().astype(np.float64)


def _setup(d_in=90, hid=128, d_out=200, B=256, seed=0, out_sigmoid=False, t_scale=1.0):
    rng = np.random.default_rng(seed)
    net = msim.MLP(d_in, hid, d_out, out_sigmoid=out_sigmoid, max_batch=B)
    p = [bf16(rng.uniform(-1, 1, (hid, d_in)) * np.sqrt(6 / d_in)), rng.normal(0, 0.1, hid),
         bf16(rng.uniform(-1, 1, (hid, hid)) * np.sqrt(6 / hid)), rng.normal(0, 0.1, hid),
         bf16(rng.uniform(-1, 1, (d_out, hid)) * np.sqrt(6 / hid)), rng.normal(0, 0.1, d_out)]
    p = [np.asarray(a, np.float32).astype(np.float64) for a in p]
    net.set(net.flatten(p))
    x = bf16(rng.uniform(-1, 1, (B, d_in)))
    t = rng.normal(0, t_scale, (B, d_out)) if not out_sigmoid else rng.uniform(0, 1, (B, d_out))
    t = np.asarray(t, np.float32).astype(np.float64)
    return net, p, x, t


def _check_forward(net, p, x, out_sigmoid, rows=None):
    Y = net.forward(net.pad_input(x))[:, : net.d_out]
    rows = np.arange(x.shape[0]) if rows is None else rows
    got = Y[torch.as_tensor(rows).cuda()].double().cpu().numpy()
    ref, bound = mlp_bf16_reference(p, x[rows], out_sigmoid)
    excess = np.abs(got - ref) - bound
    assert excess.max() <= 1e-7, "forward: %.3e above its bound" % excess.max()
    return np.abs(got - ref).max(), bound.max()


def _check_backward(net, p, x, t, out_sigmoid):
    Tt = torch.as_tensor(t, dtype=torch.float32).cuda()
    loss = net.backward(net.pad_input(x), Tt)
    g = net.unflatten(net.get(1))
    gref, bounds, lref = mlp_bf16_backward_reference(p, x, t, out_sigmoid)
    assert loss == pytest.approx(lref, rel=1e-2)
    for name, a, b, e in zip(("dW1", "db1", "dW2", "db2", "dW3", "db3"), g, gref, bounds):
        d = np.abs(np.asarray(a, np.float64) - b)
        tiny = 1e-6 * np.abs(b).max()   # FP32 storage of the gradient itself
        over = d - (e + tiny)
        assert over.max() <= 0.0, (name, float(over.max()), float(e.max()))


@pytest.mark.parametrize("out_sigmoid", [False, True])
def test_forward_matches_oracle(out_sigmoid):
    net, p, x, t = _setup(d_in=93, hid=136, d_out=203, B=333, out_sigmoid=out_sigmoid)
    _check_forward(net, p, x, out_sigmoid)


@pytest.mark.parametrize("out_sigmoid", [False, True])
def test_gradients_match_oracle(out_sigmoid):
    net, p, x, t = _setup(d_in=93, hid=136, d_out=203, B=333, seed=1, out_sigmoid=out_sigmoid)
    _check_backward(net, p, x, t, out_sigmoid)


def test_learned_geometry_network_at_its_configured_size():
    """90 -> 512 -> 512 -> 2448 (the whole body's 700 lengths and 1748 moment arms), batch 4096:
    forward on every row and all six gradients of one training step."""
    net, p, x, t = _setup(d_in=90, hid=512, d_out=2448, B=4096, seed=5)
    err, bnd = _check_forward(net, p, x, False)
    print("\nsurrogate forward: max |gpu - oracle| %.2e, largest bound %.2e" % (err, bnd))
    _check_backward(net, p, x, t, False)


def test_policy_network_at_its_configured_size():
    """2182 -> 1024 -> 1024 -> 700 with sigmoid outputs over 16384 rows (sampled rows checked)."""
    net, p, x, t = _setup(d_in=2182, hid=1024, d_out=700, B=16384, seed=6, out_sigmoid=True)
    rows = np.concatenate([[0, 16383], np.random.default_rng(2).choice(np.arange(1, 16383), 254, replace=False)])
    err, bnd = _check_forward(net, p, x, True, rows=np.sort(rows))
    print("\npolicy forward: max |gpu - oracle| %.2e, largest bound %.2e" % (err, bnd))


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

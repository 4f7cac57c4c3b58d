"""msim_mlp_forward_noalloc (fixed device scratch, no allocation in the call) against msim_mlp_forward.

Some callers cannot allocate device memory at the time they run the network: a trainer whose
memory belongs to PyTorch's caching allocator (a second allocator's cudaMalloc can fail for lack
of headroom while torch's cache holds free blocks), or a control loop that must not allocate or
free after start-up (cudaFree synchronises the device).  The no-allocation entry point serves
them with a fixed device array.

Both run the same tcgen05 GEMMs on the same BF16 weights (the network's FP32 master weights rounded
to nearest-even, which is what msim_mlp_forward's BF16 copy holds), so the outputs agree far inside
the forward tolerance of the MLP tests (2e-2 of the largest output against the FP64 oracle); the
test uses that tolerance.  Two calls in a row with different inputs and batch sizes, each checked:
the shared scratch keeps the previous call's contents, which must not leak into the next.  The
first call is also checked against the FP64 MLP oracle element by element (an independent check),
and the device's free memory must not change across the second call.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2603_29332_b300 import msim
from tests.gpu_common import mlp_bf16_reference

pytestmark = pytest.mark.gpu


def _weights(net):
    p = net.unflatten(net.get(0))
    W1 = torch.zeros((net.hidden, net.in_pitch), dtype=torch.bfloat16, device="cuda")
    W1[:, : net.d_in] = torch.as_tensor(np.ascontiguousarray(p[0])).cuda().bfloat16()
    W2 = torch.as_tensor(np.ascontiguousarray(p[2])).cuda().bfloat16().contiguous()
    W3 = torch.as_tensor(np.ascontiguousarray(p[4])).cuda().bfloat16().contiguous()
    b1, b2, b3 = (torch.as_tensor(np.ascontiguousarray(p[i]), dtype=torch.float32).cuda() for i in (1, 3, 5))
    return W1, b1, W2, b2, W3, b3


@pytest.mark.parametrize("out_sigmoid", [False, True])
def test_noalloc_forward_matches_allocating_forward(out_sigmoid):
    d_in, hid, d_out = 90, 512, 700
    net = msim.MLP(d_in, hid, d_out, out_sigmoid=out_sigmoid, max_batch=2048, seed=5, out_scale=1.0)
    W1, b1, W2, b2, W3, b3 = _weights(net)
    rng = np.random.default_rng(17)
    status = torch.full((1,), 7, dtype=torch.int32, device="cuda")
    free = []
    for call, B in enumerate((2048, 333)):   # two calls in a row; the second smaller, ragged tail
        X = net.pad_input(rng.uniform(-1, 1, (B, d_in)))
        ref = net.forward(X)[:, :d_out]
        Y = torch.empty((B, d_out), dtype=torch.float32, device="cuda")
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
        got = msim.mlp_forward_noalloc(W1, b1, W2, b2, W3, b3, X, d_in, out_sigmoid=out_sigmoid, Y=Y,
                                       status=status)
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
        assert int(status.item()) == 0
        tol = 2e-2 * float(ref.abs().max())
        assert float((got - ref).abs().max()) <= tol
        if call == 0:
            # independent check: the FP64 MLP oracle at the same BF16 weights and inputs
            params = [W1[:, :d_in].double().cpu().numpy(), b1.double().cpu().numpy(), W2.double().cpu().numpy(),
                      b2.double().cpu().numpy(), W3.double().cpu().numpy(), b3.double().cpu().numpy()]
            rows = np.arange(0, B, 37)
            x = X[rows, :d_in].double().cpu().numpy()
            y, bound = mlp_bf16_reference(params, x, out_sigmoid)
            dev = got[rows].double().cpu().numpy()
            assert np.all(np.abs(dev - y) <= bound + 1e-6)
    # nothing allocated by the second call (the first may load the module and commit the array)
    assert free[3] == free[2]
    net.close()


def test_noalloc_rejects_batches_beyond_the_scratch():
    hid = 1024
    B = msim.NOALLOC_MAX_ACT_ELEMS // hid + 1
    W1 = torch.zeros((hid, 8), dtype=torch.bfloat16, device="cuda")
    W2 = torch.zeros((hid, hid), dtype=torch.bfloat16, device="cuda")
    W3 = torch.zeros((8, hid), dtype=torch.bfloat16, device="cuda")
    b = torch.zeros(hid, device="cuda")
    X = torch.zeros((B, 8), dtype=torch.bfloat16, device="cuda")
    with pytest.raises(msim.MsimError) as ei:
        msim.mlp_forward_noalloc(W1, b, W2, b, W3, b, X, 8)
    assert msim.STATUS_NAMES[ei.value.code] == "MSIM_ERR_ARG"
    assert "MSIM_NOALLOC_MAX_ACT_ELEMS" in str(ei.value)

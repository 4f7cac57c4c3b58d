"""The tcgen05 BF16 GEMM (msim_gemm_bf16, msim_gemm_bf16_mn) against a plain PyTorch FP32 reference of the same op."""
import pytest

torch = pytest.importorskip("torch")

from paper_2603_29332_b300 import msim

pytestmark = pytest.mark.gpu


def _ref(A, B, bias, act):
    z = A.float() @ B.float().T
    if bias is not None:
        z = z + bias
    if act == 1:
        return z * torch.sigmoid(z), z
    if act == 2:
        return torch.sigmoid(z), z
    return z, z


@pytest.mark.parametrize("M,N,K,act,bias", [
    (128, 128, 64, 0, False),      # one tile, one K slice
    (300, 200, 90, 1, True),       # ragged rows, columns and K (TMA zero fill)
    (64, 48, 16, 2, True),         # smaller than a tile
    (1000, 512, 512, 1, True),     # hidden layer shape
    (4096, 2800, 512, 0, True),    # surrogate output layer (256-wide tiles)
    (257, 1024, 2184, 1, True),    # long K (policy input layer)
])
def test_gemm_matches_fp32_reference(M, N, K, act, bias):
    g = torch.Generator(device="cuda").manual_seed(M * 7 + N)
    Kp = (K + 7) // 8 * 8
    A = torch.zeros((M, Kp), device="cuda", dtype=torch.bfloat16)
    B = torch.zeros((N, Kp), device="cuda", dtype=torch.bfloat16)
    A[:, :K] = (torch.randn((M, K), device="cuda", generator=g)).bfloat16()
    B[:, :K] = (torch.randn((N, K), device="cuda", generator=g) / K ** 0.5).bfloat16()
    b = torch.randn(N, device="cuda", generator=g) if bias else None
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    C = msim.gemm_bf16(A[:, :K], B[:, :K], b, act=act, err=err)
    torch.cuda.synchronize()
    ref, _ = _ref(A[:, :K], B[:, :K], b, act)
    assert err.item() == 0
    # FP32 accumulation of exact BF16 products: error ~ K * 2^-24 * sum |a b|
    scale = (A[:, :K].float().abs() @ B[:, :K].float().abs().T) + 1.0
    assert ((C - ref).abs() / scale).max().item() < 1e-5


@pytest.mark.parametrize("M,N,K,a_mn,b_mn", [
    (300, 200, 90, 1, 0),        # ragged, A stored [K][M]
    (300, 200, 90, 0, 1),        # ragged, B stored [K][N]
    (64, 48, 16, 1, 1),          # smaller than a tile, both transposed
    (2448, 512, 4000, 1, 1),     # weight gradient dY^T H of the surrogate's output layer, ragged batch
    (4096, 512, 2448, 0, 1),     # input gradient dY W3 (W3 stored [out][hidden])
    (512, 90, 4096, 1, 1),       # first-layer weight gradient dZ1^T X
    (8192, 2048, 200, 1, 1),     # 256-wide tiles (four 64-column boxes per B stage)
])
def test_gemm_mn_contiguous_operands(M, N, K, a_mn, b_mn):
    """msim_gemm_bf16_mn reads A as [K][M] and / or B as [K][N] storage (the tensor cores'
    transposed operand mode) and must give what the K-contiguous GEMM gives on the transposes."""
    g = torch.Generator(device="cuda").manual_seed(M + 3 * N + 5 * K)
    pad = lambda x: (x + 7) // 8 * 8
    A = torch.randn((M, K), device="cuda", generator=g).bfloat16()
    B = (torch.randn((N, K), device="cuda", generator=g) / K ** 0.5).bfloat16()
    b = torch.randn(N, device="cuda", generator=g)
    if a_mn:
        As = torch.zeros((K, pad(M)), device="cuda", dtype=torch.bfloat16)
        As[:, :M] = A.T
        Aarg = As[:, :M]
    else:
        As = torch.zeros((M, pad(K)), device="cuda", dtype=torch.bfloat16)
        As[:, :K] = A
        Aarg = As[:, :K]
    if b_mn:
        Bs = torch.zeros((K, pad(N)), device="cuda", dtype=torch.bfloat16)
        Bs[:, :N] = B.T
        Barg = Bs[:, :N]
    else:
        Bs = torch.zeros((N, pad(K)), device="cuda", dtype=torch.bfloat16)
        Bs[:, :K] = B
        Barg = Bs[:, :K]
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    C = msim.gemm_bf16(Aarg, Barg, b, act=1, err=err, a_mn=bool(a_mn), b_mn=bool(b_mn))
    torch.cuda.synchronize()
    assert C.shape == (M, N) and err.item() == 0
    ref, _ = _ref(A, B, b, 1)
    scale = (A.float().abs() @ B.float().abs().T) + 1.0
    assert ((C - ref).abs() / scale).max().item() < 1e-5


@pytest.mark.parametrize("M,N,K", [(300, 200, 90), (16384, 1024, 707), (4096, 3104, 512)])
def test_gemm_addend(M, N, K):
    """An FP32 addend [M][N] joins the accumulator with the bias, before the activation: the
    product over a column subset of K kept from an earlier call completes to the whole product."""
    g = torch.Generator(device="cuda").manual_seed(M + N + K)
    Kp = (K + 7) // 8 * 8
    A = torch.zeros((M, Kp), device="cuda", dtype=torch.bfloat16)
    B = torch.zeros((N, Kp), device="cuda", dtype=torch.bfloat16)
    A[:, :K] = torch.randn((M, K), device="cuda", generator=g).bfloat16()
    B[:, :K] = (torch.randn((N, K), device="cuda", generator=g) / K ** 0.5).bfloat16()
    b = torch.randn(N, device="cuda", generator=g)
    add = torch.randn((M, N), device="cuda", generator=g)
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    C = msim.gemm_bf16(A[:, :K], B[:, :K], b, act=1, err=err, addend=add)
    Z = msim.gemm_bf16(A[:, :K], B[:, :K], b, act=0, err=err, addend=add)
    torch.cuda.synchronize()
    assert err.item() == 0
    z = A[:, :K].float() @ B[:, :K].float().T + b + add
    scale = (A[:, :K].float().abs() @ B[:, :K].float().abs().T) + add.abs() + 1.0
    assert ((Z - z).abs() / scale).max().item() < 1e-5
    assert ((C - z * torch.sigmoid(z)).abs() / scale).max().item() < 1e-5
    # splitting K at a multiple of 8 and carrying the first part as the addend
    c = (K // 2) // 8 * 8
    if c >= 8:
        pre = msim.gemm_bf16(A[:, :c], B[:, :c])
        Zs = msim.gemm_bf16(A[:, c:K], B[:, c:K], b, addend=pre)
        torch.cuda.synchronize()
        assert ((Zs - (z - add)).abs() / scale).max().item() < 1e-5


def test_gemm_bf16_output_and_preactivation():
    M, N, K = 256, 384, 160
    g = torch.Generator(device="cuda").manual_seed(3)
    A = torch.randn((M, K), device="cuda", generator=g).bfloat16()
    B = (torch.randn((N, K), device="cuda", generator=g) / K ** 0.5).bfloat16()
    b = torch.randn(N, device="cuda", generator=g)
    Z = torch.empty((M, N), device="cuda", dtype=torch.bfloat16)
    C = msim.gemm_bf16(A, B, b, act=1, out_bf16=True, Z=Z)
    torch.cuda.synchronize()
    ref, zref = _ref(A, B, b, 1)
    assert C.dtype == torch.bfloat16
    assert (C.float() - ref).abs().max().item() <= 1e-2 * ref.abs().max().item()
    assert (Z.float() - zref).abs().max().item() <= 1e-2 * zref.abs().max().item()


def test_gemm_rejects_unaligned_pitch():
    A = torch.zeros((16, 20), device="cuda", dtype=torch.bfloat16)   # pitch 20 is not a multiple of 8
    B = torch.zeros((16, 20), device="cuda", dtype=torch.bfloat16)
    with pytest.raises(msim.MsimError) as ei:
        msim.gemm_bf16(A, B)
    assert ei.value.code == 1

// mlp.cu -- forward / backward / Adam of the 3-layer MLP on the tcgen05 GEMM (see mlp.h).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "gemm_tc.h"
#include "mlp.h"

namespace msim {
namespace {

int pad8(int x) { return (x + 7) & ~7; }
size_t pad8s(size_t x) { return (x + 7) & ~size_t(7); }

// ---------------------------------------------------------------- elementwise kernels
__global__ void k_init(float* P, size_t n, size_t oW1, int hid, int in, int inp, size_t oW2, size_t oW3, int outp_rows,
                       float bound1, float bound2, float bound3, uint32_t k0, uint32_t k1) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        uint32_t c[4] = {(uint32_t)i, (uint32_t)(i >> 32), 0x5eedu, 0u};
        philox4x32_10(c, k0, k1);
        const float u = 2.f * u01_from_bits(c[0]) - 1.f;
        float v = 0.f;
        if (i >= oW1 && i < oW1 + (size_t)hid * inp) {
            const int col = (int)((i - oW1) % inp);
            v = col < in ? bound1 * u : 0.f;
        } else if (i >= oW2 && i < oW2 + (size_t)hid * hid) {
            v = bound2 * u;
        } else if (i >= oW3 && i < oW3 + (size_t)outp_rows * hid) {
            v = bound3 * u;
        }
        P[i] = v;
    }
}

__global__ void k_to_bf16(const float* P, __nv_bfloat16* Ph, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        Ph[i] = __float2bfloat16_rn(P[i]);
}

// dY = d mean((y - t)^2) / dy (times y (1 - y) for a sigmoid output), as BF16; loss sum
__global__ void k_loss_grad(const float* Y, int ldy, const float* T, int ldt, int B, int N, float scale, int sig,
                            __nv_bfloat16* dY, int ldd, float* loss_acc) {
    float acc = 0.f;
    for (int r = blockIdx.x; r < B; r += gridDim.x)   // rows per block, no flat-index division
        for (int c = threadIdx.x; c < N; c += blockDim.x) {
            const float y = Y[(size_t)r * ldy + c];
            const float d = y - T[(size_t)r * ldt + c];
            acc += d * d;
            float g = scale * d;
            if (sig) g *= y * (1.f - y);
            dY[(size_t)r * ldd + c] = __float2bfloat16_rn(g);
        }
    // the block's sum first (one atomic per block, not per warp: they all hit one address)
    __shared__ float part[32];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        acc = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0.f;
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (threadIdx.x == 0) atomicAdd(loss_acc, acc);
    }
}

// dZ = dH * silu'(Z), silu'(z) = s (1 + z (1 - s)), s = sigmoid(z)
__global__ void k_dsilu(const float* dH, const __nv_bfloat16* Z, int B, int N, int ld, __nv_bfloat16* dZ) {
    for (int r = blockIdx.x; r < B; r += gridDim.x)
        for (int c = threadIdx.x; c < N; c += blockDim.x) {
            const size_t o = (size_t)r * ld + c;
            const float z = __bfloat162float(Z[o]);
            const float sgm = 1.f / (1.f + expf(-z));
            dZ[o] = __float2bfloat16_rn(dH[o] * sgm * (1.f + z * (1.f - sgm)));
        }
}

// Column sums db[c] = sum over rows of src[r][c] in two deterministic stages: the rows in
// chunks of kColChunk, one block per (128 columns, chunk), each thread summing its column over
// the chunk (a warp's loads of a row are one contiguous run); then the chunks' partial sums in
// chunk order.
constexpr int kColChunk = 128;

__global__ void k_colsum_part(const __nv_bfloat16* src, int B, int N, int ld, float* part) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int r0 = blockIdx.y * kColChunk;
    if (c >= N) return;
    const int r1 = min(B, r0 + kColChunk);
    float s = 0.f;
#pragma unroll 8
    for (int r = r0; r < r1; ++r) s += __bfloat162float(src[(size_t)r * ld + c]);
    part[(size_t)blockIdx.y * N + c] = s;
}

__global__ void k_colsum_final(const float* part, int n_chunks, int N, float* db) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    float s = 0.f;
    for (int k = 0; k < n_chunks; ++k) s += part[(size_t)k * N + c];
    db[c] = s;
}

__global__ void k_adam(float* P, const float* G, float* Am, float* Av, size_t n, float lr, float b1, float b2,
                       float eps, float bc1, float bc2, __nv_bfloat16* Ph, const uint8_t* mask) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        if (mask && !mask[i]) continue;   // held at zero
        const float g = G[i];
        const float m = b1 * Am[i] + (1.f - b1) * g;
        const float v = b2 * Av[i] + (1.f - b2) * g * g;
        Am[i] = m;
        Av[i] = v;
        const float p = P[i] - lr * (m / bc1) / (sqrtf(v / bc2) + eps);
        P[i] = p;
        Ph[i] = __float2bfloat16_rn(p);
    }
}

// P[i] *= scale[row of i] for weights inside the mask, 0 outside it (biases untouched)
__global__ void k_mask_params(float* P, const uint8_t* mask, const float* row_scale, size_t n, size_t oW1, int inp,
                              int hid, size_t oW2, size_t oW3, int outp) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        int row = -1;
        if (i >= oW1 && i < oW1 + (size_t)hid * inp) row = (int)((i - oW1) / inp);
        else if (i >= oW2 && i < oW2 + (size_t)hid * hid) row = hid + (int)((i - oW2) / hid);
        else if (i >= oW3 && i < oW3 + (size_t)outp * hid) row = 2 * hid + (int)((i - oW3) / hid);
        if (row < 0) continue;
        P[i] = mask[i] ? P[i] * row_scale[row] : 0.f;
    }
}

// first-layer biases drawn U(-r, r), r = sum |W1 row| (the unit's largest pre-activation over
// inputs in [-1, 1]), so that the units' SiLU bends spread over the input range
__global__ void k_spread_b1(float* P, size_t oW1, size_t ob1, int inp, int hid, uint32_t k0, uint32_t k1) {
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= hid) return;
    float r = 0.f;
    for (int c = 0; c < inp; ++c) r += fabsf(P[oW1 + (size_t)u * inp + c]);
    uint32_t ctr[4] = {(uint32_t)u, 0xb1a5u, 0u, 0u};
    philox4x32_10(ctr, k0, k1);
    P[ob1 + u] = r * (2.f * u01_from_bits(ctr[0]) - 1.f);
}

cudaError_t colsum(const __nv_bfloat16* src, int B, int N, int ld, float* part, float* db, cudaStream_t s) {
    const int chunks = (B + kColChunk - 1) / kColChunk;
    k_colsum_part<<<dim3((N + 127) / 128, chunks), 128, 0, s>>>(src, B, N, ld, part);
    k_colsum_final<<<(N + 255) / 256, 256, 0, s>>>(part, chunks, N, db);
    return cudaGetLastError();
}

int nblocks(size_t n) { return (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096); }

cudaError_t gemm(const void* A, int lda, const void* B, int ldb, int M, int N, int K, void* C, int ldc, int c_bf16,
                 const float* bias, int act, void* Z, int ldz, uint32_t* err, cudaStream_t s,
                 const float* scale = nullptr, const float* shift = nullptr, int a_mn = 0, int b_mn = 0) {
    GemmArgs g;
    std::memset(&g, 0, sizeof(g));
    g.M = M; g.N = N; g.K = K; g.C = C; g.ldc = ldc; g.c_bf16 = c_bf16; g.bias = bias; g.act = act;
    g.Z = Z; g.ldz = ldz; g.err = err; g.scale = scale; g.shift = shift; g.a_mn = a_mn; g.b_mn = b_mn;
    return gemm_bf16_tc(A, lda, B, ldb, g, s);
}

// weight gradient G[M][N] (pitch ldg) = D^T S over the batch: D [B][M], S [B][N] as stored
// (both operands MN-contiguous)
cudaError_t gemm_dw(const __nv_bfloat16* D, int ldd, const __nv_bfloat16* S, int lds, int M, int N, int B, float* G,
                    int ldg, uint32_t* err, cudaStream_t s) {
    return gemm(D, ldd, S, lds, M, N, B, G, ldg, 0, nullptr, 0, nullptr, 0, err, s, nullptr, nullptr, 1, 1);
}
// input gradient dH[B][N] = D W for D [B][K] and the layer's weights W [K][N] as stored (W's
// rows are the layer's outputs: the B operand is N-contiguous)
cudaError_t gemm_dx(const __nv_bfloat16* D, int ldd, const __nv_bfloat16* W, int ldw, int B, int N, int K, float* dH,
                    int ldh, uint32_t* err, cudaStream_t s) {
    return gemm(D, ldd, W, ldw, B, N, K, dH, ldh, 0, nullptr, 0, nullptr, 0, err, s, nullptr, nullptr, 0, 1);
}

#define CK(x)                                  \
    do {                                       \
        const cudaError_t e_ = (x);            \
        if (e_ != cudaSuccess) return e_;      \
    } while (0)

}  // namespace

cudaError_t mlp_create(int in, int hid, int out, int out_act, int max_batch, Mlp** out_mlp) {
    *out_mlp = nullptr;
    if (in < 1 || hid < 8 || (hid % 8) || out < 1 || max_batch < 1) return cudaErrorInvalidValue;
    Mlp* m = new Mlp();
    std::memset(m, 0, sizeof(Mlp));
    m->in = in; m->inp = pad8(in); m->hid = hid; m->out = out; m->outp = pad8(out); m->out_act = out_act;
    m->max_batch = max_batch;
    size_t o = 0;
    m->oW1 = o; o = pad8s(o + (size_t)hid * m->inp);
    m->ob1 = o; o = pad8s(o + hid);
    m->oW2 = o; o = pad8s(o + (size_t)hid * hid);
    m->ob2 = o; o = pad8s(o + hid);
    m->oW3 = o; o = pad8s(o + (size_t)m->outp * hid);
    m->ob3 = o; o = pad8s(o + m->outp);
    m->n_params = o;
    const size_t np = m->n_params, B = (size_t)max_batch;
    cudaError_t e = cudaSuccess;
    auto A = [&](void** p, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(p, bytes);
        if (e == cudaSuccess) e = cudaMemset(*p, 0, bytes);
    };
    A((void**)&m->P, np * 4); A((void**)&m->G, np * 4); A((void**)&m->Am, np * 4); A((void**)&m->Av, np * 4);
    A((void**)&m->Ph, np * 2);
    A((void**)&m->H1, B * hid * 2); A((void**)&m->Z1, B * hid * 2); A((void**)&m->H2, B * hid * 2);
    A((void**)&m->Z2, B * hid * 2); A((void**)&m->dY, B * m->outp * 2); A((void**)&m->dZ1, B * hid * 2);
    A((void**)&m->dZ2, B * hid * 2);
    A((void**)&m->Y, B * m->outp * 4); A((void**)&m->dH, B * hid * 4);
    A((void**)&m->loss_acc, 8); A((void**)&m->err, 8);
    A((void**)&m->colpart, (size_t)((max_batch + 127) / 128) * std::max(m->outp, hid) * 4);
    if (e != cudaSuccess) {
        mlp_destroy(m);
        return e;
    }
    *out_mlp = m;
    return cudaSuccess;
}

void mlp_destroy(Mlp* m) {
    if (!m) return;
    void* ptrs[] = {m->P, m->G, m->Am, m->Av, m->Ph, m->H1, m->Z1, m->H2, m->Z2, m->dY, m->dZ1, m->dZ2, m->Y, m->dH,
                    m->loss_acc, m->err, m->mask, m->colpart};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete m;
}

cudaError_t mlp_sync_bf16(Mlp* m, cudaStream_t s) {
    ++m->version;
    k_to_bf16<<<nblocks(m->n_params), 256, 0, s>>>(m->P, m->Ph, m->n_params);
    return cudaGetLastError();
}

cudaError_t mlp_init(Mlp* m, uint64_t seed, float out_scale, cudaStream_t s) {
    const float b1 = sqrtf(6.f / m->in), b2 = sqrtf(6.f / m->hid), b3 = out_scale * sqrtf(6.f / m->hid);
    k_init<<<nblocks(m->n_params), 256, 0, s>>>(m->P, m->n_params, m->oW1, m->hid, m->in, m->inp, m->oW2, m->oW3,
                                                 m->out, b1, b2, b3, (uint32_t)seed, (uint32_t)(seed >> 32));
    CK(cudaGetLastError());
    CK(cudaMemsetAsync(m->Am, 0, m->n_params * 4, s));
    CK(cudaMemsetAsync(m->Av, 0, m->n_params * 4, s));
    m->adam_t = 0;
    return mlp_sync_bf16(m, s);
}

cudaError_t mlp_set_mask(Mlp* m, const uint8_t* host_mask, uint64_t spread_seed, cudaStream_t s) {
    // per weight row: the mlp_init bound sqrt(6 / fan_in) becomes sqrt(3 / fan) over the row's
    // unmasked entries
    const int rows = 2 * m->hid + m->outp;
    std::vector<float> scale(rows, 1.f);
    auto row_scale = [&](size_t off, int r, int width, int fan_in) {
        int fan = 0;
        for (int c = 0; c < width; ++c) fan += host_mask[off + (size_t)r * width + c] != 0;
        return fan > 0 ? std::sqrt((3.f / fan) / (6.f / fan_in)) : 0.f;
    };
    for (int r = 0; r < m->hid; ++r) scale[r] = row_scale(m->oW1, r, m->inp, m->in);
    for (int r = 0; r < m->hid; ++r) scale[m->hid + r] = row_scale(m->oW2, r, m->hid, m->hid);
    for (int r = 0; r < m->outp; ++r) scale[2 * m->hid + r] = row_scale(m->oW3, r, m->hid, m->hid);
    float* d_scale = nullptr;
    if (!m->mask) CK(cudaMalloc(&m->mask, m->n_params));
    CK(cudaMalloc(&d_scale, rows * sizeof(float)));
    cudaError_t e = cudaMemcpyAsync(m->mask, host_mask, m->n_params, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_scale, scale.data(), rows * sizeof(float), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        k_mask_params<<<nblocks(m->n_params), 256, 0, s>>>(m->P, m->mask, d_scale, m->n_params, m->oW1, m->inp, m->hid,
                                                             m->oW2, m->oW3, m->outp);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && spread_seed) {
        k_spread_b1<<<(m->hid + 127) / 128, 128, 0, s>>>(m->P, m->oW1, m->ob1, m->inp, m->hid, (uint32_t)spread_seed,
                                                        (uint32_t)(spread_seed >> 32));
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = mlp_sync_bf16(m, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // the host arrays go out of scope
    cudaFree(d_scale);
    return e;
}

cudaError_t mlp_forward(Mlp* m, const __nv_bfloat16* X, int ldx, int B, float* Y, int ldy, cudaStream_t s) {
    if (B < 1 || B > m->max_batch) return cudaErrorInvalidValue;
    const int h = m->hid;
    CK(gemm(X, ldx, m->Ph + m->oW1, m->inp, B, h, m->in, m->H1, h, 1, m->P + m->ob1, 1, m->Z1, h, m->err, s));
    CK(gemm(m->H1, h, m->Ph + m->oW2, h, B, h, h, m->H2, h, 1, m->P + m->ob2, 1, m->Z2, h, m->err, s));
    return gemm(m->H2, h, m->Ph + m->oW3, h, B, m->out, h, Y, ldy, 0, m->P + m->ob3, m->out_act, nullptr, 0, m->err, s);
}

cudaError_t mlp_infer(Mlp* m, const __nv_bfloat16* X, int ldx, int B, float* Y, int ldy, cudaStream_t s) {
    if (B < 1 || B > m->max_batch) return cudaErrorInvalidValue;
    const int h = m->hid;
    CK(gemm(X, ldx, m->Ph + m->oW1, m->inp, B, h, m->in, m->H1, h, 1, m->P + m->ob1, 1, nullptr, 0, m->err, s));
    CK(gemm(m->H1, h, m->Ph + m->oW2, h, B, h, h, m->H2, h, 1, m->P + m->ob2, 1, nullptr, 0, m->err, s));
    return gemm(m->H2, h, m->Ph + m->oW3, h, B, m->out, h, Y, ldy, 0, m->P + m->ob3, m->out_act, nullptr, 0, m->err, s);
}

cudaError_t mlp_infer_split(Mlp* m, const __nv_bfloat16* X, int ldx, int B, int c, float* Hpre, int compute_pre,
                            float* Y, int ldy, cudaStream_t s) {
    if (B < 1 || B > m->max_batch || c < 8 || c % 8 || c >= m->in) return cudaErrorInvalidValue;
    const int h = m->hid;
    const __nv_bfloat16* W1 = m->Ph + m->oW1;
    if (compute_pre) CK(gemm(X, ldx, W1, m->inp, B, h, c, Hpre, h, 0, nullptr, 0, nullptr, 0, m->err, s));
    GemmArgs g;
    std::memset(&g, 0, sizeof(g));
    g.M = B; g.N = h; g.K = m->in - c; g.C = m->H1; g.ldc = h; g.c_bf16 = 1; g.bias = m->P + m->ob1; g.act = 1;
    g.err = m->err; g.addend = Hpre; g.ld_add = h;
    CK(gemm_bf16_tc(X + c, ldx, W1 + c, m->inp, g, s));
    CK(gemm(m->H1, h, m->Ph + m->oW2, h, B, h, h, m->H2, h, 1, m->P + m->ob2, 1, nullptr, 0, m->err, s));
    return gemm(m->H2, h, m->Ph + m->oW3, h, B, m->out, h, Y, ldy, 0, m->P + m->ob3, m->out_act, nullptr, 0, m->err, s);
}

cudaError_t mlp_infer_head(Mlp* m, const __nv_bfloat16* X, int ldx, int B, const __nv_bfloat16* W3, const float* b3,
                           int N, const float* scale, const float* shift, float* Y, int ldy, cudaStream_t s) {
    if (B < 1 || B > m->max_batch) return cudaErrorInvalidValue;
    const int h = m->hid;
    CK(gemm(X, ldx, m->Ph + m->oW1, m->inp, B, h, m->in, m->H1, h, 1, m->P + m->ob1, 1, nullptr, 0, m->err, s));
    CK(gemm(m->H1, h, m->Ph + m->oW2, h, B, h, h, m->H2, h, 1, m->P + m->ob2, 1, nullptr, 0, m->err, s));
    return gemm(m->H2, h, W3, h, B, N, h, Y, ldy, 0, b3, 0, nullptr, 0, m->err, s, scale, shift);
}

cudaError_t mlp_backward(Mlp* m, const __nv_bfloat16* X, int ldx, const float* T, int ldt, int B, cudaStream_t s) {
    if (B < 1 || B > m->max_batch) return cudaErrorInvalidValue;
    const int h = m->hid;
    CK(mlp_forward(m, X, ldx, B, m->Y, m->outp, s));
    CK(cudaMemsetAsync(m->loss_acc, 0, 4, s));
    const size_t nY = (size_t)B * m->out;
    k_loss_grad<<<std::min(B, 8192), 256, 0, s>>>(m->Y, m->outp, T, ldt, B, m->out, 2.f / (float)nY, m->out_act == 2, m->dY,
                                             m->outp, m->loss_acc);
    CK(cudaGetLastError());
    // layer 3: dW3 = dY^T H2, db3 = column sums of dY, dH2 = dY W3
    CK(gemm_dw(m->dY, m->outp, m->H2, h, m->out, h, B, m->G + m->oW3, h, m->err, s));
    CK(colsum(m->dY, B, m->out, m->outp, m->colpart, m->G + m->ob3, s));
    CK(gemm_dx(m->dY, m->outp, m->Ph + m->oW3, h, B, h, m->out, m->dH, h, m->err, s));
    k_dsilu<<<std::min(B, 8192), 256, 0, s>>>(m->dH, m->Z2, B, h, h, m->dZ2);
    CK(cudaGetLastError());
    // layer 2
    CK(gemm_dw(m->dZ2, h, m->H1, h, h, h, B, m->G + m->oW2, h, m->err, s));
    CK(colsum(m->dZ2, B, h, h, m->colpart, m->G + m->ob2, s));
    CK(gemm_dx(m->dZ2, h, m->Ph + m->oW2, h, B, h, h, m->dH, h, m->err, s));
    k_dsilu<<<std::min(B, 8192), 256, 0, s>>>(m->dH, m->Z1, B, h, h, m->dZ1);
    CK(cudaGetLastError());
    // layer 1
    CK(gemm_dw(m->dZ1, h, X, ldx, h, m->in, B, m->G + m->oW1, m->inp, m->err, s));
    return colsum(m->dZ1, B, h, h, m->colpart, m->G + m->ob1, s);
}

cudaError_t mlp_adam(Mlp* m, float lr, float beta1, float beta2, float eps, cudaStream_t s) {
    m->adam_t += 1;
    ++m->version;
    const float bc1 = 1.f - powf(beta1, (float)m->adam_t), bc2 = 1.f - powf(beta2, (float)m->adam_t);
    k_adam<<<nblocks(m->n_params), 256, 0, s>>>(m->P, m->G, m->Am, m->Av, m->n_params, lr, beta1, beta2, eps, bc1,
                                                  bc2, m->Ph, m->mask);
    return cudaGetLastError();
}

}  // namespace msim

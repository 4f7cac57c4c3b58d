// mlp.h -- 3-layer MLP (SiLU hidden layers) on the tcgen05 GEMM: forward, backward, Adam.
//
// Used by the muscle-geometry surrogate (trained on the GPU) and by the policy network of the
// closed-loop rollout.  Parameters live in one flat FP32 buffer (master copy, Adam moments and
// gradients share its layout) with a BF16 copy for the GEMMs.  Activations are BF16, accumulation
// FP32, the output FP32.  The backward reads activations, gradients and weights as stored (the
// GEMM's MN-contiguous operand mode), so no transposed copies exist.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace msim {

struct Mlp {
    int in, inp;           // input width and its pitch (multiple of 8)
    int hid;               // hidden width (multiple of 8)
    int out, outp;         // output width and its pitch (multiple of 8)
    int out_act;           // 0 identity, 2 sigmoid
    int max_batch;         // batch capacity of the scratch buffers
    // flat parameter layout (FP32 element offsets; every segment starts at a multiple of 8)
    size_t oW1, ob1, oW2, ob2, oW3, ob3, n_params;
    float* P;              // master parameters
    float* G;              // gradients
    float* Am;             // Adam first moments
    float* Av;             // Adam second moments
    __nv_bfloat16* Ph;     // BF16 copy of P (same offsets)
    int adam_t;
    // scratch, max_batch rows
    __nv_bfloat16 *H1, *Z1, *H2, *Z2, *dY, *dZ1, *dZ2;
    float *Y, *dH;
    float* loss_acc;       // device scalar: sum of squared errors of the last backward
    uint32_t* err;         // device word: GEMM bounded-wait failures
    uint8_t* mask;         // [n_params] 1 = trainable, 0 = held at zero (nullptr: every parameter)
    uint64_t version;      // counts changes of the parameters (set, init, Adam steps)
    float* colpart;        // [batch chunks][max(outp, hid)] partial column sums of the bias gradients
};

cudaError_t mlp_create(int in, int hid, int out, int out_act, int max_batch, Mlp** out_mlp);
void mlp_destroy(Mlp* m);
// Kaiming-uniform weights (bound sqrt(6 / fan_in); the last layer scaled by out_scale), zero
// biases, drawn with a counter-based generator (Philox-4x32-10) keyed by seed.
cudaError_t mlp_init(Mlp* m, uint64_t seed, float out_scale, cudaStream_t s);
// refresh the BF16 copies after P changed (set from outside)
cudaError_t mlp_sync_bf16(Mlp* m, cudaStream_t s);
// Y [B][ldy] = mlp(X), X [B][ldx] BF16 (ldx multiple of 8, columns >= in ignored)
cudaError_t mlp_forward(Mlp* m, const __nv_bfloat16* X, int ldx, int B, float* Y, int ldy, cudaStream_t s);
// the same without the pre-activation copies a later backward needs (inference)
cudaError_t mlp_infer(Mlp* m, const __nv_bfloat16* X, int ldx, int B, float* Y, int ldy, cudaStream_t s);
// inference whose input columns [0, c) are the same as in an earlier call (c a multiple of 8,
// 8 <= c < in): their share of the first layer, X[:, :c] W1[:, :c]^T, is kept in Hpre [B][hid]
// (FP32; computed when compute_pre is set) and only columns [c, in) are multiplied again
cudaError_t mlp_infer_split(Mlp* m, const __nv_bfloat16* X, int ldx, int B, int c, float* Hpre, int compute_pre,
                            float* Y, int ldy, cudaStream_t s);
// inference with another output layer: layers 1-2 of m, then Y = (H2 W3^T + b3) * scale + shift
// (W3 [N][hid] BF16, b3, scale, shift [N]; identity output activation)
cudaError_t mlp_infer_head(Mlp* m, const __nv_bfloat16* X, int ldx, int B, const __nv_bfloat16* W3, const float* b3,
                           int N, const float* scale, const float* shift, float* Y, int ldy, cudaStream_t s);
// gradients of mean((y - t)^2) into G (forward included); T [B][ldt] FP32
cudaError_t mlp_backward(Mlp* m, const __nv_bfloat16* X, int ldx, const float* T, int ldt, int B, cudaStream_t s);
// one Adam step (Kingma & Ba 2015) on G, refreshes the BF16 copies; parameters outside the mask
// stay zero
cudaError_t mlp_adam(Mlp* m, float lr, float beta1, float beta2, float eps, cudaStream_t s);
// Connectivity mask (host array [n_params] in the flat layout, 1 = trainable): masked weights are
// set to zero and stay there; each weight row is re-drawn to the uniform bound sqrt(3 / fan),
// fan = its unmasked entries (variance 1 / fan), from the values mlp_init drew; with a non-zero
// spread_seed the first-layer biases are drawn U(-r, r), r the sum of the row's |weights|, so the
// units' bends spread over inputs in [-1, 1].  Call after mlp_init.  Synchronous (the host array
// may be freed on return).
cudaError_t mlp_set_mask(Mlp* m, const uint8_t* host_mask, uint64_t spread_seed, cudaStream_t s);

// Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC 2011): 4 x 32 random bits for a 128-bit counter
// and a 64-bit key.  Shared by the surrogate's sampler and the policy's exploration.
__host__ __device__ inline void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
        const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}
__host__ __device__ inline float u01_from_bits(uint32_t x) { return ((x >> 8) + 0.5f) * (1.f / 16777216.f); }

}  // namespace msim

// policy.cu -- observation assembly of the closed-loop rollout (policy network in the loop).
//
// obs row of environment e (BF16, pitch ldx): [q (n) | qd (n) | act (m) | F / F_max (m) | 0 ...],
// the state the policy sees after the previous control step.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "kernels.h"

namespace msim {
namespace {

__global__ void k_obs(const float* q, const float* qd, const float* act, const float* force, const float* inv_fmax,
                      int pitch_n, int pitch_m, int n, int m, int n_envs, __nv_bfloat16* X, int ldx) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < (size_t)n_envs * ldx;
         i += (size_t)gridDim.x * blockDim.x) {
        const int e = (int)(i / ldx), j = (int)(i % ldx);
        float v = 0.f;
        if (j < n) v = q[(size_t)e * pitch_n + j];
        else if (j < 2 * n) v = qd[(size_t)e * pitch_n + j - n];
        else if (j < 2 * n + m) v = act[(size_t)e * pitch_m + j - 2 * n];
        else if (j < 2 * n + 2 * m) v = force[(size_t)e * pitch_m + j - 2 * n - m] * inv_fmax[j - 2 * n - m];
        X[i] = __float2bfloat16_rn(v);
    }
}

}  // namespace

cudaError_t launch_obs(const float* q, const float* qd, const float* act, const float* force, const float* inv_fmax,
                       int pitch_n, int pitch_m, int n, int m, int n_envs, __nv_bfloat16* X, int ldx, cudaStream_t s) {
    const size_t tot = (size_t)n_envs * ldx;
    const int blocks = (int)((tot + 255) / 256 < 8192 ? (tot + 255) / 256 : 8192);
    k_obs<<<blocks, 256, 0, s>>>(q, qd, act, force, inv_fmax, pitch_n, pitch_m, n, m, n_envs, X, ldx);
    return cudaGetLastError();
}

}  // namespace msim

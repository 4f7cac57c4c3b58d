// policy.cu -- observation assembly of the closed-loop rollout (policy network in the loop).
//
// obs row of environment e (BF16, pitch ldx): [q (n) | qd (n) | act (m) | F / F_max (m) | 0 ...],
// the state the policy sees after the previous control step.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "kernels.h"
#include "mlp.h"

namespace msim {
namespace {

// Elementwise kernels over [environment][column] rows: one block per row at a time (no 64-bit
// division of a flat index per element).
__global__ void k_obs(const float* q, const float* qd, const float* act, const float* force, const float* inv_fmax,
                      int pitch_n, int pitch_m, int n, int m, int n_envs, __nv_bfloat16* X, int ldx) {
    for (int e = blockIdx.x; e < n_envs; e += gridDim.x)
        for (int j = threadIdx.x; j < ldx; j += blockDim.x) {
            float v = 0.f;
            if (j < n) v = q[(size_t)e * pitch_n + j];
            else if (j < 2 * n) v = qd[(size_t)e * pitch_n + j - n];
            else if (j < 2 * n + m) v = act[(size_t)e * pitch_m + j - 2 * n];
            else if (j < 2 * n + 2 * m) v = force[(size_t)e * pitch_m + j - 2 * n - m] * inv_fmax[j - 2 * n - m];
            X[(size_t)e * ldx + j] = __float2bfloat16_rn(v);
        }
}

// a = mu + sigma * eps, eps standard normal by Box-Muller on Philox-4x32-10 bits keyed by seed,
// counter (environment, muscle pair, control-step counter)
__global__ void k_flow_init(const float* mu, int ldmu, float* a, int lda, int n_envs, int m, float sigma,
                            uint32_t seed, const uint32_t* act_ctr) {
    const uint32_t step = *act_ctr;
    const int pairs = (m + 1) / 2;
    for (int e = blockIdx.x; e < n_envs; e += gridDim.x)
    for (int jp = threadIdx.x; jp < pairs; jp += blockDim.x) {
        const int j = 2 * jp;
        float z0 = 0.f, z1 = 0.f;
        if (sigma > 0.f) {
            uint32_t c[4] = {(uint32_t)e, (uint32_t)j, step, 0x666c6f77u};
            philox4x32_10(c, seed, 0xa5a5a5a5u);
            const float u1 = u01_from_bits(c[0]), u2 = u01_from_bits(c[1]);
            const float r = sqrtf(-2.f * logf(u1));
            float sn, cs;
            sincospif(2.f * u2, &sn, &cs);
            z0 = r * cs;
            z1 = r * sn;
        }
        a[(size_t)e * lda + j] = mu[(size_t)e * ldmu + j] + sigma * z0;
        if (j + 1 < m) a[(size_t)e * lda + j + 1] = mu[(size_t)e * ldmu + j + 1] + sigma * z1;
    }
}

// flow-network input columns that change per Euler step: X[e][off + j] = a[e][j], X[e][off + m] = t
__global__ void k_flow_input(const float* a, int lda, int n_envs, int m, float t, __nv_bfloat16* X, int ldx, int off) {
    for (int e = blockIdx.x; e < n_envs; e += gridDim.x)
        for (int j = threadIdx.x; j <= m; j += blockDim.x) {
            const float v = j < m ? a[(size_t)e * lda + j] : t;
            X[(size_t)e * ldx + off + j] = __float2bfloat16_rn(v);
        }
}

// copy the observation columns into the flow-network input rows (once per control step)
__global__ void k_copy_cols(const __nv_bfloat16* src, int lds, int n_envs, int cols, __nv_bfloat16* dst, int ldd) {
    for (int e = blockIdx.x; e < n_envs; e += gridDim.x)
        for (int j = threadIdx.x; j < cols; j += blockDim.x) dst[(size_t)e * ldd + j] = src[(size_t)e * lds + j];
}

// Euler step a += dt v; then either the next step's flow-input columns (X != nullptr: a and the
// time t_next, as k_flow_input writes them) or, after the last step, the excitations
// u = clamp(a, 0, 1)
__global__ void k_flow_axpy(float* a, int lda, const float* v, int ldv, int n_envs, int m, float dt, float* u, int ldu,
                            __nv_bfloat16* X, int ldx, int off, float t_next) {
    for (int e = blockIdx.x; e < n_envs; e += gridDim.x)
        for (int j = threadIdx.x; j <= m; j += blockDim.x) {
            if (j == m) {
                if (X) X[(size_t)e * ldx + off + m] = __float2bfloat16_rn(t_next);
                continue;
            }
            const float x = __fadd_rn(a[(size_t)e * lda + j], __fmul_rn(dt, v[(size_t)e * ldv + j]));   // no FMA
            a[(size_t)e * lda + j] = x;
            if (u) u[(size_t)e * ldu + j] = fminf(fmaxf(x, 0.f), 1.f);
            if (X) X[(size_t)e * ldx + off + j] = __float2bfloat16_rn(x);
        }
}

__global__ void k_bump(uint32_t* ctr) { *ctr += 1u; }

// tracking error Delta = [q - q_ref | x_body(q) - x_body(q_ref)]: BF16 network rows (pitch ldx,
// pad columns 0) and, optionally, FP32 rows
__global__ void k_delta(const float* q, const float* qr, int pitch_n, const float* xs, const float* xr, int n, int nb,
                        int n_envs, __nv_bfloat16* X, int ldx, float* D, int ldd) {
    for (int e = blockIdx.x; e < n_envs; e += gridDim.x)
        for (int j = threadIdx.x; j < ldx; j += blockDim.x) {
            float v = 0.f;
            if (j < n) v = q[(size_t)e * pitch_n + j] - qr[(size_t)e * pitch_n + j];
            else if (j < n + 3 * nb) v = xs[(size_t)e * 3 * nb + j - n] - xr[(size_t)e * 3 * nb + j - n];
            X[(size_t)e * ldx + j] = __float2bfloat16_rn(v);
            if (D && j < n + 3 * nb) D[(size_t)e * ldd + j] = v;
        }
}

// r = -log(1 - D(Delta)) + w_power r_power, r_power = -(1/m) sum_k |F_k v_k|; one warp per env
__global__ void k_reward(const float* Dout, int ldo, const float* F, const float* vm, int pitch_m, int m, int n_envs,
                         float w_power, float* r, float* parts) {
    const int warp = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (warp >= n_envs) return;
    float s = 0.f;
    for (int k = lane; k < m; k += 32) s += fabsf(F[(size_t)warp * pitch_m + k] * vm[(size_t)warp * pitch_m + k]);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
        const float d = fminf(Dout[(size_t)warp * ldo], 1.f - 1e-7f);   // keeps the reward finite
        const float rt = -log1pf(-d);
        const float rp = -s / (float)m;
        r[warp] = rt + w_power * rp;
        if (parts) {
            parts[2 * warp] = rt;
            parts[2 * warp + 1] = rp;
        }
    }
}

// one 256-thread block per environment row, at most 8192 blocks (rows loop)
int rows_grid(int n_envs) { return n_envs < 1 ? 1 : (n_envs < 8192 ? n_envs : 8192); }

}  // namespace

cudaError_t launch_flow_init(const float* mu, int ldmu, float* a, int lda, int n_envs, int m, float sigma,
                             uint32_t seed, uint32_t* act_ctr, cudaStream_t s) {
    k_bump<<<1, 1, 0, s>>>(act_ctr);
    k_flow_init<<<rows_grid(n_envs), 256, 0, s>>>(mu, ldmu, a, lda, n_envs, m, sigma, seed,
                                                                           act_ctr);
    return cudaGetLastError();
}

cudaError_t launch_flow_input(const float* a, int lda, int n_envs, int m, float t, __nv_bfloat16* X, int ldx, int off,
                              cudaStream_t s) {
    k_flow_input<<<rows_grid(n_envs), 256, 0, s>>>(a, lda, n_envs, m, t, X, ldx, off);
    return cudaGetLastError();
}

cudaError_t launch_copy_cols(const __nv_bfloat16* src, int lds, int n_envs, int cols, __nv_bfloat16* dst, int ldd,
                             cudaStream_t s) {
    k_copy_cols<<<rows_grid(n_envs), 256, 0, s>>>(src, lds, n_envs, cols, dst, ldd);
    return cudaGetLastError();
}

cudaError_t launch_flow_axpy(float* a, int lda, const float* v, int ldv, int n_envs, int m, float dt, float* u, int ldu,
                             __nv_bfloat16* X, int ldx, int off, float t_next, cudaStream_t s) {
    k_flow_axpy<<<rows_grid(n_envs), 256, 0, s>>>(a, lda, v, ldv, n_envs, m, dt, u, ldu, X, ldx, off, t_next);
    return cudaGetLastError();
}

cudaError_t launch_delta(const float* q, const float* qr, int pitch_n, const float* xs, const float* xr, int n, int nb,
                         int n_envs, __nv_bfloat16* X, int ldx, float* D, int ldd, cudaStream_t s) {
    k_delta<<<rows_grid(n_envs), 256, 0, s>>>(q, qr, pitch_n, xs, xr, n, nb, n_envs, X, ldx, D, ldd);
    return cudaGetLastError();
}

cudaError_t launch_reward(const float* Dout, int ldo, const float* F, const float* vm, int pitch_m, int m, int n_envs,
                          float w_power, float* r, float* parts, cudaStream_t s) {
    k_reward<<<(n_envs + 7) / 8, 256, 0, s>>>(Dout, ldo, F, vm, pitch_m, m, n_envs, w_power, r, parts);
    return cudaGetLastError();
}

cudaError_t launch_obs(const float* q, const float* qd, const float* act, const float* force, const float* inv_fmax,
                       int pitch_n, int pitch_m, int n, int m, int n_envs, __nv_bfloat16* X, int ldx, cudaStream_t s) {
    k_obs<<<rows_grid(n_envs), 256, 0, s>>>(q, qd, act, force, inv_fmax, pitch_n, pitch_m, n, m, n_envs, X, ldx);
    return cudaGetLastError();
}

}  // namespace msim

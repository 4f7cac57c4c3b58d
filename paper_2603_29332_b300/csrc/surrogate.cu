// surrogate.cu -- data kernels of the geometry surrogate's training: box sampling, label
// statistics and normalisation.  The labels themselves come from the step kernel's geometry mode
// and the network from mlp.cu.
#include "surrogate.h"

namespace msim {
namespace {

__global__ void k_sample(float* q, int pitch_n, __nv_bfloat16* X, int ldx, int n_rows, int n, const float* c,
                         const float* s, uint32_t seed, uint64_t row0) {
    const int groups = (ldx + 3) / 4;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < (size_t)n_rows * groups;
         i += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)(i / groups), j0 = 4 * (int)(i % groups);
        const uint64_t row = row0 + r;
        uint32_t ctr[4] = {(uint32_t)row, (uint32_t)(row >> 32), (uint32_t)j0, 0x5a17u};
        philox4x32_10(ctr, seed, 0x3c6ef372u);
        for (int t = 0; t < 4; ++t) {
            const int j = j0 + t;
            if (j >= ldx) break;
            float v = 0.f;
            if (j < n) {
                const float u = 2.f * u01_from_bits(ctr[t]) - 1.f;
                const float qj = c[j] + s[j] * u;
                q[(size_t)r * pitch_n + j] = qj;
                v = (qj - c[j]) / s[j];
            } else if (j < pitch_n) {
                q[(size_t)r * pitch_n + j] = 0.f;
            }
            X[(size_t)r * ldx + j] = __float2bfloat16_rn(v);
        }
    }
}

// block (32, 8): 32 columns, 8 row lanes; grid (column tiles, row chunks)
__global__ void k_col_stats(const float* T, int ldt, int n_rows, int cols, double* acc) {
    __shared__ double s1[8][32], s2[8][32];
    const int col = blockIdx.x * 32 + threadIdx.x;
    double a = 0.0, b = 0.0;
    if (col < cols)
        for (int r = blockIdx.y * 8 + threadIdx.y; r < n_rows; r += gridDim.y * 8) {
            const double v = T[(size_t)r * ldt + col];
            a += v;
            b += v * v;
        }
    s1[threadIdx.y][threadIdx.x] = a;
    s2[threadIdx.y][threadIdx.x] = b;
    __syncthreads();
    if (threadIdx.y == 0 && col < cols) {
        for (int k = 1; k < 8; ++k) {
            a += s1[k][threadIdx.x];
            b += s2[k][threadIdx.x];
        }
        atomicAdd(&acc[2 * col], a);
        atomicAdd(&acc[2 * col + 1], b);
    }
}

__global__ void k_finalize(const double* acc, int cols, int colp, double N, float sd_floor, float* mu, float* sd) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < colp; j += gridDim.x * blockDim.x) {
        if (j < cols) {
            const double mean = acc[2 * j] / N;
            const double var = fmax(acc[2 * j + 1] / N - mean * mean, 0.0);
            mu[j] = (float)mean;
            sd[j] = fmaxf((float)sqrt(var), sd_floor);
        } else {
            mu[j] = 0.f;
            sd[j] = 1.f;
        }
    }
}

__global__ void k_normalize(float* T, int ldt, int64_t n_rows, int cols, const float* mu, const float* sd) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < (size_t)n_rows * ldt;
         i += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)(i % ldt);
        T[i] = j < cols ? (T[i] - mu[j]) / sd[j] : 0.f;
    }
}

__global__ void k_gather_head(const __nv_bfloat16* W3, const float* b3, const float* mu, const float* sd, int hid,
                              const int* head_src, int cols, __nv_bfloat16* W3h, float* b3h, float* scale_h,
                              float* shift_h) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < (size_t)cols * hid;
         i += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)(i / hid), j = (int)(i % hid);
        const int src = head_src[c];
        W3h[i] = src >= 0 ? W3[(size_t)src * hid + j] : __float2bfloat16_rn(0.f);
        if (j == 0) {
            b3h[c] = src >= 0 ? b3[src] : 0.f;
            scale_h[c] = src >= 0 ? sd[src] : 0.f;
            shift_h[c] = src >= 0 ? mu[src] : 0.f;
        }
    }
}

__global__ void k_unpermute(const float* Yh, int ldh, int n_rows, const int* head_src, int cols, float* out, int ldo) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < (size_t)n_rows * cols;
         i += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)(i / cols), c = (int)(i % cols);
        const int src = head_src[c];
        if (src >= 0) out[(size_t)r * ldo + src] = Yh[(size_t)r * ldh + c];
    }
}

int blocks_for(size_t work, int threads) {
    const size_t b = (work + threads - 1) / threads;
    return (int)(b < 8192 ? (b > 0 ? b : 1) : 8192);
}

}  // namespace

cudaError_t surr_sample(float* q, int pitch_n, __nv_bfloat16* X, int ldx, int n_rows, int n, const float* c,
                        const float* s, uint32_t seed, uint64_t row0, cudaStream_t st) {
    if (n_rows <= 0) return cudaSuccess;
    k_sample<<<blocks_for((size_t)n_rows * ((ldx + 3) / 4), 256), 256, 0, st>>>(q, pitch_n, X, ldx, n_rows, n, c, s,
                                                                                  seed, row0);
    return cudaGetLastError();
}

cudaError_t surr_col_stats(const float* T, int ldt, int n_rows, int cols, double* acc, cudaStream_t st) {
    if (n_rows <= 0 || cols <= 0) return cudaSuccess;
    const int chunks = n_rows / 256 + 1 < 64 ? n_rows / 256 + 1 : 64;
    k_col_stats<<<dim3((cols + 31) / 32, chunks), dim3(32, 8), 0, st>>>(T, ldt, n_rows, cols, acc);
    return cudaGetLastError();
}

cudaError_t surr_finalize(const double* acc, int cols, int colp, double N, float sd_floor, float* mu, float* sd,
                          cudaStream_t st) {
    k_finalize<<<blocks_for(colp, 256), 256, 0, st>>>(acc, cols, colp, N, sd_floor, mu, sd);
    return cudaGetLastError();
}

cudaError_t surr_gather_head(const __nv_bfloat16* W3, const float* b3, const float* mu, const float* sd, int hid,
                             const int* head_src, int cols, __nv_bfloat16* W3h, float* b3h, float* scale_h,
                             float* shift_h, cudaStream_t st) {
    k_gather_head<<<blocks_for((size_t)cols * hid, 256), 256, 0, st>>>(W3, b3, mu, sd, hid, head_src, cols, W3h, b3h,
                                                                        scale_h, shift_h);
    return cudaGetLastError();
}

cudaError_t surr_unpermute(const float* Yh, int ldh, int n_rows, const int* head_src, int cols, float* out, int ldo,
                           cudaStream_t st) {
    if (n_rows <= 0) return cudaSuccess;
    k_unpermute<<<blocks_for((size_t)n_rows * cols, 256), 256, 0, st>>>(Yh, ldh, n_rows, head_src, cols, out, ldo);
    return cudaGetLastError();
}

cudaError_t surr_normalize(float* T, int ldt, int64_t n_rows, int cols, const float* mu, const float* sd,
                           cudaStream_t st) {
    if (n_rows <= 0) return cudaSuccess;
    k_normalize<<<blocks_for((size_t)n_rows * ldt, 256), 256, 0, st>>>(T, ldt, n_rows, cols, mu, sd);
    return cudaGetLastError();
}

}  // namespace msim

// surrogate.h -- learned muscle geometry: q -> (L, sparse R) by a 3-layer MLP.
//
// The network reads q normalised to the training box, (q - c) / s in [-1, 1] per DoF, and
// predicts every output normalised by its mean and standard deviation over the training labels;
// outputs are the m muscle lengths (caller's muscle order) followed by the nnz moment-arm entries
// in the library's sparse order (the crossed DoFs of each muscle, msim_get_layout).  Labels come
// from the exact via-point geometry kernel.  In the step, an environment falls back to the exact
// geometry when q leaves the box, or for good after a sampled check exceeds the tolerance.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "mlp.h"

namespace msim {

constexpr int kSurrHidden = 512;
// joint-structured network: first-layer biases spread over each unit's input range at init
constexpr bool kSurrSpreadBias = false;

struct Surrogate {
    int n = 0, m = 0, nnz = 0, out = 0;   // DoFs, muscles, moment-arm entries, outputs m + nnz
    Mlp* net = nullptr;
    float* mu = nullptr;                  // [outp] output means
    float* sd = nullptr;                  // [outp] output standard deviations (floored)
    float* box_c = nullptr;               // [pitch_n] training-box centre
    float* box_s = nullptr;               // [pitch_n] training-box half-width
    __nv_bfloat16* X = nullptr;           // [n_envs][inp] network input of the current substep
    float* Y = nullptr;                   // [n_envs][outp] network output of the current substep
    uint8_t* fallback = nullptr;          // [n_envs] 1: exact geometry until msim_reset
    unsigned long long* stats = nullptr;  // [8] counters (msim_surrogate_stats)
    uint32_t* step_ctr = nullptr;         // device substep counter of the check draw
    float* out_tmp = nullptr;             // [n_envs][outp] network output for msim_surrogate_predict
    uint32_t seed = 0;
    float check_frac = 0.01f, tol = 1e-3f;
    float box_margin = 0.05f;             // box half-width = (1 + margin) x half the limit range
    int trained = 0;
    int structured = 0;                   // 1: joint-block connectivity (msim_surrogate_set_structure)
    float loss = 0.f;                     // mean squared normalised error of the last epoch
};

// q rows [n_rows][pitch_n] drawn uniformly in the box (Philox-4x32-10 keyed by seed, counter =
// global row, DoF group), and the network input X = bf16((q - c) / s) beside them.
cudaError_t surr_sample(float* q, int pitch_n, __nv_bfloat16* X, int ldx, int n_rows, int n, const float* c,
                        const float* s, uint32_t seed, uint64_t row0, cudaStream_t st);
// per-column sums and sums of squares (FP64) of T [n_rows][ldt], first `cols` columns, added to acc
cudaError_t surr_col_stats(const float* T, int ldt, int n_rows, int cols, double* acc, cudaStream_t st);
// mu = mean, sd = max(std, sd_floor) from acc over N rows; columns [cols, colp) get mu 0, sd 1
cudaError_t surr_finalize(const double* acc, int cols, int colp, double N, float sd_floor, float* mu, float* sd,
                          cudaStream_t st);
// out[r][j] = Y[r][j] * sd[j] + mu[j] for j < cols
cudaError_t surr_denorm(const float* Y, int ldy, int n_rows, int cols, const float* mu, const float* sd, float* out,
                        int ldo, cudaStream_t st);
// T = (T - mu) / sd over the first `cols` columns; the pad columns become 0
cudaError_t surr_normalize(float* T, int ldt, int64_t n_rows, int cols, const float* mu, const float* sd,
                           cudaStream_t st);

}  // namespace msim

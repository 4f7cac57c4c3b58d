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
// Each output is normalised by its standard deviation over the labels, floored at this value
// (metres: lengths and moment arms), so the training loss weighs an output's error by
// 1 / max(sd, floor)^2 in physical units.
#ifndef MSIM_SURR_SD_FLOOR
#define MSIM_SURR_SD_FLOOR 1e-4f
#endif
constexpr float kSurrSdFloor = MSIM_SURR_SD_FLOOR;

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
    // inference head in the step kernel's order: output column c = colbase[g] + 32 s + l holds
    // entry s (0 the length, 1.. the moment arms) of muscle record 32 g + l, so that a warp's 32
    // lanes read one contiguous run; head_src[c] = the network output it comes from (-1: padding).
    // Its rows are those of the network's output layer, gathered, with the de-normalisation as the
    // GEMM epilogue's scale (sd) and shift (mu): the values are the network's, in physical units.
    int cols = 0;                         // C, a multiple of 32
    int* colbase = nullptr;               // [record groups]
    int* head_src = nullptr;              // [C]
    __nv_bfloat16* W3h = nullptr;         // [C][hid]
    float* b3h = nullptr;                 // [C]
    float* scale_h = nullptr;             // [C] sd of the source output (0 for padding)
    float* shift_h = nullptr;             // [C] mu of the source output
    uint64_t head_version = ~0ull;        // network version the head was gathered from
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
// the inference head from the network's output layer (rows of W3 [outp][hid] BF16 and b3), mu
// and sd, per head_src (see Surrogate)
cudaError_t surr_gather_head(const __nv_bfloat16* W3, const float* b3, const float* mu, const float* sd, int hid,
                             const int* head_src, int cols, __nv_bfloat16* W3h, float* b3h, float* scale_h,
                             float* shift_h, cudaStream_t st);
// out[r][head_src[c]] = Yh[r][c] for the head's non-padding columns (back to the network's order)
cudaError_t surr_unpermute(const float* Yh, int ldh, int n_rows, const int* head_src, int cols, float* out, int ldo,
                           cudaStream_t st);
// T = (T - mu) / sd over the first `cols` columns; the pad columns become 0
cudaError_t surr_normalize(float* T, int ldt, int64_t n_rows, int cols, const float* mu, const float* sd,
                           cudaStream_t st);

}  // namespace msim

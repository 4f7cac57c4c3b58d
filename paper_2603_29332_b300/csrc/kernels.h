// kernels.h -- launch interface between the C ABI (msim_api.cu) and the device code.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "image.h"

namespace msim {

struct EvalPtrs {                 // per-stage outputs of one substep (msim_eval); any may be null
    float *L, *lm, *vm, *force, *act_next, *R, *tau_m, *tau_c, *tau_l, *bias, *rhs, *qdd, *M, *A;
    int nnz_pitch, packed_pitch;
};

struct StepArgs {
    const uint8_t* img;           // device image of the model (16-byte multiple)
    int staged_bytes;             // prefix copied to shared memory (whole image, or all but the points)
    int points_in_smem;           // 0: path points are read from the global image
    int env_begin, env_end;       // environments of this model
    float* q;                     // state rows (pitch_n / pitch_m)
    float* qd;
    float* act;
    const float* exc;
    int pitch_n, pitch_m;
    float* qdd_out;               // optional: last substep's accelerations
    float* force_out;             // optional: last substep's muscle forces
    uint32_t* env_status;
    uint32_t* gflags;
    int n_sub;
    float dt;
    int envs_per_block;
    int wpe;                      // warps per environment: 1, 2 or 4
    EvalPtrs ev;                  // used by the eval kernel only
    unsigned long long* timers;   // per-phase cycle counters (profiling builds only)
};

// dynamic shared memory of a launch with `epb` environments per block
size_t step_smem_bytes(const ImgHeader& h, int epb, bool points_in_smem, int wpe);
constexpr int kMaxEnvsPerBlock = 16;

cudaError_t launch_step(const StepArgs& a, int grid, size_t smem, cudaStream_t s);
cudaError_t launch_eval(const StepArgs& a, int grid, size_t smem, cudaStream_t s);
cudaError_t launch_set_l0(uint8_t* img, const float* L, int m, cudaStream_t s);
cudaError_t launch_reset(float* q, float* qd, float* act, uint32_t* status, const float* q0, const float* qd0,
                         const float* act0, const int32_t* ids, int n_rows, int pitch_n, int pitch_m, int n_envs,
                         cudaStream_t s);
cudaError_t set_step_smem_limit(size_t bytes);
int step_blocks_per_sm(int threads, size_t smem, int wpe);

}  // namespace msim

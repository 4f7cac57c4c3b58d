// kernels.h -- launch interface between the C ABI (msim_api.cu) and the device code.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "image.h"

namespace msim {

struct EvalPtrs {                 // per-stage outputs of one substep (msim_eval); any may be null
    float *L, *lm, *vm, *force, *act_next, *R, *tau_m, *tau_c, *tau_l, *bias, *rhs, *qdd, *M, *A;
    int nnz_pitch, packed_pitch;
    float* xpos;                  // body-position mode: rows [env][xpos_pitch], body origins x, y, z
    int xpos_pitch;
    float* eps_next;              // eval: tendon strains after the substep (pitch_m)
};

struct StepArgs {
    const uint8_t* img;           // device image of the model (16-byte multiple)
    int staged_bytes;             // prefix copied to shared memory (staged_bytes in image.h)
    int stage;                    // staging level: 1 all, 0 all but via points / cylinders, 2 also
                                  // without muscle records / crossed DoFs (read from the global image)
    int env_begin, env_end;       // environments of this model
    float* q;                     // state rows (pitch_n / pitch_m)
    float* qd;
    float* act;
    float* eps;                   // tendon strains (pitch_m; the eval input rows in eval mode, may
                                  // be null there: zero strain)
    const float* exc;
    int pitch_n, pitch_m;
    float* qdd_out;               // optional: last substep's accelerations
    float* force_out;             // optional: last substep's muscle forces
    float* vm_out;                // optional: last substep's normalised fibre velocities
    uint32_t* env_status;
    uint32_t* gflags;
    int n_sub;
    float dt;
    int envs_per_block;
    int wpe;                      // warps per environment: 1, 2 or 4
    int wrap;                     // 1: the model has wrapping surfaces or compliant tendons (step
                                  // launches take the variant with those branches, uses_ext)
    EvalPtrs ev;                  // eval: per-stage outputs; geometry mode: ev.L = label rows
                                  // [env][ev.nnz_pitch] (L then R), rows from env_begin
    // surrogate step (one substep per launch)
    const float* surr_Y;          // network output rows, row (e - env_begin), pitch surr_ld
    int surr_ld;
    const int* surr_colbase;      // head layout: first column of each group of 32 muscle records
    const float* box_c;           // training box: |q - box_c| <= box_s per DoF
    const float* box_s;
    uint8_t* fallback;            // per environment: 1 = exact geometry until reset
    unsigned long long* surr_stats;
    float check_frac, tol;
    uint32_t surr_seed;
    const uint32_t* step_ctr;     // substep counter of the check draw (advanced by the input kernel)
    unsigned long long* timers;   // per-phase cycle counters (profiling builds only)
};

// dynamic shared memory of a launch with `epb` environments per block
size_t step_smem_bytes(const ImgHeader& h, int epb, int stage, int wpe);
constexpr int kMaxEnvsPerBlock = 16;

cudaError_t launch_step(const StepArgs& a, int grid, size_t smem, cudaStream_t s);
cudaError_t launch_eval(const StepArgs& a, int grid, size_t smem, cudaStream_t s);
// One model of a mixed launch, in queue order.
struct MixedModel {
    const uint8_t* img;
    int staged_bytes;             // bytes of the image staged to shared memory (multiple of 16)
    int stage;                    // staging level (0 or 1 in a mixed launch)
    int env_begin, env_end;
    int epb;                      // environments per work item (<= slots)
    int item_begin;               // first work item of this model
};
// All models in one persistent launch: a.q ... a.gflags, a.n_sub, a.dt and a.wpe are shared;
// a.img / env range / envs_per_block are unused.
struct MixedArgs {
    StepArgs a;
    int n_models;
    MixedModel mdl[kMaxModels];
    int n_items;
    int slots;                    // environment slots per block (threads = 32 wpe slots)
    int img_region;               // shared bytes reserved for the image (max over models, 128-aligned)
    uint32_t* queue;              // work counter (zeroed by launch_mixed before the kernel)
    int wrap;                     // 1: some model has wrapping surfaces or compliant tendons
};
cudaError_t launch_mixed(const MixedArgs& m, int grid, size_t smem, cudaStream_t s);
int mixed_blocks_per_sm(int threads, size_t smem, int wpe, bool wrap);
cudaError_t launch_geom(const StepArgs& a, int grid, size_t smem, cudaStream_t s);
// body origins of the configurations a.q rows [env_begin, env_end) into a.ev.xpos (pitch a.ev.xpos_pitch)
cudaError_t launch_fk(const StepArgs& a, int grid, size_t smem, cudaStream_t s);
cudaError_t launch_surr_step(const StepArgs& a, int grid, size_t smem, cudaStream_t s);
// network input rows X[r] = bf16((q[env_begin + r] - c) / sc), pad columns 0; advances *step_ctr
// (optional) by one
cudaError_t launch_surr_input(const float* q, int pitch_n, int env_begin, int n_envs, const float* c, const float* sc,
                              int n, __nv_bfloat16* X, int ldx, uint32_t* step_ctr, cudaStream_t s);
cudaError_t launch_set_l0(uint8_t* img, const float* L, int m, cudaStream_t s);
// policy observation rows [q | qd | act | force * inv_fmax | 0], BF16, pitch ldx (policy.cu)
cudaError_t launch_obs(const float* q, const float* qd, const float* act, const float* force, const float* inv_fmax,
                       int pitch_n, int pitch_m, int n, int m, int n_envs, __nv_bfloat16* X, int ldx, cudaStream_t s);
// fallback (optional): per-environment surrogate fallback flags, cleared with the state; eps
// (optional): tendon strains, zeroed
cudaError_t launch_reset(float* q, float* qd, float* act, float* eps, uint32_t* status, uint8_t* fallback, const float* q0,
                         const float* qd0, const float* act0, const int32_t* ids, int n_rows, int pitch_n, int pitch_m,
                         int n_envs, cudaStream_t s);
// flow refinement of the policy's action (policy.cu): a = mu + sigma N(0, 1) (advances *act_ctr),
// the per-step input columns [a | t] of the flow network, the observation columns, and the Euler
// step a += dt v (with u = clamp(a, 0, 1) when u is given, and the next step's input columns
// [a | t_next] when X is given)
cudaError_t launch_flow_init(const float* mu, int ldmu, float* a, int lda, int n_envs, int m, float sigma,
                             uint32_t seed, uint32_t* act_ctr, cudaStream_t s);
cudaError_t launch_flow_input(const float* a, int lda, int n_envs, int m, float t, __nv_bfloat16* X, int ldx, int off,
                              cudaStream_t s);
cudaError_t launch_copy_cols(const __nv_bfloat16* src, int lds, int n_envs, int cols, __nv_bfloat16* dst, int ldd,
                             cudaStream_t s);
cudaError_t launch_flow_axpy(float* a, int lda, const float* v, int ldv, int n_envs, int m, float dt, float* u, int ldu,
                             __nv_bfloat16* X, int ldx, int off, float t_next, cudaStream_t s);
// imitation reward (policy.cu): tracking-error rows of the discriminator, then the reward
cudaError_t launch_delta(const float* q, const float* qr, int pitch_n, const float* xs, const float* xr, int n, int nb,
                         int n_envs, __nv_bfloat16* X, int ldx, float* D, int ldd, cudaStream_t s);
cudaError_t launch_reward(const float* Dout, int ldo, const float* F, const float* vm, int pitch_m, int m, int n_envs,
                          float w_power, float* r, float* parts, cudaStream_t s);
cudaError_t set_step_smem_limit(size_t bytes);
int step_blocks_per_sm(int threads, size_t smem, int wpe, bool wrap);

}  // namespace msim

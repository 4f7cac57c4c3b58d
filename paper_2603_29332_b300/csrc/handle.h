// handle.h -- host-side state of a simulator handle, shared by the C-ABI translation units
// (msim_api.cu: create / step / state / learned geometry; tune.cu: mixed launch and autotuner).
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/msim.h"
#include "image.h"
#include "kernels.h"
#include "mlp.h"
#include "surrogate.h"

namespace msim {

struct ModelHost {
    ImgHeader hdr;
    std::vector<uint8_t> blob;
    std::vector<int32_t> dof_parent, dof_depth, packed_row, mus_ptr, mus_dof;
    // joint structure of the muscle geometry (the learned geometry's connectivity): the body
    // owning each crossed DoF (parallel to mus_dof), and per muscle whether every path segment
    // crosses at most one joint (its length then depends on that joint's DoFs alone)
    std::vector<int32_t> mus_body;
    std::vector<uint8_t> mus_one_joint_segments;
};

}  // namespace msim

struct msim_mlp_ {
    msim::Mlp* m = nullptr;
    bool borrowed = false;   // owned by a simulator handle (its surrogate network)
};

struct msim_handle_ {
    int device = 0;
    int geometry_mode = 0;
    uint32_t seed = 0;
    msim::Surrogate* sur = nullptr;
    float box_margin = 0.05f;   // training box of the next msim_surrogate_train
    int surr_hidden = msim::kSurrHidden;   // hidden width of the next msim_surrogate_train
    int surr_structured = 1;               // joint-block connectivity for the next training
    msim_mlp_ sur_view;
    int n_models = 0, n_envs = 0, pitch_n = 0, pitch_m = 0;
    float dt = 0.f;
    int num_sms = 0;
    size_t smem_optin = 0;
    msim::ModelHost models[msim::kMaxModels];
    uint8_t* d_img[msim::kMaxModels] = {};
    int env_begin[msim::kMaxModels + 1] = {};
    // per-model launches
    int epb[msim::kMaxModels] = {};
    int pts_smem[msim::kMaxModels] = {};
    int wpe[msim::kMaxModels] = {};
    // one persistent launch for all models (msim_set_mixed_launch / msim_autotune)
    int mixed = 0;
    int mixed_wpe = 2, mixed_slots = 4;
    int mixed_pts[msim::kMaxModels] = {};
    uint32_t* queue = nullptr;
    // policy in the loop (msim_policy_attach / msim_policy_step)
    msim::Mlp* policy = nullptr;             // borrowed from the caller's msim_mlp
    __nv_bfloat16* obs = nullptr;            // [n_envs][policy in pitch]
    float* exc_policy = nullptr;             // [n_envs][pitch_m] policy output = excitations
    float* inv_fmax = nullptr;               // [pitch_m] 1 / F_max, caller's muscle order
    // flow refinement of the policy's action (msim_flow_attach)
    msim::Mlp* flow = nullptr;               // borrowed: psi(t, s, a), in = obs width + m + 1, out = m
    __nv_bfloat16* flow_x = nullptr;         // [n_envs][flow in pitch]: obs | a | t
    float* flow_a = nullptr;                 // [n_envs][pitch_m] the action being refined
    float* flow_mu = nullptr;                // [n_envs][pitch_m] the initial sampler's mean
    float* flow_v = nullptr;                 // [n_envs][flow out pitch] velocity
    float* flow_pre = nullptr;               // [n_envs][flow hidden] first-layer share of the observation
    int flow_split = 0;                      // its input columns (a multiple of 8; 0: no split)
    uint32_t* act_ctr = nullptr;             // device control-step counter of the noise draw
    // imitation reward (msim_reward_attach / msim_reward)
    msim::Mlp* disc = nullptr;               // borrowed: D(Delta), in = n + 3 nb, out = 1, sigmoid
    float* vm = nullptr;                     // [n_envs][pitch_m] last substep's fibre velocities
    float* xpos_sim = nullptr;               // [n_envs][3 nb]
    float* xpos_ref = nullptr;               // [n_envs][3 nb]
    __nv_bfloat16* delta_x = nullptr;        // [n_envs][disc in pitch]
    float* disc_out = nullptr;               // [n_envs][disc out pitch]
    float w_power = 0.f;
    int flow_steps = 20;
    float flow_dt = 0.05f, flow_sigma = 0.f;
    float *q = nullptr, *qd = nullptr, *act = nullptr, *qdd = nullptr, *force = nullptr, *exc_stage = nullptr;
    float* eps = nullptr;                    // [n_envs][pitch_m] tendon strains (compliant tendons)
    // pipelined host stepping (msim_step_host_async): upload / download streams, two staging
    // slots of excitations and of q | qd, and the events that order them
    cudaStream_t pipe_up = nullptr, pipe_down = nullptr;
    float* pipe_exc[2] = {};
    float* pipe_out[2] = {};
    cudaEvent_t pipe_in[2] = {}, pipe_used[2] = {}, pipe_snap[2] = {}, pipe_done[2] = {};
    int pipe_slot = 0;
    uint32_t* env_status = nullptr;
    uint32_t* gflags = nullptr;
    unsigned long long* timers = nullptr;   // profiling builds (MSIM_PHASE_TIMERS) only
    std::string err;
};

namespace msim {
namespace host {

msim_status cuda_fail(msim_handle h, cudaError_t e, const char* what);
msim_status arg_fail(msim_handle h, const char* what);
bool aligned16(const void* p);
int model_grid(msim_handle h, int i);
StepArgs base_args(msim_handle h, int i);
int max_epb(msim_handle h, int i, int stage, int wpe);
void auto_launch(msim_handle h, int i);
// mixed launch of all models with the handle's mixed_* settings; false if they do not fit
bool mixed_args(msim_handle h, int wpe, int slots, const int* pts, MixedArgs* out, size_t* smem, int* grid);
cudaError_t launch_all(msim_handle h, const float* exc, int n_sub, cudaStream_t s);

}  // namespace host
}  // namespace msim

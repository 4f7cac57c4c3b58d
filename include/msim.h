/*
 * msim.h -- C ABI of the batched muscle-driven forward-dynamics step (one B300, sm_103a).
 *
 * The library steps E independent environments of a muscle-actuated skeleton from neural
 * excitations u in [0,1]^m, following the paper's statement of the problem (Methods,
 * "Musculoskeletal dynamics"): M(q) q_dd + C(q, q_d) = J_m(q)^T F + tau_ext, with
 * Hill-type muscle force F (Eq. 1) and first-order activation dynamics (Eq. 2).
 *
 * Conventions for every entry point:
 *   - Every call returns msim_status; MSIM_OK is 0.  Argument checks are synchronous and
 *     nothing is launched when they fail.  msim_last_error() describes the last failure.
 *   - Unless stated otherwise, array arguments are caller-owned DEVICE pointers (e.g. a
 *     torch CUDA tensor's data_ptr()), FP32, row-major [env][column], rows padded to the
 *     handle's pitches (msim_dims.pitch_n for per-DoF rows, pitch_m for per-muscle rows);
 *     padding columns are ignored on input and left untouched on output.  Pointers must be
 *     16-byte aligned (pitches are multiples of 4 floats).
 *   - Work is enqueued on the given stream (NULL = the legacy default stream) and is
 *     asynchronous; device-side numeric trouble never traps: it sets per-environment status
 *     bits (MSIM_ENV_*) and a global flag read by msim_get_status().
 *   - Environments of model i occupy the contiguous env range
 *     [msim_dims.env_begin[i], msim_dims.env_begin[i+1]) in creation order.
 *   - A handle is used by one host thread at a time.
 */
#ifndef MSIM_H
#define MSIM_H

#include <stddef.h>
#include <stdint.h>

#include "msim_model.h"

#if defined(__GNUC__)
#define MSIM_API __attribute__((visibility("default")))
#else
#define MSIM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct msim_handle_* msim_handle;     /* opaque; owned by the library */
typedef struct CUstream_st* msim_stream_t;    /* a cudaStream_t */

typedef enum {
    MSIM_OK = 0,
    MSIM_ERR_ARG = 1,          /* bad argument (NULL, size, alignment, range) */
    MSIM_ERR_CUDA = 2,         /* a CUDA runtime call failed */
    MSIM_ERR_OOM = 3,          /* device allocation failed */
    MSIM_ERR_MODEL = 4,        /* model description rejected (see msim_last_error) */
    MSIM_ERR_TIMEOUT = 5,      /* a bounded device-side wait gave up */
    MSIM_ERR_STATE = 6,        /* an environment's state went non-finite or its M was not SPD */
    MSIM_ERR_UNSUPPORTED = 7   /* valid request this build does not provide */
} msim_status;

/* per-environment status bits (msim_get_state env_status) and the global flag word */
#define MSIM_ENV_NONFINITE 0x1u  /* q, q_d or act not finite after a call */
#define MSIM_ENV_NOT_SPD 0x2u    /* a pivot of the (M + dt D) factorisation was not positive */
#define MSIM_FLAG_TIMEOUT 0x100u /* a bounded wait (model staging) expired in some block */

typedef struct {
    int32_t n_models;
    const msim_model_desc* models;  /* host array [n_models] */
    const int32_t* envs_per_model;  /* host array [n_models], each >= 0, total >= 1 */
    int32_t geometry_mode;          /* 0 = exact via-point geometry, 1 = learned (msim_set_geometry_mode) */
    float dt;                       /* substep length [s], > 0 */
    uint64_t seed;                  /* reserved for stochastic parts; 0 is fine */
    int32_t device;                 /* CUDA device ordinal */
} msim_create_args;

typedef struct {
    int32_t n_envs, n_models, pitch_n, pitch_m;
    int32_t env_begin[9];           /* first env of each model (n_models + 1 entries used) */
    int32_t n_dofs[8], n_muscles[8], n_bodies[8], nnz[8], n_packed[8], envs_per_block[8];
    int32_t image_bytes[8], workspace_bytes_per_env[8], points_in_smem[8], warps_per_env[8];
    /* points_in_smem: the staging level of msim_set_launch's stage_points (1 whole image in
     * shared memory, 0 via points in global memory, 2 via points and muscle records there) */
} msim_dims;

/* msim_create -- build a simulator for one or more models (<= 8) on one device.
 *   Copies every model description (host memory, caller keeps ownership; nothing is retained),
 *   validates it (MSIM_ERR_MODEL: parent order, DoF counts 1..3 (6 for a free root, without
 *   limits), unit axes, muscle paths that do not follow one ancestor chain, wrapping surfaces
 *   off the wrapped segment's chain or of an unknown kind, sizes above the limits in
 *   msim_model.h), builds the
 *   device model images, computes each muscle's reference length L0 = L(q = 0) on the device
 *   and allocates the state (q, q_d, act all zero).  Synchronises the device before returning.
 *   *out receives the handle, owned by the library until msim_destroy. */
MSIM_API msim_status msim_create(const msim_create_args* args, msim_handle* out);

/* msim_destroy -- free every device buffer of the handle (synchronises). NULL is a no-op. */
MSIM_API msim_status msim_destroy(msim_handle h);

/* msim_get_dims -- sizes and layout of a handle (host struct, filled synchronously). */
MSIM_API msim_status msim_get_dims(msim_handle h, msim_dims* out);

/* msim_reset -- set the state of environments (Eq. 2's act and the generalised coordinates).
 *   q0, qd0: [rows][pitch_n]; act0: [rows][pitch_m] (device).  rows = n_ids if env_ids is
 *   non-NULL (device int32 [n_ids], each in [0, n_envs)), else n_envs.  Any of q0, qd0, act0
 *   may be NULL: that part is set to zero.  Clears the status bits of those environments and
 *   sets their tendon strains to zero (compliant tendons at slack length). */
MSIM_API msim_status msim_reset(msim_handle h, const float* q0, const float* qd0, const float* act0,
                       const int32_t* env_ids, int32_t n_ids, msim_stream_t stream);

/* msim_step -- advance every environment by n_substeps substeps of length dt.
 *   excitations: device [n_envs][pitch_m], held constant over the substeps and clamped to the
 *   action space [0, 1] (Methods, "Action space").  Per substep, for each environment
 *   (Methods, Eq. 1, Eq. 2, equations of motion):
 *     act_dot = (u - act) / tau(u, act);  F = F_max [act f_l(l_m) f_v(v_m) + f_p(l_m)];
 *     (M + dt D) q_dd = R^T F + tau_contact + tau_limits - C;
 *     q_d += dt q_dd;  q += dt q_d;  act = clamp(act + dt act_dot, 0, 1)
 *   where D collects the velocity derivatives of the muscle, contact and joint damping forces
 *   (linearly implicit damping).  A compliant tendon (msim_model.h) replaces F by its tendon
 *   force and advances its strain.  1 <= n_substeps <= 100000.  Asynchronous. */
MSIM_API msim_status msim_step(msim_handle h, const float* excitations, int32_t n_substeps, msim_stream_t stream);

/* msim_step_host -- msim_step from HOST excitations with the resulting q and q_d copied back
 *   to HOST memory: excitations_host [n_envs][pitch_m] is copied to the device, the step runs,
 *   then q_host and qd_host ([n_envs][pitch_n], either may be NULL) receive the new state.
 *   Host buffers should be pinned for full speed.  Synchronises the stream before returning. */
MSIM_API msim_status msim_step_host(msim_handle h, const float* excitations_host, int32_t n_substeps, float* q_host,
                           float* qd_host, msim_stream_t stream);

/* msim_step_host_async -- msim_step_host, pipelined: the call returns once its work is queued.
 *   The excitations go up on the handle's upload stream into one of two device staging buffers,
 *   the step runs on `stream` once they have landed, q and q_d are then copied (device to
 *   device) into one of two output staging buffers and go down on the handle's download stream.
 *   So the copies of one call overlap the steps of its neighbours.  Call t + 2 reuses call t's
 *   staging buffers and waits for call t's copies.  The host buffers must be pinned and left
 *   untouched until msim_host_wait returns; q_host / qd_host (either may be NULL) receive the
 *   state after this call's step, the calls' copies landing in call order. */
MSIM_API msim_status msim_step_host_async(msim_handle h, const float* excitations_host, int32_t n_substeps,
                                          float* q_host, float* qd_host, msim_stream_t stream);
/* msim_host_wait -- block until every copy of the earlier msim_step_host_async calls (up and
 *   down) has landed. */
MSIM_API msim_status msim_host_wait(msim_handle h);

/* msim_get_state -- copy state out (device pointers, any may be NULL):
 *   q, qd, qdd: [n_envs][pitch_n] (qdd: the accelerations of the last substep);
 *   act, muscle_force: [n_envs][pitch_m] (force: F of the last substep, Eq. 1);
 *   env_status: uint32 [n_envs] (MSIM_ENV_* bits). */
MSIM_API msim_status msim_get_state(msim_handle h, float* q, float* qd, float* act, float* qdd, float* muscle_force,
                           uint32_t* env_status, msim_stream_t stream);

/* msim_tendon_strain -- the tendon strain state of compliant tendons (msim_model.h),
 *   [n_envs][pitch_m] rows (device): `set` (if non-NULL) replaces it, then `get` (if non-NULL)
 *   receives it.  Rigid muscles carry zeros.  Asynchronous. */
MSIM_API msim_status msim_tendon_strain(msim_handle h, const float* set, float* get, msim_stream_t stream);

/* msim_get_status -- synchronise the handle's device work and return the global flag word
 *   (OR of all MSIM_ENV_* bits and MSIM_FLAG_*).  Returns MSIM_ERR_STATE if any
 *   environment bit is set, MSIM_ERR_TIMEOUT if a bounded wait expired, else MSIM_OK. */
MSIM_API msim_status msim_get_status(msim_handle h, uint32_t* global_flags);

/* msim_clear_status -- zero the per-environment bits and the global flag (async). */
MSIM_API msim_status msim_clear_status(msim_handle h, msim_stream_t stream);

/* msim_eval -- every intermediate of ONE substep at caller-given states, without touching the
 *   handle's state.  Inputs q, qd [n_envs][pitch_n], act, exc [n_envs][pitch_m] (device).
 *   Outputs (device; any may be NULL), per environment row:
 *     L, lm, vm, force, act_next: [pitch_m]   muscle-tendon length, normalised fibre length
 *                                             and velocity, Hill force (Eq. 1), next activation
 *     R: [nnz_pitch] moment arms -dL/dq in each model's sparse order (msim_get_layout)
 *     tau_m, tau_c, tau_l, bias, rhs, qdd: [pitch_n]   R^T F, contact, limits, C(q, qd),
 *                                             R^T F + tau_c + tau_l - C, solved accelerations
 *     M, A: [packed_pitch] mass matrix and M + dt D in tree-packed order (msim_get_layout)
 *   nnz_pitch and packed_pitch are the row pitches the caller chose (>= each model's nnz /
 *   n_packed, multiples of 4).  Used by tests to compare every stage with a reference. */
typedef struct {
    float *L, *lm, *vm, *force, *act_next, *R, *tau_m, *tau_c, *tau_l, *bias, *rhs, *qdd, *M, *A;
    int32_t nnz_pitch, packed_pitch;
    /* compliant tendons: tendon_strain, an INPUT [n_envs][pitch_m] (NULL: zero strain), and
     * tendon_strain_next [n_envs][pitch_m], the strain after the substep (rigid muscles: the
     * input copied through) */
    const float* tendon_strain;
    float* tendon_strain_next;
} msim_eval_out;
MSIM_API msim_status msim_eval(msim_handle h, const float* q, const float* qd, const float* act, const float* exc,
                      const msim_eval_out* out, msim_stream_t stream);

/* msim_get_layout -- sparse orders of model `model` (host arrays, caller-allocated):
 *   dof_parent[n] (-1 for DoFs of root bodies), dof_depth[n] (number of ancestor DoFs),
 *   packed_row[n]: row d of the tree-packed lower triangle holds entries (d, a_0..a_depth)
 *     where a_k is d's ancestor DoF at depth k (a_depth = d) at packed_row[d] + k;
 *   muscle_dof_ptr[m+1], muscle_dof[nnz]: the DoFs each muscle crosses (root to leaf), the
 *     order of msim_eval's R.  Any pointer may be NULL. */
MSIM_API msim_status msim_get_layout(msim_handle h, int32_t model, int32_t* dof_parent, int32_t* dof_depth,
                            int32_t* packed_row, int32_t* muscle_dof_ptr, int32_t* muscle_dof);

/* msim_set_launch -- launch shape of a model's step kernel (the autotuner's knobs):
 *   warps_per_env in {1, 2, 4} (0 = keep): the warps that work on one environment together;
 *   envs_per_block in [1, 16] (0 = as many as shared memory holds, at most 8; at most 512
 *   threads and 15 environments per block when warps_per_env > 1); stage_points: 1 = copy the
 *   whole model image into shared memory, 0 = leave the via points (and wrapping cylinders) in
 *   global memory (read through the cache) to make room for more environments per block, 2 =
 *   also leave the muscle records and the crossed-DoF table there, -1 = keep.
 *   (0, -1, 0) restores the default.  MSIM_ERR_ARG if shared memory or the thread limit do not
 *   fit.  Results do not depend on the launch shape. */
MSIM_API msim_status msim_set_launch(msim_handle h, int32_t model, int32_t envs_per_block, int32_t stage_points,
                                     int32_t warps_per_env);

/* ---- batching environments of different skeletons ------------------------------------------
 * The paper runs thousands of environments of one model per GPU (Methods, "GPU-accelerated
 * simulation framework"); a handle may hold up to 8 models.  By default msim_step issues one
 * launch per model.  A mixed launch steps every model in ONE persistent launch: blocks take work
 * items (a group of environments of one model for the whole call) from a queue ordered by cost
 * per environment, re-staging a model image only when the next item belongs to another model.
 * Results are identical to the per-model launches for the same warps_per_env.
 *
 * msim_set_mixed_launch -- enable (1) or disable (0).  warps_per_env 1, 2 or 4 (0: 2);
 * slots_per_block = environments per block (0: the largest <= 8 that fits); stage_points_mask bit
 * i = stage model i's whole image in shared memory, else bit 8 + i = leave its muscle records as
 * well as its via points in global memory (staging levels 1, 2, else 0 as in msim_set_launch;
 * -1: as in the per-model setting).
 * MSIM_ERR_ARG if the shape does not fit (threads <= 512, shared memory). */
MSIM_API msim_status msim_set_mixed_launch(msim_handle h, int32_t enable, int32_t warps_per_env,
                                           int32_t slots_per_block, int32_t stage_points_mask);
typedef struct {
    int32_t mixed;                   /* 1: msim_step uses the mixed launch */
    int32_t mixed_warps_per_env, mixed_slots, mixed_stage_points_mask;
    int32_t warps_per_env[8], envs_per_block[8], stage_points[8];   /* per-model launches */
    float ms_per_model;              /* best per-model launches, back to back, one call */
    float ms_mixed;                  /* best mixed launch, one call (0: none fits) */
    int32_t candidates;              /* configurations timed */
    int32_t from_cache;              /* 1: taken from cache_path without timing */
} msim_tune_result;
/* msim_autotune -- synchronous.  Times, on the handle's own environments with n_substeps
 * substeps per call (excitation 0), every per-model launch shape (warps per environment 1/2/4 x
 * environments per block x via points in shared memory or not) and every mixed-launch shape,
 * applies the fastest (per-model shapes always; the mixed launch, timed only when two or more
 * models have environments, if it beats the per-model launches back to back), and restores the
 * state.  cache_path (may be NULL): a text file; a line
 * whose key (models, environment counts, device, n_substeps, library version) matches is applied
 * without timing; otherwise the result is appended.  The result goes to *out (may be NULL). */
MSIM_API msim_status msim_autotune(msim_handle h, const char* cache_path, int32_t n_substeps, msim_tune_result* out);

/* msim_gemm_bf16 -- the tensor-core building block of the learned parts (surrogate, policy):
 *   C = act(A B^T + bias), A [M][K] BF16 with row pitch lda, B [N][K] BF16 with row pitch ldb
 *   (both K-contiguous; pitches multiples of 8 elements, bases 16-byte aligned), accumulated in
 *   FP32 on the tcgen05 tensor cores; C row-major with pitch ldc, FP32 (c_bf16 = 0) or BF16
 *   (c_bf16 = 1); bias optional [N] FP32; act 0 = none, 1 = SiLU, 2 = sigmoid; Z optional BF16
 *   copy of the pre-activation (pitch ldz).  err (optional device uint32) gets bit 0 if a bounded
 *   wait inside the kernel expired.  Device pointers; asynchronous on `stream`.
 *   MSIM_ERR_ARG on bad sizes or alignment, MSIM_ERR_UNSUPPORTED if the driver lacks tensor maps.
 *   The paper has no GEMM of its own; its networks are 3-layer MLPs (Methods, "Training hyperparameters"). */
MSIM_API msim_status msim_gemm_bf16(const void* A, int32_t lda, const void* B, int32_t ldb, const float* bias, void* C,
                                    int32_t ldc, int32_t M, int32_t N, int32_t K, int32_t c_bf16, int32_t act, void* Z,
                                    int32_t ldz, uint32_t* err, msim_stream_t stream);

/* msim_gemm_bf16_mn -- msim_gemm_bf16 with either operand stored MN-contiguous, read by the
 *   tensor cores' transposed operand mode (no transposed copy is made), and an optional FP32
 *   addend: C = act(A B^T + bias + addend).
 *   a_mn = 0: A [M][K], pitch lda >= K;  a_mn = 1: A stored as its transpose [K][M], lda >= M;
 *   b_mn = 0: B [N][K], pitch ldb >= K;  b_mn = 1: B stored as its transpose [K][N], ldb >= N.
 *   So C = dY^T H (a_mn = b_mn = 1, K = rows of dY and H) and C = dY W (b_mn = 1) read the
 *   stored matrices as they are: the weight and input gradients of an MLP layer.
 *   addend (may be NULL): device FP32 [M][ld_add], ld_add >= N, added to the FP32 accumulator
 *   after the bias and before the activation: the product over a subset of K's columns kept from
 *   an earlier call (the flow refinement reuses the observation's share of its first layer this
 *   way).  Pitches, alignment, outputs and errors as msim_gemm_bf16; a_mn, b_mn other than 0 or 1,
 *   or ld_add < N with an addend: MSIM_ERR_ARG. */
MSIM_API msim_status msim_gemm_bf16_mn(const void* A, int32_t lda, int32_t a_mn, const void* B, int32_t ldb,
                                       int32_t b_mn, const float* bias, const float* addend, int32_t ld_add,
                                       void* C, int32_t ldc, int32_t M, int32_t N, int32_t K, int32_t c_bf16,
                                       int32_t act, void* Z, int32_t ldz, uint32_t* err, msim_stream_t stream);

/* ---- 3-layer MLP on the tensor cores (the surrogate's and the policy's network) ----------
 * A network x -> silu(W1 x + b1) -> silu(W2 h1 + b2) -> out(W3 h2 + b3), out = identity or
 * sigmoid (the paper's networks are 3-layer MLPs, Methods, "Training hyperparameters").  BF16 weights and activations,
 * FP32 accumulation, FP32 master weights, gradients and Adam moments (Kingma & Ba 2015), all in
 * one flat FP32 layout (msim_mlp_layout).  Device work is asynchronous on `stream` unless noted. */
typedef struct msim_mlp_* msim_mlp;

/* msim_mlp_create -- allocate a network (in >= 1, hidden a multiple of 8, out >= 1) with scratch
 *   for batches up to max_batch; out_act 0 = identity, 2 = sigmoid; weights Kaiming-uniform
 *   (bound sqrt(6 / fan_in), output layer scaled by out_scale) from a Philox-4x32-10 stream keyed
 *   by seed, biases zero.  Synchronous.  *net owned by the library until msim_mlp_destroy. */
MSIM_API msim_status msim_mlp_create(int32_t in, int32_t hidden, int32_t out, int32_t out_act, int32_t max_batch,
                                     uint64_t seed, float out_scale, msim_mlp* net);
MSIM_API msim_status msim_mlp_destroy(msim_mlp m);
/* msim_mlp_layout -- element offsets of W1 [hidden][in_pitch], b1, W2 [hidden][hidden], b2,
 *   W3 [out_pitch][hidden], b3 in the flat buffers, their total length, and the pitches. */
MSIM_API msim_status msim_mlp_layout(msim_mlp m, int64_t offsets[6], int64_t* n_params, int32_t* in_pitch,
                                     int32_t* out_pitch);
/* msim_mlp_get / msim_mlp_set -- synchronous copy of a flat buffer to / from HOST memory:
 *   which 0 = parameters, 1 = gradients, 2 = Adam first moments, 3 = Adam second moments; n must be
 *   the n_params of msim_mlp_layout.  Setting parameters refreshes the BF16 copies; setting the
 *   moments also sets the Adam step counter to `adam_step` (ignored otherwise). */
MSIM_API msim_status msim_mlp_get(msim_mlp m, int32_t which, float* host, int64_t n);
MSIM_API msim_status msim_mlp_set(msim_mlp m, int32_t which, const float* host, int64_t n, int32_t adam_step);
/* msim_mlp_forward -- Y [B][ldy] FP32 = network(X), X [B][ldx] BF16 (device; ldx >= in_pitch,
 *   a multiple of 8), 1 <= B <= max_batch. */
MSIM_API msim_status msim_mlp_forward(msim_mlp m, const void* X, int32_t ldx, int32_t B, float* Y, int32_t ldy,
                                      msim_stream_t stream);
/* msim_mlp_backward -- gradients of mean((y - t)^2) over the batch and outputs into the gradient
 *   buffer (forward included); T [B][ldt] FP32 device.  If loss is non-NULL the call synchronises
 *   the stream and writes the loss there (host). */
MSIM_API msim_status msim_mlp_backward(msim_mlp m, const void* X, int32_t ldx, const float* T, int32_t ldt, int32_t B,
                                       float* loss, msim_stream_t stream);
/* msim_mlp_adam -- one Adam step from the gradient buffer (bias-corrected, step counter + 1). */
MSIM_API msim_status msim_mlp_adam(msim_mlp m, float lr, float beta1, float beta2, float eps, msim_stream_t stream);

/* ---- learned muscle geometry (surrogate) ---------------------------------------------------
 * The equation of motion (Methods, "Musculoskeletal dynamics") needs the muscle lengths (for l_m,
 * v_m of Eq. 1) and the moment-arm matrix J_m(q) of the muscle paths.  The paper computes them
 * from the paths; a learned map q -> (lengths, moment arms) is this library's option, with no
 * counterpart in the paper, checked against the exact path it replaces.  Single-model handles
 * only (MSIM_ERR_UNSUPPORTED otherwise).  Outputs of
 * msim_geometry / msim_surrogate_predict are rows [L (m, caller's muscle order) | R (nnz, the
 * sparse order of msim_get_layout's muscle_dof)], FP32, pitch ld_out >= m + nnz.
 *
 * msim_surrogate_train -- synchronous.  Draws n_samples configurations uniformly in the training
 * box (each DoF's limit range widened by `margin` half-ranges on both sides, margin 0.05 unless
 * msim_surrogate_set_box says otherwise; +-pi for a DoF without limits), labels
 * them with the exact geometry kernel, normalises every output by its mean and standard deviation,
 * and trains a 3-layer MLP (n -> 512 -> 512 -> m + nnz by default, msim_surrogate_set_width; SiLU,
 * BF16 tensor-core GEMMs with FP32
 * accumulation) for `epochs` passes of n_samples / batch minibatches with Adam (beta 0.9, 0.999,
 * eps 1e-8; learning rate lr with cosine decay to lr / 100).  Randomness from the create seed.
 * Needs about n_samples * (4 (m + nnz) + 2 n) bytes of device memory while it runs (MSIM_ERR_OOM
 * otherwise).  1 <= batch <= 65536, batch <= n_samples, epochs >= 1, lr > 0. */
MSIM_API msim_status msim_surrogate_train(msim_handle h, int64_t n_samples, int32_t epochs, int32_t batch, float lr,
                                          msim_stream_t stream);
/* msim_set_geometry_mode -- 0 exact via-point geometry, 1 learned.  In mode 1 each substep runs
 * the network on every environment's q, then the step kernel uses its outputs except for
 * environments whose q is outside the training box, or that a failed check has flagged (these
 * use the exact geometry).  Each substep, a Philox-4x32-10 draw keyed by the create seed selects a
 * fraction check_frac (default 0.01) of the other environments for a check: they compute both and
 * use the exact one.  The check error of an environment is the larger of the root-mean-square
 * errors of its moment arms (over its nnz entries) and of its muscle-tendon lengths (over its m
 * muscles) against the exact geometry; an error above tol (default 1e-3, i.e. 1 mm), or a
 * non-finite one, flags the environment until its msim_reset.  Mode 1 before
 * msim_surrogate_train: MSIM_ERR_STATE. */
MSIM_API msim_status msim_set_geometry_mode(msim_handle h, int32_t mode);
/* msim_surrogate_set_box -- training-box margin in half-ranges, 0 <= margin <= 10, for the next
 * msim_surrogate_train (the penalty joint limits let states pass the limits, so a box wider than
 * the limits keeps more environments on the network). */
MSIM_API msim_status msim_surrogate_set_box(msim_handle h, float margin);
/* msim_surrogate_set_width -- hidden width of the next msim_surrogate_train's network (default
 * 512; a multiple of 64 in [64, 4096]): accuracy against cost. */
MSIM_API msim_status msim_surrogate_set_width(msim_handle h, int32_t hidden);
/* msim_surrogate_set_structure -- connectivity of the next msim_surrogate_train's network.  1
 * (default): joint blocks.  When every muscle path segment joins points on the same or on
 * adjacent bodies, each length is a sum of one-joint terms and each moment arm R_kd depends on
 * the DoFs of d's joint alone (the structure of J_m(q) in the equation of motion, Methods,
 * "Musculoskeletal dynamics"); the hidden units are then split into one block per joint, in
 * proportion to sqrt(outputs depending on the joint) x (its DoFs)^2 with at least 2 units each, a
 * block reading only its joint's DoFs, the second layer block diagonal, and each output reading
 * the blocks its value depends on.  The network keeps its dense shape and dense GEMMs (masked
 * weights are zeros held by the training); models with a segment spanning several joints, or
 * widths below 2 units per joint, get the dense network.  0: dense network. */
MSIM_API msim_status msim_surrogate_set_structure(msim_handle h, int32_t structured);
/* msim_surrogate_set_check -- check fraction in [0, 1] and tolerance > 0 (metres). */
MSIM_API msim_status msim_surrogate_set_check(msim_handle h, float check_frac, float tol);

typedef struct {
    uint64_t env_substeps;      /* environment-substeps stepped in mode 1 */
    uint64_t learned;           /* ... of which used the network's geometry */
    uint64_t out_of_box;        /* ... of which had q outside the training box */
    uint64_t flagged;           /* ... of which were flagged by an earlier failed check */
    uint64_t checked;           /* ... of which were checked against the exact geometry */
    uint64_t check_failed;      /* ... of which exceeded the tolerance */
    float max_check_error;      /* largest check error seen (metres; msim_set_geometry_mode) */
    float train_loss;           /* mean squared normalised error, last training epoch */
    int32_t flagged_envs;       /* environments flagged now */
    int32_t trained;
    int32_t structured;         /* 1: the trained network has the joint-block connectivity */
    int32_t hidden;             /* its hidden width */
} msim_surrogate_info;
/* msim_surrogate_stats -- synchronises; counters since training or the last reset_counters. */
MSIM_API msim_status msim_surrogate_stats(msim_handle h, msim_surrogate_info* out, int32_t reset_counters);
/* msim_surrogate_network -- the trained network (borrowed: owned by the handle, valid until the
 * next msim_surrogate_train or msim_destroy; msim_mlp_destroy refuses it).  Its parameters can be
 * read and replaced with msim_mlp_get / msim_mlp_set. */
MSIM_API msim_status msim_surrogate_network(msim_handle h, struct msim_mlp_** net);
/* msim_geometry -- exact geometry of model `model` at n_rows configurations q [n_rows][ldq]
 * (device, ldq >= n_dofs) into out [n_rows][ld_out] (device).  Asynchronous. */
MSIM_API msim_status msim_geometry(msim_handle h, int32_t model, const float* q, int32_t ldq, int32_t n_rows,
                                   float* out, int32_t ld_out, msim_stream_t stream);
/* msim_surrogate_predict -- the network's de-normalised geometry at n_rows configurations (same
 * layout as msim_geometry).  Uses the handle's inference buffers: stream-ordered with msim_step. */
MSIM_API msim_status msim_surrogate_predict(msim_handle h, const float* q, int32_t ldq, int32_t n_rows, float* out,
                                            int32_t ld_out, msim_stream_t stream);

/* msim_mlp_forward_noalloc -- Y [B][ldy] FP32 = the 3-layer MLP of msim_mlp_forward at caller-held
 * weights, for callers that cannot allocate device memory.  The paper has no counterpart: it is an
 * entry point of this library.  It allocates nothing (no cudaMalloc / cudaFree, no allocating
 * library call): its hidden activations go to one fixed file-scope device array of
 * MSIM_NOALLOC_MAX_ACT_ELEMS x 2 BF16 values (32 MiB) plus a 256-byte header, so B * hidden must
 * not exceed MSIM_NOALLOC_MAX_ACT_ELEMS (MSIM_ERR_ARG with a message in msim_last_error(NULL)
 * otherwise; split larger batches).  The first call on a device, made with that device current,
 * looks up the array's device address (cudaGetSymbolAddress) once.  With lazy module loading (the
 * CUDA default) that first call may also load this library's device code on that device, and the
 * driver then commits the array's memory: make the first call at start-up, while memory is still
 * available, and before any stream capture; later calls allocate nothing.  Every call on a device
 * shares the array, which keeps the last call's
 * contents; the GEMMs' wait-expiry word in it is cleared by each call.  Calls whose GPU work
 * overlaps (streams not ordered with each other) race on the array.
 *   W1 [hidden][ldw1] BF16 (ldw1 >= in, multiple of 8), b1 [hidden] FP32, W2 [hidden][hidden] BF16,
 *   b2 [hidden] FP32, W3 [out][hidden] BF16, b3 [out] FP32, X [B][ldx] BF16 (ldx >= in, multiple of
 *   8): all device pointers, BF16 ones 16-byte aligned.  out_act 0 identity, 2 sigmoid.
 *   status: optional device word; receives 0, or bit 0 set if a GEMM wait expired (Y invalid).
 * Asynchronous on `stream`; argument checks are synchronous. */
#define MSIM_NOALLOC_MAX_ACT_ELEMS (8u * 1024u * 1024u)
MSIM_API msim_status msim_mlp_forward_noalloc(int32_t in, int32_t hidden, int32_t out, int32_t out_act, const void* W1,
                                              int32_t ldw1, const float* b1, const void* W2, const float* b2,
                                              const void* W3, const float* b3, const void* X, int32_t ldx, int32_t B,
                                              float* Y, int32_t ldy, uint32_t* status, msim_stream_t stream);

/* ---- policy in the loop ----------------------------------------------------------------------
 * The paper's training loop queries the control policy every 10 simulation substeps and keeps
 * simulation and network inference on the GPU with no host round trips (Methods, "GPU-accelerated
 * simulation framework", "Simulation parameters"); its networks are 3-layer MLPs (Methods,
 * "Training hyperparameters").  Single-model handles.
 *
 * msim_policy_attach -- bind a policy network (msim_mlp_create with in >= 2 n + 2 m, out = m,
 * sigmoid output for excitations in [0, 1], max_batch >= the handle's environments; NULL
 * detaches).  Allocates the observation and excitation buffers (synchronous), so that
 * msim_policy_step allocates nothing.  The network stays owned by the caller and must outlive
 * the binding.
 * msim_policy_step -- n_acts control steps: per step, the observation of every environment,
 * [q (n) | qd (n) | act (m) | F / F_max (m) | 0 ...] in BF16, goes through the policy (BF16 tensor
 * cores, FP32 accumulation) to the excitations, then msim_step advances n_substeps_per_act
 * substeps (exact or learned geometry, per msim_set_geometry_mode).  Asynchronous: a whole
 * rollout can be captured in a CUDA graph.
 * msim_policy_excitations -- copy the last excitations [n_envs][pitch_m] (device pointer). */
MSIM_API msim_status msim_policy_attach(msim_handle h, msim_mlp policy);
MSIM_API msim_status msim_policy_step(msim_handle h, int32_t n_substeps_per_act, int32_t n_acts,
                                      msim_stream_t stream);
MSIM_API msim_status msim_policy_excitations(msim_handle h, float* out, msim_stream_t stream);
/* msim_flow_attach -- refine the policy's action with a flow network before each control step
 * (Methods, "Reinforcement learning with flow-based exploration", the action ODE and
 * "Training hyperparameters": N_ODE = 20 Euler steps of dt_ODE = 0.05).  The attached policy
 * becomes the initial sampler: a0 = mu(s) + sigma eps, eps standard normal (Box-Muller on
 * Philox-4x32-10 keyed by the create seed, counter = environment, muscle pair, control step), then
 * n_steps times a <- a + dt psi(t, s, a) with t = 0, dt, ...; excitations u = clamp(a, 0, 1).
 * psi is an msim_mlp with in = (policy in) + m + 1, reading [observation | a | t] in BF16, out = m,
 * max_batch >= the environments.  Allocates its buffers (synchronous); NULL detaches; attaching
 * another policy detaches the flow.  0 <= n_steps <= 1000, dt >= 0, sigma >= 0.
 * msim_flow_actions -- copy the sampler's mean and the last refined action [n_envs][pitch_m]
 * (device pointers, either may be NULL). */
MSIM_API msim_status msim_flow_attach(msim_handle h, msim_mlp flow, int32_t n_steps, float dt, float sigma);
MSIM_API msim_status msim_flow_actions(msim_handle h, float* mu, float* a, msim_stream_t stream);

/* ---- imitation reward -------------------------------------------------------------------------
 * The paper's unified imitation environment (Methods, "Unified imitation environment") turns the
 * tracking error Delta (joint angles and body positions against the reference motion) into the
 * reward r = -log(1 - D(Delta)) with a discriminator D, and "Training regularization" adds the
 * power penalty r_power = -(1/|A|) sum_i |F_m^(i) v_m^(i)| with weight w_power.  Single-model
 * handles.  The discriminator is trained elsewhere; here it is only evaluated.
 *
 * msim_reward_attach -- bind D (msim_mlp with in = n + 3 nb, out = 1, sigmoid output, max_batch
 * >= the environments; NULL detaches) and w_power.  Allocates its buffers (synchronous); from then
 * on every step also stores the last substep's normalised fibre velocities v_m (Eq. 1).
 * msim_reward -- for every environment: Delta = [q - q_ref (n) | x_b(q) - x_b(q_ref) (3 nb, body
 * origins in the world frame, bodies in model order)], D(Delta) on the tensor cores (BF16 input,
 * FP32 accumulation), r = -log(1 - min(D, 1 - 1e-7)) + w_power r_power with F and v_m of the last
 * substep of the last step (0 before the first step).  q_ref: device [n_envs][pitch_n]; reward:
 * device [n_envs]; parts (optional): device [n_envs][2] = (tracking, power) terms; delta
 * (optional): device [n_envs][ld_delta] FP32.  Asynchronous.
 * msim_body_positions -- body origins [n_rows][3 nb] (device) at configurations q [n_rows][ldq]. */
MSIM_API msim_status msim_reward_attach(msim_handle h, msim_mlp disc, float w_power);
MSIM_API msim_status msim_reward(msim_handle h, const float* q_ref, float* reward, float* parts, float* delta,
                                 int32_t ld_delta, msim_stream_t stream);
MSIM_API msim_status msim_body_positions(msim_handle h, const float* q, int32_t ldq, int32_t n_rows, float* xpos,
                                         msim_stream_t stream);

/* msim_measure_fp32_peak -- synchronous FP32 FMA throughput microbenchmark on `device` (8
 * independent FMA chains per thread, 8 blocks of 256 threads per SM, best of three timed
 * launches), in TFLOP/s.  The paper has no counterpart: it is the measured denominator of the
 * step kernel's ALU roofline.  Allocates a small device buffer. */
MSIM_API msim_status msim_measure_fp32_peak(int32_t device, double* tflops);

/* msim_last_error -- text of the last failure on this handle (or of the last failed create
 *   when h is NULL).  Owned by the library, valid until the next call. */
MSIM_API const char* msim_last_error(msim_handle h);

/* msim_version -- ABI version of this library. */
MSIM_API int32_t msim_version(void);

#ifdef __cplusplus
}
#endif
#endif /* MSIM_H */

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
    int32_t geometry_mode;          /* 0 = exact via-point geometry */
    float dt;                       /* substep length [s], > 0 */
    uint64_t seed;                  /* reserved for stochastic parts; 0 is fine */
    int32_t device;                 /* CUDA device ordinal */
} msim_create_args;

typedef struct {
    int32_t n_envs, n_models, pitch_n, pitch_m;
    int32_t env_begin[9];           /* first env of each model (n_models + 1 entries used) */
    int32_t n_dofs[8], n_muscles[8], n_bodies[8], nnz[8], n_packed[8], envs_per_block[8];
    int32_t image_bytes[8], workspace_bytes_per_env[8], points_in_smem[8], warps_per_env[8];
} msim_dims;

/* msim_create -- build a simulator for one or more models (<= 8) on one device.
 *   Copies every model description (host memory, caller keeps ownership; nothing is retained),
 *   validates it (MSIM_ERR_MODEL: parent order, DoF counts 1..3, unit axes, muscle paths that
 *   do not follow one ancestor chain, sizes above the limits in msim_model.h), builds the
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
 *   may be NULL: that part is set to zero.  Clears the status bits of those environments. */
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
 *   (linearly implicit damping).  1 <= n_substeps <= 100000.  Asynchronous. */
MSIM_API msim_status msim_step(msim_handle h, const float* excitations, int32_t n_substeps, msim_stream_t stream);

/* msim_step_host -- msim_step from HOST excitations with the resulting q and q_d copied back
 *   to HOST memory: excitations_host [n_envs][pitch_m] is copied to the device, the step runs,
 *   then q_host and qd_host ([n_envs][pitch_n], either may be NULL) receive the new state.
 *   Host buffers should be pinned for full speed.  Synchronises the stream before returning. */
MSIM_API msim_status msim_step_host(msim_handle h, const float* excitations_host, int32_t n_substeps, float* q_host,
                           float* qd_host, msim_stream_t stream);

/* msim_get_state -- copy state out (device pointers, any may be NULL):
 *   q, qd, qdd: [n_envs][pitch_n] (qdd: the accelerations of the last substep);
 *   act, muscle_force: [n_envs][pitch_m] (force: F of the last substep, Eq. 1);
 *   env_status: uint32 [n_envs] (MSIM_ENV_* bits). */
MSIM_API msim_status msim_get_state(msim_handle h, float* q, float* qd, float* act, float* qdd, float* muscle_force,
                           uint32_t* env_status, msim_stream_t stream);

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
 *   via-point table into shared memory with the rest of the model, 0 = leave it in global memory
 *   (read through the cache) to make room for more environments per block, -1 = keep.
 *   (0, -1, 0) restores the default.  MSIM_ERR_ARG if shared memory or the thread limit do not
 *   fit.  Results do not depend on the launch shape. */
MSIM_API msim_status msim_set_launch(msim_handle h, int32_t model, int32_t envs_per_block, int32_t stage_points,
                                     int32_t warps_per_env);

/* msim_gemm_bf16 -- the tensor-core building block of the learned parts (surrogate, policy):
 *   C = act(A B^T + bias), A [M][K] BF16 with row pitch lda, B [N][K] BF16 with row pitch ldb
 *   (both K-contiguous; pitches multiples of 8 elements, bases 16-byte aligned), accumulated in
 *   FP32 on the tcgen05 tensor cores; C row-major with pitch ldc, FP32 (c_bf16 = 0) or BF16
 *   (c_bf16 = 1); bias optional [N] FP32; act 0 = none, 1 = SiLU, 2 = sigmoid; Z optional BF16
 *   copy of the pre-activation (pitch ldz).  err (optional device uint32) gets bit 0 if a bounded
 *   wait inside the kernel expired.  Device pointers; asynchronous on `stream`.
 *   MSIM_ERR_ARG on bad sizes or alignment, MSIM_ERR_UNSUPPORTED if the driver lacks tensor maps.
 *   The paper has no GEMM of its own; its networks are 3-layer MLPs (Methods). */
MSIM_API msim_status msim_gemm_bf16(const void* A, int32_t lda, const void* B, int32_t ldb, const float* bias, void* C,
                                    int32_t ldc, int32_t M, int32_t N, int32_t K, int32_t c_bf16, int32_t act, void* Z,
                                    int32_t ldz, uint32_t* err, msim_stream_t stream);

/* msim_last_error -- text of the last failure on this handle (or of the last failed create
 *   when h is NULL).  Owned by the library, valid until the next call. */
MSIM_API const char* msim_last_error(msim_handle h);

/* msim_version -- ABI version of this library. */
MSIM_API int32_t msim_version(void);

#ifdef __cplusplus
}
#endif
#endif /* MSIM_H */

// image.h -- flat device image of one model, and the per-environment shared-memory workspace.
//
// The image is one contiguous, 16-byte aligned blob: a header, then fixed-size records and
// small index tables.  A step kernel copies it into shared memory with one bulk copy
// (cp.async.bulk) per block and keeps it resident across substeps and environments.
#pragma once
#include <stdint.h>

namespace msim {

constexpr int kMaxPts = 8;      // path points per muscle
constexpr int kMaxCross = 12;   // DoFs crossed by one muscle
constexpr int kMaxDepth = 63;   // DoF tree depth
constexpr int kMaxModels = 8;
constexpr int kMaxSpheres = 32;
constexpr int kFiStride = 20;   // floats per body in the fi workspace (float-float inertia)

struct alignas(16) BodyRec {    // 64 B
    float off[3];               // joint origin in the parent frame (world for roots)
    float mass;
    float com[3];               // body frame
    int32_t parent;             // -1: world
    float I[6];                 // inertia about the COM, body frame: xx yy zz xy xz yz
    int16_t dof0, ndof;         // hinge DoFs of this body
    int16_t child0, nchild;     // range in the child table
};

struct alignas(16) DofRec {     // 32 B
    float axis[3];              // unit, frame before the hinge
    float lo, hi;               // limits (lo >= hi: none)
    float damp;                 // joint damping
    int32_t row;                // packed row start (lower triangle, ancestors by depth)
    int16_t parent;             // parent DoF (-1: none)
    uint8_t depth;              // number of ancestor DoFs
    uint8_t body;
};

// Muscle records are sorted by (wrapped segment, points, crossed DoFs) so that the 32 muscles a
// warp handles together run the same loop trip counts and take the wrapping branch together;
// `orig` is the muscle's index in the caller's order.
struct alignas(16) MuscleRec {  // 32 B
    float fmax;
    float inv_lopt;             // 1 / l_opt
    float L0;                   // reference length L(q = 0), filled on the device at create
    float inv_vmax;             // 1 / (vmax_per_lopt * l_opt)
    int32_t p0;                 // first path point; point j at p0 + 32 j (the point table holds
                                // the points of each group of 32 records interleaved)
    int32_t x0;                 // first entry in the crossed-DoF table (== offset in sparse R)
    uint8_t np, nx;             // number of points, number of crossed DoFs
    uint8_t dep0;               // depth of the first crossed DoF (the others follow it, +1 each)
    uint8_t wrap;               // 0: none; else 1 + index into the wrap table
    int32_t orig;
};

// Crossed-DoF table entry: dof | body << 8 | packed row << 16.  A muscle's crossed DoFs form
// one contiguous ancestor chain, so entry (d_i, d_j), j <= i, of the packed matrix is at
// row(d_i) + dep0 + j.
// a node of the factorisation's level order (the dorder table): DoF, depth, packed row start
__host__ __device__ inline int node_dof(uint32_t w) { return w & 0xff; }
__host__ __device__ inline int node_depth(uint32_t w) { return (w >> 8) & 0xff; }
__host__ __device__ inline int node_row(uint32_t w) { return w >> 16; }

__host__ __device__ inline int cross_dof(uint32_t c) { return c & 0xff; }
__host__ __device__ inline int cross_body(uint32_t c) { return (c >> 8) & 0xff; }
__host__ __device__ inline int cross_row(uint32_t c) { return c >> 16; }

struct alignas(16) PointRec {   // 16 B
    float pos[3];               // body frame
    int32_t body_cross;         // body | (crossed DoFs at or above this point's body) << 8
};

struct alignas(16) WrapRec {    // 32 B, a muscle's wrapping surface (MuscleRec::wrap = index + 1)
    float center[3];            // body frame
    float radius;
    float axis[3];              // unit, body frame (cylinders; zero for spheres)
    int32_t body_cross;         // body | (crossed DoFs at or above this body) << 8, as PointRec,
                                // | (number of the muscle point that ends the wrapped segment) << 16
                                // | kind << 24 (0 cylinder, 1 sphere)
};

struct alignas(16) TendonRec {  // 16 B, per muscle record (same order) when the model has
                                // compliant tendons
    float inv_eps0;             // 1 / tendon strain at F_max; 0: rigid tendon
    float lopt;                 // optimal fibre length
    float vmax;                 // maximum fibre velocity (vmax_per_lopt l_opt)
    float pad;
};

struct alignas(16) SphereRec {  // 32 B
    float pos[3];
    float radius;
    int32_t body;
    int32_t last_dof;           // the DoF whose frame carries the sphere
    int32_t pad[2];
};

struct alignas(16) ImgHeader {
    int32_t n, m, nb, np, ns;
    int32_t n_packed;           // sum over DoFs of (depth + 1)
    int32_t nnz;                // crossed-DoF entries of all muscles (non-zeros of R)
    int32_t n_blevels, n_dlevels, max_depth, n_tri, total_bytes;
    // byte offsets of the sections
    int32_t o_body, o_dof, o_muscle, o_sphere, o_cross, o_border, o_blevel, o_child, o_anc, o_dorder, o_dlevel,
        o_tri, o_point, o_rowanc, o_crba, o_wrap;
    // per-environment workspace layout (float offsets inside the environment's slot)
    int32_t w_q, w_qd, w_frame, w_v, w_fi, w_S, w_A, w_rhs, w_racc, w_y, w_sph, w_rk,
        max_nx,                 // most DoFs one muscle crosses (rows of the moment-arm region)
        w_f,                    // body forces (inside the A region, kinematics to subtree sums)
        n_tendons,              // compliant tendons (0: none, and no tendon table)
        o_tendon;               // byte offset of the tendon table (after the wrapping surfaces)
    float gravity[3];
    float contact_k, contact_c, contact_mu, contact_eps2;
    float limit_k, limit_c, tau_act, tau_deact;
    float fp_den;               // exp(4) - 1 of the passive curve
    float fp_slope;             // slope of the passive curve's linear extension
    int32_t free_root;          // 1: body 0 has the six free DoFs 0-5 (msim_model.h)
    int32_t n_wraps;            // wrapping cylinders (their records follow the via points)
    float ft_den;               // e^3 - 4 of the tendon curve's toe
    float ft_slope;             // slope of the tendon curve's linear part (per unit eps / eps0)
    // body chains (maximal runs of single-child bodies) for the subtree sums: at o_chain,
    // int16 round starts [n_crounds + 1] (indices into the chains, a round's chains hang only
    // below chains of earlier rounds), int16 chain starts [n_chains + 1] (indices into the body
    // list), uint8 bodies [nb] (each chain bottom to top)
    int32_t o_chain, n_crounds, n_chains;
    float limit_delta;          // onset width of the joint-limit penalty (msim_model.h)
};

// Models with wrapping surfaces or compliant tendons take the step variants that compile those
// branches in.
__host__ __device__ inline bool uses_ext(const ImgHeader& h) { return h.n_wraps > 0 || h.n_tendons > 0; }

// Per environment workspace (floats), laid out by the host (msim_api.cu).  Regions whose
// lifetimes do not overlap share storage, so that more environments fit a block:
//   q[n], qd[n]                       state, resident across substeps (act stays in global memory)
//   frame[nb][12]                     body rotation (9, row-major) and origin (3), world
//   fi[nb][20]                        spatial inertia about the world origin (m, h, Ibar) as 10
//                                     float-float pairs, summed over subtrees in place
//   S[n][6]                           joint motion axis [s; o x s]
//   A[max(n_packed, 12 nb)][2]        packed M + dt D as float-float (hi, lo) pairs, factorised in
//                                     place.  Before that it holds, during the kinematics pass and
//                                     the subtree sums, the bias accelerations a[nb][6] and the
//                                     spatial velocities v[nb][6] = [w; v_O] (w_v), FP32, and the
//                                     body forces f[nb][6] = [n; f] (w_f, float-float, summed over
//                                     subtrees);
//                                     then the damping sums dt D as fixed-point int32 pairs (see
//                                     fx_red) until the mass matrix is added
//   rhs[n]                            tau_l (FP32)
//   racc[n][2]                        -C + R^T F + tau_c as fixed-point int32 pairs; the
//                                     float-float solution y of the triangular solves replaces it
//                                     (w_y)
//   rk[max(max_nx 32 wpe, 2 n, 12 ns)] per-lane moment arms of the muscle being processed (last);
//                                     sin, cos of the joint angles during the kinematics pass;
//                                     per-sphere contact point, force, damping, flags during the
//                                     contact pass (w_sph)

// Bytes of the image a block copies to shared memory at staging level `stage`: 1 = all of it;
// 0 = all but the via points, wrapping surfaces and tendon table (read through the cache); 2 =
// also without the muscle records and the crossed-DoF table (the image places these five
// sections last, in this order: muscles, crossed DoFs, via points, wrapping surfaces, tendons).
__host__ __device__ inline int staged_bytes(const ImgHeader& h, int stage) {
    return stage == 1 ? h.total_bytes : (stage == 2 ? h.o_muscle : h.o_point);
}

// floats per environment slot for a group of `wpe` warps per environment (the moment-arm
// region also holds the joint sines and cosines, and the contact scratch); a multiple of 4, so
// that every slot, and every region in it, starts on a 16-byte boundary
__host__ __device__ inline int ws_floats(const ImgHeader& h, int wpe) {
    int r = h.max_nx * 32 * wpe;
    if (2 * h.n > r) r = 2 * h.n;
    if (12 * h.ns > r) r = 12 * h.ns;
    return (h.w_rk + r + 3) & ~3;
}

}  // namespace msim

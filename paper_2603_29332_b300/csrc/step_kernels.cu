// step_kernels.cu -- the batched muscle-driven forward-dynamics substep on sm_103a.
//
// Mapping: a group of WPE warps (1, 2 or 4) per environment, several environments per block
// sharing one copy of the model image in shared memory (staged by cp.async.bulk + mbarrier,
// kept resident across all substeps and all environments the block processes).  A group
// synchronises on its own named barrier.  Blocks are persistent: each loops over groups of
// environments.  Per substep and environment (paper, Methods: Eq. 1, Eq. 2 and the
// generalised-coordinate equations of motion):
//   1. kinematics, top-down over body levels: frames, joint axes S, spatial velocities, bias
//      accelerations (gravity as a base acceleration), body forces f = I a + v x* I v and
//      spatial inertias, all in world Plücker coordinates so that subtree sums need no
//      transforms;
//   2. bottom-up over body levels: subtree sums of forces and inertias; rhs = -C = -S^T f;
//   3. CRBA: M(d, a) = S_a^T (I^c_d S_d) for every DoF and each of its ancestors (tree-packed),
//      added to the damping terms of steps 4-5, which run before it;
// Precision: kinematics, forces, muscles and contact in FP32; the parallel-axis terms of the
// inertias, their subtree sums, the entries of M and the factorisation / solves in float-float
// (dfloat.cuh).  FP32 geometry perturbs the mechanism consistently and costs ~1e-6 in q_dd,
// but independent FP32 rounding of the entries of the ill-conditioned M costs up to ~1e-3.
//   4. muscles, one lane per muscle: via-point lengths, moment arms R = -dL/dq of the crossed
//      DoFs, Hill force (Eq. 1), activation update (Eq. 2), rhs += R^T F and
//      A += dt R^T (dF/dLdot) R (linearly implicit force-velocity damping);
//   5. penalty ground contact with smoothed Coulomb friction, rhs += J^T F, A += dt J^T D J;
//   6. joint-limit penalty (linearly implicit in position and velocity) and joint damping;
//   7. tree-sparse factorisation A = L^T L (no fill-in), leaves first, by DoF depth levels;
//   8. solves L^T y = rhs (leaves first) and L qdd = y (root first);
//   9. semi-implicit Euler.
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "dfloat.cuh"
#include "image.h"
#include "kernels.h"
#include "mlp.h"

namespace msim {

namespace {

// kernel modes: one substep loop, one-substep evaluation with every intermediate, muscle
// geometry only (surrogate training labels), surrogate step (geometry from the learned model)
// kModeStepW / kModeSurrW: the step and the learned-geometry substep with the wrapping-surface
// and compliant-tendon branches compiled in (models that have either); kModeStep and kModeSurr
// leave them out (so that the two stay alike instruction for instruction, their exact geometry
// agrees bit for bit); the other modes always keep them.
constexpr int kModeStep = 0, kModeEval = 1, kModeGeom = 2, kModeSurr = 3, kModeFk = 4, kModeStepW = 5,
              kModeSurrW = 6;
__host__ __device__ constexpr bool is_surr(int mode) { return mode == kModeSurr || mode == kModeSurrW; }
__host__ __device__ constexpr bool has_ext(int mode) { return mode != kModeStep && mode != kModeSurr; }

constexpr uint32_t kEnvNonFinite = 0x1u;
constexpr uint32_t kEnvNotSpd = 0x2u;
constexpr uint32_t kFlagTimeout = 0x100u;
constexpr long long kWaitLimit = 1LL << 22;   // bounded mbarrier wait (iterations of try_wait)

// Views of the workspace regions, the image tables and the environment's global rows.  In the
// normal build a view is the raw pointer.  Built with -DMSIM_BOUNDS_CHECK (the stand-in for a
// memory checker: compute-sanitizer is not used), every index through a view is checked against
// the extent of its region, table or row; an index outside it is recorded (count, and site =
// source line, index and extent of the first one) and replaced by 0, so the access itself stays
// in bounds and the run goes on.  The host reads the record with msim_debug_bounds.
#ifdef MSIM_BOUNDS_CHECK
__device__ unsigned int g_bounds_rec[4];   // hits, first site, first index, first extent

__device__ __noinline__ void bounds_hit(int site, long long i, int n) {
    if (atomicAdd(&g_bounds_rec[0], 1u) == 0u) {
        g_bounds_rec[1] = (unsigned)site;
        g_bounds_rec[2] = (unsigned)i;
        g_bounds_rec[3] = (unsigned)n;
    }
}

template <class T>
struct View {
    T* p;
    int n;      // elements in range
    int site;   // source line that made the view
    template <class I>
    __device__ __forceinline__ T& operator[](I i) const {
        long long k = (long long)i;
        if (k < 0 || k >= n) {
            bounds_hit(site, k, n);
            k = 0;
        }
        return p[k];
    }
    template <class I>
    __device__ __forceinline__ View operator+(I i) const {
        long long k = (long long)i;
        if (k < 0 || k > n) {
            bounds_hit(site, k, n);
            k = 0;
        }
        return View{p + k, n - (int)k, site};
    }
    __device__ __forceinline__ operator T*() const { return p; }
};
#define VIEW_T(T) View<T>
template <class T>
__device__ __forceinline__ View<T> mkview(T* p, int n, int site) {
    return View<T>{p, n, site};
}
#else
#define VIEW_T(T) T*
template <class T>
__device__ __forceinline__ T* mkview(T* p, int, int) {
    return p;
}
#endif

// the raw pointer of a view (or of a pointer)
template <class T>
__device__ __forceinline__ T* raw(T* p) { return p; }
#ifdef MSIM_BOUNDS_CHECK
template <class T>
__device__ __forceinline__ T* raw(const View<T>& v) { return v.p; }
#endif

#ifdef MSIM_BOUNDS_CHECK
// end (float offset) of the workspace region holding float offset `off`: the regions are laid
// out q, qd, frame, fi, S, A, rhs, racc, rk (msim_api.cu), the last sized by the warps per env
__device__ __forceinline__ int ws_region_end(const ImgHeader& H, int off, int wpe) {
    const int ends[8] = {H.w_qd, H.w_frame, H.w_fi, H.w_S, H.w_A, H.w_rhs, H.w_racc, H.w_rk};
    for (int i = 0; i < 8; ++i)
        if (off < ends[i]) return ends[i];
    return ws_floats(H, wpe);
}
#endif

// view of the workspace from float offset `off` to the end of its region, as elements of T
#ifdef MSIM_BOUNDS_CHECK
#define WS(T, off) mkview(reinterpret_cast<T*>(ws + (off)), \
                          (int)((ws_region_end(H, (off), WPE) - (off)) * sizeof(float) / sizeof(T)), __LINE__)
#else
#define WS(T, off) reinterpret_cast<T*>(ws + (off))
#endif

struct Tables {
    const ImgHeader* H;
    VIEW_T(const BodyRec) body;
    VIEW_T(const DofRec) dof;
    VIEW_T(const MuscleRec) mus;
    VIEW_T(const PointRec) pt;
    VIEW_T(const WrapRec) wrap;
    VIEW_T(const SphereRec) sph;
    VIEW_T(const uint32_t) cross;
    VIEW_T(const uint8_t) border;
    VIEW_T(const int16_t) blevel;
    VIEW_T(const uint8_t) child;
    VIEW_T(const uint8_t) anc;
    VIEW_T(const uint32_t) dorder;     // factorisation nodes by level (node_dof / node_depth / node_row)
    VIEW_T(const int16_t) dlevel;
    VIEW_T(const uint16_t) tri;
    VIEW_T(const uint16_t) rowanc;
    VIEW_T(const uint2) crba_order;    // CRBA rows, longest first: {DoF | body << 8 | depth << 16, packed row}
    VIEW_T(const TendonRec) ten;       // null: every tendon rigid
    VIEW_T(const int16_t) cround;      // body chains of the subtree sums (ImgHeader::o_chain)
    VIEW_T(const int16_t) cstart;
    VIEW_T(const uint8_t) cbody;
};

#ifdef MSIM_BOUNDS_CHECK
// byte extent of the image section starting at byte offset `o`: up to the next section's start
// (the sections are placed in the order of msim_api.cu's image builder) or the image's end
__device__ __forceinline__ int img_section_end(const ImgHeader& h, int o) {
    const int starts[18] = {h.o_body, h.o_dof, h.o_sphere, h.o_border, h.o_blevel, h.o_child, h.o_anc,
                            h.o_dorder, h.o_dlevel, h.o_chain, h.o_tri, h.o_rowanc, h.o_crba, h.o_muscle,
                            h.o_cross, h.o_point, h.o_wrap, h.n_tendons ? h.o_tendon : h.total_bytes};
    int e = h.total_bytes;
    for (int i = 0; i < 18; ++i)
        if (starts[i] > o && starts[i] < e) e = starts[i];
    return e;
}
#endif

// view of the table of type T at byte offset o of an image (staged in shared memory or global)
#ifdef MSIM_BOUNDS_CHECK
#define TAB(T, base, o) mkview(reinterpret_cast<T*>((base) + (o)), \
                               (int)((img_section_end(h, (o)) - (o)) / (int)sizeof(T)), __LINE__)
#else
#define TAB(T, base, o) reinterpret_cast<T*>((base) + (o))
#endif

__device__ __forceinline__ Tables make_tables(const uint8_t* img) {
    Tables t;
    t.H = reinterpret_cast<const ImgHeader*>(img);
    const ImgHeader& h = *t.H;
    t.body = TAB(const BodyRec, img, h.o_body);
    t.dof = TAB(const DofRec, img, h.o_dof);
    t.mus = TAB(const MuscleRec, img, h.o_muscle);
    t.pt = TAB(const PointRec, img, h.o_point);
    t.wrap = TAB(const WrapRec, img, h.o_wrap);
    t.sph = TAB(const SphereRec, img, h.o_sphere);
    t.cross = TAB(const uint32_t, img, h.o_cross);
    t.border = TAB(const uint8_t, img, h.o_border);
    t.blevel = TAB(const int16_t, img, h.o_blevel);
    t.child = TAB(const uint8_t, img, h.o_child);
    t.anc = TAB(const uint8_t, img, h.o_anc);
    t.dorder = TAB(const uint32_t, img, h.o_dorder);
    t.dlevel = TAB(const int16_t, img, h.o_dlevel);
    t.tri = TAB(const uint16_t, img, h.o_tri);
    t.rowanc = TAB(const uint16_t, img, h.o_rowanc);
    t.crba_order = TAB(const uint2, img, h.o_crba);
#ifdef MSIM_BOUNDS_CHECK
    t.ten = h.n_tendons ? TAB(const TendonRec, img, h.o_tendon) : mkview<const TendonRec>(nullptr, 0, __LINE__);
#else
    t.ten = h.n_tendons ? reinterpret_cast<const TendonRec*>(img + h.o_tendon) : nullptr;
#endif
    // the chain section holds three arrays: round starts, chain starts, bodies
    const int16_t* cr = reinterpret_cast<const int16_t*>(img + h.o_chain);
    const int16_t* cs = cr + h.n_crounds + 1;
    t.cround = mkview(cr, h.n_crounds + 1, __LINE__);
    t.cstart = mkview(cs, h.n_chains + 1, __LINE__);
    t.cbody = mkview(reinterpret_cast<const uint8_t*>(cs + h.n_chains + 1), h.nb, __LINE__);
    return t;
}

// Sections left out of the staged prefix are read from the image in global memory.
__device__ __forceinline__ void unstaged_tables(Tables& T, const uint8_t* gimg, int stage) {
    if (stage == 1) return;
    const ImgHeader& h = *T.H;
    T.pt = TAB(const PointRec, gimg, h.o_point);
    T.wrap = TAB(const WrapRec, gimg, h.o_wrap);
    if (h.n_tendons) T.ten = TAB(const TendonRec, gimg, h.o_tendon);
    if (stage == 2) {
        T.mus = TAB(const MuscleRec, gimg, h.o_muscle);
        T.cross = TAB(const uint32_t, gimg, h.o_cross);
    }
}

__device__ __forceinline__ void cross3(const float a[3], const float b[3], float c[3]) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}
__device__ __forceinline__ float dot3(const float a[3], const float b[3]) {
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}
// A body frame in the workspace is 12 floats, 16-byte aligned: the rotation row-major, then the
// origin.  Read and written as three 16-byte words: lanes working on different bodies then meet
// in shared memory as 16-byte accesses (a quarter-warp per wavefront) rather than as twelve
// 4-byte accesses spread over only eight banks by the 12-float stride.
__device__ __forceinline__ void frame_load(const float* f, float R[9], float p[3]) {
    const float4 a = reinterpret_cast<const float4*>(f)[0];
    const float4 b = reinterpret_cast<const float4*>(f)[1];
    const float4 c = reinterpret_cast<const float4*>(f)[2];
    R[0] = a.x; R[1] = a.y; R[2] = a.z; R[3] = a.w;
    R[4] = b.x; R[5] = b.y; R[6] = b.z; R[7] = b.w;
    R[8] = c.x; p[0] = c.y; p[1] = c.z; p[2] = c.w;
}
// the origin alone: the last 16-byte word (R22, origin)
__device__ __forceinline__ void frame_origin(const float* f, float p[3]) {
    const float4 c = reinterpret_cast<const float4*>(f)[2];
    p[0] = c.y; p[1] = c.z; p[2] = c.w;
}
__device__ __forceinline__ void frame_store(float* f, const float R[9], const float p[3]) {
    reinterpret_cast<float4*>(f)[0] = make_float4(R[0], R[1], R[2], R[3]);
    reinterpret_cast<float4*>(f)[1] = make_float4(R[4], R[5], R[6], R[7]);
    reinterpret_cast<float4*>(f)[2] = make_float4(R[8], p[0], p[1], p[2]);
}

// out = R v (R row-major 3x3)
__device__ __forceinline__ void rot3(const float* R, const float v[3], float out[3]) {
    out[0] = R[0] * v[0] + R[1] * v[1] + R[2] * v[2];
    out[1] = R[3] * v[0] + R[4] * v[1] + R[5] * v[2];
    out[2] = R[6] * v[0] + R[7] * v[1] + R[8] * v[2];
}

// Profiling builds (MSIM_PHASE_TIMERS): lane 0 adds cycles since the previous mark to a slot.
#ifdef MSIM_PHASE_TIMERS
#define SUB_T0() long long st0_ = clock64()
#define SUB_MARK(i)                                                                               \
    do {                                                                                          \
        const long long t_ = clock64();                                                           \
        if (g.lane == 0 && g_timers) atomicAdd(&g_timers[(i)], (unsigned long long)(t_ - st0_));   \
        st0_ = clock64();                                                                         \
    } while (0)
__device__ unsigned long long* g_timers = nullptr;
#else
#define SUB_T0() \
    do {         \
    } while (0)
#define SUB_MARK(i) \
    do {            \
    } while (0)
#endif

// The threads working on one environment: WPE warps, N = 32 WPE lanes, synchronised on named
// barrier `bar` (one per environment slot of the block; id 0 is __syncthreads).
template <int WPE>
struct Grp {
    static constexpr int N = 32 * WPE;
    int lane;   // 0 .. N-1
    int wl;     // lane within the warp
    int wi;     // warp within the group
    int bar;
    __device__ __forceinline__ void sync() const {
        if (WPE == 1) __syncwarp();
        else asm volatile("bar.sync %0, %1;" ::"r"(bar), "n"(N) : "memory");
    }
    __device__ __forceinline__ bool all(bool v) const {
        if (WPE == 1) return __all_sync(0xffffffffu, v);
        uint32_t r;
        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %1, 0;\n\tbar.red.and.pred p, %2, %3, p;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(r) : "r"((uint32_t)v), "r"(bar), "n"(N) : "memory");
        return r != 0;
    }
    __device__ __forceinline__ bool any(bool v) const {
        if (WPE == 1) return __any_sync(0xffffffffu, v);
        uint32_t r;
        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %1, 0;\n\tbar.red.or.pred p, %2, %3, p;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(r) : "r"((uint32_t)v), "r"(bar), "n"(N) : "memory");
        return r != 0;
    }
};

// Exact, order-independent accumulation in shared memory with native 32-bit integer reductions
// (shared-memory float atomics are emulated with compare-and-swap loops and serialise under
// contention).  A value v is split into a coarse word round(v 2^8) and a fine word holding the
// remainder at 2^-28; each word is reduced with red.shared.add.u32.  Range +-8e6, resolution
// 3.7e-9, exact sums for up to 2^12 contributions per target.
constexpr float kFxCoarse = 256.f;          // 2^8
constexpr float kFxInvCoarse = 1.f / 256.f;
constexpr float kFxFine = 268435456.f;      // 2^28
constexpr float kFxInvFine = 1.f / 268435456.f;

__device__ __forceinline__ void red_add_i32(int32_t* p, int32_t v) {
    asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(static_cast<uint32_t>(__cvta_generic_to_shared(p))), "r"(v));
}
__device__ __forceinline__ void fx_red(int32_t* acc2, float v) {
    const int32_t hi = __float2int_rn(v * kFxCoarse);
    const float rem = fmaf(-static_cast<float>(hi), kFxInvCoarse, v);
    const int32_t lo = __float2int_rn(rem * kFxFine);
    red_add_i32(acc2, hi);
    red_add_i32(acc2 + 1, lo);
}
// the fixed-point pair of a float-float value (plain store: the accumulator's first term)
__device__ __forceinline__ void fx_store(int32_t* acc2, df v) {
    const int32_t hi = __float2int_rn(v.hi * kFxCoarse);
    const float rem = fmaf(-static_cast<float>(hi), kFxInvCoarse, v.hi) + v.lo;
    acc2[0] = hi;
    acc2[1] = __float2int_rn(rem * kFxFine);
}
__device__ __forceinline__ df df_from_i32(int32_t x) {
    const float f = __int2float_rn(x);
    const long long r = static_cast<long long>(x) - __float2ll_rn(f);
    return {f, static_cast<float>(r)};
}
__device__ __forceinline__ df fx_decode(int32_t hi, int32_t lo) {
    const df a = df_from_i32(hi), b = df_from_i32(lo);
    return df_add({a.hi * kFxInvCoarse, a.lo * kFxInvCoarse}, {b.hi * kFxInvFine, b.lo * kFxInvFine});
}

// ------------------------------------------------------------------ bulk staging of the image
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ bool mbar_wait(uint32_t mbar, uint32_t phase) {
    for (long long i = 0; i < kWaitLimit; ++i) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(mbar), "r"(phase)
            : "memory");
        if (done) return true;
    }
    return false;
}

// Copies `bytes` (multiple of 16) from global `src` to shared `dst` with bulk async copies
// completing on one mbarrier.  Every thread of the block must call it.  Returns false (and
// sets the timeout flag) if the bounded wait expired.
__device__ bool stage_image(uint8_t* dst, const uint8_t* src, int bytes, uint64_t* bar, uint32_t* gflags) {
    const uint32_t mb = smem_u32(bar);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb), "r"(bytes) : "memory");
        const uint32_t d = smem_u32(dst);
        constexpr int kChunk = 32768;
        for (int off = 0; off < bytes; off += kChunk) {
            const int sz = (bytes - off) < kChunk ? (bytes - off) : kChunk;
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                    d + off),
                "l"(src + off), "r"(sz), "r"(mb)
                : "memory");
        }
    }
    bool ok = mbar_wait(mb, 0);
    if (!ok) {
        if (threadIdx.x == 0) atomicOr(gflags, kFlagTimeout);
        mbar_wait(mb, 0);   // give copies still in flight a second bounded chance to land
    }
    return __syncthreads_and(ok) != 0;   // one outcome for the whole block
}

// ------------------------------------------------------------------ phase 1: kinematics
template <int WPE>
__device__ void phase_kinematics(const Tables& T, float* ws, const Grp<WPE>& g) {
    const ImgHeader& H = *T.H;
    auto q = WS(const float, H.w_q);
    auto qd = WS(const float, H.w_qd);
    auto frame = WS(float, H.w_frame);
    auto V = WS(float, H.w_v);     // in the A region during this pass (with Acc and FB)
    auto FI = WS(float, H.w_fi);
    auto FB = WS(df, H.w_f);
    auto S = WS(float, H.w_S);
    auto Acc = WS(float, H.w_A);   // bias accelerations live in the A region during this pass
    auto SC = WS(float, H.w_rk);   // sin, cos of every joint angle (the moment-arm scratch is free here)
    SUB_T0();
    // 1. joint-angle sines and cosines, all DoFs in parallel (off the level-by-level chain)
    for (int d = g.lane; d < H.n; d += g.N) sincosf(q[d], &SC[2 * d], &SC[2 * d + 1]);
    g.sync();
    // 2. frames, velocities and bias accelerations: one lane per body walks the DoF chain from
    // the root to the body's last DoF (the ancestor table of that DoF's packed row) in
    // registers, entering each body on the way at its joint origin.  A lane repeats its
    // ancestors' steps in the same order as their own lanes, so every body gets the values of a
    // root-first recursion, bit for bit, without a barrier per tree level.
    for (int b = g.lane; b < H.nb; b += g.N) {
        const BodyRec& Bb = T.body[b];
        const DofRec& Dl = T.dof[Bb.dof0 + Bb.ndof - 1];
        float R[9], p[3], w[3], vl[3], aw[3], al[3];
#pragma unroll
        for (int k = 0; k < 9; ++k) R[k] = (k % 4 == 0) ? 1.f : 0.f;
#pragma unroll
        for (int k = 0; k < 3; ++k) { p[k] = 0.f; w[k] = 0.f; vl[k] = 0.f; aw[k] = 0.f; al[k] = -H.gravity[k]; }
        int j0 = 0, cur = -1;
        if (H.free_root && T.anc[Dl.row] == 0) {   // the chain starts at the free root (body 0)
            // free root (body 0, DoFs 0-5): origin at offset + q[0..2], orientation exp(q[3..5])
            // (Rodrigues: R = I + (sin t / t) K + ((1 - cos t) / t^2) K^2, K = [r]x, with
            // 1 - cos t = 2 sin^2(t / 2)); axes world x, y, z: slides S = [0; e], turns
            // S = [e; p x e]
            const BodyRec& B0 = T.body[0];
            const float r0 = q[3], r1 = q[4], r2 = q[5];
            const float t2 = r0 * r0 + r1 * r1 + r2 * r2, t = sqrtf(t2);
            float sh, ch;
            sincosf(0.5f * t, &sh, &ch);
            const float ka = t > 1e-20f ? 2.f * sh * ch / t : 1.f;
            const float kb = t > 1e-20f ? 2.f * sh * sh / t2 : 0.5f;
            const float rr[3] = {r0, r1, r2};
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int k = 0; k < 3; ++k) R[3 * i + k] = kb * rr[i] * rr[k] + (i == k ? 1.f - kb * t2 : 0.f);
            R[1] -= ka * r2; R[2] += ka * r1; R[3] += ka * r2; R[5] -= ka * r0; R[6] -= ka * r1; R[7] += ka * r0;
            p[0] = B0.off[0] + q[0]; p[1] = B0.off[1] + q[1]; p[2] = B0.off[2] + q[2];
            const float om[3] = {qd[3], qd[4], qd[5]}, vp[3] = {qd[0], qd[1], qd[2]};
            if (b == 0) {
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    float* St = S + 6 * i;
                    float* Sr = S + 6 * (3 + i);
                    const float e[3] = {i == 0 ? 1.f : 0.f, i == 1 ? 1.f : 0.f, i == 2 ? 1.f : 0.f};
                    float pe[3];
                    cross3(p, e, pe);
                    St[0] = St[1] = St[2] = 0.f; St[3] = e[0]; St[4] = e[1]; St[5] = e[2];
                    Sr[0] = e[0]; Sr[1] = e[1]; Sr[2] = e[2]; Sr[3] = pe[0]; Sr[4] = pe[1]; Sr[5] = pe[2];
                }
            }
            // velocity [w; v_p + p x w]; bias [0; v_p x w] (the turn axes move with the origin)
            float pw[3], vw[3];
            cross3(p, om, pw);
            cross3(vp, om, vw);
#pragma unroll
            for (int k = 0; k < 3; ++k) { w[k] = om[k]; vl[k] = vp[k] + pw[k]; al[k] += vw[k]; }
            j0 = 6;
            cur = 0;
        }
        const int own0 = Dl.depth + 1 - Bb.ndof;   // chain position of the body's first DoF
        for (int j = j0; j <= Dl.depth; ++j) {
            const int d = T.anc[Dl.row + j];
            const DofRec& D = T.dof[d];
            if (D.body != cur) {   // entering the next body: its joint origin in the parent frame
                cur = D.body;
                float o[3];
                rot3(R, T.body[cur].off, o);
                p[0] += o[0]; p[1] += o[1]; p[2] += o[2];
            }
            float sv[3], ps[3];
            rot3(R, D.axis, sv);
            cross3(p, sv, ps);
            if (j >= own0) {
                float* Sd = S + 6 * d;
                Sd[0] = sv[0]; Sd[1] = sv[1]; Sd[2] = sv[2]; Sd[3] = ps[0]; Sd[4] = ps[1]; Sd[5] = ps[2];
            }
            const float qdj = qd[d];
            const float sw[3] = {sv[0] * qdj, sv[1] * qdj, sv[2] * qdj};
            const float sl[3] = {ps[0] * qdj, ps[1] * qdj, ps[2] * qdj};
            float c1[3], c2[3], c3[3];
            cross3(w, sw, c1);      // a += v x (S qd)
            cross3(w, sl, c2);
            cross3(vl, sw, c3);
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                aw[k] += c1[k];
                al[k] += c2[k] + c3[k];
                w[k] += sw[k];
                vl[k] += sl[k];
            }
            // R <- R Rot(axis, q) = c R + s (rows x axis) + (1 - c) (R axis) axis^T
            const float sn = SC[2 * d], cs = SC[2 * d + 1];
            const float* ax = D.axis;
            const float omc = 1.f - cs;
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                const float r0 = R[3 * r], r1 = R[3 * r + 1], r2 = R[3 * r + 2];
                const float x0 = r1 * ax[2] - r2 * ax[1];
                const float x1 = r2 * ax[0] - r0 * ax[2];
                const float x2 = r0 * ax[1] - r1 * ax[0];
                R[3 * r] = cs * r0 + sn * x0 + omc * sv[r] * ax[0];
                R[3 * r + 1] = cs * r1 + sn * x1 + omc * sv[r] * ax[1];
                R[3 * r + 2] = cs * r2 + sn * x2 + omc * sv[r] * ax[2];
            }
        }
        frame_store(raw(frame + 12 * b), R, p);
        float2* Vb = reinterpret_cast<float2*>(raw(V + 6 * b));     // 8-byte aligned (6 floats per body)
        float2* Ab = reinterpret_cast<float2*>(raw(Acc + 6 * b));
        Vb[0] = make_float2(w[0], w[1]); Vb[1] = make_float2(w[2], vl[0]); Vb[2] = make_float2(vl[1], vl[2]);
        Ab[0] = make_float2(aw[0], aw[1]); Ab[1] = make_float2(aw[2], al[0]); Ab[2] = make_float2(al[1], al[2]);
    }
    g.sync();
    SUB_MARK(15);   // profiling builds: sines, cosines and the recursion
    // 3. spatial inertia and body force of every body, all bodies in parallel
    for (int b = g.lane; b < H.nb; b += g.N) {
        const BodyRec& B = T.body[b];
        const float2* Vb = reinterpret_cast<const float2*>(raw(V + 6 * b));
        const float2* Ab = reinterpret_cast<const float2*>(raw(Acc + 6 * b));
        float R[9], p[3];
        frame_load(raw(frame + 12 * b), R, p);
        const float2 v0 = Vb[0], v1 = Vb[1], v2 = Vb[2], a0 = Ab[0], a1 = Ab[1], a2 = Ab[2];
        const float w[3] = {v0.x, v0.y, v1.x}, vl[3] = {v1.y, v2.x, v2.y};
        const float aw[3] = {a0.x, a0.y, a1.x}, al[3] = {a1.y, a2.x, a2.y};
        // spatial inertia about the world origin: m, h = m c, Ibar = R Ic R^T + m (|c|^2 1 - c c^T).
        // R Ic R^T in FP32 (a consistent perturbation of the body's own inertia); the
        // parallel-axis part, exact products of the FP32 COM, in float-float.
        const float m = B.mass;
        float c[3];
        rot3(R, B.com, c);
        c[0] += p[0]; c[1] += p[1]; c[2] += p[2];
        const float I9[9] = {B.I[0], B.I[3], B.I[4], B.I[3], B.I[1], B.I[5], B.I[4], B.I[5], B.I[2]};
        float TI[9];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int cc = 0; cc < 3; ++cc)
                TI[3 * r + cc] = R[3 * r] * I9[cc] + R[3 * r + 1] * I9[3 + cc] + R[3 * r + 2] * I9[6 + cc];
        const df c00 = two_prod(c[0], c[0]), c11 = two_prod(c[1], c[1]), c22 = two_prod(c[2], c[2]);
        const df cc2 = df_add(df_add(c00, c11), c22);
        df Ibd[6];   // xx yy zz xy xz yz
        {
            const float rxx = TI[0] * R[0] + TI[1] * R[1] + TI[2] * R[2];
            const float ryy = TI[3] * R[3] + TI[4] * R[4] + TI[5] * R[5];
            const float rzz = TI[6] * R[6] + TI[7] * R[7] + TI[8] * R[8];
            const float rxy = TI[0] * R[3] + TI[1] * R[4] + TI[2] * R[5];
            const float rxz = TI[0] * R[6] + TI[1] * R[7] + TI[2] * R[8];
            const float ryz = TI[3] * R[6] + TI[4] * R[7] + TI[5] * R[8];
            Ibd[0] = df_add_f(df_mul_f(df_add(cc2, df_neg(c00)), m), rxx);
            Ibd[1] = df_add_f(df_mul_f(df_add(cc2, df_neg(c11)), m), ryy);
            Ibd[2] = df_add_f(df_mul_f(df_add(cc2, df_neg(c22)), m), rzz);
            Ibd[3] = df_add_f(df_neg(df_mul_f(two_prod(c[0], c[1]), m)), rxy);
            Ibd[4] = df_add_f(df_neg(df_mul_f(two_prod(c[0], c[2]), m)), rxz);
            Ibd[5] = df_add_f(df_neg(df_mul_f(two_prod(c[1], c[2]), m)), ryz);
        }
        const df hd[3] = {two_prod(m, c[0]), two_prod(m, c[1]), two_prod(m, c[2])};
        // float-float body force f = I a + v x* (I v) from the float-float inertia (the bias
        // enters the right-hand side exactly, so that the conditioning of M does not amplify
        // FP32 rounding of the force sums)
        auto imul = [&](const float xw[3], const float xl[3], df ow[3], df ol[3]) {
            // ow = Ibar xw + h x xl, ol = m xl - h x xw
            const df hxl[3] = {df_add(df_mul_f(hd[1], xl[2]), df_neg(df_mul_f(hd[2], xl[1]))),
                               df_add(df_mul_f(hd[2], xl[0]), df_neg(df_mul_f(hd[0], xl[2]))),
                               df_add(df_mul_f(hd[0], xl[1]), df_neg(df_mul_f(hd[1], xl[0])))};
            const df hxw[3] = {df_add(df_mul_f(hd[1], xw[2]), df_neg(df_mul_f(hd[2], xw[1]))),
                               df_add(df_mul_f(hd[2], xw[0]), df_neg(df_mul_f(hd[0], xw[2]))),
                               df_add(df_mul_f(hd[0], xw[1]), df_neg(df_mul_f(hd[1], xw[0])))};
            ow[0] = df_add(df_add(df_add(df_mul_f(Ibd[0], xw[0]), df_mul_f(Ibd[3], xw[1])), df_mul_f(Ibd[4], xw[2])), hxl[0]);
            ow[1] = df_add(df_add(df_add(df_mul_f(Ibd[3], xw[0]), df_mul_f(Ibd[1], xw[1])), df_mul_f(Ibd[5], xw[2])), hxl[1]);
            ow[2] = df_add(df_add(df_add(df_mul_f(Ibd[4], xw[0]), df_mul_f(Ibd[5], xw[1])), df_mul_f(Ibd[2], xw[2])), hxl[2]);
#pragma unroll
            for (int k = 0; k < 3; ++k) ol[k] = df_add(two_prod(m, xl[k]), df_neg(hxw[k]));
        };
        // a x b, a FP32, b float-float
        auto xfd = [](const float a[3], const df bb[3], df o[3]) {
            o[0] = df_add(df_mul_f(bb[2], a[1]), df_neg(df_mul_f(bb[1], a[2])));
            o[1] = df_add(df_mul_f(bb[0], a[2]), df_neg(df_mul_f(bb[2], a[0])));
            o[2] = df_add(df_mul_f(bb[1], a[0]), df_neg(df_mul_f(bb[0], a[1])));
        };
        df Ivw[3], Ivl[3], Iaw[3], Ial[3];
        imul(w, vl, Ivw, Ivl);
        imul(aw, al, Iaw, Ial);
        df t1[3], t2[3], t3[3];
        xfd(w, Ivw, t1);
        xfd(vl, Ivl, t2);
        xfd(w, Ivl, t3);
        // force (6 float-float, 48 bytes) and inertia (m, h[3], Ibar[6]: 80 bytes) of the body,
        // stored as 16-byte words
        df fo[6];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            fo[k] = df_add(df_add(Iaw[k], t1[k]), t2[k]);
            fo[3 + k] = df_add(Ial[k], t3[k]);
        }
        float4* fb4 = reinterpret_cast<float4*>(raw(FB + 6 * b));
#pragma unroll
        for (int k = 0; k < 3; ++k) fb4[k] = make_float4(fo[2 * k].hi, fo[2 * k].lo, fo[2 * k + 1].hi, fo[2 * k + 1].lo);
        float4* I4 = reinterpret_cast<float4*>(raw(FI + kFiStride * b));
        I4[0] = make_float4(m, 0.f, hd[0].hi, hd[0].lo);
        I4[1] = make_float4(hd[1].hi, hd[1].lo, hd[2].hi, hd[2].lo);
#pragma unroll
        for (int e = 0; e < 3; ++e)
            I4[2 + e] = make_float4(Ibd[2 * e].hi, Ibd[2 * e].lo, Ibd[2 * e + 1].hi, Ibd[2 * e + 1].lo);
    }
    g.sync();
}

// ------------------------------------------------------------------ phase 2: subtree sums, bias
template <int WPE>
__device__ void phase_subtree(const Tables& T, float* ws, const Grp<WPE>& g) {
    const ImgHeader& H = *T.H;
    auto FI = WS(float, H.w_fi);
    auto FB = WS(df, H.w_f);
    auto S = WS(const float, H.w_S);
    auto rhs = WS(float, H.w_rhs);
    auto racc = WS(int32_t, H.w_racc);
    // subtree sums, leaves first, along the body chains (maximal runs of single-child bodies):
    // every chain's 16 components (force 6, float-float inertia 10) go to their own lanes, which
    // walk the chain bottom to top carrying the running sum; the bottom body adds its children
    // (tops of chains of earlier rounds), so a round costs one barrier.  Each body's sum is its
    // own term plus its children's sums in child order, as a leaves-first level pass would add.
    for (int r = 0; r < H.n_crounds; ++r) {
        const int c0 = T.cround[r], c1 = T.cround[r + 1];
        for (int t = g.lane; t < 16 * (c1 - c0); t += g.N) {
            const int c = c0 + t / 16, comp = t % 16;
            const int j0 = T.cstart[c], j1 = T.cstart[c + 1];
            df* base = comp < 6 ? raw(FB + comp) : reinterpret_cast<df*>(raw(FI)) + (comp - 6);
            const int stride = comp < 6 ? 6 : kFiStride / 2;   // df entries per body
            const BodyRec& Bb = T.body[T.cbody[j0]];
            df f = base[stride * T.cbody[j0]];
            for (int k = 0; k < Bb.nchild; ++k) f = df_add(f, base[stride * T.child[Bb.child0 + k]]);
            base[stride * T.cbody[j0]] = f;
            for (int j = j0 + 1; j < j1; ++j) {
                const int b = T.cbody[j];
                f = df_add(base[stride * b], f);
                base[stride * b] = f;
            }
        }
        g.sync();
    }
    // bias of every DoF from its body's subtree force, all DoFs in parallel, in float-float:
    // -S^T f starts the exact fixed-point accumulator of the right-hand side (the muscle and
    // contact terms follow); rhs keeps the FP32 terms (limits, damping)
    for (int d = g.lane; d < H.n; d += g.N) {
        const float2* S2 = reinterpret_cast<const float2*>(raw(S + 6 * d));
        const float4* f4 = reinterpret_cast<const float4*>(raw(FB + 6 * T.dof[d].body));
        const float2 s01 = S2[0], s23 = S2[1], s45 = S2[2];
        const float4 fa = f4[0], fbb = f4[1], fc = f4[2];
        const float Sd[6] = {s01.x, s01.y, s23.x, s23.y, s45.x, s45.y};
        const df f[6] = {df{fa.x, fa.y}, df{fa.z, fa.w}, df{fbb.x, fbb.y}, df{fbb.z, fbb.w}, df{fc.x, fc.y}, df{fc.z, fc.w}};
        df c = df_mul_f(f[0], Sd[0]);
#pragma unroll
        for (int k = 1; k < 6; ++k) c = df_fma_f(c, f[k], Sd[k]);
        fx_store(&racc[2 * d], df_neg(c));
        rhs[d] = 0.f;
    }
    g.sync();
}

// Arithmetic of the system matrix A = M + dt D, its factorisation and the solves: float-float
// pairs by default; FP64 with MSIM_FP64_FACTOR (same 8 bytes per entry).
#ifdef MSIM_FP64_FACTOR
using fac = double;
__device__ __forceinline__ fac fac_of(df x) { return static_cast<double>(x.hi) + static_cast<double>(x.lo); }
__device__ __forceinline__ fac fac_add_f(fac a, float b) { return a + static_cast<double>(b); }
__device__ __forceinline__ fac fac_mul(fac a, fac b) { return a * b; }
__device__ __forceinline__ fac fac_fms(fac acc, fac x, fac y) { return fma(-x, y, acc); }
__device__ __forceinline__ fac fac_rsqrt(fac x) { return rsqrt(x); }
__device__ __forceinline__ float fac_f(fac x) { return static_cast<float>(x); }
__device__ __forceinline__ bool fac_pos(fac x) { return x > 0.0; }
__device__ __forceinline__ fac fac_one() { return 1.0; }
__device__ __forceinline__ fac fac_decode(int32_t hi, int32_t lo) {
    return static_cast<double>(hi) * (1.0 / 256.0) + static_cast<double>(lo) * (1.0 / 268435456.0);
}
#else
using fac = df;
__device__ __forceinline__ fac fac_add_f(fac a, float b) { return df_add_f(a, b); }
__device__ __forceinline__ fac fac_mul(fac a, fac b) { return df_mul(a, b); }
__device__ __forceinline__ fac fac_fms(fac acc, fac x, fac y) { return df_fms(acc, x, y); }
__device__ __forceinline__ fac fac_rsqrt(fac x) { return df_rsqrt(x); }
__device__ __forceinline__ float fac_f(fac x) { return x.hi + x.lo; }
__device__ __forceinline__ bool fac_pos(fac x) { return x.hi > 0.f; }
__device__ __forceinline__ fac fac_one() { return df_make(1.f); }
__device__ __forceinline__ fac fac_decode(int32_t hi, int32_t lo) { return fx_decode(hi, lo); }
#endif

// ------------------------------------------------------------------ phase 3: CRBA (float-float)
// Adds M to the damping sums already accumulated (fixed point) in the same storage.  DoFs are
// taken longest row first and dealt to the lanes in a snake (similar entry counts per lane).
template <int WPE>
__device__ void phase_crba(const Tables& T, float* ws, const Grp<WPE>& g, float* evM) {
    const ImgHeader& H = *T.H;
    auto FI = WS(const float, H.w_fi);
    auto S = WS(const float, H.w_S);
    auto A = WS(fac, H.w_A);
    auto Ai = WS(const int32_t, H.w_A);
    // rows by decreasing length, dealt to the group's lanes in a snake (0..N-1, N-1..0, ...)
    for (int r0 = 0; r0 < H.n; r0 += g.N) {
        const int t = r0 + (((r0 / g.N) & 1) ? g.N - 1 - g.lane : g.lane);
        if (t >= H.n) continue;
        const uint2 ce = T.crba_order[t];
        const int d = ce.x & 0xff, body = (ce.x >> 8) & 0xff, dep = (ce.x >> 16) & 0xff;
        // the body's composite inertia as five 16-byte words (80-byte stride): m, h, then
        // Ibar xx yy zz xy xz yz, float-float each
        df m, h0, h1, h2, Ib[6];
        {
            const float4* I4 = reinterpret_cast<const float4*>(raw(FI + kFiStride * body));
            const float4 w0 = I4[0], w1 = I4[1], w2 = I4[2], w3 = I4[3], w4 = I4[4];
            m = df{w0.x, w0.y}; h0 = df{w0.z, w0.w}; h1 = df{w1.x, w1.y}; h2 = df{w1.z, w1.w};
            Ib[0] = df{w2.x, w2.y}; Ib[1] = df{w2.z, w2.w}; Ib[2] = df{w3.x, w3.y}; Ib[3] = df{w3.z, w3.w};
            Ib[4] = df{w4.x, w4.y}; Ib[5] = df{w4.z, w4.w};
        }
        const float2* Sd = reinterpret_cast<const float2*>(raw(S + 6 * d));   // 8-byte aligned
        const float2 sa = Sd[0], sb = Sd[1], sc = Sd[2];
        const float s0 = sa.x, s1 = sa.y, s2 = sb.x, p0 = sb.y, p1 = sc.x, p2 = sc.y;
        // F = I^c S: Fw = Ibar s + h x ps, Fl = m ps - h x s
        df Fw[3], Fl[3];
        Fw[0] = df_add(df_add(df_add(df_mul_f(Ib[0], s0), df_mul_f(Ib[3], s1)), df_mul_f(Ib[4], s2)),
                       df_add(df_mul_f(h1, p2), df_neg(df_mul_f(h2, p1))));
        Fw[1] = df_add(df_add(df_add(df_mul_f(Ib[3], s0), df_mul_f(Ib[1], s1)), df_mul_f(Ib[5], s2)),
                       df_add(df_mul_f(h2, p0), df_neg(df_mul_f(h0, p2))));
        Fw[2] = df_add(df_add(df_add(df_mul_f(Ib[4], s0), df_mul_f(Ib[5], s1)), df_mul_f(Ib[2], s2)),
                       df_add(df_mul_f(h0, p1), df_neg(df_mul_f(h1, p0))));
        Fl[0] = df_add(df_mul_f(m, p0), df_neg(df_add(df_mul_f(h1, s2), df_neg(df_mul_f(h2, s1)))));
        Fl[1] = df_add(df_mul_f(m, p1), df_neg(df_add(df_mul_f(h2, s0), df_neg(df_mul_f(h0, s2)))));
        Fl[2] = df_add(df_mul_f(m, p2), df_neg(df_add(df_mul_f(h0, s1), df_neg(df_mul_f(h1, s0)))));
        const int row = (int)ce.y;
        for (int k = 0; k <= dep; ++k) {
            const float2* Sa = reinterpret_cast<const float2*>(raw(S + 6 * T.anc[row + k]));
            const float2 a01 = Sa[0], a23 = Sa[1], a45 = Sa[2];
            df acc = df_mul_f(Fw[0], a01.x);
            acc = df_fma_f(acc, Fw[1], a01.y);
            acc = df_fma_f(acc, Fw[2], a23.x);
            acc = df_fma_f(acc, Fl[0], a23.y);
            acc = df_fma_f(acc, Fl[1], a45.x);
            acc = df_fma_f(acc, Fl[2], a45.y);
            if (evM) evM[row + k] = acc.hi + acc.lo;
#ifdef MSIM_FP64_FACTOR
            A[row + k] = fac_of(acc) + fac_decode(Ai[2 * (row + k)], Ai[2 * (row + k) + 1]);
#else
            A[row + k] = df_add(acc, fx_decode(Ai[2 * (row + k)], Ai[2 * (row + k) + 1]));
#endif
        }
    }
    g.sync();
}

// ------------------------------------------------------------------ Hill curves (Eq. 1)
// Readings of the curves the paper takes from Millard 2013 (not printed there): Gaussian
// active force-length of width 0.45, exponential passive curve reaching 1 at 1.6 l_opt with a
// linear extension, Hill hyperbola when shortening and a saturating branch (to 1.4) when
// lengthening, slope 5 at v = 0 on both sides.
__device__ __forceinline__ float hill_fl(float l) {
    const float x = l - 1.f;
    return expf(-x * x * (1.f / 0.45f));
}
__device__ __forceinline__ float hill_fp(float l, float den, float slope) {
    if (l <= 1.f) return 0.f;
    if (l <= 1.6f) return (expf((l - 1.f) * (4.f / 0.6f)) - 1.f) / den;
    return 1.f + slope * (l - 1.6f);
}
__device__ __forceinline__ float hill_fv(float v) {
    if (v < -1.f) return 0.f;
    if (v <= 0.f) return (1.f + v) / (1.f - 4.f * v);
    return 1.f + 0.4f * v / (v + 0.08f);
}
__device__ __forceinline__ float hill_dfv(float v) {
    if (v < -1.f) return 0.f;
    if (v <= 0.f) {
        const float den = 1.f - 4.f * v;
        return 5.f / (den * den);
    }
    const float den = v + 0.08f;
    return 0.032f / (den * den);
}
__device__ __forceinline__ float hill_dfl(float l) { return (l - 1.f) * (-2.f / 0.45f) * hill_fl(l); }
__device__ __forceinline__ float hill_dfp(float l, float den, float slope) {
    if (l <= 1.f) return 0.f;
    if (l <= 1.6f) return (4.f / 0.6f) * expf((l - 1.f) * (4.f / 0.6f)) / den;
    return slope;
}

// ------------------------------------------------------------------ compliant tendon
// Reading of the Hill model's series elastic tendon (the paper's is rigid), damped-equilibrium
// form (Millard 2013): the tendon strain eps is a state; tendon curve f_t(x), x = eps / eps0,
// (e^{3x} - 1 - 3x)/(e^3 - 4) on [0, 1] (zero slope at slack, 1 at x = 1), linear beyond with
// the same slope, 0 when slack; the fibre, with a parallel damper beta, carries the tendon's
// force.
constexpr float kTendonBeta = 0.1f;
__device__ __forceinline__ float tendon_f(float x, float den, float slope) {
    if (x <= 0.f) return 0.f;
    if (x <= 1.f) return (expm1f(3.f * x) - 3.f * x) / den;
    return 1.f + slope * (x - 1.f);
}
__device__ __forceinline__ float tendon_df(float x, float den, float slope) {
    if (x <= 0.f) return 0.f;
    if (x <= 1.f) return 3.f * expm1f(3.f * x) / den;
    return slope;
}
// Root v of A f_v(v) + beta v + c0 = 0 (A >= 0).  The left side increases strictly with v, so
// its signs at the joins of f_v's branches (v = -1: c0 - beta; v = 0: A + c0) select the branch,
// where the equation is linear (v < -1, f_v = 0) or, cleared of f_v's denominator, a quadratic
// with one root in the branch, taken in the form without cancellation.
__device__ __forceinline__ float fibre_velocity(float A, float c0) {
    constexpr float b = kTendonBeta;
    if (c0 - b >= 0.f) return -c0 * (1.f / b);
    if (A + c0 >= 0.f) {
        // (1 - 4v) g = 0:  4b v^2 - B v - C = 0, B = A + b - 4 c0, C = A + c0 >= 0; the root <= 0
        const float B = A + b - 4.f * c0, C = A + c0;
        const float sq = sqrtf(fmaf(B, B, 16.f * b * C));
        return B >= 0.f ? -2.f * C / (B + sq) : (B - sq) * (1.f / (8.f * b));
    }
    // (v + 0.08) g = 0:  b v^2 + B v + C = 0, B = 1.4 A + 0.08 b + c0, C = 0.08 (A + c0) < 0; the root > 0
    const float B = fmaf(1.4f, A, 0.08f * b + c0), C = 0.08f * (A + c0);
    const float sq = sqrtf(fmaf(B, B, -4.f * b * C));
    return B <= 0.f ? (sq - B) * (1.f / (2.f * b)) : -2.f * C / (B + sq);
}

// Per-environment context of a surrogate step: the network's normalised output row and its
// de-normalisation, whether this environment must use the exact geometry (outside the training
// box, or flagged), whether this substep cross-checks the two, and the check's tolerance.
struct SurrCtx {
    const float* Y;               // the environment's row of the inference head (physical units)
    const int* colbase;           // first column of each group of 32 muscle records
    bool use_exact;
    bool check;
    float tol;
    unsigned int* max_err_bits;   // global running maximum of the check error (float bits)
};

// Shortest path x0 -> x1 around an infinite cylinder (world centre c, unit axis a, radius r):
// in the plane normal to the axis, tangent - arc - tangent on the side of the shorter arc;
// along the axis a straight line once the cylinder is unrolled.  Wraps (returns true, with the
// length, the tangent points Q, T and the unit directions u1 of x0 -> Q and u2 of T -> x1) when
// both points are outside the cylinder and the straight segment passes within r of the axis.
// With p, s the two points' in-plane offsets from the axis, the shorter arc is the one on the
// side the chord passes (counter-clockwise about a when p x s >= 0): for an active wrap both
// arcs are psi - alpha_p - alpha_s and 2 pi - psi - alpha_p - alpha_s, psi the angle from p to s
// the short way round.  The tangent points come from the angle-sum identities
// (cos alpha = r / rho, sin alpha = l / rho, l the tangent length), the arc from one atan2, the
// directions from the circle's tangent at Q and T and the unrolled slope.
__device__ bool wrap_path(const float x0[3], const float x1[3], const float c[3], const float a[3], float r,
                          float& len, float Q[3], float T[3], float u1[3], float u2[3]) {
    float e1[3];
    const float ref[3] = {fabsf(a[0]) < 0.9f ? 1.f : 0.f, fabsf(a[0]) < 0.9f ? 0.f : 1.f, 0.f};
    cross3(a, ref, e1);
    const float in1 = rsqrtf(dot3(e1, e1));
    e1[0] *= in1; e1[1] *= in1; e1[2] *= in1;
    float e2[3];
    cross3(a, e1, e2);
    const float p[3] = {x0[0] - c[0], x0[1] - c[1], x0[2] - c[2]};
    const float q[3] = {x1[0] - c[0], x1[1] - c[1], x1[2] - c[2]};
    const float px = dot3(p, e1), py = dot3(p, e2), pz = dot3(p, a);
    const float sx = dot3(q, e1), sy = dot3(q, e2), sz = dot3(q, a);
    const float rp2 = px * px + py * py, rs2 = sx * sx + sy * sy, r2 = r * r;
    if (!(rp2 > r2 && rs2 > r2)) return false;
    const float ex = sx - px, ey = sy - py, ee = ex * ex + ey * ey;
    float t = ee > 0.f ? -(px * ex + py * ey) / ee : 0.f;
    t = fminf(fmaxf(t, 0.f), 1.f);
    const float cx = px + t * ex, cy = py + t * ey;
    if (cx * cx + cy * cy >= r2) return false;
    const float turn = (px * sy - py * sx >= 0.f) ? 1.f : -1.f;   // +1: counter-clockwise about a
    const float lp = sqrtf(rp2 - r2), ls = sqrtf(rs2 - r2);
    const float ip = 1.f / rp2, is = 1.f / rs2;
    // Q at the angle of p advanced by alpha_p, T at the angle of s moved back by alpha_s
    const float cq = (px * r - turn * py * lp) * ip, sq = (py * r + turn * px * lp) * ip;
    const float ct = (sx * r + turn * sy * ls) * is, st = (sy * r - turn * sx * ls) * is;
    const float arc = fmaxf(atan2f(turn * (cq * st - sq * ct), cq * ct + sq * st), 0.f);
    const float lplane = lp + r * arc + ls, dz = sz - pz;
    const float zq = pz + dz * lp / lplane, zt = pz + dz * (lp + r * arc) / lplane;
    len = sqrtf(lplane * lplane + dz * dz);
    const float il = 1.f / len, kp = lplane * il * turn, kz = dz * il;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        Q[i] = c[i] + r * cq * e1[i] + r * sq * e2[i] + zq * a[i];
        T[i] = c[i] + r * ct * e1[i] + r * st * e2[i] + zt * a[i];
        u1[i] = kp * (cq * e2[i] - sq * e1[i]) + kz * a[i];   // direction of travel at Q
        u2[i] = kp * (ct * e2[i] - st * e1[i]) + kz * a[i];   // and at T
    }
    return true;
}

// ------------------------------------------------------------------ phase 4: muscles
#pragma nv_diag_suppress 128
// One lane per muscle.  act: this environment's activation row in global memory (read;
// written unless MODE == kModeEval).
// Returns bit 0: a force was not finite; bit 1 (surrogate step): the cross-check exceeded the
// tolerance.  Geometry mode writes L to ev->L[k] and the moment arms to ev->R and stops there.
// (The statements after its `continue` are unreachable in that mode only: warning 128 is off.)
template <int MODE, int WPE>
__device__ uint32_t phase_muscles(const Tables& T, float* ws, const Grp<WPE>& g, float dt, const float* exc,
                                  float* act, float* eps, float* force_out, float* vm_out, const EvalPtrs* ev,
                                  const SurrCtx* sc) {
    const ImgHeader& H = *T.H;
    auto qd = WS(const float, H.w_qd);
    auto frame = WS(const float, H.w_frame);
    auto S = WS(const float, H.w_S);
    auto Ai = WS(int32_t, H.w_A);   // damping sums, fixed point
    auto racc = WS(int32_t, H.w_racc);
    auto rk = WS(float, H.w_rk);                                  // [max_nx][N]
    bool bad = false;
    float se_len = 0.f, se_arm = 0.f;   // check: squared errors of the learned lengths and arms
    SUB_T0();
    for (int r = g.lane; r < H.m; r += g.N) {
        const MuscleRec M = T.mus[r];
        const int k = M.orig;
        const float a = MODE == kModeGeom ? 0.f : act[k];
        const float u = MODE == kModeGeom ? 0.f : fminf(fmaxf(exc[k], 0.f), 1.f);
        const bool learned = is_surr(MODE) && !sc->use_exact;   // geometry from the network
        float L = 0.f, ldot = 0.f;
        if (!learned || sc->check) {
            // exact via-point geometry: L = sum |x_{j+1} - x_j|, R = -dL/dq of the crossed DoFs
            PointRec P = T.pt[M.p0];
            PointRec Pn = T.pt[M.p0 + 32];   // the next point is loaded one segment ahead
            int b = P.body_cross & 0xff;
            int cprev = P.body_cross >> 8;
            float x0[3];
            {
                float Rb[9], pb[3];
                frame_load(raw(frame + 12 * b), Rb, pb);
                rot3(Rb, P.pos, x0);
                x0[0] += pb[0]; x0[1] += pb[1]; x0[2] += pb[2];
            }
            // moment arms of the crossed DoFs [i0, i1) for a straight piece with unit direction
            // uu whose distal end xd moves with them: R = -dL/dq = -s_d . ((xd - o_d) x uu)
            auto arms = [&](int i0, int i1, const float xd[3], const float uu[3]) {
                for (int i = i0; i < i1; ++i) {
                    const uint32_t ce = T.cross[M.x0 + i];
                    const int d = cross_dof(ce);
                    const float2 s01 = *reinterpret_cast<const float2*>(raw(S + 6 * d));   // 8-byte aligned
                    const float s2 = S[6 * d + 2];
                    float o[3];
                    frame_origin(raw(frame + 12 * cross_body(ce)), o);
                    const float rr[3] = {xd[0] - o[0], xd[1] - o[1], xd[2] - o[2]};
                    float rxu[3];
                    cross3(rr, uu, rxu);
                    const float Rv = -(s01.x * rxu[0] + s01.y * rxu[1] + s2 * rxu[2]);
                    rk[i * g.N + g.lane] = Rv;
                    ldot -= Rv * qd[d];
                }
            };
            const int wseg = (has_ext(MODE) && M.wrap) ? ((T.wrap[M.wrap - 1].body_cross >> 16) & 0xff) : 0;
            for (int j = 1; j < M.np; ++j) {
                P = Pn;   // points interleaved by groups of 32 records: point j at p0 + 32 j
                if (j + 1 < M.np) Pn = T.pt[M.p0 + 32 * (j + 1)];
                b = P.body_cross & 0xff;
                const int c = P.body_cross >> 8;
                float x1[3];
                {
                    float Rb[9], pb[3];
                    frame_load(raw(frame + 12 * b), Rb, pb);
                    rot3(Rb, P.pos, x1);
                    x1[0] += pb[0]; x1[1] += pb[1]; x1[2] += pb[2];
                }
                bool wrapped = false;
                if (has_ext(MODE) && j == wseg) {
                    // the wrapped segment: tangent points held on the cylinder's body for the arms
                    const WrapRec W = T.wrap[M.wrap - 1];
                    const float* fw = frame + 12 * (W.body_cross & 0xff);
                    float cw[3], aw[3], Q[3], Tp[3], u1[3], u2[3], lw;
                    rot3(fw, W.center, cw);
                    cw[0] += fw[9]; cw[1] += fw[10]; cw[2] += fw[11];
                    if (W.body_cross >> 24) {
                        // sphere: the cylinder case about the normal of the plane through the
                        // two points and the centre (a perpendicular to x1 - x0 if collinear)
                        const float pp[3] = {x0[0] - cw[0], x0[1] - cw[1], x0[2] - cw[2]};
                        const float qq[3] = {x1[0] - cw[0], x1[1] - cw[1], x1[2] - cw[2]};
                        cross3(pp, qq, aw);
                        float nn = dot3(aw, aw);
                        if (!(nn > 1e-12f * dot3(pp, pp) * dot3(qq, qq))) {
                            const float dd[3] = {x1[0] - x0[0], x1[1] - x0[1], x1[2] - x0[2]};
                            const float a0 = fabsf(dd[0]), a1 = fabsf(dd[1]), a2 = fabsf(dd[2]);
                            const float ref[3] = {a0 <= a1 && a0 <= a2 ? 1.f : 0.f, a0 > a1 && a1 <= a2 ? 1.f : 0.f,
                                                  a2 < a0 && a2 < a1 ? 1.f : 0.f};
                            cross3(dd, ref, aw);
                            nn = dot3(aw, aw);
                        }
                        const float in = rsqrtf(nn);
                        aw[0] *= in; aw[1] *= in; aw[2] *= in;
                    } else {
                        rot3(fw, W.axis, aw);
                    }
                    wrapped = wrap_path(x0, x1, cw, aw, W.radius, lw, Q, Tp, u1, u2);
                    if (wrapped) {
                        L += lw;
                        const int cw_i = (W.body_cross >> 8) & 0xff;
                        arms(cprev, cw_i, Q, u1);   // DoFs that move the cylinder with x1
                        arms(cw_i, c, x1, u2);      // DoFs that move x1 alone
                    }
                }
                if (!wrapped) {
                    const float dv[3] = {x1[0] - x0[0], x1[1] - x0[1], x1[2] - x0[2]};
                    const float len2 = dot3(dv, dv);
                    const float inv = rsqrtf(len2);
                    L += len2 * inv;
                    const float uu[3] = {dv[0] * inv, dv[1] * inv, dv[2] * inv};
                    arms(cprev, c, x1, uu);
                }
                x0[0] = x1[0]; x0[1] = x1[1]; x0[2] = x1[2];
                cprev = c;
            }
        }
        if (is_surr(MODE) && learned) {
            // learned geometry: the record's length and moment arms from the inference head, entry
            // e at column colbase[r / 32] + 32 e + r % 32 (a warp reads each entry as one run)
            const float* Yr = sc->Y + sc->colbase[r >> 5] + (r & 31);
            const float Ls = Yr[0];
            if (sc->check) {
                // squared errors against the exact geometry, summed over the environment below
                const float dl = Ls - L;
                se_len += dl * dl;
                for (int i = 0; i < M.nx; ++i) {
                    const float dr = Yr[32 * (i + 1)] - rk[i * g.N + g.lane];
                    se_arm += dr * dr;
                }
            } else {
                L = Ls;
                // every load of the record issued before the first use: one latency per record
                float Rl[kMaxCross];
                uint32_t cl[kMaxCross];
#pragma unroll
                for (int i = 0; i < kMaxCross; ++i) {
                    Rl[i] = i < M.nx ? Yr[32 * (i + 1)] : 0.f;
                    cl[i] = i < M.nx ? T.cross[M.x0 + i] : 0u;
                }
#pragma unroll
                for (int i = 0; i < kMaxCross; ++i)
                    if (i < M.nx) {
                        rk[i * g.N + g.lane] = Rl[i];
                        ldot -= Rl[i] * qd[cross_dof(cl[i])];
                    }
            }
        }
        if (MODE == kModeGeom) {
            ev->L[k] = L;
            for (int i = 0; i < M.nx; ++i) ev->R[M.x0 + i] = rk[i * g.N + g.lane];
            continue;
        }
        SUB_MARK(8);
        float lm, vm, F, dFdl, en = 0.f;
        const TendonRec Tn = (has_ext(MODE) && T.ten) ? T.ten[r] : TendonRec{0.f, 0.f, 0.f, 0.f};
        if (has_ext(MODE) && Tn.inv_eps0 > 0.f) {
            // compliant tendon: fibre velocity from the damped equilibrium at the current strain,
            // strain advanced linearly implicitly, the tendon force at the new strain
            const float ls = M.L0 - Tn.lopt;
            const float inv_ls = 1.f / ls;
            const float e0 = eps ? eps[k] : 0.f;
            const float x = e0 * Tn.inv_eps0;
            lm = (L - ls * (1.f + e0)) * M.inv_lopt;
            const float fl = hill_fl(lm);
            const float A = a * fl;
            vm = fibre_velocity(A, hill_fp(lm, H.fp_den, H.fp_slope) - tendon_f(x, H.ft_den, H.ft_slope));
            const float num = tendon_df(x, H.ft_den, H.ft_slope) * Tn.inv_eps0 +
                              (a * hill_dfl(lm) * hill_fv(vm) + hill_dfp(lm, H.fp_den, H.fp_slope)) * ls * M.inv_lopt;
            const float J = fmaxf(num / fmaf(A, hill_dfv(vm), kTendonBeta), 0.f);
            const float gi = 1.f / fmaf(dt * Tn.vmax * J, inv_ls, 1.f);
            en = e0 + dt * (ldot - Tn.vmax * vm) * inv_ls * gi;
            const float xn = en * Tn.inv_eps0;
            F = M.fmax * tendon_f(xn, H.ft_den, H.ft_slope);
            dFdl = M.fmax * tendon_df(xn, H.ft_den, H.ft_slope) * Tn.inv_eps0 * dt * inv_ls * gi;
            if (MODE != kModeEval && eps) eps[k] = en;
        } else {
            lm = 1.f + (L - M.L0) * M.inv_lopt;
            vm = ldot * M.inv_vmax;
            const float fl = hill_fl(lm);
            F = M.fmax * (a * fl * hill_fv(vm) + hill_fp(lm, H.fp_den, H.fp_slope));
            dFdl = M.fmax * a * fl * hill_dfv(vm) * M.inv_vmax;
            if (has_ext(MODE)) en = eps ? eps[k] : 0.f;
        }
        const float tau = (u > a) ? H.tau_act * (0.5f + 1.5f * a) : H.tau_deact / (0.5f + 1.5f * a);
        const float an = fminf(fmaxf(a + dt * (u - a) / tau, 0.f), 1.f);
        if (MODE != kModeEval) act[k] = an;
        if (force_out) force_out[k] = F;
        if (vm_out) vm_out[k] = vm;
        SUB_MARK(9);
        // rhs += R^T F; A += dt R^T (dF/dLdot) R as g g^T with g = sqrt(dt dF/dLdot) R.  All
        // operands are loaded first, then the reductions issue back to back.
        const float sq = sqrtf(dt * dFdl);
        bad |= !(isfinite(F) && isfinite(sq));
        float Rr[kMaxCross];
        uint32_t cr[kMaxCross];
#pragma unroll
        for (int i = 0; i < kMaxCross; ++i) {
            Rr[i] = i < M.nx ? rk[i * g.N + g.lane] : 0.f;
            cr[i] = i < M.nx ? T.cross[M.x0 + i] : 0u;
        }
#pragma unroll
        for (int i = 0; i < kMaxCross; ++i) {
            if (i < M.nx) {
                fx_red(&racc[2 * cross_dof(cr[i])], Rr[i] * F);
                if ((MODE == kModeEval) && ev->tau_m) atomicAdd(&ev->tau_m[cross_dof(cr[i])], Rr[i] * F);
                if (sq != 0.f) {
                    const float gi = sq * Rr[i];
                    const int base = cross_row(cr[i]) + M.dep0;
#pragma unroll
                    for (int j = 0; j <= i; ++j) fx_red(&Ai[2 * (base + j)], gi * (sq * Rr[j]));
                }
            }
        }
        if ((MODE == kModeEval)) {
            if (ev->L) ev->L[k] = L;
            if (ev->lm) ev->lm[k] = lm;
            if (ev->vm) ev->vm[k] = vm;
            if (ev->force) ev->force[k] = F;
            if (ev->act_next) ev->act_next[k] = an;
            if (ev->eps_next) ev->eps_next[k] = en;
            if (ev->R)
                for (int i = 0; i < M.nx; ++i) ev->R[M.x0 + i] = Rr[i];
        }
        SUB_MARK(10);
    }
    bool fail = false;
    if (is_surr(MODE) && sc->check) {
        // the environment's check error: the larger of the root-mean-square errors of its moment
        // arms (over the nnz entries) and of its lengths (over the m muscles); a non-finite state
        // or output fails.  Warp sums, then the warps' sums in a fixed order through the
        // moment-arm region, which every lane has finished with after the first barrier.
        float v0 = se_arm, v1 = se_len;
        for (int o = 16; o > 0; o >>= 1) {
            v0 += __shfl_xor_sync(0xffffffffu, v0, o);
            v1 += __shfl_xor_sync(0xffffffffu, v1, o);
        }
        if (WPE > 1) {
            g.sync();
            if (g.wl == 0) {
                rk[2 * g.wi] = v0;
                rk[2 * g.wi + 1] = v1;
            }
            g.sync();
            v0 = v1 = 0.f;
            for (int w = 0; w < WPE; ++w) {
                v0 += rk[2 * w];
                v1 += rk[2 * w + 1];
            }
        }
        const float e = fmaxf(sqrtf(v0 / (float)max(H.nnz, 1)), sqrtf(v1 / (float)max(H.m, 1)));
        fail = !(e <= sc->tol);
        if (g.lane == 0) atomicMax(sc->max_err_bits, __float_as_uint(fail && !(e > 0.f) ? INFINITY : e));
    }
    // also orders the reductions (and the check's reads of the moment-arm region) before the
    // next phase
    return (g.any(bad) ? 1u : 0u) | (fail ? 2u : 0u);
}

// ------------------------------------------------------------------ phase 5: contact
template <int MODE, int WPE>
__device__ void phase_contact(const Tables& T, float* ws, const Grp<WPE>& g, float dt, const EvalPtrs* ev) {
    const ImgHeader& H = *T.H;
    if (H.ns == 0) return;
    auto frame = WS(const float, H.w_frame);
    auto qd = WS(const float, H.w_qd);
    auto S = WS(const float, H.w_S);
    auto Ai = WS(int32_t, H.w_A);
    auto racc = WS(int32_t, H.w_racc);
    auto sph = WS(float, H.w_sph);   // the moment-arm region, free after the muscles
    for (int i = g.lane; i < H.ns; i += g.N) {
        const SphereRec& Sp = T.sph[i];
        const float* fr = frame + 12 * Sp.body;
        float x[3];
        rot3(fr, Sp.pos, x);
        x[0] += fr[9]; x[1] += fr[10]; x[2] += fr[11];
        const float depth = Sp.radius - x[2];
        const float y[3] = {x[0], x[1], x[2] - Sp.radius};   // lowest point of the sphere
        // spatial velocity of the sphere's body from the joint rates, sum of S_d qd_d over the
        // DoFs that move it (root first, as the kinematics pass sums them)
        const DofRec& Dl = T.dof[Sp.last_dof];
        float Vb[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (int j = 0; j <= Dl.depth; ++j) {
            const int d = T.anc[Dl.row + j];
            const float* Sd = S + 6 * d;
            const float qv = qd[d];
#pragma unroll
            for (int k = 0; k < 6; ++k) Vb[k] += Sd[k] * qv;
        }
        float wy[3];
        cross3(Vb, y, wy);
        const float vy[3] = {Vb[3] + wy[0], Vb[4] + wy[1], Vb[5] + wy[2]};
        const float fn = H.contact_k * depth - H.contact_c * vy[2];
        float* o = sph + 12 * i;
        o[0] = y[0]; o[1] = y[1]; o[2] = y[2];
        if (depth > 0.f && fn > 0.f) {
            const float sm = sqrtf(vy[0] * vy[0] + vy[1] * vy[1] + H.contact_eps2);
            const float mfs = H.contact_mu * fn / sm;
            o[3] = -mfs * vy[0]; o[4] = -mfs * vy[1]; o[5] = fn;
            // square roots of dt * damping: A += (h J)^T (h J) per axis
            o[6] = sqrtf(dt * mfs); o[7] = o[6]; o[8] = sqrtf(dt * H.contact_c);
            o[9] = 1.f;
        } else {
            o[3] = o[4] = o[5] = o[6] = o[7] = o[8] = 0.f;
            o[9] = 0.f;
        }
    }
    g.sync();
    for (int i = 0; i < H.ns; ++i) {
        const float* o = sph + 12 * i;
        if (o[9] == 0.f) continue;
        const int dl = T.sph[i].last_dof;
        const int rowl = T.dof[dl].row;
        const int dep = T.dof[dl].depth;
        const int npairs = (dep + 1) * (dep + 2) / 2;
        for (int p0 = g.lane; p0 < npairs; p0 += 2 * g.N) {
            float val[2], tdiag[2];
            int tgt[2], dd[2];
            bool on[2], diag[2];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int p = p0 + g.N * u;
                on[u] = p < npairs;
                const int tv = T.tri[on[u] ? p : 0];
                const int ia = tv & 0xff, ib = tv >> 8;
                const int da = T.anc[rowl + ia], db = T.anc[rowl + ib];
                const float* Sa = S + 6 * da;
                const float* Sb = S + 6 * db;
                const float* oa = frame + 12 * T.dof[da].body + 9;
                const float* ob = frame + 12 * T.dof[db].body + 9;
                const float ra[3] = {o[0] - oa[0], o[1] - oa[1], o[2] - oa[2]};
                const float rb[3] = {o[0] - ob[0], o[1] - ob[1], o[2] - ob[2]};
                float Ja[3], Jb[3];
                cross3(Sa, ra, Ja);
                cross3(Sb, rb, Jb);
                if (H.free_root) {   // a slide of the free root moves the point along its axis
                    if (da < 3) { Ja[0] = Sa[3]; Ja[1] = Sa[4]; Ja[2] = Sa[5]; }
                    if (db < 3) { Jb[0] = Sb[3]; Jb[1] = Sb[4]; Jb[2] = Sb[5]; }
                }
                val[u] = (o[6] * Ja[0]) * (o[6] * Jb[0]) + (o[7] * Ja[1]) * (o[7] * Jb[1]) +
                         (o[8] * Ja[2]) * (o[8] * Jb[2]);
                tgt[u] = T.dof[da].row + ib;
                dd[u] = da;
                diag[u] = ia == ib;
                tdiag[u] = Ja[0] * o[3] + Ja[1] * o[4] + Ja[2] * o[5];
            }
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                if (!on[u]) continue;
                fx_red(&Ai[2 * tgt[u]], val[u]);
                if (diag[u]) {
                    fx_red(&racc[2 * dd[u]], tdiag[u]);
                    if ((MODE == kModeEval) && ev->tau_c) atomicAdd(&ev->tau_c[dd[u]], tdiag[u]);
                }
            }
        }
    }
    g.sync();
}

// ------------------------------------------------------------------ phase 6: limits, damping
template <int MODE, int WPE>
__device__ void phase_limits(const Tables& T, float* ws, const Grp<WPE>& g, float dt, const EvalPtrs* ev) {
    const ImgHeader& H = *T.H;
    auto q = WS(const float, H.w_q);
    auto qd = WS(const float, H.w_qd);
    auto A = WS(fac, H.w_A);
    auto rhs = WS(float, H.w_rhs);
    for (int d = g.lane; d < H.n; d += g.N) {
        const DofRec& D = T.dof[d];
        const float qv = q[d], qdv = qd[d];
        // limit spring-damper on the excess x past the limit, evaluated at the predicted
        // end-of-step state (linearly implicit in position and velocity): spring k_l phi(x),
        // damper c_l psi(x) with a smooth onset over limit_delta (phi = x^2 / (2 delta),
        // psi = x / delta below it; x - delta / 2 and 1 beyond), explicit part to rhs,
        // dt (dt k_l + c_l) psi to the diagonal
        float t = -D.damp * qdv, dd = D.damp;
        if (D.lo < D.hi && (qv > D.hi || qv < D.lo)) {
            const float x = qv > D.hi ? qv - D.hi : D.lo - qv;
            float phi, psi;
            if (x < H.limit_delta) { psi = x / H.limit_delta; phi = 0.5f * x * psi; }
            else { psi = 1.f; phi = x - 0.5f * H.limit_delta; }
            const float spring = H.limit_k * phi, kd = (H.limit_k * dt + H.limit_c) * psi;
            t += (qv > D.hi ? -spring : spring) - kd * qdv;
            dd += kd;
        }
        rhs[d] += t;
        A[D.row + D.depth] = fac_add_f(A[D.row + D.depth], dt * dd);
        if ((MODE == kModeEval) && ev->tau_l) ev->tau_l[d] = t;
    }
    g.sync();
}

// ------------------------------------------------------------------ phase 7-8: factor and solve
// A = L^T L with L lower triangular in the tree pattern (no fill-in), eliminating DoFs leaves
// first, in float-float.  Row k of the packed storage holds (k, ancestor at depth j) at
// row + j; after the factorisation the diagonal slot holds 1 / L_kk.  The right-hand side is
// carried as one more column, so L^T y = rhs is solved during the elimination; L qdd = y
// follows root first, the nodes of a level in parallel.
#ifndef MSIM_ELIM_UNROLL
#define MSIM_ELIM_UNROLL 4
#endif
constexpr int kElimU = MSIM_ELIM_UNROLL;

template <int WPE>
__device__ bool phase_factor_solve(const Tables& T, float* ws, const Grp<WPE>& g) {
    const ImgHeader& H = *T.H;
    auto A = WS(fac, H.w_A);
    auto rhs = WS(const float, H.w_rhs);
    auto Y = WS(fac, H.w_y);
    auto racc = WS(const int32_t, H.w_racc);
    bool ok = true;
    SUB_T0();
    for (int d = g.lane; d < H.n; d += g.N) Y[d] = fac_add_f(fac_decode(racc[2 * d], racc[2 * d + 1]), rhs[d]);
    g.sync();
    for (int l = H.n_dlevels - 1; l >= 0; --l) {
        const int i0 = T.dlevel[l], i1 = T.dlevel[l + 1];
        // pivots of this level (1 / L_kk into the diagonal slots)
        for (int i = i0 + g.lane; i < i1; i += g.N) {
            const uint32_t nd = T.dorder[i];
            const int kk = node_row(nd) + node_depth(nd);
            fac akk = A[kk];
            if (!fac_pos(akk)) { ok = false; akk = fac_one(); }
            A[kk] = fac_rsqrt(akk);
        }
        g.sync();
        SUB_MARK(11);
        // scale rows and rhs of the level's nodes: L_kj = A_kj / L_kk, y_k = b_k / L_kk; four
        // nodes at a time, every load before the first store (entry j of each node per lane)
        for (int c0 = i0; c0 < i1; c0 += 4) {
            for (int j = g.lane; j <= kMaxDepth; j += g.N) {
                fac* ptr[4];
                fac val[4], inv[4];
                bool on[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int i = c0 + u;
                    const uint32_t nd = T.dorder[i < i1 ? i : i0];
                    const int k = node_dof(nd), dep = node_depth(nd), row = node_row(nd);
                    on[u] = i < i1 && j <= dep;
                    ptr[u] = j < dep ? &A[row + j] : &Y[k];
                    inv[u] = A[row + dep];
                    val[u] = on[u] ? *ptr[u] : inv[u];
                }
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (on[u]) *ptr[u] = fac_mul(val[u], inv[u]);
            }
        }
        g.sync();
        SUB_MARK(12);
        // eliminate node by node: A_ab -= L_ka L_kb for ancestors b <= a of k (kElimU independent
        // updates per lane per iteration, loads first), then y_a -= L_ka y_k
        for (int i = i0; i < i1; ++i) {
            const uint32_t nd = T.dorder[i];
            const int k = node_dof(nd), dep = node_depth(nd), row = node_row(nd);
            const int np = dep * (dep + 1) / 2;
            const fac* Lk = A + row;
            // U targets per lane per iteration, U as small as the node's triangle allows (the
            // group's lanes share the node, so the choice is uniform): a shallow node does not
            // issue updates for lanes that have none
            auto eliminate = [&](auto u_count) {
                constexpr int U = decltype(u_count)::value;
                for (int p0 = g.lane; p0 < np; p0 += U * g.N) {
                    fac* tg[U];
                    fac av[U], xv[U], yv[U];
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        const int p = p0 + g.N * u;
                        const int tv = T.tri[p < np ? p : 0];
                        const int ja = tv & 0xff, jb = tv >> 8;      // jb <= ja < depth
                        tg[u] = &A[T.rowanc[row + ja] + jb];
                        xv[u] = Lk[ja];
                        yv[u] = Lk[jb];
                    }
#pragma unroll
                    for (int u = 0; u < U; ++u) av[u] = *tg[u];
#pragma unroll
                    for (int u = 0; u < U; ++u)
                        if (p0 + g.N * u < np) *tg[u] = fac_fms(av[u], xv[u], yv[u]);
                }
            };
            if (np <= g.N) eliminate(std::integral_constant<int, 1>{});
            else if (np <= 2 * g.N) eliminate(std::integral_constant<int, 2>{});
            else eliminate(std::integral_constant<int, kElimU>{});
            const fac yk = Y[k];
            for (int j = g.lane; j < dep; j += g.N) {
                fac* t = &Y[T.anc[row + j]];
                *t = fac_fms(*t, Lk[j], yk);
            }
            g.sync();
        }
        SUB_MARK(13);
    }
    // L x = y, root first (x overwrites y), by columns: once the nodes of depth l are final,
    // every deeper node k subtracts L_{k,a} x_a for its ancestor a of depth l (exactly one per
    // node and level, so the level's updates are independent); a node of depth l + 1 has then
    // received all its terms and is scaled by 1 / L_kk in the same pass.
    const int n_all = T.dlevel[H.n_dlevels];
    for (int i = g.lane; i < T.dlevel[1]; i += g.N) {   // roots
        const uint32_t nd = T.dorder[i];
        Y[node_dof(nd)] = fac_mul(Y[node_dof(nd)], A[node_row(nd) + node_depth(nd)]);
    }
    g.sync();
    for (int l = 0; l + 1 < H.n_dlevels; ++l) {
        const int next_end = T.dlevel[l + 2];
        for (int i = T.dlevel[l + 1] + g.lane; i < n_all; i += g.N) {
            const uint32_t nd = T.dorder[i];
            const int k = node_dof(nd), row = node_row(nd);
            fac y = fac_fms(Y[k], A[row + l], Y[T.anc[row + l]]);
            if (i < next_end) y = fac_mul(y, A[row + node_depth(nd)]);   // depth l + 1: complete
            Y[k] = y;
        }
        g.sync();
    }
    SUB_MARK(14);
    return g.all(ok);
}

// Free root: the rotation vector r of the orientation after a step with world angular velocity
// w, R <- exp(dt w) R, by unit quaternions (product of the step's rotation and the current one,
// sign chosen so that the angle stays in [0, pi]).
__device__ void free_root_turn(float* r, const float* w, float dt) {
    auto quat = [](float x, float y, float z, float o[4]) {
        const float t = sqrtf(x * x + y * y + z * z);
        float sh, ch;
        sincosf(0.5f * t, &sh, &ch);
        const float k = t > 1e-20f ? sh / t : 0.5f;
        o[0] = ch; o[1] = k * x; o[2] = k * y; o[3] = k * z;
    };
    float a[4], b[4], c[4];
    quat(r[0], r[1], r[2], a);
    quat(dt * w[0], dt * w[1], dt * w[2], b);
    c[0] = b[0] * a[0] - b[1] * a[1] - b[2] * a[2] - b[3] * a[3];
    c[1] = b[0] * a[1] + b[1] * a[0] + b[2] * a[3] - b[3] * a[2];
    c[2] = b[0] * a[2] - b[1] * a[3] + b[2] * a[0] + b[3] * a[1];
    c[3] = b[0] * a[3] + b[1] * a[2] - b[2] * a[1] + b[3] * a[0];
    const float sg = c[0] < 0.f ? -1.f : 1.f;
    const float vn = sqrtf(c[1] * c[1] + c[2] * c[2] + c[3] * c[3]);
    const float k = vn > 1e-30f ? 2.f * atan2f(vn, sg * c[0]) * sg / vn : 2.f * sg;
    r[0] = k * c[1]; r[1] = k * c[2]; r[2] = k * c[3];
}

// ------------------------------------------------------------------ one substep
// With MSIM_PHASE_TIMERS defined (profiling builds only), lane 0 of every group adds the
// cycles spent in each phase to timers[0..7].
#ifdef MSIM_PHASE_TIMERS
#define PHASE_MARK(i)                                                                   \
    do {                                                                                \
        const long long t_ = clock64();                                                 \
        if (g.lane == 0 && timers) atomicAdd(&timers[(i)], (unsigned long long)(t_ - t0_)); \
        t0_ = clock64();                                                                \
    } while (0)
#else
#define PHASE_MARK(i) \
    do {              \
    } while (0)
#endif

// Returns the environment status bits; in a surrogate step bit 8 reports a failed cross-check.
template <int MODE, int WPE>
__device__ uint32_t substep(const Tables& T, float* ws, const Grp<WPE>& g, float dt, const float* exc, float* act,
                            float* eps, float* force_out, float* vm_out, const EvalPtrs* ev, const SurrCtx* sc,
                            unsigned long long* timers) {
    const ImgHeader& H = *T.H;
    if (MODE == kModeGeom) {
        phase_kinematics(T, ws, g);
        phase_muscles<kModeGeom>(T, ws, g, dt, exc, act, nullptr, nullptr, nullptr, ev, nullptr);
        return 0u;
    }
    if (MODE == kModeFk) {   // body origins only
        phase_kinematics(T, ws, g);
        auto frame = WS(const float, H.w_frame);
        for (int i = g.lane; i < 3 * H.nb; i += g.N) ev->xpos[i] = frame[12 * (i / 3) + 9 + i % 3];
        return 0u;
    }
#ifdef MSIM_PHASE_TIMERS
    long long t0_ = clock64();
#else
    (void)timers;
#endif
    phase_kinematics(T, ws, g);
    PHASE_MARK(0);
    phase_subtree(T, ws, g);
    PHASE_MARK(1);
    {   // fixed-point accumulator of the damping sums in the A storage (the velocities, bias
        // accelerations and body forces it held are no longer needed); the right-hand side's
        // accumulator already holds -C
        auto Ai = WS(int32_t, H.w_A);
        for (int t = g.lane; t < 2 * H.n_packed; t += g.N) Ai[t] = 0;
    }
    if ((MODE == kModeEval)) {
        auto racc = WS(const int32_t, H.w_racc);
        for (int d = g.lane; d < H.n; d += g.N) {
            const df c = fx_decode(racc[2 * d], racc[2 * d + 1]);
            if (ev->bias) ev->bias[d] = -(c.hi + c.lo);
        }
    }
    g.sync();
    const uint32_t mflags = phase_muscles<MODE>(T, ws, g, dt, exc, act, eps, force_out, vm_out, ev, sc);
    const bool bad = (mflags & 1u) != 0;
    PHASE_MARK(3);
    phase_contact<MODE>(T, ws, g, dt, ev);
    PHASE_MARK(4);
    phase_crba(T, ws, g, (MODE == kModeEval) ? ev->M : nullptr);
    PHASE_MARK(2);
    phase_limits<MODE>(T, ws, g, dt, ev);
    PHASE_MARK(5);
    auto A = WS(const fac, H.w_A);
    if ((MODE == kModeEval)) {
        for (int t = g.lane; t < H.n_packed; t += g.N)
            if (ev->A) ev->A[t] = fac_f(A[t]);
        auto racc = WS(const int32_t, H.w_racc);
        for (int d = g.lane; d < H.n; d += g.N) {
            const df r = df_add_f(fx_decode(racc[2 * d], racc[2 * d + 1]), ws[H.w_rhs + d]);
            if (ev->rhs) ev->rhs[d] = r.hi + r.lo;
        }
        g.sync();
    }
    const bool ok = phase_factor_solve(T, ws, g);
    PHASE_MARK(6);
    uint32_t st = (ok ? 0u : kEnvNotSpd) | (bad ? kEnvNonFinite : 0u) | ((mflags & 2u) ? 0x100u : 0u);
    auto Y = WS(const fac, H.w_y);
    if (!(MODE == kModeEval)) {
        auto q = WS(float, H.w_q);
        auto qd = WS(float, H.w_qd);
        for (int d = g.lane; d < H.n; d += g.N) {
            const float v = qd[d] + dt * fac_f(Y[d]);
            qd[d] = v;
            if (!(H.free_root && d >= 3 && d < 6)) q[d] += dt * v;
        }
        g.sync();
        if (H.free_root) {
            if (g.lane == 0) free_root_turn(q + 3, qd + 3, dt);
            g.sync();
        }
    } else if (ev->qdd) {
        for (int d = g.lane; d < H.n; d += g.N) ev->qdd[d] = fac_f(Y[d]);
    }
    return st;
}

// One environment e through one call (n_sub substeps, or one eval / geometry / learned-geometry
// substep): state row from global memory into the group's workspace, the substeps, state and
// status back.  Every lane of the group calls it.
template <int MODE, int WPE>
__device__ __forceinline__ void run_env(const StepArgs& a, const Tables& T, float* ws, const Grp<WPE>& g, int e) {
    const ImgHeader& H = *T.H;
    const size_t rn = (size_t)e * a.pitch_n, rm = (size_t)e * a.pitch_m;
    for (int i = g.lane; i < H.n; i += g.N) {
        ws[H.w_q + i] = a.q[rn + i];
        ws[H.w_qd + i] = a.qd[rn + i];
    }
    g.sync();
    uint32_t st = 0;
    if ((MODE == kModeEval)) {
        EvalPtrs ev = a.ev;
        auto off = [&](float* p, size_t pitch) { return p ? p + (size_t)e * pitch : p; };
        ev.L = off(ev.L, a.pitch_m); ev.lm = off(ev.lm, a.pitch_m); ev.vm = off(ev.vm, a.pitch_m);
        ev.force = off(ev.force, a.pitch_m); ev.act_next = off(ev.act_next, a.pitch_m);
        ev.R = off(ev.R, ev.nnz_pitch);
        ev.tau_m = off(ev.tau_m, a.pitch_n); ev.tau_c = off(ev.tau_c, a.pitch_n);
        ev.tau_l = off(ev.tau_l, a.pitch_n); ev.bias = off(ev.bias, a.pitch_n); ev.rhs = off(ev.rhs, a.pitch_n);
        ev.qdd = off(ev.qdd, a.pitch_n);
        ev.M = off(ev.M, ev.packed_pitch); ev.A = off(ev.A, ev.packed_pitch);
        ev.eps_next = off(ev.eps_next, a.pitch_m);
        for (int d = g.lane; d < H.n; d += g.N) {
            if (ev.tau_m) ev.tau_m[d] = 0.f;
            if (ev.tau_c) ev.tau_c[d] = 0.f;
            if (ev.tau_l) ev.tau_l[d] = 0.f;
        }
        g.sync();
        st |= substep<kModeEval>(T, ws, g, a.dt, a.exc + rm, a.act + rm, a.eps ? a.eps + rm : nullptr, nullptr,
                                 nullptr, &ev, nullptr, a.timers);
    } else if (MODE == kModeGeom) {
        EvalPtrs ev = a.ev;
        ev.L = a.ev.L + (size_t)(e - a.env_begin) * ev.nnz_pitch;   // label row: L then R
        ev.R = ev.L + H.m;
        substep<kModeGeom>(T, ws, g, a.dt, nullptr, nullptr, nullptr, nullptr, nullptr, &ev, nullptr, a.timers);
    } else if (MODE == kModeFk) {
        EvalPtrs ev = a.ev;
        ev.xpos = a.ev.xpos + (size_t)(e - a.env_begin) * ev.xpos_pitch;
        substep<kModeFk>(T, ws, g, a.dt, nullptr, nullptr, nullptr, nullptr, nullptr, &ev, nullptr, a.timers);
    } else {
        if (is_surr(MODE)) {
            // one substep with the learned geometry (the host loops over substeps)
            bool oob = false;
            for (int d = g.lane; d < H.n; d += g.N)   // a non-finite q counts as outside
                oob |= !(fabsf(ws[H.w_q + d] - a.box_c[d]) <= a.box_s[d]);
            oob = g.any(oob);
            const bool flagged = a.fallback[e] != 0;
            uint32_t c[4] = {(uint32_t)e, *a.step_ctr, 0x73u, 0x75u};
            philox4x32_10(c, a.surr_seed, 0x9e3779b9u);
            SurrCtx sc;
            sc.Y = a.surr_Y + (size_t)(e - a.env_begin) * a.surr_ld;
            sc.colbase = a.surr_colbase;
            sc.use_exact = oob || flagged;
            sc.check = !sc.use_exact && u01_from_bits(c[0]) < a.check_frac;
            sc.tol = a.tol;
            sc.max_err_bits = reinterpret_cast<unsigned int*>(a.surr_stats + 6);
            const uint32_t s1 = substep<MODE>(T, ws, g, a.dt, a.exc + rm, a.act + rm, a.eps ? a.eps + rm : nullptr,
                                                   a.force_out ? a.force_out + rm : nullptr,
                                                   a.vm_out ? a.vm_out + rm : nullptr, nullptr, &sc, a.timers);
            st |= s1 & 0xffu;
            if (g.lane == 0) {
                unsigned long long* cs = a.surr_stats;   // see msim_surrogate_stats
                atomicAdd(&cs[0], 1ull);
                if (!sc.use_exact && !sc.check) atomicAdd(&cs[1], 1ull);
                if (oob) atomicAdd(&cs[2], 1ull);
                if (flagged) atomicAdd(&cs[3], 1ull);
                if (sc.check) atomicAdd(&cs[4], 1ull);
                if (s1 & 0x100u) {
                    atomicAdd(&cs[5], 1ull);
                    a.fallback[e] = 1;   // exact geometry for this environment until its reset
                }
            }
        } else {
            for (int s = 0; s < a.n_sub; ++s) {
                const bool last = (s == a.n_sub - 1);
                st |= substep<MODE == kModeStepW ? kModeStepW : kModeStep>(T, ws, g, a.dt, a.exc + rm, a.act + rm,
                                         a.eps ? a.eps + rm : nullptr,
                                         (last && a.force_out) ? a.force_out + rm : nullptr,
                                         (last && a.vm_out) ? a.vm_out + rm : nullptr, nullptr, nullptr,
                                         a.timers);
            }
        }
        bool bad = false;
        auto Y = WS(const fac, H.w_y);
        for (int d = g.lane; d < H.n; d += g.N) {
            const float v0 = ws[H.w_q + d], v1 = ws[H.w_qd + d];
            bad |= !(isfinite(v0) && isfinite(v1));
            a.q[rn + d] = v0;
            a.qd[rn + d] = v1;
            if (a.qdd_out) a.qdd_out[rn + d] = fac_f(Y[d]);
        }
        for (int k = g.lane; k < H.m; k += g.N) bad |= !isfinite(a.act[rm + k]);
        if (g.any(bad)) st |= kEnvNonFinite;
    }
    if (st && g.lane == 0) {
        atomicOr(&a.env_status[e], st);
        atomicOr(a.gflags, st);
    }
    g.sync();
}

// ------------------------------------------------------------------ kernels
template <int MODE, int WPE>
__global__ void __launch_bounds__(512, 1) k_step(StepArgs a) {
    extern __shared__ __align__(128) uint8_t smem[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
    uint8_t* img = smem + 16;
    if (!stage_image(img, a.img, a.staged_bytes, bar, a.gflags)) return;
#ifdef MSIM_PHASE_TIMERS
    if (threadIdx.x == 0 && blockIdx.x == 0) g_timers = a.timers;
    __syncthreads();
#endif
    Tables T = make_tables(img);
    unstaged_tables(T, a.img, a.stage);
    const ImgHeader& H = *T.H;
    const int warp = threadIdx.x >> 5;
    const int slot = warp / WPE;
    Grp<WPE> g;
    g.wl = threadIdx.x & 31;
    g.wi = warp % WPE;
    g.lane = g.wi * 32 + g.wl;
    g.bar = 1 + slot;
    const int ws_stride = ws_floats(H, WPE);
    float* ws_all = reinterpret_cast<float*>(img + ((a.staged_bytes + 127) & ~127));
    float* ws = ws_all + (size_t)slot * ws_stride;
    const int n_envs = a.env_end - a.env_begin;
    const int n_groups = (n_envs + a.envs_per_block - 1) / a.envs_per_block;
    for (int gi = blockIdx.x; gi < n_groups; gi += gridDim.x) {
        const int e = a.env_begin + gi * a.envs_per_block + slot;
        if (e >= a.env_end) continue;
        run_env<MODE, WPE>(a, T, ws, g, e);
    }
}

// ------------------------------------------------------------------ mixed-model persistent kernel
// All models of a handle in one launch.  Work items (one group of up to `epb` environments of one
// model, n_sub substeps) are taken from a global counter in queue order (models ordered by cost
// per environment, most expensive first, so the cheap items fill the tail).  A block re-stages
// the model image only when its next item belongs to another model.
template <int WPE, int MODE>
__global__ void __launch_bounds__(512, 1) k_step_mixed(MixedArgs ma) {
    extern __shared__ __align__(128) uint8_t smem[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
    int* s_item = reinterpret_cast<int*>(smem + 8);
    uint8_t* img = smem + 16;
    const uint32_t mb = smem_u32(bar);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5;
    const int slot = warp / WPE;
    Grp<WPE> g;
    g.wl = threadIdx.x & 31;
    g.wi = warp % WPE;
    g.lane = g.wi * 32 + g.wl;
    g.bar = 1 + slot;
    float* ws_all = reinterpret_cast<float*>(img + ma.img_region);
    uint32_t phase = 0;
    int cur = -1;
    for (;;) {
        if (threadIdx.x == 0) *s_item = (int)atomicAdd(ma.queue, 1u);
        __syncthreads();
        const int item = *s_item;
        __syncthreads();   // every thread has read the item (and left the previous one's image)
        if (item >= ma.n_items) break;
        int i = 0;
        while (i + 1 < ma.n_models && item >= ma.mdl[i + 1].item_begin) ++i;
        const MixedModel& M = ma.mdl[i];
        if (i != cur) {
            if (threadIdx.x == 0) {
                // the generic-proxy reads of the previous image are ordered before the async copies
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb), "r"(M.staged_bytes)
                             : "memory");
                const uint32_t d = smem_u32(img);
                constexpr int kChunk = 32768;
                for (int off = 0; off < M.staged_bytes; off += kChunk) {
                    const int sz = (M.staged_bytes - off) < kChunk ? (M.staged_bytes - off) : kChunk;
                    asm volatile(
                        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                            d + off),
                        "l"(M.img + off), "r"(sz), "r"(mb)
                        : "memory");
                }
            }
            bool ok = mbar_wait(mb, phase & 1u);
            if (!ok) {
                if (threadIdx.x == 0) atomicOr(ma.a.gflags, kFlagTimeout);
                mbar_wait(mb, phase & 1u);   // a second bounded chance for copies in flight
            }
            ++phase;
            if (!__syncthreads_and(ok)) return;
            cur = i;
        }
        Tables T = make_tables(img);
        unstaged_tables(T, M.img, M.stage);
        float* ws = ws_all + (size_t)slot * ws_floats(*T.H, WPE);
        if (slot < M.epb) {
            const int e = M.env_begin + (item - M.item_begin) * M.epb + slot;
            // a model without wrapping surfaces or compliant tendons takes the variant without
            // those branches, as in its own launch
            if (e < M.env_end) {
                if constexpr (MODE == kModeStepW) {
                    if (!uses_ext(*T.H)) run_env<kModeStep, WPE>(ma.a, T, ws, g, e);
                    else run_env<kModeStepW, WPE>(ma.a, T, ws, g, e);
                } else {
                    run_env<MODE, WPE>(ma.a, T, ws, g, e);
                }
            }
        }
    }
}

__global__ void k_set_l0(uint8_t* img, const float* L, int m) {
    const ImgHeader* H = reinterpret_cast<const ImgHeader*>(img);
    MuscleRec* mus = reinterpret_cast<MuscleRec*>(img + H->o_muscle);
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < m; r += gridDim.x * blockDim.x) mus[r].L0 = L[mus[r].orig];
}

__global__ void k_reset(float* q, float* qd, float* act, float* eps, uint32_t* status, uint8_t* fallback, const float* q0,
                        const float* qd0, const float* act0, const int32_t* ids, int n_rows, int pitch_n, int pitch_m,
                        int n_envs) {
    const int r = blockIdx.x;
    if (r >= n_rows) return;
    const int e = ids ? ids[r] : r;
    if (e < 0 || e >= n_envs) return;
    for (int i = threadIdx.x; i < pitch_n; i += blockDim.x) {
        q[(size_t)e * pitch_n + i] = q0 ? q0[(size_t)r * pitch_n + i] : 0.f;
        qd[(size_t)e * pitch_n + i] = qd0 ? qd0[(size_t)r * pitch_n + i] : 0.f;
    }
    for (int i = threadIdx.x; i < pitch_m; i += blockDim.x)
        act[(size_t)e * pitch_m + i] = act0 ? act0[(size_t)r * pitch_m + i] : 0.f;
    if (eps)
        for (int i = threadIdx.x; i < pitch_m; i += blockDim.x) eps[(size_t)e * pitch_m + i] = 0.f;
    if (threadIdx.x == 0) {
        status[e] = 0u;
        if (fallback) fallback[e] = 0;
    }
}

}  // namespace

size_t step_smem_bytes(const ImgHeader& h, int epb, int stage, int wpe) {
    const size_t staged = (size_t)staged_bytes(h, stage);
    return 16 + ((staged + 127) & ~(size_t)127) + (size_t)epb * ws_floats(h, wpe) * sizeof(float);
}

template <int MODE>
static int step_occ(int threads, size_t smem, int wpe) {
    int n = 0;
    cudaError_t e;
    if (wpe == 4) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step<MODE, 4>, threads, smem);
    else if (wpe == 2) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step<MODE, 2>, threads, smem);
    else e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step<MODE, 1>, threads, smem);
    return e == cudaSuccess ? n : 1;
}

int step_blocks_per_sm(int threads, size_t smem, int wpe, bool wrap) {
    return wrap ? step_occ<kModeStepW>(threads, smem, wpe) : step_occ<kModeStep>(threads, smem, wpe);
}

cudaError_t set_step_smem_limit(size_t bytes) {
    const int b = (int)bytes;
    const void* fns[] = {(const void*)k_step<kModeStep, 1>,        (const void*)k_step<kModeStep, 2>,
                         (const void*)k_step<kModeStep, 4>,        (const void*)k_step<kModeStepW, 1>,
                         (const void*)k_step<kModeStepW, 2>,       (const void*)k_step<kModeStepW, 4>,
                         (const void*)k_step<kModeEval, 1>,        (const void*)k_step<kModeEval, 2>,
                         (const void*)k_step<kModeEval, 4>,        (const void*)k_step<kModeGeom, 1>,
                         (const void*)k_step<kModeGeom, 2>,        (const void*)k_step<kModeFk, 1>,
                         (const void*)k_step<kModeFk, 2>,          (const void*)k_step<kModeSurr, 1>,
                         (const void*)k_step<kModeSurr, 2>,        (const void*)k_step<kModeSurr, 4>,
                         (const void*)k_step<kModeSurrW, 1>,       (const void*)k_step<kModeSurrW, 2>,
                         (const void*)k_step<kModeSurrW, 4>,
                         (const void*)k_step_mixed<1, kModeStep>,  (const void*)k_step_mixed<2, kModeStep>,
                         (const void*)k_step_mixed<4, kModeStep>,  (const void*)k_step_mixed<1, kModeStepW>,
                         (const void*)k_step_mixed<2, kModeStepW>, (const void*)k_step_mixed<4, kModeStepW>};
    for (const void* f : fns) {
        const cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <int MODE>
static void step_launch(const StepArgs& a, int grid, size_t smem, cudaStream_t s) {
    const int threads = 32 * a.wpe * a.envs_per_block;
    if (a.wpe == 4) k_step<MODE, 4><<<grid, threads, smem, s>>>(a);
    else if (a.wpe == 2) k_step<MODE, 2><<<grid, threads, smem, s>>>(a);
    else k_step<MODE, 1><<<grid, threads, smem, s>>>(a);
}

cudaError_t launch_step(const StepArgs& a, int grid, size_t smem, cudaStream_t s) {
    if (a.wrap) step_launch<kModeStepW>(a, grid, smem, s);
    else step_launch<kModeStep>(a, grid, smem, s);
    return cudaGetLastError();
}

template <int MODE>
static void mixed_launch(const MixedArgs& m, int grid, size_t smem, cudaStream_t s) {
    const int threads = 32 * m.a.wpe * m.slots;
    if (m.a.wpe == 4) k_step_mixed<4, MODE><<<grid, threads, smem, s>>>(m);
    else if (m.a.wpe == 2) k_step_mixed<2, MODE><<<grid, threads, smem, s>>>(m);
    else k_step_mixed<1, MODE><<<grid, threads, smem, s>>>(m);
}

cudaError_t launch_mixed(const MixedArgs& m, int grid, size_t smem, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(m.queue, 0, sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    if (m.wrap) mixed_launch<kModeStepW>(m, grid, smem, s);
    else mixed_launch<kModeStep>(m, grid, smem, s);
    return cudaGetLastError();
}

template <int MODE>
static int mixed_occ(int threads, size_t smem, int wpe) {
    int n = 0;
    cudaError_t e;
    if (wpe == 4) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step_mixed<4, MODE>, threads, smem);
    else if (wpe == 2) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step_mixed<2, MODE>, threads, smem);
    else e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step_mixed<1, MODE>, threads, smem);
    return e == cudaSuccess ? n : 0;
}

int mixed_blocks_per_sm(int threads, size_t smem, int wpe, bool wrap) {
    return wrap ? mixed_occ<kModeStepW>(threads, smem, wpe) : mixed_occ<kModeStep>(threads, smem, wpe);
}

cudaError_t launch_eval(const StepArgs& a, int grid, size_t smem, cudaStream_t s) {
    const int threads = 32 * a.wpe * a.envs_per_block;
    if (a.wpe == 4) k_step<kModeEval, 4><<<grid, threads, smem, s>>>(a);
    else if (a.wpe == 2) k_step<kModeEval, 2><<<grid, threads, smem, s>>>(a);
    else k_step<kModeEval, 1><<<grid, threads, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_geom(const StepArgs& a, int grid, size_t smem, cudaStream_t s) {
    const int threads = 32 * a.wpe * a.envs_per_block;
    if (a.wpe == 2) k_step<kModeGeom, 2><<<grid, threads, smem, s>>>(a);
    else k_step<kModeGeom, 1><<<grid, threads, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_fk(const StepArgs& a, int grid, size_t smem, cudaStream_t s) {
    const int threads = 32 * a.wpe * a.envs_per_block;
    if (a.wpe == 2) k_step<kModeFk, 2><<<grid, threads, smem, s>>>(a);
    else k_step<kModeFk, 1><<<grid, threads, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_surr_step(const StepArgs& a, int grid, size_t smem, cudaStream_t s) {
    const int threads = 32 * a.wpe * a.envs_per_block;
    if (a.wrap) {
        if (a.wpe == 4) k_step<kModeSurrW, 4><<<grid, threads, smem, s>>>(a);
        else if (a.wpe == 2) k_step<kModeSurrW, 2><<<grid, threads, smem, s>>>(a);
        else k_step<kModeSurrW, 1><<<grid, threads, smem, s>>>(a);
    } else {
        if (a.wpe == 4) k_step<kModeSurr, 4><<<grid, threads, smem, s>>>(a);
        else if (a.wpe == 2) k_step<kModeSurr, 2><<<grid, threads, smem, s>>>(a);
        else k_step<kModeSurr, 1><<<grid, threads, smem, s>>>(a);
    }
    return cudaGetLastError();
}

__global__ void k_surr_input(const float* q, int pitch_n, int env_begin, int n_envs, const float* c, const float* sc,
                             int n, __nv_bfloat16* X, int ldx, uint32_t* step_ctr) {
    if (step_ctr && blockIdx.x == 0 && threadIdx.x == 0) *step_ctr += 1u;   // read by the next step kernel
    // a warp per row (rows are short), no flat-index division
    const int wpb = blockDim.x >> 5, lane = threadIdx.x & 31;
    for (int r = blockIdx.x * wpb + (threadIdx.x >> 5); r < n_envs; r += gridDim.x * wpb)
        for (int j = lane; j < ldx; j += 32) {
            const float v = j < n ? (q[(size_t)(env_begin + r) * pitch_n + j] - c[j]) / sc[j] : 0.f;
            X[(size_t)r * ldx + j] = __float2bfloat16_rn(v);
        }
}

cudaError_t launch_surr_input(const float* q, int pitch_n, int env_begin, int n_envs, const float* c, const float* sc,
                              int n, __nv_bfloat16* X, int ldx, uint32_t* step_ctr, cudaStream_t s) {
    const int blocks = std::max(1, std::min((n_envs + 7) / 8, 4096));   // eight rows per block
    k_surr_input<<<blocks, 256, 0, s>>>(q, pitch_n, env_begin, n_envs, c, sc, n, X, ldx, step_ctr);
    return cudaGetLastError();
}

cudaError_t launch_set_l0(uint8_t* img, const float* L, int m, cudaStream_t s) {
    k_set_l0<<<(m + 255) / 256, 256, 0, s>>>(img, L, m);
    return cudaGetLastError();
}

cudaError_t launch_reset(float* q, float* qd, float* act, float* eps, uint32_t* status, uint8_t* fallback, const float* q0,
                         const float* qd0, const float* act0, const int32_t* ids, int n_rows, int pitch_n, int pitch_m,
                         int n_envs, cudaStream_t s) {
    if (n_rows <= 0) return cudaSuccess;
    k_reset<<<n_rows, 128, 0, s>>>(q, qd, act, eps, status, fallback, q0, qd0, act0, ids, n_rows, pitch_n, pitch_m,
                                   n_envs);
    return cudaGetLastError();
}

}  // namespace msim

#ifdef MSIM_BOUNDS_CHECK
// Bounds-checking build only (not part of the public ABI in include/msim.h): copies the record of
// out-of-range indices through the kernels' views, [count, source line of the first, its index,
// its extent], to out (host, 4 words) and clears it.  Returns a cudaError_t code.
extern "C" __attribute__((visibility("default"))) int msim_debug_bounds(unsigned int* out) {
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpyFromSymbol(out, msim::g_bounds_rec, 4 * sizeof(unsigned int));
    const unsigned int zero[4] = {0u, 0u, 0u, 0u};
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(msim::g_bounds_rec, zero, sizeof(zero));
    return (int)e;
}
#endif

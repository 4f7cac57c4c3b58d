// gemm_tc.cu -- BF16 x BF16 -> FP32 GEMM on the 5th-generation tensor cores (tcgen05, sm_103a).
//
//   C[m][n] = act( sum_k A[m][k] B[n][k] + bias[n] )
//
// Each operand is read either K-contiguous (A [M][K], B [N][K]) or MN-contiguous (A stored as
// [K][M], B as [K][N]: the MMA's transposed operand mode), so the gradients of an MLP,
// dW = dY^T H and dH = dY W, read the stored activations, gradients and weights as they are.
//
// One 128 x BN output tile per block (two blocks per SM, so one block's epilogue overlaps the
// other's main loop), 192 threads in three roles:
//   warp 0   TMA producer: 2-D tiled bulk copies (128-byte swizzle) of A and B K-slices into a
//            ring of STAGES shared-memory slots, completion counted on the slot's `full` mbarrier;
//   warp 1   allocates BN TMEM columns for the FP32 accumulator; one elected thread issues
//            tcgen05.mma (kind::f16, M = 128, N = BN, K = 16 per instruction, 4 per 64-wide slice)
//            and tcgen05.commit to release each slot (`empty`) and, at the end, the accumulator;
//   warps 2-5 epilogue: tcgen05.ld of their 32 TMEM lanes (32 rows) x 32 columns at a time, bias,
//            activation, then through a padded shared-memory block (the drained operand ring) so
//            that the global stores run along rows, coalesced (FP32 or BF16 output, optionally
//            also the pre-activation in BF16).
// Every wait on an mbarrier is bounded; on expiry the block records an error code, skips its
// stores and still frees its TMEM.  Out-of-range rows / columns of A and B read as zero (TMA
// fill), so M, N and K need not be multiples of the tile; only the row pitches must be multiples
// of 8 elements (16 bytes) and the base addresses 16-byte aligned.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <mutex>

#include "gemm_tc.h"

// operand-ring depth per tile width (compile-time tuning constants)
#ifndef MSIM_GEMM_STAGES_256
#define MSIM_GEMM_STAGES_256 2
#endif
#ifndef MSIM_GEMM_STAGES_128
#define MSIM_GEMM_STAGES_128 3
#endif

namespace msim {
namespace {

constexpr int kBM = 128;
constexpr int kBK = 64;                 // 64 BF16 = 128 bytes = one swizzle row
constexpr int kStage = 36;              // epilogue staging row pitch (floats): 16-byte rows, no bank conflicts
constexpr long long kSpinLimit = 1LL << 24;

__device__ __forceinline__ uint32_t saddr(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(b)), "r"(bytes) : "memory");
}
// bounded parity wait; false if the limit expired
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity) {
    const uint32_t a = saddr(b);
    for (long long i = 0; i < kSpinLimit; ++i) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(a), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            saddr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(saddr(bar))
        : "memory");
}

// Shared-memory matrix descriptor, 128-byte swizzle.  Either layout is built from 1024-byte
// atoms of 8 rows x 128 bytes, as the TMA writes a 64-element-wide box:
//   K-major:  rows along M (N), 64 K-elements per row; 8-row groups 1024 bytes apart (stride
//             byte offset); the leading offset is unused.  A K-step of 16 advances 32 bytes.
//   MN-major: rows along K, 64 M- (N-) elements per row; 8-row K groups 1024 bytes apart (stride
//             byte offset), 64-element M (N) blocks kMnBlock bytes apart (leading byte offset,
//             one TMA box each).  A K-step of 16 advances two groups, 2048 bytes.
constexpr uint32_t kMnBlock = 64 * 64 * 2;   // one 64 (MN) x 64 (K) BF16 box
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lead_bytes) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFF) >> 4);          // start address
    d |= (uint64_t)((lead_bytes >> 4) & 0x3FFF) << 16;   // leading byte offset
    d |= (uint64_t)(1024 >> 4) << 32;                // stride byte offset
    d |= (uint64_t)1 << 46;                          // descriptor version
    d |= (uint64_t)2 << 61;                          // 128-byte swizzle
    return d;
}
// instruction descriptor, kind::f16: BF16 A and B, FP32 accumulator, M x N; bits 15 / 16 select
// the MN-major (transposed) form of A / B
__host__ __device__ constexpr uint32_t instr_desc(int M, int N, int a_mn, int b_mn) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(a_mn & 1) << 15) | ((uint32_t)(b_mn & 1) << 16) |
           ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// exponent clamped so that 1 + e^-x stays below 2^126, the range of the fast divide
__device__ __forceinline__ float act_fn(float x, int act) {
    if (act == 1) return __fdividef(x, 1.f + __expf(fminf(-x, 80.f)));     // SiLU
    if (act == 2) return __fdividef(1.f, 1.f + __expf(fminf(-x, 80.f)));   // sigmoid
    return x;
}

// One warp's 32 rows x 32 columns of values (row = lane) from registers to global memory through
// shared memory: written by rows, read back so that consecutive lanes store consecutive columns.
// FP32: 8 lanes x 16 bytes per row; BF16: 4 lanes x 16 bytes per row.  Columns >= N and rows >= M
// are not stored.
__device__ __forceinline__ void store_block(float* stg, const float (&v)[32], int lane, void* out, int ld, bool bf16,
                                            int row0, int col0, int M, int N, bool vec) {
#pragma unroll
    for (int j = 0; j < 32; j += 4)
        *reinterpret_cast<float4*>(&stg[lane * kStage + j]) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
    __syncwarp();
    if (!bf16) {
        const int rs = lane >> 3, cs = (lane & 7) * 4;
        float* C = reinterpret_cast<float*>(out);
#pragma unroll
        for (int it = 0; it < 8; ++it) {
            const int r = it * 4 + rs, row = row0 + r, col = col0 + cs;
            if (row >= M) continue;
            const float4 w = *reinterpret_cast<const float4*>(&stg[r * kStage + cs]);
            float* dst = C + (size_t)row * ld + col;
            if (vec && col + 4 <= N) {
                *reinterpret_cast<float4*>(dst) = w;
            } else {
                const float a[4] = {w.x, w.y, w.z, w.w};
                for (int j = 0; j < 4 && col + j < N; ++j) dst[j] = a[j];
            }
        }
    } else {
        const int rs = lane >> 2, cs = (lane & 3) * 8;
        __nv_bfloat16* C = reinterpret_cast<__nv_bfloat16*>(out);
#pragma unroll
        for (int it = 0; it < 4; ++it) {
            const int r = it * 8 + rs, row = row0 + r, col = col0 + cs;
            if (row >= M) continue;
            const float4 a = *reinterpret_cast<const float4*>(&stg[r * kStage + cs]);
            const float4 b = *reinterpret_cast<const float4*>(&stg[r * kStage + cs + 4]);
            __nv_bfloat16* dst = C + (size_t)row * ld + col;
            if (vec && col + 8 <= N) {
                uint4 w;
                __nv_bfloat162 h0 = __floats2bfloat162_rn(a.x, a.y), h1 = __floats2bfloat162_rn(a.z, a.w);
                __nv_bfloat162 h2 = __floats2bfloat162_rn(b.x, b.y), h3 = __floats2bfloat162_rn(b.z, b.w);
                w.x = *reinterpret_cast<uint32_t*>(&h0); w.y = *reinterpret_cast<uint32_t*>(&h1);
                w.z = *reinterpret_cast<uint32_t*>(&h2); w.w = *reinterpret_cast<uint32_t*>(&h3);
                *reinterpret_cast<uint4*>(dst) = w;
            } else {
                const float f[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
                for (int j = 0; j < 8 && col + j < N; ++j) dst[j] = __float2bfloat16_rn(f[j]);
            }
        }
    }
    __syncwarp();
}

template <int BN, int kStages>
__global__ void __launch_bounds__(192, 2)
    k_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, GemmArgs p) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    constexpr int kABytes = kBM * kBK * 2, kBBytes = BN * kBK * 2;
    static_assert(kABytes == (kBM / 64) * (int)kMnBlock && kBBytes == (BN / 64) * (int)kMnBlock,
                  "an MN-major stage is whole 64 x 64 boxes");
    uint8_t* sA = smem;
    uint8_t* sB = smem + kStages * kABytes;
    uint64_t* full = reinterpret_cast<uint64_t*>(sB + kStages * kBBytes);
    uint64_t* empty = full + kStages;
    uint64_t* done = empty + kStages;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
    int* failed = reinterpret_cast<int*>(tmem_slot + 1);
    float* sbias = reinterpret_cast<float*>(tmem_slot + 4);   // BN floats
    float* sscale = sbias + BN;                                  // BN floats (with p.scale)
    float* sshift = sscale + BN;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * BN;
    const int ktiles = (p.K + kBK - 1) / kBK;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(done, 1);
        *failed = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(tmem_slot)),
                     "r"(BN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0) {
        // producer
        for (int kt = 0; kt < ktiles; ++kt) {
            const int s = kt % kStages;
            const uint32_t ph = (kt / kStages) & 1;
            if (kt >= kStages && !mbar_wait(&empty[s], ph ^ 1)) {
                atomicExch(failed, 1);
                break;
            }
            mbar_expect_tx(&full[s], kABytes + kBBytes);
            if (p.a_mn) {
                for (int i = 0; i < kBM / 64; ++i)
                    tma_load_2d(sA + s * kABytes + i * kMnBlock, &tmA, m0 + 64 * i, kt * kBK, &full[s]);
            } else {
                tma_load_2d(sA + s * kABytes, &tmA, kt * kBK, m0, &full[s]);
            }
            if (p.b_mn) {
                for (int j = 0; j < BN / 64; ++j)
                    tma_load_2d(sB + s * kBBytes + j * kMnBlock, &tmB, n0 + 64 * j, kt * kBK, &full[s]);
            } else {
                tma_load_2d(sB + s * kBBytes, &tmB, kt * kBK, n0, &full[s]);
            }
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        const uint32_t idesc = instr_desc(kBM, BN, p.a_mn, p.b_mn);
        const uint32_t a_step = p.a_mn ? 2048u : 32u, b_step = p.b_mn ? 2048u : 32u;
        const uint32_t a_lead = p.a_mn ? kMnBlock : 16u, b_lead = p.b_mn ? kMnBlock : 16u;
        for (int kt = 0; kt < ktiles; ++kt) {
            const int s = kt % kStages;
            const uint32_t ph = (kt / kStages) & 1;
            if (!mbar_wait(&full[s], ph)) {
                atomicExch(failed, 1);
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a0 = saddr(sA + s * kABytes), b0 = saddr(sB + s * kBBytes);
#pragma unroll
            for (int kk = 0; kk < kBK / 16; ++kk) {
                const uint64_t ad = smem_desc(a0 + kk * a_step, a_lead), bd = smem_desc(b0 + kk * b_step, b_lead);
                const uint32_t accum = (kt > 0 || kk > 0) ? 1u : 0u;
                asm volatile(
                    "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(idesc), "r"(accum)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             saddr(&empty[s]))
                         : "memory");
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(done))
                     : "memory");
    } else if (warp >= 2) {
        // epilogue: warp w reads TMEM lanes 32 (w % 4) .. +31, i.e. output rows of that quarter;
        // once `done` fired every MMA has completed, so the operand ring is free for staging.
        // The tile's bias goes to shared memory while the main loop runs.
        for (int j = threadIdx.x - 64; j < BN; j += 128) {
            sbias[j] = (p.bias && n0 + j < p.N) ? p.bias[n0 + j] : 0.f;
            if (p.scale) {
                sscale[j] = n0 + j < p.N ? p.scale[n0 + j] : 0.f;
                sshift[j] = n0 + j < p.N ? p.shift[n0 + j] : 0.f;
            }
        }
        asm volatile("bar.sync 1, 128;" ::: "memory");
        const bool ok = mbar_wait(done, 0);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int quarter = warp & 3;
        const int row0 = m0 + quarter * 32;
        if (!ok) atomicExch(failed, 1);
        // warp-uniform: store_block synchronises the warp
        const bool store = __all_sync(0xffffffffu, ok && (*reinterpret_cast<volatile int*>(failed) == 0));
        float* stg = reinterpret_cast<float*>(smem) + quarter * 32 * kStage;
#pragma unroll 1
        for (int c = 0; c < BN; c += 32) {
            uint32_t r[32];
            const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)c;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
                "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                  "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                  "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
                  "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                : "r"(taddr)
                : "memory");
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (!store || n0 + c >= p.N) continue;
            const int cn = n0 + c;
            float v[32], z[32];
#pragma unroll
            for (int j = 0; j < 32; ++j) z[j] = __uint_as_float(r[j]) + sbias[c + j];
            if (p.addend && row0 + lane < p.M) {
                // this lane's row of the addend: 32 consecutive floats (one 128-byte line)
                const float* ad = p.addend + (size_t)(row0 + lane) * p.ld_add + cn;
                if (p.add_vec_ok && cn + 32 <= p.N) {
#pragma unroll
                    for (int j = 0; j < 32; j += 4) {
                        const float4 w = __ldg(reinterpret_cast<const float4*>(ad + j));
                        z[j] += w.x; z[j + 1] += w.y; z[j + 2] += w.z; z[j + 3] += w.w;
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < 32; ++j)
                        if (cn + j < p.N) z[j] += __ldg(ad + j);
                }
            }
#pragma unroll
            for (int j = 0; j < 32; ++j) v[j] = act_fn(z[j], p.act);
            if (p.scale) {
#pragma unroll
                for (int j = 0; j < 32; ++j) v[j] = fmaf(v[j], sscale[c + j], sshift[c + j]);
            }
            store_block(stg, v, lane, p.C, p.ldc, p.c_bf16 != 0, row0, cn, p.M, p.N, p.vec_ok != 0);
            if (p.Z) store_block(stg, z, lane, p.Z, p.ldz, true, row0, cn, p.M, p.N, p.z_vec_ok != 0);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0 && *failed && p.err) atomicOr(p.err, 1u);
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BN) : "memory");
    }
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;

// the driver's tensor-map encoder, looked up once per process (thread-safe)
bool get_encode() {
    std::call_once(g_encode_once, [] {
        cudaDriverEntryPointQueryResult q;
        void* fn = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess && fn)
            g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    });
    return g_encode != nullptr;
}

// 2-D tensor map over a row-major [rows][ld] BF16 matrix with `cols` valid columns; box of
// 64 columns x box_rows rows, 128-byte swizzle, zero fill out of range.  A K-major operand is
// mapped as [M or N][K] with box rows = tile rows, an MN-major one as [K][M or N] with 64-row boxes.
bool make_map(CUtensorMap* m, const void* base, int rows, int cols, int ld, int box_rows) {
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    const cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return g_encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int BN, int kStages>
constexpr size_t gemm_smem() {
    return 1024 + (size_t)kStages * (kBM * kBK * 2 + BN * kBK * 2) + (2 * kStages + 1) * 8 + 16 + 3 * BN * 4;
}
// the epilogue staging (4 warps x 32 rows x kStage floats) reuses the operand ring
static_assert(4 * 32 * kStage * 4 <= 2 * (kBM * kBK * 2 + 128 * kBK * 2), "staging must fit in the ring");

// Per-device launch state: the dynamic shared-memory attribute of each kernel instance is a
// property of the device it was set on, and the tile choice depends on the device's SM count.
// Both are set once per device under a lock (host threads may launch concurrently).
constexpr int kMaxDevices = 64;
std::mutex g_dev_mu;

int current_device() {
    int dev = -1;
    return cudaGetDevice(&dev) == cudaSuccess ? dev : -1;
}

template <int BN, int kStages>
cudaError_t ensure_smem_attr(int dev) {
    static bool done[kMaxDevices] = {};
    std::lock_guard<std::mutex> lock(g_dev_mu);
    if (!done[dev]) {
        const cudaError_t e = cudaFuncSetAttribute(k_gemm<BN, kStages>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)gemm_smem<BN, kStages>());
        if (e != cudaSuccess) return e;
        done[dev] = true;
    }
    return cudaSuccess;
}

int block_slots(int dev) {
    static int slots[kMaxDevices] = {};
    std::lock_guard<std::mutex> lock(g_dev_mu);
    if (!slots[dev]) {
        int sms = 148;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) sms = 148;
        slots[dev] = 2 * sms;
    }
    return slots[dev];
}

template <int BN, int kStages>
cudaError_t launch_bn(const GemmArgs& a, const void* A, int lda, const void* B, int ldb, int dev, cudaStream_t s) {
    CUtensorMap ma, mb;
    const bool okA = a.a_mn ? make_map(&ma, A, a.K, a.M, lda, kBK) : make_map(&ma, A, a.M, a.K, lda, kBM);
    const bool okB = a.b_mn ? make_map(&mb, B, a.K, a.N, ldb, kBK) : make_map(&mb, B, a.N, a.K, ldb, BN);
    if (!okA || !okB) return cudaErrorInvalidValue;
    const cudaError_t e = ensure_smem_attr<BN, kStages>(dev);
    if (e != cudaSuccess) return e;
    dim3 grid((a.N + BN - 1) / BN, (a.M + kBM - 1) / kBM);
    k_gemm<BN, kStages><<<grid, 192, gemm_smem<BN, kStages>(), s>>>(ma, mb, a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t gemm_bf16_tc(const void* A, int lda, const void* B, int ldb, GemmArgs args, cudaStream_t s) {
    if (!get_encode()) return cudaErrorNotSupported;
    if (args.M <= 0 || args.N <= 0 || args.K <= 0) return cudaErrorInvalidValue;
    args.a_mn = args.a_mn ? 1 : 0;
    args.b_mn = args.b_mn ? 1 : 0;
    if ((lda % 8) || (ldb % 8) || (reinterpret_cast<uintptr_t>(A) & 15) || (reinterpret_cast<uintptr_t>(B) & 15))
        return cudaErrorInvalidValue;
    const int vec_align = args.c_bf16 ? 8 : 4;
    args.vec_ok = (args.ldc % vec_align == 0) && ((reinterpret_cast<uintptr_t>(args.C) & 15) == 0);
    args.z_vec_ok = args.Z && (args.ldz % 8 == 0) && ((reinterpret_cast<uintptr_t>(args.Z) & 15) == 0);
    args.add_vec_ok = args.addend && (args.ld_add % 4 == 0) && ((reinterpret_cast<uintptr_t>(args.addend) & 15) == 0);
    // two blocks per SM (<= 113 KB of shared memory and <= 256 TMEM columns each).  Tile width:
    // fewest waves of tiles over the 2 x SMs block slots, a 128-wide tile costing half a 256-wide
    // one; ties go to 256 (more reuse of each A tile)
    const int dev = current_device();
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    const int slots = block_slots(dev);
    const long long mt = (args.M + kBM - 1) / kBM;
    const long long w256 = (mt * ((args.N + 255) / 256) + slots - 1) / slots;
    const long long w128 = (mt * ((args.N + 127) / 128) + slots - 1) / slots;
    if (args.N > 128 && 2 * w256 <= w128) return launch_bn<256, MSIM_GEMM_STAGES_256>(args, A, lda, B, ldb, dev, s);
    return launch_bn<128, MSIM_GEMM_STAGES_128>(args, A, lda, B, ldb, dev, s);
}

}  // namespace msim

// gemm_tc.h -- BF16 tensor-core GEMM (tcgen05) used by the geometry surrogate and the policy MLP.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace msim {

struct GemmArgs {
    int M, N, K;          // C is M x N, reduction over K
    void* C;              // output, row-major, pitch ldc elements
    int ldc;
    int c_bf16;           // 1: BF16 output, 0: FP32 output
    const float* bias;    // optional, [N]
    int act;              // 0: none, 1: SiLU, 2: sigmoid
    void* Z;              // optional BF16 pre-activation output (pitch ldz)
    int ldz;
    uint32_t* err;        // optional device word: bit 0 set if a bounded wait expired
    const float* scale;   // optional, [N]: out = act(...) * scale[n] + shift[n] (FP32 output only)
    const float* shift;   // [N], read when scale is set
    const float* addend;  // optional FP32 [M][ld_add], added to the accumulator with the bias
    int ld_add;
    int a_mn;             // 1: A is stored as [K][M] (M-contiguous, pitch lda) instead of [M][K]
    int b_mn;             // 1: B is stored as [K][N] (N-contiguous, pitch ldb) instead of [N][K]
    int vec_ok;           // set by gemm_bf16_tc
    int z_vec_ok;         // set by gemm_bf16_tc
    int add_vec_ok;       // set by gemm_bf16_tc
};

// C = act(A B^T + bias + addend) (then * scale + shift, per column, if scale is set): A [M][K] BF16 (pitch
// lda; [K][M] with a_mn), B [N][K] BF16 (pitch ldb; [K][N] with b_mn), pitches multiples of 8,
// bases 16-byte aligned.  Asynchronous on stream s.
cudaError_t gemm_bf16_tc(const void* A, int lda, const void* B, int ldb, GemmArgs args, cudaStream_t s);

}  // namespace msim

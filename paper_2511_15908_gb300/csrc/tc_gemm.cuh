// tc_gemm.cuh -- BF16 tensor-core GEMM on sm_103a (tcgen05 + TMEM), FP32 accumulation.
//
//   C[M, N] = A[M, K] * B[N, K]^T      (both operands "row = output index, K = contraction")
//
// One CTA of 128 threads computes a 128 x Nt tile (Nt <= 256, multiple of 16; Nt = 32 when
// M fits one row tile, so that small batches use several SMs).  For every
// 64-wide K chunk the threads convert their part of A and B to BF16 and write it to shared
// memory in the canonical no-swizzle K-major layout (8 x 8 core matrices of 128 bytes:
// rows of a core matrix 16 B apart, core matrices along K 128 B apart = LBO, 8-row groups
// 1024 B apart = SBO); one elected thread issues four K=16 tcgen05.mma into the TMEM
// accumulator and commits them to an mbarrier, which every thread waits on with a bounded
// spin.  The epilogue reads the accumulator with tcgen05.ld (warp w owns TMEM lanes
// 32w..32w+31, i.e. tile rows) and applies a fused per-element operation.
//
// Operands may be stored K-contiguous ([row][k]) or row-contiguous ([k][row]) in global
// memory, as BF16 or FP32; the loader transposes/converts, so the tensor core always sees
// K-major shared-memory operands.
#pragma once
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace sphgb {

constexpr int kTcThreads = 128;
constexpr int kTcM = 128;          // rows per CTA tile (UMMA M)
constexpr int kTcKChunk = 64;      // K per shared-memory stage
constexpr int kTcMaxN = 256;       // columns per CTA tile (UMMA N <= 256)
constexpr int kTcSmallN = 32;      // columns per CTA tile when M fits one row tile
constexpr unsigned kTcSpin = 1u << 22;

enum TcEpilogue : int {
    TC_STORE = 0,        // C = acc                                   (FP32)
    TC_BIAS_GELU = 1,    // Z = acc + bias -> C (FP32); H = gelu(Z) -> aux_out (BF16)
    TC_GELU_GRAD = 2,    // G = acc * gelu'(aux_in) -> aux_out (BF16); C (FP32) optional
    TC_BIAS = 3,         // C = acc + bias                            (FP32)
};

struct TcGemm {
    const void *A;       // M x K
    const void *B;       // N x K
    int lda, ldb;        // leading dimensions in elements
    int a_kcontig, b_kcontig;   // 1: [row][k] storage, 0: [k][row] storage
    int a_f32, b_f32;    // 1: FP32 storage (converted to BF16), 0: BF16 storage
    int M, N, K;         // K multiple of 16 (zero-padded past K by the loader)
    float *C;            // M x N FP32 (ldc), may be null for TC_GELU_GRAD
    int ldc;
    const float *bias;   // N (TC_BIAS_GELU, TC_BIAS)
    const float *aux_in; // M x N FP32 pre-activation Z (TC_GELU_GRAD), ld = ldaux
    __nv_bfloat16 *aux_out;  // M x N BF16 (TC_BIAS_GELU, TC_GELU_GRAD), ld = ldaux
    int ldaux;
    int epilogue;
    unsigned *status;    // ST_TIMEOUT latched when the mbarrier wait gives up
};

// GELU, tanh form: 0.5 z (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3)))
__device__ __forceinline__ float gelu_f(float z)
{
    const float c = 0.7978845608028654f, a = 0.044715f;
    return 0.5f * z * (1.0f + tanhf(c * (z + a * z * z * z)));
}

__device__ __forceinline__ float gelu_grad_f(float z)
{
    const float c = 0.7978845608028654f, a = 0.044715f;
    float t = tanhf(c * (z + a * z * z * z));
    return 0.5f * (1.0f + t) + 0.5f * z * (1.0f - t * t) * c * (1.0f + 3.0f * a * z * z);
}

cudaError_t tc_gemm(const TcGemm &g, cudaStream_t s);

}  // namespace sphgb

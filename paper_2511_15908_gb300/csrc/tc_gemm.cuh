// tc_gemm.cuh -- BF16 tensor-core GEMM on sm_103a (tcgen05 + TMEM + TMA), FP32 accumulation.
//
//   C[M, N] = A[M, K] * B[N, K]^T      (both operands "row = output index, K = contraction")
//
// Both operands are BF16 and K-contiguous in global memory ([row][k], leading dimension a
// multiple of 8 elements, 16-byte aligned base).  One CTA of 128 threads computes a 128 x Nt
// tile (Nt = 256, 128, ..., 16: the widest that still gives kTcMinCtas CTAs, so that the
// small GEMMs of the surrogate spread over many SMs).  The K dimension is walked in 64-wide
// chunks through a 4-stage shared-memory ring:
//   - thread 0 (the producer) waits until a stage is free and has the tensor memory
//     accelerator copy the A and B boxes of the next chunk into it (cp.async.bulk.tensor,
//     128-byte swizzle, rows past M / N and k past K read as zeros), completing on the
//     stage's "full" mbarrier;
//   - thread 32 (the MMA issuer) waits for a full stage, issues four K = 16 tcgen05.mma into
//     the TMEM accumulator and commits them to the stage's "empty" mbarrier, which frees the
//     stage for the producer once the tensor core has read it; after the last chunk it
//     commits to the "done" mbarrier;
//   - every thread waits for "done" and runs the epilogue: tcgen05.ld of its TMEM lane (= tile
//     row), the fused per-element operation, and 16-byte stores of 16 consecutive columns
//     (plus, where asked, a transposed BF16 copy whose stores are coalesced across the warp,
//     and the column sums of the tile's FP32 results: a fixed shuffle tree within each warp,
//     then the four warps in order).
// Every wait is bounded: a wait that gives up latches ST_TIMEOUT in *status and the tile is
// not written.
//
// A K split (ksplit > 1, TC_STORE only) spreads the chunks over grid.z; CTA z writes its
// partial sum to C + z * split_stride, and the caller sums the slices in a fixed order.
#pragma once
#include <atomic>
#include <cstdint>
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace sphgb {

constexpr int kTcThreads = 128;
constexpr int kTcM = 128;          // rows per CTA tile (UMMA M)
constexpr int kTcKChunk = 64;      // K per pipeline stage (one 128-byte swizzle row)
constexpr int kTcMaxN = 256;       // columns per CTA tile (UMMA N <= 256)
constexpr int kTcMinCtas = 64;     // column tiles narrow (to 16) until a GEMM has this many CTAs
constexpr int kTcStages = 4;       // shared-memory ring depth
constexpr unsigned kTcSpin = 1u << 22;

enum TcEpilogue : int {
    TC_STORE = 0,        // C = acc                                   (FP32)
    TC_BIAS_GELU = 1,    // Z = acc + bias -> C (FP32); H = gelu(Z) -> aux_out (BF16)
    TC_GELU_GRAD = 2,    // G = acc * gelu'(aux_in) -> aux_out (BF16); C (FP32) optional
    TC_BIAS = 3,         // C = acc + bias                            (FP32)
};

struct TcGemm {
    const __nv_bfloat16 *A;   // M x K, [row][k], leading dimension lda
    const __nv_bfloat16 *B;   // N x K, [row][k], leading dimension ldb
    int lda, ldb;        // in elements, multiples of 8
    int M, N, K;
    float *C;            // M x N FP32 (ldc), may be null for TC_GELU_GRAD
    int ldc;
    const float *bias;   // N (TC_BIAS_GELU, TC_BIAS)
    const float *aux_in; // M x N FP32 pre-activation Z (TC_GELU_GRAD), ld = ldaux
    __nv_bfloat16 *aux_out;  // M x N BF16 (TC_BIAS_GELU, TC_GELU_GRAD), ld = ldaux
    int ldaux;
    __nv_bfloat16 *aux_out_t;  // optional N x M BF16 transposed copy of aux_out ([col][row])
    int ldaux_t;
    int epilogue;
    float *colsum;       // optional: per row tile, the column sums of the FP32 epilogue values
    int ld_colsum;       // (the values C receives) over the tile's rows: colsum[tile * ld + col]
    int ksplit;          // >= 1; > 1 only with TC_STORE
    size_t split_stride; // elements between the partial slices of C
    unsigned *status;    // ST_TIMEOUT latched when an mbarrier wait gives up
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

// Tensor map of a K-contiguous BF16 operand [rows][K] (leading dimension ld elements, a
// multiple of 8; 16-byte aligned base) for TMA boxes of 64 K x box_rows rows with the
// 128-byte swizzle, elements past rows / K reading as zero; false if the driver refuses it.
bool tc_operand_map(CUtensorMap *map, const __nv_bfloat16 *p, int rows, int K, int ld, int box_rows);

// Opt a kernel into `bytes` of dynamic shared memory on the current device, once per device
// (the attribute is per device; `done` remembers the devices, up to 64, already set).
template <class Kernel>
inline cudaError_t smem_opt_in(Kernel *kernel, int bytes, std::atomic<unsigned long long> &done)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = dev < 64 ? 1ull << dev : 0ull;
    if (bit && (done.load() & bit)) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess && bit) done.fetch_or(bit);
    return e;
}

// Number of K slices tc_gemm writes for g (1 without a split): the caller sums this many.
int tc_gemm_splits(const TcGemm &g);
// cudaErrorInvalidValue when the operands break the layout rules above or the tensor maps
// cannot be built.
cudaError_t tc_gemm(const TcGemm &g, cudaStream_t s);

}  // namespace sphgb

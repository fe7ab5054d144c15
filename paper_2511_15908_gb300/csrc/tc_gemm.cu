// tc_gemm.cu -- tcgen05 BF16 GEMM fed by TMA through an mbarrier ring, with fused
// epilogues (see tc_gemm.cuh for the roles and the layout).
#include <cuda.h>

#include "sph_internal.cuh"
#include "tc_gemm.cuh"
#include "tc_ptx.cuh"

namespace sphgb {

namespace {

using namespace tcx;

constexpr int kStageA = kTcM * kTcKChunk * 2;          // 16 KB: 128 rows x 128 B
constexpr int kStageB = kTcMaxN * kTcKChunk * 2;       // 32 KB: up to 256 rows x 128 B
constexpr int kStageBytes = kStageA + kStageB;
// the ring, 1 KB of slack to align it to the 1024-byte swizzle period, and the barriers
constexpr int kSmemBytes = kTcStages * kStageBytes + 1024 + 256;

// The fused per-element operation of one accumulator value at (row, col); returns the value
// the transposed copy (if any) receives.
__device__ __forceinline__ float epilogue_value(int ep, float acc, float bias, float zin, float &c_out)
{
    switch (ep) {
    case TC_BIAS_GELU: {
        const float z = acc + bias;
        c_out = z;
        return gelu_f(z);
    }
    case TC_GELU_GRAD: {
        const float gz = acc * gelu_grad_f(zin);
        c_out = gz;
        return gz;
    }
    case TC_BIAS: c_out = acc + bias; return 0.0f;
    default: c_out = acc; return 0.0f;
    }
}

__global__ void __launch_bounds__(kTcThreads, 1)
    k_tc_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, TcGemm g,
              int ntile, int box_b, int chunks_per_split)
{
    extern __shared__ unsigned char smem_raw[];
    __shared__ uint32_t s_tmem;
    __shared__ int s_fail;
    __shared__ float s_cs[kTcThreads / 32][16];
    const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
    const uint32_t bar = base + kTcStages * kStageBytes;   // full[S], empty[S], done
    auto full = [&](int s) { return bar + 8u * (uint32_t)s; };
    auto empty = [&](int s) { return bar + 8u * (uint32_t)(kTcStages + s); };
    const uint32_t done = bar + 16u * kTcStages;

    const int m0 = blockIdx.x * kTcM;
    const int n0 = blockIdx.y * ntile;
    const int nt_raw = min(ntile, g.N - n0);
    const int nt = (nt_raw + 15) & ~15;              // UMMA N: multiple of 16
    int ncols = 32;
    while (ncols < nt) ncols <<= 1;                  // TMEM allocation: power of two >= 32
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nk = (g.K + kTcKChunk - 1) / kTcKChunk;
    const int kc0 = blockIdx.z * chunks_per_split;
    const int kc1 = min(nk, kc0 + chunks_per_split);
    const int row = m0 + warp * 32 + lane;
    float *C = g.C ? g.C + (size_t)blockIdx.z * g.split_stride : nullptr;

    if (kc0 >= kc1) {
        // an empty K slice (more slices than chunks): its partial sum is zero
        if (C && row < g.M)
            for (int j = 0; j < nt_raw; ++j) C[(size_t)row * g.ldc + n0 + j] = 0.0f;
        return;
    }

    if (threadIdx.x == 0) {
        s_fail = 0;
        for (int s = 0; s < 2 * kTcStages + 1; ++s) mbar_init(bar + 8u * (uint32_t)s);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(ncols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = s_tmem;

    if (threadIdx.x == 0) {
        // producer: chunk i goes to stage i % S once the MMAs of chunk i - S have read it
        const uint32_t tx = (uint32_t)(kTcM + box_b) * kTcKChunk * 2;
        for (int kc = kc0, i = 0; kc < kc1; ++kc, ++i) {
            const int s = i % kTcStages;
            if (i >= kTcStages && !mbar_wait(empty(s), ((i / kTcStages) & 1) ^ 1)) {
                s_fail = 1;
                break;
            }
            const uint32_t sa = base + (uint32_t)s * kStageBytes;
            mbar_expect_tx(full(s), tx);
            tma_load_2d(sa, &tmA, kc * kTcKChunk, m0, full(s));
            tma_load_2d(sa + kStageA, &tmB, kc * kTcKChunk, n0, full(s));
        }
    } else if (threadIdx.x == 32) {
        // MMA issuer: four K = 16 steps per chunk into the TMEM accumulator
        const uint32_t idesc = instr_desc(nt);
        for (int kc = kc0, i = 0; kc < kc1; ++kc, ++i) {
            const int s = i % kTcStages;
            if (!mbar_wait(full(s), (i / kTcStages) & 1)) {
                s_fail = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t sa = base + (uint32_t)s * kStageBytes, sb = sa + kStageA;
#pragma unroll
            for (int j = 0; j < kTcKChunk / 16; ++j) {
                const uint64_t ad = smem_desc_sw128(sa + 32u * (uint32_t)j);
                const uint64_t bd = smem_desc_sw128(sb + 32u * (uint32_t)j);
                const uint32_t acc = (i > 0 || j > 0) ? 1u : 0u;
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
            }
            mma_commit(empty(s));
        }
        mma_commit(done);                            // fires once every issued MMA completed
    }
    __syncwarp();
    if (!mbar_wait(done, 0)) s_fail = 1;
    asm volatile("tcgen05.fence::after_thread_sync;");
    __syncthreads();
    if (s_fail) {
        if (threadIdx.x == 0 && g.status) atomicOr(g.status, (unsigned)ST_TIMEOUT);
    } else {
        // epilogue: thread = tile row (TMEM lane 32 warp + lane), 16 columns per load
        const int ep = g.epilogue;
        const bool vec_c = C && (g.ldc & 3) == 0 && (reinterpret_cast<uintptr_t>(C) & 15u) == 0;
        const bool vec_aux = (g.ldaux & 7) == 0 && (reinterpret_cast<uintptr_t>(g.aux_out) & 15u) == 0 &&
                             (reinterpret_cast<uintptr_t>(g.aux_in) & 15u) == 0 && (g.ldaux & 3) == 0;
        for (int c0 = 0; c0 < nt; c0 += 16) {
            uint32_t r[16];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
                "%12, %13, %14, %15}, [%16];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                  "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                  "=r"(r[14]), "=r"(r[15])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            float cv[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) cv[j] = 0.0f;
            if (row < g.M && c0 < nt_raw) {
            const int col0 = n0 + c0;
            const bool whole = c0 + 16 <= nt_raw;
            float zin[16], hv[16];
            if (ep == TC_GELU_GRAD) {
                const float *zp = g.aux_in + (size_t)row * g.ldaux + col0;
                if (whole && vec_aux) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const float4 v = __ldg(reinterpret_cast<const float4 *>(zp) + q);
                        zin[4 * q] = v.x; zin[4 * q + 1] = v.y; zin[4 * q + 2] = v.z; zin[4 * q + 3] = v.w;
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < 16; ++j) zin[j] = c0 + j < nt_raw ? zp[j] : 0.0f;
                }
            }
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const float b = (ep == TC_BIAS_GELU || ep == TC_BIAS) && c0 + j < nt_raw ? __ldg(g.bias + col0 + j)
                                                                                         : 0.0f;
                hv[j] = epilogue_value(ep, __uint_as_float(r[j]), b, ep == TC_GELU_GRAD ? zin[j] : 0.0f, cv[j]);
            }
            if (C) {
                float *cp = C + (size_t)row * g.ldc + col0;
                if (whole && vec_c) {
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        reinterpret_cast<float4 *>(cp)[q] =
                            make_float4(cv[4 * q], cv[4 * q + 1], cv[4 * q + 2], cv[4 * q + 3]);
                } else {
                    for (int j = 0; j < 16 && c0 + j < nt_raw; ++j) cp[j] = cv[j];
                }
            }
            if (ep == TC_BIAS_GELU || ep == TC_GELU_GRAD) {
                __nv_bfloat16 *hp = g.aux_out + (size_t)row * g.ldaux + col0;
                __align__(16) __nv_bfloat16 hb[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) hb[j] = __float2bfloat16_rn(hv[j]);
                if (whole && vec_aux) {
                    reinterpret_cast<uint4 *>(hp)[0] = reinterpret_cast<const uint4 *>(hb)[0];
                    reinterpret_cast<uint4 *>(hp)[1] = reinterpret_cast<const uint4 *>(hb)[1];
                } else {
                    for (int j = 0; j < 16 && c0 + j < nt_raw; ++j) hp[j] = hb[j];
                }
                if (g.aux_out_t) {
                    // column-major copy: the lanes of a warp hold consecutive rows
                    for (int j = 0; j < 16 && c0 + j < nt_raw; ++j)
                        g.aux_out_t[(size_t)(col0 + j) * g.ldaux_t + row] = hb[j];
                }
            }
            }
            if (g.colsum && c0 < nt_raw) {
                // the 16 column sums of the warp by a halving exchange: after the xor-16, -8,
                // -4 and -2 steps each lane pair holds one column (lane bits 4..1 pick it)
                const unsigned full = 0xffffffffu;
                float v8[8], v4[4], v2[2];
                const bool h16 = lane & 16, h8 = lane & 8, h4 = lane & 4, h2 = lane & 2;
#pragma unroll
                for (int k = 0; k < 8; ++k)
                    v8[k] = (h16 ? cv[k + 8] : cv[k]) + __shfl_xor_sync(full, h16 ? cv[k] : cv[k + 8], 16);
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    v4[k] = (h8 ? v8[k + 4] : v8[k]) + __shfl_xor_sync(full, h8 ? v8[k] : v8[k + 4], 8);
#pragma unroll
                for (int k = 0; k < 2; ++k)
                    v2[k] = (h4 ? v4[k + 2] : v4[k]) + __shfl_xor_sync(full, h4 ? v4[k] : v4[k + 2], 4);
                float v1 = (h2 ? v2[1] : v2[0]) + __shfl_xor_sync(full, h2 ? v2[0] : v2[1], 2);
                v1 += __shfl_xor_sync(full, v1, 1);
                const int col = (h16 ? 8 : 0) + (h8 ? 4 : 0) + (h4 ? 2 : 0) + (h2 ? 1 : 0);
                if ((lane & 1) == 0) s_cs[warp][col] = v1;
                __syncthreads();
                if (threadIdx.x < 16 && c0 + (int)threadIdx.x < nt_raw) {
                    float t = 0.0f;
                    for (int w = 0; w < kTcThreads / 32; ++w) t += s_cs[w][threadIdx.x];
                    g.colsum[(size_t)blockIdx.x * g.ld_colsum + n0 + c0 + threadIdx.x] = t;
                }
                __syncthreads();
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
    }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return (EncodeTiledFn) nullptr;
        return reinterpret_cast<EncodeTiledFn>(p);
    }();
    return fn;
}

}  // namespace

// Tensor map of a K-contiguous BF16 operand [rows][K] (leading dimension ld elements): boxes
// of 64 K x box_rows rows with the 128-byte swizzle; out-of-range elements read as zero.
bool tc_operand_map(CUtensorMap *map, const __nv_bfloat16 *p, int rows, int K, int ld, int box_rows)
{
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * 2u};
    const cuuint32_t box[2] = {(cuuint32_t)kTcKChunk, (cuuint32_t)box_rows};
    const cuuint32_t estride[2] = {1u, 1u};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16 *>(p), dims, strides, box, estride,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Columns per CTA tile: the widest of 256, 128, ..., 16 that still gives at least
// kTcMinCtas CTAs (row tiles x column tiles x K slices).  These GEMMs are small: a CTA's
// epilogue (one thread per row, one warp per SM sub-partition) is latency bound, so more,
// narrower tiles finish sooner than few wide ones; A is re-read from L2 per column tile.
namespace {

int ntile_of(const TcGemm &g, int slices)
{
    const int mt = (g.M + kTcM - 1) / kTcM;
    int nt = kTcMaxN;
    while (nt > 16 && mt * ((g.N + nt - 1) / nt) * slices < kTcMinCtas) nt >>= 1;
    return nt;
}

// (slices, chunks per slice) of the K split
void split_of(const TcGemm &g, int &slices, int &cps)
{
    const int nk = (g.K + kTcKChunk - 1) / kTcKChunk;
    const int want = (g.ksplit > 1 && g.epilogue == TC_STORE) ? g.ksplit : 1;
    cps = (nk + want - 1) / want;
    slices = want;
}

}  // namespace

int tc_gemm_splits(const TcGemm &g)
{
    int slices, cps;
    split_of(g, slices, cps);
    return slices;
}

cudaError_t tc_gemm(const TcGemm &g, cudaStream_t s)
{
    static std::atomic<unsigned long long> configured{0};
    {
        cudaError_t e = smem_opt_in(k_tc_gemm, kSmemBytes, configured);
        if (e != cudaSuccess) return e;
    }
    if (g.M <= 0 || g.N <= 0 || g.K <= 0) return cudaSuccess;
    if (!g.A || !g.B || (g.lda & 7) || (g.ldb & 7) || g.lda < g.K || g.ldb < g.K ||
        (reinterpret_cast<uintptr_t>(g.A) & 15u) || (reinterpret_cast<uintptr_t>(g.B) & 15u))
        return cudaErrorInvalidValue;
    int slices, cps;
    split_of(g, slices, cps);
    const int ntile = ntile_of(g, slices);
    const int box_b = ntile;
    CUtensorMap ma, mb;
    if (!tc_operand_map(&ma, g.A, g.M, g.K, g.lda, kTcM) || !tc_operand_map(&mb, g.B, g.N, g.K, g.ldb, box_b))
        return cudaErrorInvalidValue;
    dim3 grid((g.M + kTcM - 1) / kTcM, (g.N + ntile - 1) / ntile, slices);
    k_tc_gemm<<<grid, kTcThreads, kSmemBytes, s>>>(ma, mb, g, ntile, box_b, cps);
    return cudaGetLastError();
}

}  // namespace sphgb

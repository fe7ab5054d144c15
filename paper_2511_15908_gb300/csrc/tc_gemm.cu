// tc_gemm.cu -- tcgen05 BF16 GEMM with fused epilogues (see tc_gemm.cuh for the layout).
#include "sph_internal.cuh"
#include "tc_gemm.cuh"

namespace sphgb {

namespace {

constexpr int kABytes = kTcM * kTcKChunk * 2;          // 16 KB
constexpr int kBBytes = kTcMaxN * kTcKChunk * 2;       // 32 KB
// The tile uses 48 KB; the launch reserves a larger window so that every address an
// operand descriptor can form stays inside this CTA's shared memory.
constexpr int kSmemBytes = 160 * 1024;

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor, canonical K-major layout without swizzle:
// start address, LBO (core-matrix stride along K) and SBO (stride between 8-row groups),
// all in 16-byte units; descriptor version 1; layout type 0 (no swizzle).
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1u << 46;
    return d;
}

// Instruction descriptor of kind::f16: D = F32, A = B = BF16, both K-major, N, M = 128.
__device__ __forceinline__ uint32_t instr_desc(int n)
{
    uint32_t d = 0;
    d |= 1u << 4;                          // D format: F32
    d |= 1u << 7;                          // A format: BF16
    d |= 1u << 10;                         // B format: BF16
    d |= (uint32_t)(n >> 3) << 17;         // N / 8
    d |= (uint32_t)(kTcM >> 4) << 24;      // M / 16
    return d;
}

__device__ __forceinline__ void mbar_init(uint32_t addr)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(addr));
    asm volatile("fence.mbarrier_init.release.cluster;");
}

// Bounded wait for the given phase parity; false when it gave up.
__device__ __forceinline__ bool mbar_wait(uint32_t addr, uint32_t parity)
{
    for (unsigned it = 0; it < kTcSpin; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(addr), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ float load_elem(const void *p, int f32, size_t idx)
{
    if (f32) return __ldg(reinterpret_cast<const float *>(p) + idx);
    return __bfloat162float(reinterpret_cast<const __nv_bfloat16 *>(p)[idx]);
}

// Canonical K-major offset (bytes) of element (r, k) inside a [rows x 64] chunk.
__device__ __forceinline__ uint32_t kmajor_off(int r, int k)
{
    return (uint32_t)((((r >> 3) * (kTcKChunk / 8) + (k >> 3)) * 128) + (r & 7) * 16 + (k & 7) * 2);
}

// Load rows [r0, r0 + rows) x K-chunk [k0, k0 + 64) of an operand into shared memory.
// A K-contiguous BF16 operand whose rows start on 16-byte boundaries moves 8 elements (one
// core-matrix row) per 16-byte load, and rows past the operand's end are zero-filled
// without a load; other operands go element by element.  Both write the same bytes.
__device__ __forceinline__ void load_chunk(unsigned char *dst, const void *src, int ld, int kcontig,
                                           int f32, int r0, int rows, int nrows, int k0, int K)
{
    if (kcontig && !f32 && (ld & 7) == 0 && (reinterpret_cast<uintptr_t>(src) & 15u) == 0) {
        const __nv_bfloat16 *b = reinterpret_cast<const __nv_bfloat16 *>(src);
        constexpr int kGroups = kTcKChunk / 8;
        for (int idx = threadIdx.x; idx < rows * kGroups; idx += kTcThreads) {
            const int r = idx / kGroups, k = (idx % kGroups) * 8;
            const int gr = r0 + r, gk = k0 + k;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (gr < nrows && gk < K) {
                const __nv_bfloat16 *row = b + (size_t)gr * ld + gk;
                if (gk + 8 <= K) {
                    v = __ldg(reinterpret_cast<const uint4 *>(row));
                } else {
                    __align__(16) __nv_bfloat16 e[8];
                    for (int j = 0; j < 8; ++j) e[j] = gk + j < K ? row[j] : __float2bfloat16_rn(0.0f);
                    v = *reinterpret_cast<const uint4 *>(e);
                }
            }
            *reinterpret_cast<uint4 *>(dst + kmajor_off(r, k)) = v;
        }
        return;
    }
    if (!kcontig && !f32 && (ld & 7) == 0 && (r0 & 7) == 0 && (rows & 7) == 0 &&
        (reinterpret_cast<uintptr_t>(src) & 15u) == 0) {
        // row-contiguous BF16: 8 rows of one k per 16-byte load, scattered into 8 core-matrix rows
        const __nv_bfloat16 *b = reinterpret_cast<const __nv_bfloat16 *>(src);
        const int groups = rows / 8;
        for (int idx = threadIdx.x; idx < groups * kTcKChunk; idx += kTcThreads) {
            const int r = (idx % groups) * 8, k = idx / groups;
            const int gr = r0 + r, gk = k0 + k;
            __align__(16) __nv_bfloat16 e[8];
            if (gk < K && gr + 8 <= nrows) {
                *reinterpret_cast<uint4 *>(e) = __ldg(reinterpret_cast<const uint4 *>(b + (size_t)gk * ld + gr));
            } else {
                for (int j = 0; j < 8; ++j)
                    e[j] = (gk < K && gr + j < nrows) ? b[(size_t)gk * ld + gr + j] : __float2bfloat16_rn(0.0f);
            }
            for (int j = 0; j < 8; ++j)
                *reinterpret_cast<__nv_bfloat16 *>(dst + kmajor_off(r + j, k)) = e[j];
        }
        return;
    }
    const int total = rows * kTcKChunk;
    for (int idx = threadIdx.x; idx < total; idx += kTcThreads) {
        int r, k;
        if (kcontig) { r = idx / kTcKChunk; k = idx % kTcKChunk; }
        else { k = idx / rows; r = idx % rows; }
        const int gr = r0 + r, gk = k0 + k;
        float v = 0.0f;
        if (gr < nrows && gk < K)
            v = load_elem(src, f32, kcontig ? (size_t)gr * ld + gk : (size_t)gk * ld + gr);
        *reinterpret_cast<__nv_bfloat16 *>(dst + kmajor_off(r, k)) = __float2bfloat16_rn(v);
    }
}

__global__ void __launch_bounds__(kTcThreads, 1) k_tc_gemm(TcGemm g, int ntile)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *sA = smem;
    unsigned char *sB = smem + kABytes;
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem + kABytes + kBBytes);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(smem + kABytes + kBBytes + 16);
    __shared__ int s_fail;

    const int m0 = blockIdx.x * kTcM;
    const int n0 = blockIdx.y * ntile;
    const int nt_raw = min(ntile, g.N - n0);
    const int nt = (nt_raw + 15) & ~15;              // UMMA N: multiple of 16
    int ncols = 32;
    while (ncols < nt) ncols <<= 1;                  // TMEM allocation: power of two >= 32
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        s_fail = 0;
        mbar_init(smem_u32(mbar));
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(ncols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tslot;
    const uint32_t idesc = instr_desc(nt);

    uint32_t phase = 0;
    const int nk = (g.K + kTcKChunk - 1) / kTcKChunk;
    for (int kc = 0; kc < nk; ++kc) {
        const int k0 = kc * kTcKChunk;
        load_chunk(sA, g.A, g.lda, g.a_kcontig, g.a_f32, m0, kTcM, g.M, k0, g.K);
        load_chunk(sB, g.B, g.ldb, g.b_kcontig, g.b_f32, n0, nt, g.N, k0, g.K);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (threadIdx.x == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            const int ksteps = min(kTcKChunk, ((g.K - k0) + 15) & ~15) / 16;
            for (int j = 0; j < ksteps; ++j) {
                const uint64_t ad = smem_desc(smem_u32(sA) + j * 256, 128, 1024);
                const uint64_t bd = smem_desc(smem_u32(sB) + j * 256, 128, 1024);
                const uint32_t acc = (kc > 0 || j > 0) ? 1u : 0u;
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(mbar)));
        }
        if (!mbar_wait(smem_u32(mbar), phase)) {
            s_fail = 1;
            if (g.status) atomicOr(g.status, (unsigned)ST_TIMEOUT);
        }
        phase ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;");
        __syncthreads();
        if (s_fail) break;
    }

    if (!s_fail) {
        // epilogue: thread = tile row (TMEM lane 32 warp + lane), 16 columns per load
        const int row = m0 + warp * 32 + lane;
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
            if (row < g.M) {
                for (int j = 0; j < 16; ++j) {
                    const int col = n0 + c0 + j;
                    if (col >= g.N || c0 + j >= nt_raw) break;
                    float acc = __uint_as_float(r[j]);
                    switch (g.epilogue) {
                    case TC_BIAS_GELU: {
                        float z = acc + g.bias[col];
                        g.C[(size_t)row * g.ldc + col] = z;
                        g.aux_out[(size_t)row * g.ldaux + col] = __float2bfloat16_rn(gelu_f(z));
                        break;
                    }
                    case TC_GELU_GRAD: {
                        float z = g.aux_in[(size_t)row * g.ldaux + col];
                        float gz = acc * gelu_grad_f(z);
                        if (g.C) g.C[(size_t)row * g.ldc + col] = gz;
                        g.aux_out[(size_t)row * g.ldaux + col] = __float2bfloat16_rn(gz);
                        break;
                    }
                    case TC_BIAS: g.C[(size_t)row * g.ldc + col] = acc + g.bias[col]; break;
                    default: g.C[(size_t)row * g.ldc + col] = acc; break;
                    }
                }
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

}  // namespace

cudaError_t tc_gemm(const TcGemm &g, cudaStream_t s)
{
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(k_tc_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    if (g.M <= 0 || g.N <= 0 || g.K <= 0) return cudaSuccess;
    // A single row tile (small batches, e.g. one haptic tick) spreads its columns over
    // CTAs of 32, so that B is loaded by several SMs at once; larger M keeps wide tiles.
    const int ntile = g.M <= kTcM ? kTcSmallN : kTcMaxN;
    dim3 grid((g.M + kTcM - 1) / kTcM, (g.N + ntile - 1) / ntile);
    k_tc_gemm<<<grid, kTcThreads, kSmemBytes, s>>>(g, ntile);
    return cudaGetLastError();
}

}  // namespace sphgb

// tc_ptx.cuh -- inline PTX for the tensor-core kernels on sm_103a: shared-memory matrix and
// instruction descriptors of tcgen05.mma (BF16 x BF16 -> FP32, K-major operands written by
// TMA with the 128-byte swizzle), mbarrier waits with an iteration limit, 2-D tiled TMA
// loads, and the tcgen05 commit.  Used by the GEMM (tc_gemm.cu) and the fused haptic tick
// (sph_mlp.cu).
#pragma once
#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

#include "tc_gemm.cuh"

namespace sphgb {
namespace tcx {

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor of a K-major operand written by TMA with the 128-byte
// swizzle: rows of 128 bytes (64 BF16 of K), 8-row groups 1024 bytes apart (SBO); the
// leading-byte offset is unused for a swizzled K-major operand whose K step stays inside
// one 128-byte row (encoded as 1); descriptor version 1 (bit 46); swizzle mode 2 = 128 B.
// The K = 16 steps inside a chunk advance the start address by 32 bytes: the hardware
// applies the swizzle to the absolute address bits, so the offset composes with it.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)1u << 16;
    d |= (uint64_t)(1024u >> 4) << 32;
    d |= (uint64_t)1u << 46;
    d |= (uint64_t)2u << 61;
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
}

// Bounded wait for the completion of the phase with the given parity; false when it gave up.
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

__device__ __forceinline__ void mbar_expect_tx(uint32_t addr, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(addr), "r"(bytes) : "memory");
}

// 2-D tiled TMA load of the box at (x = k, y = row) into shared memory, completing on mbar.
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t mbar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(mbar)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}


// D (TMEM) [+]= A (smem descriptor) x B (smem descriptor)^T, kind::f16 (BF16 operands)
__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}

// 16 consecutive FP32 columns of the calling thread's TMEM lane (32x32b shape), waited for
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t r[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
        "%12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

}  // namespace tcx
}  // namespace sphgb

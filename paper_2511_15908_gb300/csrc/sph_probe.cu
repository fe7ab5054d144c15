// sph_probe.cu -- measurement hook: the FP32 FMA throughput of the GPU this library runs on,
// the ALU peak the density and force passes are reported against.  Not part of the method.
#include <cuda_runtime.h>

#include "sph.h"

namespace {

constexpr int kChains = 8;        // independent FMA chains per thread (hide the FMA latency)
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) k_fma_peak(int iters, float b, float c, float *sink)
{
    float a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = (float)(threadIdx.x + k);
#pragma unroll 1
    for (int i = 0; i < iters; i += 16) {
#pragma unroll
        for (int u = 0; u < 16; ++u)
#pragma unroll
            for (int k = 0; k < kChains; ++k) a[k] = __fmaf_rn(a[k], b, c);
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    if (s == 1.2345f) sink[threadIdx.x] = s;     // never true for the arguments used; keeps the work
}

}  // namespace

extern "C" sph_status sph_measure_fp32_fma(void *cuda_stream, int32_t blocks, int32_t iters, float *d_sink,
                                           double *out_flops)
{
    if (blocks <= 0 || iters <= 0 || (iters & 15) || !d_sink || !out_flops) return SPH_ERR_ARG;
    k_fma_peak<<<blocks, kThreads, 0, (cudaStream_t)cuda_stream>>>(iters, 0.999999f, 1e-7f, d_sink);
    *out_flops = 2.0 * kChains * (double)iters * (double)blocks * kThreads;
    return cudaGetLastError() == cudaSuccess ? SPH_OK : SPH_ERR_CUDA;
}

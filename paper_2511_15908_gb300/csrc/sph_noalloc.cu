// sph_noalloc.cu -- the spatial-hash sort for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at all: an engine plugin whose device memory belongs
// to the host engine's allocator, a real-time haptic loop that forbids allocation after
// start-up, code that runs while a stream is being captured into a CUDA graph (where
// cudaMalloc is not allowed).  sph_cell_sort_noalloc gives them the cell keys, the stable
// sorted order and the cell ranges of a particle set (the same result as a substep's
// spatial hash) without the library allocating anything: the caller passes inputs and
// outputs, and the per-cell counters and per-particle ranks live in one file-scope device
// array of fixed size that every GPU loading this library holds until the process exits.
#include <cmath>
#include <cstring>
#include <mutex>

#include "sph.h"
#include "sph_device.cuh"

namespace sphgb {

namespace {

// scratch layout (32-bit words): cnt[max_cells + 1] | tile_sum[max tiles] | key[max_n] |
// rank[max_n] | perm[max_n] | status[4]
constexpr size_t kNaMaxTiles = (SPH_NOALLOC_MAX_CELLS + kScanTile - 1) / kScanTile;
constexpr size_t kNaWords = (size_t)SPH_NOALLOC_MAX_CELLS + 1 + kNaMaxTiles + 3 * (size_t)SPH_NOALLOC_MAX_PARTICLES + 4;

static __device__ __align__(256) uint32_t g_noalloc_scratch[kNaWords];

__global__ void k_na_hash(SimConst c)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= c.n) return;
    uint32_t bad = 0;
    int cx, cy, cz;
    cell_of(c, c.xB[e], cx, cy, cz, bad);
    const uint32_t k = (uint32_t)((cz * c.ny + cy) * c.nx + cx);
    c.key[e] = k;
    c.rank[e] = atomicAdd(c.cnt + k, 1u);
    report(c, bad);
}

__global__ void k_na_scan_tiles(SimConst c) { scan_tiles_item(c, blockIdx.x); }
__global__ void k_na_scan_apply(SimConst c) { scan_apply_item(c, blockIdx.x); }
__global__ void k_na_scatter(SimConst c) { scatter_item(c, blockIdx.x); }

// Stable order inside each cell: particle e goes to cell_start + #{members with smaller e}.
// A cell of more than kMaxCell (512) particles takes the atomic claim order instead: still
// a permutation with the keys ascending, but ties in that cell are not in input order.
__global__ void k_na_rank(SimConst c, uint32_t *keys_out, int *order_out)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= c.n) return;
    const uint32_t e = c.perm[p];
    const uint32_t k = c.key[e];
    const int cs = (int)c.cell_start[k], ce = (int)c.cell_start[k + 1];
    int dst;
    if (ce - cs <= kMaxCell) {
        int r = 0;
        for (int q = cs; q < ce; ++q) r += (c.perm[q] < e);
        dst = cs + r;
    } else {
        dst = cs + (int)c.rank[e];
        atomicOr(c.status, (uint32_t)ST_CAPACITY);
    }
    keys_out[dst] = k;
    order_out[dst] = (int)e;
}

// Device address of the scratch array, looked up once per device.
uint32_t *g_scratch_ptr[64] = {};
std::mutex g_scratch_mu;

cudaError_t scratch_for_current_device(uint32_t **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = reinterpret_cast<uint32_t *>(p);
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace

}  // namespace sphgb

using namespace sphgb;

extern "C" sph_status sph_cell_sort_noalloc(const sph_params *p, const float *d_xyzm, int32_t n,
                                            uint32_t *d_keys, int32_t *d_order, uint32_t *d_cell_start,
                                            void *cuda_stream)
{
    if (!p || n < 0 || (n > 0 && (!d_xyzm || !d_keys || !d_order)) || !d_cell_start) return SPH_ERR_ARG;
    if (!(p->cell > 0.0f)) return SPH_ERR_ARG;
    if (((uintptr_t)d_xyzm & 15u) != 0) return SPH_ERR_ARG;      // float4 loads
    if (n > SPH_NOALLOC_MAX_PARTICLES) return SPH_ERR_CAPACITY;
    // grid exactly as sph_create builds it: origin lo - cell, floor((hi - o) / cell) + 2 cells
    SimConst c;
    std::memset(&c, 0, sizeof c);
    const float inv = 1.0f / p->cell;
    int dims[3];
    for (int a = 0; a < 3; ++a) {
        c.o[a] = p->domain_lo[a] - p->cell;
        if (!(p->domain_hi[a] > p->domain_lo[a])) return SPH_ERR_ARG;
        // range-checked in floating point before the conversion (a huge domain or a tiny
        // cell gives a count beyond int, or infinity)
        const float u = (p->domain_hi[a] - c.o[a]) * inv;
        if (!(u >= 0.0f && u < (float)SPH_NOALLOC_MAX_CELLS)) return SPH_ERR_CAPACITY;
        dims[a] = (int)std::floor(u) + 2;
        if (dims[a] > SPH_NOALLOC_MAX_CELLS) return SPH_ERR_CAPACITY;
    }
    const long long ncell = (long long)dims[0] * dims[1] * dims[2];
    if (ncell > SPH_NOALLOC_MAX_CELLS) return SPH_ERR_CAPACITY;
    uint32_t *s = nullptr;
    if (scratch_for_current_device(&s) != cudaSuccess) return SPH_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    c.n = n;
    c.nf = n;
    c.nx = dims[0]; c.ny = dims[1]; c.nz = dims[2]; c.ncell = (int)ncell;
    c.inv_cell = inv;
    c.n_scan_tiles = (int)((ncell + kScanTile - 1) / kScanTile);
    c.xB = reinterpret_cast<float4 *>(const_cast<float *>(d_xyzm));
    c.cnt = s;
    c.tile_sum = s + SPH_NOALLOC_MAX_CELLS + 1;
    c.key = c.tile_sum + kNaMaxTiles;
    c.rank = c.key + SPH_NOALLOC_MAX_PARTICLES;
    c.perm = c.rank + SPH_NOALLOC_MAX_PARTICLES;
    c.status = c.perm + SPH_NOALLOC_MAX_PARTICLES;
    c.cell_start = d_cell_start;
    // the counters and the status words keep the previous call's contents: start from zero
    if (cudaMemsetAsync(c.cnt, 0, 4 * ((size_t)ncell + 1), st) != cudaSuccess) return SPH_ERR_CUDA;
    if (cudaMemsetAsync(c.status, 0, 4 * 4, st) != cudaSuccess) return SPH_ERR_CUDA;
    const int nb = (n + kTile - 1) / kTile;
    if (n > 0) k_na_hash<<<nb, kTile, 0, st>>>(c);
    k_na_scan_tiles<<<c.n_scan_tiles, kTile, 0, st>>>(c);
    k_na_scan_apply<<<c.n_scan_tiles, kTile, 0, st>>>(c);
    if (n > 0) {
        k_na_scatter<<<nb, kTile, 0, st>>>(c);
        k_na_rank<<<nb, kTile, 0, st>>>(c, d_keys, d_order);
    }
    return cudaGetLastError() == cudaSuccess ? SPH_OK : SPH_ERR_CUDA;
}

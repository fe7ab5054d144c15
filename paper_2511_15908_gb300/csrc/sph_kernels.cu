// sph_kernels.cu -- plain path: one launch per substep phase on the handle's stream
// (captured once into a CUDA graph).  The arithmetic lives in sph_device.cuh.
#include "sph_device.cuh"

// Block shape and resident blocks per SM each pass is built for (its register budget).
// Measured on the 1.16 M-particle coupled scene: density in 512-thread blocks, 2 per SM (62
// registers) 305 us, against 317 for 256 x 4, 354 for 256 x 6 (40 registers), 320 for
// 128 x 8 and 316 for 1024 x 1; force in 256-thread blocks, 5 per SM, with two neighbours'
// loads in flight 136 us against 146 at 4 and 158 at 6.  Scenes too small to fill two
// waves of the wide blocks (kDensityWideMin particles) take 256 x 4: on 64 scenes of
// 8k-256k particles the wide blocks alone cost 4 % more.
#ifndef SPH_DENSITY_THREADS
#define SPH_DENSITY_THREADS 512
#endif
#ifndef SPH_DENSITY_MINB
#define SPH_DENSITY_MINB 2
#endif
#ifndef SPH_FORCE_MINB
#define SPH_FORCE_MINB 4
#endif
constexpr int kDensityWideMin = 300000;   // ~ 2 x 152 SMs x 2 blocks x 512 threads
// Low-latency density pass (SPH_FLAG_LOW_LATENCY): G lanes per particle, 32 up to
// kLowLatency32Max particles, else 16.  Measured (density pass, us) on the dam break (12k
// particles) / a compact stirring tank (4.8k) / the coupled scene with 60k fluid (83k):
// one thread 129 / 94 / 154; G = 4: 148 / 81 / 205; G = 8: 67 / 37 / 109; G = 16: 34 / 22
// / 94; G = 32: 25 / 16 / 111 (4 resident blocks; 3 and 2 the same).
#ifndef SPH_LOW_LATENCY_MINB
#define SPH_LOW_LATENCY_MINB 4
#endif
constexpr int kLowLatency32Max = 20000;

namespace sphgb {

__global__ void __launch_bounds__(kTile) k_hash(SimConst c) { hash_item(c, blockIdx.x); }
__global__ void __launch_bounds__(kTile) k_scan_tiles(SimConst c) { scan_tiles_item(c, blockIdx.x); }
__global__ void __launch_bounds__(kTile) k_scan_apply(SimConst c) { scan_apply_item(c, blockIdx.x); }
__global__ void __launch_bounds__(kTile) k_scan_lookback(SimConst c) { scan_lookback_item(c); }
// the substep's scan: single-pass (one launch; timed as the tile pass, the apply pass reads
// ~0) unless built with SPH_SCAN_LOOKBACK=0
#ifndef SPH_SCAN_LOOKBACK
#define SPH_SCAN_LOOKBACK 1
#endif
__global__ void __launch_bounds__(kTile) k_scatter(SimConst c) { scatter_item(c, blockIdx.x); }
__global__ void __launch_bounds__(kTile) k_rank_gather(SimConst c) { rank_gather_item(c, blockIdx.x); }
__global__ void __launch_bounds__(SPH_DENSITY_THREADS, SPH_DENSITY_MINB) k_density(SimConst c)
{
    density_item<SPH_DENSITY_THREADS>(c, blockIdx.x);
}
__global__ void __launch_bounds__(kTile, 4) k_density_narrow(SimConst c) { density_item<kTile>(c, blockIdx.x); }
template <int G>
__global__ void __launch_bounds__(kTile, SPH_LOW_LATENCY_MINB) k_density_coop(SimConst c)
{
    density_coop_item<G>(c, blockIdx.x);
}
#if SPH_DENSITY_BRICK
__global__ void __launch_bounds__(kBrickThreads, 2) k_density_brick(SimConst c)
{
    extern __shared__ __align__(16) unsigned char dsm[];
    density_brick(c, *reinterpret_cast<BrickShared *>(dsm));
}
#endif
__global__ void __launch_bounds__(kTile) k_boundary_volume(SimConst c) { boundary_volume_item(c, blockIdx.x); }
__global__ void __launch_bounds__(kTile, SPH_FORCE_MINB) k_force(SimConst c) { force_item(c, blockIdx.x); }
template <int G>
__global__ void __launch_bounds__(kTile, SPH_FORCE_MINB) k_force_coop(SimConst c)
{
    force_coop_item<G>(c, blockIdx.x);
}
__global__ void __launch_bounds__(kTile) k_wrench(SimConst c) { wrench_item(c, blockIdx.x); }
// the last substep of an update cycle: the cycle's end (the rolling-average log) in the
// block that finished the wrench, after its sums (the same values k_cycle_end would read)
__global__ void __launch_bounds__(kTile) k_wrench_cycle(SimConst c)
{
    if (wrench_item(c, blockIdx.x) && threadIdx.x == 0) cycle_end_item(c);
}
__global__ void k_cycle_end(SimConst c) { cycle_end_item(c); }

__global__ void k_set_grab(SimConst c, int body, int grab, float pv0, float pv1, float pv2,
                           float pv3, float pv4, float pv5, float pv6, float pv7, float pv8,
                           float pv9, float pv10, float pv11, float pv12, float g0, float g1,
                           float g2, int set_pose, int path_n)
{
    const float pv[13] = {pv0, pv1, pv2, pv3, pv4, pv5, pv6, pv7, pv8, pv9, pv10, pv11, pv12};
    for (int b = 0; b < c.nb; ++b) {
        DevBody &B = c.body[b];
        if (b != body) {
            if (grab) B.grabbed = 0;        // one grabbed body at a time
            continue;
        }
        B.grabbed = grab;
        if (!grab) { B.path_n = 0; continue; }
        B.grab_local[0] = g0; B.grab_local[1] = g1; B.grab_local[2] = g2;
        if (set_pose) {
            for (int a = 0; a < 3; ++a) { B.t[a] = pv[a]; B.v[a] = pv[7 + a]; B.w[a] = pv[10 + a]; }
            for (int a = 0; a < 4; ++a) B.q[a] = pv[3 + a];
        }
        B.path_n = path_n;
        B.path_step0 = (int)c.ctr[0];
    }
}

// Cell key and id of each sorted slot (test hook): recomputed from the sorted positions.
__global__ void k_sorted_keys(SimConst c, uint32_t *keys, int *ids)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= c.n) return;
    uint32_t bad = 0;
    int cx, cy, cz;
    cell_of(c, c.xA[p], cx, cy, cz, bad);
    keys[p] = (uint32_t)((cz * c.ny + cy) * c.nx + cx);
    ids[p] = __float_as_int(c.vA[p].w);
}

// ----------------------------------------------------------------------- launchers

static inline int blocks_for(int n, int t) { return (n + t - 1) / t; }

cudaError_t launch_substep(const SimConst &c, cudaStream_t s, cudaEvent_t *ev, bool external,
                           bool cycle_end, unsigned ev_mask)
{
    const int nb = blocks_for(c.n, 256);
    int k = 0;
    auto mark = [&]() {
        if (ev && (ev_mask >> k & 1u)) cudaEventRecordWithFlags(ev[k], s, external ? cudaEventRecordExternal : 0);
        ++k;
    };
    mark();
    k_hash<<<nb, kTile, 0, s>>>(c);
    mark();
    if (SPH_SCAN_LOOKBACK) {
        k_scan_lookback<<<c.n_scan_tiles, kTile, 0, s>>>(c);
        mark();
    } else {
        k_scan_tiles<<<c.n_scan_tiles, kTile, 0, s>>>(c);
        mark();
        k_scan_apply<<<c.n_scan_tiles, kTile, 0, s>>>(c);
    }
    mark();
    k_scatter<<<nb, kTile, 0, s>>>(c);
    mark();
    k_rank_gather<<<nb, kTile, 0, s>>>(c);
    mark();
    // volume-based boundaries: their weights first (timed with the density pass)
    if (c.flags & FLAG_VOLUME) k_boundary_volume<<<nb, kTile, 0, s>>>(c);
#if SPH_DENSITY_BRICK
    static bool brick_attr = false;
    if (!brick_attr) {
        cudaFuncSetAttribute(k_density_brick, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(BrickShared));
        brick_attr = true;
    }
    if (c.n >= kDensityWideMin && !(c.flags & FLAG_VOLUME))
        k_density_brick<<<dim3((c.nx + kBX - 1) / kBX, (c.ny + kBY - 1) / kBY, (c.nz + kBZ - 1) / kBZ), kBrickThreads,
                          sizeof(BrickShared), s>>>(c);
    else
#endif
    // the group's rows fit its 6 x 6 table while Rc < 2.5 (cells >= h give Rc ~ 2)
    if ((c.flags & FLAG_LOW_LATENCY) && !(c.flags & FLAG_VOLUME) && c.Rc < 2.5f && c.n <= kLowLatency32Max)
        k_density_coop<32><<<(unsigned)(((long long)c.n * 32 + kTile - 1) / kTile), kTile, 0, s>>>(c);
    else if ((c.flags & FLAG_LOW_LATENCY) && !(c.flags & FLAG_VOLUME) && c.Rc < 2.5f)
        k_density_coop<16><<<(unsigned)(((long long)c.n * 16 + kTile - 1) / kTile), kTile, 0, s>>>(c);
    else
    if (c.n >= kDensityWideMin)
        k_density<<<blocks_for(c.n, SPH_DENSITY_THREADS), SPH_DENSITY_THREADS, 0, s>>>(c);
    else
        k_density_narrow<<<nb, kTile, 0, s>>>(c);
    mark();
    // (a flagged scene's n_force_blocks counts blocks of 256 / G particles)
    if ((c.flags & FLAG_LOW_LATENCY) && !(c.flags & FLAG_VOLUME))
        k_force_coop<kLowLatencyForceG><<<c.n_force_blocks, kTile, 0, s>>>(c);
    else
        k_force<<<c.n_force_blocks, kTile, 0, s>>>(c);
    mark();
    if (cycle_end) k_wrench_cycle<<<c.n_wgrid, kTile, 0, s>>>(c);
    else k_wrench<<<c.n_wgrid, kTile, 0, s>>>(c);
    mark();
    return cudaGetLastError();
}

__global__ void __launch_bounds__(kTile) k_cut(SimConst c, Blade t, unsigned *count)
{
    cut_item(c, blockIdx.x, t, count);
}

cudaError_t launch_cut(const SimConst &c, cudaStream_t s, const float tri[9], unsigned *count)
{
    Blade t;
    for (int i = 0; i < 9; ++i) t.v[i] = tri[i];
    const int nbody = c.n - c.nf;
    if (nbody <= 0) return cudaSuccess;
    const cudaError_t e = launch_sort(c, s);          // sorted current state + slot_of_id
    if (e != cudaSuccess) return e;
    k_cut<<<blocks_for(nbody, 256), kTile, 0, s>>>(c, t, count);
    return cudaGetLastError();
}

cudaError_t launch_sort(const SimConst &c, cudaStream_t s)
{
    const int nb = blocks_for(c.n, 256);
    k_hash<<<nb, kTile, 0, s>>>(c);
    k_scan_tiles<<<c.n_scan_tiles, kTile, 0, s>>>(c);
    k_scan_apply<<<c.n_scan_tiles, kTile, 0, s>>>(c);
    k_scatter<<<nb, kTile, 0, s>>>(c);
    k_rank_gather<<<nb, kTile, 0, s>>>(c);
    return cudaGetLastError();
}

cudaError_t launch_cycle_end(const SimConst &c, cudaStream_t s)
{
    k_cycle_end<<<1, 1, 0, s>>>(c);
    return cudaGetLastError();
}

cudaError_t launch_set_grab(const SimConst &c, cudaStream_t s, int body, int grab,
                            const float *pv, const float *gl, int set_pose, int path_n)
{
    k_set_grab<<<1, 1, 0, s>>>(c, body, grab, pv[0], pv[1], pv[2], pv[3], pv[4], pv[5], pv[6],
                               pv[7], pv[8], pv[9], pv[10], pv[11], pv[12], gl[0], gl[1], gl[2],
                               set_pose, path_n);
    return cudaGetLastError();
}

cudaError_t launch_sorted_keys(const SimConst &c, cudaStream_t s, uint32_t *keys, int *ids)
{
    k_sorted_keys<<<blocks_for(c.n, 256), 256, 0, s>>>(c, keys, ids);
    return cudaGetLastError();
}

}  // namespace sphgb

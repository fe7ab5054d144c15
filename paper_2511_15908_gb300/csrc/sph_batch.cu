// sph_batch.cu -- many independent scenes of uneven size in ONE persistent launch.
//
// Every scene keeps its own handle and workspace (set up with the single-scene calls).
// The batch uploads each scene's SimConst into a table and runs all phases of a substep
// for all scenes in one cooperative kernel: per phase, blocks take tiles from a global
// work queue (a tile = one scene's 256-particle block, scan tile or reduction block,
// exactly the tiles the single-scene kernels use), and a bounded grid barrier separates
// the phases.  Because the tiles and their arithmetic are the single-scene ones, a
// batched substep is bit-identical to stepping each scene alone.  The launch is captured
// into a CUDA graph; an autotuner picks the resident blocks per SM and the number of tiles
// taken per queue fetch by timing candidate launches.
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "sph.h"
#include "sph_device.cuh"

namespace sphgb {

enum Phase { P_HASH, P_SCAN_T, P_SCAN_A, P_SCATTER, P_GATHER, P_VOLUME, P_DENSITY, P_FORCE, P_WRENCH,
             kPhases };

constexpr unsigned kBarrierSpin = 1u << 22;   // x 64 ns sleep: the barrier gives up after ~0.3 s

struct BatchConst {
    int n_scenes;
    int chunk;                    // tiles per queue fetch
    int total[kPhases];           // tiles of each phase over all scenes
    const int *prefix;            // kPhases x (n_scenes + 1) tile prefix per phase
    const SimConst *scenes;
    unsigned *queue;              // kPhases work-queue counters
    unsigned *bar;                // [0] arrivals, [1] generation
    unsigned *status;             // batch status word (ST_TIMEOUT)
    unsigned spin_limit;
    unsigned expect_extra;        // test hook: arrivals the barrier waits for beyond the grid
};

// Bounded grid barrier: every block arrives once; the last arrival resets the count and
// bumps the generation.  A block that waits longer than spin_limit sleeps latches
// ST_TIMEOUT and returns false, so no launch can hang on a missing block.
__device__ bool grid_barrier(const BatchConst &b)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *gen = b.bar + 1;
        const unsigned g0 = *gen;
        __threadfence();
        const unsigned arrived = atomicAdd(b.bar, 1u) + 1u;
        int ok = 1;
        if (arrived == gridDim.x + b.expect_extra) {
            atomicExch(b.bar, 0u);
            __threadfence();
            atomicAdd(b.bar + 1, 1u);
        } else {
            unsigned it = 0;
            while (*gen == g0) {
                if (++it > b.spin_limit) {
                    ok = 0;
                    atomicOr(b.status, (unsigned)ST_TIMEOUT);
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

__device__ __forceinline__ int scene_of(const int *prefix, int n, int item)
{
    int lo = 0, hi = n;                       // prefix[lo] <= item < prefix[hi]
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (prefix[mid] <= item) lo = mid; else hi = mid;
    }
    return lo;
}

#ifndef SPH_BATCH_MINB
#define SPH_BATCH_MINB 3      // resident blocks per SM the persistent kernel is built for
#endif

// The scene's constants are staged in shared memory for each tile: read through a global
// reference they would be reloaded after every global store (possible aliasing), while
// shared-memory loads cannot alias the particle arrays.
__global__ void __launch_bounds__(kTile, SPH_BATCH_MINB) k_batch(BatchConst b, int n_substeps, int cycle_end)
{
    __shared__ int s_item;
    __shared__ __align__(16) SimConst s_c;
    static_assert(sizeof(SimConst) % 16 == 0, "SimConst is copied as int4");
    int staged = -1;                  // the scene whose constants s_c holds (block-uniform)
    for (int sub = 0; sub < n_substeps; ++sub) {
        for (int ph = 0; ph < kPhases; ++ph) {
            const int *pre = b.prefix + ph * (b.n_scenes + 1);
            for (;;) {
                if (threadIdx.x == 0) s_item = (int)atomicAdd(b.queue + ph, (unsigned)b.chunk);
                __syncthreads();
                const int base = s_item;
                __syncthreads();
                if (base >= b.total[ph]) break;
                const int end = min(base + b.chunk, b.total[ph]);
                for (int it = base; it < end; ++it) {
                    const int s = scene_of(pre, b.n_scenes, it);
                    const int blk = it - pre[s];
                    // consecutive tiles mostly belong to one scene: stage its constants only
                    // when the scene changes (a substep's counter lives in global memory,
                    // so the staged copy stays valid across phases and substeps)
                    if (s != staged) {
                        const int4 *src = reinterpret_cast<const int4 *>(b.scenes + s);
                        int4 *dst = reinterpret_cast<int4 *>(&s_c);
                        for (int w = threadIdx.x; w < (int)(sizeof(SimConst) / 16); w += kTile)
                            dst[w] = __ldg(src + w);
                        staged = s;
                    }
                    __syncthreads();
                    const SimConst &c = s_c;
                    switch (ph) {
                    case P_HASH: hash_item(c, blk); break;
                    case P_SCAN_T: scan_tiles_item(c, blk); break;
                    case P_SCAN_A: scan_apply_item(c, blk); break;
                    case P_SCATTER: scatter_item(c, blk); break;
                    case P_GATHER: rank_gather_item(c, blk); break;
                    case P_VOLUME: boundary_volume_item(c, blk); break;
                    case P_DENSITY: density_item<kTile, false>(c, blk); break;
                    case P_FORCE: force_item(c, blk); break;
                    default: wrench_item(c, blk); break;
                    }
                    __syncthreads();
                }
            }
            if (!grid_barrier(b)) return;
            // nobody fetches from this queue again before the same phase of the next
            // substep, which is several barriers away
            if (blockIdx.x == 0 && threadIdx.x == 0) b.queue[ph] = 0u;
        }
    }
    if (cycle_end && threadIdx.x == 0)
        for (int s = blockIdx.x; s < b.n_scenes; s += gridDim.x) cycle_end_item(b.scenes[s]);
}

// Per-phase alternative: one kernel per phase whose blocks are that phase's tiles over all
// scenes (no grid barrier; each phase keeps its own register budget and occupancy).
// Resident blocks per SM each phase is built for.  Without a bound the density phase took
// 64 registers (4 blocks); 5 blocks give 51 without spilling (6 spill: the scene's
// parameters live in shared memory here), per-phase batch 4.29 -> 3.90 ms on 64 scenes.
template <int PH>
constexpr int batch_phase_minb() { return PH == P_DENSITY ? 4 : PH == P_FORCE ? 3 : 1; }

template <int PH>
__global__ void __launch_bounds__(kTile, batch_phase_minb<PH>()) k_batch_phase(BatchConst b)
{
    __shared__ __align__(16) SimConst s_c;
    const int *pre = b.prefix + PH * (b.n_scenes + 1);
    const int it = blockIdx.x;
    const int s = scene_of(pre, b.n_scenes, it);
    const int blk = it - pre[s];
    {
        const int4 *src = reinterpret_cast<const int4 *>(b.scenes + s);
        int4 *dst = reinterpret_cast<int4 *>(&s_c);
        for (int w = threadIdx.x; w < (int)(sizeof(SimConst) / 16); w += kTile) dst[w] = __ldg(src + w);
    }
    __syncthreads();
    const SimConst &c = s_c;
    switch (PH) {
    case P_HASH: hash_item(c, blk); break;
    case P_SCAN_T: scan_tiles_item(c, blk); break;
    case P_SCAN_A: scan_apply_item(c, blk); break;
    case P_SCATTER: scatter_item(c, blk); break;
    case P_GATHER: rank_gather_item(c, blk); break;
    case P_VOLUME: boundary_volume_item(c, blk); break;
    case P_DENSITY: density_item<kTile, false>(c, blk); break;
    case P_FORCE: force_item(c, blk); break;
    default: wrench_item(c, blk); break;
    }
}

__global__ void k_batch_cycle_end(BatchConst b)
{
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < b.n_scenes; s += gridDim.x * blockDim.x)
        cycle_end_item(b.scenes[s]);
}

// One barrier and nothing else (exercises the bounded wait of the barrier).
__global__ void __launch_bounds__(kTile) k_batch_barrier_only(BatchConst b) { grid_barrier(b); }

}  // namespace sphgb

using namespace sphgb;

// internal accessor implemented in sph_api.cu
namespace sphgb {
sph_status scene_for_batch(sph_handle *h, SimConst *out);
void scene_advanced(sph_handle *h, int n);
}

constexpr int kBranchStreams = 64;   // scene-graph structure: at most this many branches

struct sph_batch {
    int n = 0;
    std::vector<sph_handle *> handles;
    std::vector<SimConst> table;         // every scene's parameters (host copy)
    char *ws = nullptr;
    cudaStream_t stream = nullptr;
    BatchConst bc;
    // bps > 0: the persistent kernel; 0: one kernel per phase over all scenes' tiles;
    // -1: every scene's own substep kernels as parallel branches of one graph
    int sms = 0, max_bps = 0, bps = 0;
    cudaStream_t branch[kBranchStreams] = {};
    cudaEvent_t fork = nullptr, join[kBranchStreams] = {};
    int n_branches = 0;
    std::vector<int> branch_of;          // scene -> branch, balanced by particle count
    cudaGraphExec_t exec1 = nullptr, exec16 = nullptr;
    bool use_graph = true;
    std::string err;
};

namespace {

size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

struct BatchLayout {
    size_t scenes, prefix, queue, bar, status, total;
};

BatchLayout batch_layout(int n)
{
    BatchLayout L;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t r = off; off = a256(off + bytes); return r; };
    L.scenes = take(sizeof(SimConst) * (size_t)n);
    L.prefix = take(4 * (size_t)kPhases * (n + 1));
    L.queue = take(4 * kPhases);
    L.bar = take(8);
    L.status = take(4);
    L.total = off;
    return L;
}

sph_status bfail(sph_batch *b, sph_status s, const std::string &m)
{
    if (b) b->err = m;
    return s;
}

#define BATCH_CUDA(b, call)                                                         \
    do {                                                                            \
        cudaError_t e_ = (call);                                                    \
        if (e_ != cudaSuccess)                                                      \
            return bfail((b), SPH_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

cudaError_t launch_phases(sph_batch *b, int n_substeps, int cycle_end)
{
    const BatchConst &bc = b->bc;
    for (int i = 0; i < n_substeps; ++i) {
        if (bc.total[P_HASH]) k_batch_phase<P_HASH><<<bc.total[P_HASH], kTile, 0, b->stream>>>(bc);
        if (bc.total[P_SCAN_T]) k_batch_phase<P_SCAN_T><<<bc.total[P_SCAN_T], kTile, 0, b->stream>>>(bc);
        if (bc.total[P_SCAN_A]) k_batch_phase<P_SCAN_A><<<bc.total[P_SCAN_A], kTile, 0, b->stream>>>(bc);
        if (bc.total[P_SCATTER]) k_batch_phase<P_SCATTER><<<bc.total[P_SCATTER], kTile, 0, b->stream>>>(bc);
        if (bc.total[P_GATHER]) k_batch_phase<P_GATHER><<<bc.total[P_GATHER], kTile, 0, b->stream>>>(bc);
        if (bc.total[P_VOLUME]) k_batch_phase<P_VOLUME><<<bc.total[P_VOLUME], kTile, 0, b->stream>>>(bc);
        if (bc.total[P_DENSITY]) k_batch_phase<P_DENSITY><<<bc.total[P_DENSITY], kTile, 0, b->stream>>>(bc);
        if (bc.total[P_FORCE]) k_batch_phase<P_FORCE><<<bc.total[P_FORCE], kTile, 0, b->stream>>>(bc);
        if (bc.total[P_WRENCH]) k_batch_phase<P_WRENCH><<<bc.total[P_WRENCH], kTile, 0, b->stream>>>(bc);
    }
    if (cycle_end) k_batch_cycle_end<<<(bc.n_scenes + 127) / 128, 128, 0, b->stream>>>(bc);
    return cudaGetLastError();
}

// Scene-graph structure: the batch stream forks into one stream per scene (up to
// kBranchStreams; with more scenes, the largest go first to the least-loaded branch), each
// scene's substep kernels (the single-scene kernels, parameters in the constant bank) run
// on its branch, and the branches join back before the cycle end.  Captured, this is one
// graph whose branches the GPU runs side by side; a substep lasts as long as its most
// loaded branch, hence the balancing.
cudaError_t launch_branches(sph_batch *b, int n_substeps, int cycle_end)
{
    cudaError_t e = cudaSuccess;
    if (!b->fork) {
        b->n_branches = std::min(b->n, kBranchStreams);
        std::vector<int> order(b->n);
        for (int sc = 0; sc < b->n; ++sc) order[sc] = sc;
        std::stable_sort(order.begin(), order.end(),
                         [&](int x, int y) { return b->table[x].n > b->table[y].n; });
        std::vector<long long> load(b->n_branches, 0);
        b->branch_of.assign(b->n, 0);
        for (int sc : order) {
            const int k = (int)(std::min_element(load.begin(), load.end()) - load.begin());
            b->branch_of[sc] = k;
            load[k] += b->table[sc].n;
        }
        e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
        for (int k = 0; e == cudaSuccess && k < b->n_branches; ++k) {
            e = cudaStreamCreateWithFlags(&b->branch[k], cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join[k], cudaEventDisableTiming);
        }
        if (e != cudaSuccess) return e;
    }
    if (n_substeps > 0) {
        e = cudaEventRecord(b->fork, b->stream);
        for (int k = 0; e == cudaSuccess && k < b->n_branches; ++k)
            e = cudaStreamWaitEvent(b->branch[k], b->fork, 0);
        for (int sc = 0; e == cudaSuccess && sc < b->n; ++sc)
            for (int i = 0; e == cudaSuccess && i < n_substeps; ++i)
                e = launch_substep(b->table[sc], b->branch[b->branch_of[sc]]);
        for (int k = 0; e == cudaSuccess && k < b->n_branches; ++k) {
            e = cudaEventRecord(b->join[k], b->branch[k]);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->join[k], 0);
        }
        if (e != cudaSuccess) return e;
    }
    if (cycle_end) k_batch_cycle_end<<<(b->bc.n_scenes + 127) / 128, 128, 0, b->stream>>>(b->bc);
    return cudaGetLastError();
}

cudaError_t launch_batch(sph_batch *b, int n_substeps, int cycle_end)
{
    if (b->bps < 0) return launch_branches(b, n_substeps, cycle_end);
    if (b->bps == 0) return launch_phases(b, n_substeps, cycle_end);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(b->bps * b->sms));
    cfg.blockDim = dim3(kTile);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = b->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_batch, b->bc, n_substeps, cycle_end);
}

sph_status capture_batch(sph_batch *b, int n_substeps, cudaGraphExec_t *out)
{
    cudaGraph_t g = nullptr;
    BATCH_CUDA(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t le = launch_batch(b, n_substeps, 0);
    cudaError_t ce = cudaStreamEndCapture(b->stream, &g);
    if (le != cudaSuccess || ce != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return bfail(b, SPH_ERR_CUDA, std::string("batch capture: ") +
                                          cudaGetErrorString(le != cudaSuccess ? le : ce));
    }
    cudaError_t ie = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) return bfail(b, SPH_ERR_CUDA, std::string("batch instantiate: ") + cudaGetErrorString(ie));
    return SPH_OK;
}

void drop_graphs(sph_batch *b)
{
    if (b->exec1) cudaGraphExecDestroy(b->exec1);
    if (b->exec16) cudaGraphExecDestroy(b->exec16);
    b->exec1 = b->exec16 = nullptr;
}

sph_status batch_status(sph_batch *b)
{
    unsigned st = 0;
    BATCH_CUDA(b, cudaMemcpyAsync(&st, b->bc.status, 4, cudaMemcpyDeviceToHost, b->stream));
    BATCH_CUDA(b, cudaStreamSynchronize(b->stream));
    if (st & ST_TIMEOUT) {
        // the barrier state is unknown after a timeout: reset it with the status
        BATCH_CUDA(b, cudaMemsetAsync(b->bc.bar, 0, 8, b->stream));
        BATCH_CUDA(b, cudaMemsetAsync(b->bc.queue, 0, 4 * kPhases, b->stream));
        BATCH_CUDA(b, cudaMemsetAsync(b->bc.status, 0, 4, b->stream));
        BATCH_CUDA(b, cudaStreamSynchronize(b->stream));
        return bfail(b, SPH_ERR_TIMEOUT, "a grid barrier of the batched launch gave up");
    }
    return SPH_OK;
}

}  // namespace

extern "C" {

size_t sph_batch_workspace_bytes(int32_t n_scenes)
{
    if (n_scenes <= 0) return 0;
    return batch_layout(n_scenes).total;
}

sph_status sph_batch_create(sph_handle *const *scenes, int32_t n_scenes, void *d_workspace,
                            size_t bytes, void *cuda_stream, sph_batch **out)
{
    if (!out) return SPH_ERR_ARG;
    *out = nullptr;
    if (!scenes || n_scenes <= 0) return SPH_ERR_ARG;
    BatchLayout L = batch_layout(n_scenes);
    if (!d_workspace || bytes < L.total || ((uintptr_t)d_workspace & 255u)) return SPH_ERR_WORKSPACE;
    std::vector<SimConst> table(n_scenes);
    for (int s = 0; s < n_scenes; ++s) {
        if (!scenes[s]) return SPH_ERR_ARG;
        sph_status st = scene_for_batch(scenes[s], &table[s]);
        if (st != SPH_OK) return st;
        // a small reduction grid per scene: many scenes already fill the GPU
        table[s].n_wgrid = std::max(table[s].n_wblocks, 4);
        // every structure runs one thread per particle in the density pass, so that all of
        // them give the same results (a batch fills the GPU; the low-latency pass is not
        // what it needs)
        table[s].flags &= ~FLAG_LOW_LATENCY;
        table[s].n_force_blocks = (table[s].n + 255) / 256;
    }
    sph_batch *b = new sph_batch();
    b->n = n_scenes;
    b->handles.assign(scenes, scenes + n_scenes);
    b->table = table;
    b->ws = (char *)d_workspace;
    b->stream = (cudaStream_t)cuda_stream;
    BatchConst &bc = b->bc;
    std::memset(&bc, 0, sizeof bc);
    bc.n_scenes = n_scenes;
    bc.chunk = 1;
    bc.spin_limit = kBarrierSpin;
    std::vector<int> prefix((size_t)kPhases * (n_scenes + 1), 0);
    for (int ph = 0; ph < kPhases; ++ph) {
        int run = 0;
        for (int s = 0; s < n_scenes; ++s) {
            prefix[(size_t)ph * (n_scenes + 1) + s] = run;
            const SimConst &c = table[s];
            int tiles = (ph == P_SCAN_T || ph == P_SCAN_A) ? c.n_scan_tiles
                        : (ph == P_WRENCH) ? c.n_wgrid
                        : (ph == P_VOLUME && !(c.flags & FLAG_VOLUME)) ? 0
                        : (c.n + kTile - 1) / kTile;
            run += tiles;
        }
        prefix[(size_t)ph * (n_scenes + 1) + n_scenes] = run;
        bc.total[ph] = run;
    }
    bc.scenes = (const SimConst *)(b->ws + L.scenes);
    bc.prefix = (const int *)(b->ws + L.prefix);
    bc.queue = (unsigned *)(b->ws + L.queue);
    bc.bar = (unsigned *)(b->ws + L.bar);
    bc.status = (unsigned *)(b->ws + L.status);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b->max_bps, k_batch, kTile, 0);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->ws, 0, L.total, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync((void *)bc.scenes, table.data(), sizeof(SimConst) * n_scenes,
                            cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync((void *)bc.prefix, prefix.data(), 4 * prefix.size(), cudaMemcpyHostToDevice,
                            b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess || b->max_bps < 1) {
        delete b;
        return SPH_ERR_CUDA;
    }
    b->bps = b->max_bps;
    *out = b;
    return SPH_OK;
}

sph_status sph_batch_configure(sph_batch *b, int32_t blocks_per_sm, int32_t tiles_per_fetch)
{
    if (!b) return SPH_ERR_ARG;
    if (blocks_per_sm < -1 || blocks_per_sm > b->max_bps || tiles_per_fetch < 1 || tiles_per_fetch > 64)
        return bfail(b, SPH_ERR_ARG, "geometry outside the resident limit");
    if (blocks_per_sm != b->bps || tiles_per_fetch != b->bc.chunk) drop_graphs(b);
    b->bps = blocks_per_sm;
    b->bc.chunk = tiles_per_fetch;
    return SPH_OK;
}

sph_status sph_batch_step(sph_batch *b, int32_t n_substeps)
{
    if (!b || n_substeps < 0) return SPH_ERR_ARG;
    if (n_substeps == 0) return SPH_OK;
    int left = n_substeps;
    if (b->use_graph && b->stream) {
        if (!b->exec1 && capture_batch(b, 1, &b->exec1) != SPH_OK) b->use_graph = false;
        if (b->use_graph && left >= 16 && !b->exec16 && capture_batch(b, 16, &b->exec16) != SPH_OK)
            b->use_graph = false;
    }
    if (b->use_graph && b->stream) {
        for (; left >= 16; left -= 16) BATCH_CUDA(b, cudaGraphLaunch(b->exec16, b->stream));
        for (; left > 0; --left) BATCH_CUDA(b, cudaGraphLaunch(b->exec1, b->stream));
        BATCH_CUDA(b, launch_batch(b, 0, 1));           // end of the update cycle
    } else {
        BATCH_CUDA(b, launch_batch(b, left, 1));
    }
    for (sph_handle *h : b->handles) scene_advanced(h, n_substeps);
    return SPH_OK;
}

sph_status sph_batch_tune(sph_batch *b, int32_t substeps_per_trial, int32_t out_choice[2])
{
    if (!b || substeps_per_trial < 1) return SPH_ERR_ARG;
    cudaEvent_t e0, e1;
    BATCH_CUDA(b, cudaEventCreate(&e0));
    BATCH_CUDA(b, cudaEventCreate(&e1));
    float best = 1e30f;
    int best_bps = b->bps, best_chunk = b->bc.chunk;
    const int chunks[3] = {1, 2, 4};
    int trials = 0;
    for (int bps = -1; bps <= b->max_bps; ++bps)
        for (int ci = 0; ci < (bps <= 0 ? 1 : 3); ++ci) {
            ++trials;
            sph_status st = sph_batch_configure(b, bps, chunks[ci]);
            if (st != SPH_OK) return st;
            BATCH_CUDA(b, launch_batch(b, 1, 0));          // warm-up
            BATCH_CUDA(b, cudaEventRecord(e0, b->stream));
            BATCH_CUDA(b, launch_batch(b, substeps_per_trial, 0));
            BATCH_CUDA(b, cudaEventRecord(e1, b->stream));
            BATCH_CUDA(b, cudaEventSynchronize(e1));
            st = batch_status(b);
            if (st != SPH_OK) return st;
            float ms = 0.0f;
            BATCH_CUDA(b, cudaEventElapsedTime(&ms, e0, e1));
            if (ms < best) { best = ms; best_bps = bps; best_chunk = chunks[ci]; }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    for (sph_handle *h : b->handles) scene_advanced(h, trials * (1 + substeps_per_trial));
    sph_status st = sph_batch_configure(b, best_bps, best_chunk);
    if (out_choice) { out_choice[0] = best_bps; out_choice[1] = best_chunk; }
    return st;
}

sph_status sph_batch_sync(sph_batch *b)
{
    if (!b) return SPH_ERR_ARG;
    return batch_status(b);
}

sph_status sph_batch_info(sph_batch *b, int32_t out[4])
{
    if (!b || !out) return SPH_ERR_ARG;
    out[0] = b->n;
    out[1] = b->sms;
    out[2] = b->bps;
    out[3] = b->bc.chunk;
    return SPH_OK;
}

sph_status sph_batch_test_barrier(sph_batch *b, int32_t missing_blocks, int32_t spin_limit)
{
    if (!b || missing_blocks < 0 || spin_limit < 1) return SPH_ERR_ARG;
    BatchConst bc = b->bc;
    bc.expect_extra = (unsigned)missing_blocks;
    bc.spin_limit = (unsigned)spin_limit;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(std::max(b->bps, 1) * b->sms));
    cfg.blockDim = dim3(kTile);
    cfg.stream = b->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    // zero substeps and no cycle end: the kernel only meets one barrier
    BATCH_CUDA(b, cudaLaunchKernelEx(&cfg, k_batch_barrier_only, bc));
    return SPH_OK;
}

const char *sph_batch_last_error(const sph_batch *b) { return b ? b->err.c_str() : "null batch"; }

void sph_batch_destroy(sph_batch *b)
{
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    drop_graphs(b);
    for (int k = 0; k < kBranchStreams; ++k) {
        if (b->branch[k]) cudaStreamDestroy(b->branch[k]);
        if (b->join[k]) cudaEventDestroy(b->join[k]);
    }
    if (b->fork) cudaEventDestroy(b->fork);
    delete b;
}

}  // extern "C"

// sph_device.cuh -- per-tile device functions of one SPH substep (SPHaptics, arXiv 2511.15908).
//
// Each *_item function processes one tile (one 256-thread block's worth of work) of one
// phase for one scene.  The plain path launches one kernel per phase whose blocks are the
// tiles (sph_kernels.cu); the batched path runs every phase of many scenes in one
// persistent kernel that takes tiles from a work queue (sph_batch.cu).  Both therefore do
// exactly the same arithmetic in the same order.
//
// Phases (Alg. 2 inner loop and Alg. 1):
//   hash        "calculate uniform grid cell": rigid boundary particles follow their body
//               (Sec. 3.2), FP32 cell key, atomic per-cell count
//   scan_tiles  "cumulative sum of cell particle count", level 1 (tile sums)
//   scan_apply  level 2: exclusive scan into cell_start, counts reset for the next substep
//   scatter     "sorted index": every particle claims a slot in its cell
//   rank_gather stable order inside each cell (ascending previous slot), SoA float4 gather
//   density     Alg. 1 loop 1: rho_i = sum_j m_j W_ij (Eq. density), p = k(rho - rho0)
//               (Eq. pressure); 9 contiguous x-runs of 3 cells cover the 27-cell block
//   force       Alg. 1 loops 2-3: pressure + viscosity pair forces, soft springs (Sec. 3.2),
//               gravity, semi-implicit Euler (Eq. euler); boundary particles store their
//               coupling force; FP64 momentum diagnostics
//   wrench      FP64 reduction of coupling forces into per-body force and torque about
//               the grab point (Sec. 3.3); the last tile integrates free rigid bodies
//               (Sec. 3.2) and advances the substep counter
#pragma once
#include "sph_internal.cuh"

namespace sphgb {

constexpr int kTile = 256;     // threads per block = particles per tile



constexpr int KIND_STATIC = 1, KIND_RIGID = 2, KIND_SOFT = 3;
constexpr uint32_t FLAG_CLAMP = 1u, FLAG_RECORD = 2u, FLAG_TAIT = 8u, FLAG_VOLUME = 16u,
                   FLAG_LOW_LATENCY = 32u;

// ------------------------------------------------------------------ small helpers

// Neighbour loads the force pass issues together from a list quad (1, 2 or 4): with 2 the
// pass ran 187 -> 155 us (same registers); 4 needs more registers than the occupancy the
// pass wants.
#ifndef SPH_FORCE_BATCH
#define SPH_FORCE_BATCH 2
#endif
// Candidates per unrolled step of the density pass's distance-mask loop.
#ifndef SPH_MASK_UNROLL
#define SPH_MASK_UNROLL 4
#endif
constexpr int kMaskUnroll = SPH_MASK_UNROLL;
// Cell rows per unrolled step of the neighbour-row walk (along y); 2 measured 321 us
// against 317 for the density pass.
#ifndef SPH_ROW_UNROLL
#define SPH_ROW_UNROLL 1
#endif
constexpr int kRowUnroll = SPH_ROW_UNROLL;

// Index check of the bounds-checked build (compiled with -DSPH_CHECKED): an index that
// comes from data (a cell key, a sorted slot, a particle id, a list entry) and falls
// outside [0, n) latches ST_BOUNDS and is replaced by 0, so the access stays inside its
// buffer.  The default build compiles the check away.
__device__ __forceinline__ int in_range(const SimConst &c, long long i, long long n)
{
#ifdef SPH_CHECKED
    if (i >= 0 && i < n) return (int)i;
    atomicOr(c.status, ST_BOUNDS);
    return 0;
#else
    (void)c; (void)n;
    return (int)i;
#endif
}

__device__ __forceinline__ int body_of(const SimConst &c, int id)
{
    int b = 0;
    while (b < c.nb - 1 && id >= c.body_end[b]) ++b;
    return b;
}

struct Pose {
    float t[3], q[4], v[3], w[3];
};

// Pose used during substep `step`: a grabbed body with a path follows the path entry.
__device__ __forceinline__ Pose body_pose(const SimConst &c, const DevBody &B, uint32_t step)
{
    Pose P;
    if (B.grabbed && B.path_n > 0) {
        int s = (int)(step - (uint32_t)B.path_step0);
        s = s < 0 ? 0 : (s >= B.path_n ? B.path_n - 1 : s);
        const float *r = c.path + 13 * s;
        for (int a = 0; a < 3; ++a) { P.t[a] = r[a]; P.v[a] = r[7 + a]; P.w[a] = r[10 + a]; }
        for (int a = 0; a < 4; ++a) P.q[a] = r[3 + a];
    } else {
        for (int a = 0; a < 3; ++a) { P.t[a] = B.t[a]; P.v[a] = B.v[a]; P.w[a] = B.w[a]; }
        for (int a = 0; a < 4; ++a) P.q[a] = B.q[a];
    }
    return P;
}

// FP32 rotation matrix of (w,x,y,z), every product and sum rounded separately (no FMA),
// so boundary positions -- which decide cell keys -- are bit-defined.
__device__ __forceinline__ void rot_f32(const float q[4], float R[9])
{
    float w = q[0], x = q[1], y = q[2], z = q[3];
    float xx = __fmul_rn(x, x), yy = __fmul_rn(y, y), zz = __fmul_rn(z, z);
    float xy = __fmul_rn(x, y), xz = __fmul_rn(x, z), yz = __fmul_rn(y, z);
    float wx = __fmul_rn(w, x), wy = __fmul_rn(w, y), wz = __fmul_rn(w, z);
    R[0] = __fsub_rn(1.0f, __fmul_rn(2.0f, __fadd_rn(yy, zz)));
    R[1] = __fmul_rn(2.0f, __fsub_rn(xy, wz));
    R[2] = __fmul_rn(2.0f, __fadd_rn(xz, wy));
    R[3] = __fmul_rn(2.0f, __fadd_rn(xy, wz));
    R[4] = __fsub_rn(1.0f, __fmul_rn(2.0f, __fadd_rn(xx, zz)));
    R[5] = __fmul_rn(2.0f, __fsub_rn(yz, wx));
    R[6] = __fmul_rn(2.0f, __fsub_rn(xz, wy));
    R[7] = __fmul_rn(2.0f, __fadd_rn(yz, wx));
    R[8] = __fsub_rn(1.0f, __fmul_rn(2.0f, __fadd_rn(xx, yy)));
}

__device__ __forceinline__ float body_coord(const float R[9], const float t[3], float4 l, int a)
{
    float s = __fmul_rn(R[3 * a], l.x);
    s = __fadd_rn(s, __fmul_rn(R[3 * a + 1], l.y));
    s = __fadd_rn(s, __fmul_rn(R[3 * a + 2], l.z));
    return __fadd_rn(s, t[a]);
}

// Cell coordinate on one axis: floor((x - o) * inv) in FP32, clamped to [0, n-1].
__device__ __forceinline__ int cell_axis(float x, float o, float inv, int n, uint32_t &bad)
{
    if (!isfinite(x)) { bad |= ST_NONFINITE; return 0; }
    float f = floorf(__fmul_rn(__fsub_rn(x, o), inv));
    if (f < 0.0f) { bad |= ST_DOMAIN; return 0; }
    if (f > (float)(n - 1)) { bad |= ST_DOMAIN; return n - 1; }
    return (int)f;
}

__device__ __forceinline__ void cell_of(const SimConst &c, float4 x, int &cx, int &cy, int &cz,
                                        uint32_t &bad)
{
    cx = cell_axis(x.x, c.o[0], c.inv_cell, c.nx, bad);
    cy = cell_axis(x.y, c.o[1], c.inv_cell, c.ny, bad);
    cz = cell_axis(x.z, c.o[2], c.inv_cell, c.nz, bad);
}

// Neighbour predicate: d = x_j - x_i, r2 = fma(dz,dz, fma(dy,dy, dx*dx)) < R2 (FP32).
__device__ __forceinline__ float dist2(float4 xi, float4 xj, float &dx, float &dy, float &dz)
{
    dx = __fsub_rn(xj.x, xi.x);
    dy = __fsub_rn(xj.y, xi.y);
    dz = __fsub_rn(xj.z, xi.z);
    return __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
}

// Floor of a cell coordinate clamped to [0, n): out-of-range and non-finite inputs land on
// a valid cell.
__device__ __forceinline__ int cell_floor(float u, int n)
{
    return min(max(__float2int_rd(u), 0), n - 1);
}

// Lower bound, in cell units, of the distance along one axis from cell coordinate u (own
// cell cu) to any particle whose cell index along that axis is j: the distance to cell
// j's near face, less the margin.
__device__ __forceinline__ float cell_gap(float u, int j, int cu, float mc)
{
    if (j == cu) return 0.0f;
    const float g = j > cu ? (float)j - u : u - (float)(j + 1);
    return fmaxf(g - mc, 0.0f);
}

// Calls f(s, e) for every row of cells (fixed y and z) that can hold a particle within
// the search radius of x; [s, e) is the range of sorted slots of the row's cells whose
// x-extent can reach that far (cells along x are consecutive in the key, so the range is
// contiguous).  Each row is clipped to the chord of the search sphere at the row's
// nearest y-z distance, so for a cell near h the candidates fill about 2.5 times the
// sphere's volume instead of the 6.5 times of a 27-cell block of 2h cells.  The bounds
// work in cell coordinates u = (x - o) / cell, rounded exactly as the hash rounds them;
// every bound is a lower bound on the distance and rounding is monotone, so no particle
// that passes the FP32 predicate is ever outside the visited cells (the margin, ~2e-3
// cells, is far above the rounding of u).
template <class F>
__device__ __forceinline__ void for_each_row(const SimConst &c, float4 x, uint32_t &bad, F &&f)
{
    const float ux = __fmul_rn(__fsub_rn(x.x, c.o[0]), c.inv_cell);
    const float uy = __fmul_rn(__fsub_rn(x.y, c.o[1]), c.inv_cell);
    const float uz = __fmul_rn(__fsub_rn(x.z, c.o[2]), c.inv_cell);
    const float Rc = c.Rc, Rc2 = Rc * Rc, mc = c.mc;
    const int cy = cell_floor(uy, c.ny), cz = cell_floor(uz, c.nz);
    const int z0 = cell_floor(uz - Rc, c.nz), z1 = cell_floor(uz + Rc, c.nz);
    const int y0 = cell_floor(uy - Rc, c.ny), y1 = cell_floor(uy + Rc, c.ny);
#pragma unroll 1
    for (int z = z0; z <= z1; ++z) {
        const float gz = cell_gap(uz, z, cz, mc);
        const float rz2 = Rc2 - gz * gz;
#pragma unroll kRowUnroll
        for (int y = y0; y <= y1; ++y) {
            const float gy = cell_gap(uy, y, cy, mc);
            const float w2 = rz2 - gy * gy;
            if (!(w2 >= 0.0f)) continue;
            // chord half-width; the rsqrt error (~1e-7 relative) is far inside the margin
            const float w = w2 * rsqrtf(fmaxf(w2, 1e-30f)) + mc;
            const int xa = cell_floor(ux - w, c.nx), xb = cell_floor(ux + w, c.nx);
            const int base = (z * c.ny + y) * c.nx;
            const int s = in_range(c, __ldg(c.cell_start + in_range(c, base + xa, c.ncell)), c.n + 1);
            int e = in_range(c, __ldg(c.cell_start + in_range(c, base + xb + 1, c.ncell + 1)), c.n + 1);
            if (e - s > kMaxCellRun) { e = s + kMaxCellRun; bad |= ST_CAPACITY; }
            f(s, e);
        }
    }
}

// Body kind of a particle id and the id range whose pair forces it ignores: a static or
// rigid particle does not interact with the particles of its own body (their relative
// positions are fixed); fluid and soft particles ignore nobody (range empty).
__device__ __forceinline__ void pair_scope(const SimConst &c, int id, int &kind, int &excl_lo,
                                           int &excl_n)
{
    kind = 0; excl_lo = 0; excl_n = 0;
    if (id >= c.nf) {
        const int b = body_of(c, id);
        kind = c.body_kind[b];
        if (kind != KIND_SOFT) {
            excl_lo = b == 0 ? c.nf : c.body_end[b - 1];
            excl_n = c.body_end[b] - excl_lo;
        }
    }
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ void report(const SimConst &c, uint32_t bad)
{
    if (bad) {
        atomicOr(c.status, bad);
        if (bad & ST_NONFINITE) atomicAdd(c.status + 1, 1u);
        if (bad & ST_DOMAIN) atomicAdd(c.status + 2, 1u);
    }
}

// ------------------------------------------------------------------ spatial hash

__device__ __forceinline__ void hash_item(const SimConst &c, int blk)
{
    int e = blk * kTile + threadIdx.x;
    if (e >= c.n) return;
    // the single-pass scan's tile states and tile counter, ready for this substep's scan
    for (int t = e; t <= c.n_scan_tiles; t += c.n) c.tile_state[t] = 0ull;
    float4 x = c.xB[e];
    if (x.w < 0.0f) {                       // boundary particle (negative mass tag)
        float4 v = c.vB[e];
        int id = __float_as_int(v.w);
        int b = body_of(c, id);
        if (c.body_kind[b] == KIND_RIGID) {
            Pose P = body_pose(c, c.body[b], c.ctr[0]);
            float R[9];
            rot_f32(P.q, R);
            float4 l = c.locals[in_range(c, id - c.nf, c.n_body_particles)];
            x.x = body_coord(R, P.t, l, 0);
            x.y = body_coord(R, P.t, l, 1);
            x.z = body_coord(R, P.t, l, 2);
            float r0 = x.x - P.t[0], r1 = x.y - P.t[1], r2 = x.z - P.t[2];
            v.x = P.v[0] + (P.w[1] * r2 - P.w[2] * r1);
            v.y = P.v[1] + (P.w[2] * r0 - P.w[0] * r2);
            v.z = P.v[2] + (P.w[0] * r1 - P.w[1] * r0);
            c.xB[e] = x;
            c.vB[e] = v;
        }
    }
    uint32_t bad = 0;
    int cx, cy, cz;
    cell_of(c, x, cx, cy, cz, bad);
    uint32_t k = (uint32_t)in_range(c, (cz * c.ny + cy) * c.nx + cx, c.ncell);
    c.key[e] = k;
    c.rank[e] = atomicAdd(c.cnt + k, 1u);
    report(c, bad);
}

// --------------------------------------------------------------- two-level scan

__device__ __forceinline__ void scan_tiles_item(const SimConst &c, int blk)
{
    __shared__ uint32_t ws[8];
    int base = blk * kScanTile;
    uint32_t s = 0;
    for (int i = threadIdx.x; i < kScanTile; i += 256) {
        int ci = base + i;
        if (ci < c.ncell) s += c.cnt[ci];
    }
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int w = 0; w < 8; ++w) t += ws[w];
        c.tile_sum[blk] = t;
    }
}

__device__ __forceinline__ void scan_apply_item(const SimConst &c, int blk)
{
    __shared__ uint32_t ws[8];
    __shared__ uint32_t s_pre;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    // prefix of the earlier tiles
    uint32_t pre = 0;
    for (int t = threadIdx.x; t < blk; t += 256) pre += c.tile_sum[t];
    pre = warp_sum(pre);
    if (lane == 0) ws[wid] = pre;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int w = 0; w < 8; ++w) t += ws[w];
        s_pre = t;
    }
    __syncthreads();
    // 8 consecutive cells per thread, moved as two 16-byte vectors when all 8 exist and
    // both arrays are 16-byte aligned (the workspace's are; a caller's array may not be)
    const int base = blk * kScanTile + threadIdx.x * 8;
    const bool full = base + 8 <= c.ncell &&
                      (((uintptr_t)c.cnt | (uintptr_t)c.cell_start) & 15u) == 0;
    uint32_t v[8], tot = 0;
    if (full) {
        const uint4 a = *reinterpret_cast<const uint4 *>(c.cnt + base);
        const uint4 b = *reinterpret_cast<const uint4 *>(c.cnt + base + 4);
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
        v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
    } else {
#pragma unroll
        for (int i = 0; i < 8; ++i) v[i] = (base + i < c.ncell) ? c.cnt[base + i] : 0u;
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) tot += v[i];
    // inclusive warp scan of the thread totals
    uint32_t inc = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t u = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += u;
    }
    __syncthreads();
    if (lane == 31) ws[wid] = inc;
    __syncthreads();
    uint32_t wpre = 0;
    for (int w = 0; w < wid; ++w) wpre += ws[w];
    uint32_t run = s_pre + wpre + inc - tot;
    if (full) {
        uint32_t st[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) { st[i] = run; run += v[i]; }
        *reinterpret_cast<uint4 *>(c.cell_start + base) = make_uint4(st[0], st[1], st[2], st[3]);
        *reinterpret_cast<uint4 *>(c.cell_start + base + 4) = make_uint4(st[4], st[5], st[6], st[7]);
        // counts ready for the next substep's hash
        *reinterpret_cast<uint4 *>(c.cnt + base) = make_uint4(0u, 0u, 0u, 0u);
        *reinterpret_cast<uint4 *>(c.cnt + base + 4) = make_uint4(0u, 0u, 0u, 0u);
        if (base + 8 == c.ncell) c.cell_start[c.ncell] = run;
        return;
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        int ci = base + i;
        if (ci < c.ncell) {
            c.cell_start[ci] = run;
            c.cnt[ci] = 0u;                 // ready for the next substep's count
            run += v[i];
            if (ci == c.ncell - 1) c.cell_start[c.ncell] = run;
        }
    }
}

// Single-pass exclusive scan of the cell counts (decoupled look-back): one launch instead of
// the tile sums and the apply pass above, the counts read once.  A block takes the next tile
// index in the order blocks start (so every earlier tile is running or done), sums its 2048
// counts, publishes that aggregate, then warp 0 walks back over the earlier tiles 32 at a
// time, adding aggregates up to the first tile that has published its inclusive prefix, and
// publishes its own inclusive prefix; the cells then get their starts as in scan_apply_item.
// A state word is (kind << 32 | value), kind 1 = aggregate, 2 = inclusive prefix, 0 = not
// yet (the hash pass zeroes them).  Each wait is bounded: a wait that gives up latches
// ST_TIMEOUT and counts the tile as a prefix of 0.  The same integer sums as the two-pass
// scan, so the same cell_start.
constexpr unsigned kScanSpin = 1u << 20;
__device__ __forceinline__ void scan_lookback_item(const SimConst &c)
{
    __shared__ uint32_t ws[8];
    __shared__ uint32_t s_pre;
    __shared__ int s_tile;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (threadIdx.x == 0)
        s_tile = (int)atomicAdd(reinterpret_cast<unsigned *>(c.tile_state + c.n_scan_tiles), 1u);
    __syncthreads();
    const int blk = s_tile;
    const int base = blk * kScanTile + threadIdx.x * 8;
    const bool full = base + 8 <= c.ncell &&
                      (((uintptr_t)c.cnt | (uintptr_t)c.cell_start) & 15u) == 0;
    uint32_t v[8], tot = 0;
    if (full) {
        const uint4 a = *reinterpret_cast<const uint4 *>(c.cnt + base);
        const uint4 b = *reinterpret_cast<const uint4 *>(c.cnt + base + 4);
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
        v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
    } else {
#pragma unroll
        for (int i = 0; i < 8; ++i) v[i] = (base + i < c.ncell) ? c.cnt[base + i] : 0u;
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) tot += v[i];
    // inclusive warp scan of the thread totals, the warp totals in ws
    uint32_t inc = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t u = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += u;
    }
    if (lane == 31) ws[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        uint32_t agg = 0;
        for (int w = 0; w < 8; ++w) agg += ws[w];
        uint32_t excl = 0, bad = 0;
        volatile unsigned long long *st = c.tile_state;
        if (blk == 0) {
            if (lane == 0) atomicExch(c.tile_state, (2ull << 32) | agg);
        } else {
            if (lane == 0) atomicExch(c.tile_state + blk, (1ull << 32) | agg);
            for (int j = blk - 1;; j -= 32) {
                const int jj = j - lane;
                unsigned kind = 2u, val = 0u;        // before tile 0: a prefix of 0
                if (jj >= 0) {
                    unsigned long long w = st[jj];
                    for (unsigned it = 0; (w >> 32) == 0ull && it < kScanSpin; ++it) w = st[jj];
                    if ((w >> 32) == 0ull) {
                        bad |= ST_TIMEOUT;
                        w = 2ull << 32;
                    }
                    kind = (unsigned)(w >> 32);
                    val = (unsigned)w;
                }
                // the nearest tile with an inclusive prefix ends the walk; the tiles after
                // it contribute their aggregates
                const unsigned pm = __ballot_sync(0xffffffffu, kind == 2u);
                const int first = pm ? __ffs(pm) - 1 : 31;
                excl += warp_sum(lane <= first ? val : 0u);
                if (pm) break;
            }
            if (lane == 0) atomicExch(c.tile_state + blk, (2ull << 32) | (excl + agg));
        }
        if (lane == 0) s_pre = excl;
        report(c, bad);
    }
    __syncthreads();
    uint32_t wpre = 0;
    for (int w = 0; w < wid; ++w) wpre += ws[w];
    uint32_t run = s_pre + wpre + inc - tot;
    if (full) {
        uint32_t stv[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) { stv[i] = run; run += v[i]; }
        *reinterpret_cast<uint4 *>(c.cell_start + base) = make_uint4(stv[0], stv[1], stv[2], stv[3]);
        *reinterpret_cast<uint4 *>(c.cell_start + base + 4) = make_uint4(stv[4], stv[5], stv[6], stv[7]);
        // counts ready for the next substep's hash
        *reinterpret_cast<uint4 *>(c.cnt + base) = make_uint4(0u, 0u, 0u, 0u);
        *reinterpret_cast<uint4 *>(c.cnt + base + 4) = make_uint4(0u, 0u, 0u, 0u);
        if (base + 8 == c.ncell) c.cell_start[c.ncell] = run;
        return;
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        int ci = base + i;
        if (ci < c.ncell) {
            c.cell_start[ci] = run;
            c.cnt[ci] = 0u;                 // ready for the next substep's count
            run += v[i];
            if (ci == c.ncell - 1) c.cell_start[c.ncell] = run;
        }
    }
}

// --------------------------------------------------------- scatter + stable gather

__device__ __forceinline__ void scatter_item(const SimConst &c, int blk)
{
    int e = blk * kTile + threadIdx.x;
    if (e >= c.n) return;
    c.perm[in_range(c, (long long)c.cell_start[in_range(c, c.key[e], c.ncell)] + c.rank[e], c.n)] =
        (uint32_t)e;
}

// Within a cell the atomic claim order is arbitrary; the final slot of particle e is
// cell_start + #{members with a smaller previous slot}, i.e. a stable counting sort.
__device__ __forceinline__ void rank_gather_item(const SimConst &c, int blk)
{
    int p = blk * kTile + threadIdx.x;
    if (p >= c.n) return;
    uint32_t e = (uint32_t)in_range(c, c.perm[p], c.n);
    uint32_t k = (uint32_t)in_range(c, c.key[e], c.ncell);
    int cs = in_range(c, c.cell_start[k], c.n), ce = in_range(c, c.cell_start[k + 1], c.n + 1);
    int dst;
    if (ce - cs <= kMaxCell) {
        int r = 0;
        for (int q = cs; q < ce; ++q) r += (c.perm[q] < e);
        dst = cs + r;
    } else {
        dst = cs + (int)c.rank[e];          // still a permutation; order not stable
        atomicOr(c.status, (uint32_t)ST_CAPACITY);
    }
    dst = in_range(c, dst, c.n);
    float4 x = c.xB[e];
    float4 v = c.vB[e];
    c.xA[dst] = x;
    c.vA[dst] = v;
    int id = __float_as_int(v.w);
    if (id >= c.nf && c.body_kind[body_of(c, id)] == KIND_SOFT) c.slot_of_id[in_range(c, id, c.n)] = dst;
}

// ------------------------------------------------------------------- density pass

// Error-free transformations (Knuth's TwoSum; Dekker's Fast2Sum for |a| >= |b|; the FMA
// product residual).  Every operation is an explicit round-to-nearest intrinsic, so the
// compiler neither contracts nor reorders them.
__device__ __forceinline__ float two_sum(float a, float b, float &err)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    err = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return s;
}

// (th + tl)^3 as hi + lo for a small tl: th^3 exactly as t3 + e3 + e2 th (two FMA
// residuals), plus the first-order term 3 th^2 tl.
__device__ __forceinline__ float cube_pair(float th, float tl, float &lo)
{
    const float t2 = __fmul_rn(th, th), e2 = __fmaf_rn(th, th, -t2);
    const float t3 = __fmul_rn(t2, th), e3 = __fmaf_rn(t2, th, -t3);
    lo = __fmaf_rn(__fmul_rn(3.0f, t2), tl, __fmaf_rn(e2, th, e3));
    return t3;
}

// The low part of an FP32 difference: (a - b) - fl(a - b), exact (TwoSum of a and -b).
// Nonzero only when a or b lies near zero (for |a| >= 2|a - b| the difference is exact).
__device__ __forceinline__ float diff_lo(float a, float b, float d)
{
    const float bb = __fsub_rn(d, a);
    return __fadd_rn(__fsub_rn(a, __fsub_rn(d, bb)), __fsub_rn(-b, bb));
}

// ---------------------------------------------- two neighbours at once (packed FP32)
// sm_100 and later issue a pair of FP32 additions, multiplications or FMAs as one
// instruction (__fadd2_rn, __fmul2_rn, __ffma2_rn), each component rounded exactly as the
// scalar operation.  The float-pair arithmetic below evaluates two neighbours' terms that
// way: component for component the same operations as the scalar functions above, so the
// same values; the passes are bound by instruction issue, which the pairing halves for
// this part.
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 f2s(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, neg2(b)); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

__device__ __forceinline__ float2 two_sum2(float2 a, float2 b, float2 &err)
{
    const float2 s = add2(a, b);
    const float2 bb = sub2(s, a);
    err = add2(sub2(a, sub2(s, bb)), sub2(b, bb));
    return s;
}

__device__ __forceinline__ float2 cube_pair2(float2 th, float2 tl, float2 &lo)
{
    const float2 t2 = mul2(th, th), e2 = fma2(th, th, neg2(t2));
    const float2 t3 = mul2(t2, th), e3 = fma2(t2, th, neg2(t3));
    lo = fma2(mul2(f2s(3.0f), t2), tl, fma2(e2, th, e3));
    return t3;
}

__device__ __forceinline__ float2 diff_lo2(float2 a, float2 b, float2 d)
{
    const float2 bb = sub2(d, a);
    return add2(sub2(a, sub2(d, bb)), sub2(neg2(b), bb));
}

// pair_offset for two neighbours (x, y, z components of xa and xb packed)
__device__ __forceinline__ void pair_offset2(float4 xi, float4 xa, float4 xb, bool near0, float2 &dx, float2 &dy,
                                             float2 &dz, float2 &r2x, float2 &lx, float2 &ly, float2 &lz)
{
    const float2 ax = f2(xa.x, xb.x), ay = f2(xa.y, xb.y), az = f2(xa.z, xb.z);
    const float2 ix = f2s(xi.x), iy = f2s(xi.y), iz = f2s(xi.z);
    dx = sub2(ax, ix);
    dy = sub2(ay, iy);
    dz = sub2(az, iz);
    r2x = f2s(0.0f);
    lx = ly = lz = f2s(0.0f);
    if (near0) {
        lx = diff_lo2(ax, ix, dx);
        ly = diff_lo2(ay, iy, dy);
        lz = diff_lo2(az, iz, dz);
        r2x = mul2(f2s(2.0f), fma2(dx, lx, fma2(dy, ly, mul2(dz, lz))));
    }
}

struct PairQ2 {
    float2 qh, ql;
};
__device__ __forceinline__ PairQ2 pair_q2(const SimConst &c, float2 dx, float2 dy, float2 dz, float2 r2x)
{
    const float2 px = mul2(dx, dx), py = mul2(dy, dy), pz = mul2(dz, dz);
    const float2 ex = fma2(dx, dx, neg2(px)), ey = fma2(dy, dy, neg2(py));
    const float2 ez = fma2(dz, dz, neg2(pz));
    float2 e1, e2;
    const float2 s1 = two_sum2(px, py, e1);
    const float2 r2h = two_sum2(s1, pz, e2);
    const float2 r2l = add2(add2(add2(ex, ey), ez), add2(add2(e1, e2), r2x));
    const float2 rs = f2(rsqrtf(fmaxf(r2h.x, 1e-30f)), rsqrtf(fmaxf(r2h.y, 1e-30f)));
    const float2 hrs = mul2(f2s(0.5f), rs);
    float2 r = mul2(r2h, rs);
    r = fma2(hrs, fma2(neg2(r), r, r2h), r);
    const float2 rl = mul2(add2(fma2(neg2(r), r, r2h), r2l), hrs);
    PairQ2 o;
    o.qh = mul2(r, f2s(c.invh_hi));
    o.ql = add2(fma2(r, f2s(c.invh_hi), neg2(o.qh)), fma2(r, f2s(c.invh_lo), mul2(rl, f2s(c.invh_hi))));
    return o;
}

// the density terms (mh + ml)(6 w(q)) of two neighbours as float pairs (hi, lo): the
// arithmetic of PairDensitySum::add_q before its accumulation
__device__ __forceinline__ void density_term2(const PairQ2 &pq, float2 mh, float2 ml, float2 &hi, float2 &lo)
{
    const float2 qh = pq.qh, ql = pq.ql;
    const float2 th = sub2(f2s(2.0f), qh);
    const float2 tl = sub2(sub2(sub2(f2s(2.0f), th), qh), ql);
    float2 uh = sub2(f2s(1.0f), qh);
    float2 ul = sub2(sub2(sub2(f2s(1.0f), uh), qh), ql);
    if (!(uh.x > 0.0f)) { uh.x = 0.0f; ul.x = 0.0f; }
    if (!(uh.y > 0.0f)) { uh.y = 0.0f; ul.y = 0.0f; }
    float2 t3l;
    const float2 t3 = cube_pair2(th, tl, t3l);
    const float2 u2 = mul2(uh, uh);
    const float2 u3 = mul2(u2, uh);
    const float2 u3l = mul2(mul2(f2s(3.0f), u2), ul);
    const float2 m4u3 = mul2(f2s(-4.0f), u3);
    const float2 w6h = add2(t3, m4u3);
    const float2 w6l = add2(sub2(m4u3, sub2(w6h, t3)), fma2(f2s(-4.0f), u3l, t3l));
    hi = mul2(mh, w6h);
    lo = fma2(ml, w6h, fma2(mh, w6l, fma2(mh, w6h, neg2(hi))));
}

// Sum of m_j * 6 w(q_ij) over a particle's neighbours with an error of a few units of the
// second order in FP32 rounding (~1e-13 relative), i.e. as good as the FP64 definition for
// the pressure the force pass needs: p = k (rho - rho0) turns one FP32 ulp of rho ~ 1000
// (6e-5) into a pressure change that moves wall-adjacent accelerations by ~1e-4 m/s^2,
// and every FP32 stage of the plain evaluation (r^2, sqrt, q, the cubic, the product with
// m, the summation) costs about that much.  So each stage carries its rounding error: q as
// a float pair (pair_q), 6 w = t^3 - 4 u^3 with t = 2 - q and u = max(1 - q, 0) as pairs
// and both cubes as pairs (Fast2Sum for the difference, t^3 >= 4 u^3), the term m 6w as a
// pair, and the running sum by TwoSum; all low parts are summed in L.  The value is S + L.
// q = |x_j - x_i| / h as an unevaluated float pair qh + ql (relative error ~1e-13): r^2 =
// dx^2 + dy^2 + dz^2 from FMA product residuals and TwoSums, r = sqrt(r^2) from rsqrt, one
// Newton step and the residual r2 - r^2 over 2r, q with 1/h as a float pair.  d = x_j - x_i
// in FP32; r2x = the first-order r^2 correction 2 d . d_lo when a difference was not exact.
struct PairQ {
    float qh, ql;
    float r2h;                 // r^2, high part
    float rs;                  // ~ 1 / r (rsqrt of r2h)
};
__device__ __forceinline__ PairQ pair_q(const SimConst &c, float dx, float dy, float dz, float r2x)
{
    const float px = __fmul_rn(dx, dx), py = __fmul_rn(dy, dy), pz = __fmul_rn(dz, dz);
    const float ex = __fmaf_rn(dx, dx, -px), ey = __fmaf_rn(dy, dy, -py);
    const float ez = __fmaf_rn(dz, dz, -pz);
    float e1, e2;
    const float s1 = two_sum(px, py, e1);
    const float r2h = two_sum(s1, pz, e2);
    const float r2l = __fadd_rn(__fadd_rn(__fadd_rn(ex, ey), ez), __fadd_rn(__fadd_rn(e1, e2), r2x));
    // r: rsqrt, one Newton step, then the residual r2 - r^2 over 2r
    const float rs = rsqrtf(fmaxf(r2h, 1e-30f));
    const float hrs = __fmul_rn(0.5f, rs);
    float r = __fmul_rn(r2h, rs);
    r = __fmaf_rn(hrs, __fmaf_rn(-r, r, r2h), r);
    const float rl = __fmul_rn(__fadd_rn(__fmaf_rn(-r, r, r2h), r2l), hrs);
    // q = r (1/h)_hi + r (1/h)_lo + rl (1/h)_hi
    PairQ o;
    o.r2h = r2h;
    o.rs = rs;
    o.qh = __fmul_rn(r, c.invh_hi);
    o.ql = __fadd_rn(__fmaf_rn(r, c.invh_hi, -o.qh), __fmaf_rn(r, c.invh_lo, __fmul_rn(rl, c.invh_hi)));
    return o;
}

struct PairDensitySum {
    float S = 0.0f, L = 0.0f;
    int cnt = 0;
    // the particle itself (q = 0: 6 w = 4)
    __device__ __forceinline__ void self(float mi)
    {
        S = __fmul_rn(4.0f, mi);
        cnt = 1;
    }
    // neighbour of weight (mh + ml) at d = x_j - x_i (FP32 differences; r2x = the first-order
    // r^2 correction 2 d . d_lo when a difference was not exact)
    __device__ __forceinline__ void add(const SimConst &c, float mh, float ml, float dx, float dy,
                                        float dz, float r2x)
    {
        const PairQ pq = pair_q(c, dx, dy, dz, r2x);
        const float qh = pq.qh, ql = pq.ql;
        // t = 2 - q: 2 - th and (2 - th) - qh are exact (Sterbenz); likewise u = 1 - q
        const float th = __fsub_rn(2.0f, qh);
        const float tl = __fsub_rn(__fsub_rn(__fsub_rn(2.0f, th), qh), ql);
        float uh = __fsub_rn(1.0f, qh);
        float ul = __fsub_rn(__fsub_rn(__fsub_rn(1.0f, uh), qh), ql);
        if (!(uh > 0.0f)) { uh = 0.0f; ul = 0.0f; }
        float t3l;
        const float t3 = cube_pair(th, tl, t3l);
        // u^3 <= 1 weighs little: its rounding residuals are below the needed precision
        // (measured on an emulation of the arithmetic: same error as the full pair), only
        // the first-order term of ul is kept
        const float u2 = __fmul_rn(uh, uh);
        const float u3 = __fmul_rn(u2, uh);
        const float u3l = __fmul_rn(__fmul_rn(3.0f, u2), ul);
        const float m4u3 = __fmul_rn(-4.0f, u3);                 // exact
        const float w6h = __fadd_rn(t3, m4u3);
        const float w6l = __fadd_rn(__fsub_rn(m4u3, __fsub_rn(w6h, t3)), __fmaf_rn(-4.0f, u3l, t3l));
        // term (mh + ml)(w6h + w6l)
        const float th_ = __fmul_rn(mh, w6h);
        const float lo = __fmaf_rn(ml, w6h, __fmaf_rn(mh, w6l, __fmaf_rn(mh, w6h, -th_)));
        add_term(th_, lo);
    }
    // a term (hi, lo) computed elsewhere (density_term2)
    __device__ __forceinline__ void add_term(float th_, float lo)
    {
        float es;
        S = two_sum(S, th_, es);
        L = __fadd_rn(L, __fadd_rn(lo, es));
        ++cnt;
    }
    // alpha/6 (S + L) - rho0 with alpha/6 = hi + lo
    __device__ __forceinline__ float excess(const SimConst &c, float rho0) const
    {
        return __fadd_rn(__fmaf_rn(c.alpha6_hi, S, -rho0),
                         __fmaf_rn(c.alpha6_lo, S, __fmul_rn(c.alpha6_hi, L)));
    }
};

// d = x_j - x_i with the first-order r^2 correction of inexact differences (only particles
// within 2R of a coordinate plane through the origin can have them).
__device__ __forceinline__ void pair_offset(float4 xi, float4 xj, bool near0, float &dx, float &dy,
                                            float &dz, float &r2x, float &lx, float &ly, float &lz)
{
    dx = __fsub_rn(xj.x, xi.x);
    dy = __fsub_rn(xj.y, xi.y);
    dz = __fsub_rn(xj.z, xi.z);
    r2x = 0.0f;
    lx = 0.0f; ly = 0.0f; lz = 0.0f;
    if (near0) {
        lx = diff_lo(xj.x, xi.x, dx);
        ly = diff_lo(xj.y, xi.y, dy);
        lz = diff_lo(xj.z, xi.z, dz);
        r2x = __fmul_rn(2.0f, __fmaf_rn(dx, lx, __fmaf_rn(dy, ly, __fmul_rn(dz, lz))));
    }
}

__device__ __forceinline__ void pair_offset(float4 xi, float4 xj, bool near0, float &dx, float &dy,
                                            float &dz, float &r2x)
{
    float lx, ly, lz;
    pair_offset(xi, xj, near0, dx, dy, dz, r2x, lx, ly, lz);
}

// w'(q) / q of the cubic spline as a float pair gh + gl from q = qh + ql:
//   q < 1: -2 + 1.5 q;   1 <= q < 2: -0.5 (2 - q)^2 / q
// (the two agree at q = 1).  The quotient takes an approximate 1/qh and one residual step,
// so its error is second order in the reciprocal's.
__device__ __forceinline__ float gradq_pair(float qh, float ql, float &gl)
{
    // inner piece: p = 1.5 qh as a pair, then Fast2Sum with -2 (|p| <= 1.5 < 2)
    const float p = __fmul_rn(1.5f, qh), pe = __fmaf_rn(1.5f, qh, -p);
    const float gi = __fadd_rn(-2.0f, p);
    const float gil = __fadd_rn(__fsub_rn(p, __fadd_rn(gi, 2.0f)), __fmaf_rn(1.5f, ql, pe));
    // outer piece: A = t^2 as a pair (t = 2 - q), divided by q
    const float th = __fsub_rn(2.0f, qh);
    const float tl = __fsub_rn(__fsub_rn(__fsub_rn(2.0f, th), qh), ql);
    const float ah = __fmul_rn(th, th);
    const float al = __fmaf_rn(__fmul_rn(2.0f, th), tl, __fmaf_rn(th, th, -ah));
    const float iq = __fdividef(1.0f, qh);
    const float g0 = __fmul_rn(ah, iq);
    const float g1 = __fmul_rn(__fadd_rn(__fmaf_rn(-g0, qh, ah), __fmaf_rn(-g0, ql, al)), iq);
    if (qh < 1.0f) {
        gl = gil;
        return gi;
    }
    gl = __fmul_rn(-0.5f, g1);
    return __fmul_rn(-0.5f, g0);
}

// Sum over a particle's interaction partners of w_j (w'(q)/q) d_j, d_j = x_j - x_i, with
// w'(q)/q as a float pair, every product's residual kept and each component summed by
// TwoSum: a kernel-gradient sum that cancels (to ~0 for a full neighbourhood) is exact to
// ~1e-13 of its terms.  The force pass multiplies it by the particle's own pressure term.
struct PairGradSum {
    float Sx = 0.0f, Sy = 0.0f, Sz = 0.0f, Lx = 0.0f, Ly = 0.0f, Lz = 0.0f;
    __device__ __forceinline__ void add(float w, float gh, float gl, float dx, float dy, float dz,
                                        float lx, float ly, float lz)
    {
        const float mh = __fmul_rn(w, gh);
        const float ml = __fmaf_rn(w, gl, __fmaf_rn(w, gh, -mh));
        add1(Sx, Lx, mh, ml, dx, lx);
        add1(Sy, Ly, mh, ml, dy, ly);
        add1(Sz, Lz, mh, ml, dz, lz);
    }
    static __device__ __forceinline__ void add1(float &S, float &L, float mh, float ml, float d, float dl)
    {
        const float th = __fmul_rn(mh, d);
        const float tl = __fmaf_rn(mh, dl, __fmaf_rn(ml, d, __fmaf_rn(mh, d, -th)));
        acc1(S, L, th, tl);
    }
    static __device__ __forceinline__ void acc1(float &S, float &L, float th, float tl)
    {
        float e;
        S = two_sum(S, th, e);
        L = __fadd_rn(L, __fadd_rn(tl, e));
    }
};

__device__ __forceinline__ bool near_origin_planes(const SimConst &c, float4 x)
{
    const float lim = 4.0f * c.h;                 // 2R
    return fabsf(x.x) < lim || fabsf(x.y) < lim || fabsf(x.z) < lim;
}

// Compensated FP32 sum of m_j * 6 w(q_ij) (Kahan), for the isosurface field, whose
// tolerance is far looser than the pressure's.
struct DensitySum {
    float S = 0.0f, C = 0.0f;
    int cnt = 0;
    __device__ __forceinline__ void add(const SimConst &c, float4 xj, float r2)
    {
        add_m(c, fabsf(xj.w), r2);
    }
    // the same with the neighbour's weight given (its mass, or a boundary volume weight)
    __device__ __forceinline__ void add_m(const SimConst &c, float mj, float r2)
    {
        // sqrt: rsqrt + one Newton step (~1 ulp); r2 = 0 (the particle itself) gives r = 0
        float rs = rsqrtf(fmaxf(r2, 1e-30f));
        float r = r2 * rs;
        r = __fmaf_rn(0.5f * rs, __fmaf_rn(-r, r, r2), r);
        // q = r / h with a single rounding of r * (1/h)_hi + r * (1/h)_lo
        float s = __fmaf_rn(r, c.invh_hi, r * c.invh_lo);
        // 6 w(q) = (2-q)^3 - 4 (1-q)^3 for q < 1, (2-q)^3 for 1 <= q < 2
        float t = 2.0f - s, u1 = 1.0f - s;
        float w6 = t * t * t;
        if (s < 1.0f) w6 = __fmaf_rn(-4.0f * u1, u1 * u1, w6);
        float y = __fsub_rn(mj * w6, C);
        float u = __fadd_rn(S, y);
        C = __fsub_rn(__fsub_rn(u, S), y);
        S = u;
        ++cnt;
    }
};

// Appends slots to a particle's neighbour list four at a time: entries shift into a
// register quad and leave as one 16-byte store, so a warp issues a quarter of the stores.
// Entries beyond the capacity are counted, not stored.
struct ListWriter {
    uint4 *dst;                // this particle's quad 0; quad g at dst[g * n]
    size_t n;
    int cap, nl = 0;
    uint4 quad = make_uint4(0u, 0u, 0u, 0u);   // the last four entries pushed
    __device__ __forceinline__ void push(uint32_t q)
    {
        quad = make_uint4(quad.y, quad.z, quad.w, q);
        ++nl;
        if ((nl & 3) == 0 && nl <= cap) dst[(size_t)(nl / 4 - 1) * n] = quad;
    }
    __device__ __forceinline__ void flush()
    {
        const int r = nl & 3;
        if (r == 0 || nl > cap) return;
        // the last r entries sit in the top r components; move them to the bottom
        uint4 o = quad;
        if (r == 1) {
            o.x = quad.w;
        } else if (r == 2) {
            o.x = quad.z; o.y = quad.w;
        } else {
            o.x = quad.y; o.y = quad.z; o.z = quad.w;
        }
        dst[(size_t)(nl / 4) * n] = o;
    }
};

// Density and pressure (Eq. density, Eq. pressure) with the pair sum above, so that
// rho - rho0 (and p) carry no FP32 rounding of their own beyond the final one.
//
// Each row of candidates is taken 32 at a time by a branch-free distance test that sets one
// bit per neighbour.  The float-pair evaluation of the neighbours -- the expensive part --
// waits until the rows of a whole z-plane of cells are tested: the (chunk start, bit mask)
// pairs of the plane are kept in shared memory and then evaluated in one flat loop, one
// neighbour per iteration, so that each lane evaluates some seven neighbours per plane and
// the lanes of a warp run the evaluation together instead of each row's uneven one or two.
// Neighbours are evaluated in the order a plain walk visits them (rows in order,
// ascending slots).  The pass also records the particle's interaction partners
// (neighbours other than itself and, for a static or rigid particle, other than its own
// body's particles) in the neighbour list the force pass reads.  Static particles take no
// force, so they record nothing unless the debug record is on.
// Pending (chunk, mask) pairs per thread, and the count above which a plane's end drains
// them.  Measured on the stirred 1.16 M scene: 8 / 0 (drain every plane) 525 us; 12 / 6
// 839; 16 / 10 909 (the larger shared arrays shrink L1, where the candidates hit 91 %);
// 24, drained once per particle, 580.
#ifndef SPH_DENSITY_PENDING
#define SPH_DENSITY_PENDING 8
#endif
#ifndef SPH_DENSITY_PAIRED
#define SPH_DENSITY_PAIRED 1
#endif
#ifndef SPH_PAIR_UNROLL
#define SPH_PAIR_UNROLL 1
#endif
constexpr int kPairUnroll = SPH_PAIR_UNROLL;
#ifndef SPH_DENSITY_DRAIN_AT
#define SPH_DENSITY_DRAIN_AT 0
#endif
constexpr int kPending = SPH_DENSITY_PENDING;   // (chunk start, mask) pairs kept per thread
constexpr int kDrainAt = SPH_DENSITY_DRAIN_AT;  // a plane's end drains when more are pending

template <bool VOL, int THREADS, bool PAIRED>
__device__ __forceinline__ void density_item_v(const SimConst &c, int blk, int2 *s_pend)
{
    const int p = blk * THREADS + (int)threadIdx.x;
    if (p >= c.n) return;
    const float4 xi = c.xA[p];
    uint32_t bad = 0;
    int kind = 0, excl_lo = 0, excl_n = 0;
    if (xi.w < 0.0f) pair_scope(c, __float_as_int(c.vA[p].w), kind, excl_lo, excl_n);
    const bool keep_list = kind != KIND_STATIC || (c.flags & FLAG_RECORD);
    // volume-based boundaries: boundary neighbours weigh psi (in their (rho, P) slot) and
    // a boundary particle interacts with none of them
    constexpr bool vol = VOL;
    const bool vol_boundary = vol && xi.w < 0.0f;
    const float *vw = reinterpret_cast<const float *>(c.vA) + 3;   // id bits, stride 4
    const bool near0 = near_origin_planes(c, xi);
    PairDensitySum acc;
    acc.self(fabsf(xi.w));
    ListWriter list;
    list.dst = c.nlist4 + p;
    list.n = (size_t)c.n;
    list.cap = c.nl_cap;
    int2 *pend = s_pend + threadIdx.x;            // entry k at pend[k * THREADS]
    int np = 0;

    // The neighbours are evaluated two at a time with packed FP32 instructions (the
    // terms, component for component the scalar arithmetic) and accumulated in the order
    // they are found, so the sum is the one-at-a-time sum bit for bit.  An odd neighbour
    // waits (held) for the next drain's first, or for the end of the walk.
    bool held = false;
    float4 hx = xi;
    float hmh = 0.0f, hml = 0.0f;
    auto eval2 = [&](float4 xa, float mah, float mal, float4 xb, float mbh, float mbl, bool has_b) {
        float2 dx, dy, dz, r2x, lx, ly, lz;
        pair_offset2(xi, xa, xb, near0, dx, dy, dz, r2x, lx, ly, lz);
        const PairQ2 pq = pair_q2(c, dx, dy, dz, r2x);
        float2 hi, lo;
        density_term2(pq, f2(mah, mbh), f2(mal, mbl), hi, lo);
        acc.add_term(hi.x, lo.x);
        if (has_b) acc.add_term(hi.y, lo.y);
    };
    auto drain_paired = [&]() {
        if (np == 0) return;
        int k = 0;
        int2 e = pend[0];
        uint32_t mm = (uint32_t)e.y;
        auto next = [&](int &q) {
            while (mm == 0u) {
                if (++k >= np) return false;
                e = pend[k * THREADS];
                mm = (uint32_t)e.y;
            }
            q = e.x + __ffs(mm) - 1;
            mm &= mm - 1u;
            return true;
        };
        // the neighbour's position and weight (a boundary neighbour of the volume variant
        // weighs psi, kept in its (rho, P) slot as a float pair), and its partner entry: a
        // volume-boundary particle interacts with fluid and soft ones only, a static or
        // rigid one not with its own body
        auto take = [&](int q, float4 &xj, float &mh, float &ml) {
            xj = __ldg(c.xA + q);
            mh = fabsf(xj.w);
            ml = 0.0f;
            if (vol && !vol_boundary && xj.w < 0.0f) {
                const float2 psi = __ldg(&c.prho[q]);
                mh = psi.x;
                ml = psi.y;
            }
            if (keep_list && !(vol_boundary && xj.w < 0.0f) &&
                !(excl_n && (unsigned)(__float_as_int(__ldg(vw + 4 * (size_t)q)) - excl_lo) < (unsigned)excl_n))
                list.push((uint32_t)q);
        };
        int q;
        float4 xb;
        float mbh, mbl;
        if (vol_boundary) {                        // counted; the slot keeps psi
            while (next(q)) {
                take(q, xb, mbh, mbl);
                ++acc.cnt;
            }
            np = 0;
            return;
        }
        for (;;) {
            if (!held) {
                if (!next(q)) break;
                take(q, hx, hmh, hml);
                held = true;
            }
            if (!next(q)) break;
            take(q, xb, mbh, mbl);
            eval2(hx, hmh, hml, xb, mbh, mbl, true);
            held = false;
        }
        np = 0;
    };
    // evaluate the pending neighbours in one flat loop (every stored mask is non-empty)
    auto drain_scalar = [&]() {
        if (np == 0) return;
        int k = 0;
        int2 e = pend[0];
        uint32_t mm = (uint32_t)e.y;
        for (;;) {
            if (mm == 0u) {
                if (++k == np) break;
                e = pend[k * THREADS];
                mm = (uint32_t)e.y;
            }
            const int q = e.x + __ffs(mm) - 1;
            mm &= mm - 1u;
            const float4 xj = __ldg(c.xA + q);
            if (vol_boundary) {
                ++acc.cnt;                         // counted; the slot keeps psi
            } else if (vol && xj.w < 0.0f) {
                // a boundary neighbour weighs psi = (rho, P) slot as a float pair
                const float2 psi = __ldg(&c.prho[q]);
                float dx, dy, dz, r2x;
                pair_offset(xi, xj, near0, dx, dy, dz, r2x);
                acc.add(c, psi.x, psi.y, dx, dy, dz, r2x);
            } else {
                float dx, dy, dz, r2x;
                pair_offset(xi, xj, near0, dx, dy, dz, r2x);
                acc.add(c, fabsf(xj.w), 0.0f, dx, dy, dz, r2x);
            }
            // partners: a volume-boundary particle interacts with fluid and soft ones only
            if (!keep_list || (vol_boundary && xj.w < 0.0f)) continue;
            if (excl_n && (unsigned)(__float_as_int(__ldg(vw + 4 * (size_t)q)) - excl_lo) <
                              (unsigned)excl_n)
                continue;
            list.push((uint32_t)q);
        }
        np = 0;
    };

    // PAIRED: the packed evaluation above; otherwise one neighbour at a time (same sums)
    auto drain = [&]() {
        if constexpr (PAIRED) drain_paired();
        else drain_scalar();
    };

    // rows of cells around the particle (bounds as for_each_row)
    const float ux = __fmul_rn(__fsub_rn(xi.x, c.o[0]), c.inv_cell);
    const float uy = __fmul_rn(__fsub_rn(xi.y, c.o[1]), c.inv_cell);
    const float uz = __fmul_rn(__fsub_rn(xi.z, c.o[2]), c.inv_cell);
    const float Rc = c.Rc, Rc2 = Rc * Rc, mc = c.mc;
    const int cy = cell_floor(uy, c.ny), cz = cell_floor(uz, c.nz);
    const int z0 = cell_floor(uz - Rc, c.nz), z1 = cell_floor(uz + Rc, c.nz);
    const int y0 = cell_floor(uy - Rc, c.ny), y1 = cell_floor(uy + Rc, c.ny);
#pragma unroll 1
    for (int z = z0; z <= z1; ++z) {
        const float gz = cell_gap(uz, z, cz, mc);
        const float rz2 = Rc2 - gz * gz;
#pragma unroll 1
        for (int y = y0; y <= y1; ++y) {
            const float gy = cell_gap(uy, y, cy, mc);
            const float w2 = rz2 - gy * gy;
            if (!(w2 >= 0.0f)) continue;
            // chord half-width; the rsqrt error (~1e-7 relative) is far inside the margin
            const float w = w2 * rsqrtf(fmaxf(w2, 1e-30f)) + mc;
            const int xa = cell_floor(ux - w, c.nx), xb = cell_floor(ux + w, c.nx);
            const int base = (z * c.ny + y) * c.nx;
            const int s0 = in_range(c, __ldg(c.cell_start + in_range(c, base + xa, c.ncell)), c.n + 1);
            int e0 = in_range(c, __ldg(c.cell_start + in_range(c, base + xb + 1, c.ncell + 1)), c.n + 1);
            if (e0 - s0 > kMaxCellRun) { e0 = s0 + kMaxCellRun; bad |= ST_CAPACITY; }
#pragma unroll 1
            for (int b = s0; b < e0; b += 32) {
                const int end = min(e0, b + 32);
                uint32_t mm = 0u, bit = 1u;
                if constexpr (PAIRED) {
                // two candidates per step: the predicate of dist2, component for component
                const float2 ix = f2s(xi.x), iy = f2s(xi.y), iz = f2s(xi.z);
                int q = b;
#pragma unroll kPairUnroll
                for (; q + 1 < end; q += 2) {
                    const float4 xa = __ldg(c.xA + q), xb = __ldg(c.xA + q + 1);
                    const float2 dx = sub2(f2(xa.x, xb.x), ix), dy = sub2(f2(xa.y, xb.y), iy);
                    const float2 dz = sub2(f2(xa.z, xb.z), iz);
                    const float2 r2 = fma2(dz, dz, fma2(dy, dy, mul2(dx, dx)));
                    if (r2.x < c.R2) mm |= bit;
                    if (r2.y < c.R2) mm |= bit << 1;
                    bit <<= 2;
                }
                if (q < end) {
                    const float4 xj = __ldg(c.xA + q);
                    float dx, dy, dz;
                    if (dist2(xi, xj, dx, dy, dz) < c.R2) mm |= bit;
                }
                } else {
#pragma unroll kMaskUnroll
                for (int q = b; q < end; ++q) {
                    const float4 xj = __ldg(c.xA + q);
                    float dx, dy, dz;
                    if (dist2(xi, xj, dx, dy, dz) < c.R2) mm |= bit;
                    bit <<= 1;
                }
                }
                if ((unsigned)(p - b) < 32u) mm &= ~(1u << (p - b));   // self: summed above
                if (!mm) continue;
                if (np == kPending) drain();
                pend[np * THREADS] = make_int2(b, (int)mm);
                ++np;
            }
        }
        if (np > kDrainAt) drain();                // the plane's neighbours
    }
    drain();
    if constexpr (PAIRED) {
        if (held) eval2(hx, hmh, hml, xi, 0.0f, 0.0f, false);
    }
    list.flush();
    c.nlist_n[p] = list.nl;
    const float drho = acc.excess(c, c.rho0);
    const float rho = __fadd_rn(c.rho0, drho);
    float pr;
    if (c.flags & FLAG_TAIT) {
        // Tait variation (Sec. 3.1): B ((rho/rho0)^7 - 1), B = k rho0 / 7; (1+x)^7 - 1 by its
        // binomial expansion, which has no cancellation near rest (x = drho / rho0 ~ 1e-3)
        const float x = drho / c.rho0;
        pr = c.tait_B * (x * (7.0f + x * (21.0f + x * (35.0f + x * (35.0f + x * (21.0f + x * (7.0f + x)))))));
    } else {
        pr = c.k * drho;
    }
    if ((c.flags & FLAG_CLAMP) && pr < 0.0f) pr = 0.0f;
    if (!vol_boundary) c.prho[p] = make_float2(rho, pr / (rho * rho));   // else psi stays
    if (c.flags & FLAG_RECORD) c.nnbr[p] = acc.cnt - 1;
    report(c, bad);
}

// The volume-boundary variant is a separate instance, so the default path carries none of
// its per-neighbour tests.
// PAIRED = false keeps the register footprint of the one-at-a-time evaluation (kernels that
// carry more state, such as the batched phases), with the same results.
template <int THREADS, bool PAIRED = (SPH_DENSITY_PAIRED != 0)>
__device__ __forceinline__ void density_item(const SimConst &c, int blk)
{
    __shared__ int2 s_pend[kPending * THREADS];      // the block's pending neighbour masks
    if (c.flags & FLAG_VOLUME) density_item_v<true, THREADS, PAIRED>(c, blk, s_pend);
    else density_item_v<false, THREADS, PAIRED>(c, blk, s_pend);
}

// Low-latency density pass (SPH_FLAG_LOW_LATENCY; mass boundaries): G cooperating lanes
// per particle.  The lanes of a group set up the particle's clipped rows of cells together,
// test the flattened candidates G at a time (ascending slots, the order of the row walk),
// queue the neighbours in shared memory and evaluate them G at a time, one neighbour per
// lane, each lane summing its float-pair share; a shuffle tree of TwoSums adds the lanes'
// shares.  Same neighbours, same neighbour list (in the same order) and the same counts as
// density_item_v; the density sum, exact to ~1e-13 in any order, may round differently in
// its last bit.  A scene too small to fill the GPU waits for its slowest particles: a body
// sampled at half spacing has ~226 neighbours, which one thread walks and evaluates in
// series, and splitting them over G lanes shortens that chain (measured: the dam break's
// density pass 129 -> 25 us at G = 32).  On a scene that fills the GPU the group's set-up,
// compaction and queue round trips cost more than the lanes it keeps busy (the stirred
// coupled scene: 2.1x slower at best, G = 8; the 250k stirring tank 234 -> 387 us at G =
// 16), so the flag is for small interactive scenes.
template <int G>
__device__ __forceinline__ void density_coop_item(const SimConst &c, int blk)
{
    constexpr int kGroups = kTile / G;
    constexpr int kRowsMax = 36;                     // (z1 - z0 + 1) (y1 - y0 + 1) <= 6 x 6
    __shared__ int s_rs[kGroups][kRowsMax];          // first slot of each row's range
    __shared__ int s_pre[kGroups][kRowsMax + 1];     // exclusive prefix of the ranges' lengths
    __shared__ int s_nb[kGroups][2 * G];             // queued neighbours
    const int g = threadIdx.x / G, l = threadIdx.x % G;
    const int gbase = (threadIdx.x & 31) & ~(G - 1);
    const unsigned gmask = G == 32 ? 0xffffffffu : ((1u << G) - 1u) << gbase;
    const int p = blk * kGroups + g;
    if (p >= c.n) return;                            // the whole group
    const float4 xi = c.xA[p];
    uint32_t bad = 0;
    int kind = 0, excl_lo = 0, excl_n = 0;
    if (xi.w < 0.0f) pair_scope(c, __float_as_int(c.vA[p].w), kind, excl_lo, excl_n);
    const bool keep_list = kind != KIND_STATIC || (c.flags & FLAG_RECORD);
    const float *vw = reinterpret_cast<const float *>(c.vA) + 3;   // id bits, stride 4
    const bool near0 = near_origin_planes(c, xi);

    // rows of cells (bounds as for_each_row), G rows at a time
    const float ux = __fmul_rn(__fsub_rn(xi.x, c.o[0]), c.inv_cell);
    const float uy = __fmul_rn(__fsub_rn(xi.y, c.o[1]), c.inv_cell);
    const float uz = __fmul_rn(__fsub_rn(xi.z, c.o[2]), c.inv_cell);
    const float Rc = c.Rc, Rc2 = Rc * Rc, mc = c.mc;
    const int cy = cell_floor(uy, c.ny), cz = cell_floor(uz, c.nz);
    const int z0 = cell_floor(uz - Rc, c.nz), z1 = cell_floor(uz + Rc, c.nz);
    const int y0 = cell_floor(uy - Rc, c.ny), y1 = cell_floor(uy + Rc, c.ny);
    const int nyw = y1 - y0 + 1;
    if ((z1 - z0 + 1) * nyw > kRowsMax) bad |= ST_CAPACITY;   // the launcher keeps Rc < 2.5
    const int nrows = min((z1 - z0 + 1) * nyw, kRowsMax);
    for (int r = l; r < nrows; r += G) {
        const int z = z0 + r / nyw, y = y0 + r % nyw;
        const float gz = cell_gap(uz, z, cz, mc), gy = cell_gap(uy, y, cy, mc);
        const float w2 = (Rc2 - gz * gz) - gy * gy;
        int s0 = 0, len = 0;
        if (w2 >= 0.0f) {
            const float w = w2 * rsqrtf(fmaxf(w2, 1e-30f)) + mc;
            const int xa = cell_floor(ux - w, c.nx), xb = cell_floor(ux + w, c.nx);
            const int base = (z * c.ny + y) * c.nx;
            s0 = in_range(c, __ldg(c.cell_start + in_range(c, base + xa, c.ncell)), c.n + 1);
            const int e0 = in_range(c, __ldg(c.cell_start + in_range(c, base + xb + 1, c.ncell + 1)), c.n + 1);
            len = max(e0 - s0, 0);
            if (len > kMaxCellRun) { len = kMaxCellRun; bad |= ST_CAPACITY; }
        }
        s_rs[g][r] = s0;
        s_pre[g][r + 1] = len;
    }
    __syncwarp(gmask);
    if (l == 0) {
        int a = 0;
        s_pre[g][0] = 0;
        for (int r = 1; r <= nrows; ++r) { a += s_pre[g][r]; s_pre[g][r] = a; }
    }
    __syncwarp(gmask);
    const int T = s_pre[g][nrows];

    PairDensitySum acc;
    if (l == 0) acc.self(fabsf(xi.w));
    else acc.cnt = 0;
    int nq = 0;                                      // queued neighbours (group-uniform)
    int nl = 0;                                      // partners listed (group-uniform)
    int row = 0;                                     // row of the round's first candidate
    uint32_t *list = reinterpret_cast<uint32_t *>(c.nlist4 + p);
    const size_t lstride = 4 * (size_t)c.n;          // words between quads of one particle
    const unsigned lt = (1u << l) - 1u;
    // one neighbour per lane (lanes l < m): density term, and the partner list in queue order
    auto eval = [&](int m) {
        bool partner = false;
        int q = 0;
        if (l < m) {
            q = s_nb[g][l];
            const float4 xj = __ldg(c.xA + q);
            float dx, dy, dz, r2x;
            pair_offset(xi, xj, near0, dx, dy, dz, r2x);
            acc.add(c, fabsf(xj.w), 0.0f, dx, dy, dz, r2x);
            partner = keep_list &&
                      !(excl_n && (unsigned)(__float_as_int(__ldg(vw + 4 * (size_t)q)) - excl_lo) < (unsigned)excl_n);
        }
        const unsigned pb = (__ballot_sync(gmask, partner) >> gbase) & ((G == 32) ? 0xffffffffu : ((1u << G) - 1u));
        if (partner) {
            const int k = nl + __popc(pb & lt);
            if (k < c.nl_cap) list[(size_t)(k >> 2) * lstride + (k & 3)] = (uint32_t)q;
        }
        nl += __popc(pb);
    };
    for (int k0 = 0; k0 < T; k0 += G) {
        const int k = k0 + l;
        bool nbr = false;
        int q = 0;
        if (k < T) {
            int r = row;
            while (s_pre[g][r + 1] <= k) ++r;
            q = s_rs[g][r] + (k - s_pre[g][r]);
            const float4 xj = __ldg(c.xA + q);
            float dx, dy, dz;
            nbr = dist2(xi, xj, dx, dy, dz) < c.R2 && q != p;
        }
        {
            int r = row;
            const int kn = k0 + G;
            while (r < nrows && s_pre[g][r + 1] <= kn) ++r;
            row = r;
        }
        const unsigned bm = (__ballot_sync(gmask, nbr) >> gbase) & ((G == 32) ? 0xffffffffu : ((1u << G) - 1u));
        if (nbr) s_nb[g][nq + __popc(bm & lt)] = q;
        nq += __popc(bm);
        __syncwarp(gmask);
        if (nq >= G) {
            eval(G);
            __syncwarp(gmask);
            if (l < nq - G) s_nb[g][l] = s_nb[g][G + l];
            __syncwarp(gmask);
            nq -= G;
        }
    }
    if (nq > 0) eval(nq);

    // the lanes' shares, added by a fixed shuffle tree
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) {
        const float S2 = __shfl_down_sync(gmask, acc.S, off, G);
        const float L2 = __shfl_down_sync(gmask, acc.L, off, G);
        const int n2 = __shfl_down_sync(gmask, acc.cnt, off, G);
        const unsigned b2 = __shfl_down_sync(gmask, bad, off, G);
        float e;
        acc.S = two_sum(acc.S, S2, e);
        acc.L = __fadd_rn(acc.L, __fadd_rn(L2, e));
        acc.cnt += n2;
        bad |= b2;
    }
    if (l == 0) {
        c.nlist_n[p] = nl;
        const float drho = acc.excess(c, c.rho0);
        const float rho = __fadd_rn(c.rho0, drho);
        float pr;
        if (c.flags & FLAG_TAIT) {
            const float x = drho / c.rho0;
            pr = c.tait_B * (x * (7.0f + x * (21.0f + x * (35.0f + x * (35.0f + x * (21.0f + x * (7.0f + x)))))));
        } else {
            pr = c.k * drho;
        }
        if ((c.flags & FLAG_CLAMP) && pr < 0.0f) pr = 0.0f;
        c.prho[p] = make_float2(rho, pr / (rho * rho));
        if (c.flags & FLAG_RECORD) c.nnbr[p] = acc.cnt - 1;
        report(c, bad);
    }
}

#if SPH_DENSITY_BRICK
// Alternative density pass, built only with -DSPH_DENSITY_BRICK=1 (and SPH_BRICK_X/Y/Z/CAP):
// one CTA per brick of kBX x kBY x kBZ cells.  The positions of the brick's cells and of a
// halo of kBH cells around them are staged in shared memory once (row by row: the slots of
// a row of cells are contiguous), and every particle of the brick walks its rows against
// the staged copy; rows outside it, which the FP32 margin of the search can add, are read
// from global memory.  Same neighbours in the same order as density_item_v, hence the same
// results bit for bit.  Mass boundaries only (volume boundaries keep density_item_v).
// Measured against the row walk on the stirred coupled scene and rejected (1.76x slower at
// best): it executes as many instructions plus the staging, and the bricks' uneven particle
// counts (h/2 walls, air above the free surface) leave thread slots idle.
constexpr int kBX = SPH_BRICK_X, kBY = SPH_BRICK_Y, kBZ = SPH_BRICK_Z, kBH = 2;
constexpr int kSY = kBY + 2 * kBH, kSZ = kBZ + 2 * kBH, kSRows = kSY * kSZ;
constexpr int kStageCap = SPH_BRICK_CAP;
constexpr int kBrickThreads = 512;

struct BrickShared {
    float4 x[kStageCap];
    int2 pend[kPending * kBrickThreads];
    int pdel[kPending * kBrickThreads];
    int row_g[kSRows], row_s[kSRows], row_n[kSRows], row_xs[kSRows], row_xe[kSRows];
    int inner_pre[kBY * kBZ + 1];
    int ok;
};

__device__ __forceinline__ void density_brick(const SimConst &c, BrickShared &sh)
{
    const int x0 = blockIdx.x * kBX, y0 = blockIdx.y * kBY, z0 = blockIdx.z * kBZ;
    const int tid = threadIdx.x;
    // rows of the staged block: counts, then offsets
    if (tid < kSRows) {
        const int zz = z0 - kBH + tid / kSY, yy = y0 - kBH + tid % kSY;
        int g = 0, n = 0, xs = 0, xe = 0;
        if (zz >= 0 && zz < c.nz && yy >= 0 && yy < c.ny) {
            xs = max(x0 - kBH, 0);
            xe = min(x0 + kBX + kBH, c.nx);
            const int base = (zz * c.ny + yy) * c.nx;
            g = (int)__ldg(c.cell_start + base + xs);
            n = (int)__ldg(c.cell_start + base + xe) - g;
        }
        sh.row_g[tid] = g;
        sh.row_n[tid] = n;
        sh.row_xs[tid] = xs;
        sh.row_xe[tid] = xe;
    }
    if (tid == 0) {
        int pre = 0;
        for (int k = 0; k <= kBY * kBZ; ++k) {
            sh.inner_pre[k] = pre;
            if (k == kBY * kBZ) break;
            const int zz = z0 + k / kBY, yy = y0 + k % kBY;
            if (zz < c.nz && yy < c.ny && x0 < c.nx) {
                const int base = (zz * c.ny + yy) * c.nx;
                pre += (int)__ldg(c.cell_start + base + min(x0 + kBX, c.nx)) - (int)__ldg(c.cell_start + base + x0);
            }
        }
    }
    __syncthreads();
    const int n_inner = sh.inner_pre[kBY * kBZ];
    if (n_inner == 0) return;
    if (tid == 0) {
        int off = 0;
        for (int r = 0; r < kSRows; ++r) {
            sh.row_s[r] = off;
            off += sh.row_n[r];
        }
        sh.ok = off <= kStageCap;
    }
    __syncthreads();
    const bool ok = sh.ok;
    if (ok) {
        // each warp copies whole rows
        const int warp = tid >> 5, lane = tid & 31;
        for (int r = warp; r < kSRows; r += kBrickThreads / 32) {
            const int g = sh.row_g[r], s0 = sh.row_s[r], n = sh.row_n[r];
            for (int k = lane; k < n; k += 32) sh.x[s0 + k] = __ldg(c.xA + g + k);
        }
    }
    __syncthreads();

    for (int item = tid; item < n_inner; item += kBrickThreads) {
        // the particle's inner row and slot
        int ir = 0;
        while (sh.inner_pre[ir + 1] <= item) ++ir;
        const int zz = z0 + ir / kBY, yy = y0 + ir % kBY;
        const int p = (int)__ldg(c.cell_start + (zz * c.ny + yy) * c.nx + x0) + (item - sh.inner_pre[ir]);
        const float4 xi = c.xA[p];
        uint32_t bad = 0;
        int kind = 0, excl_lo = 0, excl_n = 0;
        if (xi.w < 0.0f) pair_scope(c, __float_as_int(c.vA[p].w), kind, excl_lo, excl_n);
        const bool keep_list = kind != KIND_STATIC || (c.flags & FLAG_RECORD);
        const float *vw = reinterpret_cast<const float *>(c.vA) + 3;
        const bool near0 = near_origin_planes(c, xi);
        PairDensitySum acc;
        acc.self(fabsf(xi.w));
        ListWriter list;
        list.dst = c.nlist4 + p;
        list.n = (size_t)c.n;
        list.cap = c.nl_cap;
        int2 *pend = sh.pend + tid;
        int *pdel = sh.pdel + tid;
        int np = 0;
        constexpr int kGlobal = -2147483647 - 1;
        auto drain = [&]() {
            if (np == 0) return;
            int k = 0;
            int2 e = pend[0];
            int d = pdel[0];
            uint32_t mm = (uint32_t)e.y;
            for (;;) {
                if (mm == 0u) {
                    if (++k == np) break;
                    e = pend[k * kBrickThreads];
                    d = pdel[k * kBrickThreads];
                    mm = (uint32_t)e.y;
                }
                const int qs = e.x + __ffs(mm) - 1;
                mm &= mm - 1u;
                float4 xj;
                int q;
                if (d != kGlobal) { xj = sh.x[qs]; q = qs + d; }
                else { q = qs; xj = __ldg(c.xA + q); }
                float dx, dy, dz, r2x;
                pair_offset(xi, xj, near0, dx, dy, dz, r2x);
                acc.add(c, fabsf(xj.w), 0.0f, dx, dy, dz, r2x);
                if (!keep_list) continue;
                if (excl_n && (unsigned)(__float_as_int(__ldg(vw + 4 * (size_t)q)) - excl_lo) < (unsigned)excl_n)
                    continue;
                list.push((uint32_t)q);
            }
            np = 0;
        };
        const float ux = __fmul_rn(__fsub_rn(xi.x, c.o[0]), c.inv_cell);
        const float uy = __fmul_rn(__fsub_rn(xi.y, c.o[1]), c.inv_cell);
        const float uz = __fmul_rn(__fsub_rn(xi.z, c.o[2]), c.inv_cell);
        const float Rc = c.Rc, Rc2 = Rc * Rc, mc = c.mc;
        const int cy = cell_floor(uy, c.ny), cz = cell_floor(uz, c.nz);
        const int zl = cell_floor(uz - Rc, c.nz), zh = cell_floor(uz + Rc, c.nz);
        const int yl = cell_floor(uy - Rc, c.ny), yh = cell_floor(uy + Rc, c.ny);
#pragma unroll 1
        for (int z = zl; z <= zh; ++z) {
            const float gz = cell_gap(uz, z, cz, mc);
            const float rz2 = Rc2 - gz * gz;
#pragma unroll 1
            for (int y = yl; y <= yh; ++y) {
                const float gy = cell_gap(uy, y, cy, mc);
                const float w2 = rz2 - gy * gy;
                if (!(w2 >= 0.0f)) continue;
                const float w = w2 * rsqrtf(fmaxf(w2, 1e-30f)) + mc;
                const int xa = cell_floor(ux - w, c.nx), xb = cell_floor(ux + w, c.nx);
                const int base = (z * c.ny + y) * c.nx;
                const int s0 = in_range(c, __ldg(c.cell_start + in_range(c, base + xa, c.ncell)), c.n + 1);
                int e0 = in_range(c, __ldg(c.cell_start + in_range(c, base + xb + 1, c.ncell + 1)), c.n + 1);
                if (e0 - s0 > kMaxCellRun) { e0 = s0 + kMaxCellRun; bad |= ST_CAPACITY; }
                // staged row?
                const int rz = z - (z0 - kBH), ry = y - (y0 - kBH);
                int d = kGlobal;
                if (ok && (unsigned)rz < (unsigned)kSZ && (unsigned)ry < (unsigned)kSY) {
                    const int r = rz * kSY + ry;
                    if (xa >= sh.row_xs[r] && xb < sh.row_xe[r]) d = sh.row_g[r] - sh.row_s[r];
                }
                const int sb = d == kGlobal ? s0 : s0 - d, se = d == kGlobal ? e0 : e0 - d;
                const int pself = d == kGlobal ? p : p - d;
#pragma unroll 1
                for (int b = sb; b < se; b += 32) {
                    const int end = min(se, b + 32);
                    uint32_t mm = 0u, bit = 1u;
                    if (d != kGlobal) {
#pragma unroll kMaskUnroll
                        for (int q = b; q < end; ++q) {
                            const float4 xj = sh.x[q];
                            float dx, dy, dz;
                            if (dist2(xi, xj, dx, dy, dz) < c.R2) mm |= bit;
                            bit <<= 1;
                        }
                    } else {
#pragma unroll kMaskUnroll
                        for (int q = b; q < end; ++q) {
                            const float4 xj = __ldg(c.xA + q);
                            float dx, dy, dz;
                            if (dist2(xi, xj, dx, dy, dz) < c.R2) mm |= bit;
                            bit <<= 1;
                        }
                    }
                    if ((unsigned)(pself - b) < 32u) mm &= ~(1u << (pself - b));
                    if (!mm) continue;
                    if (np == kPending) drain();
                    pend[np * kBrickThreads] = make_int2(b, (int)mm);
                    pdel[np * kBrickThreads] = d;
                    ++np;
                }
            }
            if (np > kDrainAt) drain();
        }
        drain();
        list.flush();
        c.nlist_n[p] = list.nl;
        const float drho = acc.excess(c, c.rho0);
        const float rho = __fadd_rn(c.rho0, drho);
        float pr;
        if (c.flags & FLAG_TAIT) {
            const float x = drho / c.rho0;
            pr = c.tait_B * (x * (7.0f + x * (21.0f + x * (35.0f + x * (35.0f + x * (21.0f + x * (7.0f + x)))))));
        } else {
            pr = c.k * drho;
        }
        if ((c.flags & FLAG_CLAMP) && pr < 0.0f) pr = 0.0f;
        c.prho[p] = make_float2(rho, pr / (rho * rho));
        if (c.flags & FLAG_RECORD) c.nnbr[p] = acc.cnt - 1;
        report(c, bad);
    }
}
#endif

// Volume-based boundaries (Akinci et al.): each static or rigid particle's weight
// psi_b = rho0 / sum_{k boundary} W_bk (self included), stored in its (rho, P) slot as
// (psi_b, its low part) before the density pass reads it.
__device__ __forceinline__ void boundary_volume_item(const SimConst &c, int blk)
{
    const int p = blk * kTile + threadIdx.x;
    if (p >= c.n) return;
    const float4 xi = c.xA[p];
    if (!(xi.w < 0.0f)) return;
    const bool near0 = near_origin_planes(c, xi);
    PairDensitySum acc;
    acc.self(1.0f);
    uint32_t bad = 0;
    for_each_row(c, xi, bad, [&](int s0, int e0) {
        for (int q = s0; q < e0; ++q) {
            const float4 xj = __ldg(c.xA + q);
            if (q == p || !(xj.w < 0.0f)) continue;
            float dx, dy, dz;
            if (!(dist2(xi, xj, dx, dy, dz) < c.R2)) continue;
            float r2x;
            pair_offset(xi, xj, near0, dx, dy, dz, r2x);
            acc.add(c, 1.0f, 0.0f, dx, dy, dz, r2x);
        }
    });
    // sum W = alpha6 (S + L) as a float pair (Wh, Wl); psi = rho0 / sum W as a float pair
    const float Wh = __fmul_rn(c.alpha6_hi, acc.S);
    const float Wl = __fadd_rn(__fmaf_rn(c.alpha6_hi, acc.S, -Wh),
                               __fmaf_rn(c.alpha6_lo, acc.S, __fmul_rn(c.alpha6_hi, acc.L)));
    const float ph = __fdiv_rn(c.rho0, Wh);
    const float pl = __fdiv_rn(__fmaf_rn(-ph, Wl, __fmaf_rn(-ph, Wh, c.rho0)), Wh);
    c.prho[p] = make_float2(ph, pl);
    report(c, bad);
}

// -------------------------------------------------------------- force + integrate

// The end of a force-pass particle: the pair force, its soft springs, the explicit Euler
// step (Eq. euler) for a fluid or soft particle or the coupling force of a boundary one,
// the writes and the particle's diagnostic values dg (pair force xyz, |f|, m v xyz, m|v|).
__device__ __forceinline__ void force_tail(const SimConst &c, int p, float4 xi, float4 vi, int id, int kind,
                                           float mi, float ax, float ay, float az, float (&dg)[8],
                                           uint32_t &bad)
{
    float fx = mi * ax, fy = mi * ay, fz = mi * az;   // pair force on i
    dg[0] = fx; dg[1] = fy; dg[2] = fz;
    dg[3] = sqrtf(fx * fx + fy * fy + fz * fz);
    if (kind == 0 || kind == KIND_SOFT) {
        float sx = 0.0f, sy = 0.0f, sz = 0.0f;
        bool anchored = false;
        if (kind == KIND_SOFT) {
            int l = in_range(c, id - c.nf, c.n_body_particles);
            anchored = c.locals[l].w != 0.0f;      // pinned soft particle (cloth anchor)
            for (int e = c.spring_row[l]; e < c.spring_row[l + 1]; ++e) {
                float4 sp = c.spring_e[e];
                if (sp.z == 0.0f && sp.w == 0.0f) continue;   // cut spring
                int q = in_range(c, c.slot_of_id[in_range(c, __float_as_int(sp.x), c.n)], c.n);
                float4 xj = c.xA[q], vj = c.vA[q];
                float d0 = xi.x - xj.x, d1 = xi.y - xj.y, d2 = xi.z - xj.z;
                float L = sqrtf(d0 * d0 + d1 * d1 + d2 * d2);
                float il = 1.0f / L;
                d0 *= il; d1 *= il; d2 *= il;
                float vr = (vi.x - vj.x) * d0 + (vi.y - vj.y) * d1 + (vi.z - vj.z) * d2;
                float f = -sp.z * (L - sp.y) - sp.w * vr;
                sx += f * d0; sy += f * d1; sz += f * d2;
            }
        }
        float im = 1.0f / mi;
        float a0 = ax + sx * im + c.g[0];
        float a1 = ay + sy * im + c.g[1];
        float a2 = az + sz * im + c.g[2];
        float4 vn = make_float4(vi.x + a0 * c.dt, vi.y + a1 * c.dt, vi.z + a2 * c.dt, vi.w);
        float4 xn = make_float4(xi.x + vn.x * c.dt, xi.y + vn.y * c.dt, xi.z + vn.z * c.dt, xi.w);
        if (anchored) {                        // an anchor stays where it is, at rest
            vn = make_float4(0.0f, 0.0f, 0.0f, vi.w);
            xn = xi;
        }
        if (!(isfinite(xn.x) && isfinite(xn.y) && isfinite(xn.z))) bad |= ST_NONFINITE;
        c.xB[p] = xn;
        c.vB[p] = vn;
        dg[4] = mi * vn.x; dg[5] = mi * vn.y; dg[6] = mi * vn.z;
        dg[7] = mi * sqrtf(vn.x * vn.x + vn.y * vn.y + vn.z * vn.z);
        if (c.flags & FLAG_RECORD) c.acc_dbg[p] = make_float4(a0, a1, a2, 0.0f);
    } else {
        c.xB[p] = xi;
        c.vB[p] = vi;
        int l = in_range(c, id - c.nf, c.n_body_particles);
        c.fb[l] = make_float4(fx, fy, fz, 0.0f);
        c.xb[l] = xi;
        if (c.flags & FLAG_RECORD) c.acc_dbg[p] = make_float4(ax, ay, az, 0.0f);
    }
}

// The block's row of the momentum diagnostics (dg summed over its particles): FP32 within
// the warp, FP64 above it; the last warp of the block to finish sums the per-warp partials
// in a fixed order (no block barrier, so no warp waits for another).
__device__ __forceinline__ void force_diag_row(const SimConst &c, int blk, const float (&dg)[8],
                                               double (&sd)[8][8], unsigned &s_done)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    {
        // the 8 warp sums by a halving exchange: after the xor-16, -8 and -4 steps each lane
        // holds one component (bits 4, 3, 2 of the lane pick it), then xor-2 and -1 finish
        const unsigned full = 0xffffffffu;
        const bool h16 = lane & 16, h8 = lane & 8, h4 = lane & 4;
        float v4[4], v2[2];
#pragma unroll
        for (int k = 0; k < 4; ++k)
            v4[k] = (h16 ? dg[k + 4] : dg[k]) + __shfl_xor_sync(full, h16 ? dg[k] : dg[k + 4], 16);
#pragma unroll
        for (int k = 0; k < 2; ++k)
            v2[k] = (h8 ? v4[k + 2] : v4[k]) + __shfl_xor_sync(full, h8 ? v4[k] : v4[k + 2], 8);
        float v1 = (h4 ? v2[1] : v2[0]) + __shfl_xor_sync(full, h4 ? v2[0] : v2[1], 4);
        v1 += __shfl_xor_sync(full, v1, 2);
        v1 += __shfl_xor_sync(full, v1, 1);
        if ((lane & 3) == 0) sd[wid][(h16 ? 4 : 0) + (h8 ? 2 : 0) + (h4 ? 1 : 0)] = (double)v1;
    }
    unsigned last = 0;
    if (lane == 0) {
        __threadfence_block();
        last = atomicAdd(&s_done, 1u) == (blockDim.x >> 5) - 1;
    }
    last = __shfl_sync(0xffffffffu, last, 0);
    if (last && lane < 8) {
        __threadfence_block();
        volatile double *v = &sd[0][0];
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += v[w * 8 + lane];
        c.diag_part[(size_t)blk * 8 + lane] = t;
    }
}

template <bool VOL>
__device__ __forceinline__ void force_item_v(const SimConst &c, int blk)
{
    __shared__ double sd[8][8];
    __shared__ unsigned s_done;
    if (threadIdx.x == 0) s_done = 0u;
    __syncthreads();
    const int p = blk * kTile + threadIdx.x;
    float dg[8] = {0, 0, 0, 0, 0, 0, 0, 0};   // pair force xyz, |f|, m v xyz, m|v|
    uint32_t bad = 0;
    if (p < c.n) {
        const float4 xi = c.xA[p];
        const float4 vi = c.vA[p];
        const float2 pi = c.prho[p];
        const int id = __float_as_int(vi.w);
        const float mi = fabsf(xi.w);
        int kind, excl_lo, excl_n;
        pair_scope(c, id, kind, excl_lo, excl_n);
        const bool skip = (kind == KIND_STATIC) && !(c.flags & FLAG_RECORD);
        constexpr bool vol = VOL;
        const float inv_mi = 1.0f / mi;
        const bool near0 = near_origin_planes(c, xi);
        float ax = 0.0f, ay = 0.0f, az = 0.0f;
        // The pressure term sum_j m_j (P_i + P_j) gq_j d_j is split as
        //   P_i * sum_j 2 m_j gq_j d_j  +  sum_j m_j (P_j - P_i) gq_j d_j :
        // at depth every pair term is large (P ~ rho0 g d / rho^2) and the sum cancels to
        // about the weight, so FP32 pair terms alone would carry errors of the order of the
        // acceptance bar.  The first sum is purely geometric and taken exactly (float pairs,
        // PairGradSum); the second has terms about (P_j - P_i) / P_i smaller (P_j - P_i is
        // exact, Sterbenz) and stays FP32 together with the viscous term.
        PairGradSum G;
        if (!skip) {
            // check_own: skip the particle's own rigid body (the neighbour list has no such
            // entries, so only the re-search needs the test)
            auto pair = [&](float4 xj, float4 vj, float2 pj, float dx, float dy, float dz, float r2,
                            bool check_own) {
                int jd = __float_as_int(vj.w);
                if (check_own && (unsigned)(jd - excl_lo) < (unsigned)excl_n) return;
                const bool bi = xi.w < 0.0f, bj = xj.w < 0.0f;
                if (vol && bi && bj) return;       // volume boundaries: no boundary pairs
                float r2x, lx, ly, lz;
                pair_offset(xi, xj, near0, dx, dy, dz, r2x, lx, ly, lz);
                const PairQ pq = pair_q(c, dx, dy, dz, r2x);
                // w'(q)/q of the cubic spline as a float pair (finite at q -> 0; coincident
                // particles have d = 0 and exert no force)
                float gl;
                const float gq = gradq_pair(pq.qh, pq.ql, gl);
                // v_ij . x_ij with x_ij = -d
                float vx = -((vi.x - vj.x) * dx + (vi.y - vj.y) * dy + (vi.z - vj.z) * dz);
                float coef;
                if (vol && (bi || bj)) {
                    // the fluid side's density and pressure only; the boundary side
                    // weighs psi (its (rho, P) slot holds psi as a float pair)
                    const float rf = bi ? pj.x : pi.x, Pf = bi ? pj.y : pi.y;
                    const float w = bi ? fabsf(xj.w) * pi.x * inv_mi : pj.x;
                    const float visc = __fdividef(c.nu20 * vx, (rf + rf) * (r2 + c.eps_h2));
                    if (bi) {
                        coef = w * (visc - Pf) * gq;
                    } else {                       // fluid i: -P_i w gq d goes to G
                        coef = w * visc * gq;
                        G.add(w, gq, gl, dx, dy, dz, lx, ly, lz);
                    }
                } else {
                    const float mj = fabsf(xj.w);
                    float visc = __fdividef(c.nu20 * vx, (pi.x + pj.x) * (r2 + c.eps_h2));
                    coef = mj * (visc - __fsub_rn(pj.y, pi.y)) * gq;
                    G.add(__fmul_rn(2.0f, mj), gq, gl, dx, dy, dz, lx, ly, lz);
                }
                ax -= coef * dx;
                ay -= coef * dy;
                az -= coef * dz;
            };
            const int nl = __ldg(c.nlist_n + p);
            if (nl <= c.nl_cap) {
                // the partners the density pass recorded, four per 16-byte load; the next
                // quad is fetched while this one is evaluated
                const uint4 *lq = c.nlist4 + p;
                uint4 nxt = nl > 0 ? __ldg(lq) : make_uint4(0u, 0u, 0u, 0u);
                for (int g = 0; 4 * g < nl; ++g) {
                    const uint4 e = nxt;
                    if (4 * (g + 1) < nl) nxt = __ldg(lq + (size_t)(g + 1) * c.n);
                    const int m = min(4, nl - 4 * g);
#if SPH_FORCE_BATCH > 1
                    // all of the quad's neighbour loads are issued before the first pair is
                    // evaluated (a short last quad repeats its first entry, unused)
                    constexpr int B = SPH_FORCE_BATCH;
                    const uint32_t qq[4] = {e.x, m > 1 ? e.y : e.x, m > 2 ? e.z : e.x, m > 3 ? e.w : e.x};
#pragma unroll
                    for (int j0 = 0; j0 < 4; j0 += B) {
                        float4 xs[B], vs[B];
                        float2 ps[B];
#pragma unroll
                        for (int j = 0; j < B; ++j) {
                            const int q = in_range(c, qq[j0 + j], c.n);
                            xs[j] = __ldg(c.xA + q);
                            vs[j] = __ldg(c.vA + q);
                            ps[j] = __ldg(c.prho + q);
                        }
#pragma unroll
                        for (int j = 0; j < B; ++j) {
                            if (j0 + j < m) {
                                float dx, dy, dz;
                                const float r2 = dist2(xi, xs[j], dx, dy, dz);
                                pair(xs[j], vs[j], ps[j], dx, dy, dz, r2, false);
                            }
                        }
                    }
#else
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        if (j >= m) break;
                        const int q = in_range(c, j == 0 ? e.x : j == 1 ? e.y : j == 2 ? e.z : e.w, c.n);
                        const float4 xj = __ldg(c.xA + q);
                        float dx, dy, dz;
                        const float r2 = dist2(xi, xj, dx, dy, dz);
                        pair(xj, __ldg(c.vA + q), __ldg(c.prho + q), dx, dy, dz, r2, false);
                    }
#endif
                }
            } else {
                // more partners than list slots: search again
                for_each_row(c, xi, bad, [&](int s0, int e0) {
                    for (int q = s0; q < e0; ++q) {
                        if (q == p) continue;
                        const float4 xj = __ldg(c.xA + q);
                        float dx, dy, dz;
                        const float r2 = dist2(xi, xj, dx, dy, dz);
                        if (r2 < c.R2) pair(xj, __ldg(c.vA + q), __ldg(c.prho + q), dx, dy, dz, r2, true);
                    }
                });
            }
            // + P_i * G (G cancels to ~0 in a full neighbourhood, so one rounding suffices)
            ax = __fmaf_rn(pi.y, __fadd_rn(G.Sx, G.Lx), ax);
            ay = __fmaf_rn(pi.y, __fadd_rn(G.Sy, G.Ly), ay);
            az = __fmaf_rn(pi.y, __fadd_rn(G.Sz, G.Lz), az);
            ax *= c.alpha_g;
            ay *= c.alpha_g;
            az *= c.alpha_g;
        }
        force_tail(c, p, xi, vi, id, kind, mi, ax, ay, az, dg, bad);
    }
    report(c, bad);
    force_diag_row(c, blk, dg, sd, s_done);
}

__device__ __forceinline__ void force_item(const SimConst &c, int blk)
{
    if (c.flags & FLAG_VOLUME) force_item_v<true>(c, blk);
    else force_item_v<false>(c, blk);
}

// Low-latency force pass (SPH_FLAG_LOW_LATENCY; mass boundaries): G cooperating lanes per
// particle, for scenes too small to fill the GPU, whose force pass waits for the serial
// partner loop of each fluid particle (~37 partners, two dependent loads each).  Lane l of a
// group evaluates partners l, l + G, ... of the particle's list (or, past the list's
// capacity, every G-th candidate of the row walk) with the pair terms of force_item_v; a
// fixed shuffle tree adds the lanes' FP32 sums and, by TwoSums, their float-pair kernel-
// gradient sums; lane 0 then does the springs, the integration, the writes and the
// diagnostics.  The same forces up to the order of the FP32 sums.  The grid has G blocks
// for each 256 particles, each writing its own diagnostic row (n_force_blocks is set to
// match for flagged scenes).
template <int G>
__device__ __forceinline__ void force_coop_item(const SimConst &c, int blk)
{
    __shared__ double sd[8][8];
    __shared__ unsigned s_done;
    if (threadIdx.x == 0) s_done = 0u;
    __syncthreads();
    constexpr int kGroups = kTile / G;
    const int l = threadIdx.x % G;
    const int gbase = (threadIdx.x & 31) & ~(G - 1);
    const unsigned gmask = G == 32 ? 0xffffffffu : ((1u << G) - 1u) << gbase;
    const int p = blk * kGroups + (int)threadIdx.x / G;
    float dg[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    uint32_t bad = 0;
    if (p < c.n) {                                   // group-uniform
        const float4 xi = c.xA[p];
        const float4 vi = c.vA[p];
        const float2 pi = c.prho[p];
        const int id = __float_as_int(vi.w);
        const float mi = fabsf(xi.w);
        int kind, excl_lo, excl_n;
        pair_scope(c, id, kind, excl_lo, excl_n);
        const bool skip = (kind == KIND_STATIC) && !(c.flags & FLAG_RECORD);
        const bool near0 = near_origin_planes(c, xi);
        float ax = 0.0f, ay = 0.0f, az = 0.0f;
        PairGradSum Gs;
        if (!skip) {
            auto pair = [&](float4 xj, float4 vj, float2 pj, float dx, float dy, float dz, float r2,
                            bool check_own) {
                const int jd = __float_as_int(vj.w);
                if (check_own && (unsigned)(jd - excl_lo) < (unsigned)excl_n) return;
                float r2x, lx, ly, lz;
                pair_offset(xi, xj, near0, dx, dy, dz, r2x, lx, ly, lz);
                const PairQ pq = pair_q(c, dx, dy, dz, r2x);
                float gl;
                const float gq = gradq_pair(pq.qh, pq.ql, gl);
                const float vx = -((vi.x - vj.x) * dx + (vi.y - vj.y) * dy + (vi.z - vj.z) * dz);
                const float mj = fabsf(xj.w);
                const float visc = __fdividef(c.nu20 * vx, (pi.x + pj.x) * (r2 + c.eps_h2));
                const float coef = mj * (visc - __fsub_rn(pj.y, pi.y)) * gq;
                Gs.add(__fmul_rn(2.0f, mj), gq, gl, dx, dy, dz, lx, ly, lz);
                ax -= coef * dx;
                ay -= coef * dy;
                az -= coef * dz;
            };
            const int nl = __ldg(c.nlist_n + p);
            if (nl <= c.nl_cap) {
                // entry k: component k % 4 of quad (k / 4) of the particle
                const uint32_t *list = reinterpret_cast<const uint32_t *>(c.nlist4 + p);
                const size_t lstride = 4 * (size_t)c.n;
                for (int k = l; k < nl; k += G) {
                    const int q = in_range(c, (int)__ldg(list + (size_t)(k >> 2) * lstride + (k & 3)), c.n);
                    const float4 xj = __ldg(c.xA + q);
                    float dx, dy, dz;
                    const float r2 = dist2(xi, xj, dx, dy, dz);
                    pair(xj, __ldg(c.vA + q), __ldg(c.prho + q), dx, dy, dz, r2, false);
                }
            } else {
                // more partners than list slots: every G-th candidate of the row walk
                int t = 0;
                for_each_row(c, xi, bad, [&](int s0, int e0) {
                    for (int q = s0; q < e0; ++q, ++t) {
                        if (q == p || t % G != l) continue;
                        const float4 xj = __ldg(c.xA + q);
                        float dx, dy, dz;
                        const float r2 = dist2(xi, xj, dx, dy, dz);
                        if (r2 < c.R2) pair(xj, __ldg(c.vA + q), __ldg(c.prho + q), dx, dy, dz, r2, true);
                    }
                });
            }
        }
        // the lanes' shares, added by a fixed shuffle tree (lane 0 of the group holds the sums)
#pragma unroll
        for (int off = G / 2; off > 0; off >>= 1) {
            ax = __fadd_rn(ax, __shfl_down_sync(gmask, ax, off, G));
            ay = __fadd_rn(ay, __shfl_down_sync(gmask, ay, off, G));
            az = __fadd_rn(az, __shfl_down_sync(gmask, az, off, G));
            float e;
            const float sx = __shfl_down_sync(gmask, Gs.Sx, off, G), lx = __shfl_down_sync(gmask, Gs.Lx, off, G);
            const float sy = __shfl_down_sync(gmask, Gs.Sy, off, G), ly = __shfl_down_sync(gmask, Gs.Ly, off, G);
            const float sz = __shfl_down_sync(gmask, Gs.Sz, off, G), lz = __shfl_down_sync(gmask, Gs.Lz, off, G);
            Gs.Sx = two_sum(Gs.Sx, sx, e);
            Gs.Lx = __fadd_rn(Gs.Lx, __fadd_rn(lx, e));
            Gs.Sy = two_sum(Gs.Sy, sy, e);
            Gs.Ly = __fadd_rn(Gs.Ly, __fadd_rn(ly, e));
            Gs.Sz = two_sum(Gs.Sz, sz, e);
            Gs.Lz = __fadd_rn(Gs.Lz, __fadd_rn(lz, e));
            bad |= __shfl_down_sync(gmask, bad, off, G);
        }
        if (l == 0) {
            if (!skip) {
                ax = __fmaf_rn(pi.y, __fadd_rn(Gs.Sx, Gs.Lx), ax);
                ay = __fmaf_rn(pi.y, __fadd_rn(Gs.Sy, Gs.Ly), ay);
                az = __fmaf_rn(pi.y, __fadd_rn(Gs.Sz, Gs.Lz), az);
                ax *= c.alpha_g;
                ay *= c.alpha_g;
                az *= c.alpha_g;
            }
            force_tail(c, p, xi, vi, id, kind, mi, ax, ay, az, dg, bad);
        }
    }
    if (l == 0) report(c, bad);
    force_diag_row(c, blk, dg, sd, s_done);   // only lane 0 of a group holds values
}

// ------------------------------------------------------------------ spring cutting

struct Blade {
    float v[9];                // triangle corners v0, v1, v2
};

// Does segment a-b meet triangle t (closed)?  Moller and Trumbore's ray-triangle test in
// FP32, with the segment parameter limited to [0, 1]; parallel (|det| tiny) counts as no.
__device__ __forceinline__ bool segment_meets_triangle(float3 a, float3 b, const Blade &t)
{
    const float e1x = t.v[3] - t.v[0], e1y = t.v[4] - t.v[1], e1z = t.v[5] - t.v[2];
    const float e2x = t.v[6] - t.v[0], e2y = t.v[7] - t.v[1], e2z = t.v[8] - t.v[2];
    const float dx = b.x - a.x, dy = b.y - a.y, dz = b.z - a.z;
    const float px = dy * e2z - dz * e2y, py = dz * e2x - dx * e2z, pz = dx * e2y - dy * e2x;
    const float det = e1x * px + e1y * py + e1z * pz;
    const float scale = (fabsf(e1x) + fabsf(e1y) + fabsf(e1z)) * (fabsf(px) + fabsf(py) + fabsf(pz));
    if (!(fabsf(det) > 1e-7f * scale)) return false;
    const float inv = 1.0f / det;
    const float tx = a.x - t.v[0], ty = a.y - t.v[1], tz = a.z - t.v[2];
    const float u = (tx * px + ty * py + tz * pz) * inv;
    if (u < 0.0f || u > 1.0f) return false;
    const float qx = ty * e1z - tz * e1y, qy = tz * e1x - tx * e1z, qz = tx * e1y - ty * e1x;
    const float v = (dx * qx + dy * qy + dz * qz) * inv;
    if (v < 0.0f || u + v > 1.0f) return false;
    const float s = (e2x * qx + e2y * qy + e2z * qz) * inv;
    return s >= 0.0f && s <= 1.0f;
}

// Cuts (sets k_s = c_d = 0) every active spring of a soft body whose current segment meets
// the blade.  One thread per body particle over its CSR row; both entries of a spring
// decide on the same endpoint order (lower id first), so they agree.  Reads the sorted
// copy of the current state (the caller sorts it first), where slot_of_id points.
__device__ __forceinline__ void cut_item(const SimConst &c, int blk, const Blade &t, unsigned *count)
{
    const int l = blk * kTile + threadIdx.x;
    if (l >= c.n - c.nf) return;
    const int id = c.nf + l;
    if (c.body_kind[body_of(c, id)] != KIND_SOFT) return;
    for (int e = c.spring_row[l]; e < c.spring_row[l + 1]; ++e) {
        float4 sp = c.spring_e[e];
        if (sp.z == 0.0f && sp.w == 0.0f) continue;
        const int pid = __float_as_int(sp.x);
        const int lo = in_range(c, min(id, pid), c.n), hi = in_range(c, max(id, pid), c.n);
        const float4 xa = c.xA[in_range(c, c.slot_of_id[lo], c.n)];
        const float4 xb = c.xA[in_range(c, c.slot_of_id[hi], c.n)];
        if (!segment_meets_triangle(make_float3(xa.x, xa.y, xa.z), make_float3(xb.x, xb.y, xb.z), t))
            continue;
        sp.z = 0.0f;
        sp.w = 0.0f;
        c.spring_e[e] = sp;
        if (id == lo) atomicAdd(count, 1u);
    }
}

// ------------------------------------------------------- FP64 wrench + rigid update

static __device__ void rot_f64(const double q[4], double R[9])
{
    double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

static __device__ void grab_point(const Pose &P, const DevBody &B, double xg[3], double R[9])
{
    double q[4] = {P.q[0], P.q[1], P.q[2], P.q[3]};
    rot_f64(q, R);
    for (int a = 0; a < 3; ++a)
        xg[a] = R[3 * a] * B.grab_local[0] + R[3 * a + 1] * B.grab_local[1] +
                R[3 * a + 2] * B.grab_local[2] + (double)P.t[a];
}

static __device__ void cross3d(const double a[3], const double b[3], double o[3])
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

// Semi-implicit rigid update in FP64 from the FP64 wrench (force, torque about x_g).
static __device__ void rigid_update(const SimConst &c, DevBody &B, const Pose &P, const double W[6])
{
    double R[9], xg[3];
    grab_point(P, B, xg, R);
    const double dt = c.dt;
    double vn[3], arm[3], tc[3], w[3], F[3] = {W[0], W[1], W[2]};
    for (int a = 0; a < 3; ++a) {
        vn[a] = (double)P.v[a] + (W[a] * (double)B.inv_mass + (double)c.g[a]) * dt;
        arm[a] = xg[a] - (double)P.t[a];
        w[a] = P.w[a];
    }
    cross3d(arm, F, tc);
    for (int a = 0; a < 3; ++a) tc[a] += W[3 + a];
    // I_w = R I_b R^T and I_w^-1 = R I_b^-1 R^T (the body-frame inverse is precomputed),
    // applied as matrix-vector products through the body frame (no 3 x 3 world matrices
    // are formed, which keeps the batched persistent kernel's register budget small)
    double wb[3], Lb[3], L[3], gyro[3], rb[3], ab[3], wn[3];
    for (int k = 0; k < 3; ++k) wb[k] = R[k] * w[0] + R[3 + k] * w[1] + R[6 + k] * w[2];
    for (int k = 0; k < 3; ++k)
        Lb[k] = (double)B.inertia[3 * k] * wb[0] + (double)B.inertia[3 * k + 1] * wb[1] +
                (double)B.inertia[3 * k + 2] * wb[2];
    for (int i = 0; i < 3; ++i) L[i] = R[3 * i] * Lb[0] + R[3 * i + 1] * Lb[1] + R[3 * i + 2] * Lb[2];
    cross3d(w, L, gyro);
    for (int k = 0; k < 3; ++k)
        rb[k] = R[k] * (tc[0] - gyro[0]) + R[3 + k] * (tc[1] - gyro[1]) + R[6 + k] * (tc[2] - gyro[2]);
    for (int k = 0; k < 3; ++k)
        ab[k] = (double)B.inertia_inv[3 * k] * rb[0] + (double)B.inertia_inv[3 * k + 1] * rb[1] +
                (double)B.inertia_inv[3 * k + 2] * rb[2];
    for (int i = 0; i < 3; ++i)
        wn[i] = w[i] + (R[3 * i] * ab[0] + R[3 * i + 1] * ab[1] + R[3 * i + 2] * ab[2]) * dt;
    double qv[3] = {P.q[1], P.q[2], P.q[3]}, wq[3], qn[4], nq = 0.0;
    cross3d(wn, qv, wq);
    double dq0 = -(wn[0] * qv[0] + wn[1] * qv[1] + wn[2] * qv[2]);
    qn[0] = (double)P.q[0] + 0.5 * dt * dq0;
    for (int a = 0; a < 3; ++a) qn[1 + a] = qv[a] + 0.5 * dt * ((double)P.q[0] * wn[a] + wq[a]);
    for (int a = 0; a < 4; ++a) nq += qn[a] * qn[a];
    nq = rsqrt(nq);
    for (int a = 0; a < 3; ++a) {
        B.v[a] = (float)vn[a];
        B.t[a] = (float)((double)P.t[a] + vn[a] * dt);
        B.w[a] = (float)wn[a];
    }
    for (int a = 0; a < 4; ++a) B.q[a] = (float)(qn[a] * nq);
}

constexpr int kWrenchThreads = kTile;

// Grid = max(n_wblocks, kWrenchMinBlocks) blocks: block k reduces body chunk k (if any) in
// FP64 and a slice of the force pass's FP64 diagnostic partials; the last block to finish
// forms the per-body wrenches and diagnostics in a fixed order and updates rigid bodies.
// GB300 runs FP64 at a small fraction of FP32, so this work is spread over many SMs.
// true in the block that took the last ticket (and ran the sums and the rigid update)
__device__ __forceinline__ bool wrench_item(const SimConst &c, int blk)
{
    __shared__ double sw[kWrenchThreads / 32][6];
    __shared__ double sdg[kWrenchThreads / 32][8];
    __shared__ double sxg[3];
    __shared__ bool s_last;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = kWrenchThreads / 32;
    const uint32_t step = c.ctr[0];
    const int G = c.n_wgrid;
    const bool has_body = blk < c.n_wblocks;
    int4 wb = make_int4(0, 0, 0, 0);
    if (has_body) {
        wb = c.wblock[blk];
        if (threadIdx.x == 0) {
            Pose P = body_pose(c, c.body[wb.x], step);
            double R[9], xg[3];
            grab_point(P, c.body[wb.x], xg, R);
            sxg[0] = xg[0]; sxg[1] = xg[1]; sxg[2] = xg[2];
        }
    }
    __syncthreads();
    double acc[6] = {0, 0, 0, 0, 0, 0};
    if (has_body) {
        const int l = wb.y + threadIdx.x;
        if (l < wb.z) {
            int i = in_range(c, c.body[wb.x].first - c.nf + l, c.n_body_particles);
            float4 f = c.fb[i], x = c.xb[i];
            double fd[3] = {f.x, f.y, f.z};
            double r[3] = {(double)x.x - sxg[0], (double)x.y - sxg[1], (double)x.z - sxg[2]}, t[3];
            cross3d(r, fd, t);
            for (int a = 0; a < 3; ++a) { acc[a] = fd[a]; acc[3 + a] = t[a]; }
        }
    }
    // slice of the diagnostic partials: component threadIdx.x & 7, fixed block partition
    double dacc = 0.0;
    {
        const long long F = c.n_force_blocks;
        const int lo = (int)(F * blk / G), hi = (int)(F * (blk + 1) / G);
        const int a = threadIdx.x & 7;
        for (int b = lo + (threadIdx.x >> 3); b < hi; b += kWrenchThreads >> 3)
            dacc += __ldcg(c.diag_part + (size_t)b * 8 + a);
    }
#pragma unroll
    for (int a = 0; a < 6; ++a) {
        double s = warp_sum(acc[a]);
        if (lane == 0) sw[wid][a] = s;
    }
    dacc += __shfl_xor_sync(0xffffffffu, dacc, 8);
    dacc += __shfl_xor_sync(0xffffffffu, dacc, 16);
    if (lane < 8) sdg[wid][lane] = dacc;
    __syncthreads();
    if (threadIdx.x < 6 && has_body) {
        double t = 0.0;
        for (int w = 0; w < nw; ++w) t += sw[w][threadIdx.x];
        c.wrench_part[(size_t)blk * 6 + threadIdx.x] = t;
    }
    if (threadIdx.x >= 32 && threadIdx.x < 40) {
        const int a = threadIdx.x - 32;
        double t = 0.0;
        for (int w = 0; w < nw; ++w) t += sdg[w][a];
        c.diag_part2[(size_t)blk * 8 + a] = t;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(c.ctr + 1, 1u) == (unsigned)G - 1);
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
    // ---- last block: fixed-order sums
    // Every column is summed by 32 threads (rows strided by 32) and a fixed shuffle tree,
    // so the L2 loads overlap instead of forming one dependent chain.
    {
        // diagnostics: 8 columns x G rows -> warps 0..7, column = warp index
        for (int col = wid; col < 8; col += nw) {
            double t = 0.0;
            for (int b = lane; b < G; b += 32) t += __ldcg(c.diag_part2 + (size_t)b * 8 + col);
            t = warp_sum(t);
            if (lane == 0) c.diag[col] = t;
        }
        // wrenches: 6 columns per body x wcount rows
        for (int col = wid; col < 6 * c.nb; col += nw) {
            const int b = col / 6, a = col % 6;
            double t = 0.0;
            for (int k = lane; k < c.wcount[b]; k += 32)
                t += __ldcg(c.wrench_part + (size_t)(c.wfirst[b] + k) * 6 + a);
            t = warp_sum(t);
            if (lane == 0) c.wrench[6 * b + a] = t;
        }
    }
    __syncthreads();
    // ---- rigid bodies (one thread per body): grabbed bodies log, free bodies integrate
    if ((int)threadIdx.x < c.nb) {
        const int b = threadIdx.x;
        DevBody &B = c.body[b];
        if (B.kind == KIND_RIGID) {
            Pose P = body_pose(c, B, step);
            if (B.grabbed) {
                for (int a = 0; a < 3; ++a) { B.t[a] = P.t[a]; B.v[a] = P.v[a]; B.w[a] = P.w[a]; }
                for (int a = 0; a < 4; ++a) B.q[a] = P.q[a];
                if (c.max_path > 0)
                    for (int a = 0; a < 6; ++a)
                        c.wlog[(size_t)(step % (uint32_t)c.max_path) * 6 + a] = c.wrench[6 * b + a];
            } else if (B.mass > 0.0f) {
                rigid_update(c, B, P, c.wrench + 6 * b);
            }
        }
    }
    if (threadIdx.x == 0) {
        c.ctr[1] = 0u;
        c.ctr[0] = step + 1u;
        __threadfence();
    }
    return true;
}

// ---------------------------------------------------------------- per-call kernels

// End of an update cycle: record the grabbed body's wrench for the rolling average.
__device__ __forceinline__ void cycle_end_item(const SimConst &c)
{
    uint32_t cyc = c.ctr[2];
    int g = -1;
    for (int b = 0; b < c.nb; ++b)
        if (c.body[b].grabbed) g = b;
    if (c.smooth_window > 0) {
        double *dst = c.cyc_log + (size_t)(cyc % (uint32_t)c.smooth_window) * 6;
        for (int a = 0; a < 6; ++a) dst[a] = g >= 0 ? c.wrench[6 * g + a] : 0.0;
    }
    c.ctr[2] = cyc + 1u;
}

}  // namespace sphgb

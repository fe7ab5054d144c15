// sph_api.cu -- C ABI of the GB300 SPH coupling substep (declared in include/sph.h).
//
// The handle owns no device memory: every buffer is carved out of the caller's
// workspace.  Setup calls stage particles and bodies on the host; the first call that
// needs the device state ("finalize") uploads them, builds the per-body reduction
// table, and the first sph_step captures the substep's kernel sequence into CUDA
// graphs (1 and 16 substeps) that later calls replay.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "sph.h"
#include "sph_internal.cuh"

using namespace sphgb;

namespace {

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

struct Layout {
    size_t xA, vA, xB, vB, prho, key, rank, perm, cnt, cell_start, tile_sum, tile_state, slot_of_id, locals,
        spring_row, spring_e, fb, xb, acc_dbg, nnbr, body, path, wrench, wrench_part, wblock,
        diag_part, diag_part2, nlist, nlist_n, cut, diag, wlog, cyc_log, status, ctr, total;
    int dims[3], ncell, n_scan_tiles, max_wblocks, max_force_blocks, nl_cap;
};

// Grid of the FP32 cell hash: origin lo - cell, n = floor((hi - o) / cell) + 2 per axis.
// Cells per axis; an axis whose cell count is not finite or exceeds 2^30 gets 0 (the
// callers reject a grid with a zero axis), so the float is range-checked before the cast.
void grid_dims(const sph_params &p, int dims[3], float o[3], float &inv)
{
    inv = 1.0f / p.cell;
    for (int a = 0; a < 3; ++a) {
        o[a] = p.domain_lo[a] - p.cell;
        const float u = (p.domain_hi[a] - o[a]) * inv;
        dims[a] = (u >= 0.0f && u < 1073741824.0f) ? (int)std::floor(u) + 2 : 0;
    }
}

bool valid_params(const sph_params *p, const sph_capacity *cap)
{
    if (!p || !cap) return false;
    if (!(p->h > 0.0f) || !(p->rho0 > 0.0f) || !(p->dt > 0.0f) || !(p->cell >= p->h))
        return false;
    if (!(p->fluid_spacing > 0.0f) || p->k < 0.0f || p->nu < 0.0f) return false;
    for (int a = 0; a < 3; ++a)
        if (!(p->domain_hi[a] > p->domain_lo[a])) return false;
    if (cap->max_particles < 0 || cap->max_bodies < 0 || cap->max_bodies > kMaxBodies ||
        cap->max_springs < 0 || cap->max_path < 0 || cap->max_neighbours < 0)
        return false;
    int dims[3];
    float o[3], inv;
    grid_dims(*p, dims, o, inv);
    double cells = (double)dims[0] * dims[1] * dims[2];
    return cells < 2.0e9 && dims[0] > 0 && dims[1] > 0 && dims[2] > 0;
}

Layout make_layout(const sph_params &p, const sph_capacity &cap)
{
    Layout L;
    float o[3], inv;
    grid_dims(p, L.dims, o, inv);
    L.ncell = L.dims[0] * L.dims[1] * L.dims[2];
    L.n_scan_tiles = (L.ncell + kScanTile - 1) / kScanTile;
    const size_t N = (size_t)std::max(cap.max_particles, 1);
    L.max_wblocks = (int)((N + kReduceChunk - 1) / kReduceChunk) + kMaxBodies;
    L.max_force_blocks = (int)((N + 255) / 256);
    // the low-latency force pass writes a diagnostic row per block of 256 / G particles
    if ((p.flags & SPH_FLAG_LOW_LATENCY) && !(p.flags & SPH_FLAG_VOLUME_BOUNDARY))
        L.max_force_blocks = (int)((N * kLowLatencyForceG + 255) / 256);
    const int W = std::max(p.smooth_window, 1);
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t r = off; off = align256(off + bytes); return r; };
    L.xA = take(16 * N); L.vA = take(16 * N); L.xB = take(16 * N); L.vB = take(16 * N);
    L.prho = take(8 * N);
    L.key = take(4 * N); L.rank = take(4 * N); L.perm = take(4 * N);
    L.cnt = take(4 * ((size_t)L.ncell + 1));
    L.cell_start = take(4 * ((size_t)L.ncell + 1));
    L.tile_sum = take(4 * (size_t)L.n_scan_tiles);
    L.tile_state = take(8 * ((size_t)L.n_scan_tiles + 1));
    L.slot_of_id = take(4 * N);
    L.locals = take(16 * N);
    L.spring_row = take(4 * (N + 1));
    L.spring_e = take(16 * 2 * (size_t)std::max(cap.max_springs, 1));
    L.fb = take(16 * N); L.xb = take(16 * N);
    L.acc_dbg = take(16 * N); L.nnbr = take(4 * N);
    L.body = take(sizeof(DevBody) * kMaxBodies);
    L.path = take(4 * 13 * (size_t)std::max(cap.max_path, 1));
    L.wrench = take(8 * 6 * kMaxBodies);
    L.wrench_part = take(8 * 6 * (size_t)L.max_wblocks);
    L.wblock = take(16 * (size_t)L.max_wblocks);
    L.diag_part = take(8 * 8 * (size_t)L.max_force_blocks);
    L.diag_part2 = take(8 * 8 * (size_t)std::max(L.max_wblocks, kWrenchMinBlocks));
    L.nl_cap = ((cap.max_neighbours > 0 ? cap.max_neighbours : kDefaultNeighbours) + 3) & ~3;
    L.nlist = take(4 * (size_t)L.nl_cap * N);
    L.nlist_n = take(4 * N);
    L.cut = take(16);
    L.diag = take(8 * 8);
    L.wlog = take(8 * 6 * (size_t)std::max(cap.max_path, 1));
    L.cyc_log = take(8 * 6 * (size_t)W);
    L.status = take(16);
    L.ctr = take(16);
    L.total = off;
    return L;
}

}  // namespace

struct sph_handle {
    sph_params p;
    sph_capacity cap;
    Layout L;
    char *ws = nullptr;
    cudaStream_t stream = nullptr;
    SimConst c;
    std::vector<float4> hx, hv, hlocal;     // staged in id order until finalize
    std::vector<DevBody> bodies;
    std::vector<int> spring_row;            // per body particle (id - nf)
    std::vector<float4> spring_e;
    std::vector<float> path;
    int n_springs = 0;
    int grab = -1;
    bool finalized = false;
    // graphs: 1 and 16 substeps, 1 substep followed by the update cycle's end (the last
    // launch of a call), and the profiling substep with event nodes
    cudaGraphExec_t exec1 = nullptr, exec16 = nullptr, exec1c = nullptr, exec_prof = nullptr;
    int profiling = 0;                      // 0 off, 1 every kernel, 2 the density pass only
    int prof_graph = 0;                     // the level exec_prof was captured for
    int prof_last = 0;                      // the level of the last profiled substep
    cudaEvent_t ev[kSubstepKernels + 1] = {};
    int64_t substeps = 0;
    std::string err;
    // pinned host memory for the synchronising reads (status at 0, the read's data from
    // 64 on): the copies are truly asynchronous and one stream synchronisation ends a read
    unsigned char *pin = nullptr;
    size_t pin_bytes = 0;
};

namespace {

sph_status fail(sph_handle *h, sph_status s, const std::string &msg)
{
    if (h) h->err = msg;
    return s;
}

sph_status cuda_fail(sph_handle *h, cudaError_t e, const char *where)
{
    return fail(h, SPH_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define SPH_CUDA(h, call)                                           \
    do {                                                            \
        cudaError_t e_ = (call);                                    \
        if (e_ != cudaSuccess) return cuda_fail((h), e_, #call);    \
    } while (0)

template <typename T>
T *at(sph_handle *h, size_t off) { return reinterpret_cast<T *>(h->ws + off); }

// FP32 world position of a body-frame offset: ((R0 l0 + R1 l1) + R2 l2) + t per row.
void place(const float pose[7], const float l[3], float out[3])
{
    const float w = pose[3], x = pose[4], y = pose[5], z = pose[6];
    volatile float xx = x * x, yy = y * y, zz = z * z, xy = x * y, xz = x * z, yz = y * z;
    volatile float wx = w * x, wy = w * y, wz = w * z;
    float R[9];
    R[0] = 1.0f - 2.0f * (yy + zz); R[1] = 2.0f * (xy - wz);        R[2] = 2.0f * (xz + wy);
    R[3] = 2.0f * (xy + wz);        R[4] = 1.0f - 2.0f * (xx + zz); R[5] = 2.0f * (yz - wx);
    R[6] = 2.0f * (xz - wy);        R[7] = 2.0f * (yz + wx);        R[8] = 1.0f - 2.0f * (xx + yy);
    for (int a = 0; a < 3; ++a) {
        volatile float s = R[3 * a] * l[0];
        volatile float u = R[3 * a + 1] * l[1];
        s = s + u;
        u = R[3 * a + 2] * l[2];
        s = s + u;
        out[a] = s + pose[a];
    }
}

// Turns a fetched status word into the call's result; clears it on the device if set.
sph_status eval_status(sph_handle *h, const uint32_t st[3])
{
    if (st[0] == 0) return SPH_OK;
    SPH_CUDA(h, cudaMemsetAsync(at<uint32_t>(h, h->L.status), 0, 12, h->stream));
    SPH_CUDA(h, cudaStreamSynchronize(h->stream));
    char buf[160];
    if (st[0] & ST_BOUNDS) return fail(h, SPH_ERR_BOUNDS, "an index check failed (bounds-checked build)");
    if (st[0] & ST_NONFINITE) {
        snprintf(buf, sizeof buf, "non-finite particle state (%u reports)", st[1]);
        return fail(h, SPH_ERR_NONFINITE, buf);
    }
    if (st[0] & ST_DOMAIN) {
        snprintf(buf, sizeof buf, "particles outside the grid domain (%u reports)", st[2]);
        return fail(h, SPH_ERR_DOMAIN, buf);
    }
    if (st[0] & ST_CAPACITY) return fail(h, SPH_ERR_CAPACITY, "cell occupancy above the limit");
    if (st[0] & ST_TIMEOUT) return fail(h, SPH_ERR_TIMEOUT, "a bounded device wait gave up");
    return fail(h, SPH_ERR_CUDA, "unknown device status");
}

// Waits for the stream and reports the device status word; `extra`/`bytes` (device, may be
// null) is fetched in the same synchronisation into `dst`.
sph_status read_status_with(sph_handle *h, const void *extra, size_t bytes, void *dst)
{
    uint32_t st[3];
    if (h->pin && 64 + bytes <= h->pin_bytes) {
        if (extra) SPH_CUDA(h, cudaMemcpyAsync(h->pin + 64, extra, bytes, cudaMemcpyDeviceToHost, h->stream));
        SPH_CUDA(h, cudaMemcpyAsync(h->pin, at<uint32_t>(h, h->L.status), 12,
                                    cudaMemcpyDeviceToHost, h->stream));
        SPH_CUDA(h, cudaStreamSynchronize(h->stream));
        if (extra) std::memcpy(dst, h->pin + 64, bytes);
        std::memcpy(st, h->pin, 12);
    } else {
        if (extra) SPH_CUDA(h, cudaMemcpyAsync(dst, extra, bytes, cudaMemcpyDeviceToHost, h->stream));
        SPH_CUDA(h, cudaMemcpyAsync(st, at<uint32_t>(h, h->L.status), 12, cudaMemcpyDeviceToHost,
                                    h->stream));
        SPH_CUDA(h, cudaStreamSynchronize(h->stream));
    }
    return eval_status(h, st);
}

sph_status read_status(sph_handle *h) { return read_status_with(h, nullptr, 0, nullptr); }

sph_status finalize(sph_handle *h)
{
    if (h->finalized) return SPH_OK;
    SimConst &c = h->c;
    const int n = (int)h->hx.size();
    c.n = n;
    c.nb = (int)h->bodies.size();
    c.n_body_particles = n - c.nf;
    c.n_force_blocks = (n + 255) / 256;
    if ((h->p.flags & SPH_FLAG_LOW_LATENCY) && !(h->p.flags & SPH_FLAG_VOLUME_BOUNDARY))
        c.n_force_blocks = (int)(((long long)n * kLowLatencyForceG + 255) / 256);
    for (int b = 0; b < kMaxBodies; ++b) {
        c.body_end[b] = b < c.nb ? h->bodies[b].first + h->bodies[b].n : n;
        c.body_kind[b] = b < c.nb ? h->bodies[b].kind : 0;
    }
    // reduction table: rigid bodies (and static ones when recording)
    std::vector<int4> wb;
    for (int b = 0; b < kMaxBodies; ++b) { c.wfirst[b] = 0; c.wcount[b] = 0; }
    for (int b = 0; b < c.nb; ++b) {
        const DevBody &B = h->bodies[b];
        bool want = B.kind == SPH_BODY_RIGID || (B.kind == SPH_BODY_STATIC && (h->p.flags & SPH_FLAG_RECORD));
        c.wfirst[b] = (int)wb.size();
        if (!want) continue;
        for (int l0 = 0; l0 < B.n; l0 += kReduceChunk)
            wb.push_back(make_int4(b, l0, std::min(B.n, l0 + kReduceChunk), 0));
        c.wcount[b] = (int)wb.size() - c.wfirst[b];
    }
    if ((int)wb.size() > h->L.max_wblocks) return fail(h, SPH_ERR_CAPACITY, "too many reduction blocks");
    c.n_wblocks = (int)wb.size();
    c.n_wgrid = std::max(c.n_wblocks, kWrenchMinBlocks);
    cudaStream_t s = h->stream;
    if (n > 0) {
        SPH_CUDA(h, cudaMemcpyAsync(c.xB, h->hx.data(), 16 * (size_t)n, cudaMemcpyHostToDevice, s));
        SPH_CUDA(h, cudaMemcpyAsync(c.vB, h->hv.data(), 16 * (size_t)n, cudaMemcpyHostToDevice, s));
    }
    if (!h->hlocal.empty())
        SPH_CUDA(h, cudaMemcpyAsync(c.locals, h->hlocal.data(), 16 * h->hlocal.size(),
                                    cudaMemcpyHostToDevice, s));
    std::vector<int> rows(h->spring_row);
    rows.resize((size_t)c.n_body_particles + 1, h->spring_row.empty() ? 0 : h->spring_row.back());
    if (rows.empty()) rows.push_back(0);
    SPH_CUDA(h, cudaMemcpyAsync(c.spring_row, rows.data(), 4 * rows.size(), cudaMemcpyHostToDevice, s));
    if (!h->spring_e.empty())
        SPH_CUDA(h, cudaMemcpyAsync(c.spring_e, h->spring_e.data(), 16 * h->spring_e.size(),
                                    cudaMemcpyHostToDevice, s));
    if (c.nb > 0)
        SPH_CUDA(h, cudaMemcpyAsync(c.body, h->bodies.data(), sizeof(DevBody) * c.nb,
                                    cudaMemcpyHostToDevice, s));
    if (!wb.empty())
        SPH_CUDA(h, cudaMemcpyAsync(c.wblock, wb.data(), 16 * wb.size(), cudaMemcpyHostToDevice, s));
    SPH_CUDA(h, cudaStreamSynchronize(s));
    h->finalized = true;
    return SPH_OK;
}

sph_status capture(sph_handle *h, int count, cudaGraphExec_t *out, bool prof = false,
                   bool cycle_end = false, unsigned ev_mask = ~0u)
{
    cudaGraph_t g = nullptr;
    SPH_CUDA(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t le = cudaSuccess;
    for (int i = 0; i < count && le == cudaSuccess; ++i)
        le = launch_substep(h->c, h->stream, prof ? h->ev : nullptr, prof, cycle_end && i == count - 1,
                            ev_mask);
    cudaError_t ce = cudaStreamEndCapture(h->stream, &g);
    if (le != cudaSuccess) { if (g) cudaGraphDestroy(g); return cuda_fail(h, le, "capture launch"); }
    if (ce != cudaSuccess) return cuda_fail(h, ce, "cudaStreamEndCapture");
    cudaError_t ie = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) return cuda_fail(h, ie, "cudaGraphInstantiate");
    return SPH_OK;
}

}  // namespace

namespace sphgb {

// Batch support: finalize a scene, wait for its stream, and hand out its SimConst.
sph_status scene_for_batch(sph_handle *h, SimConst *out)
{
    sph_status st = finalize(h);
    if (st != SPH_OK) return st;
    SPH_CUDA(h, cudaStreamSynchronize(h->stream));
    *out = h->c;
    return SPH_OK;
}

// Batch support: the batch advanced this scene by n substeps (one update cycle).
void scene_advanced(sph_handle *h, int n) { h->substeps += n; }

// Isosurface support: the handle's stream and parameters.
cudaStream_t scene_stream(sph_handle *h) { return h->stream; }
const sph_params *scene_params(sph_handle *h) { return &h->p; }

}  // namespace sphgb

namespace sphgb {
void handle_surrogate_view(const sph_handle *h, cudaStream_t *stream, const SimConst **c, int *grab,
                           long long *substeps)
{
    *stream = h->stream;
    *c = &h->c;
    *grab = h->grab;
    *substeps = (long long)h->substeps;
}
}  // namespace sphgb

extern "C" {

size_t sph_workspace_bytes(const sph_params *p, const sph_capacity *cap)
{
    if (!valid_params(p, cap)) return 0;
    return make_layout(*p, *cap).total;
}

sph_status sph_create(const sph_params *p, const sph_capacity *cap, void *d_workspace,
                      size_t bytes, void *cuda_stream, int32_t n_fluid, const float *h_xyz,
                      const float *h_vel, sph_handle **out)
{
    if (!out) return SPH_ERR_ARG;
    *out = nullptr;
    if (!valid_params(p, cap) || n_fluid < 0 || (n_fluid > 0 && !h_xyz)) return SPH_ERR_ARG;
    if (n_fluid > cap->max_particles) return SPH_ERR_CAPACITY;
    Layout L = make_layout(*p, *cap);
    if (!d_workspace || bytes < L.total || ((uintptr_t)d_workspace & 255u)) return SPH_ERR_WORKSPACE;
    sph_handle *h = new sph_handle();
    h->p = *p;
    h->cap = *cap;
    h->L = L;
    h->ws = (char *)d_workspace;
    h->stream = (cudaStream_t)cuda_stream;
    SimConst &c = h->c;
    std::memset(&c, 0, sizeof c);
    c.nf = n_fluid;
    c.nx = L.dims[0]; c.ny = L.dims[1]; c.nz = L.dims[2]; c.ncell = L.ncell;
    grid_dims(*p, L.dims, c.o, c.inv_cell);
    float R = 2.0f * p->h;
    c.R2 = R * R;
    {
        // The search radius exceeds R by a margin far above the FP32 rounding of the
        // predicate (relative ~1e-6) and of cell coordinates (a few ulp of the coordinates).
        float M = 0.0f;
        for (int a = 0; a < 3; ++a)
            M = std::max(M, std::max(std::fabs(c.o[a]), std::fabs(c.o[a] + (float)L.dims[a] * p->cell)));
        const float margin = std::max(1e-3f * R, 64.0f * M * 1.1920929e-7f);
        c.Rc = (R + margin) / p->cell;
        c.mc = margin / p->cell;
    }
    c.h = p->h;
    c.inv_h = 1.0f / p->h;
    c.rho0 = p->rho0;
    c.k = p->k;
    c.tait_B = (float)((double)p->k * (double)p->rho0 / 7.0);
    c.nu20 = 20.0f * p->nu;
    c.eps_h2 = p->visc_eps * p->h * p->h;
    {
        const double hd = (double)p->h;
        const double a6 = 1.0 / (4.0 * M_PI * hd * hd * hd), ih = 1.0 / hd;
        c.alpha6_hi = (float)a6;
        c.alpha6_lo = (float)(a6 - (double)c.alpha6_hi);
        c.invh_hi = (float)ih;
        c.invh_lo = (float)(ih - (double)c.invh_hi);
    }
    c.alpha_g = (float)(3.0 / (2.0 * M_PI * (double)p->h * p->h * p->h) / ((double)p->h * p->h));
    for (int a = 0; a < 3; ++a) c.g[a] = p->g[a];
    c.dt = p->dt;
    c.flags = p->flags;
    c.max_path = cap->max_path;
    c.n_scan_tiles = L.n_scan_tiles;
    c.smooth_window = std::max(p->smooth_window, 1);
    c.xA = at<float4>(h, L.xA); c.vA = at<float4>(h, L.vA);
    c.xB = at<float4>(h, L.xB); c.vB = at<float4>(h, L.vB);
    c.prho = at<float2>(h, L.prho);
    c.key = at<uint32_t>(h, L.key); c.rank = at<uint32_t>(h, L.rank); c.perm = at<uint32_t>(h, L.perm);
    c.cnt = at<uint32_t>(h, L.cnt); c.cell_start = at<uint32_t>(h, L.cell_start);
    c.tile_sum = at<uint32_t>(h, L.tile_sum);
    c.tile_state = at<unsigned long long>(h, L.tile_state);
    c.slot_of_id = at<int>(h, L.slot_of_id);
    c.locals = at<float4>(h, L.locals);
    c.spring_row = at<int>(h, L.spring_row);
    c.spring_e = at<float4>(h, L.spring_e);
    c.fb = at<float4>(h, L.fb); c.xb = at<float4>(h, L.xb);
    c.acc_dbg = at<float4>(h, L.acc_dbg); c.nnbr = at<int>(h, L.nnbr);
    c.body = at<DevBody>(h, L.body);
    c.path = at<float>(h, L.path);
    c.wrench = at<double>(h, L.wrench);
    c.wrench_part = at<double>(h, L.wrench_part);
    c.wblock = at<int4>(h, L.wblock);
    c.diag_part = at<double>(h, L.diag_part);
    c.diag_part2 = at<double>(h, L.diag_part2);
    c.nlist4 = at<uint4>(h, L.nlist);
    c.nlist_n = at<int>(h, L.nlist_n);
    c.nl_cap = L.nl_cap;
    c.diag = at<double>(h, L.diag);
    c.wlog = at<double>(h, L.wlog);
    c.cyc_log = at<double>(h, L.cyc_log);
    c.status = at<uint32_t>(h, L.status);
    c.ctr = at<uint32_t>(h, L.ctr);
    const float m = p->rho0 * (p->fluid_spacing * p->fluid_spacing * p->fluid_spacing);
    h->hx.resize(n_fluid);
    h->hv.resize(n_fluid);
    for (int i = 0; i < n_fluid; ++i) {
        h->hx[i] = make_float4(h_xyz[3 * i], h_xyz[3 * i + 1], h_xyz[3 * i + 2], m);
        float vx = h_vel ? h_vel[3 * i] : 0.0f, vy = h_vel ? h_vel[3 * i + 1] : 0.0f;
        float vz = h_vel ? h_vel[3 * i + 2] : 0.0f;
        int id = i;
        float idf;
        std::memcpy(&idf, &id, 4);
        h->hv[i] = make_float4(vx, vy, vz, idf);
    }
    cudaError_t e = cudaMemsetAsync(h->ws, 0, L.total, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
        delete h;
        return SPH_ERR_CUDA;
    }
    // pinned staging for the synchronising reads: status, then the counters and the
    // smoothing window's cycle log (host memory; unpinned copies if refused)
    h->pin_bytes = 64 + 16 + 48 * (size_t)c.smooth_window;
    if (cudaHostAlloc((void **)&h->pin, h->pin_bytes, cudaHostAllocDefault) != cudaSuccess) {
        h->pin = nullptr;
        h->pin_bytes = 0;
        cudaGetLastError();
    }
    *out = h;
    return SPH_OK;
}

static sph_status add_particles(sph_handle *h, int kind, int32_t n, const float *xyz, float spacing,
                                float mass, const float inertia[9], const float pose[7],
                                const float vel[6], int32_t *out_id, DevBody **made)
{
    if (!h) return SPH_ERR_ARG;
    if (h->finalized) return fail(h, SPH_ERR_STATE, "bodies can only be added before the first step");
    if (n <= 0 || !xyz || !(spacing > 0.0f)) return fail(h, SPH_ERR_ARG, "bad body arguments");
    if ((int)h->bodies.size() >= h->cap.max_bodies || (int)h->bodies.size() >= kMaxBodies)
        return fail(h, SPH_ERR_CAPACITY, "too many bodies");
    if ((int64_t)h->hx.size() + n > h->cap.max_particles)
        return fail(h, SPH_ERR_CAPACITY, "too many particles");
    DevBody B;
    std::memset(&B, 0, sizeof B);
    B.kind = kind;
    B.first = (int)h->hx.size();
    B.n = n;
    B.mass = mass;
    float q0[7] = {0, 0, 0, 1, 0, 0, 0};
    const float *ps = pose ? pose : q0;
    for (int a = 0; a < 3; ++a) {
        B.t[a] = ps[a];
        B.v[a] = vel ? vel[a] : 0.0f;
        B.w[a] = vel ? vel[3 + a] : 0.0f;
    }
    for (int a = 0; a < 4; ++a) B.q[a] = ps[3 + a];
    if (inertia) {
        double I[9], det;
        for (int a = 0; a < 9; ++a) { B.inertia[a] = inertia[a]; I[a] = inertia[a]; }
        det = I[0] * (I[4] * I[8] - I[5] * I[7]) - I[1] * (I[3] * I[8] - I[5] * I[6]) +
              I[2] * (I[3] * I[7] - I[4] * I[6]);
        if (kind == SPH_BODY_RIGID && !(std::fabs(det) > 0.0))
            return fail(h, SPH_ERR_ARG, "singular inertia tensor");
        if (kind == SPH_BODY_RIGID) {
            const double inv[9] = {I[4] * I[8] - I[5] * I[7], I[2] * I[7] - I[1] * I[8],
                                   I[1] * I[5] - I[2] * I[4], I[5] * I[6] - I[3] * I[8],
                                   I[0] * I[8] - I[2] * I[6], I[2] * I[3] - I[0] * I[5],
                                   I[3] * I[7] - I[4] * I[6], I[1] * I[6] - I[0] * I[7],
                                   I[0] * I[4] - I[1] * I[3]};
            for (int a = 0; a < 9; ++a) B.inertia_inv[a] = (float)(inv[a] / det);
        }
    }
    B.inv_mass = mass > 0.0f ? 1.0f / mass : 0.0f;
    const float pm = h->p.rho0 * (spacing * spacing * spacing);
    const float tagged = (kind == SPH_BODY_SOFT) ? pm : -pm;   // negative mass tags boundary
    for (int i = 0; i < n; ++i) {
        int id = B.first + i;
        float idf;
        std::memcpy(&idf, &id, 4);
        float w[3] = {xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2]};
        if (kind == SPH_BODY_STATIC || kind == SPH_BODY_RIGID) place(ps, xyz + 3 * i, w);
        h->hx.push_back(make_float4(w[0], w[1], w[2], tagged));
        h->hv.push_back(make_float4(0.0f, 0.0f, 0.0f, idf));
        h->hlocal.push_back(make_float4(xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], 0.0f));
        if (h->spring_row.empty()) h->spring_row.push_back(0);
        h->spring_row.push_back(h->spring_row.back());
    }
    h->bodies.push_back(B);
    if (out_id) *out_id = (int)h->bodies.size() - 1;
    if (made) *made = &h->bodies.back();
    return SPH_OK;
}

sph_status sph_add_rigid(sph_handle *h, int32_t n, const float *h_local, float spacing,
                         float body_mass, const float inertia[9], const float pose[7],
                         const float vel[6], int32_t *out_body_id)
{
    if (!h) return SPH_ERR_ARG;
    if (body_mass < 0.0f || (body_mass > 0.0f && !inertia))
        return fail(h, SPH_ERR_ARG, "rigid body needs mass >= 0 and an inertia tensor");
    int kind = body_mass > 0.0f ? SPH_BODY_RIGID : SPH_BODY_STATIC;
    return add_particles(h, kind, n, h_local, spacing, body_mass, inertia, pose,
                         kind == SPH_BODY_RIGID ? vel : nullptr, out_body_id, nullptr);
}

sph_status sph_add_soft(sph_handle *h, int32_t n, const float *h_xyz, float spacing,
                        int32_t n_springs, const int32_t *h_pairs, float young_E,
                        float poisson_nu, int32_t *out_body_id)
{
    (void)poisson_nu;   // a spring lattice cannot represent a Poisson ratio
    if (!h) return SPH_ERR_ARG;
    if (n_springs < 0 || (n_springs > 0 && !h_pairs) || !(young_E >= 0.0f))
        return fail(h, SPH_ERR_ARG, "bad spring arguments");
    if (h->n_springs + n_springs > h->cap.max_springs)
        return fail(h, SPH_ERR_CAPACITY, "too many springs");
    for (int s = 0; s < n_springs; ++s) {
        int a = h_pairs[2 * s], b = h_pairs[2 * s + 1];
        if (a < 0 || b < 0 || a >= n || b >= n || a == b) return fail(h, SPH_ERR_ARG, "bad spring pair");
    }
    DevBody *B = nullptr;
    sph_status st = add_particles(h, SPH_BODY_SOFT, n, h_xyz, spacing, 0.0f, nullptr, nullptr,
                                  nullptr, out_body_id, &B);
    if (st != SPH_OK) return st;
    // lookup table of Alg. 2's spring pass: CSR per particle, both directions
    const int first = B->first, nf = h->c.nf;
    const float m = h->p.rho0 * (spacing * spacing * spacing);
    std::vector<std::vector<float4>> rows(n);
    for (int s = 0; s < n_springs; ++s) {
        int a = h_pairs[2 * s], b = h_pairs[2 * s + 1];
        float d0 = h_xyz[3 * a] - h_xyz[3 * b], d1 = h_xyz[3 * a + 1] - h_xyz[3 * b + 1];
        float d2 = h_xyz[3 * a + 2] - h_xyz[3 * b + 2];
        float L0 = std::sqrt(d0 * d0 + d1 * d1 + d2 * d2);
        float ks = young_E * spacing * spacing / L0;
        float cd = 2.0f * h->p.spring_zeta * std::sqrt(ks * m / 2.0f);
        int ia = first + a, ib = first + b;
        float fa, fb;
        std::memcpy(&fa, &ia, 4);
        std::memcpy(&fb, &ib, 4);
        rows[a].push_back(make_float4(fb, L0, ks, cd));
        rows[b].push_back(make_float4(fa, L0, ks, cd));
    }
    // rewrite this body's CSR rows (they were appended empty)
    const int l0 = first - nf;
    int run = h->spring_row[l0];
    for (int i = 0; i < n; ++i) {
        for (const float4 &e : rows[i]) h->spring_e.push_back(e);
        run += (int)rows[i].size();
        h->spring_row[l0 + i + 1] = run;
    }
    h->n_springs += n_springs;
    return SPH_OK;
}

sph_status sph_set_grab_pose(sph_handle *h, int32_t body_id, const float pose[7],
                             const float vel[6], const float grab_point_local[3])
{
    if (!h) return SPH_ERR_ARG;
    if (body_id >= (int)h->bodies.size() || body_id < -1) return fail(h, SPH_ERR_ARG, "bad body id");
    if (body_id >= 0 && h->bodies[body_id].kind != SPH_BODY_RIGID)
        return fail(h, SPH_ERR_ARG, "only rigid bodies can be grabbed");
    sph_status st = finalize(h);
    if (st != SPH_OK) return st;
    float pv[13] = {0, 0, 0, 1, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    float gl[3] = {0, 0, 0};
    if (pose)
        for (int a = 0; a < 7; ++a) pv[a] = pose[a];
    if (vel)
        for (int a = 0; a < 6; ++a) pv[7 + a] = vel[a];
    if (grab_point_local)
        for (int a = 0; a < 3; ++a) gl[a] = grab_point_local[a];
    int b = body_id >= 0 ? body_id : h->grab;
    if (b < 0) return SPH_OK;
    SPH_CUDA(h, launch_set_grab(h->c, h->stream, b, body_id >= 0 ? 1 : 0, pv, gl, pose ? 1 : 0, 0));
    h->grab = body_id;
    return SPH_OK;
}

sph_status sph_set_grab_path(sph_handle *h, int32_t n, const float *h_path)
{
    if (!h) return SPH_ERR_ARG;
    if (h->grab < 0) return fail(h, SPH_ERR_STATE, "no grabbed body");
    if (n < 0 || n > h->cap.max_path || (n > 0 && !h_path)) return fail(h, SPH_ERR_ARG, "bad path");
    sph_status st = finalize(h);
    if (st != SPH_OK) return st;
    if (n > 0)
        SPH_CUDA(h, cudaMemcpyAsync(h->c.path, h_path, 4 * 13 * (size_t)n, cudaMemcpyHostToDevice,
                                    h->stream));
    // keep the grab point; pose comes from the path
    DevBody B;
    SPH_CUDA(h, cudaMemcpyAsync(&B, h->c.body + h->grab, sizeof B, cudaMemcpyDeviceToHost, h->stream));
    SPH_CUDA(h, cudaStreamSynchronize(h->stream));
    float pv[13] = {0};
    SPH_CUDA(h, launch_set_grab(h->c, h->stream, h->grab, 1, pv, B.grab_local, 0, n));
    SPH_CUDA(h, cudaStreamSynchronize(h->stream));
    return SPH_OK;
}

sph_status sph_step(sph_handle *h, int32_t n_substeps)
{
    if (!h || n_substeps < 0) return SPH_ERR_ARG;
    sph_status st = finalize(h);
    if (st != SPH_OK) return st;
    if (h->c.n == 0 || n_substeps == 0) return SPH_OK;
    const bool graphs = !(h->p.flags & SPH_FLAG_NO_GRAPH) && h->stream != nullptr;
    int left = n_substeps;
    bool cycle_done = false;
    if (h->profiling) {
        const unsigned mask = h->profiling == 2 ? kDensityEvents : ~0u;
        if (graphs && h->exec_prof && h->prof_graph != h->profiling) {
            cudaGraphExecDestroy(h->exec_prof);
            h->exec_prof = nullptr;
        }
        if (graphs && !h->exec_prof) {
            st = capture(h, 1, &h->exec_prof, true, false, mask);
            if (st != SPH_OK) return st;
            h->prof_graph = h->profiling;
        }
        for (; left > 0; --left) {
            if (graphs) SPH_CUDA(h, cudaGraphLaunch(h->exec_prof, h->stream));
            else SPH_CUDA(h, launch_substep(h->c, h->stream, h->ev, false, false, mask));
        }
        h->prof_last = h->profiling;
    } else if (graphs) {
        if (!h->exec1) {
            st = capture(h, 1, &h->exec1);
            if (st != SPH_OK) return st;
        }
        if (left >= 16 && !h->exec16) {
            st = capture(h, 16, &h->exec16);
            if (st != SPH_OK) return st;
        }
        if (left % 16 && !h->exec1c) {
            st = capture(h, 1, &h->exec1c, false, true);
            if (st != SPH_OK) return st;
        }
        for (; left >= 16; left -= 16) SPH_CUDA(h, cudaGraphLaunch(h->exec16, h->stream));
        for (; left > 1; --left) SPH_CUDA(h, cudaGraphLaunch(h->exec1, h->stream));
        if (left == 1) {
            // the last substep and the cycle's end in one launch (a haptic tick's step)
            SPH_CUDA(h, cudaGraphLaunch(h->exec1c, h->stream));
            cycle_done = true;
        }
    } else {
        for (; left > 0; --left) SPH_CUDA(h, launch_substep(h->c, h->stream));
    }
    if (!cycle_done) SPH_CUDA(h, launch_cycle_end(h->c, h->stream));
    h->substeps += n_substeps;
    return SPH_OK;
}

sph_status sph_get_body_wrench(sph_handle *h, int32_t body_id, double out[6])
{
    if (!h || !out || body_id < 0 || body_id >= (int)h->bodies.size()) return SPH_ERR_ARG;
    sph_status st = finalize(h);
    if (st != SPH_OK) return st;
    return read_status_with(h, h->c.wrench + 6 * body_id, 48, out);
}

sph_status sph_get_grab_wrench(sph_handle *h, double out[6], int32_t smoothed)
{
    if (!h || !out) return SPH_ERR_ARG;
    if (h->grab < 0) return fail(h, SPH_ERR_STATE, "no grabbed body");
    if (!smoothed) return sph_get_body_wrench(h, h->grab, out);
    const int W = h->c.smooth_window;
    std::vector<double> log(6 * (size_t)W);
    uint32_t ctr[3];
    sph_status st;
    if (h->pin) {
        // counters at 64, the log at 80, the status at 0: one synchronisation
        SPH_CUDA(h, cudaMemcpyAsync(h->pin + 64, h->c.ctr, 12, cudaMemcpyDeviceToHost, h->stream));
        SPH_CUDA(h, cudaMemcpyAsync(h->pin + 80, h->c.cyc_log, 48 * (size_t)W, cudaMemcpyDeviceToHost,
                                    h->stream));
        st = read_status_with(h, nullptr, 0, nullptr);
        std::memcpy(ctr, h->pin + 64, 12);
        std::memcpy(log.data(), h->pin + 80, 48 * (size_t)W);
    } else {
        SPH_CUDA(h, cudaMemcpyAsync(log.data(), h->c.cyc_log, 48 * (size_t)W, cudaMemcpyDeviceToHost,
                                    h->stream));
        SPH_CUDA(h, cudaMemcpyAsync(ctr, h->c.ctr, 12, cudaMemcpyDeviceToHost, h->stream));
        st = read_status(h);
    }
    uint32_t cycles = ctr[2];
    int m = (int)std::min<uint32_t>(cycles, (uint32_t)W);
    for (int a = 0; a < 6; ++a) out[a] = 0.0;
    if (m == 0) return st;
    // mean of the last m cycle-end wrenches, oldest first
    for (int k = 0; k < m; ++k) {
        uint32_t cyc = cycles - (uint32_t)m + (uint32_t)k;
        const double *e = log.data() + 6 * (cyc % (uint32_t)W);
        for (int a = 0; a < 6; ++a) out[a] += e[a];
    }
    for (int a = 0; a < 6; ++a) out[a] /= (double)m;
    return st;
}

sph_status sph_get_wrench_log(sph_handle *h, int32_t n, double *out)
{
    if (!h || (n > 0 && !out) || n < 0) return SPH_ERR_ARG;
    if (n > h->substeps || n > h->cap.max_path) return fail(h, SPH_ERR_ARG, "log shorter than n");
    const int P = h->cap.max_path;
    std::vector<double> log(6 * (size_t)std::max(P, 1));
    if (P > 0)
        SPH_CUDA(h, cudaMemcpyAsync(log.data(), h->c.wlog, 48 * (size_t)P, cudaMemcpyDeviceToHost,
                                    h->stream));
    sph_status st = read_status(h);
    for (int k = 0; k < n; ++k) {
        int64_t s = h->substeps - n + k;
        std::memcpy(out + 6 * k, log.data() + 6 * (s % P), 48);
    }
    return st;
}

sph_status sph_get_body(sph_handle *h, int32_t body_id, float out[13])
{
    if (!h || !out || body_id < 0 || body_id >= (int)h->bodies.size()) return SPH_ERR_ARG;
    sph_status st = finalize(h);
    if (st != SPH_OK) return st;
    DevBody B;
    SPH_CUDA(h, cudaMemcpyAsync(&B, h->c.body + body_id, sizeof B, cudaMemcpyDeviceToHost, h->stream));
    st = read_status(h);
    for (int a = 0; a < 3; ++a) { out[a] = B.t[a]; out[7 + a] = B.v[a]; out[10 + a] = B.w[a]; }
    for (int a = 0; a < 4; ++a) out[3 + a] = B.q[a];
    return st;
}

sph_status sph_get_state(sph_handle *h, float *h_x, float *h_v, float *h_rho, int32_t *h_nnbr,
                         float *h_acc)
{
    if (!h) return SPH_ERR_ARG;
    sph_status st = finalize(h);
    if (st != SPH_OK) return st;
    const int n = h->c.n;
    std::vector<float4> x(n), v(n), acc(h_acc ? n : 0);
    std::vector<float2> pr(h_rho ? n : 0);
    std::vector<int> nn(h_nnbr ? n : 0);
    cudaStream_t s = h->stream;
    SPH_CUDA(h, cudaMemcpyAsync(x.data(), h->c.xB, 16 * (size_t)n, cudaMemcpyDeviceToHost, s));
    SPH_CUDA(h, cudaMemcpyAsync(v.data(), h->c.vB, 16 * (size_t)n, cudaMemcpyDeviceToHost, s));
    if (h_rho) SPH_CUDA(h, cudaMemcpyAsync(pr.data(), h->c.prho, 8 * (size_t)n, cudaMemcpyDeviceToHost, s));
    if (h_nnbr) SPH_CUDA(h, cudaMemcpyAsync(nn.data(), h->c.nnbr, 4 * (size_t)n, cudaMemcpyDeviceToHost, s));
    if (h_acc) SPH_CUDA(h, cudaMemcpyAsync(acc.data(), h->c.acc_dbg, 16 * (size_t)n, cudaMemcpyDeviceToHost, s));
    st = read_status(h);
    for (int p = 0; p < n; ++p) {
        int id;
        std::memcpy(&id, &v[p].w, 4);
        if (id < 0 || id >= n) return fail(h, SPH_ERR_STATE, "corrupt particle id");
        if (h_x) { h_x[3 * id] = x[p].x; h_x[3 * id + 1] = x[p].y; h_x[3 * id + 2] = x[p].z; }
        if (h_v) { h_v[3 * id] = v[p].x; h_v[3 * id + 1] = v[p].y; h_v[3 * id + 2] = v[p].z; }
        if (h_rho) h_rho[id] = pr[p].x;
        if (h_nnbr) h_nnbr[id] = nn[p];
        if (h_acc) { h_acc[3 * id] = acc[p].x; h_acc[3 * id + 1] = acc[p].y; h_acc[3 * id + 2] = acc[p].z; }
    }
    return st;
}

sph_status sph_set_state(sph_handle *h, const float *h_x, const float *h_v)
{
    if (!h) return SPH_ERR_ARG;
    sph_status st = finalize(h);
    if (st != SPH_OK) return st;
    const int n = h->c.n;
    std::vector<float4> x(n), v(n);
    cudaStream_t s = h->stream;
    SPH_CUDA(h, cudaMemcpyAsync(x.data(), h->c.xB, 16 * (size_t)n, cudaMemcpyDeviceToHost, s));
    SPH_CUDA(h, cudaMemcpyAsync(v.data(), h->c.vB, 16 * (size_t)n, cudaMemcpyDeviceToHost, s));
    SPH_CUDA(h, cudaStreamSynchronize(s));
    for (int p = 0; p < n; ++p) {
        int id;
        std::memcpy(&id, &v[p].w, 4);
        if (id < 0 || id >= n) return fail(h, SPH_ERR_STATE, "corrupt particle id");
        if (x[p].w < 0.0f) continue;          // boundary particles follow their bodies
        if (h_x) { x[p].x = h_x[3 * id]; x[p].y = h_x[3 * id + 1]; x[p].z = h_x[3 * id + 2]; }
        if (h_v) { v[p].x = h_v[3 * id]; v[p].y = h_v[3 * id + 1]; v[p].z = h_v[3 * id + 2]; }
    }
    SPH_CUDA(h, cudaMemcpyAsync(h->c.xB, x.data(), 16 * (size_t)n, cudaMemcpyHostToDevice, s));
    SPH_CUDA(h, cudaMemcpyAsync(h->c.vB, v.data(), 16 * (size_t)n, cudaMemcpyHostToDevice, s));
    SPH_CUDA(h, cudaStreamSynchronize(s));
    return SPH_OK;
}

// ---------------------------------------------------------------- checkpoint / resume

namespace {

struct CkptHeader {
    char magic[8];
    int64_t substeps;
    int32_t n, nf, n_bodies, grab;
    uint64_t payload;
};

// Workspace regions that carry over from one substep to the next (everything else is
// recomputed by every substep): the state in its current slot order (the stable sort ties
// on it), body-frame offsets and anchor flags, the spring table (with its cuts), the body
// table, the grab path, the last wrenches, both wrench logs, status word and counters.
std::vector<std::pair<size_t, size_t>> ckpt_regions(const sph_handle *h)
{
    const size_t N = (size_t)std::max(h->cap.max_particles, 1);
    const size_t n = (size_t)h->c.n;
    const size_t P = (size_t)std::max(h->cap.max_path, 1);
    return {{h->L.xB, 16 * n}, {h->L.vB, 16 * n}, {h->L.locals, 16 * N},
            {h->L.spring_e, 16 * 2 * (size_t)std::max(h->cap.max_springs, 1)},
            {h->L.body, sizeof(DevBody) * kMaxBodies}, {h->L.path, 4 * 13 * P},
            {h->L.wrench, 8 * 6 * kMaxBodies}, {h->L.wlog, 8 * 6 * P},
            {h->L.cyc_log, 8 * 6 * (size_t)std::max(h->p.smooth_window, 1)},
            {h->L.status, 16}, {h->L.ctr, 16}};
}

size_t ckpt_total(const sph_handle *h)
{
    size_t t = sizeof(CkptHeader);
    for (const auto &r : ckpt_regions(h)) t += r.second;
    return t;
}

const char kCkptMagic[8] = {'S', 'P', 'H', 'C', 'K', 'P', 'T', '1'};

}  // namespace

size_t sph_checkpoint_bytes(sph_handle *h)
{
    if (!h || finalize(h) != SPH_OK) return 0;
    return ckpt_total(h);
}

sph_status sph_checkpoint_save(sph_handle *h, void *h_buf, size_t bytes)
{
    if (!h || !h_buf) return SPH_ERR_ARG;
    sph_status st = finalize(h);
    if (st != SPH_OK) return st;
    if (bytes < ckpt_total(h)) return fail(h, SPH_ERR_ARG, "checkpoint buffer too small");
    CkptHeader hd;
    std::memset(&hd, 0, sizeof hd);
    std::memcpy(hd.magic, kCkptMagic, 8);
    hd.substeps = h->substeps;
    hd.n = h->c.n;
    hd.nf = h->c.nf;
    hd.n_bodies = (int32_t)h->bodies.size();
    hd.grab = h->grab;
    hd.payload = ckpt_total(h) - sizeof hd;
    char *out = (char *)h_buf;
    std::memcpy(out, &hd, sizeof hd);
    size_t off = sizeof hd;
    for (const auto &r : ckpt_regions(h)) {
        SPH_CUDA(h, cudaMemcpyAsync(out + off, h->ws + r.first, r.second, cudaMemcpyDeviceToHost, h->stream));
        off += r.second;
    }
    SPH_CUDA(h, cudaStreamSynchronize(h->stream));
    return SPH_OK;
}

sph_status sph_checkpoint_load(sph_handle *h, const void *h_buf, size_t bytes)
{
    if (!h || !h_buf) return SPH_ERR_ARG;
    sph_status st = finalize(h);
    if (st != SPH_OK) return st;
    CkptHeader hd;
    if (bytes < sizeof hd) return fail(h, SPH_ERR_ARG, "not a checkpoint");
    std::memcpy(&hd, h_buf, sizeof hd);
    if (std::memcmp(hd.magic, kCkptMagic, 8) != 0) return fail(h, SPH_ERR_ARG, "not a checkpoint");
    if (hd.n != h->c.n || hd.nf != h->c.nf || hd.n_bodies != (int32_t)h->bodies.size() ||
        hd.payload != ckpt_total(h) - sizeof hd || bytes < ckpt_total(h))
        return fail(h, SPH_ERR_ARG, "checkpoint of a different scene or capacity");
    if (hd.grab >= hd.n_bodies || hd.grab < -1) return fail(h, SPH_ERR_ARG, "corrupt checkpoint");
    const char *in = (const char *)h_buf;
    size_t off = sizeof hd;
    for (const auto &r : ckpt_regions(h)) {
        SPH_CUDA(h, cudaMemcpyAsync(h->ws + r.first, in + off, r.second, cudaMemcpyHostToDevice, h->stream));
        off += r.second;
    }
    SPH_CUDA(h, cudaStreamSynchronize(h->stream));
    h->substeps = hd.substeps;
    h->grab = hd.grab;
    return SPH_OK;
}

sph_status sph_haptic_cycle(sph_handle *h, int32_t body_id, const float pose[7], const float vel[6],
                            int32_t n_substeps, int32_t smoothed, double out[6])
{
    if (!h || !out) return SPH_ERR_ARG;
    sph_status st = sph_set_grab_pose(h, body_id, pose, vel, nullptr);
    if (st != SPH_OK) return st;
    st = sph_step(h, n_substeps);
    if (st != SPH_OK) return st;
    return sph_get_grab_wrench(h, out, smoothed);
}

sph_status sph_get_sort(sph_handle *h, uint32_t *h_keys, int32_t *h_ids, uint32_t *h_cell_start)
{
    if (!h) return SPH_ERR_ARG;
    sph_status st = finalize(h);
    if (st != SPH_OK) return st;
    if (h->substeps == 0) return fail(h, SPH_ERR_STATE, "no substep has run");
    const int n = h->c.n;
    cudaStream_t s = h->stream;
    // the rank/perm arrays are free between substeps: use them as output staging
    SPH_CUDA(h, launch_sorted_keys(h->c, s, h->c.rank, (int *)h->c.perm));
    if (h_keys) SPH_CUDA(h, cudaMemcpyAsync(h_keys, h->c.rank, 4 * (size_t)n, cudaMemcpyDeviceToHost, s));
    if (h_ids) SPH_CUDA(h, cudaMemcpyAsync(h_ids, h->c.perm, 4 * (size_t)n, cudaMemcpyDeviceToHost, s));
    if (h_cell_start)
        SPH_CUDA(h, cudaMemcpyAsync(h_cell_start, h->c.cell_start, 4 * ((size_t)h->c.ncell + 1),
                                    cudaMemcpyDeviceToHost, s));
    return read_status(h);
}

sph_status sph_set_anchors(sph_handle *h, int32_t body, int32_t n, const int32_t *h_local)
{
    if (!h || n < 0 || (n > 0 && !h_local)) return SPH_ERR_ARG;
    if (h->finalized) return fail(h, SPH_ERR_STATE, "anchors can only be set before the first step");
    if (body < 0 || body >= (int)h->bodies.size() || h->bodies[body].kind != SPH_BODY_SOFT)
        return fail(h, SPH_ERR_ARG, "anchors need a soft body");
    const DevBody &B = h->bodies[body];
    for (int i = 0; i < n; ++i)
        if (h_local[i] < 0 || h_local[i] >= B.n) return fail(h, SPH_ERR_ARG, "anchor index out of range");
    for (int i = 0; i < n; ++i) {
        float4 &l = h->hlocal[(size_t)(B.first - h->c.nf + h_local[i])];
        l.w = 1.0f;
    }
    return SPH_OK;
}

sph_status sph_cut_springs(sph_handle *h, const float tri[9], int64_t *h_n_cut)
{
    if (!h || !tri || !h_n_cut) return SPH_ERR_ARG;
    for (int i = 0; i < 9; ++i)
        if (!std::isfinite(tri[i])) return fail(h, SPH_ERR_ARG, "non-finite blade");
    sph_status st = finalize(h);
    if (st != SPH_OK) return st;
    unsigned *cnt = at<unsigned>(h, h->L.cut);
    SPH_CUDA(h, cudaMemsetAsync(cnt, 0, 4, h->stream));
    SPH_CUDA(h, launch_cut(h->c, h->stream, tri, cnt));
    unsigned n = 0;
    SPH_CUDA(h, cudaMemcpyAsync(&n, cnt, 4, cudaMemcpyDeviceToHost, h->stream));
    SPH_CUDA(h, cudaStreamSynchronize(h->stream));
    *h_n_cut = (int64_t)n;
    return read_status(h);
}

sph_status sph_get_descriptor(sph_handle *h, float *d_out)
{
    if (!h || !d_out) return SPH_ERR_ARG;
    if (h->grab < 0) return fail(h, SPH_ERR_STATE, "no grabbed body");
    if (h->substeps == 0) return fail(h, SPH_ERR_STATE, "no substep has run");
    SPH_CUDA(h, launch_descriptor(h->c, h->stream, h->grab, d_out));
    return SPH_OK;
}

sph_status sph_get_diag(sph_handle *h, double out[8])
{
    if (!h || !out) return SPH_ERR_ARG;
    sph_status st = finalize(h);
    if (st != SPH_OK) return st;
    SPH_CUDA(h, cudaMemcpyAsync(out, h->c.diag, 64, cudaMemcpyDeviceToHost, h->stream));
    return read_status(h);
}

sph_status sph_get_info(sph_handle *h, int64_t out[5])
{
    if (!h || !out) return SPH_ERR_ARG;
    out[0] = (int64_t)h->hx.size();
    out[1] = h->c.nf;
    out[2] = h->c.ncell;
    out[3] = (int64_t)h->bodies.size();
    out[4] = h->substeps;
    return SPH_OK;
}

sph_status sph_set_profiling(sph_handle *h, int32_t on)
{
    if (!h) return SPH_ERR_ARG;
    if (on && !h->ev[0])
        for (int i = 0; i <= kSubstepKernels; ++i) SPH_CUDA(h, cudaEventCreate(&h->ev[i]));
    if (on < 0 || on > 2) return fail(h, SPH_ERR_ARG, "profiling level 0, 1 or 2");
    h->profiling = on;
    return SPH_OK;
}

sph_status sph_get_kernel_times(sph_handle *h, float out_ms[8])
{
    if (!h || !out_ms) return SPH_ERR_ARG;
    if (!h->ev[0]) return fail(h, SPH_ERR_STATE, "profiling was never enabled");
    SPH_CUDA(h, cudaStreamSynchronize(h->stream));
    for (int i = 0; i < kSubstepKernels; ++i) {
        out_ms[i] = 0.0f;
        // level 2 records the density pass's two events only (kernel 5)
        if (h->prof_last == 2 && i != 5) continue;
        SPH_CUDA(h, cudaEventElapsedTime(&out_ms[i], h->ev[i], h->ev[i + 1]));
    }
    return read_status(h);
}

sph_status sph_sync(sph_handle *h)
{
    if (!h) return SPH_ERR_ARG;
    return read_status(h);
}

const char *sph_last_error(const sph_handle *h)
{
    return h ? h->err.c_str() : "null handle";
}

void sph_destroy(sph_handle *h)
{
    if (!h) return;
    if (h->stream || h->finalized) cudaStreamSynchronize(h->stream);
    if (h->exec1) cudaGraphExecDestroy(h->exec1);
    if (h->exec16) cudaGraphExecDestroy(h->exec16);
    if (h->exec1c) cudaGraphExecDestroy(h->exec1c);
    if (h->exec_prof) cudaGraphExecDestroy(h->exec_prof);
    for (int i = 0; i <= kSubstepKernels; ++i)
        if (h->ev[i]) cudaEventDestroy(h->ev[i]);
    if (h->pin) cudaFreeHost(h->pin);
    delete h;
}

}  // extern "C"

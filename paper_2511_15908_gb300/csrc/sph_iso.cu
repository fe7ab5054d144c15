// sph_iso.cu -- isosurface of the fluid: density field at the corners of a cube grid and
// marching cubes over it (Alg. 2's isosurface compute kernels, Sec. 3.4).
//
// Sec. 3.4 builds the fluid surface as the isosurface of a density field that the fluid
// particles generate through the smoothing kernel, sampled at the corners of a uniform grid
// of cubes offset from the hash grid, with triangles interpolated along the cube edges
// where the field crosses the isovalue (marching cubes); the hash is reused for the field.
//
// Triangulation rule.  Each cube's corners are inside when the field exceeds the isovalue.
// On every face the cut edges are joined by segments: a face with two cut edges joins
// them; a face with four (diagonal corners alike) cuts off each inside corner with the
// segment between its two face edges.  The rule depends only on the face's four corners,
// so two cubes sharing a face draw the same segments there and the surface has no holes.
// The segments close into loops through the cut edges; loops are taken in the order of
// their smallest edge, each starting there and running so that its normal (Newell's
// formula over the edge midpoints) points from the inside corners to the outside ones.
// A loop is split into a fan of triangles from its first vertex unless one of the fan's
// diagonals would join two vertices on a common face of the cube (the loop crosses an
// ambiguous face twice, and the neighbouring cube could draw the same diagonal); then it
// is fanned from an added centre vertex, the mean of its vertices, one triangle per side.
// The table of loops per corner case is built on the host at load time from this rule.
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "sph.h"
#include "sph_device.cuh"

namespace sphgb {

sph_status scene_for_batch(sph_handle *h, SimConst *out);
cudaStream_t scene_stream(sph_handle *h);
const sph_params *scene_params(sph_handle *h);

namespace {

constexpr int kIsoMaxLoop = 4;         // loops per cube (each has >= 3 of the 12 edges)

// corner v sits at offset (v & 1, v >> 1 & 1, v >> 2 & 1); edge e joins kIsoEdge[e]
constexpr int kIsoEdge[12][2] = {{0, 1}, {2, 3}, {4, 5}, {6, 7},     // along x
                                 {0, 2}, {1, 3}, {4, 6}, {5, 7},     // along y
                                 {0, 4}, {1, 5}, {2, 6}, {3, 7}};    // along z

struct IsoCase {
    uint8_t ntri, nloop, centre;        // triangles; loops; bit l: loop l is centre-fanned
    uint8_t len[kIsoMaxLoop];
    uint8_t edge[12];                   // the loops' edges, one loop after the other
};

struct IsoTable {
    IsoCase cs[256];
};

__constant__ IsoTable c_iso;

bool face_shared(int e1, int e2)
{
    for (int axis = 0; axis < 3; ++axis)
        for (int side = 0; side < 2; ++side) {
            auto on = [&](int e) {
                return ((kIsoEdge[e][0] >> axis) & 1) == side && ((kIsoEdge[e][1] >> axis) & 1) == side;
            };
            if (on(e1) && on(e2)) return true;
        }
    return false;
}

// Builds the loops of one corner case by the rule in the file header; false if they do
// not fit the table.
bool build_case(int cs, IsoCase &out)
{
    std::memset(&out, 0, sizeof out);
    bool in[8];
    for (int v = 0; v < 8; ++v) in[v] = (cs >> v) & 1;
    bool cut[12];
    for (int e = 0; e < 12; ++e) cut[e] = in[kIsoEdge[e][0]] != in[kIsoEdge[e][1]];
    // neighbours of each cut edge along the surface (one per face containing it)
    int nb[12][2], nnb[12] = {};
    for (int axis = 0; axis < 3; ++axis) {
        for (int side = 0; side < 2; ++side) {
            // the face: corners with bit `axis` equal to `side`; its edges lie along the
            // two other axes
            int fe[4], nfe = 0;
            for (int e = 0; e < 12; ++e) {
                const int a = kIsoEdge[e][0], b = kIsoEdge[e][1];
                if (((a >> axis) & 1) == side && ((b >> axis) & 1) == side) fe[nfe++] = e;
            }
            int ce[4], nce = 0;
            for (int i = 0; i < 4; ++i)
                if (cut[fe[i]]) ce[nce++] = fe[i];
            auto join = [&](int a, int b) {
                nb[a][nnb[a]++] = b;
                nb[b][nnb[b]++] = a;
            };
            if (nce == 2) {
                join(ce[0], ce[1]);
            } else if (nce == 4) {
                for (int v = 0; v < 8; ++v) {
                    if (((v >> axis) & 1) != side || !in[v]) continue;
                    int pe[2], np = 0;
                    for (int i = 0; i < 4; ++i)
                        if (kIsoEdge[fe[i]][0] == v || kIsoEdge[fe[i]][1] == v) pe[np++] = fe[i];
                    join(pe[0], pe[1]);
                }
            }
        }
    }
    auto corner = [](int v, int a) { return (double)((v >> a) & 1); };
    auto mid = [&](int e, int a) { return 0.5 * (corner(kIsoEdge[e][0], a) + corner(kIsoEdge[e][1], a)); };
    bool used[12] = {};
    int nedge = 0, ntri = 0;
    for (int s = 0; s < 12; ++s) {
        if (!cut[s] || used[s]) continue;
        int loop[12], n = 0;
        int prev = -1, cur = s;
        do {
            loop[n++] = cur;
            used[cur] = true;
            const int a = nb[cur][0], b = nb[cur][1];
            int nxt;
            if (prev < 0) nxt = a < b ? a : b;     // first step: the smaller neighbour
            else nxt = a == prev ? b : a;
            prev = cur;
            cur = nxt;
        } while (cur != s);
        // orientation: Newell normal of the midpoint polygon against inside -> outside
        double N[3] = {0, 0, 0}, O[3] = {0, 0, 0};
        for (int i = 0; i < n; ++i) {
            const int e0 = loop[i], e1 = loop[(i + 1) % n];
            for (int a = 0; a < 3; ++a) {
                const int b = (a + 1) % 3, c = (a + 2) % 3;
                N[a] += (mid(e0, b) - mid(e1, b)) * (mid(e0, c) + mid(e1, c));
            }
            const int va = kIsoEdge[e0][0], vb = kIsoEdge[e0][1];
            const int vin = in[va] ? va : vb, vout = in[va] ? vb : va;
            for (int a = 0; a < 3; ++a) O[a] += corner(vout, a) - corner(vin, a);
        }
        if (N[0] * O[0] + N[1] * O[1] + N[2] * O[2] < 0.0) {
            for (int i = 1, j = n - 1; i < j; ++i, --j) {
                const int t = loop[i];
                loop[i] = loop[j];
                loop[j] = t;
            }
        }
        if (out.nloop >= kIsoMaxLoop) return false;
        bool centre = false;
        for (int i = 2; i + 1 < n; ++i) centre = centre || face_shared(loop[0], loop[i]);
        out.len[out.nloop] = (uint8_t)n;
        if (centre) out.centre |= (uint8_t)(1u << out.nloop);
        ++out.nloop;
        for (int i = 0; i < n; ++i) out.edge[nedge++] = (uint8_t)loop[i];
        ntri += centre ? n : n - 2;
    }
    out.ntri = (uint8_t)ntri;
    return true;
}

std::once_flag g_table_once;
bool g_table_ok = false;
std::mutex g_upload_mu;
bool g_uploaded[64] = {};
IsoTable g_table;

cudaError_t ensure_table()
{
    std::call_once(g_table_once, [] {
        std::memset(&g_table, 0, sizeof g_table);
        g_table_ok = true;
        for (int cs = 0; cs < 256; ++cs)
            if (!build_case(cs, g_table.cs[cs])) { g_table_ok = false; return; }
    });
    if (!g_table_ok) return cudaErrorInvalidValue;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_upload_mu);
    if (!g_uploaded[dev]) {
        e = cudaMemcpyToSymbol(c_iso, &g_table, sizeof g_table);
        if (e != cudaSuccess) return e;
        g_uploaded[dev] = true;
    }
    return cudaSuccess;
}

struct IsoGrid {
    int n[3];                  // corners per axis
    float o[3];                // corner (0, 0, 0)
    float a;                   // cube edge
};

bool iso_grid(const float lo[3], const float hi[3], float a, IsoGrid &g)
{
    if (!(a > 0.0f)) return false;
    for (int k = 0; k < 3; ++k) {
        if (!(hi[k] > lo[k])) return false;
        g.o[k] = lo[k] + 0.5f * a;
        const double n = std::floor(((double)hi[k] - (double)lo[k]) / (double)a);
        if (!(n >= 2.0) || n > 1e6) return false;
        g.n[k] = (int)n;
    }
    g.a = a;
    return (double)g.n[0] * g.n[1] * g.n[2] < 2.0e9;
}

// Field of the fluid particles at every corner: sum over fluid j within 2h of m_j W.
__global__ void __launch_bounds__(kTile) k_iso_field(SimConst c, IsoGrid g, float *field)
{
    const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nv = (long long)g.n[0] * g.n[1] * g.n[2];
    if (v >= nv) return;
    const int i = (int)(v % g.n[0]);
    const int j = (int)((v / g.n[0]) % g.n[1]);
    const int k = (int)(v / ((long long)g.n[0] * g.n[1]));
    const float4 p = make_float4(__fmaf_rn((float)i, g.a, g.o[0]), __fmaf_rn((float)j, g.a, g.o[1]),
                                 __fmaf_rn((float)k, g.a, g.o[2]), 0.0f);
    const float *vw = reinterpret_cast<const float *>(c.vA) + 3;   // id bits, stride 4
    DensitySum acc;
    uint32_t bad = 0;
    for_each_row(c, p, bad, [&](int s0, int e0) {
        for (int q = s0; q < e0; ++q) {
            const float4 xj = __ldg(c.xA + q);
            if (!(xj.w > 0.0f)) continue;                   // boundary particle
            float dx, dy, dz;
            const float r2 = dist2(p, xj, dx, dy, dz);
            if (!(r2 < c.R2)) continue;
            if (__float_as_int(__ldg(vw + 4 * (size_t)q)) >= c.nf) continue;   // soft body
            acc.add(c, xj, r2);
        }
    });
    field[v] = __fmaf_rn(c.alpha6_hi, acc.S, c.alpha6_lo * acc.S - c.alpha6_hi * acc.C);
}

struct IsoCubes {
    int n[3];                  // corners per axis (cubes: n - 1)
    float o[3], a, iso;
    const float *field;
};

__device__ __forceinline__ int iso_case(const IsoCubes &g, int i, int j, int k, float phi[8])
{
    int cs = 0;
#pragma unroll
    for (int v = 0; v < 8; ++v) {
        const size_t idx = ((size_t)(k + (v >> 2)) * g.n[1] + (j + ((v >> 1) & 1))) * g.n[0] +
                           (i + (v & 1));
        phi[v] = __ldg(g.field + idx);
        cs |= (phi[v] > g.iso ? 1 : 0) << v;
    }
    return cs;
}

__device__ __forceinline__ void cube_of(const IsoCubes &g, long long cube, int &i, int &j, int &k)
{
    const int cx = g.n[0] - 1, cy = g.n[1] - 1;
    i = (int)(cube % cx);
    j = (int)((cube / cx) % cy);
    k = (int)(cube / ((long long)cx * cy));
}

__global__ void __launch_bounds__(kTile) k_iso_count(IsoCubes g, long long ncube, uint32_t *cnt)
{
    const long long cube = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (cube >= ncube) return;
    int i, j, k;
    cube_of(g, cube, i, j, k);
    float phi[8];
    cnt[cube] = c_iso.cs[iso_case(g, i, j, k, phi)].ntri;
}

// The vertex on cut edge e of cube (i, j, k): linear interpolation of the field.
__device__ __forceinline__ float3 iso_vertex(const IsoCubes &g, int i, int j, int k,
                                             const float phi[8], int e)
{
    const int axis = e >> 2, idx = e & 3;
    // the edge's lower corner: the two bits other than `axis` come from idx
    const int va = axis == 0 ? ((idx & 1) << 1) | ((idx >> 1) << 2)
                 : axis == 1 ? (idx & 1) | ((idx >> 1) << 2)
                             : (idx & 1) | ((idx >> 1) << 1);
    const int vb = va | (1 << axis);
    const float u = __fdiv_rn(g.iso - phi[va], phi[vb] - phi[va]);
    float p[3];
    const int ci[3] = {i + (va & 1), j + ((va >> 1) & 1), k + ((va >> 2) & 1)};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float base = __fmaf_rn((float)ci[a], g.a, g.o[a]);
        p[a] = a == axis ? __fmaf_rn(u, g.a, base) : base;
    }
    return make_float3(p[0], p[1], p[2]);
}

__device__ __forceinline__ void put(float *out, float3 a, float3 b, float3 c)
{
    out[0] = a.x; out[1] = a.y; out[2] = a.z;
    out[3] = b.x; out[4] = b.y; out[5] = b.z;
    out[6] = c.x; out[7] = c.y; out[8] = c.z;
}

__global__ void __launch_bounds__(kTile) k_iso_write(IsoCubes g, long long ncube,
                                                     const uint32_t *start, float *tris,
                                                     long long max_tris)
{
    const long long cube = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (cube >= ncube) return;
    int i, j, k;
    cube_of(g, cube, i, j, k);
    float phi[8];
    const IsoCase &C = c_iso.cs[iso_case(g, i, j, k, phi)];
    if (C.ntri == 0) return;
    long long t = start[cube];
    int e0 = 0;
    for (int l = 0; l < C.nloop; ++l) {
        const int n = C.len[l];
        if ((C.centre >> l) & 1) {
            // fan from the loop's centre: the mean of its vertices, summed in loop order
            float3 m = make_float3(0.0f, 0.0f, 0.0f);
            for (int s = 0; s < n; ++s) {
                const float3 v = iso_vertex(g, i, j, k, phi, C.edge[e0 + s]);
                m.x += v.x; m.y += v.y; m.z += v.z;
            }
            m.x /= (float)n; m.y /= (float)n; m.z /= (float)n;
            for (int s = 0; s < n; ++s, ++t) {
                if (t >= max_tris) return;
                put(tris + 9 * t, m, iso_vertex(g, i, j, k, phi, C.edge[e0 + s]),
                    iso_vertex(g, i, j, k, phi, C.edge[e0 + (s + 1) % n]));
            }
        } else {
            const float3 v0 = iso_vertex(g, i, j, k, phi, C.edge[e0]);
            for (int s = 1; s + 1 < n; ++s, ++t) {
                if (t >= max_tris) return;
                put(tris + 9 * t, v0, iso_vertex(g, i, j, k, phi, C.edge[e0 + s]),
                    iso_vertex(g, i, j, k, phi, C.edge[e0 + s + 1]));
            }
        }
        e0 += n;
    }
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// the cube counts are scanned by the cell scan (two levels, 2048 entries per tile)
__global__ void __launch_bounds__(kTile) k_iso_scan_tiles(SimConst c) { scan_tiles_item(c, blockIdx.x); }
__global__ void __launch_bounds__(kTile) k_iso_scan_apply(SimConst c) { scan_apply_item(c, blockIdx.x); }

struct IsoLayout {
    size_t cnt, start, tile, total;
    long long ncube;
    int ntiles;
};

bool iso_layout(const int32_t dims[3], IsoLayout &L)
{
    for (int a = 0; a < 3; ++a)
        if (dims[a] < 2) return false;
    L.ncube = (long long)(dims[0] - 1) * (dims[1] - 1) * (dims[2] - 1);
    if (L.ncube >= (1ll << 28)) return false;          // counts and starts are 32-bit
    L.ntiles = (int)((L.ncube + kScanTile - 1) / kScanTile);
    size_t off = 0;
    L.cnt = off; off = align256(off + 4 * ((size_t)L.ncube + 1));
    L.start = off; off = align256(off + 4 * ((size_t)L.ncube + 1));
    L.tile = off; off = align256(off + 4 * (size_t)L.ntiles);
    L.total = off;
    return true;
}

unsigned blocks(long long n) { return (unsigned)((n + kTile - 1) / kTile); }

}  // namespace

}  // namespace sphgb

using namespace sphgb;

extern "C" {

sph_status sph_iso_grid(const sph_params *p, float cube, int32_t dims[3], float origin[3])
{
    if (!p || !dims || !origin) return SPH_ERR_ARG;
    IsoGrid g;
    if (!iso_grid(p->domain_lo, p->domain_hi, cube, g)) return SPH_ERR_ARG;
    for (int a = 0; a < 3; ++a) {
        dims[a] = g.n[a];
        origin[a] = g.o[a];
    }
    return SPH_OK;
}

sph_status sph_iso_field(sph_handle *h, float cube, float *d_field)
{
    if (!h || !d_field) return SPH_ERR_ARG;
    const sph_params *p = scene_params(h);
    IsoGrid g;
    if (!iso_grid(p->domain_lo, p->domain_hi, cube, g)) return SPH_ERR_ARG;
    SimConst c;
    sph_status st = scene_for_batch(h, &c);
    if (st != SPH_OK) return st;
    const cudaStream_t s = scene_stream(h);
    // the hash and reorder of the current state (the next substep's own hash redoes the
    // same work from the same state), then the field from the sorted copy
    if (c.n > 0 && launch_sort(c, s) != cudaSuccess) return SPH_ERR_CUDA;
    const long long nv = (long long)g.n[0] * g.n[1] * g.n[2];
    if (c.n == 0) {
        if (cudaMemsetAsync(d_field, 0, 4 * (size_t)nv, s) != cudaSuccess) return SPH_ERR_CUDA;
        return SPH_OK;
    }
    k_iso_field<<<blocks(nv), kTile, 0, s>>>(c, g, d_field);
    return cudaGetLastError() == cudaSuccess ? SPH_OK : SPH_ERR_CUDA;
}

size_t sph_iso_workspace_bytes(const int32_t dims[3])
{
    IsoLayout L;
    if (!dims || !iso_layout(dims, L)) return 0;
    return L.total;
}

sph_status sph_iso_polygonize(const float *d_field, const int32_t dims[3], const float origin[3],
                              float cube, float iso, void *d_ws, size_t ws_bytes, float *d_tris,
                              int64_t max_tris, int64_t *h_n_tris, void *cuda_stream)
{
    if (!d_field || !dims || !origin || !h_n_tris || max_tris < 0 || (max_tris > 0 && !d_tris))
        return SPH_ERR_ARG;
    if (!(cube > 0.0f) || !std::isfinite(iso)) return SPH_ERR_ARG;
    IsoLayout L;
    if (!iso_layout(dims, L)) return SPH_ERR_ARG;
    if (!d_ws || ws_bytes < L.total || ((uintptr_t)d_ws & 255u)) return SPH_ERR_WORKSPACE;
    if (ensure_table() != cudaSuccess) return SPH_ERR_CUDA;
    const cudaStream_t s = (cudaStream_t)cuda_stream;
    char *ws = (char *)d_ws;
    uint32_t *cnt = (uint32_t *)(ws + L.cnt), *start = (uint32_t *)(ws + L.start);
    IsoCubes g;
    for (int a = 0; a < 3; ++a) {
        g.n[a] = dims[a];
        g.o[a] = origin[a];
    }
    g.a = cube;
    g.iso = iso;
    g.field = d_field;
    k_iso_count<<<blocks(L.ncube), kTile, 0, s>>>(g, L.ncube, cnt);
    SimConst c;
    std::memset(&c, 0, sizeof c);
    c.cnt = cnt;
    c.cell_start = start;
    c.tile_sum = (uint32_t *)(ws + L.tile);
    c.ncell = (int)L.ncube;
    c.n_scan_tiles = L.ntiles;
    k_iso_scan_tiles<<<L.ntiles, kTile, 0, s>>>(c);
    k_iso_scan_apply<<<L.ntiles, kTile, 0, s>>>(c);
    if (max_tris > 0) k_iso_write<<<blocks(L.ncube), kTile, 0, s>>>(g, L.ncube, start, d_tris, max_tris);
    if (cudaGetLastError() != cudaSuccess) return SPH_ERR_CUDA;
    uint32_t total = 0;
    if (cudaMemcpyAsync(&total, start + L.ncube, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return SPH_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return SPH_ERR_CUDA;
    *h_n_tris = (int64_t)total;
    return (int64_t)total > max_tris ? SPH_ERR_CAPACITY : SPH_OK;
}

}  // extern "C"

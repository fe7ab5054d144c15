// sph_internal.cuh -- device-side data layout shared by the kernels and the C ABI.
//
// Particle state is SoA float4 in HBM: x = (x, y, z, SPH mass), v = (vx, vy, vz, id bits).
// Two copies exist: B holds the state in the previous substep's sorted order (the
// "current slot order" the stable sort ties on), A the copy reordered into this
// substep's cell order, which the density and force passes read.  The force pass writes
// the new state back into B, still in A's order, so the next substep's hash reads B.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace sphgb {

constexpr int kMaxBodies = 64;
constexpr int kMaxCellRun = 1536;   // particles scanned per x-run of cells before the
                                    // status word reports SPH_ERR_CAPACITY
constexpr int kMaxCell = 512;       // particles per cell for the deterministic rank
// Lanes per particle of the low-latency force pass (SPH_FLAG_LOW_LATENCY): its grid has
// this many blocks for each 256 particles, and as many diagnostic rows.
#ifndef SPH_LOW_LATENCY_FORCE_G
#define SPH_LOW_LATENCY_FORCE_G 8
#endif
constexpr int kLowLatencyForceG = SPH_LOW_LATENCY_FORCE_G;
constexpr int kScanTile = 2048;     // cells per scan block (256 threads x 8)
constexpr int kReduceChunk = 256;   // body particles per wrench-reduction block
constexpr int kWrenchMinBlocks = 128; // the FP64 reduction is spread over at least this many
constexpr int kDefaultNeighbours = 288; // neighbour-list slots per particle when the
                                       // capacity leaves it 0

// status word bits (mirrors sph_status codes as bit positions)
enum : uint32_t {
    ST_NONFINITE = 1u << 5,
    ST_DOMAIN = 1u << 6,
    ST_TIMEOUT = 1u << 7,
    ST_CAPACITY = 1u << 4,
    ST_BOUNDS = 1u << 9,       // an index check of the bounds-checked build failed
};

struct DevBody {
    int kind, first, n, grabbed;
    int path_n, path_step0, pad0, pad1;
    float mass, inv_mass;
    float inertia[9];
    float inertia_inv[9];      // body frame, computed once at creation
    float t[3], q[4], v[3], w[3];
    float grab_local[3];
};

// Everything a substep kernel needs, passed by value (lives in the constant bank).
struct __align__(16) SimConst {
    int n, nf, nb, n_body_particles;
    int nx, ny, nz, ncell;
    float o[3], inv_cell;
    float R2, h, inv_h;
    float Rc, mc;              // search radius R + margin and the margin, in cell units;
                               // the margin covers FP32 rounding of cell coordinates and
                               // of the neighbour predicate
    float rho0, k, nu20;       // nu20 = 2 (d + 2) nu * 2 with d = 3 (the 2 from rho_bar)
    float tait_B;              // k rho0 / 7: the Tait form's scale (same slope at rest)
    float eps_h2;
    float alpha6_hi, alpha6_lo; // alpha / 6 = 1 / (4 pi h^3) as an unevaluated float pair
    float invh_hi, invh_lo;     // 1 / h as an unevaluated float pair
    float alpha_g;             // alpha / h^2, alpha = 3 / (2 pi h^3)
    float g[3], dt;
    uint32_t flags;
    int max_path;
    int n_scan_tiles;
    int n_force_blocks;
    int n_wblocks;
    int n_wgrid;               // wrench kernel grid = max(n_wblocks, kWrenchMinBlocks)
    int smooth_window;
    int nl_cap;                // neighbour-list slots per particle (a multiple of 4)
    int body_end[kMaxBodies];  // exclusive id end of each body (ids ascending)
    int body_kind[kMaxBodies];
    int wfirst[kMaxBodies];    // first reduction block of each body
    int wcount[kMaxBodies];    // its number of reduction blocks

    float4 *xA, *vA, *xB, *vB;
    float2 *prho;              // (rho, p / rho^2) in sorted order
    uint32_t *key, *rank, *perm, *cnt, *cell_start, *tile_sum;
    unsigned long long *tile_state;   // n_scan_tiles + 1 words of the single-pass scan: per
                                      // tile (kind << 32 | value), then the tile counter;
                                      // zeroed by the hash pass before every scan
    int *slot_of_id;           // id -> sorted slot (soft particles only)
    float4 *locals;            // per body particle (id - nf): body-frame offset
    int *spring_row;           // per body particle (id - nf), CSR row start (+1 entry)
    float4 *spring_e;          // (partner id bits, L0, k_s, c_d)
    float4 *fb, *xb;           // per body particle: coupling force, position
    float4 *acc_dbg;
    int *nnbr;
    DevBody *body;
    float *path;               // max_path x 13
    double *wrench;            // kMaxBodies x 6
    double *wrench_part;       // n_wblocks x 6
    int4 *wblock;              // (body, l0, l1, 0) per reduction block
    double *diag_part;         // n_force_blocks x 8
    double *diag_part2;        // wrench grid x 8 (second level)
    uint4 *nlist4;             // (nl_cap / 4) x n quads: the neighbours the density pass
                               // keeps for the force pass; entry k of particle p is
                               // component k % 4 of nlist4[(k / 4) * n + p], k < nlist_n[p]
    int *nlist_n;              // per particle: neighbours found (> nl_cap: force rescans)
    double *diag;              // 8
    double *wlog;              // max_path x 6
    double *cyc_log;           // smooth_window x 6
    uint32_t *status;          // [0] bits, [1] non-finite count, [2] domain count
    uint32_t *ctr;             // [0] substep counter, [1] reduce ticket, [2] cycle counter
};

// Launchers (sph_kernels.cu).  All enqueue on `s` and return the launch error.
constexpr int kSubstepKernels = 8;
// ev (nullable): kSubstepKernels + 1 events recorded around the kernels; external = record
// them as graph nodes when the stream is being captured.
// cycle_end: the update cycle's end (launch_cycle_end's work) folded into the wrench pass;
// ev_mask: which of the kSubstepKernels + 1 events are recorded (bit k: event k)
cudaError_t launch_substep(const SimConst &c, cudaStream_t s, cudaEvent_t *ev = nullptr,
                           bool external = false, bool cycle_end = false,
                           unsigned ev_mask = ~0u);
// the events around the density pass alone (events 5 and 6)
constexpr unsigned kDensityEvents = (1u << 5) | (1u << 6);
// spring cutting against a blade triangle (sorts the current state first, like the next
// substep would); count (device) += springs cut
cudaError_t launch_cut(const SimConst &c, cudaStream_t s, const float tri[9], unsigned *count);
// the first five substep kernels only: hash, scan, reorder of the current state
cudaError_t launch_sort(const SimConst &c, cudaStream_t s);
cudaError_t launch_cycle_end(const SimConst &c, cudaStream_t s);
cudaError_t launch_set_grab(const SimConst &c, cudaStream_t s, int body, int grab,
                            const float *pose_vel13, const float *grab_local, int set_pose,
                            int path_n);
cudaError_t launch_sorted_keys(const SimConst &c, cudaStream_t s, uint32_t *keys, int *ids);
cudaError_t launch_descriptor(const SimConst &c, cudaStream_t s, int grab_body, float *d_out);

}  // namespace sphgb

struct sph_handle;
namespace sphgb {
// The surrogate's view of a handle (sph_api.cu): its stream, constants and grabbed body
// (-1 if none), and the number of substeps run.
void handle_surrogate_view(const sph_handle *h, cudaStream_t *stream, const SimConst **c, int *grab,
                           long long *substeps);
}  // namespace sphgb

/*
 * sph.h -- C ABI of the GB300 SPH substep with two-way solid coupling
 * (SPHaptics, arXiv 2511.15908).
 *
 * One handle simulates one scene on one GPU: fluid particles, static walls, rigid
 * bodies and mass-spring soft bodies, all represented as SPH particles (Sec. 3.2).
 * Each substep runs the spatial hash of Alg. 2 (cell, count, cumulative sum, sorted
 * index), soft-body springs, the density/pressure pass and the force/integrate pass of
 * Alg. 1, reduces the boundary-particle coupling forces of every rigid body to a wrench
 * in FP64, and integrates the free rigid bodies; the grabbed body's wrench is what the
 * haptic device feels (Sec. 3.3).
 *
 * Conventions shared by every call:
 *   - Ownership: all device memory lives in ONE caller-owned device buffer (the
 *     workspace) whose size sph_workspace_bytes() returns.  The library never calls
 *     cudaMalloc or cudaFree; host arrays passed in are copied before the call returns
 *     and are never retained.  sph_destroy() frees only the host-side handle.
 *   - Streams: every device operation is enqueued on the stream given at creation, in
 *     call order.  Calls marked "synchronises" wait for that stream.
 *   - Errors: every call returns sph_status; nothing throws across the ABI.  Device-side
 *     conditions (non-finite state, particles leaving the domain, cell overflow, a
 *     bounded wait that gave up) are latched in a status word in the workspace and
 *     reported by the next synchronising call.  sph_last_error() gives a message.
 *   - Particle ids are persistent: fluid particles are 0..n_fluid-1 in the order given
 *     to sph_create, then each body's particles in the order the bodies were added.
 *   - Setup calls (sph_add_*) are legal only before the first sph_step (SPH_ERR_STATE).
 *   - Layouts: positions and velocities are packed xyz triples (n x 3 floats); poses are
 *     (x, y, z, qw, qx, qy, qz); body velocities (vx, vy, vz, wx, wy, wz); wrenches
 *     (Fx, Fy, Fz, tx, ty, tz) in doubles, torque about the grab point.
 */
#ifndef SPH_GB300_H
#define SPH_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sph_handle sph_handle;

typedef enum {
    SPH_OK = 0,
    SPH_ERR_ARG = 1,        /* bad argument (null pointer, size out of range) */
    SPH_ERR_CUDA = 2,       /* a CUDA runtime call failed */
    SPH_ERR_WORKSPACE = 3,  /* workspace too small or misaligned */
    SPH_ERR_CAPACITY = 4,   /* more particles/bodies/springs than the capacity given */
    SPH_ERR_NONFINITE = 5,  /* a particle position or velocity became NaN/Inf */
    SPH_ERR_DOMAIN = 6,     /* a particle left the grid domain (its cell was clamped) */
    SPH_ERR_TIMEOUT = 7,    /* a bounded device-side wait gave up */
    SPH_ERR_STATE = 8,      /* call not legal in the current state */
    SPH_ERR_BOUNDS = 9      /* an index check failed (only the build compiled with
                               -DSPH_CHECKED checks; the access was redirected to index 0) */
} sph_status;

/* sph_params.flags */
enum {
    SPH_FLAG_CLAMP_PRESSURE = 1u << 0, /* negative pressures from the linear EOS become 0 */
    SPH_FLAG_RECORD = 1u << 1,         /* keep per-particle acceleration, neighbour
                                          counts and static-body wrenches (test hook) */
    SPH_FLAG_NO_GRAPH = 1u << 2,       /* launch kernels directly instead of replaying a
                                          captured CUDA graph */
    SPH_FLAG_TAIT = 1u << 3,           /* Tait variation of the equation of state, which
                                          Sec. 3.1 names as the alternative to Eq. pressure:
                                          p = B ((rho / rho0)^7 - 1), B = k rho0 / 7 (the
                                          same slope as k (rho - rho0) at rest) */
    SPH_FLAG_VOLUME_BOUNDARY = 1u << 4,/* volume-based boundary particles (Akinci et al., whose
                                          coupling Sec. 2.1 cites): a static or rigid
                                          particle b weighs psi_b = rho0 / sum_{k boundary}
                                          W_bk instead of its mass in the density of fluid
                                          and soft particles; a fluid or soft particle i
                                          feels psi_b (-p_i / rho_i^2 + viscosity with
                                          rho_bar = rho_i) grad W from b and b the opposite
                                          force; boundary particles exert no SPH force on
                                          each other; sph_get_state reports psi_b as a
                                          boundary particle's density */
    SPH_FLAG_LOW_LATENCY = 1u << 5     /* for scenes too small to fill the GPU, whose
                                          substep waits for the serial neighbour loops of
                                          single threads (a body sampled at half spacing
                                          has ~226 neighbours): the density pass (Alg. 1's
                                          density loop) takes 32 cooperating threads per
                                          particle (scenes up to 20,000 particles, else
                                          16) and the force pass 8.  Same neighbours,
                                          neighbour counts and interaction lists; the
                                          densities' float-pair sums and the forces' FP32
                                          sums are added in another order, so they may
                                          round to neighbouring values.  Slower on a scene
                                          that fills the GPU.  No effect with
                                          SPH_FLAG_VOLUME_BOUNDARY or inside a batch
                                          (sph_batch_*), which runs one thread per
                                          particle */
};

/* Body kinds (Sec. 3.2 particle types). */
enum { SPH_BODY_STATIC = 1, SPH_BODY_RIGID = 2, SPH_BODY_SOFT = 3 };

/*
 * Scene parameters, copied at creation.
 *   h            smoothing length of the cubic spline (Sec. 3.1, Eq. kernel); the
 *                support radius is 2h.
 *   rho0, k      rest density and pressure constant of p = k (rho - rho0)
 *                (Sec. 3.1, Eq. pressure).
 *   nu           kinematic viscosity of F^viscosity = m nu lap v (Alg. 1).
 *   g            gravity, the external force per unit mass (Alg. 1).
 *   dt           substep of the semi-implicit Euler update (Sec. 3.1, Eq. euler).
 *   domain_lo/hi box covered by the uniform grid; one margin cell is added per side.
 *   cell         grid cell edge; must be >= h.  The neighbour search visits, per row of
 *                cells, only the cells that can hold a point within 2h (plus a rounding
 *                margin) of the particle, so any cell >= h finds every neighbour; about
 *                h (e.g. h * 1.001) scans the fewest candidates.
 *   visc_eps     regulariser of the viscous term, r^2 + visc_eps h^2.
 *   spring_zeta  damping ratio of soft-body springs.
 *   fluid_spacing lattice spacing of the fluid; fluid SPH mass = rho0 * spacing^3.
 *   flags        SPH_FLAG_*.
 *   smooth_window number of update cycles (sph_step calls) in the rolling average of
 *                the haptic wrench (Sec. 3.3); 1 disables smoothing.
 */
typedef struct {
    float h, rho0, k, nu;
    float g[3];
    float dt;
    float domain_lo[3], domain_hi[3];
    float cell;
    float visc_eps, spring_zeta;
    float fluid_spacing;
    uint32_t flags;
    int32_t smooth_window;
} sph_params;

/*
 * Capacities fixed at creation (they size the workspace).
 *   max_particles  fluid + all body particles
 *   max_bodies     static + rigid + soft bodies (at most 64)
 *   max_springs    soft-body springs (each counted once)
 *   max_path       entries of the grab path (sph_set_grab_path) and of the per-substep
 *                  wrench log
 *   max_neighbours neighbour-list slots per particle (0 = 288; rounded up to a multiple
 *                  of 4), 4 bytes each: the density pass records each particle's
 *                  interaction partners for the force pass; a particle with more partners
 *                  is re-searched by the force pass (same result, slower).  288 covers a
 *                  fluid particle among boundary particles sampled at half its spacing
 *                  (about 270 partners); slots a particle does not use are never touched
 */
typedef struct {
    int32_t max_particles, max_bodies, max_springs, max_path;
    int32_t max_neighbours;
} sph_capacity;

/* Bytes of device workspace a scene with these parameters and capacities needs
 * (0 if the arguments are invalid).  The grid size follows from domain and cell; with
 * SPH_FLAG_LOW_LATENCY the force pass's diagnostic rows take 8 times their usual
 * 256 bytes per 1,024 particles (so the flag is part of the parameters the size is
 * computed for). */
size_t sph_workspace_bytes(const sph_params *p, const sph_capacity *cap);

/*
 * Create a simulation.
 *   d_workspace  device pointer, 256-byte aligned, `bytes` >= sph_workspace_bytes();
 *                owned by the caller and used exclusively by this handle until
 *                sph_destroy.
 *   cuda_stream  cudaStream_t on which every device operation is enqueued (0 = legacy
 *                default stream).
 *   n_fluid      fluid particles; h_xyz (n_fluid x 3, host, copied) positions,
 *                h_vel (n_fluid x 3, host, nullable -> zero) velocities.
 * The handle allocates no device memory; it pins a small host buffer (64 + 16 + 48 x
 * smooth_window bytes, freed by sph_destroy) through which the synchronising reads
 * (wrenches, status) arrive in one stream synchronisation; if pinning is refused they use
 * ordinary host copies.
 * Synchronises.  Errors: SPH_ERR_ARG, SPH_ERR_WORKSPACE, SPH_ERR_CAPACITY, SPH_ERR_CUDA.
 */
sph_status sph_create(const sph_params *p, const sph_capacity *cap, void *d_workspace,
                      size_t bytes, void *cuda_stream, int32_t n_fluid, const float *h_xyz,
                      const float *h_vel, sph_handle **out);

/*
 * Add a static or rigid body sampled by n boundary particles (Sec. 3.2: a rigid body is
 * a set of particles at fixed offsets from its parent transform).
 *   h_local      n x 3 body-frame offsets about the centre of mass (host, copied).
 *   spacing      sampling spacing; each particle's SPH mass is rho0 * spacing^3.
 *   body_mass    inertial mass; 0 makes the body static (its particles are placed once
 *                at pose and never move).
 *   inertia      3x3 body-frame inertia tensor, row-major (ignored when static).
 *   pose         initial pose; vel initial (v, w) (nullable -> zero).
 * Errors: SPH_ERR_ARG, SPH_ERR_CAPACITY, SPH_ERR_STATE, SPH_ERR_CUDA.
 */
sph_status sph_add_rigid(sph_handle *h, int32_t n, const float *h_local, float spacing,
                         float body_mass, const float inertia[9], const float pose[7],
                         const float vel[6], int32_t *out_body_id);

/*
 * Add a mass-spring soft body (Sec. 3.2: surface/lattice particles joined by distance
 * springs, integrated like fluid particles and interacting with everything through SPH).
 *   h_xyz        n x 3 world positions at creation (host, copied); rest lengths are the
 *                creation distances.
 *   h_pairs      n_springs x 2 local particle indices (host, copied); the lookup table
 *                of Alg. 2's spring pass is built from it here, once.
 *   young_E      Young's modulus; each spring gets k_s = E s^2 / L0 (E s on lattice axis
 *                springs) and damping 2 zeta sqrt(k_s m / 2).
 *   poisson_nu   recorded only: a spring lattice cannot represent a Poisson ratio.
 * Errors: SPH_ERR_ARG, SPH_ERR_CAPACITY, SPH_ERR_STATE, SPH_ERR_CUDA.
 */
sph_status sph_add_soft(sph_handle *h, int32_t n, const float *h_xyz, float spacing,
                        int32_t n_springs, const int32_t *h_pairs, float young_E,
                        float poisson_nu, int32_t *out_body_id);

/*
 * Grab (or release with body_id = -1) a rigid body with the haptic device (Sec. 3.3):
 * a grabbed body stops integrating; its pose and velocity are set by the device and the
 * forces on it are read with sph_get_grab_wrench.
 *   pose, vel         device pose (7) and velocity (6) applied from the next substep.
 *   grab_point_local  grab point in the body frame (nullable -> centre of mass); the
 *                     wrench torque is taken about it.
 * Enqueued on the stream (host arrays copied before return).
 */
sph_status sph_set_grab_pose(sph_handle *h, int32_t body_id, const float pose[7],
                             const float vel[6], const float grab_point_local[3]);

/*
 * Give the grabbed body a prescribed path: substep s after this call uses entry
 * min(s, n - 1) of h_path (n x 13: pose 7, velocity 6; host, copied).  n = 0 clears the
 * path (the last pose stays).  Lets a whole device-motion trajectory run without a host
 * round trip per substep.
 */
sph_status sph_set_grab_path(sph_handle *h, int32_t n, const float *h_path);

/*
 * Advance n_substeps substeps (Alg. 2 inner loop; rigid bodies updated every substep).
 * Asynchronous on the handle's stream; replays a captured CUDA graph unless
 * SPH_FLAG_NO_GRAPH.  One call is one update cycle of the haptic smoothing window.
 */
sph_status sph_step(sph_handle *h, int32_t n_substeps);

/*
 * Wrench on the grabbed body after the last substep (raw, smoothed = 0), or its rolling
 * average over the last smooth_window update cycles (smoothed = 1) (Sec. 3.3).  Force =
 * sum of the pair forces on the body's particles (gravity excluded); torque about the
 * grab point.  Synchronises; returns latched device errors.
 */
sph_status sph_get_grab_wrench(sph_handle *h, double out[6], int32_t smoothed);

/*
 * One update cycle of the haptic loop (Sec. 3.3) in a single call: the device pose and
 * velocity of the grabbed body (as sph_set_grab_pose with grab_point_local = NULL), then
 * n_substeps substeps (as sph_step), then its wrench, raw or smoothed (as
 * sph_get_grab_wrench, which synchronises).  Equal, bit for bit, to the three calls.
 * Errors: those of the three calls, in that order.
 */
sph_status sph_haptic_cycle(sph_handle *h, int32_t body_id, const float pose[7], const float vel[6],
                            int32_t n_substeps, int32_t smoothed, double out[6]);

/* Wrench of any static or rigid body after the last substep (static bodies only with
 * SPH_FLAG_RECORD).  Synchronises. */
sph_status sph_get_body_wrench(sph_handle *h, int32_t body_id, double out[6]);

/* Per-substep wrench log of the grabbed body: the last n substeps, oldest first
 * (n <= min(substeps run, max_path)).  Synchronises. */
sph_status sph_get_wrench_log(sph_handle *h, int32_t n, double *out);

/* Body state (t 3, q 4, v 3, w 3) after the last substep.  Synchronises. */
sph_status sph_get_body(sph_handle *h, int32_t body_id, float out[13]);

/*
 * Particle state in id order (each pointer nullable; host arrays of max n entries):
 * positions and velocities (n x 3) after the last substep, density (n) of the last
 * density pass, neighbour counts (n, j != i) and accelerations (n x 3: total for fluid
 * and soft particles including gravity, pair force / mass for boundary particles) of the
 * last substep when SPH_FLAG_RECORD is set.  Synchronises.
 */
sph_status sph_get_state(sph_handle *h, float *h_x, float *h_v, float *h_rho, int32_t *h_nnbr,
                         float *h_acc);

/* Overwrite fluid and soft particle positions/velocities (id order, n x 3, host,
 * nullable); boundary particles follow their bodies.  Synchronises. */
sph_status sph_set_state(sph_handle *h, const float *h_x, const float *h_v);

/*
 * Spatial-hash result of the last substep (test hook): cell key of each sorted slot
 * (n), particle id of each sorted slot (n), cell_start (n_cells + 1).  Nullable.
 * Synchronises.
 */
sph_status sph_get_sort(sph_handle *h, uint32_t *h_keys, int32_t *h_ids, uint32_t *h_cell_start);

/*
 * Diagnostics of the last substep, FP64: [0..2] sum of all pair forces (Newton's third
 * law makes it 0), [3] sum of their magnitudes, [4..6] momentum of fluid and soft
 * particles, [7] sum of m |v|.  Synchronises.
 */
sph_status sph_get_diag(sph_handle *h, double out[8]);

/*
 * Learned haptic-rate wrench surrogate (the paper has no learned part -- it motivates one
 * by the ~60 Hz update rate of the engine loop, Sec. 3.3).
 *
 * sph_get_descriptor writes the 269 surrogate inputs of the grabbed body for the last
 * substep into DEVICE memory d_out (enqueued on the handle's stream): pose (x y z qw qx qy
 * qz), velocity (vx vy vz wx wy wz), then 4 x 4 x 4 cells of edge 2h centred on the grab
 * point (x fastest), each with the mean density of its fluid particles and their
 * mass-weighted mean velocity (zeros when empty).  Errors: SPH_ERR_STATE (nothing grabbed
 * or no substep run).
 */
sph_status sph_get_descriptor(sph_handle *h, float *d_out);

/*
 * The model: a 269-128-128-128-6 multilayer perceptron with tanh-form GELU, BF16 weights
 * and FP32 accumulation on tcgen05 tensor cores; inputs standardised and outputs
 * de-standardised by the kernels.  Parameters (68,358 FP32 master values) in the order
 * W1[128][269] b1[128] W2[128][128] b2[128] W3[128][128] b3[128] W4[6][128] b4[6].
 * All buffers live in one caller-owned workspace sized for max_batch rows.
 */
typedef struct sph_mlp sph_mlp;

int32_t sph_mlp_param_count(void);
size_t sph_mlp_workspace_bytes(int32_t max_batch);
sph_status sph_mlp_create(void *d_workspace, size_t bytes, void *cuda_stream, int32_t max_batch,
                          sph_mlp **out);

/* Host parameters (param_count FP32) and, if h_norm is not NULL, the standardisation
 * xmean[269] xstd[269] ymean[6] ystd[6]; resets the Adam state.  Synchronises. */
sph_status sph_mlp_set_params(sph_mlp *m, const float *h_params, const float *h_norm);
sph_status sph_mlp_get_params(sph_mlp *m, float *h_params);

/* d_x: DEVICE batch x 269 FP32 inputs; d_y: DEVICE batch x 6 wrench outputs.  Async. */
sph_status sph_mlp_forward(sph_mlp *m, const float *d_x, int32_t batch, float *d_y);

/* Gradient of the mean squared error on standardised outputs for targets d_t (DEVICE,
 * batch x 6); h_grad (host, param_count, nullable) and h_loss (nullable).  Synchronises. */
sph_status sph_mlp_gradients(sph_mlp *m, const float *d_x, const float *d_t, int32_t batch,
                             float *h_grad, double *h_loss);

/* One Adam step (beta 0.9 / 0.999, eps 1e-8) on that loss; h_loss nullable (if given,
 * synchronises and returns the loss before the step). */
sph_status sph_mlp_train_step(sph_mlp *m, const float *d_x, const float *d_t, int32_t batch,
                              float lr, double *h_loss);

sph_status sph_mlp_sync(sph_mlp *m);
const char *sph_mlp_last_error(const sph_mlp *m);
void sph_mlp_destroy(sph_mlp *m);

/*
 * The haptic tick on the device (Sec. 3.3: the engine hands the device a new force about
 * every 60 Hz update cycle; the device wants one every millisecond).  At the start of an
 * update cycle sph_surrogate_anchor records the last substep's descriptor and the grabbed
 * body's exact FP64 wrench into the model (enqueued on the handle's stream; the model's
 * stream waits for it).  Each tick, sph_surrogate_tick takes the grab pose and velocity at
 * that instant (host, 13 floats: x y z qw qx qy qz vx vy vz wx wy wz) and the time since
 * the anchor, builds the network's 269 scale-free inputs on the device, runs the network
 * and returns the anchor's exact wrench plus the predicted change (host, 6 doubles, world
 * frame, torque about the grab point).  Synchronises the model's stream.
 *
 * Inputs, in the anchor's body frame R_a (from its quaternion): R_a^T (x - x_a) / h,
 * tau c / h, R_a^T (v - v_a) / c, R_a^T v / c, R_a^T w h / c, then per descriptor cell
 * rho / rho0 - 1 (-1 when empty) and R_a^T v_cell / c; c = sqrt(k) is the sound speed of
 * Eq. pressure.  The network's output is the wrench change since the anchor in that frame,
 * forces over rho0 c^2 h^2, torques over rho0 c^2 h^3.  sph_surrogate_features and
 * sph_surrogate_targets build the same inputs and outputs for n logged pairs (DEVICE
 * arrays: ticks with tick_stride floats per row, anchors with anchor_stride >= 269, times
 * since the anchor, wrenches n x 6 doubles) for training, with the scales of the scene
 * given to sph_surrogate_set_scene (h, k, rho0; sph_surrogate_anchor sets them too).
 * Errors: SPH_ERR_ARG, SPH_ERR_STATE (tick without an anchor; anchor without a grabbed
 * body or before the first substep), SPH_ERR_CUDA, SPH_ERR_TIMEOUT.
 */
sph_status sph_surrogate_set_scene(sph_mlp *m, const sph_params *p);
sph_status sph_surrogate_anchor(sph_handle *h, sph_mlp *m);
sph_status sph_surrogate_tick(sph_mlp *m, const float pose_vel[13], float elapsed, double out[6]);
sph_status sph_surrogate_features(sph_mlp *m, const float *d_ticks, int32_t tick_stride,
                                  const float *d_anchors, int32_t anchor_stride, const float *d_elapsed,
                                  int32_t n, float *d_x);
sph_status sph_surrogate_targets(sph_mlp *m, const double *d_wrench, const double *d_anchor_wrench,
                                 const float *d_anchors, int32_t anchor_stride, int32_t n, float *d_t);

/* Counts: particles, fluid particles, grid cells (nx*ny*nz), bodies, substeps run. */
sph_status sph_get_info(sph_handle *h, int64_t out[5]);

/*
 * Per-kernel timing hook (benchmarks).  With profiling on (on = 1), every later substep
 * records a CUDA event before and after each of its 8 kernels (as event-record nodes inside
 * the captured graph, on the handle's stream); with on = 2 only the two around the density
 * pass, which costs the substep less (each event node adds a few microseconds).
 * sph_get_kernel_times synchronises and returns the durations of the last substep in
 * milliseconds, in launch order: hash, scan tiles (the single-pass scan), scan apply (~0
 * with it), scatter, rank + gather, density, force + integrate, wrench reduction (0 for
 * the kernels a level-2 substep does not time).  The events are created by the first
 * sph_set_profiling(h, on > 0) (no device memory is allocated).  Errors: SPH_ERR_ARG for
 * a level other than 0, 1, 2.
 */
sph_status sph_set_profiling(sph_handle *h, int32_t on);
sph_status sph_get_kernel_times(sph_handle *h, float out_ms[8]);

/*
 * Batched form: many independent scenes of uneven particle counts advanced by ONE
 * persistent cooperative launch per substep (captured into a CUDA graph).  Every scene is
 * a handle set up with the calls above; the batch only adds a small table in its own
 * caller-owned workspace (sph_batch_workspace_bytes).  A batched substep performs, tile
 * for tile, the same arithmetic as sph_step on each scene, so results are bit-identical.
 * Member handles must not be stepped or queried while a batched launch is in flight:
 * call sph_batch_sync first.  The grid barriers between phases are bounded; a barrier
 * that gives up latches SPH_ERR_TIMEOUT, reported (and reset) by sph_batch_sync.
 */
typedef struct sph_batch sph_batch;

size_t sph_batch_workspace_bytes(int32_t n_scenes);

/* scenes: n_scenes handles (finalized here, their streams synchronised); d_workspace:
 * device, 256-byte aligned, >= sph_batch_workspace_bytes(n_scenes); cuda_stream: the
 * stream of the batched launches. */
sph_status sph_batch_create(sph_handle *const *scenes, int32_t n_scenes, void *d_workspace,
                            size_t bytes, void *cuda_stream, sph_batch **out);

/* Launch structure: blocks_per_sm = 1 .. occupancy limit runs the persistent kernel with
 * that many resident blocks per SM, taking tiles_per_fetch (1 .. 64) tiles per work-queue
 * fetch; blocks_per_sm = 0 runs one kernel per phase over all scenes' tiles instead (same
 * tiles, same results; each phase at its own occupancy); blocks_per_sm = -1 runs every
 * scene's own substep kernels as parallel branches of one captured graph (one branch per
 * scene up to 64; beyond that, scenes balanced over 64 branches by particle count; same
 * results).  tiles_per_fetch matters only for the
 * persistent kernel.  Errors: SPH_ERR_ARG outside these ranges. */
sph_status sph_batch_configure(sph_batch *b, int32_t blocks_per_sm, int32_t tiles_per_fetch);

/* Autotuner: times substeps_per_trial substeps (after one warm-up substep) for every
 * launch-structure candidate -- per-phase kernels, and the persistent kernel at every
 * blocks-per-SM x {1, 2, 4} tiles per fetch -- keeps the fastest and returns it in
 * out_choice (nullable).  Advances the scenes by (3 max_bps + 1)(1 + substeps_per_trial)
 * substeps. */
sph_status sph_batch_tune(sph_batch *b, int32_t substeps_per_trial, int32_t out_choice[2]);

/* Advance every scene by n_substeps substeps (one update cycle per scene).  Asynchronous. */
sph_status sph_batch_step(sph_batch *b, int32_t n_substeps);

/* Wait for the batch stream; reports SPH_ERR_TIMEOUT if a barrier gave up. */
sph_status sph_batch_sync(sph_batch *b);

/* scenes, SMs, blocks per SM, tiles per fetch. */
sph_status sph_batch_info(sph_batch *b, int32_t out[4]);

/* Test hook for the bounded wait: launches one grid barrier that expects missing_blocks
 * more arrivals than blocks exist, so every block gives up after spin_limit sleeps of
 * ~64 ns; the next sph_batch_sync reports SPH_ERR_TIMEOUT and resets the barrier. */
sph_status sph_batch_test_barrier(sph_batch *b, int32_t missing_blocks, int32_t spin_limit);

const char *sph_batch_last_error(const sph_batch *b);

/* Free the host-side batch and its graphs (the workspace and the scenes stay). */
void sph_batch_destroy(sph_batch *b);

/*
 * Checkpoint and resume.  A checkpoint holds everything that carries over from one substep
 * to the next: particle state in its current slot order (the stable sort ties on it),
 * body-frame offsets and anchors, the spring table with its cuts, the body table, the grab
 * path, the last wrenches, both wrench logs, the status word and the counters, behind a
 * small header (magic "SPHCKPT1", substep count, particle and body counts, grabbed body).
 * Everything else is recomputed by every substep.  A handle created from the same scene
 * (same parameters, capacities, bodies and springs) that loads it continues bit-identically
 * to the uninterrupted run.
 *   sph_checkpoint_bytes  size of a checkpoint of h (0 on error)
 *   sph_checkpoint_save   writes it to host memory h_buf (>= that size); synchronises
 *   sph_checkpoint_load   restores it into h; synchronises
 * Errors: SPH_ERR_ARG (buffer too small, not a checkpoint, another scene), SPH_ERR_CUDA.
 * The paper has no checkpoint.
 */
size_t sph_checkpoint_bytes(sph_handle *h);
sph_status sph_checkpoint_save(sph_handle *h, void *h_buf, size_t bytes);
sph_status sph_checkpoint_load(sph_handle *h, const void *h_buf, size_t bytes);

/*
 * Cloth anchors (Sec. 4: a soft-body cloth plane with definable anchor points).  The listed
 * particles of soft body `body` (local indices 0..n_body-1) keep their position and stay
 * at rest; they still exert and feel SPH and spring forces (their acceleration is reported
 * under SPH_FLAG_RECORD).  Only before the first sph_step.  Errors: SPH_ERR_ARG,
 * SPH_ERR_STATE.
 */
sph_status sph_set_anchors(sph_handle *h, int32_t body, int32_t n, const int32_t *h_local);

/*
 * Incision (Sec. 4: a scalpel cutting the skin of a soft body): every active spring of every
 * soft body whose segment between its two particles' current positions meets the closed
 * triangle tri (host, v0 v1 v2, 9 floats) is cut: its stiffness and damping become 0 for
 * the rest of the run.  A stroke of the blade between two frames is two such triangles.
 * The test is Moller and Trumbore's in FP32 (segment parameter in [0, 1]; a segment
 * parallel to the triangle within |det| <= 1e-7 |e1|_1 |d x e2|_1 does not meet it), taken
 * with the spring's lower particle id as the segment start.  The current state is sorted
 * first, as the next substep's hash would (the simulation is unaffected).  *h_n_cut
 * receives the number of springs cut by this call.  Synchronises.  Errors: SPH_ERR_ARG,
 * SPH_ERR_CUDA and the handle's pending status.  The paper does not give its cutting
 * model; this is one reading of it.
 */
sph_status sph_cut_springs(sph_handle *h, const float tri[9], int64_t *h_n_cut);

/*
 * Isosurface of the fluid (Alg. 2's isosurface compute kernels; Sec. 3.4).  The fluid's
 * surface is the isosurface of a density field that the fluid particles generate through
 * the smoothing kernel, sampled at the corners of a uniform grid of cubes offset from the
 * hash grid and polygonised by marching cubes.
 *
 * Corner grid of edge `cube` over the scene's domain: corner (i, j, k) sits at
 * origin + (i, j, k) cube with origin = domain_lo + cube / 2 (half a cube off the domain
 * corner) and dims[a] = floor((domain_hi[a] - domain_lo[a]) / cube) corners per axis
 * (>= 2 each).  Errors: SPH_ERR_ARG.
 */
sph_status sph_iso_grid(const sph_params *p, float cube, int32_t dims[3], float origin[3]);

/*
 * Density field of the fluid particles at every corner of that grid:
 * phi(c) = sum over fluid particles j with |c - x_j| < 2h of m_j W(|c - x_j|, h)
 * (Eq. density without the boundary and soft-body particles), from the current state.
 *   d_field  device, dims[0] * dims[1] * dims[2] floats, x fastest; written.
 * The spatial hash and reorder of the current state run first (the grid is reused for the
 * corner search, as Sec. 3.4 says); the next substep redoes the same hash from the same
 * state, so the simulation is unaffected, but sph_get_sort afterwards reports this hash.
 * Enqueued on the handle's stream after a synchronisation.  Errors: SPH_ERR_ARG,
 * SPH_ERR_CUDA, and the handle's pending status.
 */
sph_status sph_iso_field(sph_handle *h, float cube, float *d_field);

/* Device workspace of sph_iso_polygonize for a corner grid of dims (0 if dims are invalid:
 * each >= 2 and fewer than 2^28 cubes). */
size_t sph_iso_workspace_bytes(const int32_t dims[3]);

/*
 * Marching cubes over a corner field (any field; sph_iso_field's or the caller's).
 *   d_field      device, dims[0] * dims[1] * dims[2] floats, x fastest.
 *   origin, cube corner (0,0,0) and cube edge, as sph_iso_grid returns them.
 *   iso          isovalue; a corner is inside the surface when its value exceeds it.
 *   d_ws         device workspace, 256-byte aligned, >= sph_iso_workspace_bytes(dims).
 *   d_tris       device output, max_tris x 9 floats: the three vertices (x, y, z) of each
 *                triangle, ordered by cube (x fastest) and within a cube by the rule
 *                below; vertex on the edge from corner a to b at
 *                p_a + (iso - phi_a) / (phi_b - phi_a) (p_b - p_a); the triangle's
 *                normal (v1 - v0) x (v2 - v0) points out of the surface (toward lower
 *                field values).
 *   h_n_tris     host: the number of triangles of the whole surface.
 * Rule per cube: on each face, two cut edges are joined by a segment, four cut edges by one
 * segment around each inside corner (the face decides alone, so neighbouring cubes agree and
 * the surface is closed); the segments form loops through the cut edges, taken in the
 * order of their smallest edge, each starting there (first step to the smaller of its two
 * neighbours) and running so that its normal (Newell's formula over the edge midpoints)
 * points from the inside corners to the outside ones; a loop is split into a fan from its
 * first vertex, or -- when a fan diagonal would join two vertices on a common cube face --
 * into a fan from its centre (the mean of its vertices, one triangle per side, the centre
 * first).  At most 7 triangles per cube.  Edges are numbered 0-3 along x
 * (corners 0-1, 2-3, 4-5, 6-7), 4-7 along y (0-2, 1-3, 4-6, 5-7), 8-11 along z (0-4, 1-5,
 * 2-6, 3-7), corner v at offset (v & 1, v >> 1 & 1, v >> 2 & 1).
 * Synchronises the stream.  Returns SPH_ERR_CAPACITY (with *h_n_tris set) when the surface
 * has more than max_tris triangles; only the first max_tris are written.  Errors:
 * SPH_ERR_ARG, SPH_ERR_WORKSPACE, SPH_ERR_CAPACITY, SPH_ERR_CUDA.  The paper's own grid
 * spacing and isovalue are not given; callers choose them.
 */
sph_status sph_iso_polygonize(const float *d_field, const int32_t dims[3], const float origin[3],
                              float cube, float iso, void *d_ws, size_t ws_bytes, float *d_tris,
                              int64_t max_tris, int64_t *h_n_tris, void *cuda_stream);

/*
 * Allocation-free spatial hash.  The paper has no counterpart: this entry point exists for
 * callers that cannot allocate device memory -- an engine plugin whose device memory is
 * owned by the host engine's allocator, a real-time haptic loop that must not allocate
 * after start-up, or code running while a stream is captured into a CUDA graph (where
 * cudaMalloc is not permitted).  It computes what a substep's spatial hash computes (cell
 * key of each sorted slot, stable counting-sort order, cell ranges) for n particles given
 * as DEVICE float4 (x, y, z, any) records (16-byte aligned), on the grid that sph_create
 * builds from p (domain_lo/hi, cell; the other fields are ignored).
 *   d_keys[n]          cell key of each sorted slot
 *   d_order[n]         input index of the particle in each sorted slot (ties keep input
 *                      order in every cell of at most 512 particles; a cell holding more
 *                      gets its members in an arbitrary order, without an error -- the
 *                      keys stay ascending and d_order stays a permutation)
 *   d_cell_start[C+1]  first sorted slot of each cell, C = grid cells
 * It allocates nothing: the per-cell counters and per-particle ranks live in one fixed
 * file-scope device array of about 4.2 MB, reserved on every GPU that loads this library
 * until the process exits.  Limits: n <= SPH_NOALLOC_MAX_PARTICLES and C <=
 * SPH_NOALLOC_MAX_CELLS, else SPH_ERR_CAPACITY (nothing is launched).  The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress) with that device
 * current; make that first call before any stream capture.  The address is kept per
 * device for the life of the process: after cudaDeviceReset on a device this entry point
 * must not be called on it again in the same process.  Every call shares the array:
 * calls whose work overlaps on the GPU (other streams, other threads) race -- serialise
 * them.  Enqueued on cuda_stream; particles outside the domain are clamped into the border
 * cells as in sph_step (not reported here).  Errors: SPH_ERR_ARG, SPH_ERR_CAPACITY,
 * SPH_ERR_CUDA.
 */
#define SPH_NOALLOC_MAX_PARTICLES (1 << 18)
#define SPH_NOALLOC_MAX_CELLS (1 << 18)
sph_status sph_cell_sort_noalloc(const sph_params *p, const float *d_xyzm, int32_t n,
                                 uint32_t *d_keys, int32_t *d_order, uint32_t *d_cell_start,
                                 void *cuda_stream);

/*
 * Measurement hook (not part of the method): enqueues on cuda_stream one kernel of
 * `blocks` blocks of 256 threads, each thread running `iters` (a multiple of 16) steps of
 * 8 independent FP32 FMA chains, and stores its FP32 flop count (2 per FMA) in
 * *out_flops.  The caller times the launch with events on that stream; flops / time is
 * the FP32 FMA throughput the density and force passes are reported against.  d_sink: a
 * device buffer of at least 256 floats the kernel may write (it does not for these
 * arguments).  Errors: SPH_ERR_ARG, SPH_ERR_CUDA.
 */
sph_status sph_measure_fp32_fma(void *cuda_stream, int32_t blocks, int32_t iters, float *d_sink,
                                double *out_flops);

/* Wait for the stream and report latched device errors. */
sph_status sph_sync(sph_handle *h);

/* Message of the last error on this handle (never NULL; "" if none). */
const char *sph_last_error(const sph_handle *h);

/* Free the host-side handle and its CUDA graphs; the workspace stays the caller's. */
void sph_destroy(sph_handle *h);

#ifdef __cplusplus
}
#endif

#endif /* SPH_GB300_H */

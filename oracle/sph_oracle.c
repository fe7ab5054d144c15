/*
 * sph_oracle.c -- plain, slow FP64 CPU reference of one SPH substep with two-way
 * solid coupling (SPHaptics, arXiv 2511.15908).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's CPU
 * baseline may load this library.  It shares no code, header, table or constant
 * generator with the CUDA path.
 *
 * Passages followed (section / equation / algorithm of the paper):
 *   Sec. 3.1, Alg. 1      density pass, force pass, integrate pass
 *   Sec. 3.1, Eq. kernel  cubic-spline W(r,h) with support 2h
 *   Sec. 3.1, Eq. density rho_i = sum_j m_j W(|x_i - x_j|, h)
 *   Sec. 3.1, Eq. pressure p_i = k (rho_i - rho_0); with the Tait flag the variation the
 *                         same passage names instead (see readings)
 *   Sec. 3.1, Eq. euler   v += a dt;  x += v(t+dt) dt
 *   Sec. 3.1 (uniform-grid spatial hash) and Alg. 2 (cell, count, cumulative sum,
 *                         sorted index)
 *   Sec. 3.2              particle types; rigid bodies as boundary particles whose
 *                         accelerations become point forces on the parent; soft
 *                         bodies as particles joined by springs
 *   Sec. 3.3              the grabbed body's force is read instead of integrated
 *
 * Readings of points the paper leaves open (they are also listed in the design notes):
 *   - support radius R = 2h and alpha_3 = 3 / (2 pi h^3) (unit integral);
 *   - -(m_i/rho_i) grad p_i is discretised as
 *       F^p_ij = -m_i m_j (p_i/rho_i^2 + p_j/rho_j^2) grad_i W_ij,
 *     m_i nu lap v_i as the projected (Monaghan) form
 *       F^v_ij = 2(d+2) nu m_i m_j / rho_bar (v_ij . x_ij) / (r^2 + eps h^2) grad_i W_ij,
 *     with rho_bar = (rho_i + rho_j)/2, d = 3; both antisymmetric and central;
 *   - density sums over every particle type, self term included; forces act between
 *     every pair except two particles of the same static or rigid body;
 *   - the cell of a particle, the neighbour predicate and the boundary positions fed
 *     to them are fixed FP32 operation sequences (below), so integer results are
 *     bit-defined; all physics is FP64 from the FP32 state;
 *   - the Tait variation of the equation of state (named in Sec. 3.1, form not given) is
 *     the weakly compressible form p = B ((rho / rho_0)^gamma - 1), gamma = 7, with
 *     B = k rho_0 / gamma so that dp/drho at rest equals the linear form's k;
 *   - the volume-based boundary variant (Akinci et al., cited in Sec. 2.1; the flag
 *     ORC_VOLUME_BOUNDARY): each static or rigid particle b carries the weight
 *     psi_b = rho_0 / sum_{k boundary} W_bk (self included) in place of its mass in the
 *     density of fluid and soft particles; a fluid or soft particle i feels
 *     psi_b (-p_i / rho_i^2 + viscosity with rho_bar = rho_i) grad W from b, b feels the
 *     opposite force, and two boundary particles exert no SPH force on each other;
 *     the density reported for a boundary particle is its psi_b;
 *   - the grab wrench is the sum of pair forces on the body's particles (gravity
 *     excluded) with torque about the grab point; rigid bodies are updated every
 *     substep.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Host threads the oracle's parallel loops use (the CPU baseline times 1 and all cores). */
void orc_set_threads(int n)
{
#ifdef _OPENMP
    omp_set_num_threads(n > 0 ? n : omp_get_num_procs());
#else
    (void)n;
#endif
}

#define ORC_STATIC 1
#define ORC_RIGID 2
#define ORC_SOFT 3

#define ORC_CLAMP_PRESSURE 1
#define ORC_TAIT 8
#define ORC_VOLUME_BOUNDARY 16
#define ORC_TAIT_GAMMA 7.0

#define ORC_PI 3.14159265358979323846

typedef struct {
    double h, rho0, k, nu, g[3], dt, visc_eps, spring_zeta;
    float lo[3], hi[3], cell;
    int flags;
} orc_params;

typedef struct {
    int kind, first, n, grabbed;
    double mass;            /* inertial mass (rigid) */
    double inertia[9];      /* body-frame inertia, row-major (rigid) */
    float t[3], q[4], v[3], w[3];   /* centre of mass, orientation (w,x,y,z), velocities */
    float grab_local[3];    /* grab point in the body frame */
    const float *local;     /* n x 3: rigid body-frame offsets; static world positions */
    int n_springs;
    const int *springs;     /* n_springs x 2 local indices (soft) */
    const double *spring_L0, *spring_k, *spring_c;   /* per spring (soft); a cut spring has
                                                        k = c = 0 and acts no more */
    const int *anchored;        /* soft, per local particle (may be NULL): pinned at rest */
} orc_body;

/* ---------------------------------------------------------------- kernel (Eq. kernel) */

double orc_alpha(double h) { return 3.0 / (2.0 * ORC_PI * h * h * h); }

/* W(r, h) of the cubic spline, support 2h. */
double orc_W(double r, double h)
{
    double q = r / h, a = orc_alpha(h);
    if (q < 1.0) return a * (2.0 / 3.0 - q * q + 0.5 * q * q * q);
    if (q < 2.0) { double t = 2.0 - q; return a * t * t * t / 6.0; }
    return 0.0;
}

/* grad_i W for x_ij = x_i - x_j equals orc_gradW_coef(r,h) * x_ij; the coefficient is
 * dW/dr / r = (alpha / h^2) * w'(q) / q, finite at r = 0. */
double orc_gradW_coef(double r, double h)
{
    double q = r / h, a = orc_alpha(h) / (h * h);
    if (q < 1.0) return a * (-2.0 + 1.5 * q);
    if (q < 2.0) { double t = 2.0 - q; return a * (-0.5 * t * t / q); }
    return 0.0;
}

/* ------------------------------------------------ uniform grid (Sec. 3.1, Alg. 2) */

/* Grid: origin o = lo - cell, n_a = floor((hi_a - o_a) * inv) + 2 with inv = 1/cell (FP32). */
void orc_grid_dims(const orc_params *P, int dims[3])
{
    float inv = 1.0f / P->cell;
    for (int a = 0; a < 3; ++a) {
        float o = P->lo[a] - P->cell;
        float u = (P->hi[a] - o) * inv;
        dims[a] = (int)floorf(u) + 2;
    }
}

/* Cell coordinate on one axis: floor((x - o) * inv) in FP32, clamped to [0, n-1].
 * Returns 1 when the coordinate had to be clamped (outside the domain or not finite). */
static int orc_cell_axis(float x, float o, float inv, int n, int *c)
{
    if (!isfinite(x)) { *c = 0; return 1; }
    float u = (x - o) * inv;
    float f = floorf(u);
    if (f < 0.0f) { *c = 0; return 1; }
    if (f > (float)(n - 1)) { *c = n - 1; return 1; }
    *c = (int)f;
    return 0;
}

/* Linear cell key (x fastest) of each particle. Returns the number of clamped particles. */
int orc_hash(const orc_params *P, int n, const float *x, uint32_t *key)
{
    int dims[3], bad = 0;
    orc_grid_dims(P, dims);
    float inv = 1.0f / P->cell;
    float o[3];
    for (int a = 0; a < 3; ++a) o[a] = P->lo[a] - P->cell;
    for (int i = 0; i < n; ++i) {
        int c[3], b = 0;
        for (int a = 0; a < 3; ++a) b |= orc_cell_axis(x[3 * i + a], o[a], inv, dims[a], &c[a]);
        bad += b;
        key[i] = (uint32_t)(((int64_t)c[2] * dims[1] + c[1]) * dims[0] + c[0]);
    }
    return bad;
}

/* Counting sort of Alg. 2: count per cell, cumulative sum, sorted index.  Particles are
 * placed in increasing current slot order, so the sort is stable.
 * cell_start has ncell + 1 entries; src[p] = current slot of sorted slot p. */
void orc_counting_sort(int n, const uint32_t *key, int ncell, uint32_t *cell_start, int *src)
{
    uint32_t *cnt = (uint32_t *)calloc((size_t)ncell + 1, sizeof(uint32_t));
    for (int i = 0; i < n; ++i) cnt[key[i]]++;
    uint32_t run = 0;
    for (int c = 0; c < ncell; ++c) { cell_start[c] = run; run += cnt[c]; cnt[c] = 0; }
    cell_start[ncell] = run;
    for (int i = 0; i < n; ++i) {
        uint32_t k = key[i];
        src[cell_start[k] + cnt[k]++] = i;
    }
    free(cnt);
}

/* Neighbour predicate (FP32): d = x_j - x_i per axis, r2 = fma(dz,dz, fma(dy,dy, dx*dx)),
 * neighbour iff r2 < R2 with R2 = (2h)^2 rounded to FP32. */
static inline int orc_close(const float *xi, const float *xj, float R2)
{
    float dx = xj[0] - xi[0], dy = xj[1] - xi[1], dz = xj[2] - xi[2];
    float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
    return r2 < R2;
}

float orc_support2(const orc_params *P)
{
    float R = 2.0f * (float)P->h;
    return R * R;
}

/* Brute-force O(n^2) neighbour counts (j != i). */
void orc_nnbr_brute(const orc_params *P, int n, const float *x, int *nnbr)
{
    float R2 = orc_support2(P);
#pragma omp parallel for schedule(static) if (n > 4096)
    for (int i = 0; i < n; ++i) {
        int c = 0;
        for (int j = 0; j < n; ++j)
            if (j != i && orc_close(x + 3 * i, x + 3 * j, R2)) ++c;
        nnbr[i] = c;
    }
}

/* -------------------------------------------------------------- neighbour iteration */

typedef struct {
    int mode;                  /* 0 brute force, 1 grid */
    int n, dims[3];
    const float *xs;           /* sorted FP32 positions */
    const uint32_t *key;       /* sorted keys */
    const uint32_t *cell_start;
    float R2;
    int span;                  /* grid mode: cells searched on each side of the own cell */
} orc_nbrs;

/* Two particles closer than R lie at most floor(R / cell) + 1 cells apart along an axis
 * (the small relative slack absorbs FP32 rounding of the cell coordinates), so the grid
 * search visits that many cells on each side; the brute-force mode is the definition. */
static int orc_span(const orc_params *P)
{
    double R = 2.0 * (double)P->h;
    return (int)floor(R / (double)P->cell * (1.0 + 1e-5)) + 1;
}

/* Calls visit(p, q, ctx) for every q != p with the FP32 predicate true, in a fixed order. */
typedef void (*orc_visit)(int p, int q, void *ctx);

static void orc_for_neighbours(const orc_nbrs *N, int p, orc_visit visit, void *ctx)
{
    const float *xp = N->xs + 3 * p;
    if (N->mode == 0) {
        for (int q = 0; q < N->n; ++q)
            if (q != p && orc_close(xp, N->xs + 3 * q, N->R2)) visit(p, q, ctx);
        return;
    }
    int nx = N->dims[0], ny = N->dims[1], nz = N->dims[2];
    uint32_t k = N->key[p];
    int cx = (int)(k % (uint32_t)nx), cy = (int)((k / (uint32_t)nx) % (uint32_t)ny);
    int cz = (int)(k / ((uint32_t)nx * (uint32_t)ny));
    const int S = N->span;
    for (int z = cz - S; z <= cz + S; ++z) {
        if (z < 0 || z >= nz) continue;
        for (int y = cy - S; y <= cy + S; ++y) {
            if (y < 0 || y >= ny) continue;
            for (int xx = cx - S; xx <= cx + S; ++xx) {
                if (xx < 0 || xx >= nx) continue;
                uint32_t c = (uint32_t)((z * ny + y) * nx + xx);
                for (uint32_t q = N->cell_start[c]; q < N->cell_start[c + 1]; ++q)
                    if ((int)q != p && orc_close(xp, N->xs + 3 * q, N->R2)) visit(p, (int)q, ctx);
            }
        }
    }
}

/* ------------------------------------------------------------------ FP32 rotation */

/* Rotation matrix of a unit quaternion (w,x,y,z) in FP32, each product and sum rounded. */
void orc_rot_f32(const float q[4], float R[9])
{
    float w = q[0], x = q[1], y = q[2], z = q[3];
    float xx = x * x, yy = y * y, zz = z * z, xy = x * y, xz = x * z, yz = y * z;
    float wx = w * x, wy = w * y, wz = w * z;
    R[0] = 1.0f - 2.0f * (yy + zz); R[1] = 2.0f * (xy - wz);        R[2] = 2.0f * (xz + wy);
    R[3] = 2.0f * (xy + wz);        R[4] = 1.0f - 2.0f * (xx + zz); R[5] = 2.0f * (yz - wx);
    R[6] = 2.0f * (xz - wy);        R[7] = 2.0f * (yz + wx);        R[8] = 1.0f - 2.0f * (xx + yy);
}

/* World position of a body-frame offset: ((R0 l0 + R1 l1) + R2 l2) + t per row, FP32. */
void orc_body_point_f32(const float R[9], const float t[3], const float l[3], float out[3])
{
    for (int a = 0; a < 3; ++a) {
        float s = R[3 * a] * l[0];
        float u = R[3 * a + 1] * l[1];
        s = s + u;
        u = R[3 * a + 2] * l[2];
        s = s + u;
        out[a] = s + t[a];
    }
}

static void orc_rot_f64(const double q[4], double R[9])
{
    double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

static void cross3(const double a[3], const double b[3], double c[3])
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

/* ------------------------------------------------------------------- soft springs */

/* Spring constants of a lattice soft body (mass-spring model of Sec. 3.2): rest length
 * from the creation positions, k_s = E s^2 / L0 (E s on axis springs, E s / sqrt 2 on
 * face diagonals), damping c = 2 zeta sqrt(k_s m / 2) (a damping ratio zeta per spring). */
void orc_soft_setup(int n_springs, const int *pairs, const float *rest_xyz, double young,
                    double spacing, double pmass, double zeta, double *L0, double *ks, double *cd)
{
    for (int s = 0; s < n_springs; ++s) {
        const float *a = rest_xyz + 3 * pairs[2 * s], *b = rest_xyz + 3 * pairs[2 * s + 1];
        double d0 = (double)a[0] - b[0], d1 = (double)a[1] - b[1], d2 = (double)a[2] - b[2];
        L0[s] = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
        ks[s] = young * spacing * spacing / L0[s];
        cd[s] = 2.0 * zeta * sqrt(ks[s] * pmass / 2.0);
    }
}

/* ----------------------------------------------------------------- substep driver */

typedef struct {
    const orc_params *P;
    const double *xd, *vd, *m, *rho, *pres;
    const double *psi;          /* volume-boundary weights (NULL: mass-based boundaries) */
    int weight_boundary;        /* density: weigh boundary neighbours by psi */
    const int *body_of;         /* sorted slot -> body index or -1 (fluid) */
    const int *kind_of;         /* sorted slot -> kind (0 fluid) */
    double h;
    double acc[3], rho_sum;
    double gabs, fabs_sum;      /* sum_j m_j |grad W_ij|, sum_j |F_ij| / m_i */
    int count;
} orc_pair_ctx;

static void visit_density(int p, int q, void *vctx)
{
    orc_pair_ctx *c = (orc_pair_ctx *)vctx;
    double d0 = c->xd[3 * p] - c->xd[3 * q], d1 = c->xd[3 * p + 1] - c->xd[3 * q + 1];
    double d2 = c->xd[3 * p + 2] - c->xd[3 * q + 2];
    double r = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
    int qb = c->kind_of && (c->kind_of[q] == ORC_STATIC || c->kind_of[q] == ORC_RIGID);
    c->rho_sum += (c->weight_boundary && qb ? c->psi[q] : c->m[q]) * orc_W(r, c->h);
    c->count++;
}

/* Volume-boundary weight sum: W to every boundary neighbour (the self term is added by
 * the caller). */
static void visit_boundary_sum(int p, int q, void *vctx)
{
    orc_pair_ctx *c = (orc_pair_ctx *)vctx;
    if (!(c->kind_of[q] == ORC_STATIC || c->kind_of[q] == ORC_RIGID)) return;
    double d0 = c->xd[3 * p] - c->xd[3 * q], d1 = c->xd[3 * p + 1] - c->xd[3 * q + 1];
    double d2 = c->xd[3 * p + 2] - c->xd[3 * q + 2];
    c->rho_sum += orc_W(sqrt(d0 * d0 + d1 * d1 + d2 * d2), c->h);
}

/* Pair force on p from q divided by m_p (pressure and viscosity of Alg. 1). */
static void visit_force(int p, int q, void *vctx)
{
    orc_pair_ctx *c = (orc_pair_ctx *)vctx;
    int bp = c->body_of[p];
    int kp = c->kind_of[p];
    if (bp >= 0 && bp == c->body_of[q] && (kp == ORC_STATIC || kp == ORC_RIGID)) return;
    const orc_params *P = c->P;
    double x[3], v[3];
    for (int a = 0; a < 3; ++a) {
        x[a] = c->xd[3 * p + a] - c->xd[3 * q + a];
        v[a] = c->vd[3 * p + a] - c->vd[3 * q + a];
    }
    double r2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
    double r = sqrt(r2);
    double gw = orc_gradW_coef(r, c->h);             /* grad_p W = gw * x */
    double rp = c->rho[p], rq = c->rho[q];
    double vx = v[0] * x[0] + v[1] * x[1] + v[2] * x[2];
    double fp, fv;
    int pb = kp == ORC_STATIC || kp == ORC_RIGID;
    int qb = c->kind_of[q] == ORC_STATIC || c->kind_of[q] == ORC_RIGID;
    if (c->psi && (pb || qb)) {
        /* volume-based boundary: the fluid side's own pressure and density only */
        if (pb && qb) return;
        double rf = pb ? rq : rp, pf = pb ? c->pres[q] : c->pres[p];
        double w = pb ? c->m[q] * c->psi[p] / c->m[p] : c->psi[q];
        fp = -w * pf / (rf * rf);
        fv = 2.0 * (3 + 2) * P->nu * w * (1.0 / rf) * vx / (r2 + P->visc_eps * c->h * c->h);
        c->gabs += w * fabs(gw) * r;
    } else {
        fp = -c->m[q] * (c->pres[p] / (rp * rp) + c->pres[q] / (rq * rq));
        fv = 2.0 * (3 + 2) * P->nu * c->m[q] * (2.0 / (rp + rq)) * vx
             / (r2 + P->visc_eps * c->h * c->h);
        c->gabs += c->m[q] * fabs(gw) * r;
    }
    for (int a = 0; a < 3; ++a) c->acc[a] += (fp + fv) * gw * x[a];
    c->fabs_sum += fabs(fp + fv) * fabs(gw) * r;
    c->count++;
}

/*
 * One substep from the FP32 state in the current slot order.
 *
 * Inputs: x, v (n x 3, FP32), m (n), id (n) in the current slot order; particles with
 * id < nf are fluid, the others belong to bodies (id ranges [first, first + n)).  Body
 * state B[b] is the state at the start of the substep (a grabbed body carries the pose
 * of this substep's grab path entry).  mode: 0 brute force, 1 uniform grid.
 *
 * Outputs in the sorted order: key, src (current slot of each sorted slot), cell_start
 * (ncell + 1, may be NULL), rho, pres, nnbr, acc (n x 3; total acceleration of fluid and
 * soft particles including gravity; pair force / m for boundary particles), x_new, v_new
 * (n x 3), wrench (nb x 6: force, torque about the grab point), body_new (nb x 13:
 * t, q, v, w after the rigid update), diag (8: sum of pair forces xyz, sum of their
 * magnitudes, momentum of fluid and soft particles after the update xyz, sum |m v|).
 * Returns the number of particles whose cell had to be clamped.
 */
int orc_substep(const orc_params *P, int n, int nf, const float *x, const float *v,
                const float *m, const int *id, int nb, const orc_body *B, int mode,
                uint32_t *key_out, int *src_out, uint32_t *cell_start_out, double *rho,
                double *pres, int *nnbr, double *acc, double *x_new, double *v_new,
                double *wrench, double *body_new, double *diag, double *cond)
{
    const double h = P->h;
    float *xf = (float *)malloc(sizeof(float) * 3 * (size_t)n);
    double *vcur = (double *)malloc(sizeof(double) * 3 * (size_t)n);
    int *body_of_id = (int *)malloc(sizeof(int) * (size_t)n);
    for (int i = 0; i < n; ++i) body_of_id[i] = -1;
    for (int b = 0; b < nb; ++b)
        for (int l = 0; l < B[b].n; ++l) body_of_id[B[b].first + l] = b;

    /* a1: boundary particles of static and rigid bodies follow their body (Sec. 3.2). */
    float *Rf = (float *)malloc(sizeof(float) * 9 * (size_t)(nb > 0 ? nb : 1));
    for (int b = 0; b < nb; ++b) orc_rot_f32(B[b].q, Rf + 9 * b);
    for (int e = 0; e < n; ++e) {
        int b = body_of_id[id[e]];
        if (b >= 0 && B[b].kind == ORC_STATIC) {
            const float *l = B[b].local + 3 * (id[e] - B[b].first);
            for (int a = 0; a < 3; ++a) { xf[3 * e + a] = l[a]; vcur[3 * e + a] = 0.0; }
        } else if (b >= 0 && B[b].kind == ORC_RIGID) {
            const float *l = B[b].local + 3 * (id[e] - B[b].first);
            orc_body_point_f32(Rf + 9 * b, B[b].t, l, xf + 3 * e);
            double r[3], w[3], wr[3];
            for (int a = 0; a < 3; ++a) {
                r[a] = (double)xf[3 * e + a] - (double)B[b].t[a];
                w[a] = B[b].w[a];
            }
            cross3(w, r, wr);
            for (int a = 0; a < 3; ++a) vcur[3 * e + a] = (double)B[b].v[a] + wr[a];
        } else {
            for (int a = 0; a < 3; ++a) {
                xf[3 * e + a] = x[3 * e + a];
                vcur[3 * e + a] = v[3 * e + a];
            }
        }
    }

    /* a2-a4: cell keys, counting sort, sorted index (Alg. 2). */
    int dims[3];
    orc_grid_dims(P, dims);
    int ncell = dims[0] * dims[1] * dims[2];
    uint32_t *key = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n);
    uint32_t *cs = (uint32_t *)malloc(sizeof(uint32_t) * ((size_t)ncell + 1));
    int *src = (int *)malloc(sizeof(int) * (size_t)n);
    int clamped = orc_hash(P, n, xf, key);
    orc_counting_sort(n, key, ncell, cs, src);

    float *xs = (float *)malloc(sizeof(float) * 3 * (size_t)n);
    double *xd = (double *)malloc(sizeof(double) * 3 * (size_t)n);
    double *vd = (double *)malloc(sizeof(double) * 3 * (size_t)n);
    double *ms = (double *)malloc(sizeof(double) * (size_t)n);
    uint32_t *ks = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n);
    int *ids = (int *)malloc(sizeof(int) * (size_t)n);
    int *body_of = (int *)malloc(sizeof(int) * (size_t)n);
    int *kind_of = (int *)malloc(sizeof(int) * (size_t)n);
    int *slot_of_id = (int *)malloc(sizeof(int) * (size_t)n);
    for (int p = 0; p < n; ++p) {
        int e = src[p];
        for (int a = 0; a < 3; ++a) {
            xs[3 * p + a] = xf[3 * e + a];
            xd[3 * p + a] = (double)xf[3 * e + a];
            vd[3 * p + a] = vcur[3 * e + a];
        }
        ms[p] = (double)m[e];
        ks[p] = key[e];
        ids[p] = id[e];
        body_of[p] = body_of_id[id[e]];
        kind_of[p] = body_of[p] >= 0 ? B[body_of[p]].kind : 0;
        slot_of_id[id[e]] = p;
        if (key_out) key_out[p] = key[e];
        if (src_out) src_out[p] = e;
    }
    if (cell_start_out) memcpy(cell_start_out, cs, sizeof(uint32_t) * ((size_t)ncell + 1));

    orc_nbrs N = { mode, n, { dims[0], dims[1], dims[2] }, xs, ks, cs, orc_support2(P), orc_span(P) };

    /* volume-based boundaries: psi_b = rho_0 / sum_{k boundary} W_bk (self included) */
    const int vol = (P->flags & ORC_VOLUME_BOUNDARY) != 0;
    double *psi = vol ? (double *)calloc((size_t)n, sizeof(double)) : NULL;
    if (vol) {
#pragma omp parallel for schedule(dynamic, 256) if (n > 4096)
        for (int p = 0; p < n; ++p) {
            if (!(kind_of[p] == ORC_STATIC || kind_of[p] == ORC_RIGID)) continue;
            orc_pair_ctx c;
            memset(&c, 0, sizeof c);
            c.xd = xd; c.h = h; c.kind_of = kind_of;
            c.rho_sum = orc_W(0.0, h);
            orc_for_neighbours(&N, p, visit_boundary_sum, &c);
            psi[p] = P->rho0 / c.rho_sum;
        }
    }

    /* a6: density (Eq. density, self term included) and pressure (Eq. pressure). */
#pragma omp parallel for schedule(dynamic, 256) if (n > 4096)
    for (int p = 0; p < n; ++p) {
        orc_pair_ctx c;
        memset(&c, 0, sizeof c);
        c.xd = xd; c.m = ms; c.h = h;
        c.kind_of = kind_of; c.psi = psi; c.weight_boundary = vol;
        c.rho_sum = ms[p] * orc_W(0.0, h);
        orc_for_neighbours(&N, p, visit_density, &c);
        rho[p] = c.rho_sum;
        nnbr[p] = c.count;
        if (vol && (kind_of[p] == ORC_STATIC || kind_of[p] == ORC_RIGID)) {
            rho[p] = psi[p];                   /* reported in place of a density */
            pres[p] = 0.0;
            continue;
        }
        double pr = P->k * (c.rho_sum - P->rho0);
        if (P->flags & ORC_TAIT)
            pr = P->k * P->rho0 / ORC_TAIT_GAMMA * (pow(c.rho_sum / P->rho0, ORC_TAIT_GAMMA) - 1.0);
        if ((P->flags & ORC_CLAMP_PRESSURE) && pr < 0.0) pr = 0.0;
        pres[p] = pr;
    }

    /* a5: spring forces of soft bodies (Sec. 3.2), per sorted slot, divided by mass. */
    double *fs = (double *)calloc(3 * (size_t)n, sizeof(double));
    for (int b = 0; b < nb; ++b) {
        if (B[b].kind != ORC_SOFT) continue;
        for (int s = 0; s < B[b].n_springs; ++s) {
            if (B[b].spring_k[s] == 0.0 && B[b].spring_c[s] == 0.0) continue;   /* cut */
            int pa = slot_of_id[B[b].first + B[b].springs[2 * s]];
            int pb = slot_of_id[B[b].first + B[b].springs[2 * s + 1]];
            double d[3], dv[3], L = 0.0, vd_ = 0.0;
            for (int a = 0; a < 3; ++a) {
                d[a] = xd[3 * pa + a] - xd[3 * pb + a];
                dv[a] = vd[3 * pa + a] - vd[3 * pb + a];
                L += d[a] * d[a];
            }
            L = sqrt(L);
            for (int a = 0; a < 3; ++a) { d[a] /= L; vd_ += dv[a] * d[a]; }
            double f = -B[b].spring_k[s] * (L - B[b].spring_L0[s]) - B[b].spring_c[s] * vd_;
            for (int a = 0; a < 3; ++a) {
                fs[3 * pa + a] += f * d[a];
                fs[3 * pb + a] -= f * d[a];
            }
        }
    }

    /* a7: pair forces, acceleration and semi-implicit Euler (Alg. 1, Eq. euler). */
    double dt = P->dt;
#pragma omp parallel for schedule(dynamic, 256) if (n > 4096)
    for (int p = 0; p < n; ++p) {
        orc_pair_ctx c;
        memset(&c, 0, sizeof c);
        c.P = P; c.xd = xd; c.vd = vd; c.m = ms; c.rho = rho; c.pres = pres;
        c.body_of = body_of; c.kind_of = kind_of; c.h = h; c.psi = psi;
        orc_for_neighbours(&N, p, visit_force, &c);
        if (cond) { cond[2 * p] = c.gabs; cond[2 * p + 1] = c.fabs_sum; }
        int kp = kind_of[p];
        for (int a = 0; a < 3; ++a) {
            double ap = c.acc[a] + fs[3 * p + a] / ms[p];
            if (kp == 0 || kp == ORC_SOFT) ap += P->g[a];
            acc[3 * p + a] = ap;
        }
        int pinned = 0;                  /* cloth anchor (Sec. 4): keeps its place, at rest */
        if (kp == ORC_SOFT) {
            const orc_body *bb = &B[body_of[p]];
            pinned = bb->anchored && bb->anchored[ids[p] - bb->first];
        }
        if (pinned) {
            for (int a = 0; a < 3; ++a) {
                v_new[3 * p + a] = 0.0;
                x_new[3 * p + a] = xd[3 * p + a];
            }
        } else if (kp == 0 || kp == ORC_SOFT) {
            for (int a = 0; a < 3; ++a) {
                v_new[3 * p + a] = vd[3 * p + a] + acc[3 * p + a] * dt;
                x_new[3 * p + a] = xd[3 * p + a] + v_new[3 * p + a] * dt;
            }
        } else {
            for (int a = 0; a < 3; ++a) {
                v_new[3 * p + a] = vd[3 * p + a];
                x_new[3 * p + a] = xd[3 * p + a];
            }
        }
    }

    /* diagnostics: pair forces cancel (Newton's third law); fluid and soft momentum. */
    for (int a = 0; a < 8; ++a) diag[a] = 0.0;
    for (int p = 0; p < n; ++p) {
        int kp = kind_of[p];
        double fmag = 0.0, vmag = 0.0;
        for (int a = 0; a < 3; ++a) {
            double f = ms[p] * (acc[3 * p + a] - ((kp == 0 || kp == ORC_SOFT) ? P->g[a] : 0.0))
                       - fs[3 * p + a];
            diag[a] += f;
            fmag += f * f;
        }
        diag[3] += sqrt(fmag);
        if (kp == 0 || kp == ORC_SOFT) {
            for (int a = 0; a < 3; ++a) {
                diag[4 + a] += ms[p] * v_new[3 * p + a];
                vmag += v_new[3 * p + a] * v_new[3 * p + a];
            }
            diag[7] += ms[p] * sqrt(vmag);
        }
    }

    /* a8: wrench on every static and rigid body: F = sum f_b, tau = sum (x - x_g) x f_b. */
    for (int b = 0; b < nb; ++b) {
        double F[3] = { 0, 0, 0 }, T[3] = { 0, 0, 0 };
        double qd[4] = { B[b].q[0], B[b].q[1], B[b].q[2], B[b].q[3] }, Rd[9], xg[3];
        orc_rot_f64(qd, Rd);
        for (int a = 0; a < 3; ++a)
            xg[a] = Rd[3 * a] * B[b].grab_local[0] + Rd[3 * a + 1] * B[b].grab_local[1]
                    + Rd[3 * a + 2] * B[b].grab_local[2] + (double)B[b].t[a];
        if (B[b].kind == ORC_STATIC || B[b].kind == ORC_RIGID) {
            for (int l = 0; l < B[b].n; ++l) {
                int p = slot_of_id[B[b].first + l];
                double f[3], r[3], t[3];
                for (int a = 0; a < 3; ++a) {
                    f[a] = ms[p] * acc[3 * p + a];
                    r[a] = xd[3 * p + a] - xg[a];
                }
                cross3(r, f, t);
                for (int a = 0; a < 3; ++a) { F[a] += f[a]; T[a] += t[a]; }
            }
        }
        for (int a = 0; a < 3; ++a) { wrench[6 * b + a] = F[a]; wrench[6 * b + 3 + a] = T[a]; }

        /* a9: rigid update of free dynamic bodies (Sec. 3.2 point forces -> transform). */
        double *o = body_new + 13 * b;
        for (int a = 0; a < 3; ++a) { o[a] = B[b].t[a]; o[7 + a] = B[b].v[a]; o[10 + a] = B[b].w[a]; }
        for (int a = 0; a < 4; ++a) o[3 + a] = B[b].q[a];
        if (B[b].kind != ORC_RIGID || B[b].grabbed || B[b].mass <= 0.0) continue;
        double M = B[b].mass, vnew[3], arm[3], tc[3], w[3], Iw[9], Iwinv[9], Lw[3], gyro[3];
        for (int a = 0; a < 3; ++a) {
            vnew[a] = (double)B[b].v[a] + (F[a] / M + P->g[a]) * dt;
            o[7 + a] = vnew[a];
            o[a] = (double)B[b].t[a] + vnew[a] * dt;
            arm[a] = xg[a] - (double)B[b].t[a];
            w[a] = B[b].w[a];
        }
        cross3(arm, F, tc);
        for (int a = 0; a < 3; ++a) tc[a] += T[a];           /* torque about the centre */
        /* I_w = R I_b R^T */
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double s = 0.0;
                for (int k = 0; k < 3; ++k)
                    for (int l = 0; l < 3; ++l) s += Rd[3 * i + k] * B[b].inertia[3 * k + l] * Rd[3 * j + l];
                Iw[3 * i + j] = s;
            }
        double det = Iw[0] * (Iw[4] * Iw[8] - Iw[5] * Iw[7]) - Iw[1] * (Iw[3] * Iw[8] - Iw[5] * Iw[6])
                     + Iw[2] * (Iw[3] * Iw[7] - Iw[4] * Iw[6]);
        Iwinv[0] = (Iw[4] * Iw[8] - Iw[5] * Iw[7]) / det;
        Iwinv[1] = (Iw[2] * Iw[7] - Iw[1] * Iw[8]) / det;
        Iwinv[2] = (Iw[1] * Iw[5] - Iw[2] * Iw[4]) / det;
        Iwinv[3] = (Iw[5] * Iw[6] - Iw[3] * Iw[8]) / det;
        Iwinv[4] = (Iw[0] * Iw[8] - Iw[2] * Iw[6]) / det;
        Iwinv[5] = (Iw[2] * Iw[3] - Iw[0] * Iw[5]) / det;
        Iwinv[6] = (Iw[3] * Iw[7] - Iw[4] * Iw[6]) / det;
        Iwinv[7] = (Iw[1] * Iw[6] - Iw[0] * Iw[7]) / det;
        Iwinv[8] = (Iw[0] * Iw[4] - Iw[1] * Iw[3]) / det;
        for (int i = 0; i < 3; ++i) Lw[i] = Iw[3 * i] * w[0] + Iw[3 * i + 1] * w[1] + Iw[3 * i + 2] * w[2];
        cross3(w, Lw, gyro);
        double wn[3];
        for (int i = 0; i < 3; ++i) {
            double s = 0.0;
            for (int j = 0; j < 3; ++j) s += Iwinv[3 * i + j] * (tc[j] - gyro[j]);
            wn[i] = w[i] + s * dt;
            o[10 + i] = wn[i];
        }
        /* q <- normalize(q + dt/2 (0, w) (x) q) */
        double qw = qd[0], qv[3] = { qd[1], qd[2], qd[3] }, wq[3], dq[4];
        cross3(wn, qv, wq);
        dq[0] = -(wn[0] * qv[0] + wn[1] * qv[1] + wn[2] * qv[2]);
        for (int a = 0; a < 3; ++a) dq[1 + a] = qw * wn[a] + wq[a];
        double nq = 0.0, qn[4];
        for (int a = 0; a < 4; ++a) { qn[a] = qd[a] + 0.5 * dt * dq[a]; nq += qn[a] * qn[a]; }
        nq = sqrt(nq);
        for (int a = 0; a < 4; ++a) o[3 + a] = qn[a] / nq;
    }

    free(Rf); free(fs); free(xf); free(vcur); free(body_of_id); free(key); free(cs); free(src);
    free(psi);
    free(xs); free(xd); free(vd); free(ms); free(ks); free(ids); free(body_of); free(kind_of);
    free(slot_of_id);
    return clamped;
}

/* ------------------------------------------------------- haptic smoothing (Sec. 3.3) */

/* Rolling (boxcar) average over the last `window` wrenches: out[t] = mean(in[max(0,t-w+1)..t]). */
void orc_boxcar(int n, int window, const double *in, double *out)
{
    for (int t = 0; t < n; ++t) {
        int lo = t - window + 1;
        if (lo < 0) lo = 0;
        for (int a = 0; a < 6; ++a) {
            double s = 0.0;
            for (int u = lo; u <= t; ++u) s += in[6 * u + a];
            out[6 * t + a] = s / (double)(t - lo + 1);
        }
    }
}

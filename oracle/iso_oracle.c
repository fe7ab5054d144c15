/*
 * iso_oracle.c -- FP64 CPU reference of the fluid isosurface: density field at the corners
 * of a cube grid and its marching-cubes polygonisation (Alg. 2's isosurface compute
 * kernels; Sec. 3.4).  TEST INFRASTRUCTURE ONLY (tests, smoke check, benchmark baseline).
 *
 * Field (Sec. 3.4: density from particle proximity and the smoothing kernel): at corner c,
 * phi(c) = sum over fluid particles j with |c - x_j| < 2h of m_j W(|c - x_j|, h), brute force
 * over all particles, FP64 from the FP32 positions.  Corner (i, j, k) of the grid sits at
 * the FP32 value of origin + (i, j, k) cube.
 *
 * Polygonisation, cube by cube (Sec. 3.4 / marching cubes): corners whose value exceeds
 * the isovalue are inside.  Readings where the paper is silent (listed in the design notes):
 * on a face with two cut edges the surface crosses the face along a segment joining them;
 * on a face with four cut edges each inside corner is cut off by its own segment (the
 * face alone decides, so neighbouring cubes agree and the surface is closed).  The
 * segments close into loops through the cut edges.  Loops are emitted in the order of
 * their smallest edge number, each starting at that edge, first stepping to the smaller of
 * its two neighbours and then reversed if needed so that the loop's normal (Newell's
 * formula over the edge midpoints) points from the inside corners towards the outside
 * corners.  A loop becomes a fan of triangles from its first vertex, unless one of that
 * fan's diagonals would join two vertices lying on a common face of the cube (a loop that
 * crosses an ambiguous face twice): such a diagonal could coincide with one drawn by the
 * neighbouring cube, so that loop is fanned from an added centre vertex instead, the mean
 * of its vertices, with one triangle per loop side.  Vertices are linearly interpolated
 * on the cut edges.
 *
 * Numbering: corner v at offset (v & 1, v >> 1 & 1, v >> 2 & 1); the edge between corners
 * differing in bit `axis` is 4 axis + (the two other bits, the lower axis first).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

double orc_W(double r, double h);   /* sph_oracle.c */

void orc_iso_field(int n, const float *x, const double *m, const int *is_fluid, double h,
                   const int dims[3], const float origin[3], float cube, double *out)
{
    const double R = 2.0 * h;
    const long long nv = (long long)dims[0] * dims[1] * dims[2];
#pragma omp parallel for schedule(dynamic, 64) if (nv > 4096)
    for (long long v = 0; v < nv; ++v) {
        const int i = (int)(v % dims[0]), j = (int)((v / dims[0]) % dims[1]);
        const int k = (int)(v / ((long long)dims[0] * dims[1]));
        const int ijk[3] = { i, j, k };
        double c[3];
        for (int a = 0; a < 3; ++a) c[a] = (double)(float)((double)origin[a] + (double)ijk[a] * (double)cube);
        double s = 0.0;
        for (int p = 0; p < n; ++p) {
            if (!is_fluid[p]) continue;
            double d0 = (double)x[3 * p] - c[0], d1 = (double)x[3 * p + 1] - c[1], d2 = (double)x[3 * p + 2] - c[2];
            double r = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
            if (r < R) s += m[p] * orc_W(r, h);
        }
        out[v] = s;
    }
}

/* corners of edge e (lower first) */
static void edge_corners(int e, int *a, int *b)
{
    int axis = e / 4, idx = e % 4;
    int lo_bit = axis == 0 ? 1 : 0;          /* the lower of the two other axes */
    int hi_bit = axis == 2 ? 1 : 2;
    *a = ((idx & 1) << lo_bit) | (((idx >> 1) & 1) << hi_bit);
    *b = *a | (1 << axis);
}

static int edge_of(int a, int b)
{
    int d = a ^ b, axis = d == 1 ? 0 : d == 2 ? 1 : 2;
    int lo = a < b ? a : b;
    int lo_bit = axis == 0 ? 1 : 0, hi_bit = axis == 2 ? 1 : 2;
    return 4 * axis + ((lo >> lo_bit) & 1) + 2 * ((lo >> hi_bit) & 1);
}

/* is edge e on face f (f = 2 axis + side)? */
static int on_face(int e, int f)
{
    int a, b;
    edge_corners(e, &a, &b);
    int axis = f / 2, side = f % 2;
    return ((a >> axis) & 1) == side && ((b >> axis) & 1) == side;
}

static int share_face(int e1, int e2)
{
    for (int f = 0; f < 6; ++f)
        if (on_face(e1, f) && on_face(e2, f)) return 1;
    return 0;
}

/* Triangles of one cube as edge triples (edge -1 = the loop's centre vertex, whose loop
 * is given in tri_loop); loops are written to loops/loop_len.  Returns the triangle count. */
static int cube_triangles(const int inside[8], int tri[][3], int tri_loop[], int loops[][12],
                          int loop_len[], int *nloops)
{
    /* the six faces, corners in cyclic order around the face */
    static const int face[6][4] = {
        { 0, 2, 6, 4 }, { 1, 3, 7, 5 },      /* x = 0, x = 1 */
        { 0, 1, 5, 4 }, { 2, 3, 7, 6 },      /* y = 0, y = 1 */
        { 0, 1, 3, 2 }, { 4, 5, 7, 6 },      /* z = 0, z = 1 */
    };
    int cut[12], link[12][2], nlink[12];
    for (int e = 0; e < 12; ++e) {
        int a, b;
        edge_corners(e, &a, &b);
        cut[e] = inside[a] != inside[b];
        nlink[e] = 0;
    }
    for (int f = 0; f < 6; ++f) {
        int fe[4], ncut = 0, cuts[4];
        for (int s = 0; s < 4; ++s) {
            fe[s] = edge_of(face[f][s], face[f][(s + 1) % 4]);   /* side s: corner s to s+1 */
            if (cut[fe[s]]) cuts[ncut++] = fe[s];
        }
        if (ncut == 2) {
            link[cuts[0]][nlink[cuts[0]]++] = cuts[1];
            link[cuts[1]][nlink[cuts[1]]++] = cuts[0];
        } else if (ncut == 4) {
            for (int s = 0; s < 4; ++s) {
                if (!inside[face[f][s]]) continue;
                int e1 = fe[(s + 3) % 4], e2 = fe[s];              /* the sides at corner s */
                link[e1][nlink[e1]++] = e2;
                link[e2][nlink[e2]++] = e1;
            }
        }
    }
    int done[12] = { 0 }, nt = 0;
    for (int start = 0; start < 12; ++start) {
        if (!cut[start] || done[start]) continue;
        int loop[12], len = 0, prev = -1, cur = start;
        for (;;) {
            loop[len++] = cur;
            done[cur] = 1;
            int nx;
            if (prev < 0) nx = link[cur][0] < link[cur][1] ? link[cur][0] : link[cur][1];
            else nx = link[cur][0] == prev ? link[cur][1] : link[cur][0];
            prev = cur;
            cur = nx;
            if (cur == start) break;
        }
        double N[3] = { 0, 0, 0 }, O[3] = { 0, 0, 0 };
        for (int s = 0; s < len; ++s) {
            int a, b, c, d;
            edge_corners(loop[s], &a, &b);
            edge_corners(loop[(s + 1) % len], &c, &d);
            double p[3], q[3];
            for (int ax = 0; ax < 3; ++ax) {
                p[ax] = 0.5 * (((a >> ax) & 1) + ((b >> ax) & 1));
                q[ax] = 0.5 * (((c >> ax) & 1) + ((d >> ax) & 1));
            }
            N[0] += (p[1] - q[1]) * (p[2] + q[2]);
            N[1] += (p[2] - q[2]) * (p[0] + q[0]);
            N[2] += (p[0] - q[0]) * (p[1] + q[1]);
            int vin = inside[a] ? a : b, vout = inside[a] ? b : a;
            for (int ax = 0; ax < 3; ++ax) O[ax] += (double)((vout >> ax) & 1) - (double)((vin >> ax) & 1);
        }
        if (N[0] * O[0] + N[1] * O[1] + N[2] * O[2] < 0.0) {
            int rev[12];
            rev[0] = loop[0];
            for (int s = 1; s < len; ++s) rev[s] = loop[len - s];
            memcpy(loop, rev, sizeof(int) * (size_t)len);
        }
        int li = (*nloops)++;
        memcpy(loops[li], loop, sizeof(int) * (size_t)len);
        loop_len[li] = len;
        int centre = 0;
        for (int s = 2; s + 1 < len; ++s)
            if (share_face(loop[0], loop[s])) centre = 1;
        if (!centre) {
            for (int s = 1; s + 1 < len; ++s) {
                tri[nt][0] = loop[0];
                tri[nt][1] = loop[s];
                tri[nt][2] = loop[s + 1];
                tri_loop[nt] = li;
                ++nt;
            }
        } else {
            for (int s = 0; s < len; ++s) {
                tri[nt][0] = -1;
                tri[nt][1] = loop[s];
                tri[nt][2] = loop[(s + 1) % len];
                tri_loop[nt] = li;
                ++nt;
            }
        }
    }
    return nt;
}

/*
 * Marching cubes over field (dims corners, x fastest).  Writes up to max_tris triangles:
 * xyz (9 doubles each) and, per vertex, the global id of its cube edge
 * 3 * (linear index of the edge's lower corner) + axis (3 int64 each).  Returns the total.
 */
long long orc_iso_polygonize(const double *field, const int dims[3], const double origin[3],
                             double cube, double iso, long long max_tris, double *xyz,
                             long long *vid)
{
    const int nx = dims[0], ny = dims[1], nz = dims[2];
    long long total = 0;
    for (int k = 0; k + 1 < nz; ++k)
        for (int j = 0; j + 1 < ny; ++j)
            for (int i = 0; i + 1 < nx; ++i) {
                double phi[8];
                int inside[8], any_in = 0, any_out = 0;
                for (int v = 0; v < 8; ++v) {
                    int ci = i + (v & 1), cj = j + ((v >> 1) & 1), ck = k + ((v >> 2) & 1);
                    phi[v] = field[((long long)ck * ny + cj) * nx + ci];
                    inside[v] = phi[v] > iso;
                    any_in |= inside[v];
                    any_out |= !inside[v];
                }
                if (!any_in || !any_out) continue;
                int tri[16][3], tri_loop[16], loops[6][12], loop_len[6], nloops = 0;
                int nt = cube_triangles(inside, tri, tri_loop, loops, loop_len, &nloops);
                /* vertex of every cut edge, and the centre of every loop */
                double vx[12][3], cx[6][3];
                long long ev[12];
                for (int e = 0; e < 12; ++e) {
                    int a, b;
                    edge_corners(e, &a, &b);
                    if (inside[a] == inside[b]) continue;
                    int axis = e / 4;
                    double u = (iso - phi[a]) / (phi[b] - phi[a]);
                    int ca[3] = { i + (a & 1), j + ((a >> 1) & 1), k + ((a >> 2) & 1) };
                    for (int ax = 0; ax < 3; ++ax) {
                        double base = origin[ax] + (double)ca[ax] * cube;
                        vx[e][ax] = ax == axis ? base + u * cube : base;
                    }
                    ev[e] = 3 * (((long long)ca[2] * ny + ca[1]) * nx + ca[0]) + axis;
                }
                for (int l = 0; l < nloops; ++l)
                    for (int ax = 0; ax < 3; ++ax) {
                        double sum = 0.0;
                        for (int s = 0; s < loop_len[l]; ++s) sum += vx[loops[l][s]][ax];
                        cx[l][ax] = sum / loop_len[l];
                    }
                const long long ncorner = (long long)nx * ny * nz;
                const long long cube_id = ((long long)k * ny + j) * nx + i;
                for (int t = 0; t < nt; ++t, ++total) {
                    if (total >= max_tris) continue;
                    for (int s = 0; s < 3; ++s) {
                        int e = tri[t][s];
                        const double *p = e >= 0 ? vx[e] : cx[tri_loop[t]];
                        for (int ax = 0; ax < 3; ++ax) xyz[9 * total + 3 * s + ax] = p[ax];
                        /* centre vertices: ids after all edge ids, one per (cube, loop) */
                        vid[3 * total + s] = e >= 0 ? ev[e] : 3 * ncorner + 6 * cube_id + tri_loop[t];
                    }
                }
            }
    return total;
}

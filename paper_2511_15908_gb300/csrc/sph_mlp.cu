// sph_mlp.cu -- the learned haptic-rate wrench surrogate: a 269-128-128-128-6 GELU MLP with
// BF16 weights and FP32 accumulation on tcgen05 tensor cores, trained on the GPU by these
// kernels (forward, backward, Adam), and the pooled local descriptor it reads from the SPH
// state.  The exact FP64 coupling reduction of the substep stays the fallback and reference.
//
// Parameters (FP32 master copy, logical layout, 68,358 values):
//   W1[128][269] b1[128] W2[128][128] b2[128] W3[128][128] b3[128] W4[6][128] b4[6]
// The GEMMs read zero-padded BF16 copies W1b[128][272], W2b, W3b[128][128], W4b[16][128] and,
// for the backward pass, their transposes W2t, W3t[128][128], W4t[128][16]: every GEMM operand
// is K-contiguous, as the TMA-fed tensor-core GEMM wants.  For the same reason the forward and
// backward passes also write column-major copies ([feature][batch], leading dimension the
// batch capacity rounded up to 8) of the activations and gradients the weight gradients
// contract over the batch.  The weight gradients are split over kSplit K slices (batch
// ranges) and summed, slice by slice in a fixed order, when the gradient vector is gathered.
// Inputs are standardised ((x - mean) / std) and outputs de-standardised in the kernels.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "sph.h"
#include "sph_device.cuh"
#include "tc_gemm.cuh"
#include "tc_ptx.cuh"

namespace sphgb {

constexpr int kIn = 269, kInPad = 272, kHid = 128, kOut = 6, kOutPad = 16;
constexpr int kSplit = 8;      // K slices of a weight-gradient GEMM (at most)
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kHid * kIn, kOffW2 = kOffB1 + kHid,
              kOffB2 = kOffW2 + kHid * kHid, kOffW3 = kOffB2 + kHid, kOffB3 = kOffW3 + kHid * kHid,
              kOffW4 = kOffB3 + kHid, kOffB4 = kOffW4 + kOut * kHid, kParams = kOffB4 + kOut;
static_assert(kParams == 68358, "parameter count");

// ------------------------------------------------------------------ small kernels

__global__ void k_refresh_bf16(const float *master, __nv_bfloat16 *w1, __nv_bfloat16 *w2,
                               __nv_bfloat16 *w3, __nv_bfloat16 *w4, float *b4pad, __nv_bfloat16 *w2t,
                               __nv_bfloat16 *w3t, __nv_bfloat16 *w4t)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < kHid * kInPad) {
        int r = t / kInPad, c = t % kInPad;
        w1[t] = __float2bfloat16_rn(c < kIn ? master[kOffW1 + r * kIn + c] : 0.0f);
    }
    if (t < kHid * kHid) {
        w2[t] = __float2bfloat16_rn(master[kOffW2 + t]);
        w3[t] = __float2bfloat16_rn(master[kOffW3 + t]);
        const int i = t / kHid, o = t % kHid;          // transposes: [input][output]
        w2t[t] = __float2bfloat16_rn(master[kOffW2 + o * kHid + i]);
        w3t[t] = __float2bfloat16_rn(master[kOffW3 + o * kHid + i]);
    }
    if (t < kOutPad * kHid) {
        int r = t / kHid;
        w4[t] = __float2bfloat16_rn(r < kOut ? master[kOffW4 + t] : 0.0f);
        const int i = t / kOutPad, o = t % kOutPad;    // W4t[hidden][output]
        w4t[t] = __float2bfloat16_rn(o < kOut ? master[kOffW4 + o * kHid + i] : 0.0f);
    }
    if (t < kOutPad) b4pad[t] = t < kOut ? master[kOffB4 + t] : 0.0f;
}

// Standardised BF16 input rows xb[b][c] (zero-padded to 272 columns) and, when xbT is given,
// the column-major copy xbT[c][b]: a 32 x 32 tile per block, transposed through shared memory
// so that both copies are written along their contiguous dimension.
__global__ void k_prep_input(const float *x, int B, const float *mean, const float *inv_std,
                             __nv_bfloat16 *xb, __nv_bfloat16 *xbT, int ldt)
{
    __shared__ __nv_bfloat16 tile[32][33];
    const int c0 = blockIdx.x * 32, b0 = blockIdx.y * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;
    for (int r = ty; r < 32; r += blockDim.y) {
        const int b = b0 + r, c = c0 + tx;
        if (b < B && c < kInPad) {
            const float v = c < kIn ? (x[(size_t)b * kIn + c] - mean[c]) * inv_std[c] : 0.0f;
            const __nv_bfloat16 h = __float2bfloat16_rn(v);
            xb[(size_t)b * kInPad + c] = h;
            tile[r][tx] = h;
        }
    }
    if (!xbT) return;
    __syncthreads();
    for (int r = ty; r < 32; r += blockDim.y) {
        const int c = c0 + r, b = b0 + tx;
        if (b < B && c < kInPad) xbT[(size_t)c * ldt + b] = tile[tx][r];
    }
}

__global__ void k_output(const float *y, int B, const float *mean, const float *std_, float *out)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= B * kOut) return;
    int b = t / kOut, j = t % kOut;
    out[t] = y[(size_t)b * kOutPad + j] * std_[j] + mean[j];
}

// MSE on standardised outputs: L = mean over B x 6 of (y - tn)^2; dY = 2 (y - tn) / (6 B),
// written row-major (the A operand of dZ3 = dY W4) and column-major (the B operand of dW4)
// in BF16.  One element per thread (16 rows of 16 columns per block); each block writes its
// FP64 share of the squared error and its FP32 column sums of the unrounded dY (the bias
// gradient db4), both added in a fixed order here and, block by block, by the gather.
constexpr int kLossThreads = 256;
__global__ void k_loss_grad(const float *y, const float *t, int B, const float *mean, const float *inv_std,
                            __nv_bfloat16 *dyb, __nv_bfloat16 *dybT, int ldt, double *loss_part, float *db4_part)
{
    __shared__ double s[kLossThreads];
    __shared__ float sg[kLossThreads];
    const int i = blockIdx.x * kLossThreads + threadIdx.x;
    double acc = 0.0;
    if (i < B * kOutPad) {
        const int b = i / kOutPad, j = i % kOutPad;
        float g = 0.0f;
        if (j < kOut) {
            const float tn = (t[(size_t)b * kOut + j] - mean[j]) * inv_std[j];
            const float d = y[i] - tn;
            acc = (double)d * d;
            g = 2.0f * d / (float)(kOut * B);
        }
        const __nv_bfloat16 h = __float2bfloat16_rn(g);
        dyb[i] = h;
        dybT[(size_t)j * ldt + b] = h;
        sg[threadIdx.x] = g;
    } else {
        sg[threadIdx.x] = 0.0f;
    }
    s[threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.x < kOutPad) {               // column j = threadIdx.x of the block's 16 rows
        float c = 0.0f;
        for (int r = 0; r < kLossThreads / kOutPad; ++r) c += sg[r * kOutPad + threadIdx.x];
        db4_part[(size_t)blockIdx.x * kOutPad + threadIdx.x] = c;
    }
    for (int st = kLossThreads / 2; st > 0; st >>= 1) {
        if ((int)threadIdx.x < st) s[threadIdx.x] += s[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) loss_part[blockIdx.x] = s[0];
}

// Where the gather finds the gradients: the weight-gradient GEMMs' K-slice partials
// (dW1 [128][272], dW2, dW3 [128][128], dW4^T [128][16] per slice) and the bias-gradient
// partials, per 128-row tile of the dZ GEMMs (column sums of the unrounded dZ, [tile][128])
// and per block of the loss kernel (dY, [block][16]).
struct GradSrc {
    const float *dW1, *dW2, *dW3, *dW4t;
    int slices;
    const float *db1, *db2, *db3;
    int tiles;
    const float *db4;
    int blocks;
};

// Gradient of logical parameter t: its partials summed in order.
__device__ __forceinline__ float grad_of(const GradSrc &g, int t)
{
    const float *p;
    size_t idx, stride;
    int n;
    if (t < kOffB1) {
        p = g.dW1; idx = (size_t)(t / kIn) * kInPad + t % kIn; stride = (size_t)kHid * kInPad; n = g.slices;
    } else if (t < kOffW2) {
        p = g.db1; idx = t - kOffB1; stride = kHid; n = g.tiles;
    } else if (t < kOffB2) {
        p = g.dW2; idx = t - kOffW2; stride = (size_t)kHid * kHid; n = g.slices;
    } else if (t < kOffW3) {
        p = g.db2; idx = t - kOffB2; stride = kHid; n = g.tiles;
    } else if (t < kOffB3) {
        p = g.dW3; idx = t - kOffW3; stride = (size_t)kHid * kHid; n = g.slices;
    } else if (t < kOffW4) {
        p = g.db3; idx = t - kOffB3; stride = kHid; n = g.tiles;
    } else if (t < kOffB4) {
        const int q = t - kOffW4;
        p = g.dW4t; idx = (size_t)(q % kHid) * kOutPad + q / kHid; stride = (size_t)kHid * kOutPad; n = g.slices;
    } else {
        p = g.db4; idx = t - kOffB4; stride = kOutPad; n = g.blocks;
    }
    float v = 0.0f;
    for (int k = 0; k < n; ++k) v += p[k * stride + idx];
    return v;
}

__device__ __forceinline__ void finish_loss(const double *loss_part, int nblk, int B, double *loss)
{
    double l = 0.0;
    for (int k = 0; k < nblk; ++k) l += loss_part[k];
    *loss = l / (double)(kOut * B);
}

// The logical gradient vector (and the loss).
__global__ void k_gather_grads(GradSrc src, float *grad, const double *loss_part, int nblk, int B, double *loss)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t == 0) finish_loss(loss_part, nblk, B, loss);
    if (t < kParams) grad[t] = grad_of(src, t);
}

// BF16 images of the updated weight value w of logical parameter t (biases 1-3 are read
// from the FP32 master copy; the zero padding never changes)
struct Images {
    __nv_bfloat16 *w1, *w2, *w3, *w4, *w2t, *w3t, *w4t;
    float *b4pad;
};
__device__ __forceinline__ void write_images(const Images &im, int t, float w)
{
    const __nv_bfloat16 h = __float2bfloat16_rn(w);
    if (t < kOffB1) {
        im.w1[(t / kIn) * kInPad + t % kIn] = h;
    } else if (t >= kOffW2 && t < kOffB2) {
        const int q = t - kOffW2;
        im.w2[q] = h;
        im.w2t[(q % kHid) * kHid + q / kHid] = h;
    } else if (t >= kOffW3 && t < kOffB3) {
        const int q = t - kOffW3;
        im.w3[q] = h;
        im.w3t[(q % kHid) * kHid + q / kHid] = h;
    } else if (t >= kOffW4 && t < kOffB4) {
        const int q = t - kOffW4;
        im.w4[q] = h;
        im.w4t[(q % kHid) * kOutPad + q / kHid] = h;
    } else if (t >= kOffB4) {
        im.b4pad[t - kOffB4] = w;
    }
}

// One training update per parameter: gather its gradient, take the Adam step on the FP32
// master copy and refresh the BF16 images the next forward pass reads.
__global__ void k_train_update(GradSrc src, float *w, float *m, float *v, float *grad, float lr, float b1, float b2,
                               float eps, float c1, float c2, Images im, const double *loss_part, int nblk, int B,
                               double *loss)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t == 0) finish_loss(loss_part, nblk, B, loss);
    if (t >= kParams) return;
    const float gi = grad_of(src, t);
    grad[t] = gi;
    const float mi = b1 * m[t] + (1.0f - b1) * gi;
    const float vi = b2 * v[t] + (1.0f - b2) * gi * gi;
    m[t] = mi;
    v[t] = vi;
    const float wn = w[t] - lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    w[t] = wn;
    write_images(im, t, wn);
}

// ------------------------------------------------------------- pooled descriptor

// Surrogate input for the grabbed body: pose (x 3, q 4) and velocity (v 3, w 3) of the
// substep's pose, then a 4 x 4 x 4 grid of cells of edge R = 2h centred on the grab point;
// per cell (x fastest) the mean density of the fluid particles inside and their
// mass-weighted mean velocity (zeros for an empty cell).  One warp per descriptor cell:
// the lanes stride over the grid cells that overlap it, then a fixed shuffle tree sums
// their partials (deterministic).
__global__ void __launch_bounds__(256) k_descriptor(SimConst c, int grab_body, float *out)
{
    const int cell = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);   // 0..63
    const int lane = threadIdx.x & 31;
    if (cell >= 64) return;
    const DevBody &B = c.body[grab_body];
    Pose P = body_pose(c, B, c.ctr[0] > 0 ? c.ctr[0] - 1u : 0u);
    double R9[9], xg[3];
    grab_point(P, B, xg, R9);
    const float Rs = 2.0f * c.h;
    const int ci = cell & 3, cj = (cell >> 2) & 3, ck = cell >> 4;
    const float lo[3] = {(float)xg[0] + (ci - 2) * Rs, (float)xg[1] + (cj - 2) * Rs, (float)xg[2] + (ck - 2) * Rs};
    const float hi[3] = {lo[0] + Rs, lo[1] + Rs, lo[2] + Rs};
    uint32_t bad = 0;
    int g0[3], g1[3];
    for (int a = 0; a < 3; ++a) {
        const int n = a == 0 ? c.nx : (a == 1 ? c.ny : c.nz);
        g0[a] = cell_axis(lo[a], c.o[a], c.inv_cell, n, bad);
        g1[a] = cell_axis(hi[a], c.o[a], c.inv_cell, n, bad);
    }
    float sr = 0.0f, sm = 0.0f, svx = 0.0f, svy = 0.0f, svz = 0.0f;
    int cnt = 0;
    for (int z = g0[2]; z <= g1[2]; ++z)
        for (int y = g0[1]; y <= g1[1]; ++y) {
            const int base = (z * c.ny + y) * c.nx;
            const int s = (int)c.cell_start[base + g0[0]], e = (int)c.cell_start[base + g1[0] + 1];
            for (int q = s + lane; q < e; q += 32) {
                const float4 x = c.xA[q];
                const float4 v = c.vA[q];
                if (__float_as_int(v.w) >= c.nf) continue;          // fluid particles only
                if (x.x < lo[0] || x.x >= hi[0] || x.y < lo[1] || x.y >= hi[1] || x.z < lo[2] || x.z >= hi[2])
                    continue;
                const float m = fabsf(x.w);
                sr += c.prho[q].x;
                sm += m;
                svx += m * v.x; svy += m * v.y; svz += m * v.z;
                ++cnt;
            }
        }
    sr = warp_sum(sr);
    sm = warp_sum(sm);
    svx = warp_sum(svx);
    svy = warp_sum(svy);
    svz = warp_sum(svz);
    cnt = warp_sum(cnt);
    if (lane == 0) {
        float *d = out + 13 + 4 * cell;
        d[0] = cnt ? sr / (float)cnt : 0.0f;
        d[1] = sm > 0.0f ? svx / sm : 0.0f;
        d[2] = sm > 0.0f ? svy / sm : 0.0f;
        d[3] = sm > 0.0f ? svz / sm : 0.0f;
        if (cell == 0) {
            for (int a = 0; a < 3; ++a) { out[a] = P.t[a]; out[7 + a] = P.v[a]; out[10 + a] = P.w[a]; }
            for (int a = 0; a < 4; ++a) out[3 + a] = P.q[a];
        }
    }
}

cudaError_t launch_descriptor(const SimConst &c, cudaStream_t s, int grab_body, float *d_out)
{
    k_descriptor<<<8, 256, 0, s>>>(c, grab_body, d_out);
    return cudaGetLastError();
}

// ------------------------------------------------------ scale-free tick inputs

// The scene's scales: smoothing length h, sound speed c = sqrt(k) (the pressure constant of
// Eq. pressure is c^2), rest density rho0.  Lengths are measured in h, velocities in c,
// times in h / c, densities as rho / rho0 - 1, forces in rho0 c^2 h^2 and torques in
// rho0 c^2 h^3, so that one network can read scenes of different resolution and body size.
struct SurScale {
    float h, c, rho0;
};

// R(q)^T v for q = (w, x, y, z) (the anchor's body frame), FP32.
__device__ __forceinline__ void rot_t_apply(const float q[4], const float v[3], float o[3])
{
    const float w = q[0], x = q[1], y = q[2], z = q[3];
    const float R[9] = {1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y),
                        2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
                        2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)};
    for (int i = 0; i < 3; ++i) o[i] = R[i] * v[0] + R[3 + i] * v[1] + R[6 + i] * v[2];
}

// The 269 network inputs of one tick.  t13: the grab pose and velocity at the tick (x y z
// qw qx qy qz vx vy vz wx wy wz); a: the anchor's descriptor (sph_get_descriptor: the same 13
// values at the anchor substep, then 64 cells x (density, velocity)); tau: time since the
// anchor.  Output: R_a^T (x - x_a) / h, tau c / h, R_a^T (v - v_a) / c, R_a^T v / c,
// R_a^T w h / c, then per cell rho / rho0 - 1 (-1 for an empty cell) and R_a^T v_cell / c.
__device__ __forceinline__ void sur_features(const float *t13, const float *a, float tau,
                                             const SurScale &s, float *out)
{
    const float ih = 1.0f / s.h, ic = 1.0f / s.c, irho = 1.0f / s.rho0;
    const float qa[4] = {a[3], a[4], a[5], a[6]};
    float d[3], o[3];
    for (int i = 0; i < 3; ++i) d[i] = (t13[i] - a[i]) * ih;
    rot_t_apply(qa, d, o);
    for (int i = 0; i < 3; ++i) out[i] = o[i];
    out[3] = tau * s.c * ih;
    for (int i = 0; i < 3; ++i) d[i] = (t13[7 + i] - a[7 + i]) * ic;
    rot_t_apply(qa, d, o);
    for (int i = 0; i < 3; ++i) out[4 + i] = o[i];
    for (int i = 0; i < 3; ++i) d[i] = t13[7 + i] * ic;
    rot_t_apply(qa, d, o);
    for (int i = 0; i < 3; ++i) out[7 + i] = o[i];
    for (int i = 0; i < 3; ++i) d[i] = t13[10 + i] * s.h * ic;
    rot_t_apply(qa, d, o);
    for (int i = 0; i < 3; ++i) out[10 + i] = o[i];
    for (int k = 0; k < 64; ++k) {
        const float *cell = a + 13 + 4 * k;
        out[13 + 4 * k] = cell[0] * irho - 1.0f;
        for (int i = 0; i < 3; ++i) d[i] = cell[1 + i] * ic;
        rot_t_apply(qa, d, o);
        for (int i = 0; i < 3; ++i) out[14 + 4 * k + i] = o[i];
    }
}

// One row per thread: ticks (stride tick_stride floats), anchors (stride anchor_stride),
// times since the anchor; out n x 269.
__global__ void k_sur_features(const float *ticks, int tick_stride, const float *anchors,
                               int anchor_stride, const float *taus, int n, SurScale s, float *out)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    sur_features(ticks + (size_t)r * tick_stride, anchors + (size_t)r * anchor_stride, taus[r], s,
                 out + (size_t)r * 269);
}

// Training targets: the wrench change since the anchor in the anchor's body frame, in the
// force and torque scales (FP64 difference, then FP32).
__global__ void k_sur_targets(const double *w, const double *wa, const float *anchors, int anchor_stride,
                              int n, SurScale s, float *out)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const float *a = anchors + (size_t)r * anchor_stride;
    const float qa[4] = {a[3], a[4], a[5], a[6]};
    const double fs = (double)s.rho0 * s.c * s.c * s.h * s.h;
    for (int part = 0; part < 2; ++part) {
        const double sc = part == 0 ? fs : fs * s.h;
        float d[3], o[3];
        for (int i = 0; i < 3; ++i)
            d[i] = (float)((w[(size_t)r * 6 + 3 * part + i] - wa[(size_t)r * 6 + 3 * part + i]) / sc);
        rot_t_apply(qa, d, o);
        for (int i = 0; i < 3; ++i) out[(size_t)r * 6 + 3 * part + i] = o[i];
    }
}

// The tick's inputs from its pose and velocity (kernel arguments) and the stored anchor.
__global__ void k_sur_tick_features(float t0, float t1, float t2, float t3, float t4, float t5, float t6,
                                    float t7, float t8, float t9, float t10, float t11, float t12,
                                    float tau, const float *anchor, SurScale s, float *out)
{
    if (threadIdx.x != 0) return;
    const float t13[13] = {t0, t1, t2, t3, t4, t5, t6, t7, t8, t9, t10, t11, t12};
    sur_features(t13, anchor, tau, s, out);
}

// The tick's wrench: the anchor's exact FP64 wrench plus the network's correction, taken out
// of the standardised, scale-free, body-frame output.
__device__ __forceinline__ void tick_output(const float *y, const float *ymean, const float *ystd,
                                            const float *anchor, const double *wa, const SurScale &s, double *out)
{
    const float qa[4] = {anchor[3], anchor[4], anchor[5], anchor[6]};
    const float w = qa[0], x = qa[1], yq = qa[2], z = qa[3];
    const float R[9] = {1 - 2 * (yq * yq + z * z), 2 * (x * yq - w * z), 2 * (x * z + w * yq),
                        2 * (x * yq + w * z), 1 - 2 * (x * x + z * z), 2 * (yq * z - w * x),
                        2 * (x * z - w * yq), 2 * (yq * z + w * x), 1 - 2 * (x * x + yq * yq)};
    const double fs = (double)s.rho0 * s.c * s.c * s.h * s.h;
    for (int part = 0; part < 2; ++part) {
        const double sc = part == 0 ? fs : fs * s.h;
        float b[3];
        for (int i = 0; i < 3; ++i) b[i] = y[3 * part + i] * ystd[3 * part + i] + ymean[3 * part + i];
        for (int i = 0; i < 3; ++i) {
            const float wv = R[3 * i] * b[0] + R[3 * i + 1] * b[1] + R[3 * i + 2] * b[2];
            out[3 * part + i] = wa[3 * part + i] + (double)wv * sc;
        }
    }
}

__global__ void k_sur_tick_output(const float *y, const float *ymean, const float *ystd, const float *anchor,
                                  const double *wa, SurScale s, double *out)
{
    if (threadIdx.x == 0) tick_output(y, ymean, ystd, anchor, wa, s, out);
}

// The whole haptic tick in one CTA of 128 threads: the tick's 269 inputs, the four layers as
// tcgen05 MMAs with the activations kept on chip, and the wrench.  The input row sits in
// row 0 of a 128-row BF16 A tile in shared memory (the other rows are zero), written in the
// K-major 128-byte-swizzled layout the MMA descriptors expect (row 0 is not permuted by the
// swizzle); each layer's weights arrive by TMA (the GEMM's tensor maps: 64-wide K chunks,
// zero past K), the MMAs accumulate into TMEM, and the accumulator's row 0 (TMEM lane 0)
// goes through the layer's bias and GELU, rounded to BF16, into the A tile for the next
// layer.  The rounding points and operations are those of sph_mlp_forward; the result is
// the anchor's wrench plus the de-standardised, rotated correction.
struct TickArgs {
    float t13[13];
    float tau;
    const float *anchor;
    SurScale s;
    const float *xmean, *xinv, *ymean, *ystd;
    const float *b1, *b2, *b3, *b4;
    const double *wa;
    double *out;
    unsigned *status;
};
constexpr int kTickChunk = kTcM * kTcKChunk * 2;              // one K chunk of a 128-row tile
// A tile (5 chunks), W1 (5 chunks; W3 reuses it once layer 1 is done), W2 (2), W4 (2 chunks
// of 16 rows), alignment, barriers
constexpr int kTickW4 = kOutPad * kTcKChunk * 2;
constexpr int kTickSmem = (5 + 5 + 2) * kTickChunk + 2 * kTickW4 + 1024 + 64;

__global__ void __launch_bounds__(128, 1)
    k_sur_tick_fused(const __grid_constant__ CUtensorMap m1, const __grid_constant__ CUtensorMap m2,
                     const __grid_constant__ CUtensorMap m3, const __grid_constant__ CUtensorMap m4, TickArgs a)
{
    using namespace tcx;
    extern __shared__ unsigned char smem_raw[];
    __shared__ float s_v[kInPad];                 // the features, then each layer's row
    __shared__ uint32_t s_tmem;
    __shared__ int s_fail;
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t A = (raw + 1023u) & ~1023u, W1 = A + 5u * kTickChunk, W2 = W1 + 5u * kTickChunk;
    const uint32_t W4 = W2 + 2u * kTickChunk, bar = W4 + 2u * kTickW4;
    // full[l]: layer l's weights have landed (one phase each); done: a layer's MMAs completed
    const uint32_t done = bar + 32u;
    auto full = [&](int l) { return bar + 8u * (uint32_t)l; };
    unsigned char *Ap = smem_raw + (A - raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // element k of row 0 of the A tile: chunk k / 64, byte 2 (k % 64) of the row
    auto put = [&](int k, float v) {
        *reinterpret_cast<__nv_bfloat16 *>(Ap + (size_t)(k >> 6) * kTickChunk + 2 * (k & 63)) = __float2bfloat16_rn(v);
    };
    // rows 1-127 of the A tile are never written: they only feed rows 1-127 of the
    // accumulator, which nothing reads
    const CUtensorMap *maps[4] = {&m1, &m2, &m3, &m4};
    const int nk[4] = {(kInPad + kTcKChunk - 1) / kTcKChunk, kHid / kTcKChunk, kHid / kTcKChunk, kHid / kTcKChunk};
    const int nn[4] = {kHid, kHid, kHid, kOutPad};
    const uint32_t wbase[4] = {W1, W2, W1, W4};
    const uint32_t wstride[4] = {(uint32_t)kTickChunk, (uint32_t)kTickChunk, (uint32_t)kTickChunk, (uint32_t)kTickW4};
    auto load_w = [&](int l) {
        mbar_expect_tx(full(l), (uint32_t)(nk[l] * nn[l] * kTcKChunk * 2));
        for (int c = 0; c < nk[l]; ++c) tma_load_2d(wbase[l] + (uint32_t)c * wstride[l], maps[l], c * kTcKChunk, 0, full(l));
    };
    if (tid == 0) {
        s_fail = 0;
        for (int l = 0; l < 4; ++l) mbar_init(full(l));
        mbar_init(done);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        load_w(0);                                 // W1, W2 and W4 now; W3 into W1's place later
        load_w(1);
        load_w(3);
    }
    // the inputs, sur_features' arithmetic spread over the threads: thread k < 64 the
    // descriptor cell k, thread 64 the pose and velocity part
    {
        const float *an = a.anchor;
        const float qa[4] = {an[3], an[4], an[5], an[6]};
        const float ih = 1.0f / a.s.h, ic = 1.0f / a.s.c, irho = 1.0f / a.s.rho0;
        float d[3], o[3];
        if (tid < 64) {
            const float *cell = an + 13 + 4 * tid;
            s_v[13 + 4 * tid] = cell[0] * irho - 1.0f;
            for (int i = 0; i < 3; ++i) d[i] = cell[1 + i] * ic;
            rot_t_apply(qa, d, o);
            for (int i = 0; i < 3; ++i) s_v[14 + 4 * tid + i] = o[i];
        } else if (tid == 64) {
            for (int i = 0; i < 3; ++i) d[i] = (a.t13[i] - an[i]) * ih;
            rot_t_apply(qa, d, o);
            for (int i = 0; i < 3; ++i) s_v[i] = o[i];
            s_v[3] = a.tau * a.s.c * ih;
            for (int i = 0; i < 3; ++i) d[i] = (a.t13[7 + i] - an[7 + i]) * ic;
            rot_t_apply(qa, d, o);
            for (int i = 0; i < 3; ++i) s_v[4 + i] = o[i];
            for (int i = 0; i < 3; ++i) d[i] = a.t13[7 + i] * ic;
            rot_t_apply(qa, d, o);
            for (int i = 0; i < 3; ++i) s_v[7 + i] = o[i];
            for (int i = 0; i < 3; ++i) d[i] = a.t13[10 + i] * a.s.h * ic;
            rot_t_apply(qa, d, o);
            for (int i = 0; i < 3; ++i) s_v[10 + i] = o[i];
        }
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(128));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = s_tmem;
    // row 0 over all five K chunks (320 columns): the weights' zero fill past K = 272 meets
    // zeros here, never stale shared memory
    for (int k = tid; k < 5 * kTcKChunk; k += 128) put(k, k < kIn ? (s_v[k] - a.xmean[k]) * a.xinv[k] : 0.0f);

    const float *bias[3] = {a.b1, a.b2, a.b3};
    for (int l = 0; l < 4; ++l) {
        // the A row written by the threads becomes visible to the tensor core
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (tid == 0 && l == 1) load_w(2);          // layer 1's MMAs are done with W1
        if (tid == 32) {
            if (mbar_wait(full(l), 0u)) {
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint32_t idesc = instr_desc(nn[l]);
                for (int c = 0; c < nk[l]; ++c)
#pragma unroll
                    for (int j = 0; j < kTcKChunk / 16; ++j)
                        mma_bf16(tmem, smem_desc_sw128(A + (uint32_t)c * kTickChunk + 32u * j),
                                 smem_desc_sw128(wbase[l] + (uint32_t)c * wstride[l] + 32u * j), idesc,
                                 (c > 0 || j > 0) ? 1u : 0u);
            } else {
                s_fail = 1;
            }
            mma_commit(done);                      // fires once the issued MMAs completed
        }
        __syncwarp();
        if (!mbar_wait(done, (uint32_t)(l & 1))) s_fail = 1;
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (warp == 0) {
            // row 0 of the accumulator is TMEM lane 0: lane 0 of warp 0
            for (int c0 = 0; c0 < nn[l]; c0 += 16) {
                uint32_t r[16];
                tmem_ld16(tmem + (uint32_t)c0, r);
                if (lane == 0)
                    for (int j = 0; j < 16; ++j) s_v[c0 + j] = __uint_as_float(r[j]);
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        if (l < 3) {
            put(tid, gelu_f(s_v[tid] + bias[l][tid]));     // kHid = 128 = the threads
        } else if (tid == 0) {
            float y[kOut];
            for (int j = 0; j < kOut; ++j) y[j] = s_v[j] + a.b4[j];
            if (s_fail) {
                if (a.status) atomicOr(a.status, (unsigned)ST_TIMEOUT);
            } else {
                tick_output(y, a.ymean, a.ystd, a.anchor, a.wa, a.s, a.out);
            }
            // the model's status word rides along with the wrench (one copy to the host)
            a.out[kOut] = a.status ? (double)*reinterpret_cast<volatile unsigned *>(a.status) : 0.0;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(128));
    }
}

}  // namespace sphgb

using namespace sphgb;

struct sph_mlp {
    cudaStream_t stream = nullptr;
    int max_batch = 0;
    int adam_t = 0;
    float *master, *m, *v, *grad, *norm;   // norm: xmean[269] xinv[269] ymean[6] ystd[6] yinv[6]
    __nv_bfloat16 *w1b, *w2b, *w3b, *w4b;
    float *b4pad;
    __nv_bfloat16 *xb, *h1, *h2, *h3, *dyb, *dz3, *dz2, *dz1;
    float *z1, *z2, *z3, *y, *out;
    float *dW1, *dW2, *dW3, *dW4t;     // K-slice partials of the augmented weight gradients
    double *loss, *loss_part;
    float *db4_part, *db3_part, *db2_part, *db1_part;   // bias-gradient partials
    unsigned *status;
    // K-contiguous operands of the backward GEMMs: weight transposes, and column-major
    // ([feature][batch], leading dimension ldt) copies of the input, activations and gradients
    __nv_bfloat16 *w2t, *w3t, *w4t;
    __nv_bfloat16 *xbT, *h1T, *h2T, *h3T, *dybT, *dz3T, *dz2T, *dz1T;
    int ldt = 0;
    // the haptic tick: anchor descriptor (269), anchor wrench (6 doubles), the tick's input
    // row (269) and result (6 doubles); scales; pinned host copy of the result; the event
    // that orders the anchor (handle's stream) before the ticks (model's stream)
    float *anchor, *tick_x;
    double *anchor_w, *tick_w;
    SurScale scale = {0.0f, 0.0f, 0.0f};
    double *pin = nullptr;
    cudaEvent_t anchored = nullptr;
    bool has_anchor = false;
    // the fused tick's TMA maps of the BF16 weights (built once; false: the unfused path)
    CUtensorMap wmap[4];
    bool tick_fused = false;
    std::string err;
};

namespace {

size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

struct MlpLayout {
    size_t off[64];
    size_t total;
};

int ldt_of(int B) { return (B + 7) & ~7; }

// Every buffer of the surrogate, in order; sizes in bytes for batch capacity B.
size_t mlp_sizes(int B, size_t *sz)
{
    int i = 0;
    sz[i++] = 4 * (size_t)kParams;            // master
    sz[i++] = 4 * (size_t)kParams;            // m
    sz[i++] = 4 * (size_t)kParams;            // v
    sz[i++] = 4 * (size_t)kParams;            // grad
    sz[i++] = 4 * (size_t)(2 * kIn + 3 * kOut);  // norm
    sz[i++] = 2 * (size_t)kHid * kInPad;      // w1b
    sz[i++] = 2 * (size_t)kHid * kHid;        // w2b
    sz[i++] = 2 * (size_t)kHid * kHid;        // w3b
    sz[i++] = 2 * (size_t)kOutPad * kHid;     // w4b
    sz[i++] = 4 * (size_t)kOutPad;            // b4pad
    sz[i++] = 2 * (size_t)B * kInPad;         // xb
    for (int k = 0; k < 3; ++k) sz[i++] = 2 * (size_t)B * kHid;   // h1 h2 h3
    sz[i++] = 2 * (size_t)B * kOutPad;        // dyb
    for (int k = 0; k < 3; ++k) sz[i++] = 2 * (size_t)B * kHid;   // dz3 dz2 dz1
    for (int k = 0; k < 3; ++k) sz[i++] = 4 * (size_t)B * kHid;   // z1 z2 z3
    sz[i++] = 4 * (size_t)B * kOutPad;        // y
    sz[i++] = 4 * (size_t)B * kOut;           // out
    sz[i++] = 4 * (size_t)kSplit * kHid * kInPad;   // dW1 (K slices)
    sz[i++] = 4 * (size_t)kSplit * kHid * kHid;     // dW2
    sz[i++] = 4 * (size_t)kSplit * kHid * kHid;     // dW3
    sz[i++] = 4 * (size_t)kSplit * kHid * kOutPad;  // dW4t
    sz[i++] = 8;                              // loss
    const size_t nblk = (size_t)(B * kOutPad + kLossThreads - 1) / kLossThreads;
    const size_t tiles = (size_t)(B + kTcM - 1) / kTcM;
    sz[i++] = 8 * nblk;                       // loss_part
    sz[i++] = 4 * nblk * kOutPad;             // db4_part
    for (int k = 0; k < 3; ++k) sz[i++] = 4 * tiles * kHid;   // db3_part db2_part db1_part
    sz[i++] = 16;                             // status
    sz[i++] = 4 * (size_t)kIn;                // anchor
    sz[i++] = 4 * (size_t)kIn;                // tick_x
    sz[i++] = 8 * (size_t)kOut;               // anchor_w
    sz[i++] = 8 * (size_t)(kOut + 2);         // tick_w (+ the status word)
    sz[i++] = 2 * (size_t)kHid * kHid;        // w2t
    sz[i++] = 2 * (size_t)kHid * kHid;        // w3t
    sz[i++] = 2 * (size_t)kHid * kOutPad;     // w4t
    const size_t lt = (size_t)ldt_of(B);
    sz[i++] = 2 * (size_t)kInPad * lt;        // xbT
    for (int k = 0; k < 3; ++k) sz[i++] = 2 * (size_t)kHid * lt;   // h1T h2T h3T
    sz[i++] = 2 * (size_t)kOutPad * lt;       // dybT
    for (int k = 0; k < 3; ++k) sz[i++] = 2 * (size_t)kHid * lt;   // dz3T dz2T dz1T
    return (size_t)i;
}

MlpLayout mlp_layout(int B)
{
    MlpLayout L;
    size_t sz[64];
    size_t n = mlp_sizes(B, sz), off = 0;
    for (size_t k = 0; k < n; ++k) { L.off[k] = off; off = a256(off + sz[k]); }
    L.total = off;
    return L;
}

sph_status mfail(sph_mlp *m, sph_status s, const std::string &msg)
{
    if (m) m->err = msg;
    return s;
}

#define MLP_CUDA(m, call)                                                            \
    do {                                                                             \
        cudaError_t e_ = (call);                                                     \
        if (e_ != cudaSuccess)                                                       \
            return mfail((m), SPH_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

// C[M][N] = A[M][K] B[N][K]^T with K-contiguous BF16 operands
TcGemm gemm(const __nv_bfloat16 *A, int lda, const __nv_bfloat16 *B, int ldb, int M, int N, int K, float *C,
            int ldc, unsigned *status)
{
    TcGemm g;
    std::memset(&g, 0, sizeof g);
    g.A = A; g.lda = lda;
    g.B = B; g.ldb = ldb;
    g.M = M; g.N = N; g.K = K; g.C = C; g.ldc = ldc;
    g.epilogue = TC_STORE;
    g.ksplit = 1;
    g.status = status;
    return g;
}

// Forward pass of a batch of B rows; `train` also writes the column-major copies the
// backward pass contracts over the batch.
sph_status mlp_forward(sph_mlp *m, const float *d_x, int B, bool train)
{
    cudaStream_t s = m->stream;
    const float *xmean = m->norm, *xinv = m->norm + kIn;
    k_prep_input<<<dim3((kInPad + 31) / 32, (B + 31) / 32), dim3(32, 8), 0, s>>>(d_x, B, xmean, xinv, m->xb,
                                                                                train ? m->xbT : nullptr, m->ldt);
    MLP_CUDA(m, cudaGetLastError());
    const __nv_bfloat16 *in[3] = {m->xb, m->h1, m->h2};
    const __nv_bfloat16 *w[3] = {m->w1b, m->w2b, m->w3b};
    __nv_bfloat16 *hout[3] = {m->h1, m->h2, m->h3};
    __nv_bfloat16 *hT[3] = {m->h1T, m->h2T, m->h3T};
    float *z[3] = {m->z1, m->z2, m->z3};
    const int kdim[3] = {kInPad, kHid, kHid};
    const int boff[3] = {kOffB1, kOffB2, kOffB3};
    for (int l = 0; l < 3; ++l) {
        TcGemm g = gemm(in[l], kdim[l], w[l], kdim[l], B, kHid, kdim[l], z[l], kHid, m->status);
        g.epilogue = TC_BIAS_GELU;
        g.bias = m->master + boff[l];
        g.aux_out = hout[l];
        g.ldaux = kHid;
        if (train) { g.aux_out_t = hT[l]; g.ldaux_t = m->ldt; }
        MLP_CUDA(m, tc_gemm(g, s));
    }
    TcGemm g = gemm(m->h3, kHid, m->w4b, kHid, B, kOutPad, kHid, m->y, kOutPad, m->status);
    g.epilogue = TC_BIAS;
    g.bias = m->b4pad;
    MLP_CUDA(m, tc_gemm(g, s));
    return SPH_OK;
}

// Backward pass: loss, dY, the dZ chain and the weight-gradient K slices; `src` and `nblk`
// say where the gradient gather finds them.
sph_status mlp_backward(sph_mlp *m, const float *d_t, int B, GradSrc &src, int &nblk)
{
    cudaStream_t s = m->stream;
    const float *ymean = m->norm + 2 * kIn, *yinv = m->norm + 2 * kIn + 2 * kOut;
    const int lt = m->ldt;
    nblk = (B * kOutPad + kLossThreads - 1) / kLossThreads;
    k_loss_grad<<<nblk, kLossThreads, 0, s>>>(m->y, d_t, B, ymean, yinv, m->dyb, m->dybT, lt, m->loss_part,
                                              m->db4_part);
    MLP_CUDA(m, cudaGetLastError());
    // weight gradients contract over the batch: K = B, split into `slices` batch ranges
    const int slices = std::min(kSplit, (B + kTcKChunk - 1) / kTcKChunk);
    auto wgrad = [&](const __nv_bfloat16 *AT, int M, const __nv_bfloat16 *BT, int N, float *dW) {
        TcGemm g = gemm(AT, lt, BT, lt, M, N, B, dW, N, m->status);
        g.ksplit = slices;
        g.split_stride = (size_t)M * N;
        return tc_gemm(g, s);
    };
    // dZ = (dZ_next W) * gelu'(Z): BF16 row-major and column-major, and the column sums of
    // the unrounded dZ per 128-row tile (the bias gradient's partials)
    auto dzgemm = [&](const __nv_bfloat16 *dn, int kn, const __nv_bfloat16 *wt, const float *z,
                      __nv_bfloat16 *dz, __nv_bfloat16 *dzT, float *db_part) {
        TcGemm g = gemm(dn, kn, wt, kn, B, kHid, kn, nullptr, kHid, m->status);
        g.epilogue = TC_GELU_GRAD; g.aux_in = z; g.aux_out = dz; g.ldaux = kHid;
        g.aux_out_t = dzT; g.ldaux_t = lt;
        g.colsum = db_part; g.ld_colsum = kHid;
        return tc_gemm(g, s);
    };
    // layer 4: dW4^T = H3^T dY (rows = 128 inputs, K = batch)
    MLP_CUDA(m, wgrad(m->h3T, kHid, m->dybT, kOutPad, m->dW4t));
    // dZ3 = (dY W4) * gelu'(Z3): B operand W4^T [128][16]
    MLP_CUDA(m, dzgemm(m->dyb, kOutPad, m->w4t, m->z3, m->dz3, m->dz3T, m->db3_part));
    // layers 3 and 2: dW = dZ^T H_prev, dZ_prev = (dZ W) * gelu'(Z_prev)
    MLP_CUDA(m, wgrad(m->dz3T, kHid, m->h2T, kHid, m->dW3));
    MLP_CUDA(m, dzgemm(m->dz3, kHid, m->w3t, m->z2, m->dz2, m->dz2T, m->db2_part));
    MLP_CUDA(m, wgrad(m->dz2T, kHid, m->h1T, kHid, m->dW2));
    MLP_CUDA(m, dzgemm(m->dz2, kHid, m->w2t, m->z1, m->dz1, m->dz1T, m->db1_part));
    // layer 1: dW1 = dZ1^T Xb (N = 272)
    MLP_CUDA(m, wgrad(m->dz1T, kHid, m->xbT, kInPad, m->dW1));
    src = GradSrc{m->dW1, m->dW2, m->dW3, m->dW4t, slices,
                  m->db1_part, m->db2_part, m->db3_part, (B + kTcM - 1) / kTcM, m->db4_part, nblk};
    return SPH_OK;
}

sph_status mlp_status(sph_mlp *m)
{
    unsigned st = 0;
    MLP_CUDA(m, cudaMemcpyAsync(&st, m->status, 4, cudaMemcpyDeviceToHost, m->stream));
    MLP_CUDA(m, cudaStreamSynchronize(m->stream));
    if (st) {
        MLP_CUDA(m, cudaMemsetAsync(m->status, 0, 4, m->stream));
        return mfail(m, SPH_ERR_TIMEOUT, "a tensor-core completion wait gave up");
    }
    return SPH_OK;
}

}  // namespace

extern "C" {

int32_t sph_mlp_param_count(void) { return kParams; }

size_t sph_mlp_workspace_bytes(int32_t max_batch)
{
    if (max_batch < 1 || max_batch > (1 << 20)) return 0;
    return mlp_layout(max_batch).total;
}

sph_status sph_mlp_create(void *d_workspace, size_t bytes, void *cuda_stream, int32_t max_batch,
                          sph_mlp **out)
{
    if (!out) return SPH_ERR_ARG;
    *out = nullptr;
    if (max_batch < 1) return SPH_ERR_ARG;
    MlpLayout L = mlp_layout(max_batch);
    if (!d_workspace || bytes < L.total || ((uintptr_t)d_workspace & 255u)) return SPH_ERR_WORKSPACE;
    sph_mlp *m = new sph_mlp();
    m->stream = (cudaStream_t)cuda_stream;
    m->max_batch = max_batch;
    char *ws = (char *)d_workspace;
    int i = 0;
    auto f = [&]() { return reinterpret_cast<float *>(ws + L.off[i++]); };
    auto h = [&]() { return reinterpret_cast<__nv_bfloat16 *>(ws + L.off[i++]); };
    m->master = f(); m->m = f(); m->v = f(); m->grad = f(); m->norm = f();
    m->w1b = h(); m->w2b = h(); m->w3b = h(); m->w4b = h(); m->b4pad = f();
    m->xb = h(); m->h1 = h(); m->h2 = h(); m->h3 = h(); m->dyb = h();
    m->dz3 = h(); m->dz2 = h(); m->dz1 = h();
    m->z1 = f(); m->z2 = f(); m->z3 = f(); m->y = f(); m->out = f();
    m->dW1 = f(); m->dW2 = f(); m->dW3 = f(); m->dW4t = f();
    m->loss = reinterpret_cast<double *>(ws + L.off[i++]);
    m->loss_part = reinterpret_cast<double *>(ws + L.off[i++]);
    m->db4_part = f(); m->db3_part = f(); m->db2_part = f(); m->db1_part = f();
    m->status = reinterpret_cast<unsigned *>(ws + L.off[i++]);
    m->anchor = f(); m->tick_x = f();
    m->anchor_w = reinterpret_cast<double *>(ws + L.off[i++]);
    m->tick_w = reinterpret_cast<double *>(ws + L.off[i++]);
    m->w2t = h(); m->w3t = h(); m->w4t = h();
    m->xbT = h(); m->h1T = h(); m->h2T = h(); m->h3T = h(); m->dybT = h();
    m->dz3T = h(); m->dz2T = h(); m->dz1T = h();
    m->ldt = ldt_of(max_batch);
    m->tick_fused = tc_operand_map(&m->wmap[0], m->w1b, kHid, kInPad, kInPad, kHid) &&
                    tc_operand_map(&m->wmap[1], m->w2b, kHid, kHid, kHid, kHid) &&
                    tc_operand_map(&m->wmap[2], m->w3b, kHid, kHid, kHid, kHid) &&
                    tc_operand_map(&m->wmap[3], m->w4b, kOutPad, kHid, kHid, kOutPad);
    cudaError_t e = cudaMemsetAsync(ws, 0, L.total, m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    if (e == cudaSuccess) e = cudaHostAlloc(&m->pin, 8 * (kOut + 2), cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&m->anchored, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        if (m->pin) cudaFreeHost(m->pin);
        delete m;
        return SPH_ERR_CUDA;
    }
    *out = m;
    return SPH_OK;
}

sph_status sph_mlp_set_params(sph_mlp *m, const float *h_params, const float *h_norm)
{
    if (!m || !h_params) return SPH_ERR_ARG;
    MLP_CUDA(m, cudaMemcpyAsync(m->master, h_params, 4 * (size_t)kParams, cudaMemcpyHostToDevice, m->stream));
    if (h_norm) {
        // h_norm: xmean[269] xstd[269] ymean[6] ystd[6]; stored with reciprocals
        std::vector<float> nb(2 * kIn + 3 * kOut);
        for (int c = 0; c < kIn; ++c) { nb[c] = h_norm[c]; nb[kIn + c] = 1.0f / h_norm[kIn + c]; }
        for (int j = 0; j < kOut; ++j) {
            nb[2 * kIn + j] = h_norm[2 * kIn + j];
            nb[2 * kIn + kOut + j] = h_norm[2 * kIn + kOut + j];
            nb[2 * kIn + 2 * kOut + j] = 1.0f / h_norm[2 * kIn + kOut + j];
        }
        MLP_CUDA(m, cudaMemcpyAsync(m->norm, nb.data(), 4 * nb.size(), cudaMemcpyHostToDevice, m->stream));
    }
    MLP_CUDA(m, cudaMemsetAsync(m->m, 0, 4 * (size_t)kParams, m->stream));
    MLP_CUDA(m, cudaMemsetAsync(m->v, 0, 4 * (size_t)kParams, m->stream));
    m->adam_t = 0;
    k_refresh_bf16<<<(kHid * kInPad + 255) / 256, 256, 0, m->stream>>>(m->master, m->w1b, m->w2b, m->w3b,
                                                                       m->w4b, m->b4pad, m->w2t, m->w3t,
                                                                       m->w4t);
    MLP_CUDA(m, cudaGetLastError());
    MLP_CUDA(m, cudaStreamSynchronize(m->stream));
    return SPH_OK;
}

sph_status sph_mlp_get_params(sph_mlp *m, float *h_params)
{
    if (!m || !h_params) return SPH_ERR_ARG;
    MLP_CUDA(m, cudaMemcpyAsync(h_params, m->master, 4 * (size_t)kParams, cudaMemcpyDeviceToHost, m->stream));
    return mlp_status(m);
}

sph_status sph_mlp_forward(sph_mlp *m, const float *d_x, int32_t batch, float *d_y)
{
    if (!m || !d_x || !d_y || batch < 1 || batch > m->max_batch) return SPH_ERR_ARG;
    sph_status st = mlp_forward(m, d_x, batch, false);
    if (st != SPH_OK) return st;
    const float *ymean = m->norm + 2 * kIn, *ystd = m->norm + 2 * kIn + kOut;
    k_output<<<(batch * kOut + 255) / 256, 256, 0, m->stream>>>(m->y, batch, ymean, ystd, d_y);
    MLP_CUDA(m, cudaGetLastError());
    return SPH_OK;
}

sph_status sph_mlp_gradients(sph_mlp *m, const float *d_x, const float *d_t, int32_t batch, float *h_grad,
                             double *h_loss)
{
    if (!m || !d_x || !d_t || batch < 1 || batch > m->max_batch) return SPH_ERR_ARG;
    GradSrc src;
    int nblk = 0;
    sph_status st = mlp_forward(m, d_x, batch, true);
    if (st == SPH_OK) st = mlp_backward(m, d_t, batch, src, nblk);
    if (st != SPH_OK) return st;
    k_gather_grads<<<(kParams + 255) / 256, 256, 0, m->stream>>>(src, m->grad, m->loss_part, nblk, batch, m->loss);
    MLP_CUDA(m, cudaGetLastError());
    if (h_grad)
        MLP_CUDA(m, cudaMemcpyAsync(h_grad, m->grad, 4 * (size_t)kParams, cudaMemcpyDeviceToHost, m->stream));
    if (h_loss) MLP_CUDA(m, cudaMemcpyAsync(h_loss, m->loss, 8, cudaMemcpyDeviceToHost, m->stream));
    return mlp_status(m);
}

sph_status sph_mlp_train_step(sph_mlp *m, const float *d_x, const float *d_t, int32_t batch, float lr,
                              double *h_loss)
{
    if (!m || !d_x || !d_t || batch < 1 || batch > m->max_batch || !(lr > 0.0f)) return SPH_ERR_ARG;
    GradSrc src;
    int nblk = 0;
    sph_status st = mlp_forward(m, d_x, batch, true);
    if (st == SPH_OK) st = mlp_backward(m, d_t, batch, src, nblk);
    if (st != SPH_OK) return st;
    m->adam_t += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f / (1.0f - std::pow(b1, (float)m->adam_t));
    const float c2 = 1.0f / (1.0f - std::pow(b2, (float)m->adam_t));
    const Images im{m->w1b, m->w2b, m->w3b, m->w4b, m->w2t, m->w3t, m->w4t, m->b4pad};
    k_train_update<<<(kParams + 255) / 256, 256, 0, m->stream>>>(src, m->master, m->m, m->v, m->grad, lr, b1, b2,
                                                                 1e-8f, c1, c2, im, m->loss_part, nblk, batch,
                                                                 m->loss);
    MLP_CUDA(m, cudaGetLastError());
    if (h_loss) {
        MLP_CUDA(m, cudaMemcpyAsync(h_loss, m->loss, 8, cudaMemcpyDeviceToHost, m->stream));
        return mlp_status(m);
    }
    return SPH_OK;
}

sph_status sph_mlp_sync(sph_mlp *m)
{
    if (!m) return SPH_ERR_ARG;
    return mlp_status(m);
}

const char *sph_mlp_last_error(const sph_mlp *m) { return m ? m->err.c_str() : "null model"; }

void sph_mlp_destroy(sph_mlp *m)
{
    if (!m) return;
    cudaStreamSynchronize(m->stream);
    if (m->anchored) cudaEventDestroy(m->anchored);
    if (m->pin) cudaFreeHost(m->pin);
    delete m;
}

static SurScale scale_of(const sph_params *p)
{
    SurScale s;
    s.h = p->h;
    s.c = std::sqrt(p->k);
    s.rho0 = p->rho0;
    return s;
}

sph_status sph_surrogate_set_scene(sph_mlp *m, const sph_params *p)
{
    if (!m || !p || !(p->h > 0.0f) || !(p->k > 0.0f) || !(p->rho0 > 0.0f)) return SPH_ERR_ARG;
    m->scale = scale_of(p);
    return SPH_OK;
}

sph_status sph_surrogate_features(sph_mlp *m, const float *d_ticks, int32_t tick_stride, const float *d_anchors,
                                  int32_t anchor_stride, const float *d_elapsed, int32_t n, float *d_x)
{
    if (!m || n < 0 || (n > 0 && (!d_ticks || !d_anchors || !d_elapsed || !d_x))) return SPH_ERR_ARG;
    if (tick_stride < 13 || anchor_stride < kIn || !(m->scale.h > 0.0f)) return SPH_ERR_ARG;
    if (n == 0) return SPH_OK;
    k_sur_features<<<(n + 127) / 128, 128, 0, m->stream>>>(d_ticks, tick_stride, d_anchors, anchor_stride,
                                                           d_elapsed, n, m->scale, d_x);
    MLP_CUDA(m, cudaGetLastError());
    return SPH_OK;
}

sph_status sph_surrogate_targets(sph_mlp *m, const double *d_wrench, const double *d_anchor_wrench,
                                 const float *d_anchors, int32_t anchor_stride, int32_t n, float *d_t)
{
    if (!m || n < 0 || (n > 0 && (!d_wrench || !d_anchor_wrench || !d_anchors || !d_t))) return SPH_ERR_ARG;
    if (anchor_stride < kIn || !(m->scale.h > 0.0f)) return SPH_ERR_ARG;
    if (n == 0) return SPH_OK;
    k_sur_targets<<<(n + 127) / 128, 128, 0, m->stream>>>(d_wrench, d_anchor_wrench, d_anchors, anchor_stride,
                                                          n, m->scale, d_t);
    MLP_CUDA(m, cudaGetLastError());
    return SPH_OK;
}

sph_status sph_surrogate_anchor(sph_handle *h, sph_mlp *m)
{
    if (!h || !m) return SPH_ERR_ARG;
    cudaStream_t hs;
    const SimConst *c;
    int grab;
    long long substeps;
    handle_surrogate_view(h, &hs, &c, &grab, &substeps);
    if (grab < 0 || substeps == 0) return mfail(m, SPH_ERR_STATE, "no grabbed body or no substep run");
    sph_params p;
    std::memset(&p, 0, sizeof p);
    p.h = c->h;
    p.k = c->k;
    p.rho0 = c->rho0;
    m->scale = scale_of(&p);
    MLP_CUDA(m, launch_descriptor(*c, hs, grab, m->anchor));
    MLP_CUDA(m, cudaMemcpyAsync(m->anchor_w, c->wrench + 6 * grab, 8 * kOut, cudaMemcpyDeviceToDevice, hs));
    MLP_CUDA(m, cudaEventRecord(m->anchored, hs));
    MLP_CUDA(m, cudaStreamWaitEvent(m->stream, m->anchored, 0));
    m->has_anchor = true;
    return SPH_OK;
}

sph_status sph_surrogate_tick(sph_mlp *m, const float pose_vel[13], float elapsed, double out[6])
{
    if (!m || !pose_vel || !out || !(elapsed >= 0.0f)) return SPH_ERR_ARG;
    if (!m->has_anchor) return mfail(m, SPH_ERR_STATE, "no anchor: call sph_surrogate_anchor first");
    const float *t = pose_vel;
    const float *ymean = m->norm + 2 * kIn, *ystd = m->norm + 2 * kIn + kOut;
    if (m->tick_fused) {
        // one kernel: inputs, the four layers on the tensor cores, the wrench
        static std::atomic<unsigned long long> configured{0};
        MLP_CUDA(m, smem_opt_in(k_sur_tick_fused, kTickSmem, configured));
        TickArgs a;
        for (int i = 0; i < 13; ++i) a.t13[i] = t[i];
        a.tau = elapsed;
        a.anchor = m->anchor;
        a.s = m->scale;
        a.xmean = m->norm;
        a.xinv = m->norm + kIn;
        a.ymean = ymean;
        a.ystd = ystd;
        a.b1 = m->master + kOffB1;
        a.b2 = m->master + kOffB2;
        a.b3 = m->master + kOffB3;
        a.b4 = m->b4pad;
        a.wa = m->anchor_w;
        a.out = m->tick_w;
        a.status = m->status;
        k_sur_tick_fused<<<1, 128, kTickSmem, m->stream>>>(m->wmap[0], m->wmap[1], m->wmap[2], m->wmap[3], a);
        MLP_CUDA(m, cudaGetLastError());
    } else {
        k_sur_tick_features<<<1, 32, 0, m->stream>>>(t[0], t[1], t[2], t[3], t[4], t[5], t[6], t[7], t[8], t[9],
                                                     t[10], t[11], t[12], elapsed, m->anchor, m->scale, m->tick_x);
        MLP_CUDA(m, cudaGetLastError());
        sph_status st = mlp_forward(m, m->tick_x, 1, false);
        if (st != SPH_OK) return st;
        k_sur_tick_output<<<1, 32, 0, m->stream>>>(m->y, ymean, ystd, m->anchor, m->anchor_w, m->scale, m->tick_w);
        MLP_CUDA(m, cudaGetLastError());
    }
    sph_status st;
    if (m->tick_fused) {
        // the wrench and the status word in one copy
        MLP_CUDA(m, cudaMemcpyAsync(m->pin, m->tick_w, 8 * (kOut + 1), cudaMemcpyDeviceToHost, m->stream));
        MLP_CUDA(m, cudaStreamSynchronize(m->stream));
        st = SPH_OK;
        if (m->pin[kOut] != 0.0) {
            MLP_CUDA(m, cudaMemsetAsync(m->status, 0, 4, m->stream));
            st = mfail(m, SPH_ERR_TIMEOUT, "a tensor-core completion wait gave up");
        }
    } else {
        MLP_CUDA(m, cudaMemcpyAsync(m->pin, m->tick_w, 8 * kOut, cudaMemcpyDeviceToHost, m->stream));
        st = mlp_status(m);                     // synchronises the model's stream
    }
    if (st != SPH_OK) return st;
    std::memcpy(out, m->pin, 8 * kOut);
    return SPH_OK;
}

}  // extern "C"

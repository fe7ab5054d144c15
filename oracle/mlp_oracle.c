/*
 * mlp_oracle.c -- FP64 CPU reference of the learned wrench surrogate and of its pooled
 * input descriptor.  TEST INFRASTRUCTURE ONLY (tests, smoke check, benchmark baseline).
 *
 * The paper has no learned part; it motivates one by the ~60 Hz update cycle of the
 * engine loop (Sec. 3.3, haptic smoothing).  The network and its precision: a
 * 269-128-128-128-6 multilayer perceptron with the tanh form of GELU, BF16 weights and
 * activations, accumulation in FP32 or better.  With bf16 = 1 the
 * oracle rounds to BF16 (round to nearest even) at exactly those points -- standardised
 * input, weights, hidden activations, output gradient, pre-activation gradients -- and
 * accumulates in FP64; with bf16 = 0 everything is FP64 (used for finite differences).
 *
 * Parameter layout (68,358 values): W1[128][269] b1[128] W2[128][128] b2[128]
 * W3[128][128] b3[128] W4[6][128] b4[6].  Loss: mean over batch x 6 of the squared error
 * of the standardised outputs.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define NI 269
#define NH 128
#define NO 6

enum { OW1 = 0, OB1 = OW1 + NH * NI, OW2 = OB1 + NH, OB2 = OW2 + NH * NH, OW3 = OB2 + NH,
       OB3 = OW3 + NH * NH, OW4 = OB3 + NH, OB4 = OW4 + NO * NH, NPARAM = OB4 + NO };

int orc_mlp_param_count(void) { return NPARAM; }

/* Round a float to the nearest BF16 value (ties to even). */
float orc_bf16(float x)
{
    uint32_t u;
    memcpy(&u, &x, 4);
    if ((u & 0x7f800000u) == 0x7f800000u) return x;
    u += 0x7fffu + ((u >> 16) & 1u);
    u &= 0xffff0000u;
    memcpy(&x, &u, 4);
    return x;
}

static double rnd(double x, int bf) { return bf ? (double)orc_bf16((float)x) : x; }

/* GELU, tanh form: 0.5 z (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3))), and its derivative. */
double orc_gelu(double z)
{
    const double c = 0.7978845608028654, a = 0.044715;
    return 0.5 * z * (1.0 + tanh(c * (z + a * z * z * z)));
}

double orc_gelu_grad(double z)
{
    const double c = 0.7978845608028654, a = 0.044715;
    double t = tanh(c * (z + a * z * z * z));
    return 0.5 * (1.0 + t) + 0.5 * z * (1.0 - t * t) * c * (1.0 + 3.0 * a * z * z);
}

typedef struct {
    double *xn, *z[3], *h[3], *y;   /* B x NI, B x NH (x3), B x NH (x3), B x NO */
} acts;

static void forward(const float *P, const float *norm, const float *X, int B, int bf, acts *A)
{
    const float *xm = norm, *xs = norm + NI;
    /* standardised input, FP32 like the kernel: (x - mean) * (1 / std) */
    for (int b = 0; b < B; ++b)
        for (int i = 0; i < NI; ++i) {
            float inv = 1.0f / xs[i];
            float v = (X[(size_t)b * NI + i] - xm[i]) * inv;
            A->xn[(size_t)b * NI + i] = bf ? (double)orc_bf16(v) : ((double)X[(size_t)b * NI + i] - xm[i]) / xs[i];
        }
    const double *in = A->xn;
    int nin = NI;
    const int ow[3] = { OW1, OW2, OW3 }, ob[3] = { OB1, OB2, OB3 };
    for (int l = 0; l < 3; ++l) {
        for (int b = 0; b < B; ++b)
            for (int j = 0; j < NH; ++j) {
                double s = 0.0;
                for (int i = 0; i < nin; ++i) s += in[(size_t)b * nin + i] * rnd(P[ow[l] + j * nin + i], bf);
                s += P[ob[l] + j];
                A->z[l][(size_t)b * NH + j] = s;
                A->h[l][(size_t)b * NH + j] = rnd(orc_gelu(s), bf);
            }
        in = A->h[l];
        nin = NH;
    }
    for (int b = 0; b < B; ++b)
        for (int j = 0; j < NO; ++j) {
            double s = 0.0;
            for (int i = 0; i < NH; ++i) s += A->h[2][(size_t)b * NH + i] * rnd(P[OW4 + j * NH + i], bf);
            A->y[(size_t)b * NO + j] = s + P[OB4 + j];
        }
}

static void alloc_acts(acts *A, int B)
{
    A->xn = (double *)malloc(sizeof(double) * (size_t)B * NI);
    for (int l = 0; l < 3; ++l) {
        A->z[l] = (double *)malloc(sizeof(double) * (size_t)B * NH);
        A->h[l] = (double *)malloc(sizeof(double) * (size_t)B * NH);
    }
    A->y = (double *)malloc(sizeof(double) * (size_t)B * NO);
}

static void free_acts(acts *A)
{
    free(A->xn);
    for (int l = 0; l < 3; ++l) { free(A->z[l]); free(A->h[l]); }
    free(A->y);
}

/* Forward pass: Y (B x 6) in physical units (de-standardised). */
void orc_mlp_forward(const float *P, const float *norm, const float *X, int B, int bf, double *Y)
{
    acts A;
    alloc_acts(&A, B);
    forward(P, norm, X, B, bf, &A);
    const float *ym = norm + 2 * NI, *ys = norm + 2 * NI + NO;
    for (int b = 0; b < B; ++b)
        for (int j = 0; j < NO; ++j) Y[(size_t)b * NO + j] = A.y[(size_t)b * NO + j] * ys[j] + ym[j];
    free_acts(&A);
}

/* Loss and its gradient with respect to every parameter (backpropagation, FP64 sums). */
double orc_mlp_grad(const float *P, const float *norm, const float *X, const float *T, int B, int bf,
                    double *G)
{
    acts A;
    alloc_acts(&A, B);
    forward(P, norm, X, B, bf, &A);
    const float *ym = norm + 2 * NI, *ys = norm + 2 * NI + NO;
    double loss = 0.0;
    double *dy = (double *)malloc(sizeof(double) * (size_t)B * NO);
    double *dyf = (double *)malloc(sizeof(double) * (size_t)B * NO);
    for (int b = 0; b < B; ++b)
        for (int j = 0; j < NO; ++j) {
            double tn = bf ? (double)((T[(size_t)b * NO + j] - ym[j]) * (1.0f / ys[j]))
                           : ((double)T[(size_t)b * NO + j] - ym[j]) / ys[j];
            double d = A.y[(size_t)b * NO + j] - tn;
            loss += d * d;
            dyf[(size_t)b * NO + j] = 2.0 * d / (double)(NO * B);
            dy[(size_t)b * NO + j] = rnd(dyf[(size_t)b * NO + j], bf);
        }
    loss /= (double)(NO * B);
    memset(G, 0, sizeof(double) * NPARAM);
    /* layer 4 */
    for (int j = 0; j < NO; ++j) {
        double sb = 0.0;
        for (int b = 0; b < B; ++b) sb += dyf[(size_t)b * NO + j];
        G[OB4 + j] = sb;
        for (int i = 0; i < NH; ++i) {
            double s = 0.0;
            for (int b = 0; b < B; ++b) s += A.h[2][(size_t)b * NH + i] * dy[(size_t)b * NO + j];
            G[OW4 + j * NH + i] = s;
        }
    }
    double *dz = (double *)malloc(sizeof(double) * (size_t)B * NH);    /* rounded (GEMM input) */
    double *dzf = (double *)malloc(sizeof(double) * (size_t)B * NH);   /* unrounded (bias grad) */
    for (int b = 0; b < B; ++b)
        for (int i = 0; i < NH; ++i) {
            double s = 0.0;
            for (int j = 0; j < NO; ++j) s += dy[(size_t)b * NO + j] * rnd(P[OW4 + j * NH + i], bf);
            dzf[(size_t)b * NH + i] = s * orc_gelu_grad(A.z[2][(size_t)b * NH + i]);
            dz[(size_t)b * NH + i] = rnd(dzf[(size_t)b * NH + i], bf);
        }
    /* layers 3, 2, 1 */
    const int ow[3] = { OW1, OW2, OW3 }, ob[3] = { OB1, OB2, OB3 };
    double *dzp = (double *)malloc(sizeof(double) * (size_t)B * NH);
    double *dzpf = (double *)malloc(sizeof(double) * (size_t)B * NH);
    for (int l = 2; l >= 0; --l) {
        const double *in = l == 0 ? A.xn : A.h[l - 1];
        const int nin = l == 0 ? NI : NH;
        for (int o = 0; o < NH; ++o) {
            double sb = 0.0;
            for (int b = 0; b < B; ++b) sb += dzf[(size_t)b * NH + o];
            G[ob[l] + o] = sb;
            for (int i = 0; i < nin; ++i) {
                double s = 0.0;
                for (int b = 0; b < B; ++b) s += dz[(size_t)b * NH + o] * in[(size_t)b * nin + i];
                G[ow[l] + o * nin + i] = s;
            }
        }
        if (l == 0) break;
        for (int b = 0; b < B; ++b)
            for (int i = 0; i < NH; ++i) {
                double s = 0.0;
                for (int o = 0; o < NH; ++o) s += dz[(size_t)b * NH + o] * rnd(P[ow[l] + o * NH + i], bf);
                dzpf[(size_t)b * NH + i] = s * orc_gelu_grad(A.z[l - 1][(size_t)b * NH + i]);
                dzp[(size_t)b * NH + i] = rnd(dzpf[(size_t)b * NH + i], bf);
            }
        memcpy(dz, dzp, sizeof(double) * (size_t)B * NH);
        memcpy(dzf, dzpf, sizeof(double) * (size_t)B * NH);
    }
    free(dy); free(dyf); free(dz); free(dzf); free(dzp); free(dzpf);
    free_acts(&A);
    return loss;
}

/*
 * Pooled descriptor of the grabbed body: pose (7) and velocity (6), then 4 x 4 x 4 cells of
 * edge R = fl(2h) centred on the grab point xg (x fastest).  Cell (i, j, k) spans
 * [lo, lo + R) per axis with lo = fl(fl(xg) + (i - 2) R) evaluated in FP32, so membership
 * of FP32 positions is decided exactly as on the GPU.  Per cell: mean density of the fluid
 * particles inside and their mass-weighted mean velocity; zeros when empty.  Brute force
 * over all particles.
 */
void orc_descriptor(int n, const float *x, const double *v, const double *rho, const double *m,
                    const int *is_fluid, const double xg[3], const float pose_vel[13], float h,
                    double *out)
{
    const float R = 2.0f * h;
    for (int a = 0; a < 13; ++a) out[a] = pose_vel[a];
    for (int cell = 0; cell < 64; ++cell) {
        int ci[3] = { cell & 3, (cell >> 2) & 3, cell >> 4 };
        float lo[3], hi[3];
        for (int a = 0; a < 3; ++a) {
            float off = (float)(ci[a] - 2) * R;
            lo[a] = (float)xg[a] + off;
            hi[a] = lo[a] + R;
        }
        double sr = 0.0, sm = 0.0, sv[3] = { 0, 0, 0 };
        int cnt = 0;
        for (int p = 0; p < n; ++p) {
            if (!is_fluid[p]) continue;
            const float *xp = x + 3 * p;
            if (xp[0] < lo[0] || xp[0] >= hi[0] || xp[1] < lo[1] || xp[1] >= hi[1] || xp[2] < lo[2] ||
                xp[2] >= hi[2])
                continue;
            sr += rho[p];
            sm += m[p];
            for (int a = 0; a < 3; ++a) sv[a] += m[p] * v[3 * p + a];
            ++cnt;
        }
        double *d = out + 13 + 4 * cell;
        d[0] = cnt ? sr / cnt : 0.0;
        for (int a = 0; a < 3; ++a) d[1 + a] = sm > 0.0 ? sv[a] / sm : 0.0;
    }
}

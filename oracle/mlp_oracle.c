/*
 * mlp_oracle.c -- FP64 reference for the rate-coefficient surrogate: a
 * three-layer perceptron din -> h -> h -> dout with GELU, MSE loss and Adam.
 *
 * TEST INFRASTRUCTURE ONLY (see ltpc_oracle.c).  The paper motivates the
 * surrogate by the need to resolve high-energy tails, which can take tens of
 * thousands of particles per cell (Sec. 1), and by the rate terms
 * C_kc = int sigma_kc |v| f of Eq. (1) that the fluid equations need.  The
 * network itself is not in the paper; its definition here is the reading the
 * GPU kernels follow:
 *
 *   z1 = X W1^T + b1,  a1 = GELU(z1)          W1: h x din
 *   z2 = a1 W2^T + b2, a2 = GELU(z2)          W2: h x h
 *   y  = a2 W3^T + b3                          W3: dout x h
 *   L  = mean over batch and outputs of (y - t)^2
 *
 * With bf16 != 0 the values the GPU stores in bfloat16 are rounded to
 * bfloat16 (round to nearest, ties to even) at the same points: X, W1, W2,
 * W3, a1, a2 in the forward pass, and the back-propagated dz2, dz1 before
 * they enter the weight-gradient and input-gradient products.  Everything
 * else, and every sum, stays FP64.  GELU is the exact erf form.
 *
 * Pinning: with bf16 == 0 the gradients are checked against central finite
 * differences of the loss, the forward pass against numpy matrix products,
 * and bf16 rounding against exhaustive conversion of float32 bit patterns.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Round a double to the nearest bfloat16 value (8-bit significand), ties to
 * even, returned as a double.  Rounds first to float32 the way a float32
 * accumulator holds the value, then to bfloat16. */
double orc_bf16_round(double x)
{
    float f = (float)x;
    uint32_t u;
    memcpy(&u, &f, 4);
    if ((u & 0x7F800000u) == 0x7F800000u) return (double)f;      /* inf / nan */
    uint32_t lsb = (u >> 16) & 1u;
    u += 0x7FFFu + lsb;
    u &= 0xFFFF0000u;
    memcpy(&f, &u, 4);
    return (double)f;
}

double orc_gelu(double z) { return 0.5 * z * (1.0 + erf(z / sqrt(2.0))); }

static double gelu_grad(double z)
{
    const double inv_sqrt_2pi = 0.39894228040143267794;
    return 0.5 * (1.0 + erf(z / sqrt(2.0))) + z * inv_sqrt_2pi * exp(-0.5 * z * z);
}

static double rnd(double x, int bf16) { return bf16 ? orc_bf16_round(x) : x; }

/* out[r, o] = sum_k in[r, k] W[o, k] + b[o] */
static void linear(int32_t B, int32_t din, int32_t dout, const double *in, const double *W,
                   const double *b, double *out)
{
    for (int32_t r = 0; r < B; ++r)
        for (int32_t o = 0; o < dout; ++o) {
            double s = 0.0;
            for (int32_t k = 0; k < din; ++k) s += in[(size_t)r * din + k] * W[(size_t)o * din + k];
            out[(size_t)r * dout + o] = s + b[o];
        }
}

typedef struct { double *Xb, *W1b, *W2b, *W3b, *z1, *a1, *z2, *a2; } fwd_buf;

static int forward_impl(int32_t B, int32_t din, int32_t h, int32_t dout, const double *X,
                        const double *W1, const double *b1, const double *W2, const double *b2,
                        const double *W3, const double *b3, double *Y, int bf16, fwd_buf *fb)
{
    fb->Xb = (double *)malloc(sizeof(double) * (size_t)B * din);
    fb->W1b = (double *)malloc(sizeof(double) * (size_t)h * din);
    fb->W2b = (double *)malloc(sizeof(double) * (size_t)h * h);
    fb->W3b = (double *)malloc(sizeof(double) * (size_t)dout * h);
    fb->z1 = (double *)malloc(sizeof(double) * (size_t)B * h);
    fb->a1 = (double *)malloc(sizeof(double) * (size_t)B * h);
    fb->z2 = (double *)malloc(sizeof(double) * (size_t)B * h);
    fb->a2 = (double *)malloc(sizeof(double) * (size_t)B * h);
    if (!fb->Xb || !fb->W1b || !fb->W2b || !fb->W3b || !fb->z1 || !fb->a1 || !fb->z2 || !fb->a2) return -1;
    for (size_t i = 0; i < (size_t)B * din; ++i) fb->Xb[i] = rnd(X[i], bf16);
    for (size_t i = 0; i < (size_t)h * din; ++i) fb->W1b[i] = rnd(W1[i], bf16);
    for (size_t i = 0; i < (size_t)h * h; ++i) fb->W2b[i] = rnd(W2[i], bf16);
    for (size_t i = 0; i < (size_t)dout * h; ++i) fb->W3b[i] = rnd(W3[i], bf16);
    linear(B, din, h, fb->Xb, fb->W1b, b1, fb->z1);
    for (size_t i = 0; i < (size_t)B * h; ++i) fb->a1[i] = rnd(orc_gelu(fb->z1[i]), bf16);
    linear(B, h, h, fb->a1, fb->W2b, b2, fb->z2);
    for (size_t i = 0; i < (size_t)B * h; ++i) fb->a2[i] = rnd(orc_gelu(fb->z2[i]), bf16);
    linear(B, h, dout, fb->a2, fb->W3b, b3, Y);
    return 0;
}

static void free_fwd(fwd_buf *fb)
{
    free(fb->Xb); free(fb->W1b); free(fb->W2b); free(fb->W3b);
    free(fb->z1); free(fb->a1); free(fb->z2); free(fb->a2);
}

void orc_mlp_forward(int32_t B, int32_t din, int32_t h, int32_t dout, const double *X,
                     const double *W1, const double *b1, const double *W2, const double *b2,
                     const double *W3, const double *b3, double *Y, int32_t bf16)
{
    fwd_buf fb;
    memset(&fb, 0, sizeof fb);
    forward_impl(B, din, h, dout, X, W1, b1, W2, b2, W3, b3, Y, bf16, &fb);
    free_fwd(&fb);
}

/* Loss and gradients of all parameters for one batch; returns the loss. */
double orc_mlp_loss_backward(int32_t B, int32_t din, int32_t h, int32_t dout, const double *X,
                             const double *T, const double *W1, const double *b1, const double *W2,
                             const double *b2, const double *W3, const double *b3, double *gW1,
                             double *gb1, double *gW2, double *gb2, double *gW3, double *gb3,
                             double *Y, double *unused, int32_t bf16)
{
    (void)unused;
    fwd_buf fb;
    memset(&fb, 0, sizeof fb);
    if (forward_impl(B, din, h, dout, X, W1, b1, W2, b2, W3, b3, Y, bf16, &fb)) { free_fwd(&fb); return NAN; }
    const double scale = 2.0 / ((double)B * (double)dout);
    double loss = 0.0;
    double *g = (double *)malloc(sizeof(double) * (size_t)B * dout);
    double *d2 = (double *)malloc(sizeof(double) * (size_t)B * h);
    double *d1 = (double *)malloc(sizeof(double) * (size_t)B * h);
    for (size_t i = 0; i < (size_t)B * dout; ++i) {
        double e = Y[i] - T[i];
        loss += e * e;
        g[i] = scale * e;                                   /* dL/dy */
    }
    loss /= (double)B * (double)dout;
    /* layer 3 */
    memset(gW3, 0, sizeof(double) * (size_t)dout * h);
    memset(gb3, 0, sizeof(double) * (size_t)dout);
    for (int32_t r = 0; r < B; ++r)
        for (int32_t o = 0; o < dout; ++o) {
            double gv = g[(size_t)r * dout + o];
            gb3[o] += gv;
            for (int32_t k = 0; k < h; ++k) gW3[(size_t)o * h + k] += gv * fb.a2[(size_t)r * h + k];
        }
    /* dz2 = (g W3) * GELU'(z2) */
    for (int32_t r = 0; r < B; ++r)
        for (int32_t k = 0; k < h; ++k) {
            double s = 0.0;
            for (int32_t o = 0; o < dout; ++o) s += g[(size_t)r * dout + o] * fb.W3b[(size_t)o * h + k];
            d2[(size_t)r * h + k] = rnd(s * gelu_grad(fb.z2[(size_t)r * h + k]), bf16);
        }
    /* layer 2 */
    memset(gW2, 0, sizeof(double) * (size_t)h * h);
    memset(gb2, 0, sizeof(double) * (size_t)h);
    for (int32_t r = 0; r < B; ++r)
        for (int32_t o = 0; o < h; ++o) {
            double gv = d2[(size_t)r * h + o];
            gb2[o] += gv;
            for (int32_t k = 0; k < h; ++k) gW2[(size_t)o * h + k] += gv * fb.a1[(size_t)r * h + k];
        }
    /* dz1 = (dz2 W2) * GELU'(z1) */
    for (int32_t r = 0; r < B; ++r)
        for (int32_t k = 0; k < h; ++k) {
            double s = 0.0;
            for (int32_t o = 0; o < h; ++o) s += d2[(size_t)r * h + o] * fb.W2b[(size_t)o * h + k];
            d1[(size_t)r * h + k] = rnd(s * gelu_grad(fb.z1[(size_t)r * h + k]), bf16);
        }
    /* layer 1 */
    memset(gW1, 0, sizeof(double) * (size_t)h * din);
    memset(gb1, 0, sizeof(double) * (size_t)h);
    for (int32_t r = 0; r < B; ++r)
        for (int32_t o = 0; o < h; ++o) {
            double gv = d1[(size_t)r * h + o];
            gb1[o] += gv;
            for (int32_t k = 0; k < din; ++k) gW1[(size_t)o * din + k] += gv * fb.Xb[(size_t)r * din + k];
        }
    free(g); free(d2); free(d1);
    free_fwd(&fb);
    return loss;
}

/* Adam (Kingma & Ba 2015) with bias correction, step t >= 1. */
void orc_adam_update(int64_t n, double *w, const double *g, double *m, double *v, double lr,
                     double beta1, double beta2, double eps, int32_t t)
{
    double c1 = 1.0 - pow(beta1, (double)t), c2 = 1.0 - pow(beta2, (double)t);
    for (int64_t i = 0; i < n; ++i) {
        m[i] = beta1 * m[i] + (1.0 - beta1) * g[i];
        v[i] = beta2 * v[i] + (1.0 - beta2) * g[i] * g[i];
        double mh = m[i] / c1, vh = v[i] / c2;
        w[i] -= lr * mh / (sqrt(vh) + eps);
    }
}

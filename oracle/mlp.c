/*
 * mlp.c -- oracle copy of the importance network, FP64.
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * The learned proposal is a 3-layer perceptron  in -> H -> H -> 1  with SiLU
 * hidden activations, fit by weighted least squares to log-importance
 * targets and optimised with Adam (Kingma & Ba, ICLR 2015).  The paper has no
 * such network; this file is the plain definition the GPU kernels are checked
 * against.
 *
 * Parameter vector (one flat array, this order):
 *   W1[H][in], b1[H], W2[H][H], b2[H], W3[H], b3
 * Loss over n samples with inputs X[n][in], targets y[n], weights w[n]:
 *   L = sum_i w_i (f(x_i) - y_i)^2 / sum_i w_i
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static double silu(double z) { return z / (1.0 + exp(-z)); }
static double dsilu(double z) {
    double s = 1.0 / (1.0 + exp(-z));
    return s * (1.0 + z * (1.0 - s));
}

int64_t orc_mlp_param_count(int32_t in, int32_t H)
{
    return (int64_t)H * in + H + (int64_t)H * H + H + H + 1;
}

/* one sample: forward pass, keeping pre-activations when asked */
static double forward1(int32_t in, int32_t H, const double *p, const double *x,
                       double *z1, double *h1, double *z2, double *h2)
{
    const double *W1 = p, *b1 = W1 + (int64_t)H * in, *W2 = b1 + H, *b2 = W2 + (int64_t)H * H;
    const double *W3 = b2 + H, *b3 = W3 + H;
    for (int32_t j = 0; j < H; ++j) {
        double a = b1[j];
        for (int32_t k = 0; k < in; ++k) a += W1[(int64_t)j * in + k] * x[k];
        z1[j] = a;
        h1[j] = silu(a);
    }
    for (int32_t j = 0; j < H; ++j) {
        double a = b2[j];
        for (int32_t k = 0; k < H; ++k) a += W2[(int64_t)j * H + k] * h1[k];
        z2[j] = a;
        h2[j] = silu(a);
    }
    double y = b3[0];
    for (int32_t k = 0; k < H; ++k) y += W3[k] * h2[k];
    return y;
}

void orc_mlp_forward(int32_t in, int32_t H, int32_t unused, const double *p, int64_t n,
                     const double *X, double *out)
{
    (void)unused;
    double *buf = (double *)malloc(sizeof(double) * 4 * H);
    for (int64_t i = 0; i < n; ++i)
        out[i] = forward1(in, H, p, X + i * in, buf, buf + H, buf + 2 * H, buf + 3 * H);
    free(buf);
}

/* loss and its gradient with respect to every parameter (backpropagation) */
double orc_mlp_loss_grad(int32_t in, int32_t H, int32_t unused, const double *p, int64_t n,
                         const double *X, const double *y, const double *w, double *grad)
{
    (void)unused;
    const int64_t np = orc_mlp_param_count(in, H);
    memset(grad, 0, sizeof(double) * np);
    double *gW1 = grad, *gb1 = gW1 + (int64_t)H * in, *gW2 = gb1 + H, *gb2 = gW2 + (int64_t)H * H;
    double *gW3 = gb2 + H, *gb3 = gW3 + H;
    const double *W2 = p + (int64_t)H * in + H, *W3 = W2 + (int64_t)H * H + H;
    double *buf = (double *)malloc(sizeof(double) * 6 * H);
    double *z1 = buf, *h1 = buf + H, *z2 = buf + 2 * H, *h2 = buf + 3 * H, *d2 = buf + 4 * H,
           *d1 = buf + 5 * H;
    double wsum = 0.0, loss = 0.0;
    for (int64_t i = 0; i < n; ++i) wsum += w[i];
    for (int64_t i = 0; i < n; ++i) {
        const double *x = X + i * in;
        double f = forward1(in, H, p, x, z1, h1, z2, h2);
        double r = f - y[i];
        loss += w[i] * r * r;
        double dy = 2.0 * w[i] * r / wsum;         /* dL/df */
        gb3[0] += dy;
        for (int32_t k = 0; k < H; ++k) {
            gW3[k] += dy * h2[k];
            d2[k] = dy * W3[k] * dsilu(z2[k]);      /* dL/dz2 */
        }
        for (int32_t j = 0; j < H; ++j) {
            gb2[j] += d2[j];
            for (int32_t k = 0; k < H; ++k) gW2[(int64_t)j * H + k] += d2[j] * h1[k];
        }
        for (int32_t k = 0; k < H; ++k) {
            double a = 0.0;
            for (int32_t j = 0; j < H; ++j) a += d2[j] * W2[(int64_t)j * H + k];
            d1[k] = a * dsilu(z1[k]);               /* dL/dz1 */
        }
        for (int32_t j = 0; j < H; ++j) {
            gb1[j] += d1[j];
            for (int32_t k = 0; k < in; ++k) gW1[(int64_t)j * in + k] += d1[j] * x[k];
        }
    }
    free(buf);
    return loss / wsum;
}

/* Adam: m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
 * p -= lr * (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps) */
void orc_adam_step(int64_t np, double *p, double *m, double *v, const double *g, double lr,
                   double b1, double b2, double eps, int64_t t)
{
    const double c1 = 1.0 - pow(b1, (double)t), c2 = 1.0 - pow(b2, (double)t);
    for (int64_t i = 0; i < np; ++i) {
        m[i] = b1 * m[i] + (1.0 - b1) * g[i];
        v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
        p[i] -= lr * (m[i] / c1) / (sqrt(v[i] / c2) + eps);
    }
}

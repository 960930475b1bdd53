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

/* v rounded to BF16 (8 significant bits) through FP32, to nearest with ties
 * to even: the operand precision of the network's matrix products on the
 * GPU (BF16 weights and activations, FP32 accumulation) */
static double bf16r(double v)
{
    float f = (float)v;
    uint32_t b;
    memcpy(&b, &f, 4);
    b = (uint32_t)(((uint64_t)b + 0x7FFFu + ((b >> 16) & 1u)) & 0xFFFF0000u);
    memcpy(&f, &b, 4);
    return (double)f;
}
static double dsilu(double z) {
    double s = 1.0 / (1.0 + exp(-z));
    return s * (1.0 + z * (1.0 - s));
}

int64_t orc_mlp_param_count(int32_t in, int32_t H)
{
    return (int64_t)H * in + H + (int64_t)H * H + H + H + 1;
}

/* an operand of a matrix product: as is, or rounded to BF16 when rnd */
static double opnd(double v, int32_t rnd) { return rnd ? bf16r(v) : v; }

/* one sample: forward pass, keeping pre-activations when asked; rnd rounds
 * the operands of the two hidden layers' products (x, W1, h1, W2) to BF16
 * (h1 is then kept rounded: it is also an operand of the backward pass) */
static double forward1(int32_t in, int32_t H, int32_t rnd, const double *p, const double *x,
                       double *z1, double *h1, double *z2, double *h2)
{
    const double *W1 = p, *b1 = W1 + (int64_t)H * in, *W2 = b1 + H, *b2 = W2 + (int64_t)H * H;
    const double *W3 = b2 + H, *b3 = W3 + H;
    for (int32_t j = 0; j < H; ++j) {
        double a = b1[j];
        for (int32_t k = 0; k < in; ++k) a += opnd(W1[(int64_t)j * in + k], rnd) * opnd(x[k], rnd);
        z1[j] = a;
        h1[j] = opnd(silu(a), rnd);
    }
    for (int32_t j = 0; j < H; ++j) {
        double a = b2[j];
        for (int32_t k = 0; k < H; ++k) a += opnd(W2[(int64_t)j * H + k], rnd) * h1[k];
        z2[j] = a;
        h2[j] = silu(a);
    }
    double y = b3[0];
    for (int32_t k = 0; k < H; ++k) y += W3[k] * h2[k];
    return y;
}

/* bf16: 0 evaluates the definition in FP64; 1 rounds every operand of the
 * matrix products to BF16 first (the precision the network's products run
 * in: BF16 weights and activations), everything else in FP64 */
void orc_mlp_forward(int32_t in, int32_t H, int32_t bf16, const double *p, int64_t n,
                     const double *X, double *out)
{
    double *buf = (double *)malloc(sizeof(double) * 4 * H);
    for (int64_t i = 0; i < n; ++i)
        out[i] = forward1(in, H, bf16, p, X + i * in, buf, buf + H, buf + 2 * H, buf + 3 * H);
    free(buf);
}

/* loss and its gradient with respect to every parameter (backpropagation);
 * bf16 as in orc_mlp_forward, the products of the backward pass included
 * (their operands dL/dz2, dL/dz1, h1, x and W2 in BF16) */
double orc_mlp_loss_grad(int32_t in, int32_t H, int32_t bf16, const double *p, int64_t n,
                         const double *X, const double *y, const double *w, double *grad)
{
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
        double f = forward1(in, H, bf16, p, x, z1, h1, z2, h2);
        double r = f - y[i];
        loss += w[i] * r * r;
        double dy = 2.0 * w[i] * r / wsum;         /* dL/df */
        gb3[0] += dy;
        for (int32_t k = 0; k < H; ++k) {
            gW3[k] += dy * h2[k];
            d2[k] = opnd(dy * W3[k] * dsilu(z2[k]), bf16);      /* dL/dz2 */
        }
        for (int32_t j = 0; j < H; ++j) {
            gb2[j] += d2[j];
            for (int32_t k = 0; k < H; ++k) gW2[(int64_t)j * H + k] += d2[j] * h1[k];
        }
        for (int32_t k = 0; k < H; ++k) {
            double a = 0.0;
            for (int32_t j = 0; j < H; ++j) a += d2[j] * opnd(W2[(int64_t)j * H + k], bf16);
            d1[k] = opnd(a * dsilu(z1[k]), bf16);               /* dL/dz1 */
        }
        for (int32_t j = 0; j < H; ++j) {
            gb1[j] += d1[j];
            for (int32_t k = 0; k < in; ++k) gW1[(int64_t)j * in + k] += d1[j] * opnd(x[k], bf16);
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

/*
 * Tolerance of the tensor-core evaluation (test infrastructure, not part of
 * the method): a first-order bound, per output and per gradient element, of
 * the rounding error of a computation that rounds every operand of a matrix
 * product to BF16 -- x, W1, h1, W2, dL/dz2 and dL/dz1, each with relative
 * error at most u = 2^-8 -- and accumulates every sum in FP32 (recursive
 * summation of N terms: at most N 2^-24 times the sum of the absolute terms),
 * with the activations and the output layer (W3, b3) in FP32.  Each computed
 * quantity q carries a bound e(q) on |q_computed - q|, carried through every
 * operation by the absolute value of its derivative (silu' and silu'' for
 * the activations), so a bound has the shape of the quantity itself: a sum
 * of absolute values of its terms.
 *   f_bound[n], g_bound[np], *loss_bound.
 */
static double d2silu(double z) {
    double s = 1.0 / (1.0 + exp(-z));
    return s * (1.0 - s) * (2.0 + z * (1.0 - 2.0 * s));
}

/* g_abssum, g_absmax (optional): per gradient element the sum and the
 * largest of the absolute values of its per-sample terms. */
static void term_stats(double *sum, double *mx, int64_t i, double t)
{
    if (!sum) return;
    t = fabs(t);
    sum[i] += t;
    if (t > mx[i]) mx[i] = t;
}

void orc_mlp_error_bounds(int32_t in, int32_t H, const double *p, int64_t n, const double *X,
                          const double *y, const double *w, double *f_bound, double *g_bound,
                          double *loss_bound, double *g_abssum, double *g_absmax)
{
    const double u = 1.0 / 256.0, u32 = 1.0 / 16777216.0;
    const int64_t np = orc_mlp_param_count(in, H);
    memset(g_bound, 0, sizeof(double) * np);
    if (g_abssum) {
        memset(g_abssum, 0, sizeof(double) * np);
        memset(g_absmax, 0, sizeof(double) * np);
    }
    const double *W1 = p, *b1 = W1 + (int64_t)H * in, *W2 = b1 + H, *b2 = W2 + (int64_t)H * H;
    const double *W3 = b2 + H, *b3 = W3 + H;
    const int64_t oW1 = 0, ob1 = (int64_t)H * in, oW2 = ob1 + H, ob2 = oW2 + (int64_t)H * H,
                  oW3 = ob2 + H, ob3 = oW3 + H;
    double *eW1 = g_bound, *eb1 = eW1 + (int64_t)H * in, *eW2 = eb1 + H;
    double *eb2 = eW2 + (int64_t)H * H, *eW3 = eb2 + H, *eb3 = eW3 + H;
    double *buf = (double *)malloc(sizeof(double) * 16 * H + sizeof(double) * in);
    double *z1 = buf, *h1 = z1 + H, *z2 = h1 + H, *h2 = z2 + H, *ez1 = h2 + H, *eh1 = ez1 + H,
           *ez2 = eh1 + H, *eh2 = ez2 + H, *d2 = eh2 + H, *ed2 = d2 + H, *dh = ed2 + H,
           *edh = dh + H, *d1 = edh + H, *ed1 = d1 + H, *ex = ed1 + H;
    const double acc_n = (double)n * u32;     /* sums over the samples */
    double wsum = 0.0, eloss = 0.0;
    for (int64_t i = 0; i < n; ++i) wsum += w[i];
    for (int64_t i = 0; i < n; ++i) {
        const double *x = X + i * in;
        for (int32_t k = 0; k < in; ++k) ex[k] = u * fabs(x[k]);
        for (int32_t j = 0; j < H; ++j) {               /* layer 1 */
            double a = b1[j], e = 0.0, s = fabs(b1[j]);
            for (int32_t k = 0; k < in; ++k) {
                const double t = fabs(W1[(int64_t)j * in + k]);
                a += W1[(int64_t)j * in + k] * x[k];
                e += t * ex[k] + u * t * fabs(x[k]);
                s += t * fabs(x[k]);
            }
            z1[j] = a;
            ez1[j] = e + in * u32 * s;
            h1[j] = silu(a);
            eh1[j] = fabs(dsilu(a)) * ez1[j] + u * fabs(h1[j]);   /* then rounded */
        }
        for (int32_t j = 0; j < H; ++j) {               /* layer 2 */
            double a = b2[j], e = 0.0, s = fabs(b2[j]);
            for (int32_t k = 0; k < H; ++k) {
                const double t = fabs(W2[(int64_t)j * H + k]);
                a += W2[(int64_t)j * H + k] * h1[k];
                e += t * eh1[k] + u * t * fabs(h1[k]);
                s += t * fabs(h1[k]);
            }
            z2[j] = a;
            ez2[j] = e + H * u32 * s;
            h2[j] = silu(a);
            eh2[j] = fabs(dsilu(a)) * ez2[j];
        }
        double f = b3[0], ef = 0.0, sf = fabs(b3[0]);
        for (int32_t k = 0; k < H; ++k) {
            f += W3[k] * h2[k];
            ef += fabs(W3[k]) * eh2[k];
            sf += fabs(W3[k] * h2[k]);
        }
        ef += H * u32 * sf;
        f_bound[i] = ef;
        const double r = f - y[i];
        const double dy = 2.0 * w[i] * r / wsum, edy = 2.0 * w[i] * ef / wsum;
        eloss += 2.0 * w[i] * fabs(r) * ef / wsum;
        eb3[0] += edy + acc_n * fabs(dy);
        term_stats(g_abssum, g_absmax, ob3, dy);
        for (int32_t k = 0; k < H; ++k) {
            eW3[k] += edy * fabs(h2[k]) + fabs(dy) * eh2[k] + acc_n * fabs(dy * h2[k]);
            term_stats(g_abssum, g_absmax, oW3 + k, dy * h2[k]);
            d2[k] = dy * W3[k] * dsilu(z2[k]);
            ed2[k] = fabs(W3[k]) * (edy * fabs(dsilu(z2[k])) + fabs(dy) * fabs(d2silu(z2[k])) * ez2[k])
                     + u * fabs(d2[k]);                  /* then rounded */
        }
        for (int32_t j = 0; j < H; ++j) {
            eb2[j] += ed2[j] + acc_n * fabs(d2[j]);
            term_stats(g_abssum, g_absmax, ob2 + j, d2[j]);
            for (int32_t k = 0; k < H; ++k) {
                eW2[(int64_t)j * H + k] += ed2[j] * fabs(h1[k]) + fabs(d2[j]) * eh1[k]
                                           + acc_n * fabs(d2[j] * h1[k]);
                term_stats(g_abssum, g_absmax, oW2 + (int64_t)j * H + k, d2[j] * h1[k]);
            }
        }
        for (int32_t k = 0; k < H; ++k) {               /* dL/dh1 = W2^T dL/dz2 */
            double a = 0.0, e = 0.0, s = 0.0;
            for (int32_t j = 0; j < H; ++j) {
                const double t = fabs(W2[(int64_t)j * H + k]);
                a += d2[j] * W2[(int64_t)j * H + k];
                e += ed2[j] * t + u * fabs(d2[j]) * t;
                s += fabs(d2[j]) * t;
            }
            dh[k] = a;
            edh[k] = e + H * u32 * s;
            d1[k] = a * dsilu(z1[k]);
            ed1[k] = edh[k] * fabs(dsilu(z1[k])) + fabs(a) * fabs(d2silu(z1[k])) * ez1[k]
                     + u * fabs(d1[k]);                  /* then rounded */
        }
        for (int32_t j = 0; j < H; ++j) {
            eb1[j] += ed1[j] + acc_n * fabs(d1[j]);
            term_stats(g_abssum, g_absmax, ob1 + j, d1[j]);
            for (int32_t k = 0; k < in; ++k) {
                eW1[(int64_t)j * in + k] += ed1[j] * fabs(x[k]) + fabs(d1[j]) * ex[k]
                                            + acc_n * fabs(d1[j] * x[k]);
                term_stats(g_abssum, g_absmax, oW1 + (int64_t)j * in + k, d1[j] * x[k]);
            }
        }
    }
    free(buf);
    if (loss_bound) *loss_bound = eloss;
}

/*
 * Tolerance of the warp-batched window evaluation (test infrastructure): a
 * first-order bound, per sample, of |computed output - exact output| when
 *   - every input carries an absolute error x_abs (its FP32 computation) and
 *     is then rounded to an operand format of unit roundoff u, as are W1, W2
 *     and W3;
 *   - every sum accumulates in FP32 (K terms: at most 2 K 2^-24 times the sum
 *     of the absolute terms, K the padded width: 16 or 32 inputs, 64 hidden);
 *   - every activation is computed as s = round(h + h t), h = round(z / 2),
 *     t = tanh(h) within eps_t (absolute): |s - silu(z)| <= u |z| |silu'(z)|
 *     + eps_t |z| / 2 + u |silu(z)| to first order -- the layer-1 activation is
 *     then an operand of layer 2 as it stands, the layer-2 one an operand of
 *     the output layer (a product with W3, FP32 accumulation, then + b3).
 * Bounds are carried as in orc_mlp_error_bounds.  f_bound[n].
 */
static double act_err(double z, double u, double eps_t)
{
    return u * fabs(z) * fabs(dsilu(z)) + 0.5 * eps_t * fabs(z) + u * fabs(silu(z));
}

void orc_mlp_window_bound(int32_t in, int32_t H, const double *p, int64_t n, const double *X,
                          double u, double eps_t, double x_abs, double *f_bound)
{
    const double u32 = 1.0 / 16777216.0;
    const double *W1 = p, *b1 = W1 + (int64_t)H * in, *W2 = b1 + H, *b2 = W2 + (int64_t)H * H;
    const double *W3 = b2 + H, *b3 = W3 + H;
    const double k1 = in > 16 ? 32.0 : 16.0, k2 = 64.0;
    double *buf = (double *)malloc(sizeof(double) * 4 * H + sizeof(double) * in);
    double *h1 = buf, *eh1 = h1 + H, *h2 = eh1 + H, *eh2 = h2 + H, *ex = eh2 + H;
    for (int64_t i = 0; i < n; ++i) {
        const double *x = X + i * in;
        for (int32_t k = 0; k < in; ++k) ex[k] = x_abs + u * (fabs(x[k]) + x_abs);
        for (int32_t j = 0; j < H; ++j) {               /* layer 1 */
            double a = b1[j], e = 0.0, s = fabs(b1[j]);
            for (int32_t k = 0; k < in; ++k) {
                const double t = fabs(W1[(int64_t)j * in + k]);
                a += W1[(int64_t)j * in + k] * x[k];
                e += t * ex[k] + u * t * fabs(x[k]);
                s += t * fabs(x[k]);
            }
            const double ez = e + 2.0 * k1 * u32 * s;
            h1[j] = silu(a);
            eh1[j] = fabs(dsilu(a)) * ez + act_err(a, u, eps_t);
        }
        for (int32_t j = 0; j < H; ++j) {               /* layer 2 */
            double a = b2[j], e = 0.0, s = fabs(b2[j]);
            for (int32_t k = 0; k < H; ++k) {
                const double t = fabs(W2[(int64_t)j * H + k]);
                a += W2[(int64_t)j * H + k] * h1[k];
                e += t * eh1[k] + u * t * fabs(h1[k]);
                s += t * fabs(h1[k]);
            }
            const double ez = e + 2.0 * k2 * u32 * s;
            h2[j] = silu(a);
            eh2[j] = fabs(dsilu(a)) * ez + act_err(a, u, eps_t);
        }
        double ef = 0.0, sf = fabs(b3[0]);
        for (int32_t k = 0; k < H; ++k) {
            ef += fabs(W3[k]) * eh2[k] + u * fabs(W3[k]) * fabs(h2[k]);
            sf += fabs(W3[k] * h2[k]);
        }
        f_bound[i] = ef + 2.0 * (k2 + 1.0) * u32 * sf;
    }
    free(buf);
}

/*
 * Training (test reference for the library's training call): `epochs` passes
 * over minibatches of `batch` consecutive samples (the last one shorter); per
 * minibatch the loss and gradient of orc_mlp_loss_grad (bf16 as there) and
 * one Adam step (b1 0.9, b2 0.999, eps 1e-8, step count from 1).  p is
 * updated in place; loss_first / loss_last receive the mean minibatch loss
 * of the first and the last epoch.
 */
void orc_mlp_train(int32_t in, int32_t H, int32_t bf16, double *p, int64_t n, const double *X,
                   const double *y, const double *w, int32_t epochs, int32_t batch, double lr,
                   double *loss_first, double *loss_last)
{
    const int64_t np = orc_mlp_param_count(in, H);
    double *m = (double *)calloc((size_t)np, sizeof(double));
    double *v = (double *)calloc((size_t)np, sizeof(double));
    double *g = (double *)malloc(sizeof(double) * np);
    const int64_t steps = (n + batch - 1) / batch;
    int64_t t = 0;
    for (int32_t ep = 0; ep < epochs; ++ep) {
        double ls = 0.0;
        for (int64_t b = 0; b < steps; ++b) {
            const int64_t f0 = b * batch, cnt = (f0 + batch < n ? batch : n - f0);
            ls += orc_mlp_loss_grad(in, H, bf16, p, cnt, X + f0 * in, y + f0, w + f0, g);
            orc_adam_step(np, p, m, v, g, lr, 0.9, 0.999, 1e-8, ++t);
        }
        if (ep == 0 && loss_first) *loss_first = ls / (double)steps;
        if (ep == epochs - 1 && loss_last) *loss_last = ls / (double)steps;
    }
    free(m);
    free(v);
    free(g);
}

/*
 * HRKAN FP64 CPU oracle.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path links, loads or
 * calls this file: only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark use it.  It shares no code, header, table or constant with
 * the CUDA path.
 *
 * Every routine is the plain definition from the paper, written for
 * readability, in double precision, with no blocking, no active-set
 * shortcut and no fusion:
 *
 *   support    Section 2.1/2.2: the HR basis uses "the same support as the
 *              B-spline basis" of grid size g and order k, i.e. n = g + k
 *              intervals [s_i, e_i] with s_i = lo + (i-k)h, e_i = lo + (i+1)h,
 *              h = (hi-lo)/g.
 *   basis      Section 3, Eq. 2: v_{m,i}(x) = ReLU(e_i-x)^m ReLU(x-s_i)^m c_m,
 *              c_m = (2/(e_i-s_i))^{2m}; first to fourth derivatives are the
 *              derivatives of that polynomial inside (s_i, e_i), zero outside.
 *   layer      Sections 1-3 (KAN layer as a matrix operation): output unit o of
 *              a layer is sum_j sum_i W[o][j][i] v_i(z_j), summed densely over
 *              all n bases; no bias, no base branch, no normalisation.
 *   jets       the input derivatives the PDE residuals need (Eq. 3: Laplacian;
 *              Eq. 6-8: u_t, u_x, u_xx), third to fifth derivatives along each
 *              input (the higher-order terms Section 3 motivates the order m
 *              with; it picks m = 6 for a fifth derivative), and for D = 2 the
 *              mixed derivative u_x0x1, by the forward-mode chain rule (Faa di
 *              Bruno's formula for the fourth and fifth orders).
 *   loss       Eq. 4 (Poisson) and Eq. 8 (Burgers): L = alpha L_pde + L_bnd,
 *              L_bnd the pooled mean over all boundary/initial points.
 *   backward   hand-written reverse mode of the above.
 *   adam       the Adam update used for training (Section 4), bias-corrected.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PI 3.14159265358979323846

/* ---------------------------------------------------------------- support */

void orc_support(int G, int k, double lo, double hi, double* s, double* e)
{
    double h = (hi - lo) / (double)G;
    for (int i = 0; i < G + k; ++i) {
        s[i] = lo + (double)(i - k) * h;
        e[i] = lo + (double)(i + 1) * h;
    }
}

/* ------------------------------------------------------------------ basis */

static double relu(double x) { return x > 0.0 ? x : 0.0; }

/* b^p for integer p; a negative power only ever multiplies a zero
 * coefficient in the formulas below, so it is returned as 0. */
static double ipow(double b, int p)
{
    if (p < 0) return 0.0;
    double r = 1.0;
    for (int t = 0; t < p; ++t) r *= b;
    return r;
}

/*
 * out[0..4] = v, v', v'', v''', v'''' of the order-m HR basis on [s, e] at x.
 * With p(x) = (e-x)(x-s), p' = e+s-2x, p'' = -2, p''' = 0, inside (s, e):
 *   v    = c p^m
 *   v'   = c m p^{m-1} p'
 *   v''  = c [m(m-1) p^{m-2} p'^2 - 2m p^{m-1}]
 *   v''' = c [m(m-1)(m-2) p^{m-3} p'^3 - 6m(m-1) p^{m-2} p']
 *   v''''= c [m(m-1)(m-2)(m-3) p^{m-4} p'^4 - 12m(m-1)(m-2) p^{m-3} p'^2 + 12m(m-1) p^{m-2}]
 * The value is the literal ReLU product of Eq. 2 everywhere; the derivatives
 * are taken as 0 at and outside the end points.
 */
void orc_hr_basis(int m, double s, double e, double x, double* out)
{
    double c = pow(2.0 / (e - s), 2.0 * m);
    double A = relu(e - x), B = relu(x - s);
    out[0] = ipow(A, m) * ipow(B, m) * c;
    if (!(x > s && x < e)) {
        out[1] = out[2] = out[3] = out[4] = 0.0;
        return;
    }
    double p = A * B, dp = e + s - 2.0 * x;
    double md = (double)m;
    out[1] = c * md * ipow(p, m - 1) * dp;
    out[2] = c * (md * (md - 1.0) * ipow(p, m - 2) * dp * dp - 2.0 * md * ipow(p, m - 1));
    out[3] = c * (md * (md - 1.0) * (md - 2.0) * ipow(p, m - 3) * dp * dp * dp
                  - 6.0 * md * (md - 1.0) * ipow(p, m - 2) * dp);
    out[4] = c * (md * (md - 1.0) * (md - 2.0) * (md - 3.0) * ipow(p, m - 4) * dp * dp * dp * dp
                  - 12.0 * md * (md - 1.0) * (md - 2.0) * ipow(p, m - 3) * dp * dp
                  + 12.0 * md * (md - 1.0) * ipow(p, m - 2));
}

/*
 * out[0..6] = v and its first to sixth derivatives at x.  Eq. 2 in the
 * coordinate u = (2x - s - e)/(e - s) of the support reads c p^m = (1 - u^2)^m,
 * because p = (e-x)(x-s) = ((e-s)/2)^2 (1 - u^2) and c = (2/(e-s))^{2m}.
 * Expanding (1 - u^2)^m = sum_q C(m,q) (-1)^q u^{2q} and differentiating term
 * by term, inside (s, e):
 *   v^(r)(x) = (2/(e-s))^r sum_{2q >= r} C(m,q) (-1)^q (2q)!/(2q-r)! u^{2q-r}.
 * out[0] is the literal ReLU product of Eq. 2; the derivatives are 0 at and
 * outside the end points, as in orc_hr_basis.
 */
void orc_hr_basis6(int m, double s, double e, double x, double* out)
{
    double A = relu(e - x), B = relu(x - s);
    out[0] = ipow(A, m) * ipow(B, m) * pow(2.0 / (e - s), 2.0 * m);
    for (int r = 1; r <= 6; ++r) out[r] = 0.0;
    if (!(x > s && x < e)) return;
    double a = 2.0 / (e - s), u = (2.0 * x - s - e) / (e - s);
    double binom = 1.0;                       /* C(m, q) */
    for (int q = 0; q <= m; ++q) {
        double sign = (q % 2) ? -1.0 : 1.0;
        for (int r = 1; r <= 6 && r <= 2 * q; ++r) {
            double falling = 1.0;                 /* (2q)! / (2q - r)! */
            for (int t = 0; t < r; ++t) falling *= (double)(2 * q - t);
            out[r] += binom * sign * falling * ipow(u, 2 * q - r) * ipow(a, r);
        }
        binom = binom * (double)(m - q) / (double)(q + 1);
    }
}

/*
 * Fourth and fifth derivatives of v(z(x)) along one input, by Faa di Bruno's
 * formula: f[r] = v^(r)(z), g[q] = d^q z / dx^q (q = 1..5):
 *   R4 = f4 g1^4 + 6 f3 g1^2 g2 + 3 f2 g2^2 + 4 f2 g1 g3 + f1 g4
 *   R5 = f5 g1^5 + 10 f4 g1^3 g2 + 15 f3 g1 g2^2 + 10 f3 g1^2 g3 + 10 f2 g2 g3
 *        + 5 f2 g1 g4 + f1 g5
 * d/dz of R is the same polynomial with every f[r] replaced by f[r+1]; the
 * partial derivatives in g are written out in row4_dg / row5_dg.
 */
static double row4(const double* f, const double* g)
{
    return f[4] * g[1] * g[1] * g[1] * g[1] + 6.0 * f[3] * g[1] * g[1] * g[2] + 3.0 * f[2] * g[2] * g[2]
         + 4.0 * f[2] * g[1] * g[3] + f[1] * g[4];
}

static double row5(const double* f, const double* g)
{
    return f[5] * g[1] * g[1] * g[1] * g[1] * g[1] + 10.0 * f[4] * g[1] * g[1] * g[1] * g[2]
         + 15.0 * f[3] * g[1] * g[2] * g[2] + 10.0 * f[3] * g[1] * g[1] * g[3] + 10.0 * f[2] * g[2] * g[3]
         + 5.0 * f[2] * g[1] * g[4] + f[1] * g[5];
}

/* dg[q] = dR4/dg_q, q = 1..4 */
static void row4_dg(const double* f, const double* g, double* dg)
{
    dg[1] = 4.0 * f[4] * g[1] * g[1] * g[1] + 12.0 * f[3] * g[1] * g[2] + 4.0 * f[2] * g[3];
    dg[2] = 6.0 * f[3] * g[1] * g[1] + 6.0 * f[2] * g[2];
    dg[3] = 4.0 * f[2] * g[1];
    dg[4] = f[1];
    dg[5] = 0.0;
}

/* dg[q] = dR5/dg_q, q = 1..5 */
static void row5_dg(const double* f, const double* g, double* dg)
{
    dg[1] = 5.0 * f[5] * g[1] * g[1] * g[1] * g[1] + 30.0 * f[4] * g[1] * g[1] * g[2] + 15.0 * f[3] * g[2] * g[2]
          + 20.0 * f[3] * g[1] * g[3] + 5.0 * f[2] * g[4];
    dg[2] = 10.0 * f[4] * g[1] * g[1] * g[1] + 30.0 * f[3] * g[1] * g[2] + 10.0 * f[2] * g[3];
    dg[3] = 10.0 * f[3] * g[1] * g[1] + 10.0 * f[2] * g[2];
    dg[4] = 5.0 * f[2] * g[1];
    dg[5] = f[1];
}

/* ------------------------------------------------------ reduced precision */

/*
 * Reduced-precision operands for the tensor-core variants (not a method of the
 * paper: the precision the contraction's inputs are rounded to).  The value is
 * first rounded to float32, then
 *   ORC_BF16: to bfloat16, round to nearest even (8-bit significand);
 *   ORC_TF32: to TF32, round to nearest with ties away from zero (11-bit significand);
 *   ORC_BF16W2: operands as ORC_BF16, weights as the sum of two bfloat16
 *   values (round_w below: a contraction split into A_hi W_hi + A_hi W_lo);
 *   ORC_BF16X3: both factors of every product as the sum of two bfloat16
 *   values, x = x_hi + x_lo, and the product taken as
 *   x_hi y_hi + x_hi y_lo + x_lo y_hi (the x_lo y_lo term dropped; prod3 below).
 */
enum { ORC_EXACT = 0, ORC_BF16 = 1, ORC_TF32 = 2, ORC_BF16W2 = 3, ORC_BF16X3 = 4 };

static double round_to(double x, int fmt)
{
    if (fmt == ORC_EXACT) return x;
    float f = (float)x;
    uint32_t u;
    memcpy(&u, &f, 4);
    if (fmt == ORC_BF16 || fmt == ORC_BF16W2 || fmt == ORC_BF16X3) {
        u += 0x7FFFu + ((u >> 16) & 1u);
        u &= 0xFFFF0000u;
    } else {
        u += 0x1000u;
        u &= 0xFFFFE000u;
    }
    memcpy(&f, &u, 4);
    return (double)f;
}

double orc_round(double x, int fmt) { return round_to(x, fmt); }

/* A weight as the contraction sees it: round_to, except under ORC_BF16W2 the
 * float32 weight w is carried as hi + lo with hi = bf16(w), lo = bf16(w - hi)
 * (w - hi is exact in float32: it has at most 16 significant bits). */
static double round_w(double x, int fmt)
{
    if (fmt != ORC_BF16W2) return round_to(x, fmt);
    float w = (float)x;
    float hi = (float)round_to(w, ORC_BF16);
    float lo = (float)round_to(w - hi, ORC_BF16);
    return (double)hi + (double)lo;
}

/* x rounded to float32 and carried as hi + lo: hi = bf16(x), lo = bf16(x - hi)
 * (x - hi is exact in float32). */
static void split_bf16(double x, double* hi, double* lo)
{
    float f = (float)x;
    float h = (float)round_to(f, ORC_BF16);
    *hi = (double)h;
    *lo = round_to(f - h, ORC_BF16);
}

/* The product x y as a contraction in format fmt sees it: under ORC_BF16X3 the
 * three-term split of both factors, otherwise x rounded by round_to and y by
 * wround (round_to, or round_w for weights). */
static double prod3(double x, double y)
{
    double xh, xl, yh, yl;
    split_bf16(x, &xh, &xl);
    split_bf16(y, &yh, &yl);
    return xh * yh + xh * yl + xl * yh;
}

/* A weight w times a basis-matrix entry a (or an output-jet gradient a) under fmt. */
static double wmul(double w, double a, int fmt)
{
    if (fmt == ORC_BF16X3) return prod3(a, w);
    return round_w(w, fmt) * round_to(a, fmt);
}

/* An output-jet gradient g times a basis-matrix entry a under fmt (weight gradient). */
static double gmul(double g, double a, int fmt)
{
    if (fmt == ORC_BF16X3) return prod3(g, a);
    return round_to(g, fmt) * round_to(a, fmt);
}

/* ---------------------------------------------------------------- network */

typedef struct {
    int n_widths;      /* layers + 1 */
    const int* widths; /* widths[0] = D input dims, widths[n_widths-1] = 1 */
    int G, k, m;
    double lo, hi;
} orc_net;

static int orc_nbasis(const orc_net* net) { return net->G + net->k; }

long orc_param_count(int n_widths, const int* widths, int G, int k)
{
    long P = 0;
    for (int l = 0; l + 1 < n_widths; ++l) P += (long)widths[l] * widths[l + 1] * (G + k);
    return P;
}

static long layer_offset(const orc_net* net, int l)
{
    long off = 0, n = orc_nbasis(net);
    for (int t = 0; t < l; ++t) off += (long)net->widths[t] * net->widths[t + 1] * n;
    return off;
}

static int max_width(const orc_net* net)
{
    int w = 0;
    for (int l = 0; l < net->n_widths; ++l) if (net->widths[l] > w) w = net->widths[l];
    return w;
}

/*
 * One layer, one point, full jets over D input dims.
 * z[j], dz[j*D+d] = dz_j/dx_d, d2z[j*D+d] = d2z_j/dx_d^2, d3z = d3z_j/dx_d^3,
 * mz[j] = d2z_j/dx_0dx_1 (D = 2), and when hi != 0 also d4z, d5z (fourth and
 * fifth derivatives along each input)
 *   ->  y, dy, d2y, d3y, my (d4y, d5y), by the chain rule for y = sum W v(z):
 *   y_d = v' z_d,  y_dd = v'' z_d^2 + v' z_dd,  y_ddd = v''' z_d^3 + 3 v'' z_d z_dd + v' z_ddd,
 *   y_01 = v'' z_0 z_1 + v' z_01,  y_dddd = R4,  y_ddddd = R5 (Faa di Bruno, above).
 */
static void layer_forward(const orc_net* net, int l, const double* Wl, int D,
                          const double* s, const double* e,
                          const double* z, const double* dz, const double* d2z, const double* d3z,
                          const double* mz, const double* d4z, const double* d5z,
                          double* y, double* dy, double* d2y, double* d3y, double* my, double* d4y, double* d5y,
                          int hi, int fmt)
{
    int I = net->widths[l], O = net->widths[l + 1], n = orc_nbasis(net);
    for (int o = 0; o < O; ++o) {
        y[o] = 0.0;
        my[o] = 0.0;
        for (int d = 0; d < D; ++d) dy[o * D + d] = d2y[o * D + d] = d3y[o * D + d] = 0.0;
        if (hi)
            for (int d = 0; d < D; ++d) d4y[o * D + d] = d5y[o * D + d] = 0.0;
    }
    for (int j = 0; j < I; ++j) {
        for (int i = 0; i < n; ++i) {
            double b[5];
            orc_hr_basis(net->m, s[i], e[i], z[j], b);
            /* the basis-matrix entries (jet rows) of this input unit and basis */
            double a0 = b[0], a1[8], a2[8], a3[8];
            for (int d = 0; d < D; ++d) {
                double zd = dz[j * D + d], zdd = d2z[j * D + d], zddd = d3z[j * D + d];
                a1[d] = b[1] * zd;
                a2[d] = b[2] * zd * zd + b[1] * zdd;
                a3[d] = b[3] * zd * zd * zd + 3.0 * b[2] * zd * zdd + b[1] * zddd;
            }
            double am = D == 2 ? b[2] * dz[j * D] * dz[j * D + 1] + b[1] * mz[j] : 0.0;
            double a4[8], a5[8];
            if (hi) {
                double f[7];
                orc_hr_basis6(net->m, s[i], e[i], z[j], f);
                for (int d = 0; d < D; ++d) {
                    double g[6] = {0.0, dz[j * D + d], d2z[j * D + d], d3z[j * D + d], d4z[j * D + d],
                                   d5z[j * D + d]};
                    a4[d] = row4(f, g);
                    a5[d] = row5(f, g);
                }
            }
            for (int o = 0; o < O; ++o) {
                double w = Wl[((long)o * I + j) * n + i];
                y[o] += wmul(w, a0, fmt);
                my[o] += wmul(w, am, fmt);
                for (int d = 0; d < D; ++d) {
                    dy[o * D + d] += wmul(w, a1[d], fmt);
                    d2y[o * D + d] += wmul(w, a2[d], fmt);
                    d3y[o * D + d] += wmul(w, a3[d], fmt);
                }
                if (hi)
                    for (int d = 0; d < D; ++d) {
                        d4y[o * D + d] += wmul(w, a4[d], fmt);
                        d5y[o * D + d] += wmul(w, a5[d], fmt);
                    }
            }
        }
    }
}

/* jet rows selected by mask: bit 0 = u, bit 1+d = du/dx_d, bit 1+D+d = d2u/dx_d^2,
 * bit 1+2D+d = d3u/dx_d^3; for D = 2 bit 7 = d2u/dx_0dx_1, bits 8+d the fourth and
 * bits 10+d the fifth derivatives; for D = 3 bits 10+d the fourth and 13+d the fifth. */
static int jet_bits(int D) { return D == 2 ? 12 : 1 + 5 * D; }

/* Order of the derivative bit b stands for (0 = u, 1..5, 6 = the mixed row) and its input *d. */
static int bit_order(int b, int D, int* d)
{
    *d = 0;
    if (b == 0) return 0;
    if (D == 2 && b == 7) return 6;
    int c = (D == 2 && b > 7) ? b - 2 : b - 1;
    *d = c % D;
    return c / D + 1;
}

static int mask_rows(unsigned mask, int D, int* bit_of_row)
{
    int J = 0;
    for (int b = 0; b < jet_bits(D); ++b)
        if (mask & (1u << b)) bit_of_row[J++] = b;
    return J;
}

/* Whether mask asks for a fourth or fifth derivative. */
static int mask_higher(unsigned mask, int D)
{
    int d;
    for (int b = 0; b < jet_bits(D); ++b)
        if ((mask & (1u << b)) && bit_order(b, D, &d) >= 4 && bit_order(b, D, &d) <= 5) return 1;
    return 0;
}

/* Scratch holding the per-layer input jets of one point. */
typedef struct {
    double *z, *dz, *d2z, *d3z, *mz; /* [layer][maxw], [layer][maxw*D], mixed [layer][maxw] */
    double *d4z, *d5z;               /* [layer][maxw*D] */
    int stride;                      /* maxw */
} point_tape;

static int tape_alloc(point_tape* t, const orc_net* net, int D)
{
    int L = net->n_widths - 1, w = max_width(net);
    t->stride = w;
    t->z = calloc((size_t)(L + 1) * w, sizeof(double));
    t->dz = calloc((size_t)(L + 1) * w * D, sizeof(double));
    t->d2z = calloc((size_t)(L + 1) * w * D, sizeof(double));
    t->d3z = calloc((size_t)(L + 1) * w * D, sizeof(double));
    t->mz = calloc((size_t)(L + 1) * w, sizeof(double));
    t->d4z = calloc((size_t)(L + 1) * w * D, sizeof(double));
    t->d5z = calloc((size_t)(L + 1) * w * D, sizeof(double));
    return (t->z && t->dz && t->d2z && t->d3z && t->mz && t->d4z && t->d5z) ? 0 : -1;
}

static void tape_free(point_tape* t)
{
    free(t->z); free(t->dz); free(t->d2z); free(t->d3z); free(t->mz); free(t->d4z); free(t->d5z);
}

/* Forward of one point through all layers; layer l's input jets land in the tape row l,
 * the network output in row L. */
static void point_forward(const orc_net* net, const double* W, int D, const double* s,
                          const double* e, const double* xp, point_tape* t, unsigned round_layers, int fmt,
                          int hi)
{
    int L = net->n_widths - 1, w = t->stride;
    for (int j = 0; j < D; ++j) {
        t->z[j] = xp[j];
        for (int d = 0; d < D; ++d) {
            t->dz[j * D + d] = (j == d) ? 1.0 : 0.0;
            t->d2z[j * D + d] = 0.0;
            t->d3z[j * D + d] = 0.0;
            t->d4z[j * D + d] = 0.0;
            t->d5z[j * D + d] = 0.0;
        }
        t->mz[j] = 0.0;
    }
    for (int l = 0; l < L; ++l) {
        const double* Wl = W + layer_offset(net, l);
        long a = (long)l * w, b = (long)(l + 1) * w;
        layer_forward(net, l, Wl, D, s, e, t->z + a, t->dz + a * D, t->d2z + a * D, t->d3z + a * D, t->mz + a,
                      t->d4z + a * D, t->d5z + a * D,
                      t->z + b, t->dz + b * D, t->d2z + b * D, t->d3z + b * D, t->mz + b, t->d4z + b * D,
                      t->d5z + b * D, hi, ((round_layers >> l) & 1u) ? fmt : ORC_EXACT);
    }
}

/*
 * jets[J][N] of the network output at N points x[D][N] (structure of arrays).
 * Returns 0, or -1 on a bad argument.
 */
int orc_forward_rounded(int n_widths, const int* widths, int G, int k, int m, double lo, double hi,
                        const double* W, const double* x, long N, unsigned mask, double* jets,
                        unsigned round_layers, int fmt)
{
    orc_net net = {n_widths, widths, G, k, m, lo, hi};
    int D = widths[0], L = n_widths - 1;
    if (widths[L] != 1 || !(mask & 1u)) return -1;
    int rows[16];
    int J = mask_rows(mask, D, rows), higher = mask_higher(mask, D);
    int n = G + k;
    double* s = malloc(sizeof(double) * n);
    double* e = malloc(sizeof(double) * n);
    orc_support(G, k, lo, hi, s, e);
    point_tape t;
    if (tape_alloc(&t, &net, D)) return -1;
    double xp[8];
    int w = t.stride;
    for (long p = 0; p < N; ++p) {
        for (int d = 0; d < D; ++d) xp[d] = x[(long)d * N + p];
        point_forward(&net, W, D, s, e, xp, &t, round_layers, fmt, higher);
        long a = (long)L * w;
        const double* by_order[7] = {t.z + a, t.dz + a * D, t.d2z + a * D, t.d3z + a * D, t.d4z + a * D,
                                     t.d5z + a * D, t.mz + a};
        for (int r = 0; r < J; ++r) {
            int d, q = bit_order(rows[r], D, &d);
            jets[(long)r * N + p] = (q == 0 || q == 6) ? by_order[q][0] : by_order[q][d];
        }
    }
    tape_free(&t);
    free(s); free(e);
    return 0;
}

int orc_forward(int n_widths, const int* widths, int G, int k, int m, double lo, double hi,
                const double* W, const double* x, long N, unsigned mask, double* jets)
{
    return orc_forward_rounded(n_widths, widths, G, k, m, lo, hi, W, x, N, mask, jets, 0u, ORC_EXACT);
}

/* One point's jets of unit j from rows [J][I][N] into per-order arrays (rows not in mask: zero).
 * q[0] = value [I], q[1..5] = derivatives of that order [I*D], q[6] = mixed [I]. */
static void unpack_unit(const double* zin, const int* rows, int J, int I, int D, long N, long p, int j,
                        double* const* q)
{
    q[0][j] = 0.0;
    q[6][j] = 0.0;
    for (int o = 1; o <= 5; ++o)
        for (int d = 0; d < D; ++d) q[o][j * D + d] = 0.0;
    for (int r = 0; r < J; ++r) {
        int d, o = bit_order(rows[r], D, &d);
        double v = zin[((long)r * I + j) * N + p];
        if (o == 0 || o == 6) q[o][j] = v;
        else q[o][j * D + d] = v;
    }
}

/*
 * One layer (Sections 1-3) applied to given input jets, D = 2:
 *   zin[r][j][p] for the jet rows r of mask (value and derivatives in bit
 *   order), units j < I, points p < N; rows not in mask are zero.
 *   yout[r][o][p], the same rows for the O outputs.
 * Basis-matrix entries and weights rounded to fmt (ORC_EXACT: none).
 */
int orc_layer_forward(int I, int O, int G, int k, int m, double lo, double hi, const double* Wl,
                      const double* zin, long N, unsigned mask, double* yout, int fmt)
{
    const int D = 2;
    int widths[2] = {I, O};
    orc_net net = {2, widths, G, k, m, lo, hi};
    int rows[16];
    int J = mask_rows(mask, D, rows), higher = mask_higher(mask, D);
    if (!(mask & 1u)) return -1;
    int n = G + k;
    double* s = malloc(sizeof(double) * n);
    double* e = malloc(sizeof(double) * n);
    double* q[7];
    double* out[7];
    for (int o = 0; o < 7; ++o) {
        size_t per = (o == 0 || o == 6) ? 1 : D;
        q[o] = calloc((size_t)I * per, sizeof(double));
        out[o] = calloc((size_t)O * per, sizeof(double));
    }
    orc_support(G, k, lo, hi, s, e);
    for (long p = 0; p < N; ++p) {
        for (int j = 0; j < I; ++j) unpack_unit(zin, rows, J, I, D, N, p, j, q);
        layer_forward(&net, 0, Wl, D, s, e, q[0], q[1], q[2], q[3], q[6], q[4], q[5],
                      out[0], out[1], out[2], out[3], out[6], out[4], out[5], higher, fmt);
        for (int o = 0; o < O; ++o)
            for (int r = 0; r < J; ++r) {
                int d, b = bit_order(rows[r], D, &d);
                yout[((long)r * O + o) * N + p] = (b == 0 || b == 6) ? out[b][o] : out[b][o * D + d];
            }
    }
    for (int o = 0; o < 7; ++o) { free(q[o]); free(out[o]); }
    free(s); free(e);
    return 0;
}

/*
 * Weight gradient of one layer for given output-jet gradients (the
 * contraction of Sections 2-3 differentiated w.r.t. W):
 *   dW[o][j][i] = sum_p sum_r gy[r][o][p] * A_r[p][j][i]
 * with the basis-matrix entries A_r of layer_forward (value, first, second and
 * third derivative rows of input unit j and basis i).  fmt rounds the A entries and
 * gy to BF16/TF32 before the FP64 products and sums (the reduced-precision
 * contraction's inputs; ORC_BF16X3 splits both, prod3); ORC_EXACT rounds nothing.  zin [J][I][N], gy [J][O][N],
 * dW [O][I][n] overwritten.
 */
int orc_layer_dw(int I, int O, int G, int k, int m, double lo, double hi, const double* zin,
                 const double* gy, long N, unsigned mask, double* dW, int fmt)
{
    const int D = 2;
    int rows[16];
    int J = mask_rows(mask, D, rows), higher = mask_higher(mask, D);
    if (!(mask & 1u)) return -1;
    int n = G + k;
    double* s = malloc(sizeof(double) * n);
    double* e = malloc(sizeof(double) * n);
    orc_support(G, k, lo, hi, s, e);
    memset(dW, 0, sizeof(double) * (size_t)O * I * n);
    double a[16];
    for (long p = 0; p < N; ++p) {
        for (int j = 0; j < I; ++j) {
            double z = 0.0, dz[2] = {0.0, 0.0}, d2z[2] = {0.0, 0.0}, d3z[2] = {0.0, 0.0}, mz = 0.0;
            double d4z[2] = {0.0, 0.0}, d5z[2] = {0.0, 0.0};
            double* q[7] = {&z, dz, d2z, d3z, d4z, d5z, &mz};
            for (int r = 0; r < J; ++r) {
                int d, o = bit_order(rows[r], D, &d);
                double v = zin[((long)r * I + j) * N + p];
                if (o == 0 || o == 6) *q[o] = v;
                else q[o][d] = v;
            }
            for (int i = 0; i < n; ++i) {
                double b[5], f[7];
                orc_hr_basis(m, s[i], e[i], z, b);
                if (higher) orc_hr_basis6(m, s[i], e[i], z, f);
                for (int r = 0; r < J; ++r) {
                    int bit = rows[r], dd, ord = bit_order(bit, D, &dd);
                    double v;
                    if (ord == 4 || ord == 5) {
                        double g[6] = {0.0, dz[dd], d2z[dd], d3z[dd], d4z[dd], d5z[dd]};
                        v = ord == 4 ? row4(f, g) : row5(f, g);
                    } else if (bit == 0) {
                        v = b[0];
                    } else if (bit <= D) {
                        v = b[1] * dz[bit - 1];
                    } else if (bit <= 2 * D) {
                        int d = bit - 1 - D;
                        v = b[2] * dz[d] * dz[d] + b[1] * d2z[d];
                    } else if (bit <= 3 * D) {
                        int d = bit - 1 - 2 * D;
                        v = b[3] * dz[d] * dz[d] * dz[d] + 3.0 * b[2] * dz[d] * d2z[d] + b[1] * d3z[d];
                    } else {
                        v = b[2] * dz[0] * dz[1] + b[1] * mz;
                    }
                    a[r] = v;
                }
                for (int o = 0; o < O; ++o) {
                    double acc = 0.0;
                    for (int r = 0; r < J; ++r) acc += gmul(gy[((long)r * O + o) * N + p], a[r], fmt);
                    dW[((long)o * I + j) * n + i] += acc;
                }
            }
        }
    }
    free(s); free(e);
    return 0;
}

/*
 * Input adjoint of one layer: gz = d/d(input jets) of
 * sum_p sum_r sum_o gy[r][o][p] * y_r[o][p], the chain rule of Section 3
 * reversed through the third derivative of Eq. 2.  With
 * dA_r[j][i] = sum_o gy[r][o] W[o][j][i] and v1, v2, v3 the derivatives:
 *   value row:        d/dz += dA_0 v1
 *   d-row (A = v1 z_d):  d/dz += dA_d v2 z_d,                d/dz_d += dA_d v1
 *   dd-row (A = v2 z_d^2 + v1 z_dd):
 *                     d/dz += dA_dd (v3 z_d^2 + v2 z_dd),   d/dz_d += dA_dd 2 v2 z_d,
 *                     d/dz_dd += dA_dd v1
 *   ddd-row (A = v3 z_d^3 + 3 v2 z_d z_dd + v1 z_ddd), through the fourth derivative v4:
 *                     d/dz += dA (v4 z_d^3 + 3 v3 z_d z_dd + v2 z_ddd),
 *                     d/dz_d += dA (3 v3 z_d^2 + 3 v2 z_dd),  d/dz_dd += dA 3 v2 z_d,
 *                     d/dz_ddd += dA v1
 *   01-row (A = v2 z_0 z_1 + v1 z_01):
 *                     d/dz += dA (v3 z_0 z_1 + v2 z_01),  d/dz_0 += dA v2 z_1,
 *                     d/dz_1 += dA v2 z_0,  d/dz_01 += dA v1
 *   fourth / fifth rows (A = R4 / R5): d/dz += dA R with v^(r) -> v^(r+1) (through
 *                     the sixth derivative), d/dz_d^(q) += dA dR/dg_q
 * fmt rounds gy and W before the FP64 sum over o (the reduced-precision
 * contraction's inputs; ORC_BF16X3 splits both, prod3); ORC_EXACT rounds nothing.  zin [J][I][N],
 * gy [J][O][N], gz [J][I][N] written.
 */
int orc_layer_adjoint(int I, int O, int G, int k, int m, double lo, double hi, const double* Wl,
                      const double* zin, const double* gy, long N, unsigned mask, double* gz, int fmt)
{
    const int D = 2;
    int rows[16];
    int J = mask_rows(mask, D, rows), higher = mask_higher(mask, D);
    if (!(mask & 1u)) return -1;
    int n = G + k;
    double* s = malloc(sizeof(double) * n);
    double* e = malloc(sizeof(double) * n);
    orc_support(G, k, lo, hi, s, e);
    for (long p = 0; p < N; ++p) {
        for (int j = 0; j < I; ++j) {
            double z = 0.0, dz[2] = {0.0, 0.0}, d2z[2] = {0.0, 0.0}, d3z[2] = {0.0, 0.0}, mz = 0.0;
            double d4z[2] = {0.0, 0.0}, d5z[2] = {0.0, 0.0};
            double* q[7] = {&z, dz, d2z, d3z, d4z, d5z, &mz};
            for (int r = 0; r < J; ++r) {
                int d, o = bit_order(rows[r], D, &d);
                double v = zin[((long)r * I + j) * N + p];
                if (o == 0 || o == 6) *q[o] = v;
                else q[o][d] = v;
            }
            double g_z = 0.0, g_d[2] = {0.0, 0.0}, g_dd[2] = {0.0, 0.0}, g_ddd[2] = {0.0, 0.0}, g_m = 0.0;
            double g_4[2] = {0.0, 0.0}, g_5[2] = {0.0, 0.0};
            for (int i = 0; i < n; ++i) {
                double b[5], f[7];
                orc_hr_basis(m, s[i], e[i], z, b);
                if (higher) orc_hr_basis6(m, s[i], e[i], z, f);
                for (int r = 0; r < J; ++r) {
                    double dA = 0.0;
                    for (int o = 0; o < O; ++o)
                        dA += wmul(Wl[((long)o * I + j) * n + i], gy[((long)r * O + o) * N + p], fmt);
                    int bit = rows[r], dd, ord = bit_order(bit, D, &dd);
                    if (ord == 4 || ord == 5) {
                        /* d/dz through v^(r+1); d/dz_d^(q) from the partials of R4 / R5 */
                        double g[6] = {0.0, dz[dd], d2z[dd], d3z[dd], d4z[dd], d5z[dd]}, dg[6];
                        g_z += dA * (ord == 4 ? row4(f + 1, g) : row5(f + 1, g));
                        if (ord == 4) row4_dg(f, g, dg);
                        else row5_dg(f, g, dg);
                        g_d[dd] += dA * dg[1];
                        g_dd[dd] += dA * dg[2];
                        g_ddd[dd] += dA * dg[3];
                        g_4[dd] += dA * dg[4];
                        g_5[dd] += dA * dg[5];
                    } else if (bit == 0) {
                        g_z += dA * b[1];
                    } else if (bit <= D) {
                        int d = bit - 1;
                        g_z += dA * b[2] * dz[d];
                        g_d[d] += dA * b[1];
                    } else if (bit <= 2 * D) {
                        int d = bit - 1 - D;
                        g_z += dA * (b[3] * dz[d] * dz[d] + b[2] * d2z[d]);
                        g_d[d] += dA * 2.0 * b[2] * dz[d];
                        g_dd[d] += dA * b[1];
                    } else if (bit <= 3 * D) {
                        int d = bit - 1 - 2 * D;
                        g_z += dA * (b[4] * dz[d] * dz[d] * dz[d] + 3.0 * b[3] * dz[d] * d2z[d] + b[2] * d3z[d]);
                        g_d[d] += dA * (3.0 * b[3] * dz[d] * dz[d] + 3.0 * b[2] * d2z[d]);
                        g_dd[d] += dA * 3.0 * b[2] * dz[d];
                        g_ddd[d] += dA * b[1];
                    } else {
                        g_z += dA * (b[3] * dz[0] * dz[1] + b[2] * mz);
                        g_d[0] += dA * b[2] * dz[1];
                        g_d[1] += dA * b[2] * dz[0];
                        g_m += dA * b[1];
                    }
                }
            }
            const double* by_order[7] = {&g_z, g_d, g_dd, g_ddd, g_4, g_5, &g_m};
            for (int r = 0; r < J; ++r) {
                int d, o = bit_order(rows[r], D, &d);
                gz[((long)r * I + j) * N + p] = (o == 0 || o == 6) ? *by_order[o] : by_order[o][d];
            }
        }
    }
    free(s); free(e);
    return 0;
}

/*
 * Reverse mode of point_forward.  g*, gd*, gd2* hold dL/d(output jets) of the
 * layer on entry and are overwritten with dL/d(input jets).  dW accumulates.
 */
static void layer_backward(const orc_net* net, int l, const double* Wl, double* dWl, int D,
                           const double* s, const double* e, const double* z,
                           const double* dz, const double* d2z, const double* d3z, const double* mz,
                           const double* d4z, const double* d5z,
                           const double* gy, const double* gdy, const double* gd2y, const double* gd3y,
                           const double* gmy, const double* gd4y, const double* gd5y,
                           double* gz, double* gdz, double* gd2z, double* gd3z, double* gmz, double* gd4z,
                           double* gd5z, int hi)
{
    int I = net->widths[l], O = net->widths[l + 1], n = orc_nbasis(net);
    for (int j = 0; j < I; ++j) {
        gz[j] = 0.0;
        gmz[j] = 0.0;
        for (int d = 0; d < D; ++d) gdz[j * D + d] = gd2z[j * D + d] = gd3z[j * D + d] = 0.0;
        for (int d = 0; d < D; ++d) gd4z[j * D + d] = gd5z[j * D + d] = 0.0;
    }
    for (int j = 0; j < I; ++j) {
        for (int i = 0; i < n; ++i) {
            double b[5], f[7];
            orc_hr_basis(net->m, s[i], e[i], z[j], b);
            if (hi) orc_hr_basis6(net->m, s[i], e[i], z[j], f);
            for (int o = 0; o < O; ++o) {
                long wi = ((long)o * I + j) * n + i;
                double w = Wl[wi];
                double gW = gy[o] * b[0];
                double acc_z = gy[o] * b[1];
                for (int d = 0; d < D; ++d) {
                    double zd = dz[j * D + d], zdd = d2z[j * D + d], zddd = d3z[j * D + d];
                    double g1 = gdy[o * D + d], g2 = gd2y[o * D + d], g3 = gd3y[o * D + d];
                    gW += g1 * b[1] * zd + g2 * (b[2] * zd * zd + b[1] * zdd)
                        + g3 * (b[3] * zd * zd * zd + 3.0 * b[2] * zd * zdd + b[1] * zddd);
                    acc_z += g1 * b[2] * zd + g2 * (b[3] * zd * zd + b[2] * zdd)
                           + g3 * (b[4] * zd * zd * zd + 3.0 * b[3] * zd * zdd + b[2] * zddd);
                    gdz[j * D + d] += w * (g1 * b[1] + g2 * 2.0 * b[2] * zd
                                           + g3 * (3.0 * b[3] * zd * zd + 3.0 * b[2] * zdd));
                    gd2z[j * D + d] += w * (g2 * b[1] + g3 * 3.0 * b[2] * zd);
                    gd3z[j * D + d] += w * g3 * b[1];
                }
                if (D == 2) {
                    double z0 = dz[j * D], z1 = dz[j * D + 1], gm = gmy[o];
                    gW += gm * (b[2] * z0 * z1 + b[1] * mz[j]);
                    acc_z += gm * (b[3] * z0 * z1 + b[2] * mz[j]);
                    gdz[j * D] += w * gm * b[2] * z1;
                    gdz[j * D + 1] += w * gm * b[2] * z0;
                    gmz[j] += w * gm * b[1];
                }
                if (hi)
                    for (int d = 0; d < D; ++d) {
                        int c = j * D + d;
                        double g[6] = {0.0, dz[c], d2z[c], d3z[c], d4z[c], d5z[c]}, p4[6], p5[6];
                        double g4 = gd4y[o * D + d], g5 = gd5y[o * D + d];
                        row4_dg(f, g, p4);
                        row5_dg(f, g, p5);
                        gW += g4 * row4(f, g) + g5 * row5(f, g);
                        acc_z += g4 * row4(f + 1, g) + g5 * row5(f + 1, g);
                        gdz[c] += w * (g4 * p4[1] + g5 * p5[1]);
                        gd2z[c] += w * (g4 * p4[2] + g5 * p5[2]);
                        gd3z[c] += w * (g4 * p4[3] + g5 * p5[3]);
                        gd4z[c] += w * (g4 * p4[4] + g5 * p5[4]);
                        gd5z[c] += w * g5 * p5[5];
                    }
                dWl[wi] += gW;
                gz[j] += w * acc_z;
            }
        }
    }
}

/*
 * dW (+)= d/dW sum_p sum_r dL_djets[r][p] * jets[r][p].
 * accumulate = 0 overwrites dW, 1 adds to it.
 */
int orc_backward(int n_widths, const int* widths, int G, int k, int m, double lo, double hi,
                 const double* W, const double* x, long N, unsigned mask, const double* dL_djets,
                 double* dW, int accumulate)
{
    orc_net net = {n_widths, widths, G, k, m, lo, hi};
    int D = widths[0], L = n_widths - 1;
    if (widths[L] != 1 || !(mask & 1u)) return -1;
    int rows[16];
    int J = mask_rows(mask, D, rows), higher = mask_higher(mask, D);
    int n = G + k;
    long P = orc_param_count(n_widths, widths, G, k);
    if (!accumulate) memset(dW, 0, sizeof(double) * P);
    double* s = malloc(sizeof(double) * n);
    double* e = malloc(sizeof(double) * n);
    orc_support(G, k, lo, hi, s, e);
    point_tape t;
    if (tape_alloc(&t, &net, D)) return -1;
    int w = t.stride;
    double *g = calloc(w, sizeof(double)), *gd = calloc((size_t)w * D, sizeof(double)),
           *gd2 = calloc((size_t)w * D, sizeof(double)), *gd3 = calloc((size_t)w * D, sizeof(double)),
           *gm = calloc(w, sizeof(double));
    double *h = calloc(w, sizeof(double)), *hd = calloc((size_t)w * D, sizeof(double)),
           *hd2 = calloc((size_t)w * D, sizeof(double)), *hd3 = calloc((size_t)w * D, sizeof(double)),
           *hm = calloc(w, sizeof(double));
    double *gd4 = calloc((size_t)w * D, sizeof(double)), *gd5 = calloc((size_t)w * D, sizeof(double)),
           *hd4 = calloc((size_t)w * D, sizeof(double)), *hd5 = calloc((size_t)w * D, sizeof(double));
    double xp[8];
    for (long p = 0; p < N; ++p) {
        for (int d = 0; d < D; ++d) xp[d] = x[(long)d * N + p];
        point_forward(&net, W, D, s, e, xp, &t, 0u, ORC_EXACT, higher);
        g[0] = 0.0;
        gm[0] = 0.0;
        for (int d = 0; d < D; ++d) gd[d] = gd2[d] = gd3[d] = gd4[d] = gd5[d] = 0.0;
        double* by_order[7] = {g, gd, gd2, gd3, gd4, gd5, gm};
        for (int r = 0; r < J; ++r) {
            int d, o = bit_order(rows[r], D, &d);
            by_order[o][(o == 0 || o == 6) ? 0 : d] = dL_djets[(long)r * N + p];
        }
        for (int l = L - 1; l >= 0; --l) {
            long off = layer_offset(&net, l), a = (long)l * w;
            layer_backward(&net, l, W + off, dW + off, D, s, e, t.z + a, t.dz + a * D, t.d2z + a * D,
                           t.d3z + a * D, t.mz + a, t.d4z + a * D, t.d5z + a * D,
                           g, gd, gd2, gd3, gm, gd4, gd5, h, hd, hd2, hd3, hm, hd4, hd5, higher);
            int I = widths[l];
            memcpy(g, h, sizeof(double) * I);
            memcpy(gm, hm, sizeof(double) * I);
            memcpy(gd, hd, sizeof(double) * I * D);
            memcpy(gd2, hd2, sizeof(double) * I * D);
            memcpy(gd3, hd3, sizeof(double) * I * D);
            memcpy(gd4, hd4, sizeof(double) * I * D);
            memcpy(gd5, hd5, sizeof(double) * I * D);
        }
    }
    free(g); free(gd); free(gd2); free(gd3); free(gm); free(h); free(hd); free(hd2); free(hd3); free(hm);
    free(gd4); free(gd5); free(hd4); free(hd5);
    tape_free(&t);
    free(s); free(e);
    return 0;
}

/* ------------------------------------------------------------------- loss */

enum { ORC_POISSON = 0, ORC_BURGERS = 1, ORC_KDV = 2, ORC_POISSON3 = 3 };

static int row_of(unsigned mask, int bit)
{
    if (!(mask & (1u << bit))) return -1;
    int r = 0;
    for (int b = 0; b < bit; ++b) if (mask & (1u << b)) ++r;
    return r;
}

/*
 * PDE residual and loss, D = 2 (D = 3 for the three-dimensional Poisson kind).
 *   Poisson (Eq. 3-4, generalised to u* = sin(a pi x) sin(b pi y)):
 *       r = u_xx + u_yy + (a^2+b^2) pi^2 sin(a pi x) sin(b pi y)
 *   Poisson in three dimensions (the same equation with a third coordinate z,
 *   u* = sin(a pi x) sin(b pi y) sin(c pi z), c passed in lam; x_int [3][N]):
 *       r = u_xx + u_yy + u_zz + (a^2+b^2+c^2) pi^2 sin(a pi x) sin(b pi y) sin(c pi z)
 *   Burgers (Eq. 6-8 form, coordinates (x, t)):
 *       r = u_t + lam u u_x - nu u_xx
 *   KdV (a third-order equation of the kind Section 3 picks a larger m for,
 *   coordinates (x, t)):
 *       r = u_t + lam u u_x + nu u_xxx
 *   L_pde = mean_int r^2, L_bnd = mean_bnd (u - g)^2 (pooled over all edges /
 *   initial points), L = alpha L_pde + L_bnd.
 * loss[0] = L, loss[1] = L_pde, loss[2] = L_bnd.
 * dL_djets_int has the layout of jets_int; dL_du_bnd[N_bnd].
 * Returns -1 if the mask lacks a row the residual needs.
 */
int orc_residual_loss(int kind, double a, double b, double lam, double nu, double alpha,
                      const double* x_int, long N_int, unsigned mask, const double* jets_int,
                      const double* u_bnd, const double* g_bnd, long N_bnd, double* loss,
                      double* dL_djets_int, double* dL_du_bnd)
{
    int D = kind == ORC_POISSON3 ? 3 : 2, rows[16];
    int J = mask_rows(mask, D, rows);
    double Lp = 0.0, Lb = 0.0;
    if (dL_djets_int) memset(dL_djets_int, 0, sizeof(double) * J * N_int);
    if (kind == ORC_POISSON3) {
        int rxx = row_of(mask, 1 + D + 0), ryy = row_of(mask, 1 + D + 1), rzz = row_of(mask, 1 + D + 2);
        if (rxx < 0 || ryy < 0 || rzz < 0) return -1;
        double c = lam;
        for (long p = 0; p < N_int; ++p) {
            double xx = x_int[p], yy = x_int[N_int + p], zz = x_int[2 * N_int + p];
            double f = (a * a + b * b + c * c) * ORC_PI * ORC_PI * sin(a * ORC_PI * xx) * sin(b * ORC_PI * yy) *
                       sin(c * ORC_PI * zz);
            double r = jets_int[(long)rxx * N_int + p] + jets_int[(long)ryy * N_int + p] +
                       jets_int[(long)rzz * N_int + p] + f;
            Lp += r * r;
            if (dL_djets_int) {
                double g = 2.0 * alpha * r / (double)N_int;
                dL_djets_int[(long)rxx * N_int + p] = g;
                dL_djets_int[(long)ryy * N_int + p] = g;
                dL_djets_int[(long)rzz * N_int + p] = g;
            }
        }
    } else if (kind == ORC_POISSON) {
        int rxx = row_of(mask, 1 + D + 0), ryy = row_of(mask, 1 + D + 1);
        if (rxx < 0 || ryy < 0) return -1;
        for (long p = 0; p < N_int; ++p) {
            double xx = x_int[p], yy = x_int[N_int + p];
            double f = (a * a + b * b) * ORC_PI * ORC_PI * sin(a * ORC_PI * xx) * sin(b * ORC_PI * yy);
            double r = jets_int[(long)rxx * N_int + p] + jets_int[(long)ryy * N_int + p] + f;
            Lp += r * r;
            if (dL_djets_int) {
                double g = 2.0 * alpha * r / (double)N_int;
                dL_djets_int[(long)rxx * N_int + p] = g;
                dL_djets_int[(long)ryy * N_int + p] = g;
            }
        }
    } else if (kind == ORC_BURGERS) {
        int ru = row_of(mask, 0), rx = row_of(mask, 1), rt = row_of(mask, 2),
            rxx = row_of(mask, 1 + D + 0);
        if (ru < 0 || rx < 0 || rt < 0 || rxx < 0) return -1;
        for (long p = 0; p < N_int; ++p) {
            double u = jets_int[(long)ru * N_int + p], ux = jets_int[(long)rx * N_int + p];
            double ut = jets_int[(long)rt * N_int + p], uxx = jets_int[(long)rxx * N_int + p];
            double r = ut + lam * u * ux - nu * uxx;
            Lp += r * r;
            if (dL_djets_int) {
                double g = 2.0 * alpha * r / (double)N_int;
                dL_djets_int[(long)rt * N_int + p] = g;
                dL_djets_int[(long)ru * N_int + p] = g * lam * ux;
                dL_djets_int[(long)rx * N_int + p] = g * lam * u;
                dL_djets_int[(long)rxx * N_int + p] = -g * nu;
            }
        }
    } else if (kind == ORC_KDV) {
        int ru = row_of(mask, 0), rx = row_of(mask, 1), rt = row_of(mask, 2),
            rxxx = row_of(mask, 1 + 2 * D + 0);
        if (ru < 0 || rx < 0 || rt < 0 || rxxx < 0) return -1;
        for (long p = 0; p < N_int; ++p) {
            double u = jets_int[(long)ru * N_int + p], ux = jets_int[(long)rx * N_int + p];
            double ut = jets_int[(long)rt * N_int + p], uxxx = jets_int[(long)rxxx * N_int + p];
            double r = ut + lam * u * ux + nu * uxxx;
            Lp += r * r;
            if (dL_djets_int) {
                double g = 2.0 * alpha * r / (double)N_int;
                dL_djets_int[(long)rt * N_int + p] = g;
                dL_djets_int[(long)ru * N_int + p] = g * lam * ux;
                dL_djets_int[(long)rx * N_int + p] = g * lam * u;
                dL_djets_int[(long)rxxx * N_int + p] = g * nu;
            }
        }
    } else {
        return -1;
    }
    for (long p = 0; p < N_bnd; ++p) {
        double d = u_bnd[p] - g_bnd[p];
        Lb += d * d;
        if (dL_du_bnd) dL_du_bnd[p] = 2.0 * d / (double)N_bnd;
    }
    Lp = N_int > 0 ? Lp / (double)N_int : 0.0;
    Lb = N_bnd > 0 ? Lb / (double)N_bnd : 0.0;
    loss[0] = alpha * Lp + Lb;
    loss[1] = Lp;
    loss[2] = Lb;
    return 0;
}

/* ------------------------------------------------------------------- adam */

/*
 * Bias-corrected Adam, step t >= 1:
 *   mom1 <- b1 mom1 + (1-b1) g,  mom2 <- b2 mom2 + (1-b2) g^2,
 *   W <- W - lr (mom1/(1-b1^t)) / (sqrt(mom2/(1-b2^t)) + eps)
 */
void orc_adam(long P, double* W, const double* g, double* mom1, double* mom2, double lr,
              double b1, double b2, double eps, int t)
{
    double c1 = 1.0 - pow(b1, t), c2 = 1.0 - pow(b2, t);
    for (long i = 0; i < P; ++i) {
        mom1[i] = b1 * mom1[i] + (1.0 - b1) * g[i];
        mom2[i] = b2 * mom2[i] + (1.0 - b2) * g[i] * g[i];
        W[i] -= lr * (mom1[i] / c1) / (sqrt(mom2[i] / c2) + eps);
    }
}

/* ------------------------------------------------------------- train step */

/*
 * One full-batch training step: forward jets at the interior and boundary
 * points, residual/loss, backward, Adam.  W, mom1, mom2 are updated in place;
 * loss[3] is the loss at the weights before the update; dW (may be NULL)
 * receives the gradient.
 */
int orc_train_step(int n_widths, const int* widths, int G, int k, int m, double lo, double hi,
                   int kind, double a, double b, double lam, double nu, double alpha,
                   double* W, double* mom1, double* mom2, const double* x_int, long N_int,
                   unsigned mask_int, const double* x_bnd, const double* g_bnd, long N_bnd,
                   double lr, double b1, double b2, double eps, int t, double* loss, double* dW)
{
    int D = widths[0], rows[16];
    int J = mask_rows(mask_int, D, rows);
    long P = orc_param_count(n_widths, widths, G, k);
    double* jets = malloc(sizeof(double) * (J * N_int + 1));
    double* gj = malloc(sizeof(double) * (J * N_int + 1));
    double* ub = malloc(sizeof(double) * (N_bnd + 1));
    double* gb = malloc(sizeof(double) * (N_bnd + 1));
    double* g = dW ? dW : malloc(sizeof(double) * P);
    int rc = 0;
    rc |= orc_forward(n_widths, widths, G, k, m, lo, hi, W, x_int, N_int, mask_int, jets);
    rc |= orc_forward(n_widths, widths, G, k, m, lo, hi, W, x_bnd, N_bnd, 1u, ub);
    if (!rc)
        rc |= orc_residual_loss(kind, a, b, lam, nu, alpha, x_int, N_int, mask_int, jets, ub,
                                g_bnd, N_bnd, loss, gj, gb);
    if (!rc) {
        rc |= orc_backward(n_widths, widths, G, k, m, lo, hi, W, x_int, N_int, mask_int, gj, g, 0);
        rc |= orc_backward(n_widths, widths, G, k, m, lo, hi, W, x_bnd, N_bnd, 1u, gb, g, 1);
    }
    if (!rc) orc_adam(P, W, g, mom1, mom2, lr, b1, b2, eps, t);
    free(jets); free(gj); free(ub); free(gb);
    if (!dW) free(g);
    return rc;
}

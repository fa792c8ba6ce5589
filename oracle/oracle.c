/*
 * oracle.c -- plain, slow FP64 reference for the loop nests the library
 * computes.  TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load it; the library never does.
 *
 * PENCIL (arXiv:1302.5586) defines a program's meaning as that of its
 * sequential execution (Sec. 2); each function here is that sequential loop nest,
 * written out without blocking, fusion or reordering, accumulated in FP64 from
 * inputs widened exactly.  Loops whose iterations are independent (the
 * `independent` directive of Sec. 2.2.3) run under `omp parallel for`; that
 * changes no result, since every output element is still computed by the same
 * sequence of operations.
 *
 * The paper never writes the convolution or the stencil down (it names image
 * processing and CFD as the domains, Sec. 1, and stencil computations as the
 * regular motif, Sec. 2).  The readings taken here:
 *   conv2d   out[i][j] = sum_a sum_b k[a][b] * in[clamp(i+a-kh/2)][clamp(j+b-kw/2)]
 *            -- correlation (no flip), anchor (kh/2, kw/2) in integer division,
 *            clamp-to-edge per axis (other border modes: see border_index),
 *            the same filter on every planar channel;
 *            bound[i][j] = sum_a sum_b |k[a][b]| * |in[...]|.
 *   jacobi   the 5-point average (up + down + left + right) / 4 on the interior,
 *            boundary ring fixed, two buffers (a Jacobi step, not Gauss-Seidel);
 *            a fixed number of sweeps stands for the sequential outer loop of
 *            `untilconverged` (Sec. 3.2).
 *   residual sqrt(sum over interior (4u - up - down - left - right)^2), unscaled,
 *            summed in row-major order (the `reduction` directive of Sec. 2.2.3
 *            over the interior points).
 *   binary16 IEEE 754-2008 binary16, round to nearest, ties to even.
 *
 * Parity pins: every function here is pinned by tests that do not use it
 * (library routines, closed forms, invariants, brute force on tiny inputs).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_DT_F32 0
#define ORACLE_DT_F16 1

int oracle_version(void) { return 1; }

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ---------------------------------------------------------------- binary16 */

/* Value of a binary16 bit pattern: sign, 5-bit biased exponent (bias 15),
 * 10-bit fraction; exponent 0 is zero/subnormal (fraction * 2^-24), exponent
 * 31 is infinity (fraction 0) or NaN. */
double oracle_f16_to_f64(uint16_t bits)
{
    int sign = (bits >> 15) & 1;
    int e = (bits >> 10) & 0x1f;
    int f = bits & 0x3ff;
    double v;
    if (e == 0)
        v = ldexp((double)f, -24);
    else if (e == 31)
        v = f ? NAN : INFINITY;
    else
        v = ldexp((double)(1024 + f), e - 25);
    return sign ? -v : v;
}

/* Round a double to the nearest binary16, ties to even.  The significand is
 * scaled by a power of two (exact) so that one integer step is one binary16
 * ulp, then rounded to an integer with rint() under the default
 * round-to-nearest-even mode. */
uint16_t oracle_f64_to_f16(double x)
{
    uint16_t sign = signbit(x) ? 0x8000 : 0;
    double a = fabs(x);
    if (isnan(x)) return (uint16_t)(sign | 0x7e00);
    if (isinf(a)) return (uint16_t)(sign | 0x7c00);
    if (a < ldexp(1.0, -14)) {
        /* subnormal range: ulp is 2^-24; q == 1024 lands on the smallest normal */
        double q = rint(ldexp(a, 24));
        return (uint16_t)(sign | (uint16_t)q);
    }
    int e2;
    frexp(a, &e2);               /* a = m * 2^e2, m in [0.5, 1) */
    int e = e2 - 1;              /* a in [2^e, 2^(e+1)) */
    double q = rint(ldexp(a, 10 - e)); /* in [1024, 2048] */
    if (q == 2048.0) { q = 1024.0; e += 1; }
    if (e > 15) return (uint16_t)(sign | 0x7c00);
    return (uint16_t)(sign | (uint16_t)((e + 15) << 10) | (uint16_t)((int)q - 1024));
}

void oracle_f16_to_f64_array(int64_t n, const uint16_t *in, double *out)
{
    for (int64_t i = 0; i < n; ++i) out[i] = oracle_f16_to_f64(in[i]);
}

void oracle_f64_to_f16_array(int64_t n, const double *in, uint16_t *out)
{
    for (int64_t i = 0; i < n; ++i) out[i] = oracle_f64_to_f16(in[i]);
}

/* ------------------------------------------------------------------ conv2d */

static int64_t clamp64(int64_t v, int64_t lo, int64_t hi)
{
    return v < lo ? lo : (v > hi ? hi : v);
}

/* Border modes: where index i of an axis of length n lands, or -1 for a
 * zero value.
 *   0 clamp   a a a | a b c d | d d d     (replicate the edge)
 *   1 zero    0 0 0 | a b c d | 0 0 0
 *   2 reflect c b a | a b c d | d c b     (edge repeated; period 2n)
 *   3 mirror  d c b | a b c d | c b a     (edge not repeated; period 2n-2)
 *   4 wrap    b c d | a b c d | a b c     (periodic; period n)  */
static int64_t border_index(int64_t i, int64_t n, int mode)
{
    if (i >= 0 && i < n) return i;
    switch (mode) {
    case 1: return -1;
    case 2: {
        int64_t p = 2 * n, j = ((i % p) + p) % p;
        return j < n ? j : p - 1 - j;
    }
    case 3: {
        if (n == 1) return 0;
        int64_t p = 2 * n - 2, j = ((i % p) + p) % p;
        return j < n ? j : p - j;
    }
    case 4: return ((i % n) + n) % n;
    default: return clamp64(i, 0, n - 1);
    }
}

static double load_px(const void *in, int dtype, int64_t idx)
{
    if (dtype == ORACLE_DT_F16) return oracle_f16_to_f64(((const uint16_t *)in)[idx]);
    return (double)((const float *)in)[idx];
}

/* One output pixel of one channel plane (base = first element of the plane);
 * window positions that the border mode maps to zero contribute nothing. */
static void conv_pixel(int64_t h, int64_t w, const void *in, int dtype, int64_t base,
                       int kh, int kw, const double *k, int64_t i, int64_t j,
                       double *out, double *bound, int mode)
{
    const int ah = kh / 2, aw = kw / 2;
    double s = 0.0, b = 0.0;
    for (int a = 0; a < kh; ++a) {
        const int64_t r = border_index(i + a - ah, h, mode);
        for (int bb = 0; bb < kw; ++bb) {
            const int64_t c = border_index(j + bb - aw, w, mode);
            const double x = (r < 0 || c < 0) ? 0.0 : load_px(in, dtype, base + r * w + c);
            const double wt = k[a * kw + bb];
            s += wt * x;
            b += fabs(wt) * fabs(x);
        }
    }
    *out = s;
    if (bound) *bound = b;
}

static void conv_planes(int64_t nc, int64_t h, int64_t w, const void *in, int dtype,
                        int kh, int kw, const double *k, double *out, double *bound, int mode)
{
    const int64_t rows = nc * h;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t cr = 0; cr < rows; ++cr) {
        const int64_t ch = cr / h, i = cr % h;
        const int64_t base = ch * h * w;
        for (int64_t j = 0; j < w; ++j)
            conv_pixel(h, w, in, dtype, base, kh, kw, k, i, j, out + base + i * w + j,
                       bound ? bound + base + i * w + j : NULL, mode);
    }
}

static double *widen_filter(int kh, int kw, const float *k)
{
    double *kd = (double *)malloc(sizeof(double) * (size_t)kh * (size_t)kw);
    if (!kd) return NULL;
    for (int t = 0; t < kh * kw; ++t) kd[t] = (double)k[t];
    return kd;
}

/* Direct correlation over nc planar channels with border mode `mode`
 * (0 clamp-to-edge, 1 zero, 2 reflect, 3 mirror, 4 wrap).
 * in: nc*h*w values (FP32 or binary16 bits), k: kh*kw FP32 weights row-major,
 * out/bound: nc*h*w doubles (bound may be NULL).  Returns 0, or -1 on bad
 * arguments or allocation failure. */
int oracle_conv2d_mode(int64_t nc, int64_t h, int64_t w, const void *in, int dtype,
                       int kh, int kw, const float *k, double *out, double *bound, int mode)
{
    if (nc < 0 || h <= 0 || w <= 0 || kh <= 0 || kw <= 0 || mode < 0 || mode > 4) return -1;
    double *kd = widen_filter(kh, kw, k);
    if (!kd) return -1;
    conv_planes(nc, h, w, in, dtype, kh, kw, kd, out, bound, mode);
    free(kd);
    return 0;
}

/* Clamp-to-edge correlation (mode 0). */
int oracle_conv2d(int64_t nc, int64_t h, int64_t w, const void *in, int dtype,
                  int kh, int kw, const float *k, double *out, double *bound)
{
    return oracle_conv2d_mode(nc, h, w, in, dtype, kh, kw, k, out, bound, 0);
}

/* Separable filter: the 2-D weight array is the outer product gy[a] * gx[b]
 * (formed in FP64, exact for FP32 taps); the result is the same direct
 * correlation as oracle_conv2d. */
int oracle_conv2d_sep(int64_t nc, int64_t h, int64_t w, const void *in, int dtype,
                      int kx, const float *gx, int ky, const float *gy,
                      double *out, double *bound)
{
    if (nc < 0 || h <= 0 || w <= 0 || kx <= 0 || ky <= 0) return -1;
    double *kd = (double *)malloc(sizeof(double) * (size_t)kx * (size_t)ky);
    if (!kd) return -1;
    for (int a = 0; a < ky; ++a)
        for (int b = 0; b < kx; ++b) kd[a * kx + b] = (double)gy[a] * (double)gx[b];
    conv_planes(nc, h, w, in, dtype, ky, kx, kd, out, bound, 0);
    free(kd);
    return 0;
}

/* The same definition evaluated at npts sampled pixels (ch, i, j) given as
 * int64 triples; used where the full image is too large to check. */
int oracle_conv2d_points(int64_t nc, int64_t h, int64_t w, const void *in, int dtype,
                         int kh, int kw, const float *k, int64_t npts, const int64_t *pts,
                         double *out, double *bound)
{
    if (nc <= 0 || h <= 0 || w <= 0 || kh <= 0 || kw <= 0 || npts < 0) return -1;
    double *kd = widen_filter(kh, kw, k);
    if (!kd) return -1;
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
    for (int64_t p = 0; p < npts; ++p) {
        const int64_t ch = pts[3 * p], i = pts[3 * p + 1], j = pts[3 * p + 2];
        if (ch < 0 || ch >= nc || i < 0 || i >= h || j < 0 || j >= w) { bad = 1; continue; }
        conv_pixel(h, w, in, dtype, ch * h * w, kh, kw, kd, i, j, out + p, bound ? bound + p : NULL, 0);
    }
    free(kd);
    return bad ? -1 : 0;
}

/* The separable definition (weights gy[a] * gx[b] in FP64) at sampled points. */
int oracle_conv2d_sep_points(int64_t nc, int64_t h, int64_t w, const void *in, int dtype,
                             int kx, const float *gx, int ky, const float *gy, int64_t npts,
                             const int64_t *pts, double *out, double *bound)
{
    if (nc <= 0 || h <= 0 || w <= 0 || kx <= 0 || ky <= 0 || npts < 0) return -1;
    double *kd = (double *)malloc(sizeof(double) * (size_t)kx * (size_t)ky);
    if (!kd) return -1;
    for (int a = 0; a < ky; ++a)
        for (int b = 0; b < kx; ++b) kd[a * kx + b] = (double)gy[a] * (double)gx[b];
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
    for (int64_t p = 0; p < npts; ++p) {
        const int64_t ch = pts[3 * p], i = pts[3 * p + 1], j = pts[3 * p + 2];
        if (ch < 0 || ch >= nc || i < 0 || i >= h || j < 0 || j >= w) { bad = 1; continue; }
        conv_pixel(h, w, in, dtype, ch * h * w, ky, kx, kd, i, j, out + p, bound ? bound + p : NULL, 0);
    }
    free(kd);
    return bad ? -1 : 0;
}

/* ------------------------------------------------- interleaved [h][w][c] */

/* The interleaved layout image DSLs hand over (pixels of nc channels side by
 * side, Sec. 1): channel ch of pixel (i, j) is element (i*w + j)*nc + ch.  The
 * definition is the planar one with that address: each channel is correlated
 * with k on its own, and the border mode acts on pixel rows and columns. */
static void conv_pixel_hwc(int64_t nc, int64_t h, int64_t w, const void *in, int dtype, int64_t ch,
                           int kh, int kw, const double *k, int64_t i, int64_t j,
                           double *out, double *bound, int mode)
{
    const int ah = kh / 2, aw = kw / 2;
    double s = 0.0, b = 0.0;
    for (int a = 0; a < kh; ++a) {
        const int64_t r = border_index(i + a - ah, h, mode);
        for (int bb = 0; bb < kw; ++bb) {
            const int64_t c = border_index(j + bb - aw, w, mode);
            const double x = (r < 0 || c < 0) ? 0.0 : load_px(in, dtype, (r * w + c) * nc + ch);
            const double wt = k[a * kw + bb];
            s += wt * x;
            b += fabs(wt) * fabs(x);
        }
    }
    *out = s;
    if (bound) *bound = b;
}

static void conv_hwc(int64_t nc, int64_t h, int64_t w, const void *in, int dtype,
                     int kh, int kw, const double *k, double *out, double *bound, int mode)
{
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t i = 0; i < h; ++i)
        for (int64_t j = 0; j < w; ++j)
            for (int64_t ch = 0; ch < nc; ++ch) {
                const int64_t o = (i * w + j) * nc + ch;
                conv_pixel_hwc(nc, h, w, in, dtype, ch, kh, kw, k, i, j, out + o, bound ? bound + o : NULL,
                               mode);
            }
}

/* Direct correlation of an interleaved [h][w][nc] image (FP32 or binary16
 * bits) under border mode `mode`; out/bound: h*w*nc doubles in the same
 * layout (bound may be NULL).  Returns 0, or -1 on bad arguments. */
int oracle_conv2d_hwc(int64_t nc, int64_t h, int64_t w, const void *in, int dtype,
                      int kh, int kw, const float *k, double *out, double *bound, int mode)
{
    if (nc <= 0 || h <= 0 || w <= 0 || kh <= 0 || kw <= 0 || mode < 0 || mode > 4) return -1;
    double *kd = widen_filter(kh, kw, k);
    if (!kd) return -1;
    conv_hwc(nc, h, w, in, dtype, kh, kw, kd, out, bound, mode);
    free(kd);
    return 0;
}

/* Separable weights gy[a] * gx[b] (FP64) on an interleaved image. */
int oracle_conv2d_sep_hwc(int64_t nc, int64_t h, int64_t w, const void *in, int dtype,
                          int kx, const float *gx, int ky, const float *gy,
                          double *out, double *bound, int mode)
{
    if (nc <= 0 || h <= 0 || w <= 0 || kx <= 0 || ky <= 0 || mode < 0 || mode > 4) return -1;
    double *kd = (double *)malloc(sizeof(double) * (size_t)kx * (size_t)ky);
    if (!kd) return -1;
    for (int a = 0; a < ky; ++a)
        for (int b = 0; b < kx; ++b) kd[a * kx + b] = (double)gy[a] * (double)gx[b];
    conv_hwc(nc, h, w, in, dtype, ky, kx, kd, out, bound, mode);
    free(kd);
    return 0;
}

/* The interleaved definition at sampled (ch, i, j) points. */
int oracle_conv2d_hwc_points(int64_t nc, int64_t h, int64_t w, const void *in, int dtype,
                             int kh, int kw, const float *k, int64_t npts, const int64_t *pts,
                             double *out, double *bound)
{
    if (nc <= 0 || h <= 0 || w <= 0 || kh <= 0 || kw <= 0 || npts < 0) return -1;
    double *kd = widen_filter(kh, kw, k);
    if (!kd) return -1;
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
    for (int64_t p = 0; p < npts; ++p) {
        const int64_t ch = pts[3 * p], i = pts[3 * p + 1], j = pts[3 * p + 2];
        if (ch < 0 || ch >= nc || i < 0 || i >= h || j < 0 || j >= w) { bad = 1; continue; }
        conv_pixel_hwc(nc, h, w, in, dtype, ch, kh, kw, kd, i, j, out + p, bound ? bound + p : NULL, 0);
    }
    free(kd);
    return bad ? -1 : 0;
}

/* ------------------------------------------------------- Jacobi + residual */

/* sqrt(sum over interior points of (4u - up - down - left - right)^2), summed
 * in row-major order.  Grids with no interior give 0. */
double oracle_residual2d_f64(int64_t h, int64_t w, const double *u)
{
    double acc = 0.0;
    for (int64_t i = 1; i + 1 < h; ++i)
        for (int64_t j = 1; j + 1 < w; ++j) {
            const double r = 4.0 * u[i * w + j] - u[(i - 1) * w + j] - u[(i + 1) * w + j]
                             - u[i * w + j - 1] - u[i * w + j + 1];
            acc += r * r;
        }
    return sqrt(acc);
}

/* The same residual of an FP32 grid, each value widened exactly. */
double oracle_residual2d_f32(int64_t h, int64_t w, const float *u)
{
    double acc = 0.0;
    for (int64_t i = 1; i + 1 < h; ++i)
        for (int64_t j = 1; j + 1 < w; ++j) {
            const double r = 4.0 * (double)u[i * w + j] - (double)u[(i - 1) * w + j]
                             - (double)u[(i + 1) * w + j] - (double)u[i * w + j - 1]
                             - (double)u[i * w + j + 1];
            acc += r * r;
        }
    return sqrt(acc);
}

/* One Jacobi sweep: v = average of the 4 neighbours of u on the interior,
 * boundary ring copied. */
static void jacobi_sweep(int64_t h, int64_t w, const double *u, double *v)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < h; ++i)
        for (int64_t j = 0; j < w; ++j) {
            const int64_t p = i * w + j;
            if (i == 0 || j == 0 || i == h - 1 || j == w - 1)
                v[p] = u[p];
            else
                v[p] = (u[p - w] + u[p + w] + u[p - 1] + u[p + 1]) / 4.0;
        }
}

/* iters sweeps applied to u in place (FP64).  When check_every > 0 the
 * residual of the iterate after sweep m*check_every is written to
 * res[m-1], m = 1 .. iters/check_every.  Returns 0, or -1 on bad arguments
 * or allocation failure. */
int oracle_jacobi2d(int64_t h, int64_t w, double *u, int iters, int check_every, double *res)
{
    if (h <= 0 || w <= 0 || iters < 0 || check_every < 0) return -1;
    double *v = (double *)malloc(sizeof(double) * (size_t)h * (size_t)w);
    if (!v) return -1;
    double *cur = u, *nxt = v;
    for (int s = 1; s <= iters; ++s) {
        jacobi_sweep(h, w, cur, nxt);
        double *t = cur; cur = nxt; nxt = t;
        if (check_every > 0 && s % check_every == 0)
            res[s / check_every - 1] = oracle_residual2d_f64(h, w, cur);
    }
    if (cur != u) memcpy(u, cur, sizeof(double) * (size_t)h * (size_t)w);
    free(v);
    return 0;
}

/* Red-black successive over-relaxation: one sweep updates, in place, first
 * the interior points with (i + j) even, then those with (i + j) odd, each as
 * u <- u + omega * ((up + down + left + right) / 4 - u), the odd points seeing
 * the new even values.  omega = 1 is red-black Gauss-Seidel.  Residuals as in
 * oracle_jacobi2d.  Returns 0, or -1 on bad arguments. */
int oracle_rbsor2d(int64_t h, int64_t w, double *u, int iters, double omega, int check_every,
                   double *res)
{
    if (h <= 0 || w <= 0 || iters < 0 || check_every < 0) return -1;
    for (int s = 1; s <= iters; ++s) {
        for (int color = 0; color < 2; ++color)
            for (int64_t i = 1; i + 1 < h; ++i)
                for (int64_t j = 1; j + 1 < w; ++j) {
                    if (((i + j) & 1) != color) continue;
                    const int64_t p = i * w + j;
                    const double avg = (u[p - w] + u[p + w] + u[p - 1] + u[p + 1]) / 4.0;
                    u[p] = u[p] + omega * (avg - u[p]);
                }
        if (check_every > 0 && s % check_every == 0)
            res[s / check_every - 1] = oracle_residual2d_f64(h, w, u);
    }
    return 0;
}

/* Indirect increment over an edge set (the OP2 loop of Sec. 3.1): for every
 * edge i in increasing order, the cells e2c[2i+1] and then e2c[2i] (in that
 * order) are each incremented by edge[i].  Sequential, in FP64.  Returns 0,
 * or -1 on an index outside [0, ncells). */
int oracle_op2_inc(int64_t ncells, int64_t nedges, const int32_t *e2c, const double *edge,
                   double *cell)
{
    for (int64_t i = 0; i < nedges; ++i) {
        const int32_t c1 = e2c[2 * i + 1], c0 = e2c[2 * i];
        if (c0 < 0 || c1 < 0 || c0 >= ncells || c1 >= ncells) return -1;
        cell[c1] += edge[i];
        cell[c0] += edge[i];
    }
    return 0;
}

/*
 * oracle.c -- plain FP64 reference of the w-stacking imaging path described in
 * De Rubeis et al., "Accelerating radio astronomy imaging with RICK" (§2).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark load this library.  It shares no code, header,
 * table or constant with the CUDA library; the two never call each other.
 *
 * Everything here is written for a reader checking it against the paper:
 * straight loops in the order the method states, complex128 arithmetic, no
 * blocking, no fusion.  OpenMP is used only over independent rows/pixels/
 * visibilities where the loop body does not depend on the iteration order.
 *
 * Readings of the paper that this file fixes (the paper is silent on them):
 *  - grid index i <-> u = (i - n/2)/fov, pixel p <-> l = (p - n/2) fov/n;
 *  - x = fma(u, fov, n/2) (one rounding); odd W: centre cell c = floor(x+1/2),
 *    even W: c = floor(x); footprint corner a = c - h; offsets d_j = (j-h) - (x-c);
 *    a footprint that leaves the grid drops the visibility;
 *  - w-planes: n_w equal bins over [w_min, w_max], boundaries
 *    b_j = fma(j, dw, w_min), plane k = #{j >= 1 : w >= b_j}, centre
 *    w_k = fma(k + 1/2, dw, w_min) ("closest w-plane", §2); dw == 0 -> k = 0,
 *    w_k = w_min;
 *  - separable 2D kernel G(d_x) G(d_y) in (u,v) (Eq. 3 with the closest plane in w);
 *  - taper correction C(nu) = integral_{-W/2}^{W/2} G(d) cos(2 pi nu d) dd,
 *    nu = (p - n/2)/n, C == 1 for W == 1;
 *  - image = Re(sum_k F_k e^{2 pi i w_k (n-1)}) * [n] / (C C) / [sum w]  (Eq. 2,
 *    the w-integral becoming the sum over planes and (w_max - w_min) the weight sum);
 *  - grid padding (not in the paper, whose mesh equals the image): the n x n
 *    image is computed as above and its central m x m pixels are kept, pixel
 *    p' of the crop being pixel p' + (n - m)/2 of the grid frame (m even, so
 *    the phase centre n/2 becomes m/2); the adjoint zero-pads.
 * Parity status: every function below is pinned by the CPU tests (closed forms,
 * the brute-force DFT of Eq. 1, Hermitian and weight-sum invariants, adjoint
 * identity); none is "parity unpinned".
 */
#include <complex.h>
#include <math.h>
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

enum { OR_GAUSS = 0, OR_KB = 1 };
enum { OR_N_CORRECT = 1u, OR_NORMALIZE = 2u, OR_N_DIVIDE = 4u };

typedef struct {
    int32_t n;           /* grid side == image side (cells == pixels)          */
    int32_t n_w;         /* number of w-planes                                 */
    double fov;          /* image side in direction-cosine units               */
    double w_min, w_max; /* w range in wavelengths; NaN -> exact data min/max */
    int32_t kernel;      /* OR_GAUSS / OR_KB                                   */
    int32_t support;     /* W, cells                                           */
    double kb_beta;      /* KB shape; NaN -> default                           */
    double gauss_sigma;  /* Gaussian sigma in cells; NaN -> W/6                */
    int32_t tile;        /* uv-tile side T used for the binning key            */
    uint32_t flags;      /* unused by the oracle's geometry; kept for layout   */
    int32_t image_n;     /* side m of the image kept: the central m x m pixels */
                         /*   of the n x n w-stacked image (grid padding by    */
                         /*   n/m); 0 -> n, no crop                            */
    int32_t reserved_;   /* 0                                                  */
} or_params;

/* ------------------------------------------------------------------------ */
/* Kernel G (§2: "the G kernel is a Kaiser-Bessel function", Jackson 1991).  */

/* Modified Bessel function I0 by its power series sum_j (x^2/4)^j / (j!)^2,
 * summed until the terms stop changing the sum. */
double or_i0(double x)
{
    double q = 0.25 * x * x, term = 1.0, sum = 1.0;
    for (int j = 1; j < 1000; ++j) {
        term *= q / ((double)j * (double)j);
        sum += term;
        if (term < 1e-18 * sum) break;
    }
    return sum;
}

/* KB shape for grid oversampling alpha (Beatty, Nishimura & Pauly 2005):
 * beta = pi sqrt((W / alpha)^2 (alpha - 1/2)^2 - 0.8), which puts the first zero
 * of the kernel's transform just beyond the first alias of the image edge. */
double or_kb_beta(int32_t W, double alpha)
{
    double t = (W / alpha) * (W / alpha) * (alpha - 0.5) * (alpha - 0.5) - 0.8;
    return M_PI * sqrt(t);
}

/* Default KB shape: Beatty's choice for oversampling 2. */
double or_kb_beta_default(int32_t W)
{
    return or_kb_beta(W, 2.0);
}

static double or_beta(const or_params *p)
{
    return isnan(p->kb_beta) ? or_kb_beta_default(p->support) : p->kb_beta;
}

static double or_sigma(const or_params *p)
{
    return isnan(p->gauss_sigma) ? p->support / 6.0 : p->gauss_sigma;
}

/* G(d), d in cells, peak 1 at d = 0, zero outside |d| <= W/2; W == 1 is the
 * nearest-cell delta (G == 1 on the single cell). */
double or_kernel(const or_params *p, double d)
{
    int W = p->support;
    if (W == 1) return 1.0;
    if (fabs(d) > 0.5 * W) return 0.0;
    if (p->kernel == OR_GAUSS) {
        double s = or_sigma(p);
        return exp(-d * d / (2.0 * s * s));
    }
    double beta = or_beta(p), t = 2.0 * d / W;
    return or_i0(beta * sqrt(1.0 - t * t)) / or_i0(beta);
}

/* ------------------------------------------------------------------------ */
/* Taper correction: the continuous Fourier transform of G, by adaptive       */
/* Gauss-Legendre quadrature.                                                */

#define OR_GL 16
static double or_gl_x[OR_GL], or_gl_w[OR_GL];
static int or_gl_ready = 0;

/* Gauss-Legendre nodes/weights on [-1, 1]: Newton iteration on P_n, with P_n
 * from the three-term recurrence and P_n' = n (x P_n - P_{n-1}) / (x^2 - 1). */
static void or_gl_init(void)
{
    if (or_gl_ready) return;
    int n = OR_GL;
    for (int i = 0; i < n; ++i) {
        double x = cos(M_PI * (i + 0.75) / (n + 0.5)), dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = x;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (x * p1 - p0) / (x * x - 1.0);
            double dx = p1 / dp;
            x -= dx;
            if (fabs(dx) < 1e-16) break;
        }
        or_gl_x[i] = x;
        or_gl_w[i] = 2.0 / ((1.0 - x * x) * dp * dp);
    }
    or_gl_ready = 1;
}

static double or_taper_integrand(const or_params *p, double nu, double d)
{
    return or_kernel(p, d) * cos(2.0 * M_PI * nu * d);
}

static double or_gl_rule(const or_params *p, double nu, double a, double b)
{
    double h = 0.5 * (b - a), m = 0.5 * (a + b), s = 0.0;
    for (int i = 0; i < OR_GL; ++i) s += or_gl_w[i] * or_taper_integrand(p, nu, m + h * or_gl_x[i]);
    return s * h;
}

static double or_adapt(const or_params *p, double nu, double a, double b, double whole, int depth)
{
    double m = 0.5 * (a + b);
    double left = or_gl_rule(p, nu, a, m), right = or_gl_rule(p, nu, m, b);
    if (depth <= 0 || fabs(left + right - whole) <= 1e-15 * (fabs(left + right) + 1e-300))
        return left + right;
    return or_adapt(p, nu, a, m, left, depth - 1) + or_adapt(p, nu, m, b, right, depth - 1);
}

/* C(nu) = integral_{-W/2}^{W/2} G(d) cos(2 pi nu d) dd  (C == 1 when W == 1). */
double or_taper(const or_params *p, double nu)
{
    if (p->support == 1) return 1.0;
    or_gl_init();
    double h = 0.5 * p->support;
    return or_adapt(p, nu, -h, h, or_gl_rule(p, nu, -h, h), 30);
}

/* ------------------------------------------------------------------------ */
/* FFT: iterative radix-2 Cooley-Tukey (1965), unnormalised,                 */
/* out[k] = sum_j in[j] e^{sign 2 pi i j k / n}.                             */

static void or_fft1(double complex *a, int n, const double complex *tw)
{
    for (int i = 1, j = 0; i < n; ++i) {  /* bit-reversal permutation */
        int bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) {
            double complex t = a[i];
            a[i] = a[j];
            a[j] = t;
        }
    }
    for (int len = 2; len <= n; len <<= 1) {
        int half = len >> 1, step = n / len;
        for (int i = 0; i < n; i += len)
            for (int j = 0; j < half; ++j) {
                double complex w = tw[j * step];
                double complex x = a[i + j], y = a[i + j + half] * w;
                a[i + j] = x + y;
                a[i + j + half] = x - y;
            }
    }
}

/* Twiddles tw[j] = e^{sign 2 pi i j / n}, each from cos/sin of its own angle. */
static double complex *or_twiddles(int n, int sign)
{
    double complex *tw = malloc(sizeof(double complex) * (size_t)(n / 2 + 1));
    for (int j = 0; j <= n / 2; ++j) {
        double ang = 2.0 * M_PI * (double)j / (double)n;
        tw[j] = cos(ang) + I * (sign * sin(ang));
    }
    return tw;
}

/* 1D transform exported for the FFT pins. */
void or_fft1d(double complex *a, int32_t n, int32_t sign)
{
    double complex *tw = or_twiddles(n, sign);
    or_fft1(a, n, tw);
    free(tw);
}

/* 2D transform of an n x n row-major array: rows, then columns. */
void or_fft2d(double complex *a, int32_t n, int32_t sign)
{
    double complex *tw = or_twiddles(n, sign);
#pragma omp parallel for schedule(static)
    for (int r = 0; r < n; ++r) or_fft1(a + (size_t)r * n, n, tw);
#pragma omp parallel
    {
        double complex *col = malloc(sizeof(double complex) * (size_t)n);
#pragma omp for schedule(static)
        for (int c = 0; c < n; ++c) {
            for (int r = 0; r < n; ++r) col[r] = a[(size_t)r * n + c];
            or_fft1(col, n, tw);
            for (int r = 0; r < n; ++r) a[(size_t)r * n + c] = col[r];
        }
        free(col);
    }
    free(tw);
}

/* ------------------------------------------------------------------------ */
/* Geometry of one visibility: grid coordinates, footprint, w-plane.         */

/* Exact min / max of the finite w over all input visibilities (0, 0 if none). */
void or_wrange(int64_t nvis, const double *uvw, double *wmin, double *wmax)
{
    double lo = INFINITY, hi = -INFINITY;
    for (int64_t i = 0; i < nvis; ++i) {
        double w = uvw[3 * i + 2];
        if (!isfinite(w)) continue;
        if (w < lo) lo = w;
        if (w > hi) hi = w;
    }
    if (lo > hi) lo = hi = 0.0;
    *wmin = lo == 0.0 ? 0.0 : lo; /* -0 -> +0 */
    *wmax = hi == 0.0 ? 0.0 : hi;
}

/* One axis: returns 1 and the footprint corner a and fractional offset x - c
 * when the W-cell footprint lies inside [0, n-1], else 0. */
static int or_axis(const or_params *p, double u, int32_t *a, double *frac)
{
    int W = p->support, n = p->n;
    int h = (W % 2) ? (W - 1) / 2 : W / 2 - 1;
    double x = fma(u, p->fov, 0.5 * n);
    if (!(x >= -1.0 && x <= n + 1.0)) return 0; /* also rejects NaN */
    double fl = floor(x), c = fl;
    if ((W % 2) && x - fl >= 0.5) c = fl + 1.0; /* c = floor(x + 1/2) */
    long a0 = (long)c - h;
    if (a0 < 0 || a0 + W - 1 > n - 1) return 0;
    *a = (int32_t)a0;
    *frac = x - c;
    return 1;
}

static double or_dw(const or_params *p, double wmin, double wmax)
{
    return (wmax - wmin) / p->n_w;
}

/* Closest plane: k = number of inner boundaries b_j = fma(j, dw, wmin) <= w. */
static int32_t or_plane_of(const or_params *p, double w, double wmin, double dw)
{
    if (dw == 0.0) return 0;
    int32_t k = 0;
    for (int j = 1; j < p->n_w; ++j)
        if (w >= fma((double)j, dw, wmin)) k = j;
    return k;
}

double or_plane_centre(const or_params *p, int32_t k, double wmin, double wmax)
{
    double dw = or_dw(p, wmin, wmax);
    if (dw == 0.0) return wmin;
    return fma(k + 0.5, dw, wmin);
}

/* Per-visibility geometry.  status: 0 kept, 1 dropped (footprint off the
 * grid, or u / v not finite), 2 dropped (w not finite, or outside a
 * user-given range).  Returns the kept count. */
int64_t or_coords(const or_params *p, int64_t nvis, const double *uvw, double wmin, double wmax,
                  int32_t given_range, int32_t *plane, int32_t *ax, int32_t *ay, double *fx,
                  double *fy, int32_t *status)
{
    double dw = or_dw(p, wmin, wmax);
    int64_t kept = 0;
    for (int64_t i = 0; i < nvis; ++i) {
        double u = uvw[3 * i], v = uvw[3 * i + 1], w = uvw[3 * i + 2];
        plane[i] = -1;
        ax[i] = ay[i] = -1;
        fx[i] = fy[i] = 0.0;
        if (!or_axis(p, u, &ax[i], &fx[i]) || !or_axis(p, v, &ay[i], &fy[i])) {
            ax[i] = ay[i] = -1;
            fx[i] = fy[i] = 0.0;
            status[i] = 1;
            continue;
        }
        if (!isfinite(w) || (given_range && !(w >= wmin && w <= wmax))) {
            ax[i] = ay[i] = -1;
            fx[i] = fy[i] = 0.0;
            status[i] = 2;
            continue;
        }
        plane[i] = or_plane_of(p, w, wmin, dw);
        status[i] = 0;
        ++kept;
    }
    return kept;
}

/* ------------------------------------------------------------------------ */
/* Binning (§2 gridding sub-step 1, "an array ... for each slab"), here by    */
/* (w-plane, uv-tile of the footprint corner, edge class).  The edge class   */
/* says which neighbouring tiles the footprint reaches: 0 none, 1 east only, */
/* 2 east and south, 3 south only.  The permutation is a stable counting     */
/* sort by key; offsets are the exclusive prefix sum of the bin counts.      */

int64_t or_nbins(const or_params *p)
{
    int64_t nt = p->n / p->tile;
    return 4 * (int64_t)p->n_w * nt * nt;
}

void or_bin(const or_params *p, int64_t nvis, const int32_t *plane, const int32_t *ax,
            const int32_t *ay, const int32_t *status, int32_t *key, int64_t *perm, int64_t *offsets)
{
    int64_t T = p->tile, nt = p->n / p->tile, W = p->support, nb = or_nbins(p);
    for (int64_t i = 0; i < nvis; ++i) {
        if (status[i] != 0) {
            key[i] = -1;
            continue;
        }
        int64_t tx = ax[i] / T, ty = ay[i] / T;
        int ex = (ax[i] % T) > T - W, ey = (ay[i] % T) > T - W;
        int cls = ex ? (ey ? 2 : 1) : (ey ? 3 : 0);
        key[i] = (int32_t)(((plane[i] * nt + ty) * nt + tx) * 4 + cls);
    }
    int64_t *count = calloc((size_t)nb + 1, sizeof(int64_t));
    for (int64_t i = 0; i < nvis; ++i)
        if (key[i] >= 0) count[key[i]]++;
    offsets[0] = 0;
    for (int64_t b = 0; b < nb; ++b) offsets[b + 1] = offsets[b] + count[b];
    memset(count, 0, sizeof(int64_t) * (size_t)nb);
    for (int64_t i = 0; i < nvis; ++i)
        if (key[i] >= 0) perm[offsets[key[i]] + count[key[i]]++] = i;
    free(count);
}

/* ------------------------------------------------------------------------ */
/* Shared helpers of the image pipeline.                                     */

/* n - 1 = -(l^2 + m^2) / (1 + sqrt(1 - l^2 - m^2)), the cancellation-free form. */
static double or_nm1(double l, double m)
{
    double r2 = l * l + m * m;
    return -r2 / (1.0 + sqrt(1.0 - r2));
}

/* Side m of the image kept and its offset (n - m)/2 in the grid frame. */
static int or_image_side(const or_params *p)
{
    return p->image_n > 0 ? p->image_n : p->n;
}

/* The taper along one axis of the grid frame: tap[i] = C((i - n/2) / n).
 * The row depends only on the kernel and n; the last one computed is kept
 * and handed out again for the same kernel and n (the quadrature of a
 * Kaiser-Bessel kernel to 1e-15 costs milliseconds per value). */
static double *or_tap_last;
static uint64_t or_tap_key[5];

void or_taper_row(const or_params *p, double *tap)
{
    int n = p->n;
    uint64_t key[5];
    double kb = or_beta(p), sg = or_sigma(p);
    key[0] = (uint64_t)(uint32_t)p->kernel;
    key[1] = (uint64_t)(uint32_t)p->support;
    key[2] = (uint64_t)(uint32_t)n;
    memcpy(&key[3], &kb, 8);
    memcpy(&key[4], &sg, 8);
    int hit = 0;
#pragma omp critical(or_tap)
    if (or_tap_last && memcmp(key, or_tap_key, sizeof key) == 0) {
        memcpy(tap, or_tap_last, sizeof(double) * (size_t)n);
        hit = 1;
    }
    if (hit) return;
    or_gl_init(); /* the quadrature nodes, before the threads read them */
#pragma omp parallel for schedule(dynamic, 8)
    for (int i = 0; i < n; ++i) tap[i] = or_taper(p, (double)(i - n / 2) / n);
#pragma omp critical(or_tap)
    {
        free(or_tap_last);
        or_tap_last = malloc(sizeof(double) * (size_t)n);
        memcpy(or_tap_last, tap, sizeof(double) * (size_t)n);
        memcpy(or_tap_key, key, sizeof key);
    }
}

/* Pixel scale s(p,q) = [n] [1/n] [1/sum w] / (C(nu_p) C(nu_q)). */
static void or_scale_plane(const or_params *p, uint32_t flags, double sumw, double *scale)
{
    int n = p->n;
    double dl = p->fov / n;
    double *tap = malloc(sizeof(double) * (size_t)n);
    or_taper_row(p, tap);
#pragma omp parallel for schedule(static)
    for (int q = 0; q < n; ++q)
        for (int pp = 0; pp < n; ++pp) {
            double l = (pp - n / 2) * dl, m = (q - n / 2) * dl;
            double nn = sqrt(1.0 - l * l - m * m), s = 1.0 / (tap[pp] * tap[q]);
            if (flags & OR_N_CORRECT) s *= nn;
            if (flags & OR_N_DIVIDE) s /= nn;
            if ((flags & OR_NORMALIZE) && sumw != 0.0) s /= sumw; /* nothing gridded: no scaling */
            scale[(size_t)q * n + pp] = s;
        }
    free(tap);
}

/* Kernel weights of one visibility along one axis: G(d_j), d_j = (j - h) - frac. */
static void or_axis_weights(const or_params *p, double frac, double *g)
{
    int W = p->support, h = (W % 2) ? (W - 1) / 2 : W / 2 - 1;
    for (int j = 0; j < W; ++j) g[j] = or_kernel(p, (double)(j - h) - frac);
}

/* Indices of the kept visibilities of each plane, in input order. */
static int64_t *or_plane_lists(const or_params *p, int64_t nvis, const int32_t *plane, int64_t *start)
{
    int64_t *idx = malloc(sizeof(int64_t) * (size_t)(nvis + 1));
    for (int k = 0; k <= p->n_w; ++k) start[k] = 0;
    for (int64_t i = 0; i < nvis; ++i)
        if (plane[i] >= 0) start[plane[i] + 1]++;
    for (int k = 0; k < p->n_w; ++k) start[k + 1] += start[k];
    int64_t *fill = calloc((size_t)(p->n_w > 0 ? p->n_w : 1), sizeof(int64_t));
    for (int64_t i = 0; i < nvis; ++i)
        if (plane[i] >= 0) idx[start[plane[i]] + fill[plane[i]]++] = i;
    free(fill);
    return idx;
}

typedef struct {
    int32_t *plane, *ax, *ay, *status;
    double *fx, *fy;
    double wmin, wmax, sumw;
    int64_t kept;
} or_geom;

static void or_geom_build(const or_params *p, int64_t nvis, const double *uvw, const double *weight,
                          or_geom *g)
{
    g->plane = malloc(sizeof(int32_t) * (size_t)nvis);
    g->ax = malloc(sizeof(int32_t) * (size_t)nvis);
    g->ay = malloc(sizeof(int32_t) * (size_t)nvis);
    g->status = malloc(sizeof(int32_t) * (size_t)nvis);
    g->fx = malloc(sizeof(double) * (size_t)nvis);
    g->fy = malloc(sizeof(double) * (size_t)nvis);
    int given = !(isnan(p->w_min) || isnan(p->w_max));
    if (given) {
        g->wmin = p->w_min;
        g->wmax = p->w_max;
    } else {
        or_wrange(nvis, uvw, &g->wmin, &g->wmax);
    }
    g->kept = or_coords(p, nvis, uvw, g->wmin, g->wmax, given, g->plane, g->ax, g->ay, g->fx, g->fy,
                        g->status);
    g->sumw = 0.0;
    for (int64_t i = 0; i < nvis; ++i)
        if (g->status[i] == 0) g->sumw += weight ? weight[i] : 1.0;
}

static void or_geom_free(or_geom *g)
{
    free(g->plane);
    free(g->ax);
    free(g->ay);
    free(g->status);
    free(g->fx);
    free(g->fy);
}

/* ------------------------------------------------------------------------ */
/* Gridding of one plane (Eq. 3): g[a_y + jy][a_x + jx] += w V G(d_x) G(d_y). */

void or_grid_plane(const or_params *p, const or_geom *g, int64_t cnt, const int64_t *idx,
                   const double complex *vis, const double *weight, double complex *plane)
{
    int W = p->support, n = p->n;
    memset(plane, 0, sizeof(double complex) * (size_t)n * n);
    /* kernel weights are a pure function of each visibility: computed in parallel */
    double *gx = malloc(sizeof(double) * (size_t)(cnt > 0 ? cnt : 1) * W);
    double *gy = malloc(sizeof(double) * (size_t)(cnt > 0 ? cnt : 1) * W);
#pragma omp parallel for schedule(static)
    for (int64_t t = 0; t < cnt; ++t) {
        or_axis_weights(p, g->fx[idx[t]], gx + t * W);
        or_axis_weights(p, g->fy[idx[t]], gy + t * W);
    }
    /* The sum of Eq. 3 in input order for every cell.  The threads split the
     * plane's rows (bands of 16, dealt out in turn) and each walks all the
     * visibilities in input order, adding only into its own rows: every cell
     * still receives its terms in input order, so the result is the same, bit
     * for bit, as one thread walking the visibilities. */
#pragma omp parallel
    {
        int nth = omp_get_num_threads(), th = omp_get_thread_num();
        for (int64_t t = 0; t < cnt; ++t) {
            int64_t i = idx[t];
            double complex val = vis[i] * (weight ? weight[i] : 1.0);
            for (int jy = 0; jy < W; ++jy) {
                int row = g->ay[i] + jy;
                if ((row >> 4) % nth != th) continue;
                for (int jx = 0; jx < W; ++jx)
                    plane[(size_t)row * n + (g->ax[i] + jx)] += val * gx[t * W + jx] * gy[t * W + jy];
            }
        }
    }
    free(gx);
    free(gy);
}

/* ------------------------------------------------------------------------ */
/* The image (§2 steps 2-4, Eq. 2):                                          */
/*   per plane k: grid -> x (-1)^{i+j} -> unnormalised inverse 2D DFT ->     */
/*   x (-1)^{p+q} -> x e^{2 pi i w_k (n-1)} -> sum over planes;              */
/*   image = Re(sum) * s(p,q), then the central m x m pixels are kept.       */
/* image: m x m; acc_out (if given): the n x n plane sum before scaling.     */
/* stats: kept, dropped_uv, dropped_w, sum_w, w_min, w_max.                  */

void or_image(const or_params *p, int64_t nvis, const double *uvw, const double complex *vis,
              const double *weight, uint32_t flags, double *image, double complex *acc_out,
              double *stats)
{
    int n = p->n;
    size_t nn = (size_t)n * n;
    or_geom g;
    or_geom_build(p, nvis, uvw, weight, &g);
    int64_t *start = malloc(sizeof(int64_t) * (size_t)(p->n_w + 1));
    int64_t *idx = or_plane_lists(p, nvis, g.plane, start);
    double complex *plane = malloc(sizeof(double complex) * nn);
    double complex *acc = acc_out ? acc_out : malloc(sizeof(double complex) * nn);
    memset(acc, 0, sizeof(double complex) * nn);
    double dl = p->fov / n;
    for (int k = 0; k < p->n_w; ++k) {
        or_grid_plane(p, &g, start[k + 1] - start[k], idx + start[k], vis, weight, plane);
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i)
                if ((i + j) & 1) plane[(size_t)j * n + i] = -plane[(size_t)j * n + i];
        or_fft2d(plane, n, +1);
        double wk = or_plane_centre(p, k, g.wmin, g.wmax);
#pragma omp parallel for schedule(static)
        for (int q = 0; q < n; ++q)
            for (int pp = 0; pp < n; ++pp) {
                double l = (pp - n / 2) * dl, m = (q - n / 2) * dl;
                double ph = 2.0 * M_PI * wk * or_nm1(l, m);
                double complex f = plane[(size_t)q * n + pp];
                if ((pp + q) & 1) f = -f;
                acc[(size_t)q * n + pp] += f * (cos(ph) + I * sin(ph));
            }
    }
    double *scale = malloc(sizeof(double) * nn);
    or_scale_plane(p, flags, g.sumw, scale);
    int m = or_image_side(p), o = (n - m) / 2;
    for (int q = 0; q < m; ++q)
        for (int pp = 0; pp < m; ++pp) {
            size_t t = (size_t)(q + o) * n + (pp + o);
            image[(size_t)q * m + pp] = creal(acc[t]) * scale[t];
        }
    if (stats) {
        int64_t du = 0, dw = 0;
        for (int64_t i = 0; i < nvis; ++i) {
            du += g.status[i] == 1;
            dw += g.status[i] == 2;
        }
        stats[0] = (double)g.kept;
        stats[1] = (double)du;
        stats[2] = (double)dw;
        stats[3] = g.sumw;
        stats[4] = g.wmin;
        stats[5] = g.wmax;
    }
    free(scale);
    if (!acc_out) free(acc);
    free(plane);
    free(idx);
    free(start);
    or_geom_free(&g);
}

/* Gridded planes only (for stage-wise checks): planes[k] = g_k, no shift, no FFT. */
void or_grid(const or_params *p, int64_t nvis, const double *uvw, const double complex *vis,
             const double *weight, double complex *planes, double *stats)
{
    size_t nn = (size_t)p->n * p->n;
    or_geom g;
    or_geom_build(p, nvis, uvw, weight, &g);
    int64_t *start = malloc(sizeof(int64_t) * (size_t)(p->n_w + 1));
    int64_t *idx = or_plane_lists(p, nvis, g.plane, start);
    for (int k = 0; k < p->n_w; ++k)
        or_grid_plane(p, &g, start[k + 1] - start[k], idx + start[k], vis, weight, planes + k * nn);
    if (stats) {
        stats[0] = (double)g.kept;
        stats[3] = g.sumw;
        stats[4] = g.wmin;
        stats[5] = g.wmax;
    }
    free(idx);
    free(start);
    or_geom_free(&g);
}

/* ------------------------------------------------------------------------ */
/* Adjoint of or_image under Re<.,.> (and, with other flags and no weights,  */
/* the degridding predictor): element by element the transpose of the steps */
/* above, in reverse order:                                                  */
/*   y * s(p,q) -> x e^{-2 pi i w_k (n-1)} -> x (-1)^{p+q} ->                */
/*   unnormalised forward 2D DFT -> x (-1)^{i+j} ->                          */
/*   per visibility [w_m] sum G(d_x) G(d_y) P[a_y + jy][a_x + jx].           */
/* The m x m image enters zero-padded to n x n (the transpose of the crop). */
/* wmin/wmax/sumw are those of the forward operator (the binning geometry). */

void or_adjoint(const or_params *p, int64_t nvis, const double *uvw, const double *weight,
                uint32_t flags, const double *image, double wmin, double wmax, double sumw,
                double complex *vis_out)
{
    int n = p->n, W = p->support;
    size_t nn = (size_t)n * n;
    or_params q = *p;
    q.w_min = wmin;
    q.w_max = wmax;
    or_geom g;
    or_geom_build(&q, nvis, uvw, weight, &g);
    int64_t *start = malloc(sizeof(int64_t) * (size_t)(p->n_w + 1));
    int64_t *idx = or_plane_lists(p, nvis, g.plane, start);
    double *scale = malloc(sizeof(double) * nn);
    or_scale_plane(p, flags, sumw, scale);
    double complex *plane = malloc(sizeof(double complex) * nn);
    double dl = p->fov / n;
    int mside = or_image_side(p), o = (n - mside) / 2;
    for (int64_t i = 0; i < nvis; ++i) vis_out[i] = 0.0;
    for (int k = 0; k < p->n_w; ++k) {
        double wk = or_plane_centre(p, k, wmin, wmax);
#pragma omp parallel for schedule(static)
        for (int qq = 0; qq < n; ++qq)
            for (int pp = 0; pp < n; ++pp) {
                double l = (pp - n / 2) * dl, m = (qq - n / 2) * dl;
                double ph = -2.0 * M_PI * wk * or_nm1(l, m);
                int inside = pp >= o && pp < o + mside && qq >= o && qq < o + mside;
                double complex f = 0.0; /* outside the crop (possibly off the unit circle) */
                if (inside)
                    f = image[(size_t)(qq - o) * mside + (pp - o)] * scale[(size_t)qq * n + pp] *
                        (cos(ph) + I * sin(ph));
                if ((pp + qq) & 1) f = -f;
                plane[(size_t)qq * n + pp] = f;
            }
        or_fft2d(plane, n, -1);
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i)
                if ((i + j) & 1) plane[(size_t)j * n + i] = -plane[(size_t)j * n + i];
        int64_t cnt = start[k + 1] - start[k];
#pragma omp parallel for schedule(static)
        for (int64_t t = 0; t < cnt; ++t) {
            int64_t i = idx[start[k] + t];
            double gx[64], gy[64];
            or_axis_weights(p, g.fx[i], gx);
            or_axis_weights(p, g.fy[i], gy);
            double complex s = 0.0;
            for (int jy = 0; jy < W; ++jy)
                for (int jx = 0; jx < W; ++jx)
                    s += gx[jx] * gy[jy] * plane[(size_t)(g.ay[i] + jy) * n + (g.ax[i] + jx)];
            vis_out[i] = s * (weight ? weight[i] : 1.0);
        }
    }
    free(plane);
    free(scale);
    free(idx);
    free(start);
    or_geom_free(&g);
}

/* ------------------------------------------------------------------------ */
/* Brute-force direct transform (inverse of Eq. 1, the form the w-stacked    */
/* image approximates): I(p,q) = d(p,q) sum_m w_m Re[V_m e^{+2 pi i (u l +   */
/* v m + w (n-1))}], d = [n] [1/n] [1/sum w], no taper, at pixel centres.    */

void or_dft(int32_t n, double fov, int64_t nvis, const double *uvw, const double complex *vis,
            const double *weight, uint32_t flags, double sumw, double *image)
{
    double dl = fov / n;
#pragma omp parallel for schedule(dynamic, 1)
    for (int q = 0; q < n; ++q)
        for (int pp = 0; pp < n; ++pp) {
            double l = (pp - n / 2) * dl, m = (q - n / 2) * dl, nm1 = or_nm1(l, m);
            double s = 0.0;
            for (int64_t i = 0; i < nvis; ++i) {
                double ph = 2.0 * M_PI * (uvw[3 * i] * l + uvw[3 * i + 1] * m + uvw[3 * i + 2] * nm1);
                s += (weight ? weight[i] : 1.0) * creal(vis[i] * (cos(ph) + I * sin(ph)));
            }
            double nn = 1.0 + nm1;
            if (flags & OR_N_CORRECT) s *= nn;
            if (flags & OR_N_DIVIDE) s /= nn;
            if ((flags & OR_NORMALIZE) && sumw != 0.0) s /= sumw;
            image[(size_t)q * n + pp] = s;
        }
}

/* ------------------------------------------------------------------------ */
/* The w-stacked image at chosen pixels, evaluated directly from the          */
/* visibilities: for each plane k the centred 2D DFT of its gridded cells at  */
/* (p, q) -- F_k(p, q) = sum_cells g_k(i, j) e^{2 pi i ((i-n/2)(p-n/2) +       */
/* (j-n/2)(q-n/2))/n}, which is what the checkerboarded FFT of or_image      */
/* computes -- written per visibility as w V X Y, X = sum_jx G(d_jx)          */
/* e^{2 pi i (a_x+jx-n/2)(p-n/2)/n} (Y likewise); then the w-phase of the     */
/* plane, the sum over planes and the scale of or_scale_plane (Eq. 2).  Costs */
/* O(n_vis W) per pixel instead of the FFT's O(n^2 log n) per plane, so a few */
/* pixels of a large image can be checked.  The corner's phase               */
/* (a - n/2)(p - n/2) is reduced modulo n exactly in integers before the      */
/* cosine and sine; the W cells of a footprint step from it by e^{2 pi i s/n}.*/

void or_image_pixels(const or_params *p, int64_t nvis, const double *uvw,
                     const double complex *vis, const double *weight, uint32_t flags,
                     int32_t npix, const int32_t *px, const int32_t *py, double *out)
{
    int n = p->n, W = p->support;
    or_geom g;
    or_geom_build(p, nvis, uvw, weight, &g);
    double dl = p->fov / n;
    /* per pixel: the w-phase factor of every plane */
    double complex *wph = malloc(sizeof(double complex) * (size_t)npix * p->n_w);
    for (int t = 0; t < npix; ++t) {
        double l = (px[t] - n / 2) * dl, m = (py[t] - n / 2) * dl, nm1 = or_nm1(l, m);
        for (int k = 0; k < p->n_w; ++k) {
            double ph = 2.0 * M_PI * or_plane_centre(p, k, g.wmin, g.wmax) * nm1;
            wph[(size_t)t * p->n_w + k] = cos(ph) + I * sin(ph);
        }
    }
    double complex *stepx = malloc(sizeof(double complex) * (size_t)npix);
    double complex *stepy = malloc(sizeof(double complex) * (size_t)npix);
    for (int t = 0; t < npix; ++t) {
        double ax_ = 2.0 * M_PI * (double)(((px[t] - n / 2) % n + n) % n) / n;
        double ay_ = 2.0 * M_PI * (double)(((py[t] - n / 2) % n + n) % n) / n;
        stepx[t] = cos(ax_) + I * sin(ax_);
        stepy[t] = cos(ay_) + I * sin(ay_);
    }
    double complex *acc = calloc((size_t)npix, sizeof(double complex));
#pragma omp parallel
    {
        double complex *part = calloc((size_t)npix, sizeof(double complex));
        double *gx = malloc(sizeof(double) * W), *gy = malloc(sizeof(double) * W);
#pragma omp for schedule(static)
        for (int64_t i = 0; i < nvis; ++i) {
            if (g.status[i] != 0) continue;
            or_axis_weights(p, g.fx[i], gx);
            or_axis_weights(p, g.fy[i], gy);
            double complex wv = (weight ? weight[i] : 1.0) * vis[i];
            for (int t = 0; t < npix; ++t) {
                long sp = px[t] - n / 2, sq = py[t] - n / 2;
                /* e^{2 pi i (a - n/2) s / n} at the corner, times e^{2 pi i s / n} per cell */
                long mx = (((long)(g.ax[i] - n / 2) * sp) % n + n) % n;
                long my = (((long)(g.ay[i] - n / 2) * sq) % n + n) % n;
                double bx = 2.0 * M_PI * (double)mx / n, by = 2.0 * M_PI * (double)my / n;
                double complex ex = cos(bx) + I * sin(bx), ey = cos(by) + I * sin(by);
                double complex X = 0.0, Y = 0.0;
                for (int j = 0; j < W; ++j) {
                    X += gx[j] * ex;
                    Y += gy[j] * ey;
                    ex *= stepx[t];
                    ey *= stepy[t];
                }
                part[t] += wv * X * Y * wph[(size_t)t * p->n_w + g.plane[i]];
            }
        }
#pragma omp critical
        for (int t = 0; t < npix; ++t) acc[t] += part[t];
        free(part);
        free(gx);
        free(gy);
    }
    for (int t = 0; t < npix; ++t) {
        double l = (px[t] - n / 2) * dl, m = (py[t] - n / 2) * dl;
        double nn = sqrt(1.0 - l * l - m * m);
        double s = 1.0 / (or_taper(p, (double)(px[t] - n / 2) / n) *
                          or_taper(p, (double)(py[t] - n / 2) / n));
        if (flags & OR_N_CORRECT) s *= nn;
        if (flags & OR_N_DIVIDE) s /= nn;
        if ((flags & OR_NORMALIZE) && g.sumw != 0.0) s /= g.sumw;
        out[t] = creal(acc[t]) * s;
    }
    free(acc);
    free(wph);
    free(stepx);
    free(stepy);
    or_geom_free(&g);
}

/* ------------------------------------------------------------------------ */
/* Imaging weights (the paper's §2 names Briggs 1995 for the weighting).     */
/* The density of a uv cell is the sum of the natural weights of the kept   */
/* visibilities whose centre cell c = a + h (the cell nearest to (x, y)) it  */
/* is, over all w-planes.  Uniform weighting divides each weight by its      */
/* cell's density; Briggs' robust weighting with robustness R divides it by  */
/* 1 + f^2 D, with f^2 = (5 10^-R)^2 / (sum_cells D^2 / sum_kept w).  Dropped */
/* visibilities get weight 0.                                                */

enum { OR_WEIGHT_UNIFORM = 1, OR_WEIGHT_BRIGGS = 2 };

void or_density_weights(const or_params *p, int64_t nvis, const double *uvw, const double *weight,
                        int32_t scheme, double robust, double *out)
{
    int n = p->n, W = p->support;
    int h = (W % 2) ? (W - 1) / 2 : W / 2 - 1;
    int given = !isnan(p->w_min);
    double wmin = p->w_min, wmax = p->w_max;
    if (!given) or_wrange(nvis, uvw, &wmin, &wmax);
    int32_t *plane = malloc(sizeof(int32_t) * (nvis > 0 ? nvis : 1));
    int32_t *ax = malloc(sizeof(int32_t) * (nvis > 0 ? nvis : 1));
    int32_t *ay = malloc(sizeof(int32_t) * (nvis > 0 ? nvis : 1));
    int32_t *status = malloc(sizeof(int32_t) * (nvis > 0 ? nvis : 1));
    double *fx = malloc(sizeof(double) * (nvis > 0 ? nvis : 1));
    double *fy = malloc(sizeof(double) * (nvis > 0 ? nvis : 1));
    double *dens = calloc((size_t)n * n, sizeof(double));
    or_coords(p, nvis, uvw, wmin, wmax, given, plane, ax, ay, fx, fy, status);
    double sumw = 0.0;
    for (int64_t i = 0; i < nvis; ++i) {
        if (status[i] != 0) continue;
        double w = weight ? weight[i] : 1.0;
        dens[(size_t)(ay[i] + h) * n + (ax[i] + h)] += w;
        sumw += w;
    }
    double f2 = 0.0;
    if (scheme == OR_WEIGHT_BRIGGS) {
        double s2 = 0.0;
        for (size_t k = 0; k < (size_t)n * n; ++k) s2 += dens[k] * dens[k];
        double c = 5.0 * pow(10.0, -robust);
        f2 = s2 > 0.0 ? c * c / (s2 / sumw) : 0.0;
    }
    for (int64_t i = 0; i < nvis; ++i) {
        if (status[i] != 0) {
            out[i] = 0.0;
            continue;
        }
        double w = weight ? weight[i] : 1.0;
        double d = dens[(size_t)(ay[i] + h) * n + (ax[i] + h)];
        if (scheme == OR_WEIGHT_UNIFORM)
            out[i] = d > 0.0 ? w / d : 0.0;
        else
            out[i] = w / (1.0 + f2 * d);
    }
    free(plane);
    free(ax);
    free(ay);
    free(status);
    free(fx);
    free(fy);
    free(dens);
}

/* Threads the OpenMP loops above may use (for the CPU-baseline report). */
int32_t or_max_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * synth.c -- seeded synthetic interferometer observations, shared by the tests,
 * the benchmark and the oracle runs as their only common input source.
 *
 * It holds none of the imaging method's arithmetic: it draws an antenna layout,
 * earth-rotation uvw tracks and a point-source sky, and predicts visibilities
 * with the measurement equation (Eq. 1 of De Rubeis et al.) evaluated directly.
 *
 * Random numbers: SplitMix64 (Steele, Lea & Flood 2014) as a counter-based
 * generator, value = mix(seed, stream, index), so every draw is independent of
 * thread count and identical on x86-64 and aarch64 (compile with
 * -ffp-contract=off).
 *
 * Geometry (textbook interferometry, e.g. Thompson, Moran & Swenson ch. 4):
 *   local (E, N, U) -> equatorial (X, Y, Z) at latitude phi:
 *     X = -sin(phi) N + cos(phi) U,  Y = E,  Z = cos(phi) N + sin(phi) U
 *   baseline (Lx, Ly, Lz) in wavelengths at hour angle H, declination dec:
 *     u =  sin H Lx + cos H Ly
 *     v = -sin dec cos H Lx + sin dec sin H Ly + cos dec Lz
 *     w =  cos dec cos H Lx - cos dec sin H Ly + sin dec Lz
 * Visibility order is (time, baseline, channel), channel fastest.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

static uint64_t sx_mix(uint64_t z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* Uniform double in [0, 1) from the top 53 bits of mix(seed, stream, i). */
double sx_uniform(uint64_t seed, uint64_t stream, uint64_t i)
{
    uint64_t z = sx_mix(sx_mix(sx_mix(seed) ^ (stream * 0xD1B54A32D192ED03ull)) ^ i);
    return (double)(z >> 11) * (1.0 / 9007199254740992.0);
}

/* Standard normal by Box-Muller from two uniforms of the same counter. */
double sx_normal(uint64_t seed, uint64_t stream, uint64_t i)
{
    double u1 = sx_uniform(seed, stream, 2 * i), u2 = sx_uniform(seed, stream, 2 * i + 1);
    return sqrt(-2.0 * log(1.0 - u1)) * cos(2.0 * M_PI * u2);
}

typedef struct {
    int64_t seed;
    int32_t n_ant;
    int32_t n_steps;
    int32_t n_chan;
    int32_t n_src;
    double core_frac;    /* fraction of stations in the dense core                */
    double core_radius;  /* m                                                      */
    double max_radius;   /* m, outermost remote station (log-radial between)       */
    double latitude;     /* rad                                                    */
    double dec;          /* rad, phase-centre declination                          */
    double hours;        /* observation length, centred on transit                 */
    double nu0, dnu;     /* Hz, first channel and channel width                    */
    double uv_max;       /* lambda; u,v rescaled so that max(|u|,|v|) == uv_max    */
    double w_max;        /* lambda; w rescaled so that max |w| == w_max             */
    double field;        /* rad, side of the square the sources are drawn in       */
    double flux_min, flux_max;
    double flux_index;   /* dN/dS ~ S^index; 0 -> log-uniform                      */
    double noise_sigma;  /* complex noise, re and im ~ N(0, sigma^2 / 2)           */
    int32_t weight_mode; /* 0 unit weights, 1 uniform in [0.5, 1.5)                */
    int32_t pad;
} sx_config;

enum { ST_ANT_R = 1, ST_ANT_T, ST_SRC_L, ST_SRC_M, ST_SRC_S, ST_NOISE, ST_WEIGHT, ST_CORE };

/* Station layout in local (E, N, U = 0) metres: core_frac of the stations
 * uniform in a disc of core_radius, the rest log-uniform in radius out to
 * max_radius, uniform in azimuth. */
void sx_antennas(const sx_config *c, double *enu)
{
    int n_core = (int)llround(c->core_frac * c->n_ant);
    for (int a = 0; a < c->n_ant; ++a) {
        double ur = sx_uniform(c->seed, ST_ANT_R, a), ut = sx_uniform(c->seed, ST_ANT_T, a), r;
        if (a < n_core)
            r = c->core_radius * sqrt(ur);
        else
            r = c->core_radius * exp(ur * log(c->max_radius / c->core_radius));
        enu[3 * a] = r * cos(2.0 * M_PI * ut);
        enu[3 * a + 1] = r * sin(2.0 * M_PI * ut);
        enu[3 * a + 2] = 0.0;
    }
}

/* Point sources: (l, m) uniform in the field square, flux from the power law
 * (inverse CDF) or log-uniform. */
void sx_sources(const sx_config *c, double *l, double *m, double *s)
{
    for (int k = 0; k < c->n_src; ++k) {
        l[k] = (sx_uniform(c->seed, ST_SRC_L, k) - 0.5) * c->field;
        m[k] = (sx_uniform(c->seed, ST_SRC_M, k) - 0.5) * c->field;
        double u = sx_uniform(c->seed, ST_SRC_S, k);
        if (c->flux_index == 0.0) {
            s[k] = c->flux_min * exp(u * log(c->flux_max / c->flux_min));
        } else {
            double g = c->flux_index + 1.0;
            double a = pow(c->flux_min, g), b = pow(c->flux_max, g);
            s[k] = pow(a + u * (b - a), 1.0 / g);
        }
    }
}

/* Unscaled uvw (wavelengths at nu0) of row r = t * n_bl + b. */
static void sx_row_uvw(const sx_config *c, const double *xyz, const int *bl_a, const int *bl_b,
                       int64_t n_bl, int64_t r, double *uvw)
{
    int64_t t = r / n_bl, b = r % n_bl;
    double lam = 299792458.0 / c->nu0;
    double H = ((t + 0.5) / c->n_steps - 0.5) * c->hours * (2.0 * M_PI / 24.0);
    double Lx = (xyz[3 * bl_b[b]] - xyz[3 * bl_a[b]]) / lam;
    double Ly = (xyz[3 * bl_b[b] + 1] - xyz[3 * bl_a[b] + 1]) / lam;
    double Lz = (xyz[3 * bl_b[b] + 2] - xyz[3 * bl_a[b] + 2]) / lam;
    double sh = sin(H), ch = cos(H), sd = sin(c->dec), cd = cos(c->dec);
    uvw[0] = sh * Lx + ch * Ly;
    uvw[1] = -sd * ch * Lx + sd * sh * Ly + cd * Lz;
    uvw[2] = cd * ch * Lx - cd * sh * Ly + sd * Lz;
}

/* Full observation: uvw [n_keep][3] (f64, lambda), vis [n_keep] as (re, im)
 * f32 pairs, weight [n_keep] f32, and the sky (l, m, flux) [n_src].
 * Rows are (time, baseline); each row holds n_chan channels with uvw scaled by
 * f_c = nu_c / nu0: uvw[row n_chan + c] = uvw_rows[row] * f_c, one FP64
 * product per coordinate.  uvw_rows [ceil(n_keep / n_chan)][3] and chan_f
 * [n_chan] receive those factors if not NULL.  Only the first n_keep
 * visibilities are produced. */
int64_t sx_observation(const sx_config *c, int64_t n_keep, double *uvw, float *vis, float *weight,
                       double *src_l, double *src_m, double *src_s, double *uvw_rows,
                       double *chan_f)
{
    int n_ant = c->n_ant;
    int64_t n_bl = (int64_t)n_ant * (n_ant - 1) / 2;
    int64_t n_total = n_bl * c->n_steps * c->n_chan;
    if (n_keep > n_total) n_keep = n_total;
    int64_t n_rows = (n_keep + c->n_chan - 1) / c->n_chan;

    double *enu = malloc(sizeof(double) * 3 * n_ant), *xyz = malloc(sizeof(double) * 3 * n_ant);
    sx_antennas(c, enu);
    double sp = sin(c->latitude), cp = cos(c->latitude);
    for (int a = 0; a < n_ant; ++a) {
        double E = enu[3 * a], N = enu[3 * a + 1], U = enu[3 * a + 2];
        xyz[3 * a] = -sp * N + cp * U;
        xyz[3 * a + 1] = E;
        xyz[3 * a + 2] = cp * N + sp * U;
    }
    int *bl_a = malloc(sizeof(int) * n_bl), *bl_b = malloc(sizeof(int) * n_bl);
    for (int a = 0, b = 0; a < n_ant; ++a)
        for (int j = a + 1; j < n_ant; ++j, ++b) {
            bl_a[b] = a;
            bl_b[b] = j;
        }

    /* rescaling factors from the unscaled maxima over the kept rows */
    double max_uv = 0.0, max_w = 0.0, top = 1.0 + (c->n_chan - 1) * c->dnu / c->nu0;
#pragma omp parallel for reduction(max : max_uv, max_w) schedule(static)
    for (int64_t r = 0; r < n_rows; ++r) {
        double q[3];
        sx_row_uvw(c, xyz, bl_a, bl_b, n_bl, r, q);
        double a = fmax(fabs(q[0]), fabs(q[1])) * top, bw = fabs(q[2]) * top;
        if (a > max_uv) max_uv = a;
        if (bw > max_w) max_w = bw;
    }
    double s_uv = max_uv > 0 ? c->uv_max / max_uv : 1.0, s_w = max_w > 0 ? c->w_max / max_w : 1.0;

    sx_sources(c, src_l, src_m, src_s);
    if (chan_f)
        for (int ch = 0; ch < c->n_chan; ++ch) chan_f[ch] = (c->nu0 + ch * c->dnu) / c->nu0;
    double *src_amp = malloc(sizeof(double) * (c->n_src > 0 ? c->n_src : 1));
    double *src_nm1 = malloc(sizeof(double) * (c->n_src > 0 ? c->n_src : 1));
    for (int k = 0; k < c->n_src; ++k) {
        double n = sqrt(1.0 - src_l[k] * src_l[k] - src_m[k] * src_m[k]);
        src_amp[k] = src_s[k] / n; /* Eq. 1: I / n */
        src_nm1[k] = n - 1.0;
    }

#pragma omp parallel
    {
        double *re = malloc(sizeof(double) * c->n_chan), *im = malloc(sizeof(double) * c->n_chan);
#pragma omp for schedule(static)
        for (int64_t r = 0; r < n_rows; ++r) {
            double q[3];
            sx_row_uvw(c, xyz, bl_a, bl_b, n_bl, r, q);
            double u0 = q[0] * s_uv, v0 = q[1] * s_uv, w0 = q[2] * s_w;
            if (uvw_rows) {
                uvw_rows[3 * r] = u0;
                uvw_rows[3 * r + 1] = v0;
                uvw_rows[3 * r + 2] = w0;
            }
            int64_t i0 = r * c->n_chan;
            int nc = (int)((n_keep - i0) < c->n_chan ? (n_keep - i0) : c->n_chan);
            for (int ch = 0; ch < nc; ++ch) {
                double f = (c->nu0 + ch * c->dnu) / c->nu0;
                uvw[3 * (i0 + ch)] = u0 * f;
                uvw[3 * (i0 + ch) + 1] = v0 * f;
                uvw[3 * (i0 + ch) + 2] = w0 * f;
                re[ch] = im[ch] = 0.0;
            }
            /* Eq. 1 for point sources, V = sum_s S_s/n_s e^{-2 pi i (u l + v m + w (n - 1))};
             * uvw scale with frequency, so the phase of channel ch is the channel-0
             * phase times f_ch: the phasor is advanced by a fixed per-row step. */
            for (int k = 0; k < c->n_src; ++k) {
                double ph = -2.0 * M_PI * (u0 * src_l[k] + v0 * src_m[k] + w0 * src_nm1[k]);
                double pr = cos(ph), pi = sin(ph);
                double dph = ph * (c->dnu / c->nu0), sr = cos(dph), si = sin(dph);
                for (int ch = 0; ch < nc; ++ch) {
                    re[ch] += src_amp[k] * pr;
                    im[ch] += src_amp[k] * pi;
                    double t = pr * sr - pi * si;
                    pi = pr * si + pi * sr;
                    pr = t;
                }
            }
            for (int ch = 0; ch < nc; ++ch) {
                int64_t i = i0 + ch;
                double s = c->noise_sigma * sqrt(0.5);
                vis[2 * i] = (float)(re[ch] + s * sx_normal(c->seed, ST_NOISE, 2 * (uint64_t)i));
                vis[2 * i + 1] = (float)(im[ch] + s * sx_normal(c->seed, ST_NOISE, 2 * (uint64_t)i + 1));
                weight[i] = c->weight_mode == 1 ? (float)(0.5 + sx_uniform(c->seed, ST_WEIGHT, i)) : 1.0f;
            }
        }
        free(re);
        free(im);
    }
    free(src_amp);
    free(src_nm1);
    free(enu);
    free(xyz);
    free(bl_a);
    free(bl_b);
    return n_keep;
}

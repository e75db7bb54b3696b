// rick_wphase.cuh -- per-pixel geometry and w-phase of the w-correction
// (§2 step 4, Eq. 2), shared by the plane-sum kernels (rick_wcorrect.cu) and
// the fused transform + w-correction (rick_fft.cu).
//
// The phase w_k (n - 1) reaches tens of cycles for wide fields and large |w|,
// so it is formed in double-single arithmetic (hi + lo floats, about 48
// significant bits) from the FP64 plane centres and the pixel's n - 1, which
// itself is evaluated in double-single from l, m; only its fraction in cycles
// goes to sincospif.
#pragma once

#include <cuda_fp16.h>

#include "rick_common.cuh"

struct WcArgs {
    int n, n_w;
    int m, off;  // image side and its offset (n - m)/2 in the grid frame
    const float2 *planes_in;
    float2 *planes_out;
    const float *image_in;
    float *image_out;
    const float *taper_inv;
    const WsHeader *hdr;
    const float4 *wplane;
    ff dl;        // fov / n as hi + lo
    float dl_f;   // fov / n as float
    uint32_t flags;
};

struct PixelGeom {
    ff nm1;      // n - 1 (double-single)
    float nm1_f; // n - 1 in plain FP32 (ablation)
    float scale; // s(p, q) including the checkerboard sign
};

// The output scale s(p, q) of a pixel: the taper correction 1 / (C(l) C(m)),
// the n factor (nn = n, RICK_N_CORRECT / RICK_N_DIVIDE), the weight
// normalisation and the checkerboard sign of the centred transform.
__device__ __forceinline__ float pixel_scale(const WcArgs &a, int p, int q, float nn,
                                             float inv_sumw)
{
    float s = a.taper_inv[p] * a.taper_inv[q];
    if (a.flags & RICK_N_CORRECT) s *= nn;
    if (a.flags & RICK_N_DIVIDE) s /= nn;
    if (a.flags & RICK_NORMALIZE) s *= inv_sumw;
    return ((p + q) & 1) ? -s : s;
}

// The low word of a double-single n - 1 kept in 16 bits, for kernels that hold
// n - 1 of many pixels in shared memory: lo / hi scaled by 2^24 (|lo| <=
// ulp(hi) / 2 <= 2^-24 |hi|, so the ratio lies in [-1, 1]) as a half.  The
// decoded low word carries a relative error of 2^-11, about 2^-35 of n - 1:
// below 1e-9 cycles of w-phase for |w (n - 1)| up to 100 cycles.
__device__ __forceinline__ __half nm1_lo_encode(ff v)
{
    return __float2half_rn(v.hi != 0.0f ? v.lo / v.hi * 16777216.0f : 0.0f);
}

__device__ __forceinline__ float nm1_lo_decode(float hi, __half e)
{
    return __half2float(e) * hi * 5.9604644775390625e-8f;  // 2^-24
}

__device__ __forceinline__ PixelGeom pixel_geom(const WcArgs &a, int p, int q, float inv_sumw)
{
    PixelGeom g;
    const int h = a.n / 2;
    ff r2;
    g.nm1 = ff_nm1(ff_mul_int(p - h, a.dl), ff_mul_int(q - h, a.dl), &r2);
    float l = (p - h) * a.dl_f, m = (q - h) * a.dl_f, r2f = l * l + m * m;
    g.nm1_f = -r2f / (1.0f + sqrtf(1.0f - r2f));
    g.scale = pixel_scale(a, p, q, sqrtf(1.0f - r2.hi), inv_sumw);
    return g;
}

// cos / sin of 2 pi w_k (n - 1)
__device__ __forceinline__ void wphase(const WcArgs &a, const float4 &wk, const PixelGeom &g,
                                       float *c, float *s)
{
    float f;
    if (a.flags & RICK_PHASE_FP32) {
        float th = wk.z * g.nm1_f;
        f = th - rintf(th);
    } else {
        f = ff_frac(ff_mul(ff{wk.x, wk.y}, g.nm1));
    }
    sincospif(2.0f * f, s, c);
}

// Phase factors e^{2 pi i w_k (n - 1)} of one pixel for k = 0 .. n_w - 1.  The
// plane centres are equally spaced, w_k = w_0 + k dw, so the factor of plane k
// is the previous one times the step e^{2 pi i dw (n - 1)}: one complex
// multiply per plane.  Every RICK_PHASE_ANCHOR planes the factor is recomputed
// exactly from w_k (double-single phase, sincospif), which bounds the FP32
// drift of the recurrence to a few ulps.
#define RICK_PHASE_ANCHOR 8

struct PhaseWalker {
    float c, s, cd, sd;
    __device__ __forceinline__ void start(const WcArgs &a, const float4 *w, int n_w,
                                          const PixelGeom &g)
    {
        if (a.flags & RICK_PHASE_FP32) {
            cd = 1.0f;
            sd = 0.0f;
            return;
        }
        float fd = ff_frac(ff_mul(ff{w[n_w].x, w[n_w].y}, g.nm1));
        sincospif(2.0f * fd, &sd, &cd);
    }
    __device__ __forceinline__ void at(const WcArgs &a, const float4 *w, int k, const PixelGeom &g)
    {
        if ((a.flags & RICK_PHASE_FP32) || k % RICK_PHASE_ANCHOR == 0) {
            wphase(a, w[k], g, &c, &s);
        } else {
            float c2 = c * cd - s * sd;
            s = s * cd + c * sd;
            c = c2;
        }
    }
};


// Launch arguments of a plan's w-correction (host side).
static WcArgs make_args(rick_plan *plan, const void *ws_dev, uint32_t flags)
{
    const rick_params &p = plan->p;
    WsPtrs w = rick_ws_ptrs((void *)ws_dev, rick_ws_layout(&p, plan->max_vis));
    WcArgs a;
    a.n = p.n;
    a.n_w = p.n_w;
    a.m = p.image_n ? p.image_n : p.n;
    a.off = (p.n - a.m) / 2;
    a.taper_inv = plan->taper_inv;
    a.hdr = w.hdr;
    a.wplane = w.wplane;
    double dl = p.fov / p.n;
    a.dl = ff_from_double(dl);
    a.dl_f = (float)dl;
    a.flags = flags;
    a.planes_in = NULL;
    a.planes_out = NULL;
    a.image_in = NULL;
    a.image_out = NULL;
    return a;
}

// Flags of an imaging call (w-correction, plane sum) or, with adjoint, of a
// w-spreading call, which has no imaginary part to select.
static bool valid_flags(uint32_t f, bool adjoint = false)
{
    const uint32_t known = RICK_N_CORRECT | RICK_NORMALIZE | RICK_N_DIVIDE | RICK_PHASE_FP32 |
                           (adjoint ? 0u : RICK_IMAG_PART);
    return (f & ~known) == 0 && !((f & RICK_N_CORRECT) && (f & RICK_N_DIVIDE));
}


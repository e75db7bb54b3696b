// rick_wcorrect.cu -- w-correction and plane reduction (§2 step 4: "we apply
// the phase shift and reduce the w-planes to obtain the final image"; Eq. 2,
// with the integral over w becoming the sum over the plane centres w_k), the
// taper correction, and the adjoint of all of it (w-spreading, used by
// degridding).
//
// One thread per pixel walks the n_w planes: each plane is one coalesced
// float2 read per pixel, so the kernel is bound by reading the planes once.
// The phase w_k (n - 1) reaches tens of cycles for wide fields and large |w|,
// so it is formed in double-single arithmetic (hi + lo floats, about 48
// significant bits) from the FP64 plane centres and the pixel's n - 1, which
// itself is evaluated in double-single from l, m; only its fraction in cycles
// goes to sincospif.  This keeps FP64-class accuracy without per-pixel FP64
// instructions, which GB300 issues at a small fraction of the FP32 rate.
//
// On a padded grid only the kept m x m crop is corrected (m^2 n_w plane reads
// instead of n^2 n_w); the adjoint writes zeros outside the crop.  Where the
// crop offset is even, a thread corrects two adjacent pixels (16-byte plane
// loads: 0.36 instead of 0.41 ms for 16 planes of 4096^2).
#include "rick_common.cuh"
#include "rick_wphase.cuh"

__global__ void __launch_bounds__(256) wcorrect_kernel(WcArgs a)
{
    extern __shared__ float4 s_w[];
    __shared__ float s_inv_sumw;
    for (int k = threadIdx.x; k <= a.n_w; k += blockDim.x) s_w[k] = a.wplane[k];
    if (threadIdx.x == 0) {
        double sw = a.hdr->stats.sum_weight;  // nothing gridded: no normalisation
        s_inv_sumw = sw != 0.0 ? (float)(1.0 / sw) : 1.0f;
    }
    __syncthreads();
    const size_t nn = (size_t)a.n * a.n;
    const size_t oidx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (oidx >= (size_t)a.m * a.m) return;
    const int p = (int)(oidx % a.m) + a.off, q = (int)(oidx / a.m) + a.off;
    PixelGeom g = pixel_geom(a, p, q, s_inv_sumw);
    const bool imag = (a.flags & RICK_IMAG_PART) != 0;  // Im of the sum instead of Re
    float acc = 0.0f;
    const float2 *src = a.planes_in + ((size_t)q * a.n + p);
    PhaseWalker ph;
    ph.start(a, s_w, a.n_w, g);
#pragma unroll 4
    for (int k = 0; k < a.n_w; ++k) {
        float2 F = src[(size_t)k * nn];
        ph.at(a, s_w, k, g);
        acc = imag ? fmaf(F.x, ph.s, fmaf(F.y, ph.c, acc)) : fmaf(F.x, ph.c, fmaf(-F.y, ph.s, acc));
    }
    a.image_out[oidx] = acc * g.scale;
}

// The same for two adjacent pixels per thread: one 16-byte load per plane
// brings both pixels' values.  Needs an even crop offset (16-byte aligned
// pairs) and an 8-byte aligned image.
__global__ void __launch_bounds__(256) wcorrect2_kernel(WcArgs a)
{
    extern __shared__ float4 s_w[];
    __shared__ float s_inv_sumw;
    for (int k = threadIdx.x; k <= a.n_w; k += blockDim.x) s_w[k] = a.wplane[k];
    if (threadIdx.x == 0) {
        double sw = a.hdr->stats.sum_weight;  // nothing gridded: no normalisation
        s_inv_sumw = sw != 0.0 ? (float)(1.0 / sw) : 1.0f;
    }
    __syncthreads();
    const size_t half_nn = (size_t)a.n * a.n / 2;  // planes in float4 units
    const int mh = a.m >> 1;
    const size_t pidx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;  // pixel pair
    if (pidx >= (size_t)mh * a.m) return;
    const int pp = (int)(pidx % mh) * 2, qq = (int)(pidx / mh);  // in the image
    const int p = pp + a.off, q = qq + a.off;                      // in the grid frame
    PixelGeom g0 = pixel_geom(a, p, q, s_inv_sumw), g1 = pixel_geom(a, p + 1, q, s_inv_sumw);
    const bool imag = (a.flags & RICK_IMAG_PART) != 0;  // Im of the sum instead of Re
    float acc0 = 0.0f, acc1 = 0.0f;
    const float4 *src = (const float4 *)(a.planes_in + ((size_t)q * a.n + p));
    PhaseWalker ph0, ph1;
    ph0.start(a, s_w, a.n_w, g0);
    ph1.start(a, s_w, a.n_w, g1);
#pragma unroll 4
    for (int k = 0; k < a.n_w; ++k) {
        const float4 F = src[(size_t)k * half_nn];
        ph0.at(a, s_w, k, g0);
        ph1.at(a, s_w, k, g1);
        if (imag) {
            acc0 = fmaf(F.x, ph0.s, fmaf(F.y, ph0.c, acc0));
            acc1 = fmaf(F.z, ph1.s, fmaf(F.w, ph1.c, acc1));
        } else {
            acc0 = fmaf(F.x, ph0.c, fmaf(-F.y, ph0.s, acc0));
            acc1 = fmaf(F.z, ph1.c, fmaf(-F.w, ph1.s, acc1));
        }
    }
    *(float2 *)(a.image_out + ((size_t)qq * a.m + pp)) =
        make_float2(acc0 * g0.scale, acc1 * g1.scale);
}

__global__ void __launch_bounds__(256) wspread_kernel(WcArgs a)
{
    extern __shared__ float4 s_w[];
    __shared__ float s_inv_sumw;
    for (int k = threadIdx.x; k <= a.n_w; k += blockDim.x) s_w[k] = a.wplane[k];
    if (threadIdx.x == 0) {
        double sw = a.hdr->stats.sum_weight;  // nothing gridded: no normalisation
        s_inv_sumw = sw != 0.0 ? (float)(1.0 / sw) : 1.0f;
    }
    __syncthreads();
    const size_t nn = (size_t)a.n * a.n;
    size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nn) return;
    const int p = (int)(idx % a.n), q = (int)(idx / a.n);
    float2 *dst = a.planes_out + idx;
    const int pi = p - a.off, qi = q - a.off;
    if (pi < 0 || pi >= a.m || qi < 0 || qi >= a.m) {  // zero padding
        for (int k = 0; k < a.n_w; ++k) dst[(size_t)k * nn] = make_float2(0.0f, 0.0f);
        return;
    }
    PixelGeom g = pixel_geom(a, p, q, s_inv_sumw);
    float v = a.image_in[(size_t)qi * a.m + pi] * g.scale;
    PhaseWalker ph;
    ph.start(a, s_w, a.n_w, g);
#pragma unroll 4
    for (int k = 0; k < a.n_w; ++k) {
        ph.at(a, s_w, k, g);
        dst[(size_t)k * nn] = make_float2(v * ph.c, -v * ph.s);
    }
}

extern "C" rick_status rick_wcorrect_stack(rick_plan *plan, const void *planes_dev,
                                           const void *ws_dev, float *image_dev, uint32_t flags,
                                           void *stream)
{
    if (!plan || !planes_dev || !ws_dev || !image_dev || !valid_flags(flags)) return RICK_EINVAL;
    if (plan->sticky != RICK_OK) return plan->sticky;
    if (((uintptr_t)ws_dev & 255) || ((uintptr_t)planes_dev & 7) || ((uintptr_t)image_dev & 3))
        return RICK_EINVAL;
    WcArgs a = make_args(plan, ws_dev, flags);
    a.planes_in = (const float2 *)planes_dev;
    a.image_out = image_dev;
    size_t mm = (size_t)a.m * a.m;
    if ((a.off & 1) == 0 && ((uintptr_t)planes_dev & 15) == 0 && ((uintptr_t)image_dev & 7) == 0)
        wcorrect2_kernel<<<(unsigned)((mm / 2 + 255) / 256), 256, sizeof(float4) * (a.n_w + 1),
                           (cudaStream_t)stream>>>(a);
    else
        wcorrect_kernel<<<(unsigned)((mm + 255) / 256), 256, sizeof(float4) * (a.n_w + 1),
                          (cudaStream_t)stream>>>(a);
    RICK_LAUNCH_CHECK(plan);
    return RICK_OK;
}

extern "C" rick_status rick_wspread(rick_plan *plan, const float *image_dev, const void *ws_dev,
                                    void *planes_dev, uint32_t flags, void *stream)
{
    if (!plan || !planes_dev || !ws_dev || !image_dev || !valid_flags(flags, true))
        return RICK_EINVAL;
    if (plan->sticky != RICK_OK) return plan->sticky;
    if (((uintptr_t)ws_dev & 255) || ((uintptr_t)planes_dev & 7) || ((uintptr_t)image_dev & 3))
        return RICK_EINVAL;
    WcArgs a = make_args(plan, ws_dev, flags);
    a.image_in = image_dev;
    a.planes_out = (float2 *)planes_dev;
    size_t nn = (size_t)a.n * a.n;
    wspread_kernel<<<(unsigned)((nn + 255) / 256), 256, sizeof(float4) * (a.n_w + 1),
                     (cudaStream_t)stream>>>(a);
    RICK_LAUNCH_CHECK(plan);
    return RICK_OK;
}

// rick_plan.cu -- plans, parameter checks, workspace sizing and the per-plane
// FFT stage (§2 step 3; §3.1 of De Rubeis et al. describe the cuFFT usage,
// here single-GPU and batched over w-planes instead of cuFFTMp descriptors).
#include <math.h>
#include <stddef.h>
#include <stdio.h>
#include <stdlib.h>

#include "rick_common.cuh"

extern "C" const char *rick_status_string(rick_status s)
{
    switch (s) {
    case RICK_OK: return "ok";
    case RICK_EINVAL: return "invalid argument";
    case RICK_ENOMEM: return "device out of memory";
    case RICK_ECUDA: return "CUDA error";
    case RICK_ECUFFT: return "cuFFT error";
    case RICK_ERANGE: return "size exceeds capacity";
    default: return "unknown status";
    }
}

static bool is_pow2(int64_t x) { return x > 0 && (x & (x - 1)) == 0; }

// Beatty, Nishimura & Pauly (2005): the KB shape for oversampling alpha.
extern "C" double rick_kb_beta(int32_t support, double alpha)
{
    if (support < 2 || !(alpha >= 1.0) || !isfinite(alpha)) return NAN;
    const double t = (support / alpha) * (support / alpha) * (alpha - 0.5) * (alpha - 0.5) - 0.8;
    return t > 0.0 ? M_PI * sqrt(t) : NAN;
}

static rick_status check_params(const rick_params *p)
{
    if (!p) return RICK_EINVAL;
    if (!is_pow2(p->n) || p->n < 16 || p->n > 32768) return RICK_EINVAL;
    if (p->n_w < 1 || p->n_w > 1024) return RICK_EINVAL;
    if (!(p->fov > 0.0) || !isfinite(p->fov)) return RICK_EINVAL;
    if (p->options & ~(RICK_OPT_HERMITIAN_MIRROR | RICK_OPT_DETERMINISTIC)) return RICK_EINVAL;
    // the deterministic tile holds 64-bit sums (2 T (T + 1) 8 bytes of shared
    // memory) and has its own exact accumulation in place of the compensated one
    if ((p->options & RICK_OPT_DETERMINISTIC) &&
        (p->tile > 64 || p->precision != RICK_PREC_FP32))
        return RICK_EINVAL;
    if (p->image_n != 0 && (p->image_n < 16 || p->image_n > p->n || (p->image_n & 1)))
        return RICK_EINVAL;
    // the image (the kept crop of a padded grid) must stay inside the unit
    // circle of direction cosines; its corner pixel is at l = m = -(m/2) fov/n
    const double kept = p->image_n ? (double)p->image_n / p->n : 1.0;
    if (!(p->fov * kept * 0.5 * sqrt(2.0) < 1.0)) return RICK_EINVAL;
    if (isnan(p->w_min) != isnan(p->w_max)) return RICK_EINVAL;
    if (!isnan(p->w_min) && !(isfinite(p->w_min) && isfinite(p->w_max) && p->w_min <= p->w_max))
        return RICK_EINVAL;
    if (p->kernel != RICK_KERNEL_GAUSS && p->kernel != RICK_KERNEL_KB) return RICK_EINVAL;
    if (p->support < 1 || p->support > 16) return RICK_EINVAL;
    if (!is_pow2(p->tile) || p->tile < p->support || p->tile > 128 || p->tile > p->n ||
        p->tile < 8)
        return RICK_EINVAL;
    if (p->precision != RICK_PREC_FP32 && p->precision != RICK_PREC_FP32_COMPENSATED)
        return RICK_EINVAL;
    // the compensated tile holds six T x T float arrays in shared memory
    if (p->precision == RICK_PREC_FP32_COMPENSATED && p->tile > 64) return RICK_EINVAL;
    // the binning keys are 32-bit
    int64_t nt = p->n / p->tile;
    if (4 * (int64_t)p->n_w * nt * nt >= (1ll << 31)) return RICK_EINVAL;
    if (p->kernel == RICK_KERNEL_KB && p->support > 1) {
        double b = p->kb_beta;
        if (isnan(b)) {
            if (isnan(rick_kb_beta(p->support, 2.0))) return RICK_EINVAL;
        } else if (!(b > 0.0) || !isfinite(b)) {
            return RICK_EINVAL;
        }
    }
    if (p->kernel == RICK_KERNEL_GAUSS && !isnan(p->gauss_sigma) &&
        !(p->gauss_sigma > 0.0 && isfinite(p->gauss_sigma)))
        return RICK_EINVAL;
    return RICK_OK;
}

// Taper correction C(nu) = integral_{-W/2}^{W/2} G(d) cos(2 pi nu d) dd for
// nu_p = (p - n/2)/n, stored as 1/C.  KB: closed form of Jackson (1991),
// W sinh(sqrt(beta^2 - (pi W nu)^2)) / sqrt(...) / I0(beta); Gaussian: a
// 48-point Gauss-Legendre rule (the integrand is entire).  FP64.
// Nodes and weights of the 48-point Gauss-Legendre rule on [-1, 1] (nodes in
// decreasing order), by Newton's iteration on the Legendre polynomial P_48 from
// the cosine initial guesses (the textbook method), in FP64 on the host.
#define RICK_GL_N 48
struct GaussLegendre {
    double x[RICK_GL_N], w[RICK_GL_N];
};

static GaussLegendre gauss_legendre()
{
    GaussLegendre g;
    const int N = RICK_GL_N;
    for (int i = 0; i < N; ++i) {
        double x = cos(M_PI * (i + 0.75) / (N + 0.5)), dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = x;  // P_0, P_1; recurrence up to P_N
            for (int k = 2; k <= N; ++k) {
                const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = N * (x * p1 - p0) / (x * x - 1.0);  // P_N'(x)
            const double dx = p1 / dp;
            x -= dx;
            if (fabs(dx) < 1e-16) break;
        }
        g.x[i] = x;
        g.w[i] = 2.0 / ((1.0 - x * x) * dp * dp);
    }
    return g;
}

__global__ void taper_kernel(float *taper_inv, int n, int W, int kind, double beta, double i0b,
                             double sigma, GaussLegendre gl)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    double nu = (double)(p - n / 2) / n, c;
    if (W == 1) {
        c = 1.0;
    } else if (kind == RICK_KERNEL_KB) {
        double a = beta * beta - (M_PI * W * nu) * (M_PI * W * nu);
        if (a > 1e-30) {
            double r = sqrt(a);
            c = W * sinh(r) / r;
        } else if (a < -1e-30) {
            double r = sqrt(-a);
            c = W * sin(r) / r;
        } else {
            c = W;
        }
        c /= i0b;
    } else {
        // the even integrand e^{-d^2 / (2 sigma^2)} cos(2 pi nu d) is entire and
        // at most a few oscillations long on [0, W/2]: twice its 48-point
        // Gauss-Legendre sum there is exact to rounding
        const double half = 0.25 * W;  // d = half (t + 1), t in [-1, 1]
        double s = 0.0;
        for (int i = 0; i < RICK_GL_N; ++i) {
            const double d = half * (gl.x[i] + 1.0);
            s += gl.w[i] * exp(-d * d / (2.0 * sigma * sigma)) * cos(2.0 * M_PI * nu * d);
        }
        c = 2.0 * half * s;
    }
    taper_inv[p] = (float)(1.0 / c);
}

// Kernel-weight polynomials (one thread per segment j, FP64): G((j - h) - f)
// sampled at the RICK_POLY_N Chebyshev nodes of s = 2 (f - fc) in [-1, 1],
// Chebyshev coefficients by the discrete orthogonality sums, then the
// Chebyshev series rewritten in powers of s with T_{k+1} = 2 s T_k - T_{k-1}.
__global__ void kernel_poly_kernel(float *coef, int W, int kind, double beta, double i0b,
                                   double sigma)
{
    const int j = threadIdx.x;
    if (j >= W) return;
    const int N = RICK_POLY_N;
    const int h = (W & 1) ? (W - 1) / 2 : W / 2 - 1;
    const double fc = (W & 1) ? 0.0 : 0.5;
    double val[RICK_POLY_N], a[RICK_POLY_N], c[RICK_POLY_N], t0[RICK_POLY_N], t1[RICK_POLY_N],
        t2[RICK_POLY_N];
    for (int q = 0; q < N; ++q) {
        double s = cos(M_PI * (q + 0.5) / N);
        double d = (double)(j - h) - (fc + 0.5 * s);
        double g;
        if (kind == RICK_KERNEL_KB) {
            double t = 2.0 * d / W, u = 1.0 - t * t;
            g = u > 0.0 ? cyl_bessel_i0(beta * sqrt(u)) / i0b : 1.0 / i0b;
        } else {
            g = exp(-d * d / (2.0 * sigma * sigma));
        }
        val[q] = g;
    }
    for (int k = 0; k < N; ++k) {
        double sum = 0.0;
        for (int q = 0; q < N; ++q) sum += val[q] * cos(M_PI * k * (q + 0.5) / N);
        a[k] = (k == 0 ? 1.0 : 2.0) * sum / N;
    }
    for (int k = 0; k < N; ++k) c[k] = t0[k] = t1[k] = 0.0;
    t0[0] = 1.0;
    t1[1] = 1.0;
    c[0] = a[0];
    for (int k = 0; k < N; ++k) c[k] += a[1] * t1[k];
    for (int m = 2; m < N; ++m) {
        for (int k = 0; k < N; ++k) t2[k] = (k > 0 ? 2.0 * t1[k - 1] : 0.0) - t0[k];
        for (int k = 0; k < N; ++k) {
            c[k] += a[m] * t2[k];
            t0[k] = t1[k];
            t1[k] = t2[k];
        }
    }
    for (int k = 0; k < N; ++k) coef[j * N + k] = (float)c[k];
}

// The default KB shape is Beatty's for oversampling 2 (0 where that has no
// real root: W == 1, which needs no shape).
static double kb_beta_of(const rick_params *p)
{
    if (!isnan(p->kb_beta)) return p->kb_beta;
    const double b = rick_kb_beta(p->support, 2.0);
    return isnan(b) ? 0.0 : b;
}

static double bessel_i0_host(double x)
{
    double q = 0.25 * x * x, term = 1.0, sum = 1.0;
    for (int j = 1; j < 1000 && term > 1e-18 * sum; ++j) {
        term *= q / ((double)j * j);
        sum += term;
    }
    return sum;
}

// Plan creation and destruction do not synchronise the device: the plan gets
// its own non-blocking stream, its tables and the cuFFT work area are
// allocated stream-ordered on it, and only that stream is waited for.  Work of
// other plans on other streams keeps running meanwhile.
static void plan_release(rick_plan *pl)
{
    if (pl->fft) cufftDestroy(pl->fft);
    cudaEvent_t evs[4] = {pl->ev_start, pl->ev_uvw, pl->ev_area_free[0], pl->ev_area_free[1]};
    for (cudaEvent_t e : evs)
        if (e) cudaEventDestroy(e);
    for (int b = 0; b < RICK_STREAM_BUFS; ++b) {
        if (pl->ev_ready[b]) cudaEventDestroy(pl->ev_ready[b]);
        if (pl->ev_free[b]) cudaEventDestroy(pl->ev_free[b]);
    }
    if (pl->copy) cudaStreamDestroy(pl->copy);
    if (pl->own) {
        if (pl->taper_inv) cudaFreeAsync(pl->taper_inv, pl->own);
        if (pl->twid) cudaFreeAsync(pl->twid, pl->own);
        if (pl->fft_work) cudaFreeAsync(pl->fft_work, pl->own);
        cudaStreamSynchronize(pl->own);
        cudaStreamDestroy(pl->own);
    }
    free(pl);
}

// The kernel-dependent tables of a plan: 1/C(nu) on the device and the
// kernel-weight polynomial coefficients (fitted on the device in FP64, kept on
// the host for the kernels' parameter space).  Waits for the plan's own
// stream, which holds nothing but this work.
static bool kernel_tables(rick_plan *pl)
{
    const rick_params *params = &pl->p;
    const int n = params->n;
    float *coef = NULL;
    bool ok = cudaMallocAsync((void **)&coef, sizeof(float) * RICK_MAX_W * RICK_POLY_N, pl->own) ==
              cudaSuccess;
    if (ok) {
        pl->launches += 2;
        taper_kernel<<<(n + 255) / 256, 256, 0, pl->own>>>(pl->taper_inv, n, params->support,
                                                           params->kernel, pl->beta, pl->i0_beta,
                                                           pl->sigma, gauss_legendre());
        ok = cudaGetLastError() == cudaSuccess &&
             cudaMemsetAsync(coef, 0, sizeof(float) * RICK_MAX_W * RICK_POLY_N, pl->own) ==
                 cudaSuccess;
        if (ok) {
            kernel_poly_kernel<<<1, RICK_MAX_W, 0, pl->own>>>(coef, params->support, params->kernel,
                                                             pl->beta, pl->i0_beta, pl->sigma);
            ok = cudaGetLastError() == cudaSuccess &&
                 cudaMemcpyAsync(pl->poly.c, coef, sizeof(pl->poly.c), cudaMemcpyDeviceToHost,
                                 pl->own) == cudaSuccess;
        }
        cudaFreeAsync(coef, pl->own);
        ok = ok && cudaStreamSynchronize(pl->own) == cudaSuccess;
    }
    pl->poly.fc = (params->support & 1) ? 0.0f : 0.5f;
    return ok;
}

extern "C" rick_status rick_plan_create(const rick_params *params, int64_t max_vis, rick_plan **out)
{
    if (!out) return RICK_EINVAL;
    rick_status st = check_params(params);
    if (st != RICK_OK) return st;
    if (max_vis < 0 || rick_n_records(params, max_vis) >= (1ll << 31)) return RICK_EINVAL;
    rick_plan *pl = (rick_plan *)calloc(1, sizeof(rick_plan));
    if (!pl) return RICK_ENOMEM;
    pl->p = *params;
    pl->max_vis = max_vis;
    pl->wait_polls = RICK_WAIT_POLLS;
    pl->n_w_created = params->n_w;
    if (cudaGetDevice(&pl->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&pl->num_sms, cudaDevAttrMultiProcessorCount, pl->device) !=
            cudaSuccess ||
        cudaStreamCreateWithFlags(&pl->own, cudaStreamNonBlocking) != cudaSuccess) {
        free(pl);
        return RICK_ECUDA;
    }
    pl->beta = kb_beta_of(params);
    pl->sigma = isnan(params->gauss_sigma) ? params->support / 6.0 : params->gauss_sigma;
    pl->i0_beta = bessel_i0_host(pl->beta);

    // batched 2D C2C plan; the work area is ours (stream-ordered allocation)
    int n = params->n;
    long long dims[2] = {n, n}, dist = (long long)n * n;
    cufftResult fr = cufftCreate(&pl->fft);
    if (fr == CUFFT_SUCCESS) fr = cufftSetAutoAllocation(pl->fft, 0);
    if (fr == CUFFT_SUCCESS)
        fr = cufftMakePlanMany64(pl->fft, 2, dims, NULL, 1, dist, NULL, 1, dist, CUFFT_C2C,
                                 params->n_w, &pl->fft_bytes);
    if (fr != CUFFT_SUCCESS) {
        plan_release(pl);
        return fr == CUFFT_ALLOC_FAILED ? RICK_ENOMEM : RICK_ECUFFT;
    }
    if ((pl->fft_bytes && cudaMallocAsync(&pl->fft_work, pl->fft_bytes, pl->own) != cudaSuccess) ||
        cudaMallocAsync((void **)&pl->taper_inv, sizeof(float) * n, pl->own) != cudaSuccess) {
        plan_release(pl);
        return RICK_ENOMEM;
    }
    if (pl->fft_bytes && cufftSetWorkArea(pl->fft, pl->fft_work) != CUFFT_SUCCESS) {
        plan_release(pl);
        return RICK_ECUFFT;
    }
    if (!rick_fft_tables(pl) || !kernel_tables(pl)) {
        plan_release(pl);
        return RICK_ECUDA;
    }
    pl->sticky = RICK_OK;
    *out = pl;
    return RICK_OK;
}

extern "C" rick_status rick_plan_set_kernel(rick_plan *plan, int32_t kernel, int32_t support,
                                            double kb_beta, double gauss_sigma)
{
    if (!plan) return RICK_EINVAL;
    if (plan->sticky != RICK_OK) return plan->sticky;
    rick_params q = plan->p;
    q.kernel = kernel;
    q.support = support;
    q.kb_beta = kb_beta;
    q.gauss_sigma = gauss_sigma;
    rick_status st = check_params(&q);
    if (st != RICK_OK) return st;
    plan->p = q;
    plan->beta = kb_beta_of(&q);
    plan->sigma = isnan(q.gauss_sigma) ? q.support / 6.0 : q.gauss_sigma;
    plan->i0_beta = bessel_i0_host(plan->beta);
    if (!kernel_tables(plan)) {
        plan->sticky = RICK_ECUDA;
        return RICK_ECUDA;
    }
    return RICK_OK;
}

// The caller guarantees that no work enqueued with the plan is still pending.
extern "C" rick_status rick_plan_destroy(rick_plan *plan)
{
    if (!plan) return RICK_OK;
    plan_release(plan);
    return RICK_OK;
}

extern "C" rick_status rick_plan_last_error(const rick_plan *plan)
{
    return plan ? plan->sticky : RICK_EINVAL;
}

extern "C" rick_status rick_plan_set_geometry(rick_plan *plan, double fov, double w_min,
                                              double w_max)
{
    if (!plan) return RICK_EINVAL;
    rick_params q = plan->p;
    q.fov = fov;
    q.w_min = w_min;
    q.w_max = w_max;
    rick_status st = check_params(&q);
    if (st != RICK_OK) return st;
    plan->p = q;
    return RICK_OK;
}

extern "C" rick_status rick_plan_set_image_n(rick_plan *plan, int32_t image_n)
{
    if (!plan) return RICK_EINVAL;
    rick_params q = plan->p;
    q.image_n = image_n;
    rick_status st = check_params(&q);
    if (st != RICK_OK) return st;
    plan->p = q;
    return RICK_OK;
}

extern "C" rick_status rick_plan_set_planes(rick_plan *plan, int32_t n_w)
{
    if (!plan || n_w < 1 || n_w > plan->n_w_created) return RICK_EINVAL;
    rick_params q = plan->p;
    q.n_w = n_w;
    rick_status st = check_params(&q);
    if (st != RICK_OK) return st;
    plan->p = q;
    return RICK_OK;
}

extern "C" rick_status rick_plan_set_wait_limit(rick_plan *plan, uint32_t polls)
{
    if (!plan) return RICK_EINVAL;
    plan->wait_polls = polls;
    return RICK_OK;
}

extern "C" rick_status rick_plan_launch_count(const rick_plan *plan, uint64_t *count)
{
    if (!plan || !count) return RICK_EINVAL;
    *count = plan->launches;
    return RICK_OK;
}

extern "C" rick_status rick_workspace_bytes(const rick_params *params, int64_t n_vis,
                                            size_t *bin_bytes, size_t *plane_bytes)
{
    rick_status st = check_params(params);
    if (st != RICK_OK) return st;
    if (n_vis < 0 || n_vis >= (1ll << 31)) return RICK_EINVAL;
    WsLayout L = rick_ws_layout(params, n_vis);
    if (bin_bytes) *bin_bytes = L.total;
    if (plane_bytes) *plane_bytes = (size_t)params->n_w * params->n * params->n * 8;
    return RICK_OK;
}

extern "C" rick_status rick_fused_work_bytes(const rick_params *params, size_t *work_bytes)
{
    if (!work_bytes) return RICK_EINVAL;
    rick_status st = check_params(params);
    if (st != RICK_OK) return st;
    *work_bytes = rick_fft_work_bytes(params);
    return RICK_OK;
}

extern "C" rick_status rick_plan_fft_bytes(const rick_plan *plan, size_t *fft_bytes)
{
    if (!plan || !fft_bytes) return RICK_EINVAL;
    *fft_bytes = plan->fft_bytes;
    return RICK_OK;
}

extern "C" rick_status rick_fft_wplanes(rick_plan *plan, void *planes, int32_t direction,
                                        void *stream)
{
    if (!plan || !planes || (direction != 1 && direction != -1)) return RICK_EINVAL;
    if (plan->sticky != RICK_OK) return plan->sticky;
    // the batched cuFFT plan transforms the plane count it was made for
    if (((uintptr_t)planes & 7) != 0 || plan->p.n_w != plan->n_w_created) return RICK_EINVAL;
    if (cufftSetStream(plan->fft, (cudaStream_t)stream) != CUFFT_SUCCESS ||
        cufftExecC2C(plan->fft, (cufftComplex *)planes, (cufftComplex *)planes,
                     direction > 0 ? CUFFT_INVERSE : CUFFT_FORWARD) != CUFFT_SUCCESS) {
        plan->sticky = RICK_ECUFFT;
        return RICK_ECUFFT;
    }
    return RICK_OK;
}

extern "C" rick_status rick_bin_layout(const rick_plan *plan, rick_bin_view *out)
{
    if (!plan || !out) return RICK_EINVAL;
    WsLayout L = rick_ws_layout(&plan->p, plan->max_vis);
    out->offsets = L.offsets;
    out->perm = L.perm;
    out->rec = L.rec;
    out->rec_cell = L.rcell;
    out->stats = L.header + offsetof(WsHeader, stats);
    out->n_bins = L.nbins;
    return RICK_OK;
}

// rick_weights.cu -- imaging weights from the uv-cell density: uniform and
// Briggs-robust weighting (§2 of the paper names Briggs 1995 for the
// weighting of the visibilities).
//
// The density D of a uv cell is the sum of the natural weights of the kept
// visibilities whose centre cell c = a + h (the cell nearest to (x, y)) it is,
// over all w-planes.  Uniform weighting divides each weight by its cell's D;
// Briggs' robust weighting with robustness R divides it by 1 + f^2 D, where
// f^2 = (5 10^-R)^2 / (sum_cells D^2 / sum w).  The pass reads the corners and
// keys that the binning left in the workspace, so it follows a rick_bin (or
// rick_bin_channels) of the same visibilities and weights; the new weights go
// back into the records with rick_bin_values.
#include "rick_common.cuh"

#define WFULL 0xffffffffu

struct DensityHeader {
    double sum_d2;  // sum over cells of D^2
    double f2;      // Briggs' f^2
};

#define RICK_DENSITY_PARTIALS 2048  // per-block partial sums of D^2 (at most)

struct DensityLayout {
    size_t header, partials, dens, total;
};

static DensityLayout density_layout(const rick_params *p)
{
    DensityLayout D;
    size_t o = 0;
    D.header = o;   o += rick_align256(sizeof(DensityHeader));
    D.partials = o; o += rick_align256(8 * (size_t)RICK_DENSITY_PARTIALS);
    D.dens = o;     o += rick_align256(4 * (size_t)p->n * p->n);
    D.total = o;
    return D;
}

// D[centre cell] += w over the kept inputs; consecutive lanes with the same
// cell (the channels of one baseline and time) add their weights first and
// take one atomic per run.
__global__ void __launch_bounds__(256) density_kernel(int64_t n_vis, const uint32_t *key,
                                                      const uint32_t *cell, const float *weight,
                                                      int h, int n, float *dens)
{
    const int lane = threadIdx.x & 31;
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x; i0 < n_vis;
         i0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = i0 + threadIdx.x;
        uint32_t c = 0xFFFFFFFFu;
        float w = 0.0f;
        if (i < n_vis && key[i] != 0xFFFFFFFFu) {
            c = cell[i];
            w = weight ? weight[i] : 1.0f;
        }
        const uint32_t prev = __shfl_up_sync(WFULL, c, 1);
        const unsigned starts = __ballot_sync(WFULL, lane == 0 || c != prev);
        const unsigned after = lane == 31 ? 0u : starts & (0xFFFFFFFFu << (lane + 1));
        const int end = after ? __ffs(after) - 1 : 32;  // one past the last lane of this run
        // segmented sum: lane ends up with the sum over [lane, end)
        for (int o = 1; o < 32; o <<= 1) {
            const float t = __shfl_down_sync(WFULL, w, o);
            if (lane + o < end) w += t;
        }
        if (c != 0xFFFFFFFFu && ((starts >> lane) & 1u))
            atomicAdd(&dens[(size_t)((c >> 16) + h) * n + (c & 0xFFFFu) + h], w);
    }
}

// Per-block partial sums of D^2 in FP64 (fixed order inside a block).
__global__ void __launch_bounds__(256) density_sq_kernel(const float *dens, int64_t cells,
                                                         double *partials)
{
    __shared__ double s[256];
    double t = 0.0;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < cells;
         k += (int64_t)gridDim.x * blockDim.x) {
        const double d = dens[k];
        t += d * d;
    }
    s[threadIdx.x] = t;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = s[0];
}

// f^2 = c2 / (sum D^2 / sum w), c2 = (5 10^-R)^2; sum w is the binning's.
__global__ void density_f2_kernel(const double *partials, int nparts, const WsHeader *hdr,
                                  double c2, DensityHeader *dh)
{
    double s2 = 0.0;
    for (int k = 0; k < nparts; ++k) s2 += partials[k];
    dh->sum_d2 = s2;
    dh->f2 = s2 > 0.0 ? c2 * hdr->stats.sum_weight / s2 : 0.0;
}

__global__ void __launch_bounds__(256) reweight_kernel(int64_t n_vis, const uint32_t *key,
                                                       const uint32_t *cell, const float *weight,
                                                       int h, int n, const float *dens,
                                                       const DensityHeader *dh, int uniform,
                                                       float *out)
{
    const float f2 = uniform ? 0.0f : (float)dh->f2;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_vis;
         i += (int64_t)gridDim.x * blockDim.x) {
        float r = 0.0f;
        if (key[i] != 0xFFFFFFFFu) {
            const uint32_t c = cell[i];
            const float d = dens[(size_t)((c >> 16) + h) * n + (c & 0xFFFFu) + h];
            const float w = weight ? weight[i] : 1.0f;
            if (uniform)
                r = d > 0.0f ? w / d : 0.0f;
            else
                r = w / __fmaf_rn(f2, d, 1.0f);
        }
        out[i] = r;
    }
}

extern "C" rick_status rick_density_scratch_bytes(const rick_params *params, size_t *bytes)
{
    if (!params || !bytes) return RICK_EINVAL;
    *bytes = density_layout(params).total;
    return RICK_OK;
}

extern "C" rick_status rick_density_weights(rick_plan *plan, int64_t n_vis,
                                            const float *weight_dev, void *ws_dev, int32_t scheme,
                                            double robust, void *scratch_dev,
                                            size_t scratch_bytes, float *weight_out_dev,
                                            void *stream)
{
    if (!plan || !ws_dev || !scratch_dev || (n_vis > 0 && !weight_out_dev) || n_vis < 0)
        return RICK_EINVAL;
    if (plan->sticky != RICK_OK) return plan->sticky;
    if (scheme != RICK_WEIGHT_UNIFORM && scheme != RICK_WEIGHT_BRIGGS) return RICK_EINVAL;
    if (scheme == RICK_WEIGHT_BRIGGS && !isfinite(robust)) return RICK_EINVAL;
    if (((uintptr_t)ws_dev & 255) || ((uintptr_t)scratch_dev & 255) ||
        ((uintptr_t)weight_dev & 3) || ((uintptr_t)weight_out_dev & 3))
        return RICK_EINVAL;
    if (n_vis > plan->max_vis) return RICK_ERANGE;
    const rick_params &p = plan->p;
    if (p.options & RICK_OPT_HERMITIAN_MIRROR) return RICK_EINVAL;  // per-input records only
    const DensityLayout D = density_layout(&p);
    if (scratch_bytes < D.total) return RICK_ERANGE;
    const WsPtrs w = rick_ws_ptrs(ws_dev, rick_ws_layout(&p, plan->max_vis));
    char *sb = (char *)scratch_dev;
    DensityHeader *dh = (DensityHeader *)(sb + D.header);
    double *partials = (double *)(sb + D.partials);
    float *dens = (float *)(sb + D.dens);
    cudaStream_t st = (cudaStream_t)stream;
    const int W = p.support, h = (W % 2) ? (W - 1) / 2 : W / 2 - 1;
    const int64_t cells = (int64_t)p.n * p.n;

    RICK_CUDA_TRY(plan, cudaMemsetAsync(dens, 0, 4 * (size_t)cells, st));
    int blocks = (int)((n_vis + 255) / 256);
    if (blocks > plan->num_sms * 16) blocks = plan->num_sms * 16;
    if (blocks < 1) blocks = 1;
    density_kernel<<<blocks, 256, 0, st>>>(n_vis, w.key, w.cell, weight_dev, h, p.n, dens);
    RICK_LAUNCH_CHECK(plan);
    if (scheme == RICK_WEIGHT_BRIGGS) {
        int nb = plan->num_sms * 4;
        if (nb > RICK_DENSITY_PARTIALS) nb = RICK_DENSITY_PARTIALS;
        density_sq_kernel<<<nb, 256, 0, st>>>(dens, cells, partials);
        RICK_LAUNCH_CHECK(plan);
        const double c = 5.0 * pow(10.0, -robust);
        density_f2_kernel<<<1, 1, 0, st>>>(partials, nb, w.hdr, c * c, dh);
        RICK_LAUNCH_CHECK(plan);
    }
    reweight_kernel<<<blocks, 256, 0, st>>>(n_vis, w.key, w.cell, weight_dev, h, p.n, dens, dh,
                                            scheme == RICK_WEIGHT_UNIFORM, weight_out_dev);
    RICK_LAUNCH_CHECK(plan);
    return RICK_OK;
}

// rick_grid.cu -- convolutional gridding (Eq. 3 of De Rubeis et al.) and its
// adjoint, degridding.
//
// Gridding: one CTA per work item = (uv-tile of one w-plane, chunk of at most
// chunk_cap records).  The CTA owns the T x T output cells of its tile: it sums
// into a shared-memory accumulator the records binned at the tile (footprint
// corner inside it) and the records of the west / north / north-west tiles
// whose footprints reach into it (their edge classes), each clipped to the
// tile, then writes the tile once with plain coalesced stores.  The
// checkerboard (-1)^(i+j) of the centred FFT is applied in that write.  A tile
// with more than one chunk is zeroed first and its chunks add their sums with
// float2 atomics.  No global atomics otherwise, and no separate zero-fill of
// the planes: every cell is written by the CTA that owns it.
//
// Degridding: one CTA per chunk of a non-empty tile's own bin; the CTA stages
// the (T + W - 1)^2 plane region its records can touch into shared memory and
// each thread gathers one record's W x W footprint.
#include "rick_common.cuh"

struct GridArgs {
    TileArgs t;
    float2 *planes;
    int log2T;
};

struct DegridArgs {
    TileArgs t;
    const float2 *planes;
    const float *weight;
    float2 *vis_out;
    int log2T;
};

// Largest t in [0, ntiles) with base[t] <= b (base non-decreasing).
__device__ __forceinline__ uint32_t find_tile(const uint32_t *base, uint32_t ntiles, uint32_t b)
{
    uint32_t lo = 0, hi = ntiles;
    while (hi - lo > 1) {
        uint32_t mid = (lo + hi) >> 1;
        if (base[mid] <= b)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

template <int W>
__device__ __forceinline__ void kernel_weights(const KernelShape &ks, float f, float *g)
{
    const int h = (W & 1) ? (W - 1) / 2 : W / 2 - 1;
    if (W == 1) {
        g[0] = 1.0f;
        return;
    }
    if (ks.kind == RICK_KERNEL_KB) {
#pragma unroll
        for (int j = 0; j < W; ++j) g[j] = rick_g<RICK_KERNEL_KB>(ks, (float)(j - h) - f);
    } else {
#pragma unroll
        for (int j = 0; j < W; ++j) g[j] = rick_g<RICK_KERNEL_GAUSS>(ks, (float)(j - h) - f);
    }
}

// Add one record's footprint, clipped to the tile, into the accumulator.
template <int W>
__device__ __forceinline__ void splat(float *acc_re, float *acc_im, int T, int log2T, int lx,
                                      int ly, float2 val, const float *gx, const float *gy)
{
#pragma unroll
    for (int jy = 0; jy < W; ++jy) {
        int row = ly + jy;
        if ((unsigned)row >= (unsigned)T) continue;
        float vr = val.x * gy[jy], vi = val.y * gy[jy];
        int rbase = row << log2T;
#pragma unroll
        for (int jx = 0; jx < W; ++jx) {
            int col = lx + jx;
            if ((unsigned)col >= (unsigned)T) continue;
            atomicAdd(&acc_re[rbase + col], vr * gx[jx]);
            atomicAdd(&acc_im[rbase + col], vi * gx[jx]);
        }
    }
}

// Neumaier's compensated summation of a into (s, c).
__device__ __forceinline__ void neumaier(float &s, float &c, float a)
{
    float t = s + a;
    if (fabsf(s) >= fabsf(a))
        c += (s - t) + a;
    else
        c += (a - t) + s;
    s = t;
}

template <int W, bool COMP>
__global__ void __launch_bounds__(256) grid_kernel(GridArgs a)
{
    extern __shared__ float sm[];
    const TileArgs &ta = a.t;
    const uint32_t b = blockIdx.x;
    if (b >= ta.base[ta.ntiles]) return;
    __shared__ uint32_t s_tile;
    if (threadIdx.x == 0) s_tile = find_tile(ta.base, ta.ntiles, b);
    __syncthreads();
    const uint32_t t = s_tile;
    const uint32_t chunk = b - ta.base[t], nch = ta.base[t + 1] - ta.base[t];
    const int T = 1 << a.log2T, TT = T * T, nt = ta.nt;
    const uint32_t tx = t % nt, ty = (t / nt) % nt, k = t / (nt * nt);
    const int x0 = tx << a.log2T, y0 = ty << a.log2T;
    const uint32_t *off = ta.offsets;

    // the four record ranges that can touch this tile
    uint32_t s0 = off[4 * t], L0 = off[4 * t + 4] - s0;
    uint32_t s1 = 0, L1 = 0, s2 = 0, L2 = 0, s3 = 0, L3 = 0;
    if (tx > 0) {
        s1 = off[4 * (t - 1) + 1];
        L1 = off[4 * (t - 1) + 3] - s1;
    }
    if (ty > 0) {
        s2 = off[4 * (t - nt) + 2];
        L2 = off[4 * (t - nt) + 4] - s2;
    }
    if (tx > 0 && ty > 0) {
        s3 = off[4 * (t - nt - 1) + 2];
        L3 = off[4 * (t - nt - 1) + 3] - s3;
    }
    const uint32_t Ltot = L0 + L1 + L2 + L3;
    const uint32_t vbeg = chunk * ta.chunk_cap;
    const uint32_t vend = min(Ltot, vbeg + ta.chunk_cap);

    float *acc_re = sm, *acc_im = sm + TT;
    float *sum_re = sm + 2 * TT, *sum_im = sm + 3 * TT, *cmp_re = sm + 4 * TT, *cmp_im = sm + 5 * TT;
    for (int i = threadIdx.x; i < TT; i += blockDim.x) {
        acc_re[i] = 0.0f;
        acc_im[i] = 0.0f;
        if (COMP) {
            sum_re[i] = sum_im[i] = cmp_re[i] = cmp_im[i] = 0.0f;
        }
    }
    __syncthreads();

    const uint32_t SUB = COMP ? 1024u : 0xFFFFFFFFu;  // records per compensated fold
    for (uint32_t sb = vbeg; sb < vend; sb += (COMP ? SUB : (vend - vbeg))) {
        const uint32_t se = COMP ? min(vend, sb + SUB) : vend;
        for (uint32_t v = sb + threadIdx.x; v < se; v += blockDim.x) {
            uint32_t r;
            if (v < L0)
                r = s0 + v;
            else if (v < L0 + L1)
                r = s1 + (v - L0);
            else if (v < L0 + L1 + L2)
                r = s2 + (v - L0 - L1);
            else
                r = s3 + (v - L0 - L1 - L2);
            float2 val = ta.rval[r];
            float2 fr = ta.rfrac[r];
            uint32_t cell = ta.rcell[r];
            int lx = (int)(cell & 0xFFFFu) - x0, ly = (int)(cell >> 16) - y0;
            float gx[W], gy[W];
            kernel_weights<W>(ta.ks, fr.x, gx);
            kernel_weights<W>(ta.ks, fr.y, gy);
            splat<W>(acc_re, acc_im, T, a.log2T, lx, ly, val, gx, gy);
        }
        if (COMP) {
            __syncthreads();
            for (int i = threadIdx.x; i < TT; i += blockDim.x) {
                neumaier(sum_re[i], cmp_re[i], acc_re[i]);
                neumaier(sum_im[i], cmp_im[i], acc_im[i]);
                acc_re[i] = 0.0f;
                acc_im[i] = 0.0f;
            }
            __syncthreads();
        }
    }
    if (!COMP) __syncthreads();

    // flush: (-1)^(i+j) folded in; plain stores unless the tile has several chunks
    const int n = ta.n;
    float2 *plane = a.planes + (size_t)k * n * n;
    for (int i = threadIdx.x; i < TT; i += blockDim.x) {
        int row = i >> a.log2T, col = i & (T - 1);
        int gi = x0 + col, gj = y0 + row;
        float re = COMP ? sum_re[i] + cmp_re[i] : acc_re[i];
        float im = COMP ? sum_im[i] + cmp_im[i] : acc_im[i];
        if ((gi + gj) & 1) {
            re = -re;
            im = -im;
        }
        float2 *dst = plane + (size_t)gj * n + gi;
        if (nch == 1) {
            *dst = make_float2(re, im);
        } else if (re != 0.0f || im != 0.0f) {
            atomicAdd(dst, make_float2(re, im));
        }
    }
}

// Zero the tiles that several chunks add into (grid-stride, one warp per tile).
__global__ void zero_multi_kernel(const uint32_t *base, uint32_t ntiles, int nt, int log2T, int n,
                                  float2 *planes)
{
    int lane = threadIdx.x & 31;
    uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    const int T = 1 << log2T;
    for (uint32_t t = warp; t < ntiles; t += nwarps) {
        if (base[t + 1] - base[t] <= 1) continue;
        uint32_t tx = t % nt, ty = (t / nt) % nt, k = t / (nt * nt);
        float2 *plane = planes + (size_t)k * n * n;
        for (int i = lane; i < T * T; i += 32) {
            int row = i >> log2T, col = i & (T - 1);
            plane[(size_t)((ty << log2T) + row) * n + (tx << log2T) + col] = make_float2(0.f, 0.f);
        }
    }
}

template <int W>
__global__ void __launch_bounds__(256) degrid_kernel(DegridArgs a)
{
    extern __shared__ float2 stage[];
    const TileArgs &ta = a.t;
    const uint32_t b = blockIdx.x;
    if (b >= ta.base[ta.ntiles]) return;
    __shared__ uint32_t s_tile;
    if (threadIdx.x == 0) s_tile = find_tile(ta.base, ta.ntiles, b);
    __syncthreads();
    const uint32_t t = s_tile;
    const uint32_t chunk = b - ta.base[t];
    const int T = 1 << a.log2T, S = T + W - 1, nt = ta.nt, n = ta.n;
    const uint32_t tx = t % nt, ty = (t / nt) % nt, k = t / (nt * nt);
    const int x0 = tx << a.log2T, y0 = ty << a.log2T;
    const uint32_t r0 = ta.offsets[4 * t] + chunk * ta.chunk_cap;
    const uint32_t r1 = min(ta.offsets[4 * t + 4], r0 + ta.chunk_cap);

    const float2 *plane = a.planes + (size_t)k * n * n;
    for (int i = threadIdx.x; i < S * S; i += blockDim.x) {
        int row = i / S, col = i - row * S;
        int gi = x0 + col, gj = y0 + row;
        float2 v = make_float2(0.f, 0.f);
        if (gi < n && gj < n) {
            v = plane[(size_t)gj * n + gi];
            if ((gi + gj) & 1) {
                v.x = -v.x;
                v.y = -v.y;
            }
        }
        stage[i] = v;
    }
    __syncthreads();
    for (uint32_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
        float2 fr = ta.rfrac[r];
        uint32_t cell = ta.rcell[r];
        int lx = (int)(cell & 0xFFFFu) - x0, ly = (int)(cell >> 16) - y0;
        float gx[W], gy[W];
        kernel_weights<W>(ta.ks, fr.x, gx);
        kernel_weights<W>(ta.ks, fr.y, gy);
        float sr = 0.f, si = 0.f;
#pragma unroll
        for (int jy = 0; jy < W; ++jy) {
            const float2 *rowp = stage + (ly + jy) * S + lx;
            float rr = 0.f, ri = 0.f;
#pragma unroll
            for (int jx = 0; jx < W; ++jx) {
                float2 c = rowp[jx];
                rr = fmaf(gx[jx], c.x, rr);
                ri = fmaf(gx[jx], c.y, ri);
            }
            sr = fmaf(gy[jy], rr, sr);
            si = fmaf(gy[jy], ri, si);
        }
        uint32_t m = ta.perm[r];
        float wt = a.weight ? a.weight[m] : 1.0f;
        a.vis_out[m] = make_float2(sr * wt, si * wt);
    }
}

// Dropped visibilities (key == all ones) get a zero model value.
__global__ void degrid_zero_dropped_kernel(const WsHeader *hdr, const uint32_t *key, float2 *vis_out)
{
    int64_t n = (int64_t)hdr->n_vis;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        if (key[i] == 0xFFFFFFFFu) vis_out[i] = make_float2(0.f, 0.f);
}

// ------------------------------------------------------------------------

static TileArgs make_tile_args(const rick_plan *plan, const WsPtrs &w, const uint32_t *base,
                               uint32_t cap)
{
    const rick_params &p = plan->p;
    TileArgs t;
    t.n = p.n;
    t.n_w = p.n_w;
    t.T = p.tile;
    t.nt = p.n / p.tile;
    t.W = p.support;
    t.ntiles = (uint32_t)p.n_w * t.nt * t.nt;
    t.chunk_cap = cap;
    t.offsets = w.offsets;
    t.base = base;
    t.perm = w.perm;
    t.rcell = w.rcell;
    t.rval = w.rval;
    t.rfrac = w.rfrac;
    t.hdr = w.hdr;
    t.ks.kind = p.kernel;
    t.ks.beta = (float)plan->beta;
    t.ks.inv_i0b = (float)(1.0 / plan->i0_beta);
    t.ks.two_over_w = 2.0f / p.support;
    t.ks.inv_2s2 = (float)(1.0 / (2.0 * plan->sigma * plan->sigma));
    return t;
}

static int ilog2(int x)
{
    int l = 0;
    while ((1 << l) < x) ++l;
    return l;
}

template <int W>
static cudaError_t launch_grid(const GridArgs &a, bool comp, unsigned blocks, cudaStream_t st)
{
    size_t TT = (size_t)a.t.T * a.t.T;
    size_t smem = (comp ? 6 : 2) * TT * sizeof(float);
    if (comp) {
        cudaFuncSetAttribute(grid_kernel<W, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
        grid_kernel<W, true><<<blocks, 256, smem, st>>>(a);
    } else {
        cudaFuncSetAttribute(grid_kernel<W, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
        grid_kernel<W, false><<<blocks, 256, smem, st>>>(a);
    }
    return cudaGetLastError();
}

template <int W>
static cudaError_t launch_degrid(const DegridArgs &a, unsigned blocks, cudaStream_t st)
{
    size_t S = a.t.T + W - 1;
    size_t smem = S * S * sizeof(float2);
    cudaFuncSetAttribute(degrid_kernel<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    degrid_kernel<W><<<blocks, 256, smem, st>>>(a);
    return cudaGetLastError();
}

#define RICK_W_SWITCH(W, CALL)          \
    switch (W) {                        \
    case 1: CALL(1); break;             \
    case 2: CALL(2); break;             \
    case 3: CALL(3); break;             \
    case 4: CALL(4); break;             \
    case 5: CALL(5); break;             \
    case 6: CALL(6); break;             \
    case 7: CALL(7); break;             \
    case 8: CALL(8); break;             \
    case 9: CALL(9); break;             \
    case 10: CALL(10); break;           \
    case 11: CALL(11); break;           \
    case 12: CALL(12); break;           \
    case 13: CALL(13); break;           \
    case 14: CALL(14); break;           \
    case 15: CALL(15); break;           \
    case 16: CALL(16); break;           \
    default: err = cudaErrorInvalidValue; \
    }

extern "C" rick_status rick_grid(rick_plan *plan, const void *ws_dev, void *planes_dev,
                                 void *stream)
{
    if (!plan || !ws_dev || !planes_dev) return RICK_EINVAL;
    if (plan->sticky != RICK_OK) return plan->sticky;
    if (((uintptr_t)ws_dev & 255) || ((uintptr_t)planes_dev & 15)) return RICK_EINVAL;
    const rick_params &p = plan->p;
    WsPtrs w = rick_ws_ptrs((void *)ws_dev, rick_ws_layout(&p, plan->max_vis));
    cudaStream_t st = (cudaStream_t)stream;
    // The chunk cap and work totals live on the device; the launch uses the
    // host-side bound: every tile has at least one item, and the items of the
    // records are at most 4 n_vis / cap (a record touches at most 4 tiles).
    uint32_t cap = rick_chunk_cap(plan->max_vis, plan->num_sms);
    GridArgs a;
    a.t = make_tile_args(plan, w, w.gbase, cap);
    a.planes = (float2 *)planes_dev;
    a.log2T = ilog2(p.tile);
    int64_t bound = (int64_t)a.t.ntiles + (4 * plan->max_vis + cap - 1) / cap + 1;
    cudaError_t err = cudaSuccess;
    zero_multi_kernel<<<plan->num_sms * 4, 256, 0, st>>>(w.gbase, a.t.ntiles, a.t.nt, a.log2T, p.n,
                                                         a.planes);
    RICK_LAUNCH_CHECK(plan);
    bool comp = p.precision == RICK_PREC_FP32_COMPENSATED;
#define CALL_GRID(WW) err = launch_grid<WW>(a, comp, (unsigned)bound, st)
    RICK_W_SWITCH(p.support, CALL_GRID);
#undef CALL_GRID
    ++plan->launches;
    RICK_CUDA_TRY(plan, err);
    return RICK_OK;
}

extern "C" rick_status rick_degrid(rick_plan *plan, const void *ws_dev, const void *planes_dev,
                                   const float *weight_dev, void *vis_out_dev, void *stream)
{
    if (!plan || !ws_dev || !planes_dev || !vis_out_dev) return RICK_EINVAL;
    if (plan->sticky != RICK_OK) return plan->sticky;
    if (((uintptr_t)ws_dev & 255) || ((uintptr_t)planes_dev & 15) || ((uintptr_t)vis_out_dev & 7) ||
        ((uintptr_t)weight_dev & 3))
        return RICK_EINVAL;
    const rick_params &p = plan->p;
    WsPtrs w = rick_ws_ptrs((void *)ws_dev, rick_ws_layout(&p, plan->max_vis));
    cudaStream_t st = (cudaStream_t)stream;
    uint32_t cap = rick_chunk_cap(plan->max_vis, plan->num_sms);
    DegridArgs a;
    a.t = make_tile_args(plan, w, w.dbase, cap);
    a.planes = (const float2 *)planes_dev;
    a.weight = weight_dev;
    a.vis_out = (float2 *)vis_out_dev;
    a.log2T = ilog2(p.tile);
    degrid_zero_dropped_kernel<<<plan->num_sms * 4, 256, 0, st>>>(w.hdr, w.key, a.vis_out);
    RICK_LAUNCH_CHECK(plan);
    int64_t bound = (int64_t)a.t.ntiles + (plan->max_vis + cap - 1) / cap + 1;
    cudaError_t err = cudaSuccess;
#define CALL_DEGRID(WW) err = launch_degrid<WW>(a, (unsigned)bound, st)
    RICK_W_SWITCH(p.support, CALL_DEGRID);
#undef CALL_DEGRID
    ++plan->launches;
    RICK_CUDA_TRY(plan, err);
    return RICK_OK;
}

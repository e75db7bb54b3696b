// rick_bin.cu -- binning of visibilities by (w-plane, uv-tile, edge class)
// (§2, gridding sub-step 1: "an array is created for each slab, concatenating
// the data with u-v coordinates inside the corresponding slab"; here the slab
// is a T x T uv-tile of one w-plane, and a visibility goes to the closest
// w-plane, §2).
//
// Passes, all stream-ordered:
//   1. w range: min / max of the finite w as order-preserving integer keys
//      (exact, deterministic), unless the range is given;
//   2. setup: plane width, the plane boundaries as keys, plane centres;
//   3. key: per visibility two FP64 FMAs give the grid coordinates, everything
//      else (floor, rounding, fraction, plane search) is integer work on the
//      bit patterns -- GB300 runs FP64 at a small fraction of FP32;
//      warp-aggregated histogram; deterministic weight-sum partials;
//   4. exclusive scan of the histogram -> bin offsets;
//   5. scatter: warp-aggregated cursors place each record in its bin;
//   6. work lists of the tile kernels (chunks of at most chunk_cap records).
#include <math.h>

#include <mutex>

#include "rick_common.cuh"

#define FULL 0xffffffffu

// ------------------------------------------------------------------------
// Exclusive scan of uint32 (block of 2048, recursive over block sums)

__global__ void __launch_bounds__(1024) scan_blocks_kernel(const uint32_t *in, uint32_t *out,
                                                           int64_t n, uint32_t *block_sums)
{
    __shared__ uint32_t warp_tot[32];
    int64_t base = (int64_t)blockIdx.x * 2048;
    int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    int64_t i0 = base + 2 * t;
    uint32_t a = i0 < n ? in[i0] : 0u, b = i0 + 1 < n ? in[i0 + 1] : 0u;
    uint32_t s = a + b, inc = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t v = __shfl_up_sync(FULL, inc, o);
        if (lane >= o) inc += v;
    }
    if (lane == 31) warp_tot[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        uint32_t w = warp_tot[lane], wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t v = __shfl_up_sync(FULL, wi, o);
            if (lane >= o) wi += v;
        }
        warp_tot[lane] = wi - w;  // exclusive prefix of the warps
        if (lane == 31) block_sums[blockIdx.x] = wi;
    }
    __syncthreads();
    uint32_t ex = warp_tot[wid] + inc - s;
    if (i0 < n) out[i0] = ex;
    if (i0 + 1 < n) out[i0 + 1] = ex + a;
}

__global__ void scan_add_kernel(uint32_t *out, int64_t n, const uint32_t *block_off)
{
    int64_t i = (int64_t)blockIdx.x * 2048 + threadIdx.x;
    uint32_t add = block_off[blockIdx.x];
    if (i < n) out[i] += add;
    if (i + 1024 < n) out[i + 1024] += add;
}

// out[i] = sum_{j < i} in[j]; in may equal out.  tmp: rick_scan_tmp(n) words.
// *launches counts the kernels enqueued.
static cudaError_t scan_u32(const uint32_t *in, uint32_t *out, int64_t n, uint32_t *tmp,
                            cudaStream_t st, unsigned long long *launches)
{
    if (n <= 0) return cudaSuccess;
    int64_t nb = (n + 2047) / 2048;
    scan_blocks_kernel<<<(unsigned)nb, 1024, 0, st>>>(in, out, n, tmp);
    ++*launches;
    if (nb == 1) return cudaGetLastError();
    cudaError_t e = scan_u32(tmp, tmp, nb, tmp + nb + 1, st, launches);
    if (e != cudaSuccess) return e;
    scan_add_kernel<<<(unsigned)nb, 1024, 0, st>>>(out, n, tmp);
    ++*launches;
    return cudaGetLastError();
}

// ------------------------------------------------------------------------
// Pass 1: w range

// range_src (optional): a header whose w-range keys stand in for a given
// range (the exact range of a larger set, found by an earlier pass).
// n_vis: records (inputs, or twice the inputs with the Hermitian mirror).
__global__ void bin_init_kernel(WsHeader *hdr, uint64_t n_vis, uint32_t chunk_cap, int given,
                                uint64_t wmin_key, uint64_t wmax_key, uint32_t n_key_blocks,
                                const WsHeader *range_src, uint64_t n_src, int mirror)
{
    hdr->n_vis = n_vis;
    hdr->n_src = n_src;
    hdr->mirror = (uint32_t)mirror;
    hdr->fault = 0;
    hdr->drop_uv = 0;
    hdr->drop_w = 0;
    hdr->chunk_cap = chunk_cap;
    hdr->n_key_blocks = n_key_blocks;
    if (range_src) {
        given = 1;
        wmin_key = range_src->wmin_key;
        wmax_key = range_src->wmax_key;
    }
    hdr->range_given = given;
    hdr->wmin_key = given ? wmin_key : ~0ull;
    hdr->wmax_key = given ? wmax_key : 0ull;
}

// Launch the w-range reduction of visibilities [0, n) into hdr's range keys.
void rick_launch_wrange(const rick_plan *plan, const double *uvw, int64_t n, WsHeader *hdr,
                        cudaStream_t st, int n_chan, const double *scale);


// Fold the key of w into [lo, hi] unless w is not finite.
__device__ __forceinline__ void wrange_fold(double w, uint64_t &lo, uint64_t &hi)
{
    const uint64_t b = rick_dbits(w);
    if (((b >> 52) & 0x7FF) == 0x7FF) return;  // not finite
    const uint64_t k = rick_dkey(w);
    lo = k < lo ? k : lo;
    hi = k > hi ? k : hi;
}

// w range of visibilities [0, n).  Multi-channel input (n_chan > 0): rows of
// n_chan visibilities, w = the row's w times the channel factor.  When every
// factor is positive and finite, rounding is monotone in the factor, so a
// row's extremes are its products with the smallest and the largest factor
// (unless one of those overflows, when every channel is folded).
// MIRROR: the mirrored visibilities' -w are folded in too.
template <bool MIRROR>
__global__ void wrange_kernel(const double *uvw, int64_t n, WsHeader *hdr, int n_chan,
                              const double *scale)
{
    __shared__ double s_min[32], s_max[32];
    __shared__ int s_ok[32];
    uint64_t lo = ~0ull, hi = 0ull;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (n_chan <= 0) {
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
             i += (int64_t)gridDim.x * blockDim.x) {
            const double w = uvw[3 * i + 2];
            wrange_fold(w, lo, hi);
            if (MIRROR) wrange_fold(-w, lo, hi);
        }
    } else {
        // smallest and largest factor, and whether all are positive and finite
        double fmin = INFINITY, fmax = 0.0;
        int ok = 1;
        for (int c = threadIdx.x; c < n_chan; c += blockDim.x) {
            const double f = scale[c];
            ok &= (f > 0.0 && f < INFINITY) ? 1 : 0;
            fmin = fmin < f ? fmin : f;
            fmax = fmax > f ? fmax : f;
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double a = __shfl_xor_sync(FULL, fmin, o), b = __shfl_xor_sync(FULL, fmax, o);
            fmin = fmin < a ? fmin : a;
            fmax = fmax > b ? fmax : b;
            ok &= __shfl_xor_sync(FULL, ok, o);
        }
        if (lane == 0) {
            s_min[wid] = fmin;
            s_max[wid] = fmax;
            s_ok[wid] = ok;
        }
        __syncthreads();
        for (int k = 0; k < nw; ++k) {
            fmin = fmin < s_min[k] ? fmin : s_min[k];
            fmax = fmax > s_max[k] ? fmax : s_max[k];
            ok &= s_ok[k];
        }
        const int64_t n_rows = n / n_chan;  // whole rows (callers pass n = rows * n_chan)
        for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n_rows;
             r += (int64_t)gridDim.x * blockDim.x) {
            const double w0 = uvw[3 * r + 2];
            const double a = w0 * fmin, b = w0 * fmax;
            if (ok && isfinite(a) && isfinite(b)) {
                wrange_fold(a, lo, hi);
                wrange_fold(b, lo, hi);
            } else {
                for (int c = 0; c < n_chan; ++c) wrange_fold(w0 * scale[c], lo, hi);
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        uint64_t l2 = __shfl_xor_sync(FULL, lo, o), h2 = __shfl_xor_sync(FULL, hi, o);
        lo = l2 < lo ? l2 : lo;
        hi = h2 > hi ? h2 : hi;
    }
    if (lane == 0) {
        if (lo != ~0ull) atomicMin(&hdr->wmin_key, (unsigned long long)lo);
        if (hi != 0ull) atomicMax(&hdr->wmax_key, (unsigned long long)hi);
    }
}

void rick_launch_wrange(const rick_plan *plan, const double *uvw, int64_t n, WsHeader *hdr,
                        cudaStream_t st, int n_chan, const double *scale)
{
    wrange_kernel<false><<<plan->num_sms * 4, 256, 0, st>>>(uvw, n, hdr, n_chan, scale);
}

// ------------------------------------------------------------------------
// Pass 2: plane geometry (one thread; n_w <= 1024)

__global__ void bin_setup_kernel(WsHeader *hdr, unsigned long long *bkey, float4 *wplane, int n_w)
{
    double wmin, wmax;
    if (hdr->wmin_key == ~0ull) {  // no finite w at all
        wmin = wmax = 0.0;
    } else {
        wmin = rick_dunkey(hdr->wmin_key);
        wmax = rick_dunkey(hdr->wmax_key);
    }
    double dw = (wmax - wmin) / n_w;
    hdr->dw = dw;
    hdr->stats.w_min = wmin;
    hdr->stats.w_max = wmax;
    for (int j = 1; j < n_w; ++j) bkey[j - 1] = rick_dkey(fma((double)j, dw, wmin));
    for (int k = 0; k < n_w; ++k) {
        double wk = dw == 0.0 ? wmin : fma(k + 0.5, dw, wmin);
        ff s = ff_from_double(wk);
        wplane[k] = make_float4(s.hi, s.lo, (float)wk, 0.0f);
    }
    // one more entry: the plane spacing, for the phase step between planes
    ff d = ff_from_double(dw);
    wplane[n_w] = make_float4(d.hi, d.lo, (float)dw, 0.0f);
}

// ------------------------------------------------------------------------
// Pass 3: keys, histogram, weight-sum partials

struct KeyArgs {
    int64_t n_vis;
    const double *uvw;
    const float *weight;
    int n, n_w, W, log2T, nt;
    double fov, half_n;
    uint64_t key_lo, key_hi;  // rick_dkey(-0.5), rick_dkey(n + 0.5)
    int bulk;                 // uvw (and weight) 16-byte aligned: blocks stage them by bulk copy
    int n_chan;               // > 0: uvw holds rows of n_chan visibilities, scaled per channel
    int n_corr;               // correlations per visibility (weights [n_vis][n_corr])
    const double *chan_scale;
    int64_t n_src;            // inputs; records i >= n_src mirror input i - n_src (n_vis = 2 n_src)
    uint32_t wait_polls;      // limit of the wait for the block's bulk copies
    WsPtrs ws;
};

// Dynamic shared memory of the key pass: the block's uvw and weights, then the
// plane boundary keys.
static inline size_t key_pass_smem(int n_w)
{
    return 28 * (size_t)(RICK_KEY_THREADS * RICK_KEY_ITEMS) + 8 * (size_t)(n_w > 1 ? n_w - 1 : 1);
}

// Lanes that start a run of equal keys (lane 0, or a key unlike the previous
// lane's), as a warp ballot.
__device__ __forceinline__ unsigned run_starts(uint32_t key, int lane)
{
    const uint32_t prev = __shfl_up_sync(FULL, key, 1);
    return __ballot_sync(FULL, lane == 0 || key != prev);
}

// One past the last lane of the run that starts at or before `lane`.
__device__ __forceinline__ int run_end(unsigned starts, int lane)
{
    const unsigned after = lane == 31 ? 0u : starts & (0xFFFFFFFFu << (lane + 1));
    return after ? __ffs(after) - 1 : 32;
}

// First lane of the run that holds `lane`.
__device__ __forceinline__ int run_begin(unsigned starts, int lane)
{
    return 31 - __clz(starts & (0xFFFFFFFFu >> (31 - lane)));
}

__device__ __forceinline__ uint32_t plane_of(uint64_t kw, const unsigned long long *sb, int nb)
{
    int lo = 0, hi = nb;  // number of boundaries <= w
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (sb[mid] <= kw)
            lo = mid + 1;
        else
            hi = mid;
    }
    return (uint32_t)lo;
}

__global__ void __launch_bounds__(RICK_KEY_THREADS) bin_key_kernel(KeyArgs a)
{
    constexpr int NI = RICK_KEY_THREADS * RICK_KEY_ITEMS;
    extern __shared__ __align__(128) unsigned char s_dyn[];
    double *s_uvw = (double *)s_dyn;
    float *s_wt = (float *)(s_dyn + 24 * NI);
    unsigned long long *s_bkey = (unsigned long long *)(s_dyn + 28 * NI);
    __shared__ unsigned long long s_bar;
    __shared__ double s_wsum[RICK_KEY_THREADS / 32];
    __shared__ unsigned long long s_drop[2][RICK_KEY_THREADS / 32];
    const WsHeader *hdr = a.ws.hdr;
    const int64_t blk0 = (int64_t)blockIdx.x * NI;
    const int nitems = (int)(a.n_vis - blk0 < NI ? a.n_vis - blk0 : NI);
    // The block's 1024 uvw rows and weights are contiguous: one bulk copy each
    // (TMA) into shared memory, while the plane keys load; a ragged last block
    // or unaligned inputs take plain loads instead.
    const bool bulk = a.bulk && nitems == NI && blk0 + NI <= a.n_src;
    if (bulk && threadIdx.x == 0) {
        rick_mbar_init(&s_bar, 1);
        rick_mbar_expect_tx(&s_bar, 24 * NI + (a.weight ? 4 * NI : 0));
        rick_bulk_g2s(s_uvw, a.uvw + 3 * blk0, 24 * NI, &s_bar);
        if (a.weight) rick_bulk_g2s(s_wt, a.weight + blk0, 4 * NI, &s_bar);
    }
    int nb = a.n_w - 1;
    for (int j = threadIdx.x; j < nb; j += blockDim.x) s_bkey[j] = a.ws.bkey[j];
    if (!bulk && a.n_chan > 0) {
        // multi-channel input: the uvw of channel c of row r is the row's uvw
        // times the channel factor (one FP64 product per coordinate)
        const int64_t row0 = blk0 / a.n_chan;
        const int ch0 = (int)(blk0 - row0 * a.n_chan);
        for (int i = threadIdx.x; i < nitems; i += blockDim.x) {
            const int t = ch0 + i;
            const int64_t r = row0 + t / a.n_chan;
            const double f = a.chan_scale[t % a.n_chan];
            s_uvw[3 * i] = a.uvw[3 * r] * f;
            s_uvw[3 * i + 1] = a.uvw[3 * r + 1] * f;
            s_uvw[3 * i + 2] = a.uvw[3 * r + 2] * f;
            if (a.weight && a.n_corr == 1) s_wt[i] = a.weight[blk0 + i];
        }
    } else if (!bulk) {
        // records past the inputs mirror input i - n_src: -uvw (its weight)
        for (int i = threadIdx.x; i < nitems; i += blockDim.x) {
            const int64_t r = blk0 + i, src = r < a.n_src ? r : r - a.n_src;
            const double sg = r < a.n_src ? 1.0 : -1.0;
            s_uvw[3 * i] = sg * a.uvw[3 * src];
            s_uvw[3 * i + 1] = sg * a.uvw[3 * src + 1];
            s_uvw[3 * i + 2] = sg * a.uvw[3 * src + 2];
            if (a.weight) s_wt[i] = a.weight[src];
        }
    }
    __syncthreads();
    const bool landed = !bulk || rick_mbar_wait(&s_bar, 0, a.wait_polls);
    if (!__syncthreads_and(landed)) {
        // the copy did not complete in time (never expected): leave this block's
        // inputs out of the binning, flag the fault (reported as n_binned < 0),
        // and let the copy land before the block's shared memory is released
        if (threadIdx.x == 0) {
            atomicExch(&a.ws.hdr->fault, 1u);
            a.ws.wpart[blockIdx.x] = 0.0;
        }
        for (int i = threadIdx.x; i < nitems; i += blockDim.x) a.ws.key[blk0 + i] = 0xFFFFFFFFu;
        rick_mbar_wait(&s_bar, 0, RICK_WAIT_POLLS);  // drain: the copies land before the block ends
        return;
    }
    const bool degenerate = rick_dbits(hdr->dw) == 0;
    const bool given = hdr->range_given;
    const uint64_t wlo = hdr->wmin_key, whi = hdr->wmax_key;
    const int T = 1 << a.log2T, tmask = T - 1;
    int lane = threadIdx.x & 31;

    ff ws = {0.0f, 0.0f};  // this thread's weight sum in double-single arithmetic
    unsigned long long du = 0, dwn = 0;
    int64_t base = blk0 + threadIdx.x;
#pragma unroll 2
    for (int it = 0; it < RICK_KEY_ITEMS; ++it) {
        int64_t i = base + (int64_t)it * RICK_KEY_THREADS;
        uint32_t key = 0xFFFFFFFFu;
        const int li = it * RICK_KEY_THREADS + threadIdx.x;  // index inside the block
        if (i < a.n_vis) {
            double u = s_uvw[3 * li], v = s_uvw[3 * li + 1], w = s_uvw[3 * li + 2];
            int32_t ax, ay;
            float fx, fy;
            bool ok = rick_footprint(fma(u, a.fov, a.half_n), a.n, a.W, a.key_lo, a.key_hi, &ax,
                                     &fx) &&
                      rick_footprint(fma(v, a.fov, a.half_n), a.n, a.W, a.key_lo, a.key_hi, &ay,
                                     &fy);
            if (!ok) {
                ++du;
            } else {
                uint64_t wb = rick_dbits(w);
                uint64_t kw = rick_dkey(w);
                if (((wb >> 52) & 0x7FF) == 0x7FF || (given && (kw < wlo || kw > whi))) {
                    ++dwn;
                } else {
                    uint32_t k = degenerate ? 0u : plane_of(kw, s_bkey, nb);
                    int lx = ax & tmask, ly = ay & tmask;
                    int ex = lx > T - a.W, ey = ly > T - a.W;
                    uint32_t cls = ex ? (ey ? 2u : 1u) : (ey ? 3u : 0u);
                    key = (((k * a.nt + (uint32_t)(ay >> a.log2T)) * a.nt +
                            (uint32_t)(ax >> a.log2T)) << 2) | cls;
                    a.ws.cell[i] = (uint32_t)ax | ((uint32_t)ay << 16);
                    a.ws.frac[i] = make_float2(fx, fy);
                    if (a.n_corr == 1) {
                        float wt = a.weight ? s_wt[li] : 1.0f;
                        ws = ff_add(ws, ff{wt, 0.0f});
                    } else {  // the visibility's weight is the sum of its correlations'
                        for (int c = 0; c < a.n_corr; ++c)
                            ws = ff_add(ws, ff{a.weight ? a.weight[i * a.n_corr + c] : 1.0f,
                                               0.0f});
                    }
                }
            }
            a.ws.key[i] = key;
        }
        // histogram, on this block's sub-counter of the bin: one atomic per run
        // of equal keys in consecutive lanes (consecutive inputs -- the
        // channels of one baseline and time -- mostly share a key).  The
        // counter's old value ranks the run inside the (bin, sub-counter)
        // range, so the scatter needs no atomics of its own.
        const unsigned starts = run_starts(key, lane);
        uint32_t base = 0;
        if (key != 0xFFFFFFFFu && ((starts >> lane) & 1u))
            base = atomicAdd(&a.ws.hist[key * RICK_BIN_SUBS + (blockIdx.x & (RICK_BIN_SUBS - 1))],
                             (uint32_t)(run_end(starts, lane) - lane));
        const int first = run_begin(starts, lane);
        base = __shfl_sync(FULL, base, first);
        if (i < a.n_vis) a.ws.rank[i] = base + (uint32_t)(lane - first);
    }
    // deterministic block reduction of the weight sum (double-single pairs in
    // the warp: GB300 issues FP64 slowly) and of the drop counts
    for (int o = 16; o > 0; o >>= 1) {
        ff other = {__shfl_xor_sync(FULL, ws.hi, o), __shfl_xor_sync(FULL, ws.lo, o)};
        ws = ff_add(ws, other);
        du += __shfl_xor_sync(FULL, du, o);
        dwn += __shfl_xor_sync(FULL, dwn, o);
    }
    int wid = threadIdx.x >> 5;
    if (lane == 0) {
        s_wsum[wid] = (double)ws.hi + (double)ws.lo;
        s_drop[0][wid] = du;
        s_drop[1][wid] = dwn;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        unsigned long long d0 = 0, d1 = 0;
        for (int j = 0; j < RICK_KEY_THREADS / 32; ++j) {
            t += s_wsum[j];
            d0 += s_drop[0][j];
            d1 += s_drop[1][j];
        }
        a.ws.wpart[blockIdx.x] = t;
        if (d0) atomicAdd(&a.ws.hdr->drop_uv, d0);
        if (d1) atomicAdd(&a.ws.hdr->drop_w, d1);
    }
}

// Weight sum over the block partials in a fixed order; stats.
// unit_weights > 0: no weights were given, and each kept visibility weighs
// unit_weights (its number of correlations).
__global__ void __launch_bounds__(1024) bin_finalize_kernel(WsHeader *hdr, const double *wpart,
                                                            int nparts, int unit_weights)
{
    __shared__ double s[1024];
    double t = 0.0;
    for (int i = threadIdx.x; i < nparts; i += 1024) t += wpart[i];
    s[threadIdx.x] = t;
    __syncthreads();
    for (int o = 512; o > 0; o >>= 1) {
        if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        long long binned = (long long)hdr->n_vis - (long long)hdr->drop_uv - (long long)hdr->drop_w;
        if (hdr->fault) binned = -1;  // a bounded wait ran out: the binning is incomplete
        hdr->stats.n_binned = binned;
        hdr->stats.n_dropped_uv = (long long)hdr->drop_uv;
        hdr->stats.n_dropped_w = (long long)hdr->drop_w;
        hdr->stats.sum_weight = unit_weights ? (double)binned * unit_weights : s[0];
    }
}

// ------------------------------------------------------------------------
// Pass 5: scatter records into their bins

// Each thread takes RICK_SCATTER_U inputs per pass (256 apart), so that their
// load chains -- key and rank, then the (bin, sub-counter) offset, then the
// record stores -- overlap (eight chains at two CTAs per SM beat four at four
// CTAs per SM).  Positions come from the ranks the key pass took from the
// histogram counters: no atomics here.
#define RICK_SCATTER_U 8

//
// With CORR, each visibility has n_corr correlations (vis and weight
// [n_vis][n_corr]) and its record carries their weighted sum, sum_c w_c V_c.
// MIRROR: records i >= n_src (the Hermitian mirror) carry conj(V) of input
// i - n_src.
template <bool CORR, bool MIRROR>
__global__ void __launch_bounds__(256) bin_scatter_kernel(int64_t n_vis, const float2 *vis,
                                                          const float *weight, WsPtrs ws,
                                                          int n_corr, int64_t n_src)
{
    constexpr int U = RICK_SCATTER_U;
    const int64_t step = (int64_t)gridDim.x * blockDim.x * U;
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x * U; i0 < n_vis; i0 += step) {
        int64_t idx[U];
        uint32_t key[U], rk[U], cl[U];
        float2 v[U], fr[U];
        float wt[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            idx[u] = i0 + (int64_t)u * blockDim.x + threadIdx.x;
            key[u] = 0xFFFFFFFFu;
            if (idx[u] < n_vis) {
                key[u] = ws.key[idx[u]];
                rk[u] = ws.rank[idx[u]];
                if (CORR) {
                    float2 acc = make_float2(0.0f, 0.0f);
                    for (int c = 0; c < n_corr; ++c) {
                        const float2 vc = vis[idx[u] * n_corr + c];
                        const float wc = weight ? weight[idx[u] * n_corr + c] : 1.0f;
                        acc.x = __fmaf_rn(vc.x, wc, acc.x);
                        acc.y = __fmaf_rn(vc.y, wc, acc.y);
                    }
                    v[u] = acc;
                    wt[u] = 1.0f;
                } else if (MIRROR) {
                    const bool mir = idx[u] >= n_src;
                    const int64_t src = mir ? idx[u] - n_src : idx[u];
                    v[u] = vis[src];
                    if (mir) v[u].y = -v[u].y;
                    wt[u] = weight ? weight[src] : 1.0f;
                } else {
                    v[u] = vis[idx[u]];
                    wt[u] = weight ? weight[idx[u]] : 1.0f;
                }
                fr[u] = ws.frac[idx[u]];
                cl[u] = ws.cell[idx[u]];
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (key[u] != 0xFFFFFFFFu) {
                // the sub-counter of the key pass's block that held this input
                const uint32_t sub = (uint32_t)((idx[u] / (RICK_KEY_THREADS * RICK_KEY_ITEMS)) &
                                                (RICK_BIN_SUBS - 1));
                const uint32_t pos = ws.suboff[key[u] * RICK_BIN_SUBS + sub] + rk[u];
                ws.perm[pos] = (uint32_t)idx[u];
                ws.rec[pos] = make_float4(v[u].x * wt[u], v[u].y * wt[u], fr[u].x, fr[u].y);
                ws.rcell[pos] = cl[u];
            }
        }
    }
}

// Bin offsets from the sub-counter offsets: bin b starts where its first
// sub-range starts.
__global__ void bin_offsets_kernel(const uint32_t *suboff, uint32_t *offsets, int64_t nbins)
{
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b <= nbins;
         b += (int64_t)gridDim.x * blockDim.x)
        offsets[b] = suboff[b * RICK_BIN_SUBS];
}

// Re-pack record values for new visibilities through an existing permutation,
// and sum the new weights: double-single per thread and warp, FP64 per block,
// block partials in wpart (summed in a fixed order by values_finalize_kernel).
// det: also the blocks' sums of |Re| + |Im| of the new values (the bound of the
// deterministic mode's fixed-point scale).
__global__ void __launch_bounds__(256) bin_values_kernel(const float2 *vis, const float *weight,
                                                         WsPtrs ws, int det)
{
    __shared__ double s_part[8];
    __shared__ float s_bound[8];
    float bound = 0.0f;
    const WsHeader *hdr = ws.hdr;
    const int64_t nb = hdr->stats.n_binned;
    ff acc = {0.0f, 0.0f};
    const int64_t n_src = (int64_t)hdr->n_src;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nb;
         r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i0 = ws.perm[r];
        const bool mir = i0 >= n_src;  // the Hermitian mirror: conj V of input i0 - n_src
        const int64_t i = mir ? i0 - n_src : i0;
        float2 v = vis[i];
        if (mir) v.y = -v.y;
        const float wt = weight ? weight[i] : 1.0f;
        float2 *val = (float2 *)&ws.rec[r];  // the value half of the record
        *val = make_float2(v.x * wt, v.y * wt);
        bound += fabsf(v.x * wt) + fabsf(v.y * wt);
        acc = ff_add(acc, ff{wt, 0.0f});
    }
    for (int o = 16; o > 0; o >>= 1) bound += __shfl_xor_sync(FULL, bound, o);
    if ((threadIdx.x & 31) == 0) s_bound[threadIdx.x >> 5] = bound;
    for (int o = 16; o > 0; o >>= 1) {
        const ff other = {__shfl_xor_sync(FULL, acc.hi, o), __shfl_xor_sync(FULL, acc.lo, o)};
        acc = ff_add(acc, other);
    }
    if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = (double)acc.hi + (double)acc.lo;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0, b = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
            t += s_part[k];
            b += s_bound[k];
        }
        ws.wpart[blockIdx.x] = t;
        if (det) ws.vpart[blockIdx.x] = b;
    }
}

__global__ void __launch_bounds__(1024) values_finalize_kernel(const double *wpart, int nparts,
                                                               int unit_weights, WsHeader *hdr)
{
    __shared__ double s[1024];
    double t = 0.0;
    for (int i = threadIdx.x; i < nparts; i += 1024) t += wpart[i];
    s[threadIdx.x] = t;
    __syncthreads();
    for (int o = 512; o > 0; o >>= 1) {
        if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        hdr->stats.sum_weight = unit_weights ? (double)hdr->stats.n_binned : s[0];
}

// ------------------------------------------------------------------------
// Deterministic mode (RICK_OPT_DETERMINISTIC): the ranks the key pass takes
// from atomics order a bin's records by arrival, which differs from run to
// run.  Instead, (key, input index) pairs are sorted by a stable LSD radix
// sort -- RICK_DET_DIGIT-bit digits, least significant first, over blocks of
// RICK_DET_BLOCK records -- so that the records of each bin are in input
// order, and then gathered.  A dropped record's all-ones key sorts after every
// bin in every pass.

// Per block, the count of each digit: cnt[digit * nblk + block] (digit-major,
// so that one exclusive scan gives every (digit, block) its first position).
__global__ void __launch_bounds__(256) det_hist_kernel(const uint32_t *key, int64_t n, int shift,
                                                       uint32_t *cnt, uint32_t nblk)
{
    __shared__ uint32_t h[1 << RICK_DET_DIGIT];
    for (int d = threadIdx.x; d < (1 << RICK_DET_DIGIT); d += blockDim.x) h[d] = 0;
    __syncthreads();
    const int64_t b0 = (int64_t)blockIdx.x * RICK_DET_BLOCK;
    const int lane = threadIdx.x & 31;
    for (int j = threadIdx.x; j < RICK_DET_BLOCK; j += blockDim.x) {
        const int64_t i = b0 + j;
        const uint32_t d = i < n ? (key[i] >> shift) & ((1u << RICK_DET_DIGIT) - 1) : 0xFFFFFFFFu;
        const unsigned peers = __match_any_sync(FULL, d);
        if (d != 0xFFFFFFFFu && (peers & ((1u << lane) - 1u)) == 0u)  // one add per digit
            atomicAdd(&h[d], (uint32_t)__popc(peers));
    }
    __syncthreads();
    for (int d = threadIdx.x; d < (1 << RICK_DET_DIGIT); d += blockDim.x)
        cnt[(size_t)d * nblk + blockIdx.x] = h[d];
}

// One stable pass: the block's records in rounds of 256 consecutive ones; a
// record's place is its (digit, block) start, plus the records of its digit in
// the block's earlier rounds, in earlier warps of its round and in earlier
// lanes of its warp.  idx_in NULL: the identity (the first pass).
__global__ void __launch_bounds__(256) det_scatter_kernel(const uint32_t *key_in,
                                                          const uint32_t *idx_in, int64_t n,
                                                          int shift, const uint32_t *start,
                                                          uint32_t nblk, uint32_t *key_out,
                                                          uint32_t *idx_out)
{
    constexpr int ND = 1 << RICK_DET_DIGIT;
    __shared__ uint32_t run[ND];     // next place of each digit
    __shared__ uint32_t wc[8][ND];   // this round: records of each digit per warp
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    for (int d = t; d < ND; d += 256) {
        run[d] = start[(size_t)d * nblk + blockIdx.x];
        for (int w = 0; w < 8; ++w) wc[w][d] = 0;
    }
    __syncthreads();
    const int64_t b0 = (int64_t)blockIdx.x * RICK_DET_BLOCK;
    for (int r = 0; r < RICK_DET_BLOCK / 256; ++r) {
        const int64_t i = b0 + r * 256 + t;
        const bool live = i < n;
        uint32_t k = 0, idx = 0, d = 0xFFFFFFFFu;
        if (live) {
            k = key_in[i];
            idx = idx_in ? idx_in[i] : (uint32_t)i;
            d = (k >> shift) & (ND - 1);
        }
        const unsigned peers = __match_any_sync(FULL, d);
        const int rank = __popc(peers & ((1u << lane) - 1u));
        if (live && rank == 0) wc[wid][d] = (uint32_t)__popc(peers);
        __syncthreads();
        if (live) {
            uint32_t pos = run[d] + (uint32_t)rank;
            for (int w = 0; w < wid; ++w) pos += wc[w][d];
            key_out[pos] = k;
            idx_out[pos] = idx;
        }
        __syncthreads();
        for (int dd = t; dd < ND; dd += 256) {
            uint32_t tot = 0;
            for (int w = 0; w < 8; ++w) {
                tot += wc[w][dd];
                wc[w][dd] = 0;
            }
            run[dd] += tot;
        }
        __syncthreads();
    }
}

// The records in sorted order: record r is input sidx[r] (records past n_src
// mirror input i - n_src; with CORR the weighted sum of the correlations).
// Each block also sums |Re| + |Im| of its record values (a fixed order: the
// grid-stride split and the reductions depend only on the sizes), the bound
// from which the fixed-point scale of the tile sums is chosen.
template <bool CORR>
__global__ void __launch_bounds__(256) det_records_kernel(const uint32_t *sidx, const float2 *vis,
                                                          const float *weight, WsPtrs ws,
                                                          int n_corr, int64_t n_src)
{
    __shared__ float s_part[8];
    const int64_t nb = ws.hdr->stats.n_binned;
    float bound = 0.0f;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nb;
         r += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t i = sidx[r];
        float2 v;
        if (CORR) {
            v = make_float2(0.0f, 0.0f);
            for (int c = 0; c < n_corr; ++c) {
                const float2 vc = vis[(int64_t)i * n_corr + c];
                const float wc = weight ? weight[(int64_t)i * n_corr + c] : 1.0f;
                v.x = __fmaf_rn(vc.x, wc, v.x);
                v.y = __fmaf_rn(vc.y, wc, v.y);
            }
        } else {
            const bool mir = (int64_t)i >= n_src;
            const int64_t src = mir ? (int64_t)i - n_src : (int64_t)i;
            v = vis[src];
            if (mir) v.y = -v.y;
            const float wt = weight ? weight[src] : 1.0f;
            v = make_float2(v.x * wt, v.y * wt);
        }
        const float2 fr = ws.frac[i];
        ws.perm[r] = i;
        ws.rec[r] = make_float4(v.x, v.y, fr.x, fr.y);
        ws.rcell[r] = ws.cell[i];
        bound += fabsf(v.x) + fabsf(v.y);
    }
    for (int o = 16; o > 0; o >>= 1) bound += __shfl_xor_sync(FULL, bound, o);
    if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = bound;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += s_part[k];
        ws.vpart[blockIdx.x] = t;
    }
}

// The fixed-point scale: 2^k with the sum of all |values| (each kernel weight
// is at most about 1, so every tile sum is bounded by it) below 2^60, so that
// 64-bit sums cannot overflow.
__global__ void det_scale_kernel(WsHeader *hdr, const double *vpart, int nparts)
{
    double b = 0.0;
    for (int i = 0; i < nparts; ++i) b += vpart[i];
    int e = 0;
    frexp(b * 1.01 + 1e-30, &e);  // b * 1.01 < 2^e
    int k = 60 - e;
    k = k > 100 ? 100 : (k < -100 ? -100 : k);
    hdr->fx_scale = ldexpf(1.0f, k);
    hdr->fx_inv = ldexpf(1.0f, -k);
}

// Slots of the tiles gridded by several work items (deterministic mode): a
// flag per tile, then its exclusive scan is the tile's slot.
__global__ void det_mc_flags_kernel(const uint32_t *gbase, uint32_t *slot, uint32_t ntiles)
{
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < ntiles) slot[t] = gbase[t + 1] - gbase[t] > 1 ? 1u : 0u;
    if (t == ntiles) slot[t] = 0u;
}

__global__ void det_mc_count_kernel(WsHeader *hdr, const uint32_t *slot, uint32_t ntiles)
{
    hdr->mc_count = slot[ntiles];
}

// Enqueue the deterministic ordering and the records.  Keys of n records are
// in w.key (input order); nbins bins.
static rick_status det_sort_records(rick_plan *plan, WsPtrs w, const WsLayout &L, int64_t n,
                                    const void *vis, const float *weight, int n_corr,
                                    int64_t n_src, cudaStream_t st)
{
    const uint32_t nblk = (uint32_t)((n + RICK_DET_BLOCK - 1) / RICK_DET_BLOCK);
    int passes = 1;
    while (passes * RICK_DET_DIGIT < 32 && ((int64_t)1 << (passes * RICK_DET_DIGIT)) <= L.nbins)
        ++passes;
    // ping-pong between two (key, index) buffers; the input-order keys in
    // w.key stay (degridding and the density weights read them)
    const uint32_t *kin = w.key, *iin = NULL;
    uint32_t *kbuf[2] = {w.dkey, w.dkey2}, *ibuf[2] = {w.didx, w.rank};
    if (n > 0) {
        for (int ps = 0; ps < passes; ++ps) {
            const int shift = ps * RICK_DET_DIGIT;
            det_hist_kernel<<<nblk, 256, 0, st>>>(kin, n, shift, w.dcnt, nblk);
            RICK_LAUNCH_CHECK(plan);
            RICK_CUDA_TRY(plan, scan_u32(w.dcnt, w.dcnt, (int64_t)nblk << RICK_DET_DIGIT, w.scan,
                                         st, &plan->launches));
            uint32_t *ko = kbuf[ps & 1], *io = ibuf[ps & 1];
            det_scatter_kernel<<<nblk, 256, 0, st>>>(kin, iin, n, shift, w.dcnt, nblk, ko, io);
            RICK_LAUNCH_CHECK(plan);
            kin = ko;
            iin = io;
        }
    }
    int blocks = plan->num_sms * 8;
    if (blocks > (int)L.ndetblocks + 1) blocks = (int)L.ndetblocks + 1;
    if (n > 0) {
        if (n_corr > 1)
            det_records_kernel<true><<<blocks, 256, 0, st>>>(iin, (const float2 *)vis, weight, w,
                                                             n_corr, n);
        else
            det_records_kernel<false><<<blocks, 256, 0, st>>>(iin, (const float2 *)vis, weight,
                                                              w, 1, n_src);
        RICK_LAUNCH_CHECK(plan);
    }
    det_scale_kernel<<<1, 1, 0, st>>>(w.hdr, w.vpart, n > 0 ? blocks : 0);
    RICK_LAUNCH_CHECK(plan);
    return RICK_OK;
}

// ------------------------------------------------------------------------
// Pass 6: work lists.  The grid work of tile t covers its own bin (all four
// edge classes) plus the records of the west, north and north-west tiles
// whose footprints reach into t; degridding needs only the own bin.

__global__ void tile_count_kernel(const uint32_t *off, uint32_t *gcnt, uint32_t *dcnt,
                                  uint32_t ntiles, int nt, uint32_t cap)
{
    uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t > ntiles) return;
    if (t == ntiles) {
        gcnt[t] = 0;
        dcnt[t] = 0;
        return;
    }
    uint32_t tx = t % nt, ty = (t / nt) % nt;
    uint32_t own = off[4 * t + 4] - off[4 * t];
    uint32_t L = own;
    if (tx > 0) L += off[4 * (t - 1) + 3] - off[4 * (t - 1) + 1];
    if (ty > 0) L += off[4 * (t - nt) + 4] - off[4 * (t - nt) + 2];
    if (tx > 0 && ty > 0) L += off[4 * (t - nt - 1) + 3] - off[4 * (t - nt - 1) + 2];
    gcnt[t] = (L + cap - 1) / cap;  // tiles without records: no work item
    dcnt[t] = (own + cap - 1) / cap;
}

// ------------------------------------------------------------------------

// Rows of n_chan channels that fit a plan's capacity.
static int64_t plan_max_rows(const rick_plan *plan, int32_t n_chan)
{
    return plan && n_chan > 0 ? plan->max_vis / n_chan : 0;
}

rick_status rick_bin_impl(rick_plan *plan, int64_t n_vis, const double *uvw, const void *vis,
                          const float *weight, void *ws_dev, size_t ws_bytes,
                          rick_bin_stats *stats_dev, void *stream, const WsHeader *range_src,
                          int n_chan, const double *chan_scale, int n_corr)
{
    if (!plan || !ws_dev || n_vis < 0 || n_corr < 1 || n_corr > RICK_MAX_CORR) return RICK_EINVAL;
    if (plan->sticky != RICK_OK) return plan->sticky;
    if (n_vis > 0 && (!uvw || !vis)) return RICK_EINVAL;
    if (((uintptr_t)ws_dev & 255) || ((uintptr_t)uvw & 7) || ((uintptr_t)vis & 7) ||
        ((uintptr_t)weight & 3) || ((uintptr_t)stats_dev & 7) || ((uintptr_t)chan_scale & 7))
        return RICK_EINVAL;
    if (n_chan < 0 || (n_chan > 0 && n_vis > 0 && !chan_scale)) return RICK_EINVAL;
    if (n_vis > plan->max_vis) return RICK_ERANGE;
    const rick_params &p = plan->p;
    // the Hermitian mirror: input-order records, then the mirrored ones (per-
    // visibility input only: not with channels, correlations or streaming)
    const int mirror = (p.options & RICK_OPT_HERMITIAN_MIRROR) != 0;
    if (mirror && (n_chan > 0 || n_corr != 1 || range_src)) return RICK_EINVAL;
    const int64_t n_src = n_vis;
    n_vis = rick_n_records(&p, n_src);  // records from here on
    WsLayout L = rick_ws_layout(&p, plan->max_vis);
    if (ws_bytes < L.total) return RICK_ERANGE;
    const int64_t nkb = (n_vis + RICK_KEY_THREADS * RICK_KEY_ITEMS - 1) /
                        (RICK_KEY_THREADS * RICK_KEY_ITEMS);
    WsPtrs w = rick_ws_ptrs(ws_dev, L);
    cudaStream_t st = (cudaStream_t)stream;
    const bool det = (p.options & RICK_OPT_DETERMINISTIC) != 0;
    uint32_t cap = rick_chunk_cap(n_vis, plan->num_sms);
    if (det) {
        // enough records per work item that the tiles with several items fit
        // the workspace's slots (a record is visited by at most four tiles)
        const int64_t slots = rick_det_slots(&p, rick_n_records(&p, plan->max_vis));
        int64_t c = (4 * n_vis + slots - 1) / slots;
        c = (c + 255) & ~(int64_t)255;
        if (c > cap) cap = (uint32_t)c;
    }
    int given = !isnan(p.w_min) || range_src != NULL;

    bin_init_kernel<<<1, 1, 0, st>>>(w.hdr, (uint64_t)n_vis, cap, given,
                                     isnan(p.w_min) ? 0 : rick_dkey(p.w_min),
                                     isnan(p.w_min) ? 0 : rick_dkey(p.w_max), (uint32_t)nkb,
                                     range_src, (uint64_t)n_src, mirror);
    RICK_LAUNCH_CHECK(plan);
    if (!given && n_vis > 0) {
        int blocks = plan->num_sms * 4;
        if (mirror)
            wrange_kernel<true><<<blocks, 256, 0, st>>>(uvw, n_src, w.hdr, n_chan, chan_scale);
        else
            wrange_kernel<false><<<blocks, 256, 0, st>>>(uvw, n_src, w.hdr, n_chan, chan_scale);
        RICK_LAUNCH_CHECK(plan);
    }
    bin_setup_kernel<<<1, 1, 0, st>>>(w.hdr, w.bkey, w.wplane, p.n_w);
    RICK_LAUNCH_CHECK(plan);
    RICK_CUDA_TRY(plan, cudaMemsetAsync(w.hist, 0, 4 * (size_t)(RICK_BIN_SUBS * L.nbins + 1), st));

    if (n_vis > 0) {
        KeyArgs ka;
        ka.n_vis = n_vis;
        ka.uvw = uvw;
        ka.weight = weight;
        ka.n = p.n;
        ka.n_w = p.n_w;
        ka.W = p.support;
        ka.log2T = 0;
        while ((1 << ka.log2T) < p.tile) ++ka.log2T;
        ka.nt = p.n / p.tile;
        ka.fov = p.fov;
        ka.half_n = 0.5 * p.n;
        ka.key_lo = rick_dkey(-0.5);
        ka.key_hi = rick_dkey((double)p.n + 0.5);
        ka.ws = w;
        ka.n_chan = n_chan;
        ka.n_corr = n_corr;
        ka.chan_scale = chan_scale;
        ka.n_src = mirror ? n_src : n_vis;
        ka.wait_polls = plan->wait_polls;
        ka.bulk = n_chan == 0 && n_corr == 1 && ((uintptr_t)uvw & 15) == 0 &&
                  ((uintptr_t)weight & 15) == 0;
        const size_t smem = key_pass_smem(p.n_w);
        RICK_CUDA_TRY(plan, cudaFuncSetAttribute(bin_key_kernel,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)smem));
        bin_key_kernel<<<(unsigned)nkb, RICK_KEY_THREADS, smem, st>>>(ka);
        RICK_LAUNCH_CHECK(plan);
    }
    bin_finalize_kernel<<<1, 1024, 0, st>>>(w.hdr, w.wpart, (int)nkb, weight == NULL ? n_corr : 0);
    RICK_LAUNCH_CHECK(plan);
    RICK_CUDA_TRY(plan, scan_u32(w.hist, w.suboff, RICK_BIN_SUBS * L.nbins + 1, w.scan, st,
                                 &plan->launches));
    bin_offsets_kernel<<<(unsigned)((L.nbins + 256) / 256), 256, 0, st>>>(w.suboff, w.offsets,
                                                                          L.nbins);
    RICK_LAUNCH_CHECK(plan);
    if (det) {
        rick_status ds = det_sort_records(plan, w, L, n_vis, vis, weight, n_corr,
                                          mirror ? n_src : n_vis, st);
        if (ds != RICK_OK) return ds;
    } else if (n_vis > 0) {
        int64_t blocks = (n_vis + 256 * RICK_SCATTER_U - 1) / (256 * RICK_SCATTER_U);
        if (blocks > (int64_t)plan->num_sms * 64) blocks = (int64_t)plan->num_sms * 64;
        if (n_corr > 1)
            bin_scatter_kernel<true, false><<<(unsigned)blocks, 256, 0, st>>>(
                n_vis, (const float2 *)vis, weight, w, n_corr, n_vis);
        else if (mirror)
            bin_scatter_kernel<false, true><<<(unsigned)blocks, 256, 0, st>>>(
                n_vis, (const float2 *)vis, weight, w, 1, n_src);
        else
            bin_scatter_kernel<false, false><<<(unsigned)blocks, 256, 0, st>>>(
                n_vis, (const float2 *)vis, weight, w, 1, n_vis);
        RICK_LAUNCH_CHECK(plan);
    }
    uint32_t nt = (uint32_t)L.ntiles;
    tile_count_kernel<<<(nt + 256) / 256, 256, 0, st>>>(w.offsets, w.gbase, w.dbase, nt,
                                                        p.n / p.tile, cap);
    RICK_LAUNCH_CHECK(plan);
    RICK_CUDA_TRY(plan, scan_u32(w.gbase, w.gbase, L.ntiles + 1, w.scan, st, &plan->launches));
    RICK_CUDA_TRY(plan, scan_u32(w.dbase, w.dbase, L.ntiles + 1, w.scan, st, &plan->launches));
    if (det) {  // slots of the tiles with several grid work items
        det_mc_flags_kernel<<<(nt + 256) / 256, 256, 0, st>>>(w.gbase, w.mcslot, nt);
        RICK_LAUNCH_CHECK(plan);
        RICK_CUDA_TRY(plan, scan_u32(w.mcslot, w.mcslot, L.ntiles + 1, w.scan, st,
                                     &plan->launches));
        det_mc_count_kernel<<<1, 1, 0, st>>>(w.hdr, w.mcslot, nt);
        RICK_LAUNCH_CHECK(plan);
    }
    if (stats_dev)
        RICK_CUDA_TRY(plan, cudaMemcpyAsync(stats_dev, &w.hdr->stats, sizeof(rick_bin_stats),
                                            cudaMemcpyDeviceToDevice, st));
    return RICK_OK;
}

extern "C" rick_status rick_bin(rick_plan *plan, int64_t n_vis, const double *uvw,
                                const void *vis, const float *weight, void *ws_dev,
                                size_t ws_bytes, rick_bin_stats *stats_dev, void *stream)
{
    return rick_bin_impl(plan, n_vis, uvw, vis, weight, ws_dev, ws_bytes, stats_dev, stream, NULL,
                         0, NULL, 1);
}

extern "C" rick_status rick_bin_channels(rick_plan *plan, int64_t n_rows, int32_t n_chan,
                                         const double *uvw_rows, const double *chan_scale,
                                         const void *vis, const float *weight, void *ws_dev,
                                         size_t ws_bytes, rick_bin_stats *stats_dev, void *stream)
{
    if (!plan || n_rows < 0 || n_chan < 1) return RICK_EINVAL;
    if (n_rows > 0 && !chan_scale) return RICK_EINVAL;
    if (n_rows > plan_max_rows(plan, n_chan)) return RICK_ERANGE;
    return rick_bin_impl(plan, n_rows * n_chan, uvw_rows, vis, weight, ws_dev, ws_bytes, stats_dev,
                         stream, NULL, n_chan, chan_scale, 1);
}

extern "C" rick_status rick_bin_rows(rick_plan *plan, int64_t n_rows, int32_t n_chan,
                                     int32_t n_corr, const double *uvw_rows,
                                     const double *chan_scale, const void *vis,
                                     const float *weight, void *ws_dev, size_t ws_bytes,
                                     rick_bin_stats *stats_dev, void *stream)
{
    if (!plan || n_rows < 0 || n_chan < 1 || n_corr < 1 || n_corr > RICK_MAX_CORR)
        return RICK_EINVAL;
    if (n_rows > 0 && !chan_scale) return RICK_EINVAL;
    if (n_rows > plan_max_rows(plan, n_chan)) return RICK_ERANGE;
    return rick_bin_impl(plan, n_rows * n_chan, uvw_rows, vis, weight, ws_dev, ws_bytes, stats_dev,
                         stream, NULL, n_chan, chan_scale, n_corr);
}

extern "C" rick_status rick_bin_values(rick_plan *plan, const void *vis, const float *weight,
                                       void *ws_dev, rick_bin_stats *stats_dev, void *stream)
{
    if (!plan || !vis || !ws_dev) return RICK_EINVAL;
    if (plan->sticky != RICK_OK) return plan->sticky;
    if (((uintptr_t)ws_dev & 255) || ((uintptr_t)vis & 7) || ((uintptr_t)weight & 3) ||
        ((uintptr_t)stats_dev & 7))
        return RICK_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const WsLayout L = rick_ws_layout(&plan->p, plan->max_vis);
    WsPtrs w = rick_ws_ptrs(ws_dev, L);
    // one weight partial per block: the workspace holds nkeyblocks + 1 of them
    // (and ndetblocks + 1 bound partials in deterministic mode)
    const int det = (plan->p.options & RICK_OPT_DETERMINISTIC) != 0;
    int blocks = plan->num_sms * 8;
    if (blocks > (int)L.nkeyblocks + 1) blocks = (int)L.nkeyblocks + 1;
    if (det && blocks > (int)L.ndetblocks + 1) blocks = (int)L.ndetblocks + 1;
    bin_values_kernel<<<blocks, 256, 0, st>>>((const float2 *)vis, weight, w, det);
    RICK_LAUNCH_CHECK(plan);
    values_finalize_kernel<<<1, 1024, 0, st>>>(w.wpart, blocks, weight == NULL, w.hdr);
    RICK_LAUNCH_CHECK(plan);
    if (det) {  // the fixed-point scale for the new values
        det_scale_kernel<<<1, 1, 0, st>>>(w.hdr, w.vpart, blocks);
        RICK_LAUNCH_CHECK(plan);
    }
    if (stats_dev)
        RICK_CUDA_TRY(plan, cudaMemcpyAsync(stats_dev, &w.hdr->stats, sizeof(rick_bin_stats),
                                            cudaMemcpyDeviceToDevice, st));
    return RICK_OK;
}

// ------------------------------------------------------------------------
// rick_bin_noalloc: the binning above for callers that must not allocate
// device memory.  Its temporaries -- the per-visibility ranks and fractional
// offsets, the histogram / cursor array, the scan temporaries and the
// weight-sum partials -- live in this file-scope array instead of the
// caller's workspace.  The per-visibility keys and corner cells stay in the
// caller's workspace, where rick_bin writes them: degridding and the density
// weights read them after the binning.  The array is part of the library
// image: every GPU that loads librick.so holds it (about 11.6 MB) until the
// process exits.

#define NOALLOC_MAX_VIS (1 << 18)
#define NOALLOC_MAX_BINS (1 << 17)
#define NOALLOC_FRAC (0)
#define NOALLOC_RANK (NOALLOC_FRAC + 8 * NOALLOC_MAX_VIS)
#define NOALLOC_HIST (NOALLOC_RANK + 4 * NOALLOC_MAX_VIS)
#define NOALLOC_SUBOFF (NOALLOC_HIST + 4 * (RICK_BIN_SUBS * NOALLOC_MAX_BINS + 256))
#define NOALLOC_SCAN (NOALLOC_SUBOFF + 4 * (RICK_BIN_SUBS * NOALLOC_MAX_BINS + 256))
#define NOALLOC_WPART (NOALLOC_SCAN + 4 * 4096)
#define NOALLOC_BYTES (NOALLOC_WPART + 8 * (NOALLOC_MAX_VIS / (RICK_KEY_THREADS * RICK_KEY_ITEMS) + 256))

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

// The array's device address, looked up once per device with that device
// current (a host-side name of a __device__ array is not a device address).
#define NOALLOC_MAX_DEVICES 64
static void *g_noalloc_addr[NOALLOC_MAX_DEVICES];
static std::mutex g_noalloc_mu;

static rick_status noalloc_scratch(unsigned char **out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NOALLOC_MAX_DEVICES)
        return RICK_ECUDA;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void *ptr = NULL;
        if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return RICK_ECUDA;
        g_noalloc_addr[dev] = ptr;
    }
    *out = (unsigned char *)g_noalloc_addr[dev];
    return RICK_OK;
}

extern "C" rick_status rick_bin_noalloc(rick_plan *plan, int64_t n_vis, const double *uvw,
                                        const void *vis, const float *weight, void *ws_dev,
                                        size_t ws_bytes, rick_bin_stats *stats_dev, void *stream)
{
    if (!plan || !ws_dev || n_vis < 0) return RICK_EINVAL;
    if (plan->sticky != RICK_OK) return plan->sticky;
    if (n_vis > 0 && (!uvw || !vis)) return RICK_EINVAL;
    if (((uintptr_t)ws_dev & 255) || ((uintptr_t)uvw & 7) || ((uintptr_t)vis & 7) ||
        ((uintptr_t)weight & 3) || ((uintptr_t)stats_dev & 7))
        return RICK_EINVAL;
    if (n_vis > plan->max_vis) return RICK_ERANGE;
    const rick_params &p = plan->p;
    if (p.options != 0) return RICK_EINVAL;  // plain binning only
    WsLayout L = rick_ws_layout(&p, plan->max_vis);
    if (ws_bytes < L.total) return RICK_ERANGE;
    // the fixed scratch bounds the problem size
    if (n_vis > NOALLOC_MAX_VIS || L.nbins > NOALLOC_MAX_BINS) return RICK_ERANGE;
    unsigned char *scratch = NULL;
    rick_status sst = noalloc_scratch(&scratch);
    if (sst != RICK_OK) {
        plan->sticky = sst;
        return sst;
    }
    const int64_t nkb = (n_vis + RICK_KEY_THREADS * RICK_KEY_ITEMS - 1) /
                        (RICK_KEY_THREADS * RICK_KEY_ITEMS);
    // outputs (records, offsets, work lists, and the keys and corner cells that
    // later calls read) in the caller's workspace, temporaries in the fixed array
    WsPtrs w = rick_ws_ptrs(ws_dev, L);
    w.rank = (uint32_t *)(scratch + NOALLOC_RANK);
    w.frac = (float2 *)(scratch + NOALLOC_FRAC);
    w.hist = (uint32_t *)(scratch + NOALLOC_HIST);
    w.suboff = (uint32_t *)(scratch + NOALLOC_SUBOFF);
    w.scan = (uint32_t *)(scratch + NOALLOC_SCAN);
    w.wpart = (double *)(scratch + NOALLOC_WPART);
    cudaStream_t st = (cudaStream_t)stream;
    uint32_t cap = rick_chunk_cap(n_vis, plan->num_sms);
    int given = !isnan(p.w_min);

    // the same stages as rick_bin, in the same order
    bin_init_kernel<<<1, 1, 0, st>>>(w.hdr, (uint64_t)n_vis, cap, given,
                                     given ? rick_dkey(p.w_min) : 0, given ? rick_dkey(p.w_max) : 0,
                                     (uint32_t)nkb, NULL, (uint64_t)n_vis, 0);
    RICK_LAUNCH_CHECK(plan);
    if (!given && n_vis > 0) {
        wrange_kernel<false><<<plan->num_sms * 4, 256, 0, st>>>(uvw, n_vis, w.hdr, 0, NULL);
        RICK_LAUNCH_CHECK(plan);
    }
    bin_setup_kernel<<<1, 1, 0, st>>>(w.hdr, w.bkey, w.wplane, p.n_w);
    RICK_LAUNCH_CHECK(plan);
    // the array keeps the last call's contents: the histogram must start at zero
    RICK_CUDA_TRY(plan, cudaMemsetAsync(w.hist, 0, 4 * (size_t)(RICK_BIN_SUBS * L.nbins + 1), st));
    if (n_vis > 0) {
        KeyArgs ka;
        ka.n_vis = n_vis;
        ka.uvw = uvw;
        ka.weight = weight;
        ka.n = p.n;
        ka.n_w = p.n_w;
        ka.W = p.support;
        ka.log2T = 0;
        while ((1 << ka.log2T) < p.tile) ++ka.log2T;
        ka.nt = p.n / p.tile;
        ka.fov = p.fov;
        ka.half_n = 0.5 * p.n;
        ka.key_lo = rick_dkey(-0.5);
        ka.key_hi = rick_dkey((double)p.n + 0.5);
        ka.ws = w;
        ka.n_chan = 0;
        ka.n_corr = 1;
        ka.chan_scale = NULL;
        ka.n_src = n_vis;
        ka.wait_polls = plan->wait_polls;
        ka.bulk = ((uintptr_t)uvw & 15) == 0 && ((uintptr_t)weight & 15) == 0;
        const size_t smem = key_pass_smem(p.n_w);
        RICK_CUDA_TRY(plan, cudaFuncSetAttribute(bin_key_kernel,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)smem));
        bin_key_kernel<<<(unsigned)nkb, RICK_KEY_THREADS, smem, st>>>(ka);
        RICK_LAUNCH_CHECK(plan);
    }
    bin_finalize_kernel<<<1, 1024, 0, st>>>(w.hdr, w.wpart, (int)nkb, weight == NULL);
    RICK_LAUNCH_CHECK(plan);
    RICK_CUDA_TRY(plan, scan_u32(w.hist, w.suboff, RICK_BIN_SUBS * L.nbins + 1, w.scan, st,
                                 &plan->launches));
    bin_offsets_kernel<<<(unsigned)((L.nbins + 256) / 256), 256, 0, st>>>(w.suboff, w.offsets,
                                                                          L.nbins);
    RICK_LAUNCH_CHECK(plan);
    if (n_vis > 0) {
        int64_t blocks = (n_vis + 256 * RICK_SCATTER_U - 1) / (256 * RICK_SCATTER_U);
        if (blocks > (int64_t)plan->num_sms * 64) blocks = (int64_t)plan->num_sms * 64;
        bin_scatter_kernel<false, false><<<(unsigned)blocks, 256, 0, st>>>(
            n_vis, (const float2 *)vis, weight, w, 1, n_vis);
        RICK_LAUNCH_CHECK(plan);
    }
    uint32_t nt = (uint32_t)L.ntiles;
    tile_count_kernel<<<(nt + 256) / 256, 256, 0, st>>>(w.offsets, w.gbase, w.dbase, nt,
                                                        p.n / p.tile, cap);
    RICK_LAUNCH_CHECK(plan);
    RICK_CUDA_TRY(plan, scan_u32(w.gbase, w.gbase, L.ntiles + 1, w.scan, st, &plan->launches));
    RICK_CUDA_TRY(plan, scan_u32(w.dbase, w.dbase, L.ntiles + 1, w.scan, st, &plan->launches));
    if (stats_dev)
        RICK_CUDA_TRY(plan, cudaMemcpyAsync(stats_dev, &w.hdr->stats, sizeof(rick_bin_stats),
                                            cudaMemcpyDeviceToDevice, st));
    return RICK_OK;
}

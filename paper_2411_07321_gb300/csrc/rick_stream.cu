// rick_stream.cu -- imaging a visibility set that sits in host memory,
// streamed through the GPU in chunks (§4 reads the visibilities in
// sequential chunks; §3.2 counts the offload to the GPU as part of gridding).
//
// The set is cut into chunks of at most the plan's max_vis visibilities.  A
// copy stream of the plan moves the next chunks into a ring of
// RICK_STREAM_BUFS staging buffers while the caller's stream bins chunk c and
// grids it into the planes (gridding is linear in the records, so the sum over
// chunks is the gridding of the whole set).  Where the fused transform
// (rick_fft.cu) covers n, a chunk writes only the tiles its records reach,
// overwriting those no earlier chunk reached and adding into the others (the
// tile flags the fused transform keeps say which), and the fused transform then
// reads the tiles the records of any chunk reach: no plane cell is cleared.
// Otherwise the first chunk uses rick_grid (every plane cell written) and the
// later ones rick_grid_accumulate, then cuFFT in place and the plane-sum
// kernel.  Gridded weight sums and drop counts are added up over the chunks in
// chunk order, so the normalisation is that of the whole set.
//
// The w-planes must be the same for every chunk.  With a given w range (the
// plan's) every chunk uses it.  Without one, the range of the whole set is
// needed before the first chunk is binned: uvw is then copied first, in
// chunks, into a device-resident array, each chunk's w range folded in as it
// lands, and only the visibilities and weights go through the staging
// buffers.  Every chunk is binned with that exact range as a given range,
// which drops nothing that the range-from-data binning keeps.  Calls
// alternate between two such areas, so the uvw of the next call can land
// while this call's chunks are still being binned.
//
// Calls of one plan that pass the same staging area overlap: the copy stream
// waits only for the binnings that read a buffer before refilling it, so a
// call's copies run under the previous call's gridding, FFT and w-correction.
// The ring continues across calls (a call's first chunk takes the buffer after
// the previous call's last), so every buffer is refilled only after the
// binning RICK_STREAM_BUFS chunks earlier.
#include <math.h>

#include "rick_common.cuh"

// Channels of multi-channel input the streamed call accepts (their factors
// are staged in the staging area).
#define RICK_STREAM_MAX_CHAN 4096

struct StageLayout {
    size_t range, total, scale, vis, weight, fwork, fwork_bytes, uvw, bytes;
    size_t uvw_buf, vis_buf, weight_buf;  // bytes of one staging buffer / resident area
    int64_t chunk;
    int resident_uvw;
};

// The staging area: the range header and stats totals, RICK_STREAM_BUFS chunk
// buffers of vis and of weight, the fused transform's work buffer (for the n
// it covers), then either RICK_STREAM_BUFS chunk buffers of uvw (given w range)
// or two resident uvw areas (range from the data), used by alternate calls.
// The resident area size is fixed by stage_bytes (0: the size that holds
// n_vis), so that calls with the same staging area agree on its layout.
static StageLayout stage_layout(const rick_params *p, int64_t max_vis, int64_t n_vis,
                                size_t stage_bytes)
{
    StageLayout S;
    S.chunk = max_vis > 0 ? max_vis : 1;
    S.resident_uvw = isnan(p->w_min) ? 1 : 0;
    S.vis_buf = rick_align256(8 * (size_t)S.chunk);
    S.weight_buf = rick_align256(4 * (size_t)S.chunk);
    size_t o = 0;
    S.range = o;  o += rick_align256(sizeof(WsHeader));
    S.total = o;  o += rick_align256(sizeof(rick_bin_stats));
    S.scale = o;  o += 2 * 8 * (size_t)RICK_STREAM_MAX_CHAN;  // channel factors, per area
    S.vis = o;    o += RICK_STREAM_BUFS * S.vis_buf;
    S.weight = o; o += RICK_STREAM_BUFS * S.weight_buf;
    S.fwork_bytes = rick_fft_work_bytes(p);
    S.fwork = o;  o += rick_align256(S.fwork_bytes);
    S.uvw = o;
    if (!S.resident_uvw) {
        S.uvw_buf = rick_align256(24 * (size_t)S.chunk);
    } else if (stage_bytes == 0) {
        S.uvw_buf = rick_align256(24 * (size_t)(n_vis > 0 ? n_vis : 1));
    } else {
        S.uvw_buf = stage_bytes > o ? (stage_bytes - o) / 2 / 256 * 256 : 0;
    }
    S.bytes = o + (S.resident_uvw ? 2 : RICK_STREAM_BUFS) * S.uvw_buf;
    return S;
}

__global__ void range_init_kernel(WsHeader *rh)
{
    rh->wmin_key = ~0ull;
    rh->wmax_key = 0ull;
}

// Running totals of the chunk binnings (first: start them).
__global__ void stats_add_kernel(const WsHeader *hdr, rick_bin_stats *tot, int first)
{
    const rick_bin_stats &s = hdr->stats;
    if (first) {
        *tot = s;
        return;
    }
    tot->n_binned += s.n_binned;
    tot->n_dropped_uv += s.n_dropped_uv;
    tot->n_dropped_w += s.n_dropped_w;
    tot->sum_weight += s.sum_weight;
    tot->w_min = s.w_min;
    tot->w_max = s.w_max;
}

// The whole set's stats into the workspace header (read by the w-correction
// for the weight sum) and to the caller.
__global__ void stats_finish_kernel(WsHeader *hdr, const rick_bin_stats *tot, rick_bin_stats *out)
{
    hdr->stats = *tot;
    if (out) *out = *tot;
}

extern "C" rick_status rick_stream_bytes(const rick_params *params, int64_t max_vis,
                                         int64_t n_vis, size_t *bytes)
{
    if (!params || !bytes || max_vis < 0 || n_vis < 0) return RICK_EINVAL;
    *bytes = stage_layout(params, max_vis, n_vis, 0).bytes;
    return RICK_OK;
}

static rick_status stream_resources(rick_plan *plan)
{
    if (plan->copy) return RICK_OK;
    cudaEvent_t *evs[4] = {&plan->ev_start, &plan->ev_uvw, &plan->ev_area_free[0],
                           &plan->ev_area_free[1]};
    for (cudaEvent_t *e : evs)
        RICK_CUDA_TRY(plan, cudaEventCreateWithFlags(e, cudaEventDisableTiming));
    for (int b = 0; b < RICK_STREAM_BUFS; ++b) {
        RICK_CUDA_TRY(plan, cudaEventCreateWithFlags(&plan->ev_ready[b], cudaEventDisableTiming));
        RICK_CUDA_TRY(plan, cudaEventCreateWithFlags(&plan->ev_free[b], cudaEventDisableTiming));
    }
    RICK_CUDA_TRY(plan, cudaStreamCreateWithFlags(&plan->copy, cudaStreamNonBlocking));
    return RICK_OK;
}

#define RICK_TRY(expr)                      \
    do {                                    \
        rick_status s_ = (expr);            \
        if (s_ != RICK_OK) return s_;       \
    } while (0)

// The streamed path over "units": visibilities (n_chan == 0) or rows of n_chan
// visibilities whose uvw is the row's times a per-channel factor, each
// visibility with n_corr correlations (values and weights [unit][chan][corr]).
// A chunk holds at most max_vis values, so with several correlations it holds
// max_vis / n_corr visibilities: the staging buffers keep their size.
static rick_status stream_impl(rick_plan *plan, int64_t n_units, int32_t n_chan, int32_t n_corr,
                               const double *uvw_host, const double *scale_host,
                               const void *vis_host, const float *weight_host, void *ws_dev,
                               size_t ws_bytes, void *stage_dev, size_t stage_bytes,
                               void *planes_dev, float *image_dev, uint32_t flags,
                               rick_bin_stats *stats_dev, void *stream)
{
    if (!plan || !ws_dev || !stage_dev || !planes_dev || !image_dev || n_units < 0)
        return RICK_EINVAL;
    if (plan->sticky != RICK_OK) return plan->sticky;
    if (n_chan < 0 || n_chan > RICK_STREAM_MAX_CHAN) return n_chan < 0 ? RICK_EINVAL : RICK_ERANGE;
    if (plan->p.options & RICK_OPT_HERMITIAN_MIRROR) return RICK_EINVAL;  // resident binning only
    if (n_corr < 1 || n_corr > RICK_MAX_CORR || (n_corr > 1 && n_chan < 1)) return RICK_EINVAL;
    if (n_units > 0 && (!uvw_host || !vis_host || (n_chan > 0 && !scale_host)))
        return RICK_EINVAL;
    if (((uintptr_t)stage_dev & 255) || ((uintptr_t)ws_dev & 255) ||
        ((uintptr_t)planes_dev & 15) || ((uintptr_t)image_dev & 3) ||
        ((uintptr_t)stats_dev & 7) || ((uintptr_t)uvw_host & 7) || ((uintptr_t)vis_host & 7) ||
        ((uintptr_t)weight_host & 3) || ((uintptr_t)scale_host & 7))
        return RICK_EINVAL;
    const int64_t per = n_chan > 0 ? n_chan : 1;  // visibilities per unit
    const int64_t vals = per * n_corr;              // values (and weights) per unit
    const int64_t n_vis = n_units * per;
    if (n_units > 0 && plan->max_vis < vals) return RICK_ERANGE;
    const StageLayout S = stage_layout(&plan->p, plan->max_vis, n_vis, stage_bytes);
    if (stage_bytes < S.bytes || (S.resident_uvw && S.uvw_buf < 24 * (size_t)n_units))
        return RICK_ERANGE;
    if (ws_bytes < rick_ws_layout(&plan->p, plan->max_vis).total) return RICK_ERANGE;
    RICK_TRY(stream_resources(plan));

    cudaStream_t st = (cudaStream_t)stream, cp = plan->copy;
    char *sb = (char *)stage_dev;
    WsHeader *rh = (WsHeader *)(sb + S.range);
    rick_bin_stats *tot = (rick_bin_stats *)(sb + S.total);
    WsHeader *hdr = rick_ws_ptrs(ws_dev, rick_ws_layout(&plan->p, plan->max_vis)).hdr;
    const int64_t chunk = plan->max_vis / vals;  // units per chunk (whole rows)
    const int64_t nchunks = n_units > 0 ? (n_units + chunk - 1) / chunk : 1;  // one empty chunk
    const float2 *vh = (const float2 *)vis_host;

    // Before the copy stream writes the staging area: for a staging area new
    // to this plan, everything enqueued earlier on the caller's stream (the
    // memory may have had other uses); for the same area as the plan's last
    // call, only the binnings that read its buffers -- so the copies of this
    // call overlap the previous call's gridding, FFT and w-correction.
    if (stage_dev != plan->stage_prev || stage_bytes != plan->stage_prev_bytes) {
        RICK_CUDA_TRY(plan, cudaEventRecord(plan->ev_start, st));
        RICK_CUDA_TRY(plan, cudaStreamWaitEvent(cp, plan->ev_start, 0));
        plan->stage_prev = stage_dev;
        plan->stage_prev_bytes = stage_bytes;
        plan->parity = 0;
        plan->next_buf = 0;
    }
    const int area = plan->parity;
    plan->parity ^= 1;
    // the call before last binned from this area (resident uvw, channel factors)
    RICK_CUDA_TRY(plan, cudaStreamWaitEvent(cp, plan->ev_area_free[area], 0));

    double *scale_dev = (double *)(sb + S.scale + area * 8 * (size_t)RICK_STREAM_MAX_CHAN);
    if (n_chan > 0 && n_units > 0)
        RICK_CUDA_TRY(plan, cudaMemcpyAsync(scale_dev, scale_host, 8 * (size_t)n_chan,
                                            cudaMemcpyHostToDevice, cp));
    const double *scale_c = n_chan > 0 ? scale_dev : NULL;

    double *uvw_res = (double *)(sb + S.uvw + area * S.uvw_buf);
    if (S.resident_uvw) {
        range_init_kernel<<<1, 1, 0, st>>>(rh);
        RICK_LAUNCH_CHECK(plan);
        for (int64_t c = 0; c < nchunks && n_units > 0; ++c) {
            const int64_t off = c * chunk, nc = n_units - off < chunk ? n_units - off : chunk;
            RICK_CUDA_TRY(plan, cudaMemcpyAsync(uvw_res + 3 * off, uvw_host + 3 * off, 24 * nc,
                                                cudaMemcpyHostToDevice, cp));
            RICK_CUDA_TRY(plan, cudaEventRecord(plan->ev_uvw, cp));
            RICK_CUDA_TRY(plan, cudaStreamWaitEvent(st, plan->ev_uvw, 0));
            rick_launch_wrange(plan, uvw_res + 3 * off, nc * per, rh, st, n_chan, scale_c);
            RICK_LAUNCH_CHECK(plan);
        }
    }

    // the fused transform's tile flags: the tiles earlier chunks of this call reached
    const uint8_t *touched = (const uint8_t *)(sb + S.fwork);  // its first field
    const bool chunk_tiles = S.fwork_bytes && !(plan->p.options & RICK_OPT_DETERMINISTIC);
    for (int64_t c = 0; c < nchunks; ++c) {
        const int b = plan->next_buf;
        plan->next_buf = (b + 1) % RICK_STREAM_BUFS;
        const int64_t off = c * chunk;
        const int64_t nc = n_units - off < chunk ? n_units - off : chunk;
        const double *uvw_c = NULL;
        const void *vis_c = NULL;
        const float *wt_c = NULL;
        if (nc > 0) {
            // staging buffer b was last read by the binning RICK_STREAM_BUFS
            // chunks earlier (of this call or the previous ones)
            RICK_CUDA_TRY(plan, cudaStreamWaitEvent(cp, plan->ev_free[b], 0));
            if (S.resident_uvw) {
                uvw_c = uvw_res + 3 * off;
            } else {
                double *ub = (double *)(sb + S.uvw + b * S.uvw_buf);
                RICK_CUDA_TRY(plan, cudaMemcpyAsync(ub, uvw_host + 3 * off, 24 * nc,
                                                    cudaMemcpyHostToDevice, cp));
                uvw_c = ub;
            }
            float2 *vb = (float2 *)(sb + S.vis + b * S.vis_buf);
            RICK_CUDA_TRY(plan, cudaMemcpyAsync(vb, vh + off * vals, 8 * nc * vals,
                                                cudaMemcpyHostToDevice, cp));
            vis_c = vb;
            if (weight_host) {
                float *wb = (float *)(sb + S.weight + b * S.weight_buf);
                RICK_CUDA_TRY(plan, cudaMemcpyAsync(wb, weight_host + off * vals, 4 * nc * vals,
                                                    cudaMemcpyHostToDevice, cp));
                wt_c = wb;
            }
            RICK_CUDA_TRY(plan, cudaEventRecord(plan->ev_ready[b], cp));
            RICK_CUDA_TRY(plan, cudaStreamWaitEvent(st, plan->ev_ready[b], 0));
        }
        RICK_TRY(rick_bin_impl(plan, nc > 0 ? nc * per : 0, uvw_c, vis_c, wt_c, ws_dev, ws_bytes,
                               NULL, st, S.resident_uvw ? rh : NULL, n_chan, scale_c, n_corr));
        // the binning has read staging buffer b (the records are in ws now)
        RICK_CUDA_TRY(plan, cudaEventRecord(plan->ev_free[b], st));
        stats_add_kernel<<<1, 1, 0, st>>>(hdr, tot, c == 0);
        RICK_LAUNCH_CHECK(plan);
        if (chunk_tiles)
            RICK_TRY(rick_grid_impl(plan, ws_dev, planes_dev, RICK_GRID_CHUNK_TILES, st,
                                    c > 0 ? touched : NULL));
        else
            RICK_TRY(rick_grid_impl(plan, ws_dev, planes_dev,
                                    c > 0 ? RICK_GRID_ACCUMULATE : RICK_GRID_OVERWRITE, st));
        // the tiles this chunk's records reach, for the fused transform
        if (S.fwork_bytes)
            RICK_TRY(rick_fft_tiles_impl(plan, ws_dev, sb + S.fwork, S.fwork_bytes, c > 0 ? 2 : 1,
                                         st));
    }
    // every binning of this call has read its resident uvw area and factors
    RICK_CUDA_TRY(plan, cudaEventRecord(plan->ev_area_free[area], st));
    stats_finish_kernel<<<1, 1, 0, st>>>(hdr, tot, stats_dev);
    RICK_LAUNCH_CHECK(plan);
    if (S.fwork_bytes)
        return rick_fft_wcorrect_impl(plan, planes_dev, ws_dev, sb + S.fwork, S.fwork_bytes,
                                      image_dev, flags, st);
    RICK_TRY(rick_fft_wplanes(plan, planes_dev, 1, st));
    RICK_TRY(rick_wcorrect_stack(plan, planes_dev, ws_dev, image_dev, flags, st));
    return RICK_OK;
}

extern "C" rick_status rick_image_host(rick_plan *plan, int64_t n_vis, const double *uvw_host,
                                       const void *vis_host, const float *weight_host,
                                       void *ws_dev, size_t ws_bytes, void *stage_dev,
                                       size_t stage_bytes, void *planes_dev, float *image_dev,
                                       uint32_t flags, rick_bin_stats *stats_dev, void *stream)
{
    return stream_impl(plan, n_vis, 0, 1, uvw_host, NULL, vis_host, weight_host, ws_dev, ws_bytes,
                       stage_dev, stage_bytes, planes_dev, image_dev, flags, stats_dev, stream);
}

extern "C" rick_status rick_image_host_channels(rick_plan *plan, int64_t n_rows, int32_t n_chan,
                                                const double *uvw_rows_host,
                                                const double *chan_scale_host,
                                                const void *vis_host, const float *weight_host,
                                                void *ws_dev, size_t ws_bytes, void *stage_dev,
                                                size_t stage_bytes, void *planes_dev,
                                                float *image_dev, uint32_t flags,
                                                rick_bin_stats *stats_dev, void *stream)
{
    if (n_chan < 1) return RICK_EINVAL;
    return stream_impl(plan, n_rows, n_chan, 1, uvw_rows_host, chan_scale_host, vis_host,
                       weight_host, ws_dev, ws_bytes, stage_dev, stage_bytes, planes_dev, image_dev,
                       flags, stats_dev, stream);
}

extern "C" rick_status rick_image_host_rows(rick_plan *plan, int64_t n_rows, int32_t n_chan,
                                            int32_t n_corr, const double *uvw_rows_host,
                                            const double *chan_scale_host, const void *vis_host,
                                            const float *weight_host, void *ws_dev,
                                            size_t ws_bytes, void *stage_dev, size_t stage_bytes,
                                            void *planes_dev, float *image_dev, uint32_t flags,
                                            rick_bin_stats *stats_dev, void *stream)
{
    if (n_chan < 1) return RICK_EINVAL;
    return stream_impl(plan, n_rows, n_chan, n_corr, uvw_rows_host, chan_scale_host, vis_host,
                       weight_host, ws_dev, ws_bytes, stage_dev, stage_bytes, planes_dev, image_dev,
                       flags, stats_dev, stream);
}

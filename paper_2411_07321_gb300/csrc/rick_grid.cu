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
// float2 atomics.  Tiles without records are not gridding items: the
// persistent gridding CTAs clear them in groups between their gridding items,
// so the stores of zeros overlap the gridding of the other tiles.
//
// Degridding: one CTA per chunk of a non-empty tile's own bin; the CTA stages
// the (T + W - 1)^2 plane region its records can touch into shared memory and
// each thread gathers one record's W x W footprint.
#include "rick_common.cuh"

struct GridArgs {
    TileArgs t;
    float2 *planes;
    int log2T;
    int accumulate;  // add into the planes instead of overwriting them
    const uint8_t *touched;  // per tile: add into it (tiles an earlier chunk gridded), or NULL
    uint32_t nzero;  // tile-clearing items (RICK_ZERO_GROUP tiles each); 0 when accumulating
    const uint32_t *mcslot;     // deterministic mode: slot of each multi-item tile
    unsigned long long *mcacc;  // deterministic mode: the slots' int64 (re, im) sums
};

// Accumulation modes of the grid kernel: FP32 shared-memory sums, FP32 rounds
// folded by compensated summation, or 64-bit fixed point (deterministic: the
// sums do not depend on the order of the atomics).
#define GM_PLAIN 0
#define GM_COMP 1
#define GM_DET 2

// Tiles per clearing item of the grid kernel.
#define RICK_ZERO_GROUP 8

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

// ------------------------------------------------------------------------
// Record streams.  A group of W consecutive lanes walks a contiguous run of
// records; lane j of the group owns footprint row j (W cells).  Per record,
// lane j evaluates kernel segment j at both offsets -- gx[j] = G((j - h) - fx)
// and gy[j] = G((j - h) - fy), one Horner chain on (x, y) pairs with packed
// two-wide FP32 FMAs and the segment's coefficients held (duplicated) in the
// lane's registers -- so it already has its row's v weight, scales the
// visibility by it, and takes the W u weights from its group with shuffles:
// W shuffles and W packed FMAs per record and lane (re and im of two cells per
// instruction pair).  While consecutive records share
// the footprint corner (the channels of one baseline-time land on the same
// cells) the row sums stay in registers; when the corner changes the group
// adds its rows to the tile accumulator at once -- one row per lane, so the
// group's atomics never collide.

// A record stream is a group of G consecutive lanes, lane j owning footprint
// row j < W.  G is the power of two next to W when that packs as many groups
// into a warp as W lanes would (W = 7: four groups either way, and the lane
// arithmetic is shifts), else W itself (W = 9: three groups of nine instead of
// two of sixteen).  A warp holds NG = 32 / G groups; its last 32 - NG G lanes
// stay idle.
template <int W>
struct StreamShape {
    static constexpr int P2 = W <= 1 ? 1 : W <= 2 ? 2 : W <= 4 ? 4 : W <= 8 ? 8 : 16;
    static constexpr int G = (32 / P2 == 32 / W) ? P2 : W;
    static constexpr int NG = 32 / G;
    static constexpr int LIVE = NG * G;  // lanes of a warp that carry a stream
};

// Warps of a gridding CTA (256 threads).
#define RICK_GRID_WARPS 8

// The lane's row sums into the tile accumulator: fb is the index of the row's
// first cell, bit jx of fv says whether column jx lies inside the tile (fv = 0
// when the row is outside it or the lane carries no row).  Both are set once
// per footprint corner, so the loop over records carries two registers for
// the flush instead of the corner's geometry.
template <int W>
__device__ __forceinline__ void group_flush(float *acc_re, float *acc_im, int fb, uint32_t fv,
                                            const float *ar, const float *ai)
{
    if (!fv) return;
#pragma unroll
    for (int jx = 0; jx < W; ++jx) {
        if ((fv >> jx) & 1u) {
            atomicAdd(&acc_re[fb + jx], ar[jx]);
            atomicAdd(&acc_im[fb + jx], ai[jx]);
        }
    }
}

// The same into the 64-bit fixed-point tile: each row sum scaled by 2^k and
// rounded to an integer, then added with integer atomics (exact, so the tile
// does not depend on the order in which the groups flush).
template <int W>
__device__ __forceinline__ void group_flush_det(unsigned long long *acc64, float fx, int T, int TP,
                                                int lx, int row, bool live, const float *ar,
                                                const float *ai)
{
    if (!live || (unsigned)row >= (unsigned)T) return;
#pragma unroll
    for (int jx = 0; jx < W; ++jx) {
        int col = lx + jx;
        if ((unsigned)col < (unsigned)T) {
            int i = 2 * (row * TP + col);
            atomicAdd(&acc64[i], (unsigned long long)__float2ll_rn(ar[jx] * fx));
            atomicAdd(&acc64[i + 1], (unsigned long long)__float2ll_rn(ai[jx] * fx));
        }
    }
}

// Asynchronous copies global -> shared (cp.async): 16 or 4 bytes, both
// addresses aligned to the size.
__device__ __forceinline__ void cp_async16(void *sdst, const void *gsrc)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async4(void *sdst, const void *gsrc)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// all but the most recently committed group have landed (for this thread)
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Record ring of a warp: where a warp carries at most three record streams
// (W >= 9, three CTAs per SM), the streams' next records are staged in shared
// memory by the whole warp, RICK_GRID_RB records per stream per chunk, two
// chunks in flight, so that the record loop reads them from shared memory
// instead of waiting on global loads one record ahead (large workload, W = 9:
// grid 9.92 -> 9.06 ms).  With four streams (W = 7, four CTAs per SM) the
// extra warps already hide the loads and the ring measured 2 % slower.
#define RICK_GRID_RB 16

template <int W>
struct RecRing {
    static constexpr bool ON = W > 1 && StreamShape<W>::NG <= 3;
    static constexpr int NG = StreamShape<W>::NG;
    static constexpr int SLOTS = ON ? NG * RICK_GRID_RB : 1;  // records per chunk and warp
};

// Copy chunk c of the warp's streams (iterations c RB ... c RB + RB - 1; past
// a stream's end its last record again) into buffer c & 1 of the ring.  Slot
// e = lane + 32 h holds record e % RB of stream e / RB, whose first record and
// last index are cr0[h] and clast[h].
template <int W>
__device__ __forceinline__ void ring_issue(const TileArgs &ta, float4 *wrec, uint32_t *wcel,
                                           uint32_t c, const uint32_t *cr0, const uint32_t *clast)
{
    constexpr int RB = RICK_GRID_RB, SLOTS = RecRing<W>::SLOTS;
#pragma unroll
    for (int h = 0; h < (SLOTS + 31) / 32; ++h) {
        const int e = (threadIdx.x & 31) + 32 * h;
        if (e < SLOTS) {
            const uint32_t idx = cr0[h] + min(c * RB + (uint32_t)(e % RB), clast[h]);
            const int slot = (int)(c & 1u) * SLOTS + e;
            cp_async16(wrec + slot, ta.rec + idx);
            cp_async4(wcel + slot, ta.rcell + idx);
        }
    }
    cp_async_commit();
}

// n records of one segment of the tile's record list, starting at record r0.
// DET: the flushes go to the 64-bit fixed-point tile acc64 (scale fx).
template <int W, bool DET>
__device__ __forceinline__ void grid_stream(const TileArgs &ta, uint32_t r0, uint32_t n,
                                            uint32_t ntrip, int x0,
                                            int y0, float *acc_re, float *acc_im, int T, int TP,
                                            const float2 *coef2, unsigned long long *acc64,
                                            float fx)
{
    constexpr int G = StreamShape<W>::G;
    const int lane = threadIdx.x & 31, grp = lane / G;
    const int j = lane - grp * G;  // this lane's row / kernel segment
    const bool live = lane < StreamShape<W>::LIVE && j < W && n > 0;
    if (ntrip == 0) return;
    const uint32_t last = n > 0 ? n - 1 : 0;
    float ar[W], ai[W];
#pragma unroll
    for (int jx = 0; jx < W; ++jx) ar[jx] = ai[jx] = 0.0f;
    const float4 *rec = ta.rec + r0;
    const uint32_t *rcell = ta.rcell + r0;
    // the warp's record ring: chunk c of every stream of the warp in buffer c & 1
    using Ring = RecRing<W>;
    constexpr int RB = RICK_GRID_RB, NGR = Ring::NG;
    __shared__ __align__(16) float4 s_rrec[Ring::ON ? RICK_GRID_WARPS * 2 * Ring::SLOTS : 1];
    __shared__ uint32_t s_rcel[Ring::ON ? RICK_GRID_WARPS * 2 * Ring::SLOTS : 1];
    float4 *wrec = s_rrec + (Ring::ON ? (threadIdx.x >> 5) * 2 * Ring::SLOTS : 0);
    uint32_t *wcel = s_rcel + (Ring::ON ? (threadIdx.x >> 5) * 2 * Ring::SLOTS : 0);
    const int rg = grp < NGR ? grp : NGR - 1;  // the stream this lane reads (idle lanes: any)
    // this lane's slots of a chunk (e = lane + 32 h): record rr of stream g,
    // whose first record and last index come from the stream's first lane
    constexpr int NH = (Ring::SLOTS + 31) / 32;
    uint32_t cr0[NH], clast[NH];
#pragma unroll
    for (int h = 0; h < NH; ++h) {
        const int e = (threadIdx.x & 31) + 32 * h, g = min(e / RB, NGR - 1);
        cr0[h] = Ring::ON ? __shfl_sync(0xffffffffu, r0, g * G) : 0u;
        clast[h] = Ring::ON ? __shfl_sync(0xffffffffu, last, g * G) : 0u;
    }
    auto ring_at = [&](uint32_t i) { return (int)((i / RB) & 1u) * Ring::SLOTS + rg * RB + (int)(i % RB); };
    uint32_t cur;
    float4 q;
    int ri = 0;  // ring slot of the record being read (running: reset at chunk starts)
    if constexpr (Ring::ON) {
        ring_issue<W>(ta, wrec, wcel, 0, cr0, clast);
        ring_issue<W>(ta, wrec, wcel, 1, cr0, clast);
        cp_async_wait1();
        __syncwarp();
        ri = ring_at(0);
        q = wrec[ri];
        cur = wcel[ri];
    } else {
        cur = rcell[0];
        q = rec[0];
    }
    uint32_t cell = cur;
    // the flush target of corner cur (group_flush)
    int fb;
    uint32_t fv;
    auto target = [&](uint32_t c) {
        const int lx = (int)(c & 0xFFFFu) - x0, row = (int)(c >> 16) - y0 + j;
        fb = row * TP + lx;
        uint32_t m = 0;
#pragma unroll
        for (int jx = 0; jx < W; ++jx) m |= ((unsigned)(lx + jx) < (unsigned)T ? 1u : 0u) << jx;
        fv = (live && (unsigned)row < (unsigned)T) ? m : 0u;
    };
    target(cur);
    for (uint32_t i = 0; i < ntrip; ++i) {
        // the next record; past the stream's end the last one again
        float4 nq;
        uint32_t ncell;
        if constexpr (Ring::ON) {
            const uint32_t i1 = i + 1;
            if (i1 % RB == 0) {
                if (i1 < ntrip) {
                    // entering chunk c = i1 / RB: the warp is done with chunk c - 1
                    // (record i was read last iteration), so its buffer takes chunk
                    // c + 1; chunk c has landed once only that copy is pending
                    __syncwarp();
                    ring_issue<W>(ta, wrec, wcel, i1 / RB + 1, cr0, clast);
                    cp_async_wait1();
                    __syncwarp();
                }
                ri = ring_at(i1);
            } else {
                ++ri;
            }
            nq = wrec[ri];
            ncell = wcel[ri];
        } else {
            const uint32_t ln = min(i + 1, last);
            nq = rec[ln];
            ncell = rcell[ln];
        }
        if (cell != cur) {
            if (DET)
                group_flush_det<W>(acc64, fx, T, TP, (int)(cur & 0xFFFFu) - x0,
                                   (int)(cur >> 16) - y0 + j, live, ar, ai);
            else
                group_flush<W>(acc_re, acc_im, fb, fv, ar, ai);
#pragma unroll
            for (int jx = 0; jx < W; ++jx) ar[jx] = ai[jx] = 0.0f;
            cur = cell;
            target(cur);
        }
        float gx = 1.0f, gy = 1.0f;
        if (W > 1) {
            const float2 s2 = make_float2(2.0f * (q.z - ta.kp.fc), 2.0f * (q.w - ta.kp.fc));
            float2 g2 = coef2[RICK_POLY_DEG];
#pragma unroll
            for (int k = RICK_POLY_DEG - 1; k >= 0; --k) g2 = __ffma2_rn(g2, s2, coef2[k]);
            gx = g2.x;
            gy = g2.y;
        }
        const float gz = i < n ? gy : 0.0f;
        const float2 vv = __fmul2_rn(make_float2(q.x, q.y), make_float2(gz, gz));
        const float2 vr2 = make_float2(vv.x, vv.x), vi2 = make_float2(vv.y, vv.y);
        float wv[W];
#pragma unroll
        for (int jx = 0; jx < W; ++jx) {
            // power-of-two groups: the lane inside the group is an immediate
            // (width form); groups of W lanes: the absolute lane
            wv[jx] = W == 1 ? gx
                   : (G & (G - 1)) == 0 ? __shfl_sync(0xffffffffu, gx, jx, G)
                                        : __shfl_sync(0xffffffffu, gx, grp * G + jx);
        }
#pragma unroll
        for (int jx = 0; jx + 1 < W; jx += 2) {
            const float2 w2 = make_float2(wv[jx], wv[jx + 1]);
            const float2 a2 = __ffma2_rn(vr2, w2, make_float2(ar[jx], ar[jx + 1]));
            const float2 b2 = __ffma2_rn(vi2, w2, make_float2(ai[jx], ai[jx + 1]));
            ar[jx] = a2.x; ar[jx + 1] = a2.y;
            ai[jx] = b2.x; ai[jx + 1] = b2.y;
        }
        if (W & 1) {
            ar[W - 1] = __fmaf_rn(vv.x, wv[W - 1], ar[W - 1]);
            ai[W - 1] = __fmaf_rn(vv.y, wv[W - 1], ai[W - 1]);
        }
        q = nq;
        cell = ncell;
    }
    if (DET)
        group_flush_det<W>(acc64, fx, T, TP, (int)(cur & 0xFFFFu) - x0, (int)(cur >> 16) - y0 + j,
                           live, ar, ai);
    else
        group_flush<W>(acc_re, acc_im, fb, fv, ar, ai);
    if constexpr (Ring::ON) {
        // the copies still in flight land before the ring is used again
        cp_async_wait0();
        __syncwarp();
    }
}

template <int W, int MODE>
__device__ __forceinline__ void grid_item(const GridArgs &a, uint32_t b, uint32_t t, float *sm,
                                          const float2 *coef2)
{
    constexpr bool COMP = MODE == GM_COMP, DET = MODE == GM_DET;
    const TileArgs &ta = a.t;
    const uint32_t chunk = b - ta.base[t], nch = ta.base[t + 1] - ta.base[t];
    const int T = 1 << a.log2T, TP = T + 1, TT = T * TP, nt = ta.nt;
    const uint32_t tx = t % nt, ty = (t / nt) % nt, k = t / (nt * nt);
    const int x0 = tx << a.log2T, y0 = ty << a.log2T;
    const uint32_t *off = ta.offsets;

    // the four record ranges that can touch this tile: its own bin, and the
    // edge classes of the west, north and north-west bins that reach into it
    uint32_t rs[4], rl[4];
    rs[0] = off[4 * t];
    rl[0] = off[4 * t + 4] - rs[0];
    rs[1] = rl[1] = rs[2] = rl[2] = rs[3] = rl[3] = 0;
    if (tx > 0) {
        rs[1] = off[4 * (t - 1) + 1];
        rl[1] = off[4 * (t - 1) + 3] - rs[1];
    }
    if (ty > 0) {
        rs[2] = off[4 * (t - nt) + 2];
        rl[2] = off[4 * (t - nt) + 4] - rs[2];
    }
    if (tx > 0 && ty > 0) {
        rs[3] = off[4 * (t - nt - 1) + 2];
        rl[3] = off[4 * (t - nt - 1) + 3] - rs[3];
    }
    const uint32_t Ltot = rl[0] + rl[1] + rl[2] + rl[3];
    // the ranges in shared memory, for a loop over them that is not unrolled
    // (one copy of the record loop keeps the kernel small)
    __shared__ uint32_t s_rs[4], s_rl[4];
    if (threadIdx.x < 4) {
        s_rs[threadIdx.x] = rs[threadIdx.x];
        s_rl[threadIdx.x] = rl[threadIdx.x];
    }
    const uint32_t cap = ta.hdr->chunk_cap;
    const uint32_t vbeg = chunk * cap;
    const uint32_t vend = min(Ltot, vbeg + cap);

    // accumulators with padded rows (stride T + 1): the lanes of a group own
    // different rows, which then fall in different banks
    float *acc_re = sm, *acc_im = sm + TT;
    float *sum_re = sm + 2 * TT, *sum_im = sm + 3 * TT, *cmp_re = sm + 4 * TT, *cmp_im = sm + 5 * TT;
    unsigned long long *acc64 = (unsigned long long *)sm;  // DET: (re, im) pairs
    const float fx = DET ? ta.hdr->fx_scale : 0.0f;
    for (int i = threadIdx.x; i < TT; i += blockDim.x) {
        if (DET) {
            acc64[2 * i] = 0ull;
            acc64[2 * i + 1] = 0ull;
        } else {
            acc_re[i] = 0.0f;
            acc_im[i] = 0.0f;
        }
        if (COMP) sum_re[i] = sum_im[i] = cmp_re[i] = cmp_im[i] = 0.0f;
    }
    __syncthreads();

    // plain: one round over the chunk; compensated: rounds of 4096 records,
    // each folded into the (sum, compensation) pair of every cell.  The
    // round's piece of each of the four ranges is split evenly into one
    // contiguous run per record stream, so the streams of a warp always walk
    // the same range with runs of equal length (a split of the whole round
    // would let a warp's streams straddle a range boundary, and the warp then
    // walks both ranges one after the other).
    constexpr int NG = StreamShape<W>::NG;
    const int lane = threadIdx.x & 31;
    const bool streaming = lane < StreamShape<W>::LIVE;
    const uint32_t nstreams = (blockDim.x >> 5) * NG;
    const uint32_t stream = (threadIdx.x >> 5) * NG + (streaming ? lane / StreamShape<W>::G : 0);
    const uint32_t round = COMP ? 4096u : max(vend - vbeg, 1u);
    for (uint32_t rb = vbeg; rb < vend; rb += round) {
        const uint32_t re = min(vend, rb + round);
        uint32_t base = 0;
#pragma unroll 1
        for (int g = 0; g < 4; ++g) {
            const uint32_t lg = s_rl[g];
            const uint32_t a0 = max(rb, base), a1 = min(re, base + lg);
            if (a0 < a1) {
                const uint32_t per = (a1 - a0 + nstreams - 1) / nstreams;
                const uint32_t v0 = min(a0 + stream * per, a1), v1 = min(v0 + per, a1);
                const uint32_t nv = streaming ? v1 - v0 : 0u;
                grid_stream<W, DET>(ta, s_rs[g] + ((nv ? v0 : a0) - base), nv, per, x0, y0,
                                    acc_re, acc_im,
                                        T, TP, coef2, acc64, fx);
            }
            base += lg;
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
    if (DET && nch > 1) {  // several work items: exact integer sums in the tile's slot
        unsigned long long *slot = a.mcacc + (size_t)a.mcslot[t] * 2 * T * T;
        for (int i = threadIdx.x; i < T * T; i += blockDim.x) {
            const int ip = (i >> a.log2T) * TP + (i & (T - 1));
            const unsigned long long re = acc64[2 * ip], im = acc64[2 * ip + 1];
            if (re) atomicAdd(&slot[2 * i], re);
            if (im) atomicAdd(&slot[2 * i + 1], im);
        }
        return;
    }
    const float fxi = DET ? ta.hdr->fx_inv : 0.0f;
    const bool acc = a.accumulate || (a.touched && a.touched[t]);
    for (int i = threadIdx.x; i < T * T; i += blockDim.x) {
        int row = i >> a.log2T, col = i & (T - 1), ip = row * TP + col;
        int gi = x0 + col, gj = y0 + row;
        float re = DET ? __ll2float_rn((long long)acc64[2 * ip]) * fxi
                 : COMP ? sum_re[ip] + cmp_re[ip] : acc_re[ip];
        float im = DET ? __ll2float_rn((long long)acc64[2 * ip + 1]) * fxi
                 : COMP ? sum_im[ip] + cmp_im[ip] : acc_im[ip];
        if ((gi + gj) & 1) {
            re = -re;
            im = -im;
        }
        float2 *dst = plane + (size_t)gj * n + gi;
        if (nch == 1 && !acc) {
            *dst = make_float2(re, im);
        } else if (nch == 1) {  // the only writer of this tile in this launch
            float2 o = *dst;
            *dst = make_float2(o.x + re, o.y + im);
        } else if (re != 0.0f || im != 0.0f) {
            atomicAdd(dst, make_float2(re, im));
        }
    }
}

// Clear the tiles of group z that have no work item (no records reach them):
// 16-byte stores, the CTA's threads striding over the tile.
__device__ __forceinline__ void zero_group(const GridArgs &a, uint32_t z)
{
    const TileArgs &ta = a.t;
    const int T = 1 << a.log2T, half = T >> 1, nt = ta.nt, n = ta.n;
    const uint32_t t1 = min(ta.ntiles, (z + 1) * RICK_ZERO_GROUP);
    for (uint32_t t = z * RICK_ZERO_GROUP; t < t1; ++t) {
        if (ta.base[t + 1] != ta.base[t]) continue;
        const uint32_t tx = t % nt, ty = (t / nt) % nt, k = t / (nt * nt);
        float4 *plane = (float4 *)(a.planes + (size_t)k * n * n);
        for (int i = threadIdx.x; i < T * half; i += blockDim.x) {
            const int row = i / half, col2 = i - row * half;
            plane[((size_t)((ty << a.log2T) + row) * n + (tx << a.log2T)) / 2 + col2] =
                make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
}

// Persistent: one wave of CTAs takes work items (tile, chunk) from a counter
// in the workspace header (reset by zero_tiles_kernel, launched just before),
// and with each a clearing item for a group of tiles without records, so that
// the HBM-bound clearing of the empty tiles runs under the issue-bound
// gridding of the others.  Four CTAs per SM for W <= 8 (64 registers a
// thread): the record loop is latency-bound, and the extra warps hide more of
// it than the few spilled registers cost.
template <int W, int MODE>
__global__ void __launch_bounds__(32 * RICK_GRID_WARPS, (W <= 8 && MODE == GM_PLAIN) ? 4 : 3)
    grid_kernel(GridArgs a)
{
    extern __shared__ float sm[];
    __shared__ uint32_t s_b, s_tile, s_z;
    const uint32_t total = a.t.base[a.t.ntiles];
    // this lane's kernel segment (= its footprint row within its group)
    const int seg = min((int)((threadIdx.x & 31) % StreamShape<W>::G), W - 1);
    float2 coef2[RICK_POLY_N];
#pragma unroll
    for (int k = 0; k < RICK_POLY_N; ++k) coef2[k] = make_float2(a.t.kp.c[seg][k], a.t.kp.c[seg][k]);
    for (;;) {
        if (threadIdx.x == 0) {
            const uint32_t b = atomicAdd(&a.t.hdr->grid_next, 1u);
            s_b = b;
            s_tile = b < total ? find_tile(a.t.base, a.t.ntiles, b) : 0u;
            s_z = a.nzero ? atomicAdd(&a.t.hdr->zero_next, 1u) : 0u;
        }
        __syncthreads();
        const uint32_t b = s_b, t = s_tile, z = s_z;
        __syncthreads();  // everyone has the item before thread 0 takes the next
        if (b >= total && z >= a.nzero) break;
        if (b < total) {
            grid_item<W, MODE>(a, b, t, sm, coef2);
            __syncthreads();  // the accumulator is reused by the next item
        }
        if (z < a.nzero) zero_group(a, z);
    }
}

// Several imaging jobs gridded by one launch (rick_grid_sparse_batch): the jobs'
// work items form one list, job after job, taken from one counter (the first
// job's).  Every job has the same support W and tile T, and plain FP32 sums.
// RICK_GRID_BATCH_MAX (rick.h) jobs at most: the arguments travel as one
// kernel parameter.

struct GridBatchArgs {
    int n_jobs;
    GridArgs job[RICK_GRID_BATCH_MAX];
};
static_assert(sizeof(GridBatchArgs) <= 32764, "kernel parameters are limited to 32764 bytes");

// Zero the tiles whose chunks add into them with atomics (more than one work
// item) before the grid kernel runs, and reset the grid kernel's counters.
// Grid-stride, one warp per tile, 16-byte stores.  Tiles without records are
// cleared by the grid kernel itself; when gridding adds into existing planes
// nothing is cleared, and neither are the tiles flagged in touched (a chunk of a
// streamed set adds into the tiles earlier chunks gridded).
// Deterministic mode (mcacc != NULL): the int64 slots of those tiles are
// zeroed instead, accumulating or not (the slots are added into the planes
// after gridding).
__global__ void __launch_bounds__(256) zero_tiles_kernel(const uint32_t *base, uint32_t ntiles,
                                                         int nt, int log2T, int n, float2 *planes,
                                                         WsHeader *hdr, int accumulate,
                                                         const uint32_t *mcslot,
                                                         unsigned long long *mcacc,
                                                         const uint8_t *touched)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        hdr->grid_next = 0;
        hdr->zero_next = 0;
    }
    int lane = threadIdx.x & 31;
    uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    const int T = 1 << log2T, half = T >> 1;  // float4 = two cells
    if (mcacc) {
        for (uint32_t t = warp; t < ntiles; t += nwarps) {
            if (base[t + 1] - base[t] <= 1) continue;
            ulonglong2 *slot = (ulonglong2 *)(mcacc + (size_t)mcslot[t] * 2 * T * T);
            for (int i = lane; i < T * T; i += 32) slot[i] = make_ulonglong2(0ull, 0ull);
        }
        return;
    }
    if (accumulate) return;
    for (uint32_t t = warp; t < ntiles; t += nwarps) {
        if (base[t + 1] - base[t] <= 1 || (touched && touched[t])) continue;
        uint32_t tx = t % nt, ty = (t / nt) % nt, k = t / (nt * nt);
        float4 *plane = (float4 *)(planes + (size_t)k * n * n);
        for (int i = lane; i < T * half; i += 32) {
            int row = i / half, col2 = i - row * half;
            plane[((size_t)((ty << log2T) + row) * n + (tx << log2T)) / 2 + col2] =
                make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
}

// The batch's multi-item tiles zeroed (one row of CTAs per job, blockIdx.y) and
// its item counter reset.
__global__ void __launch_bounds__(256)
    zero_tiles_batch_kernel(const __grid_constant__ GridBatchArgs ba)
{
    const GridArgs &a = ba.job[blockIdx.y];
    const TileArgs &ta = a.t;
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) ta.hdr->grid_next = 0;
    const int lane = threadIdx.x & 31, log2T = a.log2T, T = 1 << log2T, half = T >> 1;
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    const int nt = ta.nt, n = ta.n;
    for (uint32_t t = warp; t < ta.ntiles; t += nwarps) {
        if (ta.base[t + 1] - ta.base[t] <= 1) continue;
        const uint32_t tx = t % nt, ty = (t / nt) % nt, k = t / (nt * nt);
        float4 *plane = (float4 *)(a.planes + (size_t)k * n * n);
        for (int i = lane; i < T * half; i += 32) {
            const int row = i / half, col2 = i - row * half;
            plane[((size_t)((ty << log2T) + row) * n + (tx << log2T)) / 2 + col2] =
                make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
}

// Persistent over the batch's work items: item b of the list belongs to the
// job j with cum[j] <= b < cum[j + 1] (cum: running totals of the jobs' items),
// and is that job's item b - cum[j].  A CTA reloads its lanes' kernel
// coefficients when the job changes.
template <int W>
__global__ void __launch_bounds__(32 * RICK_GRID_WARPS, W <= 8 ? 4 : 3)
    grid_batch_kernel(const __grid_constant__ GridBatchArgs ba)
{
    extern __shared__ float sm[];
    __shared__ uint32_t s_cum[RICK_GRID_BATCH_MAX + 1];
    __shared__ uint32_t s_b, s_tile, s_job;
    if (threadIdx.x == 0) {
        uint32_t c = 0;
        s_cum[0] = 0;
        for (int j = 0; j < ba.n_jobs; ++j) {
            c += ba.job[j].t.base[ba.job[j].t.ntiles];
            s_cum[j + 1] = c;
        }
    }
    __syncthreads();
    const uint32_t total = s_cum[ba.n_jobs];
    const int seg = min((int)((threadIdx.x & 31) % StreamShape<W>::G), W - 1);
    float2 coef2[RICK_POLY_N];
    int cur = -1;
    for (;;) {
        if (threadIdx.x == 0) {
            const uint32_t b = atomicAdd(&ba.job[0].t.hdr->grid_next, 1u);
            int j = 0;
            while (j + 1 < ba.n_jobs && s_cum[j + 1] <= b) ++j;
            s_b = b;
            s_job = (uint32_t)j;
            s_tile = b < total ? find_tile(ba.job[j].t.base, ba.job[j].t.ntiles, b - s_cum[j]) : 0u;
        }
        __syncthreads();
        const uint32_t b = s_b, t = s_tile;
        const int j = (int)s_job;
        __syncthreads();  // everyone has the item before thread 0 takes the next
        if (b >= total) break;
        const GridArgs &a = ba.job[j];
        if (j != cur) {
#pragma unroll
            for (int k = 0; k < RICK_POLY_N; ++k)
                coef2[k] = make_float2(a.t.kp.c[seg][k], a.t.kp.c[seg][k]);
            cur = j;
        }
        grid_item<W, GM_PLAIN>(a, b - s_cum[j], t, sm, coef2);
        __syncthreads();  // the accumulator is reused by the next item
    }
}

// Deterministic mode: the tiles gridded by several work items, from their
// int64 slots into the planes (written, or added with accumulate), the
// checkerboard (-1)^(i+j) folded in.  One warp per tile.
__global__ void __launch_bounds__(256) det_mc_convert_kernel(const uint32_t *base, uint32_t ntiles,
                                                             int nt, int log2T, int n,
                                                             float2 *planes, const WsHeader *hdr,
                                                             int accumulate,
                                                             const uint32_t *mcslot,
                                                             const unsigned long long *mcacc)
{
    const int lane = threadIdx.x & 31, T = 1 << log2T;
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    const float inv = hdr->fx_inv;
    for (uint32_t t = warp; t < ntiles; t += nwarps) {
        if (base[t + 1] - base[t] <= 1) continue;
        const uint32_t tx = t % nt, ty = (t / nt) % nt, k = t / (nt * nt);
        const unsigned long long *slot = mcacc + (size_t)mcslot[t] * 2 * T * T;
        float2 *plane = planes + (size_t)k * n * n;
        for (int i = lane; i < T * T; i += 32) {
            const int row = i >> log2T, col = i & (T - 1);
            const int gi = (int)(tx << log2T) + col, gj = (int)(ty << log2T) + row;
            float re = __ll2float_rn((long long)slot[2 * i]) * inv;
            float im = __ll2float_rn((long long)slot[2 * i + 1]) * inv;
            if ((gi + gj) & 1) {
                re = -re;
                im = -im;
            }
            float2 *dst = plane + (size_t)gj * n + gi;
            if (accumulate) {
                const float2 o = *dst;
                re += o.x;
                im += o.y;
            }
            *dst = make_float2(re, im);
        }
    }
}

// n_src: with the Hermitian mirror the inputs (records from n_src on mirror
// input i - n_src), else 0.
template <int W>
__device__ __forceinline__ void degrid_item(const DegridArgs &a, uint32_t b, uint32_t t,
                                            float2 *stage, uint32_t n_src)
{
    const TileArgs &ta = a.t;
    const uint32_t chunk = b - ta.base[t];
    const int T = 1 << a.log2T, S = T + W - 1, nt = ta.nt, n = ta.n;
    const uint32_t tx = t % nt, ty = (t / nt) % nt, k = t / (nt * nt);
    const int x0 = tx << a.log2T, y0 = ty << a.log2T;
    const uint32_t cap = ta.hdr->chunk_cap;
    const uint32_t r0 = ta.offsets[4 * t] + chunk * cap;
    const uint32_t r1 = min(ta.offsets[4 * t + 4], r0 + cap);

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
        const float4 q = ta.rec[r];
        const float2 fr = make_float2(q.z, q.w);
        uint32_t cell = ta.rcell[r];
        int lx = (int)(cell & 0xFFFFu) - x0, ly = (int)(cell >> 16) - y0;
        float gx[W], gy[W];
        kernel_weights<W>(ta.kp, fr.x, gx);
        kernel_weights<W>(ta.kp, fr.y, gy);
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
        const uint32_t m = ta.perm[r];
        if (n_src == 0) {
            const float wt = a.weight ? a.weight[m] : 1.0f;
            a.vis_out[m] = make_float2(sr * wt, si * wt);
        } else {
            // the Hermitian mirror: input m' gets its record's value plus the
            // conjugate of its mirrored record's (two adds onto zero, so the
            // result does not depend on their order)
            const bool mir = m >= n_src;
            const uint32_t src = mir ? m - n_src : m;
            const float wt = a.weight ? a.weight[src] : 1.0f;
            atomicAdd(&a.vis_out[src], make_float2(sr * wt, mir ? -si * wt : si * wt));
        }
    }
}

template <int W>
__global__ void __launch_bounds__(256) degrid_kernel(DegridArgs a)
{
    extern __shared__ float2 stage[];
    __shared__ uint32_t s_b, s_tile;
    const uint32_t total = a.t.base[a.t.ntiles];
    const uint32_t n_src = a.t.hdr->mirror ? (uint32_t)a.t.hdr->n_src : 0u;
    for (;;) {
        if (threadIdx.x == 0) {
            uint32_t b = atomicAdd(&a.t.hdr->degrid_next, 1u);
            s_b = b;
            s_tile = b < total ? find_tile(a.t.base, a.t.ntiles, b) : 0u;
        }
        __syncthreads();
        const uint32_t b = s_b, t = s_tile;
        if (b >= total) break;
        degrid_item<W>(a, b, t, stage, n_src);
        __syncthreads();
    }
}

// Dropped visibilities (key == all ones) get a zero model value.  With the
// Hermitian mirror every output is zeroed: both records of an input add into it.
__global__ void degrid_zero_dropped_kernel(WsHeader *hdr, const uint32_t *key, float2 *vis_out)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) hdr->degrid_next = 0;
    const bool all = hdr->mirror != 0;
    int64_t n = (int64_t)(all ? hdr->n_src : hdr->n_vis);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        if (all || key[i] == 0xFFFFFFFFu) vis_out[i] = make_float2(0.f, 0.f);
}

// ------------------------------------------------------------------------

static TileArgs make_tile_args(const rick_plan *plan, const WsPtrs &w, const uint32_t *base)
{
    const rick_params &p = plan->p;
    TileArgs t;
    t.n = p.n;
    t.n_w = p.n_w;
    t.T = p.tile;
    t.nt = p.n / p.tile;
    t.W = p.support;
    t.ntiles = (uint32_t)p.n_w * t.nt * t.nt;
    t.offsets = w.offsets;
    t.base = base;
    t.perm = w.perm;
    t.rcell = w.rcell;
    t.rec = w.rec;
    t.hdr = w.hdr;
    t.kp = plan->poly;
    return t;
}

static int ilog2(int x)
{
    int l = 0;
    while ((1 << l) < x) ++l;
    return l;
}

// One wave of persistent CTAs: SMs x resident CTAs per SM.
template <typename K>
static unsigned persistent_blocks(K kernel, size_t smem, int num_sms)
{
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 256, smem) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    return (unsigned)(per_sm * num_sms);
}

template <int W, int MODE>
static cudaError_t launch_grid_t(const GridArgs &a, int num_sms, cudaStream_t st)
{
    // float words: two T (T + 1) arrays; compensated six; 64-bit sums four
    const int words = MODE == GM_COMP ? 6 : MODE == GM_DET ? 4 : 2;
    size_t smem = words * (size_t)a.t.T * (a.t.T + 1) * sizeof(float);
    cudaFuncSetAttribute(grid_kernel<W, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    grid_kernel<W, MODE><<<persistent_blocks(grid_kernel<W, MODE>, smem, num_sms), 32 * RICK_GRID_WARPS,
                              smem, st>>>(a);
    return cudaGetLastError();
}

template <int W>
static cudaError_t launch_grid(const GridArgs &a, int mode, int num_sms, cudaStream_t st)
{
    return mode == GM_COMP ? launch_grid_t<W, GM_COMP>(a, num_sms, st)
         : mode == GM_DET  ? launch_grid_t<W, GM_DET>(a, num_sms, st)
                           : launch_grid_t<W, GM_PLAIN>(a, num_sms, st);
}

template <int W>
static cudaError_t launch_degrid(const DegridArgs &a, int num_sms, cudaStream_t st)
{
    size_t S = a.t.T + W - 1;
    size_t smem = S * S * sizeof(float2);
    cudaFuncSetAttribute(degrid_kernel<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    degrid_kernel<W><<<persistent_blocks(degrid_kernel<W>, smem, num_sms), 256, smem, st>>>(a);
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

rick_status rick_grid_impl(rick_plan *plan, void *ws_dev, void *planes_dev, int mode,
                           void *stream, const uint8_t *touched)
{
    const int accumulate = mode == RICK_GRID_ACCUMULATE;
    if (!plan || !ws_dev || !planes_dev) return RICK_EINVAL;
    if (plan->sticky != RICK_OK) return plan->sticky;
    if (((uintptr_t)ws_dev & 255) || ((uintptr_t)planes_dev & 15)) return RICK_EINVAL;
    const rick_params &p = plan->p;
    WsPtrs w = rick_ws_ptrs(ws_dev, rick_ws_layout(&p, plan->max_vis));
    cudaStream_t st = (cudaStream_t)stream;
    GridArgs a;
    a.t = make_tile_args(plan, w, w.gbase);
    a.planes = (float2 *)planes_dev;
    a.log2T = ilog2(p.tile);
    a.accumulate = accumulate;
    a.touched = mode == RICK_GRID_CHUNK_TILES ? touched : NULL;
    a.nzero = mode != RICK_GRID_OVERWRITE ? 0u
                                          : (a.t.ntiles + RICK_ZERO_GROUP - 1) / RICK_ZERO_GROUP;
    cudaError_t err = cudaSuccess;
    const bool det = (p.options & RICK_OPT_DETERMINISTIC) != 0;
    if (det && mode == RICK_GRID_CHUNK_TILES) return RICK_EINVAL;  // its slots add per tile
    a.mcslot = det ? w.mcslot : NULL;
    a.mcacc = det ? w.mcacc : NULL;
    zero_tiles_kernel<<<(accumulate && !det) ? 1 : plan->num_sms * 8, 256, 0, st>>>(
        w.gbase, a.t.ntiles, a.t.nt, a.log2T, p.n, a.planes, w.hdr, accumulate, a.mcslot,
        a.mcacc, a.touched);
    RICK_LAUNCH_CHECK(plan);
    const int gmode = det ? GM_DET : p.precision == RICK_PREC_FP32_COMPENSATED ? GM_COMP : GM_PLAIN;
#define CALL_GRID(WW) err = launch_grid<WW>(a, gmode, plan->num_sms, st)
    RICK_W_SWITCH(p.support, CALL_GRID);
#undef CALL_GRID
    ++plan->launches;
    RICK_CUDA_TRY(plan, err);
    if (det) {
        det_mc_convert_kernel<<<plan->num_sms * 8, 256, 0, st>>>(
            w.gbase, a.t.ntiles, a.t.nt, a.log2T, p.n, a.planes, w.hdr, accumulate, a.mcslot,
            a.mcacc);
        RICK_LAUNCH_CHECK(plan);
    }
    return RICK_OK;
}

extern "C" rick_status rick_grid(rick_plan *plan, void *ws_dev, void *planes_dev, void *stream)
{
    return rick_grid_impl(plan, ws_dev, planes_dev, RICK_GRID_OVERWRITE, stream);
}

extern "C" rick_status rick_grid_sparse(rick_plan *plan, void *ws_dev, void *planes_dev, void *stream)
{
    return rick_grid_impl(plan, ws_dev, planes_dev, RICK_GRID_RECORD_TILES, stream);
}

extern "C" rick_status rick_grid_accumulate(rick_plan *plan, void *ws_dev, void *planes_dev,
                                            void *stream)
{
    return rick_grid_impl(plan, ws_dev, planes_dev, RICK_GRID_ACCUMULATE, stream);
}

template <int W>
static cudaError_t launch_grid_batch(const GridBatchArgs &ba, int num_sms, cudaStream_t st)
{
    const size_t smem = 2 * (size_t)ba.job[0].t.T * (ba.job[0].t.T + 1) * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(grid_batch_kernel<W>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    grid_batch_kernel<W><<<persistent_blocks(grid_batch_kernel<W>, smem, num_sms),
                           32 * RICK_GRID_WARPS, smem, st>>>(ba);
    return cudaGetLastError();
}

extern "C" rick_status rick_grid_sparse_batch(rick_plan *const *plans, void *const *ws_dev,
                                              void *const *planes_dev, int32_t n_jobs,
                                              void *stream)
{
    if (!plans || !ws_dev || !planes_dev) return RICK_EINVAL;
    if (n_jobs < 1 || n_jobs > RICK_GRID_BATCH_MAX) return RICK_ERANGE;
    for (int j = 0; j < n_jobs; ++j) {
        const rick_plan *pl = plans[j];
        if (!pl || !ws_dev[j] || !planes_dev[j]) return RICK_EINVAL;
        if (pl->sticky != RICK_OK) return pl->sticky;
        if (((uintptr_t)ws_dev[j] & 255) || ((uintptr_t)planes_dev[j] & 15)) return RICK_EINVAL;
        if (pl->p.support != plans[0]->p.support || pl->p.tile != plans[0]->p.tile ||
            pl->device != plans[0]->device || pl->p.precision != RICK_PREC_FP32 ||
            (pl->p.options & RICK_OPT_DETERMINISTIC))
            return RICK_EINVAL;
        for (int i = 0; i < j; ++i)  // each job needs its own workspace and planes
            if (ws_dev[i] == ws_dev[j] || planes_dev[i] == planes_dev[j]) return RICK_EINVAL;
    }
    rick_plan *p0 = plans[0];
    GridBatchArgs ba;
    memset(&ba, 0, sizeof(ba));
    ba.n_jobs = n_jobs;
    int tiles_max = 0;
    for (int j = 0; j < n_jobs; ++j) {
        const rick_params &p = plans[j]->p;
        WsPtrs w = rick_ws_ptrs(ws_dev[j], rick_ws_layout(&p, plans[j]->max_vis));
        GridArgs &a = ba.job[j];
        a.t = make_tile_args(plans[j], w, w.gbase);
        a.planes = (float2 *)planes_dev[j];
        a.log2T = ilog2(p.tile);
        a.accumulate = 0;
        a.touched = NULL;
        a.nzero = 0;
        a.mcslot = NULL;
        a.mcacc = NULL;
        tiles_max = max(tiles_max, (int)a.t.ntiles);
    }
    cudaStream_t st = (cudaStream_t)stream;
    const unsigned bx = (unsigned)max(1, min(p0->num_sms * 8 / n_jobs, (tiles_max + 7) / 8));
    zero_tiles_batch_kernel<<<dim3(bx, (unsigned)n_jobs), 256, 0, st>>>(ba);
    cudaError_t err = cudaGetLastError();
    if (err == cudaSuccess) {
#define CALL_GRID_BATCH(WW) err = launch_grid_batch<WW>(ba, p0->num_sms, st)
        RICK_W_SWITCH(p0->p.support, CALL_GRID_BATCH);
#undef CALL_GRID_BATCH
    }
    p0->launches += 2;
    if (err != cudaSuccess) {
        for (int j = 0; j < n_jobs; ++j) plans[j]->sticky = RICK_ECUDA;
        return RICK_ECUDA;
    }
    return RICK_OK;
}

extern "C" rick_status rick_degrid(rick_plan *plan, void *ws_dev, const void *planes_dev,
                                   const float *weight_dev, void *vis_out_dev, void *stream)
{
    if (!plan || !ws_dev || !planes_dev || !vis_out_dev) return RICK_EINVAL;
    if (plan->sticky != RICK_OK) return plan->sticky;
    if (((uintptr_t)ws_dev & 255) || ((uintptr_t)planes_dev & 15) || ((uintptr_t)vis_out_dev & 7) ||
        ((uintptr_t)weight_dev & 3))
        return RICK_EINVAL;
    const rick_params &p = plan->p;
    WsPtrs w = rick_ws_ptrs(ws_dev, rick_ws_layout(&p, plan->max_vis));
    cudaStream_t st = (cudaStream_t)stream;
    DegridArgs a;
    a.t = make_tile_args(plan, w, w.dbase);
    a.planes = (const float2 *)planes_dev;
    a.weight = weight_dev;
    a.vis_out = (float2 *)vis_out_dev;
    a.log2T = ilog2(p.tile);
    degrid_zero_dropped_kernel<<<plan->num_sms * 4, 256, 0, st>>>(w.hdr, w.key, a.vis_out);
    RICK_LAUNCH_CHECK(plan);
    cudaError_t err = cudaSuccess;
#define CALL_DEGRID(WW) err = launch_degrid<WW>(a, plan->num_sms, st)
    RICK_W_SWITCH(p.support, CALL_DEGRID);
#undef CALL_DEGRID
    ++plan->launches;
    RICK_CUDA_TRY(plan, err);
    return RICK_OK;
}

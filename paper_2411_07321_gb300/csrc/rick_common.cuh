// rick_common.cuh -- shared definitions of the sm_103a w-stacking library:
// plan and workspace layout, launch-argument structs, and the device helpers
// that several kernels use (coordinate split, double-single arithmetic, the
// gridding kernel G).
#pragma once

#include <cuda_runtime.h>
#include <cufft.h>
#include <stdint.h>
#include <string.h>

#include "../../include/rick.h"

#if defined(__CUDACC__)
#define RICK_HD __host__ __device__ __forceinline__
#else
#define RICK_HD inline
#endif

// ------------------------------------------------------------------------
// Gridding kernel weights.  For a visibility at fractional offset f the W
// weights are G((j - h) - f), j = 0..W-1.  Each segment j is a polynomial in
// s = 2 (f - fc) in [-1, 1) (fc = 0 for odd W, where f is in [-1/2, 1/2);
// fc = 1/2 for even W, f in [0, 1)), fitted at plan creation by Chebyshev
// interpolation of degree RICK_POLY_DEG in FP64 and evaluated by Horner's rule
// in FP32.  Degree 8 fits the Kaiser-Bessel kernels of W = 4..16 to 7e-8 of the
// peak or better (2e-9 for W = 7), below FP32 rounding of the sums; the
// Gaussians are smoother.  The coefficients travel in the kernel-argument
// (constant) space.

#define RICK_MAX_W 16
#define RICK_POLY_DEG 8
#define RICK_POLY_N (RICK_POLY_DEG + 1)

struct KernelPoly {
    float c[RICK_MAX_W][RICK_POLY_N];
    float fc;
};

#if defined(__CUDACC__)
// Weight of segment j at s = 2 (f - fc).
template <int W>
__device__ __forceinline__ float kernel_weight_one(const KernelPoly &kp, int j, float s)
{
    if (W == 1) return 1.0f;
    float y = kp.c[j][RICK_POLY_DEG];
#pragma unroll
    for (int k = RICK_POLY_DEG - 1; k >= 0; --k) y = __fmaf_rn(y, s, kp.c[j][k]);
    return y;
}

template <int W>
__device__ __forceinline__ void kernel_weights(const KernelPoly &kp, float f, float *g)
{
    if (W == 1) {
        g[0] = 1.0f;
        return;
    }
    const float s = 2.0f * (f - kp.fc);
#pragma unroll
    for (int j = 0; j < W; ++j) {
        float y = kp.c[j][RICK_POLY_DEG];
#pragma unroll
        for (int k = RICK_POLY_DEG - 1; k >= 0; --k) y = __fmaf_rn(y, s, kp.c[j][k]);
        g[j] = y;
    }
}
#endif

// ------------------------------------------------------------------------
// Plan

struct rick_plan {
    rick_params p;
    int64_t max_vis;
    int device;
    int num_sms;
    cufftHandle fft;
    size_t fft_bytes;
    void *fft_work;     // cuFFT work area (ours: stream-ordered allocation)
    cudaStream_t own;   // the plan's private stream for its own allocations
    float *taper_inv;  // device [n]: 1 / C(nu_p), nu_p = (p - n/2) / n
    float2 *twid;      // device: stage twiddle tables of the fused transform (or NULL)
    double beta, sigma, i0_beta;
    KernelPoly poly;   // kernel-weight polynomials (host copy, passed to kernels)
    rick_status sticky;
    unsigned long long launches;  // library kernels enqueued so far (cuFFT's not included)
    uint32_t wait_polls;          // poll limit of the key pass's bounded wait for its copies
    int32_t n_w_created;          // planes the plan was created for (its cuFFT batch)
    // streaming from host memory (created on first use): the copy stream and
    // its events -- start of a call, chunk copied into staging buffer b,
    // staging buffer b free again, uvw chunk resident, resident uvw area a
    // free again -- and the staging area of the last call with its parity and
    // the staging buffer its next chunk takes
    cudaStream_t copy;
    cudaEvent_t ev_start, ev_ready[RICK_STREAM_BUFS], ev_free[RICK_STREAM_BUFS], ev_uvw,
        ev_area_free[2];
    void *stage_prev;
    size_t stage_prev_bytes;
    int parity;
    int next_buf;
};

// ------------------------------------------------------------------------
// Workspace layout (caller-owned device buffer, 256-byte aligned pieces)

struct WsHeader {
    rick_bin_stats stats;               // the stats of the last rick_bin
    unsigned long long wmin_key, wmax_key;  // monotone keys of the w range
    unsigned long long n_vis;           // n_vis of the last rick_bin
    unsigned long long drop_uv, drop_w; // counters
    double dw;                          // plane width (0: one degenerate plane)
    uint32_t grid_total, degrid_total;  // work items of rick_grid / rick_degrid
    uint32_t chunk_cap;                 // records per work item (at most)
    uint32_t range_given;
    uint32_t n_key_blocks;
    uint32_t grid_next, degrid_next;    // work counters of the persistent tile kernels
    uint32_t zero_next;                 // counter of the grid kernel's tile-clearing items
    uint32_t fault;                     // a bounded device-side wait ran out (never expected)
    uint32_t mirror;                    // records i >= n_src mirror input i - n_src
    unsigned long long n_src;           // input visibilities of the last rick_bin
    // deterministic mode: tile sums in fixed point, value = integer * fx_inv
    float fx_scale, fx_inv;             // 2^k and 2^-k
    uint32_t mc_count;                  // tiles gridded by several work items
};

struct WsLayout {
    size_t header, key, rank, cell, frac, perm, rec, rcell, hist, suboff, offsets, gbase, dbase, scan,
        wpart, bkey, wplane, dkey, didx, dkey2, dcnt, vpart, mcslot, mcacc, total;
    int64_t n_vis, nbins, ntiles, nscan, nkeyblocks, ndetblocks;
};

// Key pass blocks: 1024 visibilities, staged in 28 KB of shared memory, so that
// six blocks fit an SM (the pass is bound by integer issue and needs the warps).
#define RICK_KEY_THREADS 256
#define RICK_KEY_ITEMS 4
// Each bin's histogram counter is split into RICK_BIN_SUBS sub-counters, chosen
// by the input's block of RICK_KEY_THREADS * RICK_KEY_ITEMS visibilities: the
// densest bins (the array core) then take their atomics on several addresses
// instead of one.  The value a counter held before an input's atomic is the
// input's rank within its (bin, sub-counter) range.
#define RICK_BIN_SUBS 8
// Polls of a bounded device-side wait before it gives up (and the drain wait
// of a block that gave up: its copies must land before its shared memory goes).
#define RICK_WAIT_POLLS RICK_WAIT_POLLS_DEFAULT

// Deterministic mode (RICK_OPT_DETERMINISTIC).  The records of each bin are
// put in input order by a stable radix sort of (key, input index) in passes of
// RICK_DET_DIGIT bits over blocks of RICK_DET_BLOCK records.  Tiles gridded by
// several work items add 64-bit fixed-point sums into one of at most
// RICK_DET_MAX_MC workspace slots of T x T (re, im) int64 pairs; the records
// per work item are raised so that no more tiles than that need a slot.
#define RICK_DET_DIGIT 8
#define RICK_DET_BLOCK 2048
#define RICK_DET_MAX_MC 16384
RICK_HD size_t rick_align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Temporary elements of the recursive exclusive scan of `n` elements.
static inline int64_t rick_scan_tmp(int64_t n)
{
    int64_t t = 0;
    while (n > 2048) {
        n = (n + 2047) / 2048;
        t += n + 1;
    }
    return t + 1;
}

// Records of a binning of n_vis visibilities: two per visibility with the
// Hermitian mirror (V at uvw and conj V at -uvw), else one.
RICK_HD int64_t rick_n_records(const rick_params *p, int64_t n_vis)
{
    return (p->options & RICK_OPT_HERMITIAN_MIRROR) ? 2 * n_vis : n_vis;
}

// Multi-work-item tiles of a deterministic binning of n_rec records need a
// slot each; at most RICK_DET_MAX_MC of them.
static inline int64_t rick_det_slots(const rick_params *p, int64_t n_rec)
{
    if (!(p->options & RICK_OPT_DETERMINISTIC)) return 0;
    // a tile with several work items holds more than 1024 record visits, and
    // a record is visited by at most four tiles
    const int64_t b = 4 * n_rec / 1024 + 1;
    return b < RICK_DET_MAX_MC ? b : RICK_DET_MAX_MC;
}

static inline WsLayout rick_ws_layout(const rick_params *p, int64_t n_vis_in)
{
    WsLayout L;
    int64_t nt = p->n / p->tile;
    const int64_t n_vis = rick_n_records(p, n_vis_in);
    const bool det = (p->options & RICK_OPT_DETERMINISTIC) != 0;
    L.n_vis = n_vis;
    L.ntiles = (int64_t)p->n_w * nt * nt;
    L.nbins = 4 * L.ntiles;
    L.nkeyblocks = (n_vis + RICK_KEY_THREADS * RICK_KEY_ITEMS - 1) / (RICK_KEY_THREADS * RICK_KEY_ITEMS);
    L.ndetblocks = det ? (n_vis + RICK_DET_BLOCK - 1) / RICK_DET_BLOCK : 0;
    L.nscan = rick_scan_tmp(RICK_BIN_SUBS * L.nbins + 1);
    if (det) {
        const int64_t d = rick_scan_tmp((1 << RICK_DET_DIGIT) * L.ndetblocks + 1);
        if (d > L.nscan) L.nscan = d;
    }
    int64_t nv = n_vis > 0 ? n_vis : 1;
    size_t o = 0;
    L.header = o; o += rick_align256(sizeof(WsHeader));
    L.key = o;    o += rick_align256(4 * (size_t)nv);
    L.rank = o;   o += rick_align256(4 * (size_t)nv);
    L.cell = o;   o += rick_align256(4 * (size_t)nv);
    L.frac = o;   o += rick_align256(8 * (size_t)nv);
    L.perm = o;   o += rick_align256(4 * (size_t)nv);
    // one record of padding: the gridding loop reads one record ahead
    L.rec = o;    o += rick_align256(16 * (size_t)(nv + 1));
    L.rcell = o;  o += rick_align256(4 * (size_t)(nv + 1));
    L.hist = o;   o += rick_align256(4 * (size_t)(RICK_BIN_SUBS * L.nbins + 1));
    L.suboff = o; o += rick_align256(4 * (size_t)(RICK_BIN_SUBS * L.nbins + 1));
    L.offsets = o; o += rick_align256(4 * (size_t)(L.nbins + 1));
    L.gbase = o;  o += rick_align256(4 * (size_t)(L.ntiles + 1));
    L.dbase = o;  o += rick_align256(4 * (size_t)(L.ntiles + 1));
    L.scan = o;   o += rick_align256(4 * (size_t)L.nscan);
    L.wpart = o;  o += rick_align256(8 * (size_t)(L.nkeyblocks + 1));
    L.bkey = o;   o += rick_align256(8 * (size_t)(p->n_w + 1));
    L.wplane = o; o += rick_align256(16 * (size_t)(p->n_w + 1));
    // deterministic mode only (empty otherwise): the radix sort's second
    // (key, index) buffer and digit counts, the value-bound partials of the
    // fixed-point scale, the slot of each multi-work-item tile and the slots
    const size_t dn = det ? (size_t)nv : 0;
    L.dkey = o;   o += rick_align256(4 * dn);
    L.didx = o;   o += rick_align256(4 * dn);
    L.dkey2 = o;  o += rick_align256(4 * dn);
    L.dcnt = o;   o += rick_align256(det ? 4 * (size_t)((1 << RICK_DET_DIGIT) * L.ndetblocks + 1) : 0);
    L.vpart = o;  o += rick_align256(det ? 8 * (size_t)(L.ndetblocks + 1) : 0);
    L.mcslot = o; o += rick_align256(det ? 4 * (size_t)(L.ntiles + 1) : 0);
    L.mcacc = o;  o += rick_align256(16 * (size_t)rick_det_slots(p, n_vis) * p->tile * p->tile);
    L.total = o;
    return L;
}

// Device pointers into a workspace.
struct WsPtrs {
    WsHeader *hdr;
    uint32_t *key, *rank, *cell, *perm, *rcell, *hist, *suboff, *offsets, *gbase, *dbase, *scan;
    float2 *frac;
    float4 *rec;  // per record: vis*weight (re, im), fractional offsets (fx, fy)
    double *wpart;
    unsigned long long *bkey;
    float4 *wplane;  // per plane: (w_k hi, w_k lo, w_k as float, 0)
    uint32_t *dkey, *didx, *dkey2, *dcnt, *mcslot;  // deterministic mode
    double *vpart;
    unsigned long long *mcacc;
};

static inline WsPtrs rick_ws_ptrs(void *ws, const WsLayout &L)
{
    char *b = (char *)ws;
    WsPtrs w;
    w.hdr = (WsHeader *)(b + L.header);
    w.key = (uint32_t *)(b + L.key);
    w.rank = (uint32_t *)(b + L.rank);
    w.cell = (uint32_t *)(b + L.cell);
    w.frac = (float2 *)(b + L.frac);
    w.perm = (uint32_t *)(b + L.perm);
    w.rec = (float4 *)(b + L.rec);
    w.rcell = (uint32_t *)(b + L.rcell);
    w.hist = (uint32_t *)(b + L.hist);
    w.suboff = (uint32_t *)(b + L.suboff);
    w.offsets = (uint32_t *)(b + L.offsets);
    w.gbase = (uint32_t *)(b + L.gbase);
    w.dbase = (uint32_t *)(b + L.dbase);
    w.scan = (uint32_t *)(b + L.scan);
    w.wpart = (double *)(b + L.wpart);
    w.bkey = (unsigned long long *)(b + L.bkey);
    w.wplane = (float4 *)(b + L.wplane);
    w.dkey = (uint32_t *)(b + L.dkey);
    w.didx = (uint32_t *)(b + L.didx);
    w.dkey2 = (uint32_t *)(b + L.dkey2);
    w.dcnt = (uint32_t *)(b + L.dcnt);
    w.vpart = (double *)(b + L.vpart);
    w.mcslot = (uint32_t *)(b + L.mcslot);
    w.mcacc = (unsigned long long *)(b + L.mcacc);
    return w;
}

// Records per work item of the tile kernels for a binning of n_vis
// visibilities: about 64 items per SM in total (16 per resident CTA: short
// items balance the skewed tiles of a centrally concentrated uv coverage), at
// least 1024.  Set by the binning in the workspace header, where the tile
// kernels read it.
static inline uint32_t rick_chunk_cap(int64_t n_vis, int num_sms)
{
    int64_t c = (n_vis + (int64_t)num_sms * 64 - 1) / ((int64_t)num_sms * 64);
    if (c < 1024) c = 1024;
    c = (c + 255) & ~(int64_t)255;
    if (c > (1 << 30)) c = 1 << 30;
    return (uint32_t)c;
}

// ------------------------------------------------------------------------
// Bit-level helpers (identical on host and device)

RICK_HD uint64_t rick_dbits(double x)
{
    uint64_t b;
    memcpy(&b, &x, 8);
    return b;
}

RICK_HD double rick_bitsd(uint64_t b)
{
    double x;
    memcpy(&x, &b, 8);
    return x;
}

// Order-preserving map of a double to an unsigned key (-0 is treated as +0):
// a <= b  <=>  key(a) <= key(b) for all non-NaN a, b.
RICK_HD uint64_t rick_dkey(double x)
{
    uint64_t b = rick_dbits(x);
    if (b == 0x8000000000000000ull) b = 0;
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

RICK_HD double rick_dunkey(uint64_t k)
{
    return rick_bitsd((k >> 63) ? (k & 0x7FFFFFFFFFFFFFFFull) : ~k);
}

RICK_HD int rick_clz64(uint64_t x)
{
#if defined(__CUDA_ARCH__)
    return __clzll((long long)x);
#else
    return __builtin_clzll(x);
#endif
}

// Round the exact value s * 2^-sh (|s| < 2^53, s != 0, 0 <= sh <= 60) to the
// nearest float, ties to even, with integer operations only.
//
// Device path: normalise |s| so that its top bit is bit 63, keep the upper 32
// bits with every lower bit ORed into their lowest bit (a sticky bit), and let
// the hardware round that 32-bit integer to float.  The kept integer has 32
// significant bits, so the rounding position is bit 8 and the round bit bit 7;
// folding the discarded bits into bit 0 changes neither, and keeps "exactly
// half way" and "above half way" apart -- the result is the correctly rounded
// value of s.  Scaling by the power of two 2^(32 - lz - sh) is exact.
RICK_HD float rick_scaled_int_to_float(int64_t s, int sh)
{
#if defined(__CUDA_ARCH__)
    {
        const uint64_t mag = s < 0 ? (uint64_t)(-s) : (uint64_t)s;
        const int lz = __clzll((long long)mag);
        const uint64_t norm = mag << lz;
        const uint32_t top = (uint32_t)(norm >> 32) | ((uint32_t)norm != 0u ? 1u : 0u);
        const float f = __uint2float_rn(top) * __int_as_float((32 - lz - sh + 127) << 23);
        return s < 0 ? -f : f;
    }
#endif

    uint32_t sign = s < 0 ? 0x80000000u : 0u;
    uint64_t mag = s < 0 ? (uint64_t)(-s) : (uint64_t)s;
    int lz = rick_clz64(mag);
    uint64_t norm = mag << lz;  // top bit at 63
    uint64_t hi = norm >> 40;   // 24 significant bits
    uint64_t rem = norm & 0xFFFFFFFFFFull, half = 1ull << 39;
    int e = 63 - lz - sh;       // value = (hi / 2^23) 2^e
    if (rem > half || (rem == half && (hi & 1))) {
        ++hi;
        if (hi == (1ull << 24)) {
            hi >>= 1;
            ++e;
        }
    }
    uint32_t bits = sign | ((uint32_t)(e + 127) << 23) | (uint32_t)(hi & 0x7FFFFFu);
    float f;
    memcpy(&f, &bits, 4);
    return f;
}

// -0.5 <= x < 1 (the first grid cell; x < 0 only with W odd).  Kept out of
// line so that its FP64 conversions stay on this rare path instead of being
// predicated into every call.
#if defined(__CUDACC__)
static __host__ __device__ __noinline__
#else
static inline
#endif
bool rick_footprint_first_cell(double x, bool odd, int32_t *c, float *f)
{
    uint64_t b = rick_dbits(x);
    if (b >> 63) {  // -0.5 <= x < 0: only W odd can have c = 0
        if (!odd) return false;
        *c = 0;
        *f = (float)x;
        return true;
    }
    *c = (odd && b >= 0x3FE0000000000000ull) ? 1 : 0;
    *f = (float)(x - (double)*c);
    return true;
}

// Footprint of one axis (see rick_bin in rick.h): from the FP64 grid
// coordinate x, the corner a and the offset x - c rounded to float.  Returns
// false when the footprint is not inside [0, n-1] or x is not finite.
// key_lo = rick_dkey(-0.5), key_hi = rick_dkey(n + 0.5).  Apart from the rare
// x < 1 case, only integer operations act on x.
RICK_HD bool rick_footprint(double x, int n, int W, uint64_t key_lo, uint64_t key_hi, int32_t *a,
                            float *fx)
{
    const bool odd = W & 1;
    const int h = odd ? (W - 1) / 2 : W / 2 - 1;
    uint64_t b = rick_dbits(x);
    int32_t c;
    float f;
#if defined(__CUDA_ARCH__)
    // Device path for the common case 1 <= x < n + 1/2 (n <= 2^15): the
    // integer part of x lies in the high word of its bit pattern, so the split
    // runs on 32-bit words.  The mantissa is mh 2^32 + lw with mh holding the
    // implicit one and k = 20 - e fraction bits; the fraction is
    // (fh 2^32 + lw) 2^-(k+32).
    const uint32_t hw = (uint32_t)(b >> 32), lw = (uint32_t)b;
    if (hw >= 0x3FF00000u && hw < 0x80000000u) {
        if (b >= (key_hi ^ 0x8000000000000000ull)) return false;  // x >= n + 1/2, inf, NaN
        const int k = 20 - ((int)(hw >> 20) - 1023);
        const uint32_t mh = (hw & 0xFFFFFu) | 0x100000u;
        uint32_t fh = mh & ((1u << k) - 1u), fo = lw;
        const uint32_t up = odd ? (fh >> (k - 1)) & 1u : 0u;
        c = (int32_t)((mh >> k) + up);
        if (up) {  // x - c = fraction - 1: magnitude 2^(k+32) - (fh 2^32 + lw)
            fh = (1u << k) - fh - (lw != 0u ? 1u : 0u);
            fo = 0u - lw;
        }
        if ((fh | fo) == 0u) {
            f = 0.0f;
        } else {
            // the top 32 bits of the normalised magnitude, lower bits folded
            // into a sticky bit, rounded by the hardware (see
            // rick_scaled_int_to_float), times 2^sc
            uint32_t top;
            int sc;
            if (fh != 0u) {
                const int lz = __clz((int)fh);
                top = __funnelshift_l(fo, fh, lz) | ((fo << lz) != 0u ? 1u : 0u);
                sc = -lz - k;
            } else {
                const int lz = __clz((int)fo);
                top = fo << lz;
                sc = -lz - k - 32;
            }
            f = __uint2float_rn(top) * __int_as_float((sc + 127) << 23);
            if (up) f = -f;
        }
    } else {
        const uint64_t kx = rick_dkey(x);
        if (kx < key_lo || kx >= key_hi) return false;
        if (!rick_footprint_first_cell(x, odd, &c, &f)) return false;  // -1/2 <= x < 1
    }
#else
    uint64_t kx = rick_dkey(x);
    if (kx < key_lo || kx >= key_hi) return false;
    if (b < 0x3FF0000000000000ull || (b >> 63)) {  // -0.5 <= x < 1: the first cell, rare
        if (!rick_footprint_first_cell(x, odd, &c, &f)) return false;
    } else {
        int e = (int)(b >> 52) - 1023;  // 0 <= e <= 15
        int sh = 52 - e;
        uint64_t m = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
        uint64_t fb = m & ((1ull << sh) - 1);
        int32_t fl = (int32_t)(m >> sh);
        int up = odd ? (int)((fb >> (sh - 1)) & 1) : 0;
        c = fl + up;
        int64_t s = up ? (int64_t)fb - (int64_t)(1ull << sh) : (int64_t)fb;
        f = s == 0 ? 0.0f : rick_scaled_int_to_float(s, sh);
    }
#endif
    int32_t a0 = c - h;
    if (a0 < 0 || a0 + W - 1 > n - 1) return false;
    *a = a0;
    *fx = f;
    return true;
}

// ------------------------------------------------------------------------
// Double-single ("float-float") arithmetic: a value is hi + lo with
// |lo| <= ulp(hi)/2.  Products use the exact FMA residual (Dekker/Knuth).

struct ff {
    float hi, lo;
};

RICK_HD ff ff_from_double(double x)
{
    ff r;
    r.hi = (float)x;
    r.lo = (float)(x - (double)r.hi);
    return r;
}

#if defined(__CUDACC__)
__device__ __forceinline__ ff ff_two_sum(float a, float b)
{
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

__device__ __forceinline__ ff ff_fast_two_sum(float a, float b)  // |a| >= |b|
{
    float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ ff ff_add(ff a, ff b)
{
    ff s = ff_two_sum(a.hi, b.hi);
    float e = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
    return ff_fast_two_sum(s.hi, e);
}

__device__ __forceinline__ ff ff_mul(ff a, ff b)
{
    float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e));
    return ff_fast_two_sum(p, e);
}

// i * d for an integer |i| < 2^24
__device__ __forceinline__ ff ff_mul_int(int i, ff d)
{
    float fi = (float)i;
    float p = __fmul_rn(fi, d.hi);
    float e = __fmaf_rn(fi, d.hi, -p);
    e = __fmaf_rn(fi, d.lo, e);
    return ff_fast_two_sum(p, e);
}

__device__ __forceinline__ ff ff_sqrt(ff a)  // a > 0
{
    float s = sqrtf(a.hi);
    float p = __fmul_rn(s, s);
    float e = __fmaf_rn(s, s, -p);
    float r = __fdiv_rn(__fadd_rn(__fsub_rn(__fsub_rn(a.hi, p), e), a.lo), __fmul_rn(2.0f, s));
    return ff_fast_two_sum(s, r);
}

__device__ __forceinline__ ff ff_div(ff a, ff b)
{
    float q1 = __fdiv_rn(a.hi, b.hi);
    ff qb = ff_mul({q1, 0.0f}, b);
    ff r = ff_add(a, {-qb.hi, -qb.lo});
    float q2 = __fdiv_rn(r.hi, b.hi);
    return ff_fast_two_sum(q1, q2);
}

// n - 1 = -(l^2 + m^2) / (1 + sqrt(1 - l^2 - m^2)) in double-single arithmetic.
__device__ __forceinline__ ff ff_nm1(ff l, ff m, ff *r2_out)
{
    ff r2 = ff_add(ff_mul(l, l), ff_mul(m, m));
    ff t = ff_add({1.0f, 0.0f}, {-r2.hi, -r2.lo});
    ff den = ff_add({1.0f, 0.0f}, ff_sqrt(t));
    ff q = ff_div(r2, den);
    *r2_out = r2;
    return {-q.hi, -q.lo};
}

// ------------------------------------------------------------------------
// Bulk (TMA) copies from global into shared memory, completed on an mbarrier

__device__ __forceinline__ uint32_t rick_smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// One-phase barrier for `count` arrivals, made visible to the async proxy.
__device__ __forceinline__ void rick_mbar_init(unsigned long long *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(rick_smem_addr(bar)), "r"(count)
                 : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Arrive once, announcing `bytes` of bulk copies that complete on the barrier.
__device__ __forceinline__ void rick_mbar_expect_tx(unsigned long long *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                     rick_smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

// Copy `bytes` (a multiple of 16; both addresses 16-byte aligned) from global to
// shared memory; completion is counted on `bar`.
__device__ __forceinline__ void rick_bulk_g2s(void *dst, const void *src, uint32_t bytes,
                                              unsigned long long *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(rick_smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(rick_smem_addr(bar))
        : "memory");
}

// Wait for phase `parity` of `bar`, polling at most `limit` times; false if it
// did not complete.
__device__ __forceinline__ bool rick_mbar_wait(unsigned long long *bar, uint32_t parity,
                                               uint32_t limit)
{
    for (uint32_t i = 0; i < limit; ++i) {
        uint32_t done;
        asm volatile(
            "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; "
            "selp.u32 %0, 1, 0, p; }"
            : "=r"(done)
            : "r"(rick_smem_addr(bar)), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// Fraction of a double-single phase in cycles: (hi - rint(hi)) + lo, in
// [-1/2 - |lo|, 1/2 + |lo|].  hi - rint(hi) is exact for |hi| < 2^23.
__device__ __forceinline__ float ff_frac(ff t)
{
    return __fadd_rn(__fsub_rn(t.hi, rintf(t.hi)), t.lo);
}
#endif

// ------------------------------------------------------------------------
// Error plumbing

#define RICK_CUDA_TRY(plan, expr)                                  \
    do {                                                           \
        cudaError_t e_ = (expr);                                   \
        if (e_ != cudaSuccess) {                                   \
            if (plan) (plan)->sticky = RICK_ECUDA;                 \
            return e_ == cudaErrorMemoryAllocation ? RICK_ENOMEM : RICK_ECUDA; \
        }                                                          \
    } while (0)

#define RICK_LAUNCH_CHECK(plan)                    \
    do {                                           \
        ++(plan)->launches;                        \
        RICK_CUDA_TRY(plan, cudaGetLastError());   \
    } while (0)

// Launch arguments shared by the tile kernels.
struct TileArgs {
    int n, n_w, T, nt, W;
    uint32_t ntiles;
    const uint32_t *offsets, *base, *perm, *rcell;
    const float4 *rec;
    WsHeader *hdr;
    KernelPoly kp;
};

// ------------------------------------------------------------------------
// Internal entry points shared by the translation units

// rick_bin; range_src (device, optional) supplies the w range in place of the
// plan's (a range found over a larger set by an earlier pass).
// With n_chan > 0, uvw holds rows of n_chan visibilities and the uvw of
// visibility i is uvw[i / n_chan] * chan_scale[i % n_chan] (multi-channel input).
rick_status rick_bin_impl(rick_plan *plan, int64_t n_vis, const double *uvw, const void *vis,
                          const float *weight, void *ws_dev, size_t ws_bytes,
                          rick_bin_stats *stats_dev, void *stream, const WsHeader *range_src,
                          int n_chan, const double *chan_scale, int n_corr);
// Min/max keys of the finite w of visibilities [0, n) folded into hdr->wmin_key / wmax_key.
void rick_launch_wrange(const rick_plan *plan, const double *uvw, int64_t n, WsHeader *hdr,
                        cudaStream_t st, int n_chan, const double *scale);
// rick_grid (RICK_GRID_OVERWRITE), rick_grid_accumulate (RICK_GRID_ACCUMULATE)
// or rick_grid_sparse (RICK_GRID_RECORD_TILES: only the tiles that records
// reach are written, the others keep whatever they held).  RICK_GRID_CHUNK_TILES
// (a chunk of a streamed set): as RICK_GRID_RECORD_TILES, except that a tile
// flagged in touched (byte per tile, set where an earlier chunk's records
// reached; NULL: none) is added to instead of overwritten.
#define RICK_GRID_OVERWRITE 0
#define RICK_GRID_ACCUMULATE 1
#define RICK_GRID_RECORD_TILES 2
#define RICK_GRID_CHUNK_TILES 3
rick_status rick_grid_impl(rick_plan *plan, void *ws_dev, void *planes_dev, int mode,
                           void *stream, const uint8_t *touched = NULL);
// The twiddle tables of the fused transform (rick_fft.cu), on the plan's own
// stream; nothing for sizes the fused transform does not cover.
bool rick_fft_tables(rick_plan *pl);
// Bytes of the fused transform's work buffer (0 where it does not cover n).
size_t rick_fft_work_bytes(const rick_params *p);
// Tiles the fused transform reads (mode 0: all; 1: this binning's; 2: add this
// binning's to those marked), kept in the work buffer.
rick_status rick_fft_tiles_impl(rick_plan *plan, const void *ws_dev, void *work_dev,
                                size_t work_bytes, int mode, cudaStream_t st);
// The fused inverse FFT + w-correction of the marked tiles.
rick_status rick_fft_wcorrect_impl(rick_plan *plan, const void *planes_dev, const void *ws_dev,
                                   void *work_dev, size_t work_bytes, float *image_dev,
                                   uint32_t flags, cudaStream_t st);

// rick_fft.cu -- the inverse 2D FFT of every w-plane (§2 step 3) fused with
// the w-correction, the plane sum and the taper correction (§2 step 4, Eq. 2).
// Only the uv-tiles that hold gridded records are read.
//
// The unnormalised inverse transform F[q][p] = sum_{j,i} g[j][i]
// e^{+2 pi i (i p + j q) / n} of each plane runs as two passes of 1D
// transforms:
//  1. rows: along u, for every row v of a tile-row in which some tile holds
//     records (a row of empty tiles transforms to zero and is skipped).  Tiles
//     without records are read as zeros, so the grid step need not clear them.
//     The transformed rows go out transposed, work[k][p][v], 1024/(n/16) rows
//     per CTA (4 at n = 4096) so that each 32-byte sector of the transposed
//     store comes from one CTA; at n = 8192 (two rows per CTA) columns are
//     stored in interleaved pairs, work[k][p/2][v][p%2], for the same reason.
//     Only the image's crop columns p are kept.
//  2. columns: along v, one transform per image column p and plane k, reading
//     only the touched tile-rows of work[k][p].  The CTA keeps its column's
//     pixels across the planes and sums them into the image as it goes: plane
//     k contributes Re(F_k e^{2 pi i w_k (n - 1)}), and with equally spaced
//     plane centres the phase of plane k is that of the block's first plane
//     times D^(k - k0), D = e^{2 pi i dw (n - 1)}; each block of 8 planes is
//     summed by Horner's rule (descending k) and turned by its first plane's
//     exact phase (double-single argument, sincospif).
//
// Each 1D transform of N = 2^LOGN points is a Stockham autosort FFT (the
// formulation of Govindaraju et al., SC 2008): N/16 threads with 16 points
// each, radix-16 butterflies in registers (a radix-2, -4 or -8 stage last when
// 16 does not divide; the butterflies' adds two-wide), stages exchanged
// through shared memory arrays padded by one word in 32.  Twiddles come from
// per-stage tables computed in FP64 at plan creation and rounded once, laid
// out so that a warp reads consecutive entries (they stay in L1; the plane
// data is read around it).
//
// The adjoint (w-spreading + forward FFT, for degridding) runs the same two
// passes in the opposite order on the same inverse transforms, by conjugation;
// it writes only the tiles that degridding reads (see the section below).
#include "rick_common.cuh"
#include "rick_wphase.cuh"

#define RICK_FFT_LOG_MIN 8
#define RICK_FFT_LOG_MAX 13

struct FftArgs {
    int n, n_w, nt, log2T;
    const float2 *planes;    // [n_w][n][n]
    float2 *planes_out;      // [n_w][n][n]: the adjoint's output (tiles with records)
    float2 *work;            // [n_w][m][n]: row transforms, transposed
    uint8_t *tflag;          // [n_w][nt][nt]: tile holds records (is read)
    uint8_t *trow;           // [n_w][nt]: tile-row holds records
    uint8_t *pflag;          // [n_w]: plane holds records
    ulonglong2 *pmask;       // [n_w]: bit ty = tile-row ty holds records (nt <= 128)
    ulonglong2 *tmask;       // [n_w][nt]: bit tx = tile tx of the tile-row holds records (nt <= 128)
    const float2 *tw;        // the plan's stage twiddle tables (twiddle_kernel)
    WcArgs wc;               // image geometry, flags, taper, plane centres, weight sum
};

// Shared arrays hold complex points as float2, one 8-byte access each: a warp's
// access is two half-warps of 16 points, conflict-free when the 16 fall in
// distinct 8-byte bank pairs (index mod 16).
//
// Staged rows (written out or gathered transposed): an XOR swizzle of the low
// four bits, which with a per-row rotation keeps both the row-wise and the
// column-wise accesses free of bank conflicts.
static __device__ __forceinline__ int swz(int a) { return a ^ ((a >> 4) & 15); }

// Exchange arrays: one point of padding per 16 (a + a/16) keeps the stages'
// access patterns free of bank conflicts and leaves every address a
// per-thread base plus a constant.
static __device__ __forceinline__ int pad16(int a) { return a + (a >> 4); }

static __device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// u + v and u - v, two-wide (packed) FP32
static __device__ __forceinline__ void bfly(float2 &u, float2 &v)
{
    const float2 s = __fadd2_rn(u, v);
    v = __ffma2_rn(v, make_float2(-1.0f, -1.0f), u);
    u = s;
}

// u + v e^{2 pi i e / 16} and u - v e^{2 pi i e / 16}, e = 0..7 (constant
// after unrolling)
static __device__ __forceinline__ void bfly16(float2 &u, float2 &v, int e)
{
    const float C1 = 0.923879532511286756f;  // cos(pi/8)
    const float S1 = 0.382683432365089772f;  // sin(pi/8)
    const float H = 0.707106781186547524f;   // sqrt(1/2)
    float2 r;
    switch (e) {
    case 0: bfly(u, v); return;
    case 4: {  // v i: scalar adds, no lane swap
        const float2 a = make_float2(u.x - v.y, u.y + v.x);
        v = make_float2(u.x + v.y, u.y - v.x);
        u = a;
        return;
    }
    case 2:    // v e^{i pi/4} = sqrt(1/2) (x - y, x + y): the scale rides on the packed FMAs
    case 6: {  // v e^{3 i pi/4} = sqrt(1/2) (-(x + y), x - y)
        const float2 d = e == 2 ? make_float2(v.x - v.y, v.x + v.y)
                                : make_float2(-v.x - v.y, v.x - v.y);
        v = __ffma2_rn(d, make_float2(-H, -H), u);
        u = __ffma2_rn(d, make_float2(H, H), u);
        return;
    }
    case 1: r = make_float2(v.x * C1 - v.y * S1, v.x * S1 + v.y * C1); break;
    case 3: r = make_float2(v.x * S1 - v.y * C1, v.x * C1 + v.y * S1); break;
    case 5: r = make_float2(-v.x * S1 - v.y * C1, v.x * C1 - v.y * S1); break;
    default: r = make_float2(-v.x * C1 - v.y * S1, v.x * S1 - v.y * C1); break;
    }
    v = r;
    bfly(u, v);
}

// Bit reversal of i < R (R a power of two).
__host__ __device__ constexpr int brev(int i, int R)
{
    int j = 0;
    for (int b = 1; b < R; b <<= 1, i >>= 1) j = (j << 1) | (i & 1);
    return j;
}

// One radix-2 level of the in-register DFT: butterflies of span LEN / 2.
template <int R, int LEN>
static __device__ __forceinline__ void dft_level(float2 *a)
{
#pragma unroll
    for (int i = 0; i < R; i += LEN) {
#pragma unroll
        for (int m = 0; m < LEN / 2; ++m) bfly16(a[i + m], a[i + m + LEN / 2], m * (16 / LEN));
    }
    if constexpr (LEN < R) dft_level<R, 2 * LEN>(a);
}

// In-register DFT of R points, A_m = sum_r a_r e^{+2 pi i r m / R}: radix-2
// decimation in time after a bit-reversal permutation (all indices constant).
template <int R>
static __device__ __forceinline__ void dft_inv(float2 *a)
{
#pragma unroll
    for (int i = 0; i < R; ++i) {
        const int j = brev(i, R);
        if (j > i) {
            const float2 t = a[i];
            a[i] = a[j];
            a[j] = t;
        }
    }
    if constexpr (R > 1) dft_level<R, 2>(a);
}

// The stages of an N-point transform: radix 16 while 16 divides what is left,
// then one radix-2, -4 or -8 stage.  Stage i after sub-transforms of NS points
// needs the twiddles e^{2 pi i r k / (NS R)}, r = 1..R-1, k < NS (none for the
// first stage), tabled per stage as [r - 1][k] so that the threads of a warp
// read consecutive entries.
__host__ __device__ constexpr int stage_radix(int N, int NS)
{
    return ((N / NS) % 16 == 0) ? 16 : N / NS;
}

__host__ __device__ constexpr int twiddle_entries(int N)
{
    int e = 0;
    for (int ns = 1; ns < N; ns *= stage_radix(N, ns))
        if (ns > 1) e += (stage_radix(N, ns) - 1) * ns;
    return e;
}

// One Stockham stage of radix R after sub-transforms of NS points.  x[s] holds
// element t + P s of the current array (P = N / 16 threads per transform);
// butterfly j = t + P b (b < 16 / R) takes elements j + r N/R, applies the
// twiddles e^{2 pi i r (j mod NS) / (NS R)} (table at OFF), and its outputs m
// go to (j - j mod NS) R + j mod NS + m NS.  After the last stage x[s] holds
// output t + P s.  cb is the transform's offset in the exchange arrays.
template <int N, int R, int NS, int OFF, bool LAST>
static __device__ __forceinline__ void fft_stage(float2 (&x)[16], int t, int cb, float2 *sx,
                                                 const float2 *__restrict__ tw)
{
    constexpr int P = N / 16, B = 16 / R;
    static_assert(P % 16 == 0 && (NS > 1 || R == 16), "exchange addressing assumes these");
#pragma unroll
    for (int b = 0; b < B; ++b) {
        const int j = t + P * b, k = j & (NS - 1);
        float2 y[R];
#pragma unroll
        for (int r = 0; r < R; ++r) y[r] = x[b + B * r];
        if constexpr (NS > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r) y[r] = cmul(y[r], __ldg(tw + OFF + (r - 1) * NS + k));
        }
        dft_inv<R>(y);
        if constexpr (LAST) {
#pragma unroll
            for (int m = 0; m < R; ++m) x[b + B * m] = y[m];
        } else {
            // outputs base + m NS: with NS >= 16 the padding of output m is that
            // of base plus m NS / 16; with NS = 1, base = R j and the R outputs
            // share the padding j R / 16 (R <= 16)
            const int base = (j - k) * R + k;
            float2 *dst = sx + cb + (NS >= 16 ? pad16(base) : base + (base >> 4));
#pragma unroll
            for (int m = 0; m < R; ++m) dst[m * (NS >= 16 ? NS + NS / 16 : 1)] = y[m];
        }
    }
    if constexpr (!LAST) {
        __syncthreads();
        // elements t + P s, P a multiple of 16: padding t / 16 + s P / 16
        const float2 *src = sx + cb + pad16(t);
#pragma unroll
        for (int s = 0; s < 16; ++s) {
            x[s] = src[s * (P + P / 16)];
        }
        __syncthreads();
    }
}

template <int N, int NS, int OFF>
static __device__ __forceinline__ void fft_stages(float2 (&x)[16], int t, int cb, float2 *sx,
                                                  const float2 *__restrict__ tw)
{
    constexpr int R = stage_radix(N, NS);
    constexpr bool LAST = (R == N / NS);
    fft_stage<N, R, NS, OFF, LAST>(x, t, cb, sx, tw);
    if constexpr (!LAST) fft_stages<N, NS * R, OFF + (NS > 1 ? (R - 1) * NS : 0)>(x, t, cb, sx, tw);
}

// The unnormalised inverse DFT of N points held as x[s] = element t + P s;
// on return x[s] = output t + P s.  Every thread of the CTA must call it.
// tw: the plan's stage twiddle tables.
template <int LOGN>
static __device__ __forceinline__ void fft_inv(float2 (&x)[16], int t, int cb, float2 *sx,
                                               const float2 *__restrict__ tw)
{
    fft_stages<(1 << LOGN), 1, 0>(x, t, cb, sx, tw);
}

// Tile masks of up to 128 tiles (x: bits 0..63, y: bits 64..127), for grids of
// at most RICK_FFT_MASK_TILES tiles a side; larger grids read byte flags.
#define RICK_FFT_MASK_TILES 128

static __device__ __forceinline__ bool mask_bit(const ulonglong2 &msk, int b)
{
    return ((b < 64 ? msk.x : msk.y) >> (b & 63)) & 1ull;
}

// x[s] = src[VS (t + P s)] where the tile of t + P s is set in msk, else 0
// (WIDE: up to 128 tiles; else up to 64, one word and no selection).
template <int P, bool WIDE, int VS = 1>
static __device__ __forceinline__ void load_masked(float2 (&x)[16], const float2 *src,
                                                   const ulonglong2 &msk, int t, int l2T)
{
#pragma unroll
    for (int s = 0; s < 16; ++s) {
        const int u = t + P * s;
        const bool on = WIDE ? mask_bit(msk, u >> l2T) : ((msk.x >> (u >> l2T)) & 1ull);
        x[s] = on ? __ldcg(src + VS * u) : make_float2(0.0f, 0.0f);
    }
}

// Selector of the 16 points t + P s (s < 16) of the threads of class c = t / T
// when P is a multiple of the tile side T: the points lie in tile-rows (or
// tiles) c + s S, S = P / T; bit s is set where that one holds records.
static __device__ __forceinline__ uint32_t class_sel(const ulonglong2 &msk, int c, int S)
{
    uint32_t sel = 0;
    for (int s = 0; s < 16; ++s) sel |= (uint32_t)mask_bit(msk, c + s * S) << s;
    return sel;
}

// x[s] = src[VS (t + P s)] where bit s of sel is set, else 0.
template <int P, int VS = 1>
static __device__ __forceinline__ void load_sel(float2 (&x)[16], const float2 *src, uint32_t sel,
                                                int t)
{
#pragma unroll
    for (int s = 0; s < 16; ++s)
        x[s] = ((sel >> s) & 1u) ? __ldcg(src + VS * (t + P * s)) : make_float2(0.0f, 0.0f);
}

// Classes of threads whose selectors are tabled per CTA (P / T for T >= 16).
#define RICK_FFT_SEL_CLASSES 32

// Layout of the row transforms in the work buffer, per plane k (plane stride
// m n; the image side m is even): transposed, column p's n values contiguous
// ([p][v]); or, where a row-pass block holds only two rows (n = 8192), in
// interleaved column pairs ([p/2][v][p%2]), so that the block's write-out fills
// whole 32-byte sectors (two rows of two columns) and the column pass reads
// every second point.
template <int N>
struct WorkPairs {
    static constexpr bool ON = 1024 / (N / 16) < 4;
    static constexpr int VS = ON ? 2 : 1;  // element stride of a column
};

// Exchange array of one transform: N points plus the padding.
template <int N>
struct XLen {
    static constexpr int L = N + N / 16;
};

// Tiles to read: a tile holds records iff it has gridding work items.
// mode 0: every tile; 1: the tiles of this binning; 2: add this binning's
// tiles to those already marked (planes gridded over several binnings).
__global__ void __launch_bounds__(256) fft_tiles_kernel(uint8_t *tflag, const uint32_t *gbase,
                                                        uint32_t ntiles, int mode)
{
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntiles) return;
    const uint8_t has = mode == 0 || gbase[t + 1] != gbase[t];
    tflag[t] = mode == 2 ? (uint8_t)(tflag[t] | has) : has;
}

// Tile-rows and planes with a tile to read: one block per plane.
__global__ void __launch_bounds__(256) fft_rowflags_kernel(FftArgs a)
{
    const int k = blockIdx.x, nt = a.nt;
    const uint8_t *tf = a.tflag + (size_t)k * nt * nt;
    __shared__ unsigned long long s_mask[2];
    if (threadIdx.x < 2) s_mask[threadIdx.x] = 0;
    __syncthreads();
    int any_plane = 0;
    for (int ty = threadIdx.x; ty < nt; ty += blockDim.x) {
        uint8_t any = 0;
        unsigned long long tm[2] = {0, 0};
        for (int x = 0; x < nt; ++x) {
            const uint8_t f = tf[ty * nt + x];
            any |= f;
            if (x < RICK_FFT_MASK_TILES && f) tm[x >> 6] |= 1ull << (x & 63);
        }
        a.trow[k * nt + ty] = any;
        a.tmask[k * nt + ty] = make_ulonglong2(tm[0], tm[1]);
        any_plane |= any;
        if (any && ty < RICK_FFT_MASK_TILES) atomicOr(&s_mask[ty >> 6], 1ull << (ty & 63));
    }
    any_plane = __syncthreads_or(any_plane);
    if (threadIdx.x == 0) {
        a.pflag[k] = (uint8_t)(any_plane != 0);
        a.pmask[k] = make_ulonglong2(s_mask[0], s_mask[1]);
    }
}

// Pass 1: ROWS = 1024 / P rows per CTA, transformed in two batches by 512
// threads (a thread's 16 points and twiddles then stay in registers), staged in
// shared memory and written out transposed.  Persistent over (plane, block of
// ROWS rows); blocks whose tile-rows hold no records are skipped.
template <int LOGN>
__global__ void __launch_bounds__(512, 1) fft_rows_kernel(FftArgs a)
{
    constexpr int N = 1 << LOGN, P = N / 16, ROWS = 1024 / P, RPR = 512 / P;
    constexpr int ROT = ROWS >= 16 ? 1 : 16 / ROWS;
    constexpr int L = XLen<N>::L;
    extern __shared__ float2 sx[];  // exchange arrays (row stride L); staging at row stride N
    __shared__ uint8_t s_tf[1024];  // tile flags of the block's tile-rows
    __shared__ uint16_t s_rsel[8][RICK_FFT_SEL_CLASSES];  // selectors per tile-row and class
    const int t = threadIdx.x % P;
    const int nt = a.nt, l2T = a.log2T, m = a.wc.m, off = a.wc.off;
    // selectors from the tile masks when P is a multiple of the tile side
    // and the masks take two words (one word is tested as cheaply in place)
    const int ncls = P >> l2T;
    const bool tabled = nt > 64 && nt <= RICK_FFT_MASK_TILES && ncls >= 1 &&
                        ncls <= RICK_FFT_SEL_CLASSES && ROWS <= 8 << l2T;
    const int nvb = N / ROWS, items = a.n_w * nvb;
    for (int item = blockIdx.x; item < items; item += gridDim.x) {
        const int k = item / nvb, v0 = (item - k * nvb) * ROWS;
        const int ty0 = v0 >> l2T, ty1 = (v0 + ROWS - 1) >> l2T;
        bool any = false;
        for (int ty = ty0; ty <= ty1; ++ty) any |= a.trow[k * nt + ty] != 0;
        if (!any) continue;  // the same for every thread
        __syncthreads();     // the previous block's write-out has read the staging rows
        const int ntr = ty1 - ty0 + 1;
        if (nt > RICK_FFT_MASK_TILES) {
            const uint8_t *tfg = a.tflag + ((size_t)k * nt + ty0) * nt;
            for (int i = threadIdx.x; i < ntr * nt; i += blockDim.x) s_tf[i] = tfg[i];
        } else if (tabled && threadIdx.x < ntr * ncls) {
            const int r = threadIdx.x / ncls, c = threadIdx.x - r * ncls;
            s_rsel[r][c] = (uint16_t)class_sel(a.tmask[k * nt + ty0 + r], c, ncls);
        }
        __syncthreads();
#pragma unroll 1
        for (int h = 0; h < 2; ++h) {
            // the rows of batch h use their own exchange areas; the staged rows
            // of batch 0 are not touched by batch 1
            const int c = threadIdx.x / P + h * RPR, v = v0 + c;
            const float2 *row = a.planes + ((size_t)k * N + v) * N;
            float2 x[16];
            if (tabled) {
                load_sel<P>(x, row, s_rsel[(v >> l2T) - ty0][t >> l2T], t);
            } else if (nt <= 64) {  // the row's tiles as a bit mask
                load_masked<P, false>(x, row, a.tmask[k * nt + (v >> l2T)], t, l2T);
            } else if (nt <= RICK_FFT_MASK_TILES) {
                load_masked<P, true>(x, row, a.tmask[k * nt + (v >> l2T)], t, l2T);
            } else {
                const uint8_t *tf = s_tf + ((v >> l2T) - ty0) * nt;
#pragma unroll
                for (int s = 0; s < 16; ++s) {
                    const int u = t + P * s;
                    x[s] = tf[u >> l2T] ? __ldcg(row + u) : make_float2(0.0f, 0.0f);
                }
            }
            fft_inv<LOGN>(x, t, c * L, sx, a.tw);
            // stage the row (row stride N: the staged rows of batch 0 lie below
            // the exchange arrays of batch 1), XOR-swizzled and rotated per row
            // so that the transposed read-out is free of bank conflicts too
#pragma unroll
            for (int s = 0; s < 16; ++s) sx[swz(c * N + t + P * s) ^ ((c * ROT) & 15)] = x[s];
        }
        __syncthreads();
        // lanes take consecutive rows of consecutive columns, so that each warp
        // store fills whole 32-byte sectors (ROWS x 8 bytes of a column)
        if constexpr (WorkPairs<N>::ON) {
            // column pairs: lanes take the two rows of two columns (a 32-byte
            // sector) in order
            float2 *dst = a.work + (size_t)k * m * N + 2 * v0;
            for (int i = threadIdx.x; i < ROWS * m; i += blockDim.x) {
                const int e = i % (2 * ROWS), cp = i / (2 * ROWS);
                const int r = e >> 1, pc = 2 * cp + (e & 1);
                dst[(size_t)cp * 2 * N + e] = sx[swz(r * N + pc + off) ^ ((r * ROT) & 15)];
            }
        } else {
            // lanes take consecutive rows of consecutive columns, so that each
            // warp store fills whole 32-byte sectors (ROWS x 8 bytes of a column)
            float2 *dst = a.work + (size_t)k * m * N + v0;
            for (int i = threadIdx.x; i < ROWS * m; i += blockDim.x) {
                const int r = i % ROWS, pc = i / ROWS;
                dst[(size_t)pc * N + r] = sx[swz(r * N + pc + off) ^ ((r * ROT) & 15)];
            }
        }
    }
}

// Pass 2 and the w-correction: NT threads, COLS = NT / P image columns per
// CTA, each column transformed for every plane.  Per pixel the CTA keeps in
// shared memory n - 1 (double-single with the low word in 16 bits; plain FP32
// for the FP32-phase ablation) and the running plane sum; the output scale
// (taper, n factor, weight sum, checkerboard) is formed at the end, and the
// Horner sum of the current block of planes and the step D stay in registers.
// The plane data is read around L1 (it streams), so the twiddle tables stay
// there: the shared arrays are kept small enough (148 KB per SM at n = 8192,
// and for the two CTAs per SM below) that the SM's unified L1 / shared memory
// leaves 92 KB of L1, which holds the largest transform's 65 KB of tables.
template <int LOGN>
struct ColShape {
    static constexpr int N = 1 << LOGN, P = N / 16;
    static constexpr int NT = P < 256 ? 256 : P, COLS = NT / P, NE = NT * 16;
    static constexpr int XE = COLS * XLen<N>::L;  // points of the exchange arrays
    static constexpr size_t SMEM = sizeof(float2) * XE + sizeof(float) * 2 * NE +
                                   sizeof(__half) * NE;
};

template <int LOGN>
__global__ void __launch_bounds__(ColShape<LOGN>::NT, ColShape<LOGN>::NT <= 256 ? 2 : 1)
    fft_cols_kernel(FftArgs a)
{
    using S = ColShape<LOGN>;
    constexpr int N = S::N, P = S::P, NT = S::NT, COLS = S::COLS, NE = S::NE;
    constexpr int XE = S::XE;
    extern __shared__ float fsm[];
    float2 *sx = (float2 *)fsm;
    float *g_hi = fsm + 2 * XE, *g_acc = g_hi + NE;
    __half *g_lo = (__half *)(g_acc + NE);
    const WcArgs &w = a.wc;
    const int c = threadIdx.x / P, t = threadIdx.x % P, cb = c * XLen<N>::L;
    const int m = w.m, off = w.off, nt = a.nt, l2T = a.log2T;
    const int pc = blockIdx.x * COLS + c;  // image column
    const bool live = pc < m;
    const int p = (live ? pc : 0) + off;
    const bool fp32ph = (w.flags & RICK_PHASE_FP32) != 0;
    const bool imag = (w.flags & RICK_IMAG_PART) != 0;  // Im of the plane sum instead of Re
    float inv_sumw;
    {
        const double sw = w.hdr->stats.sum_weight;  // nothing gridded: no normalisation
        inv_sumw = sw != 0.0 ? (float)(1.0 / sw) : 1.0f;
    }
    const float4 dwp = __ldg(&w.wplane[w.n_w]);
    float2 D[16];
#pragma unroll
    for (int s = 0; s < 16; ++s) {
        const int q = t + P * s, gi = s * NT + threadIdx.x;
        D[s] = make_float2(1.0f, 0.0f);
        if (live && q >= off && q < off + m) {
            const PixelGeom g = pixel_geom(w, p, q, inv_sumw);
            g_hi[gi] = fp32ph ? g.nm1_f : g.nm1.hi;
            g_lo[gi] = fp32ph ? __float2half_rn(0.0f) : nm1_lo_encode(g.nm1);
            if (!fp32ph) {
                const float fd = ff_frac(ff_mul(ff{dwp.x, dwp.y}, g.nm1));
                sincospif(2.0f * fd, &D[s].y, &D[s].x);
            }
        } else {
            g_hi[gi] = 0.0f;
            g_lo[gi] = __float2half_rn(0.0f);
        }
        g_acc[gi] = 0.0f;
    }
    const int bs = fp32ph ? 1 : RICK_PHASE_ANCHOR;
    constexpr int VS = WorkPairs<N>::VS;
    const int pl = live ? pc : 0;
    const float2 *col = a.work + (VS == 2 ? (size_t)(pl >> 1) * 2 * N + (pl & 1) : (size_t)pl * N);
    // selectors of the block's planes per thread class (P a multiple of the
    // tile side), tabled at the start of each block of planes
    __shared__ uint16_t s_sel[RICK_PHASE_ANCHOR][RICK_FFT_SEL_CLASSES];
    const int ncls = P >> l2T;
    const bool tabled = nt <= RICK_FFT_MASK_TILES && ncls >= 1 && ncls <= RICK_FFT_SEL_CLASSES;
    for (int k0 = 0; k0 < w.n_w; k0 += bs) {
        const int k1 = min(k0 + bs, w.n_w);
        if (tabled) {
            // the previous block's reads of the table precede the barriers of
            // its transforms
            for (int i = threadIdx.x; i < (k1 - k0) * ncls; i += NT) {
                const int r = i / ncls, c = i - r * ncls;
                s_sel[r][c] = (uint16_t)class_sel(a.pmask[k0 + r], c, ncls);
            }
            __syncthreads();
        }
        float2 h[16];
#pragma unroll
        for (int s = 0; s < 16; ++s) h[s] = make_float2(0.0f, 0.0f);
        for (int k = k1 - 1; k >= k0; --k) {
            if (!a.pflag[k]) {  // an empty plane adds nothing: h = h D
#pragma unroll
                for (int s = 0; s < 16; ++s) h[s] = cmul(h[s], D[s]);
                continue;
            }
            const float2 *src = col + (size_t)k * m * N;
            float2 x[16];
            if (tabled) {
                load_sel<P, VS>(x, src, live ? (uint32_t)s_sel[k - k0][t >> l2T] : 0u, t);
            } else if (nt <= RICK_FFT_MASK_TILES) {  // the plane's tile-rows as a bit mask
                const ulonglong2 msk = live ? a.pmask[k] : make_ulonglong2(0ull, 0ull);
                if (nt <= 64) load_masked<P, false, VS>(x, src, msk, t, l2T);
                else load_masked<P, true, VS>(x, src, msk, t, l2T);
            } else {
                const uint8_t *tr = a.trow + k * nt;
#pragma unroll
                for (int s = 0; s < 16; ++s) {
                    const int v = t + P * s;
                    x[s] = (live && tr[v >> l2T]) ? __ldcg(src + VS * v) : make_float2(0.0f, 0.0f);
                }
            }
            fft_inv<LOGN>(x, t, cb, sx, a.tw);
#pragma unroll
            for (int s = 0; s < 16; ++s) {
                const float2 hd = cmul(h[s], D[s]);
                h[s] = make_float2(hd.x + x[s].x, hd.y + x[s].y);
            }
        }
        // the block's sum times the exact phase of its first plane
        const float4 wk = __ldg(&w.wplane[k0]);
#pragma unroll
        for (int s = 0; s < 16; ++s) {
            const int gi = s * NT + threadIdx.x;
            PixelGeom g;
            const float hi = g_hi[gi];
            g.nm1 = ff{hi, nm1_lo_decode(hi, g_lo[gi])};
            g.nm1_f = hi;
            float cs, sn;
            wphase(w, wk, g, &cs, &sn);
            g_acc[gi] = imag ? fmaf(h[s].x, sn, fmaf(h[s].y, cs, g_acc[gi]))
                             : fmaf(h[s].x, cs, fmaf(-h[s].y, sn, g_acc[gi]));
        }
    }
    if (!live) return;
#pragma unroll
    for (int s = 0; s < 16; ++s) {
        const int q = t + P * s, gi = s * NT + threadIdx.x;
        // n = 1 + (n - 1) to FP32 rounding
        if (q >= off && q < off + m)
            w.image_out[(size_t)(q - off) * m + pc] =
                g_acc[gi] * pixel_scale(w, p, q, 1.0f + g_hi[gi], inv_sumw);
    }
}

// ------------------------------------------------------------------------
// The adjoint: w-spreading (the transpose of the w-correction) fused with the
// forward FFT of every plane, for the tiles that records reach (the only cells
// degridding reads).  Plane k of the adjoint is the forward 2D DFT of
// G_k[q][p] = image[q][p] s(p, q) e^{-2 pi i w_k (n - 1)} (s with the
// checkerboard sign; zero outside the crop).  A forward DFT is the conjugate of
// the inverse DFT of the conjugate, so both passes reuse the inverse
// transforms:
//  A. per image column p and plane k: z_k[p][v] = sum_q conj(G_k[q][p])
//     e^{+2 pi i v q / n}, conj(G) = image s e^{+2 pi i w_k (n - 1)} (the phase
//     walked by the step D with exact anchors every 8 planes, as in the plane-sum
//     kernels), stored transposed for the tile-rows with records;
//  B. per row v of those tile-rows: planes[k][v][u] = conj(sum_p z_k[p][v]
//     e^{+2 pi i u p / n}) for the tiles with records.

template <int LOGN>
struct AdjColShape {
    static constexpr int N = 1 << LOGN, P = N / 16;
    static constexpr int NT = P < 256 ? 256 : P, COLS = NT / P, NE = NT * 16;
    static constexpr int XE = COLS * XLen<N>::L;  // points of the exchange arrays
    static constexpr size_t SMEM = sizeof(float2) * XE + sizeof(float) * 2 * NE +
                                   sizeof(__half) * NE;
};

template <int LOGN>
__global__ void __launch_bounds__(AdjColShape<LOGN>::NT, AdjColShape<LOGN>::NT <= 256 ? 2 : 1)
    fft_cols_adj_kernel(FftArgs a)
{
    using S = AdjColShape<LOGN>;
    constexpr int N = S::N, P = S::P, NT = S::NT, COLS = S::COLS, NE = S::NE, XE = S::XE;
    extern __shared__ float fsm[];
    float2 *sx = (float2 *)fsm;
    float *g_hi = fsm + 2 * XE, *g_a = g_hi + NE;
    __half *g_lo = (__half *)(g_a + NE);
    const WcArgs &w = a.wc;
    const int c = threadIdx.x / P, t = threadIdx.x % P, cb = c * XLen<N>::L;
    const int m = w.m, off = w.off, nt = a.nt, l2T = a.log2T;
    const int pc = blockIdx.x * COLS + c;  // image column
    const bool live = pc < m;
    const int p = (live ? pc : 0) + off;
    const bool fp32ph = (w.flags & RICK_PHASE_FP32) != 0;
    float inv_sumw;
    {
        const double sw = w.hdr->stats.sum_weight;  // nothing gridded: no normalisation
        inv_sumw = sw != 0.0 ? (float)(1.0 / sw) : 1.0f;
    }
    const float4 dwp = __ldg(&w.wplane[w.n_w]);
    float2 D[16], ph[16];
#pragma unroll
    for (int s = 0; s < 16; ++s) {
        const int q = t + P * s, gi = s * NT + threadIdx.x;
        D[s] = make_float2(1.0f, 0.0f);
        ph[s] = make_float2(1.0f, 0.0f);
        if (live && q >= off && q < off + m) {
            const PixelGeom g = pixel_geom(w, p, q, inv_sumw);
            g_hi[gi] = fp32ph ? g.nm1_f : g.nm1.hi;
            g_lo[gi] = fp32ph ? __float2half_rn(0.0f) : nm1_lo_encode(g.nm1);
            g_a[gi] = w.image_in[(size_t)(q - off) * m + pc] * g.scale;
            if (!fp32ph) {
                const float fd = ff_frac(ff_mul(ff{dwp.x, dwp.y}, g.nm1));
                sincospif(2.0f * fd, &D[s].y, &D[s].x);
            }
        } else {
            g_hi[gi] = g_a[gi] = 0.0f;
            g_lo[gi] = __float2half_rn(0.0f);
        }
    }
    const int bs = fp32ph ? 1 : RICK_PHASE_ANCHOR;
    float2 *dst = a.work + (size_t)(live ? pc : 0) * N;
    for (int k = 0; k < w.n_w; ++k) {
        if (k % bs == 0) {  // exact phase of the anchor plane
            const float4 wk = __ldg(&w.wplane[k]);
#pragma unroll
            for (int s = 0; s < 16; ++s) {
                const int gi = s * NT + threadIdx.x;
                PixelGeom g;
                const float hi = g_hi[gi];
                g.nm1 = ff{hi, nm1_lo_decode(hi, g_lo[gi])};
                g.nm1_f = hi;
                wphase(w, wk, g, &ph[s].x, &ph[s].y);
            }
        } else {
#pragma unroll
            for (int s = 0; s < 16; ++s) ph[s] = cmul(ph[s], D[s]);
        }
        if (!a.pflag[k]) continue;  // degridding reads nothing of this plane
        float2 x[16];
#pragma unroll
        for (int s = 0; s < 16; ++s) {
            const float av = g_a[s * NT + threadIdx.x];
            x[s] = make_float2(av * ph[s].x, av * ph[s].y);
        }
        fft_inv<LOGN>(x, t, cb, sx, a.tw);
        if (!live) continue;
        float2 *col = dst + (size_t)k * m * N;
        if (nt <= RICK_FFT_MASK_TILES) {
            const ulonglong2 msk = a.pmask[k];
#pragma unroll
            for (int s = 0; s < 16; ++s) {
                const int v = t + P * s;
                if (mask_bit(msk, v >> l2T)) __stcg(col + v, x[s]);
            }
        } else {
            const uint8_t *tr = a.trow + k * nt;
#pragma unroll
            for (int s = 0; s < 16; ++s) {
                const int v = t + P * s;
                if (tr[v >> l2T]) __stcg(col + v, x[s]);
            }
        }
    }
}

// Pass B: ROWS = 1024 / P rows per CTA gathered from the transposed pass-A
// output (lanes take consecutive rows of consecutive columns: whole 32-byte
// sectors), staged in shared memory, transformed in two batches by 512 threads
// (exchange arrays after the staged rows), conjugated and written to the
// tiles with records.  Persistent over (plane, block of ROWS rows).
template <int LOGN>
__global__ void __launch_bounds__(512, 1) fft_rows_adj_kernel(FftArgs a)
{
    constexpr int N = 1 << LOGN, P = N / 16, ROWS = 1024 / P, RPR = 512 / P;
    constexpr int ROT = ROWS >= 16 ? 1 : 16 / ROWS;
    constexpr int L = XLen<N>::L;
    extern __shared__ float2 gx[];   // staged rows (row stride N)
    float2 *xx = gx + ROWS * N;      // exchange arrays (row stride L)
    __shared__ uint8_t s_tf[1024];
    const int t = threadIdx.x % P;
    const int nt = a.nt, l2T = a.log2T, m = a.wc.m, off = a.wc.off;
    const int nvb = N / ROWS, items = a.n_w * nvb;
    for (int item = blockIdx.x; item < items; item += gridDim.x) {
        const int k = item / nvb, v0 = (item - k * nvb) * ROWS;
        const int ty0 = v0 >> l2T, ty1 = (v0 + ROWS - 1) >> l2T;
        bool any = false;
        for (int ty = ty0; ty <= ty1; ++ty) any |= a.trow[k * nt + ty] != 0;
        if (!any) continue;  // the same for every thread
        __syncthreads();     // the previous block is done with the staged rows
        const int ntr = ty1 - ty0 + 1;
        if (nt > RICK_FFT_MASK_TILES) {
            const uint8_t *tfg = a.tflag + ((size_t)k * nt + ty0) * nt;
            for (int i = threadIdx.x; i < ntr * nt; i += blockDim.x) s_tf[i] = tfg[i];
        }
        // gather: rows v0 .. v0 + ROWS - 1 of the crop columns (pass A wrote only
        // the tile-rows with records); zeros elsewhere
        const float2 *src = a.work + (size_t)k * m * N + v0;
        for (int i = threadIdx.x; i < ROWS * N; i += blockDim.x) {
            const int r = i % ROWS, p = i / ROWS, pc = p - off;
            const float2 z = (pc >= 0 && pc < m && a.trow[k * nt + ((v0 + r) >> l2T)])
                                 ? __ldcg(src + (size_t)pc * N + r) : make_float2(0.0f, 0.0f);
            gx[swz(r * N + p) ^ ((r * ROT) & 15)] = z;
        }
        __syncthreads();
#pragma unroll 1
        for (int h = 0; h < 2; ++h) {
            const int c = threadIdx.x / P + h * RPR, v = v0 + c;
            float2 x[16];
#pragma unroll
            for (int s = 0; s < 16; ++s) {
                x[s] = gx[swz(c * N + t + P * s) ^ ((c * ROT) & 15)];
            }
            fft_inv<LOGN>(x, t, (threadIdx.x / P) * L, xx, a.tw);
            float2 *row = a.planes_out + ((size_t)k * N + v) * N;
            if (nt <= RICK_FFT_MASK_TILES) {
                const ulonglong2 msk = a.tmask[k * nt + (v >> l2T)];
#pragma unroll
                for (int s = 0; s < 16; ++s) {
                    const int u = t + P * s;
                    if (mask_bit(msk, u >> l2T)) row[u] = make_float2(x[s].x, -x[s].y);
                }
            } else {
                const uint8_t *tf = s_tf + ((v >> l2T) - ty0) * nt;
#pragma unroll
                for (int s = 0; s < 16; ++s) {
                    const int u = t + P * s;
                    if (tf[u >> l2T]) row[u] = make_float2(x[s].x, -x[s].y);
                }
            }
        }
    }
}

// ------------------------------------------------------------------------
// Host side

static bool fft_supported(const rick_params &p)
{
    return p.n >= (1 << RICK_FFT_LOG_MIN) && p.n <= (1 << RICK_FFT_LOG_MAX);
}

struct FftWorkLayout {
    size_t tflag, trow, pflag, pmask, tmask, work, total;
};

static FftWorkLayout fft_work_layout(const rick_params &p)
{
    const size_t nt = p.n / p.tile, m = p.image_n ? p.image_n : p.n;
    FftWorkLayout L;
    size_t o = 0;
    L.tflag = o; o += rick_align256((size_t)p.n_w * nt * nt);
    L.trow = o;  o += rick_align256((size_t)p.n_w * nt);
    L.pflag = o; o += rick_align256((size_t)p.n_w);
    L.pmask = o; o += rick_align256(sizeof(ulonglong2) * (size_t)p.n_w);
    L.tmask = o; o += rick_align256(sizeof(ulonglong2) * (size_t)p.n_w * nt);
    L.work = o;  o += (size_t)p.n_w * m * p.n * sizeof(float2);
    L.total = o;
    return L;
}

size_t rick_fft_work_bytes(const rick_params *p)
{
    return fft_supported(*p) ? fft_work_layout(*p).total : 0;
}

// The stage twiddle tables of an n-point transform: entry OFF_i + (r - 1) NS + k
// of stage i = e^{2 pi i r k / (NS R)}, in FP64, rounded once.
__global__ void twiddle_kernel(float2 *tw, int n, int entries)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= entries) return;
    int off = 0;
    for (int ns = 1; ns < n; ns *= stage_radix(n, ns)) {
        if (ns == 1) continue;
        const int R = stage_radix(n, ns), cnt = (R - 1) * ns;
        if (e < off + cnt) {
            const int r = (e - off) / ns + 1, k = (e - off) % ns;
            double s, c;
            sincospi(2.0 * r * k / ((double)ns * R), &s, &c);
            tw[e] = make_float2((float)c, (float)s);
            return;
        }
        off += cnt;
    }
}

// The plan's twiddle tables (plans whose n the fused transform covers), on the
// plan's own stream.
bool rick_fft_tables(rick_plan *pl)
{
    if (!fft_supported(pl->p)) return true;
    const int n = pl->p.n, entries = twiddle_entries(n);
    if (cudaMallocAsync((void **)&pl->twid, sizeof(float2) * entries, pl->own) != cudaSuccess)
        return false;
    twiddle_kernel<<<(entries + 255) / 256, 256, 0, pl->own>>>(pl->twid, n, entries);
    ++pl->launches;
    return cudaGetLastError() == cudaSuccess;
}

// Shared memory of a transform kernel and the unified L1 / shared-memory split
// it prefers: 70 % of the SM's 228 KB for shared memory (the 164 KB
// configuration), which holds the resident CTAs of the column passes and of the
// imaging row pass (at most 154 KB per SM) and leaves 92 KB of L1 for the
// twiddle tables.
#define RICK_FFT_SMEM_CARVEOUT 70

template <typename K>
static cudaError_t fft_smem_attrs(K kernel, size_t smem)
{
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                RICK_FFT_SMEM_CARVEOUT);
}

template <int LOGN>
static cudaError_t launch_fft_wc(const FftArgs &a, int num_sms, cudaStream_t st)
{
    using S = ColShape<LOGN>;
    const size_t rows_smem = sizeof(float2) * (1024 / S::P) * XLen<(1 << LOGN)>::L;
    cudaError_t e = fft_smem_attrs(fft_rows_kernel<LOGN>, rows_smem);
    if (e != cudaSuccess) return e;
    e = fft_smem_attrs(fft_cols_kernel<LOGN>, S::SMEM);
    if (e != cudaSuccess) return e;
    const int items = a.n_w * (a.n / (1024 / S::P));
    fft_rows_kernel<LOGN><<<(unsigned)min(items, num_sms), 512, rows_smem, st>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int m = a.wc.m;
    fft_cols_kernel<LOGN><<<(unsigned)((m + S::COLS - 1) / S::COLS), S::NT, S::SMEM, st>>>(a);
    return cudaGetLastError();
}

static bool fft_args_ok(const rick_plan *plan, const void *ws_dev, const void *work_dev,
                        size_t work_bytes)
{
    return fft_supported(plan->p) && plan->twid && !((uintptr_t)ws_dev & 255) &&
           !((uintptr_t)work_dev & 255) && work_bytes >= fft_work_layout(plan->p).total;
}

// Kernel arguments of the fused transforms (the planes and image set by the caller).
static FftArgs fft_args(rick_plan *plan, const void *ws_dev, void *work_dev, uint32_t flags)
{
    const rick_params &p = plan->p;
    const FftWorkLayout L = fft_work_layout(p);
    FftArgs a;
    a.n = p.n;
    a.n_w = p.n_w;
    a.nt = p.n / p.tile;
    a.log2T = 0;
    while ((1 << a.log2T) < p.tile) ++a.log2T;
    a.planes = NULL;
    a.planes_out = NULL;
    char *wb = (char *)work_dev;
    a.tflag = (uint8_t *)(wb + L.tflag);
    a.trow = (uint8_t *)(wb + L.trow);
    a.pflag = (uint8_t *)(wb + L.pflag);
    a.pmask = (ulonglong2 *)(wb + L.pmask);
    a.tmask = (ulonglong2 *)(wb + L.tmask);
    a.work = (float2 *)(wb + L.work);
    a.tw = plan->twid;
    a.wc = make_args(plan, ws_dev, flags);
    return a;
}

rick_status rick_fft_tiles_impl(rick_plan *plan, const void *ws_dev, void *work_dev,
                                size_t work_bytes, int mode, cudaStream_t st)
{
    if (!fft_args_ok(plan, ws_dev, work_dev, work_bytes)) return RICK_EINVAL;
    const rick_params &p = plan->p;
    const FftWorkLayout L = fft_work_layout(p);
    WsPtrs wp = rick_ws_ptrs((void *)ws_dev, rick_ws_layout(&p, plan->max_vis));
    const uint32_t nt = p.n / p.tile, ntiles = (uint32_t)p.n_w * nt * nt;
    fft_tiles_kernel<<<(ntiles + 255) / 256, 256, 0, st>>>((uint8_t *)work_dev + L.tflag,
                                                           wp.gbase, ntiles, mode);
    RICK_LAUNCH_CHECK(plan);
    return RICK_OK;
}

rick_status rick_fft_wcorrect_impl(rick_plan *plan, const void *planes_dev, const void *ws_dev,
                                   void *work_dev, size_t work_bytes, float *image_dev,
                                   uint32_t flags, cudaStream_t st)
{
    if (!fft_args_ok(plan, ws_dev, work_dev, work_bytes) || !valid_flags(flags) ||
        ((uintptr_t)planes_dev & 7) || ((uintptr_t)image_dev & 3))
        return RICK_EINVAL;
    const rick_params &p = plan->p;
    FftArgs a = fft_args(plan, ws_dev, work_dev, flags);
    a.planes = (const float2 *)planes_dev;
    a.wc.image_out = image_dev;
    fft_rowflags_kernel<<<p.n_w, 256, 0, st>>>(a);
    RICK_LAUNCH_CHECK(plan);
    cudaError_t err = cudaErrorInvalidValue;
    switch (p.n) {
    case 256: err = launch_fft_wc<8>(a, plan->num_sms, st); break;
    case 512: err = launch_fft_wc<9>(a, plan->num_sms, st); break;
    case 1024: err = launch_fft_wc<10>(a, plan->num_sms, st); break;
    case 2048: err = launch_fft_wc<11>(a, plan->num_sms, st); break;
    case 4096: err = launch_fft_wc<12>(a, plan->num_sms, st); break;
    case 8192: err = launch_fft_wc<13>(a, plan->num_sms, st); break;
    }
    plan->launches += 2;
    RICK_CUDA_TRY(plan, err);
    return RICK_OK;
}

template <int LOGN>
static cudaError_t launch_wspread_fft(const FftArgs &a, int num_sms, cudaStream_t st)
{
    using S = AdjColShape<LOGN>;
    constexpr int N = 1 << LOGN, P = N / 16, ROWS = 1024 / P, RPR = 512 / P;
    const size_t rows_smem = sizeof(float2) * (ROWS * N + RPR * XLen<N>::L);
    cudaError_t e = fft_smem_attrs(fft_cols_adj_kernel<LOGN>, S::SMEM);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(fft_rows_adj_kernel<LOGN>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rows_smem);
    if (e != cudaSuccess) return e;
    const int m = a.wc.m;
    fft_cols_adj_kernel<LOGN><<<(unsigned)((m + S::COLS - 1) / S::COLS), S::NT, S::SMEM, st>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int items = a.n_w * (N / ROWS);
    fft_rows_adj_kernel<LOGN><<<(unsigned)min(items, num_sms), 512, rows_smem, st>>>(a);
    return cudaGetLastError();
}

extern "C" rick_status rick_wspread_fft(rick_plan *plan, const float *image_dev,
                                        const void *ws_dev, void *work_dev, size_t work_bytes,
                                        void *planes_dev, uint32_t flags, void *stream)
{
    if (!plan || !image_dev || !ws_dev || !work_dev || !planes_dev || !valid_flags(flags, true))
        return RICK_EINVAL;
    if (plan->sticky != RICK_OK) return plan->sticky;
    if (!fft_args_ok(plan, ws_dev, work_dev, work_bytes) || ((uintptr_t)planes_dev & 7) ||
        ((uintptr_t)image_dev & 3))
        return RICK_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    rick_status s = rick_fft_tiles_impl(plan, ws_dev, work_dev, work_bytes, 1, st);
    if (s != RICK_OK) return s;
    const rick_params &p = plan->p;
    FftArgs a = fft_args(plan, ws_dev, work_dev, flags);
    a.wc.image_in = image_dev;
    a.planes_out = (float2 *)planes_dev;
    fft_rowflags_kernel<<<p.n_w, 256, 0, st>>>(a);
    RICK_LAUNCH_CHECK(plan);
    cudaError_t err = cudaErrorInvalidValue;
    switch (p.n) {
    case 256: err = launch_wspread_fft<8>(a, plan->num_sms, st); break;
    case 512: err = launch_wspread_fft<9>(a, plan->num_sms, st); break;
    case 1024: err = launch_wspread_fft<10>(a, plan->num_sms, st); break;
    case 2048: err = launch_wspread_fft<11>(a, plan->num_sms, st); break;
    case 4096: err = launch_wspread_fft<12>(a, plan->num_sms, st); break;
    case 8192: err = launch_wspread_fft<13>(a, plan->num_sms, st); break;
    }
    plan->launches += 2;
    RICK_CUDA_TRY(plan, err);
    return RICK_OK;
}

extern "C" rick_status rick_fft_wcorrect_bytes(const rick_plan *plan, size_t *work_bytes)
{
    if (!plan || !work_bytes) return RICK_EINVAL;
    if (!fft_supported(plan->p)) return RICK_EINVAL;
    *work_bytes = fft_work_layout(plan->p).total;
    return RICK_OK;
}

extern "C" rick_status rick_fft_wcorrect(rick_plan *plan, const void *planes_dev,
                                         const void *ws_dev, int32_t sparse, void *work_dev,
                                         size_t work_bytes, float *image_dev, uint32_t flags,
                                         void *stream)
{
    if (!plan || !planes_dev || !ws_dev || !work_dev || !image_dev || !valid_flags(flags))
        return RICK_EINVAL;
    if (plan->sticky != RICK_OK) return plan->sticky;
    if (!fft_args_ok(plan, ws_dev, work_dev, work_bytes) || ((uintptr_t)planes_dev & 7) ||
        ((uintptr_t)image_dev & 3))
        return RICK_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    rick_status s = rick_fft_tiles_impl(plan, ws_dev, work_dev, work_bytes, sparse ? 1 : 0, st);
    if (s != RICK_OK) return s;
    return rick_fft_wcorrect_impl(plan, planes_dev, ws_dev, work_dev, work_bytes, image_dev, flags,
                                  st);
}

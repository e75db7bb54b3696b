/*
 * rick.h -- C ABI of the GB300 (sm_103a) w-stacking imaging library.
 *
 * The library implements the w-stacking gridder of De Rubeis et al.,
 * "Accelerating radio astronomy imaging with RICK" (§2): visibilities are
 * binned, convolved onto a (u, v, w) mesh with a Gaussian or Kaiser-Bessel
 * kernel (Eq. 3; each visibility goes to the closest w-plane), each w-plane is
 * inverse Fourier transformed, and the planes are phase-corrected and summed
 * into the image (Eq. 2, §2 step 4).  Degridding is the exact adjoint.
 *
 * Conventions (all calls):
 *  - uvw are in wavelengths (§2, Eq. 1), float64, row-major [n_vis][3].
 *  - Visibilities are complex64 stored as interleaved (re, im) float32 pairs.
 *  - Grid cell i <-> u = (i - n/2) / fov; image pixel p <-> l = (p - n/2) fov / n.
 *  - Planes are complex64 [n_w][n][n], row-major (v row, u fastest); after the
 *    inverse FFT the same buffer holds [n_w][m row q][l column p].
 *  - The image is float32 [m][m], m = image_n (n unless the grid is padded),
 *    row q (m) major, column p (l) fastest; its pixel (p', q') is the grid-frame
 *    pixel (p' + (n - m)/2, q' + (n - m)/2).
 *  - Pointers named *_dev are device pointers, *_host host pointers.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Every call that takes a stream only enqueues work on it and returns;
 *    results are ready when the stream reaches that point.
 *  - The caller owns every buffer passed in.  A plan owns only its cuFFT plan
 *    and a few small tables; it allocates them in rick_plan_create.
 *  - No call throws; every call returns a rick_status.  Arguments are checked on
 *    the host before anything is enqueued.  A CUDA or cuFFT error seen by a call
 *    is returned by that call and kept in the plan (rick_plan_last_error) so
 *    that later calls on the same plan return it too (sticky).
 *  - A plan may be used from one host thread at a time.
 */
#ifndef RICK_H
#define RICK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t rick_status;
#define RICK_OK 0
#define RICK_EINVAL (-1)  /* invalid argument (checked before any launch)   */
#define RICK_ENOMEM (-2)  /* device allocation failed                       */
#define RICK_ECUDA (-3)   /* a CUDA runtime call or kernel launch failed    */
#define RICK_ECUFFT (-4)  /* a cuFFT call failed                            */
#define RICK_ERANGE (-5)  /* a size exceeds the plan's or workspace capacity */

#define RICK_KERNEL_GAUSS 0 /* G(d) = exp(-d^2 / (2 sigma^2)), |d| <= W/2              */
#define RICK_KERNEL_KB 1    /* G(d) = I0(beta sqrt(1 - (2d/W)^2)) / I0(beta) (Jackson 1991) */

#define RICK_PREC_FP32 0             /* FP32 shared-memory tile accumulation          */
#define RICK_PREC_FP32_COMPENSATED 1 /* FP32 sub-chunk sums folded with Neumaier's     */
                                     /* compensated summation per tile cell          */

/* Pixel scaling of rick_wcorrect_stack / rick_wspread (bit-or):               */
#define RICK_N_CORRECT 1u /* multiply by n = sqrt(1 - l^2 - m^2) (Eq. 2 left side)      */
#define RICK_NORMALIZE 2u /* divide by the sum of the binned weights                    */
#define RICK_N_DIVIDE 4u  /* divide by n (the 1/n of Eq. 1, for prediction)             */
#define RICK_PHASE_FP32 8u /* ablation: w-phase argument in plain FP32 instead of       */
                           /* double-single (~48-bit) arithmetic                         */
#define RICK_IMAG_PART 16u /* write Im of the plane sum instead of Re (imaging calls    */
                           /* only): a check that Hermitian data give a real image      */

/* Options of a plan (rick_params.options, bit-or): */
#define RICK_OPT_HERMITIAN_MIRROR 1 /* grid every visibility twice: V at (u, v, w) and    */
                                    /* conj(V) at (-u, -v, -w), the sky being real (§2:  */
                                    /* the image is the real part); with the w range     */
                                    /* from the data it is then -max|w| ... max|w|       */
#define RICK_OPT_DETERMINISTIC 2    /* bitwise repeatable binning and gridding: records  */
                                    /* of a bin in input order, tile sums in 64-bit      */
                                    /* fixed point (no floating-point atomics)           */

/* Imaging-weight schemes of rick_density_weights. */
#define RICK_WEIGHT_UNIFORM 1 /* w / D                                           */
#define RICK_WEIGHT_BRIGGS 2  /* w / (1 + f^2 D), Briggs' robust weighting        */

typedef struct rick_params {
    int32_t n;          /* grid (mesh) side, power of two, 16 ... 32768                 */
    int32_t n_w;        /* number of w-planes, >= 1                                     */
    double fov;         /* image side in direction-cosine units (> 0); cell du = 1/fov */
    double w_min;       /* w range in wavelengths; both NaN: exact min/max over all    */
    double w_max;       /*   input w.  Given: visibilities outside it are dropped.     */
    int32_t kernel;     /* RICK_KERNEL_GAUSS or RICK_KERNEL_KB                          */
    int32_t support;    /* W, kernel support in cells, 1 ... 16 (W == 1: nearest cell)  */
    double kb_beta;     /* KB shape; NaN: pi sqrt((W/2)^2 1.5^2 - 0.8) (Beatty 2005)     */
    double gauss_sigma; /* Gaussian sigma in cells; NaN: W / 6                           */
    int32_t tile;       /* uv-tile side T: power of two, max(8, W) <= T <= min(128, n);  */
                        /*   T <= 64 with RICK_PREC_FP32_COMPENSATED                    */
    int32_t precision;  /* RICK_PREC_*                                                   */
    int32_t image_n;    /* side m of the image: the central m x m pixels of the n x n    */
                        /*   w-stacked image are kept (grid padding by n/m, which moves  */
                        /*   the aliases of the kept field onto the kernel's stopband);  */
                        /*   pixel p' of the image is pixel p' + (n - m)/2 of the grid   */
                        /*   frame, so the pixel size stays fov/n and the phase centre   */
                        /*   is pixel m/2.  Even, 16 <= m <= n; 0 means m = n (no crop)  */
    int32_t options;    /* bit-or of RICK_OPT_* (0: none)                                */
} rick_params;

/* Geometry and counts of the last rick_bin, written to device memory. */
typedef struct rick_bin_stats {
    int64_t n_binned;     /* visibilities kept; -1 if a bounded device-side wait of    */
                          /*   the binning ran out (never expected; the binning is    */
                          /*   then incomplete and must not be used)                  */
    int64_t n_dropped_uv; /* footprint not inside the grid (or non-finite u, v)       */
    int64_t n_dropped_w;  /* w outside a given range                                  */
    double sum_weight;    /* sum of the kept visibilities' weights                    */
    double w_min, w_max;  /* the w range used                                         */
} rick_bin_stats;

typedef struct rick_plan rick_plan;

/* Text for a status code (static storage). */
const char *rick_status_string(rick_status s);

/* Create a plan for `params` on the current CUDA device: validates params,
 * creates the batched cuFFT plan (n_w transforms of n x n, complex64), and
 * precomputes the taper table and the kernel-weight fits.  max_vis bounds
 * n_vis in later calls.  Does not synchronise the device: the plan's own
 * allocations are stream-ordered on a private stream, and only that stream is
 * waited for, so work already running on other streams is not stalled.
 * Errors: RICK_EINVAL (bad params or max_vis < 0 or >= 2^31), RICK_ENOMEM,
 * RICK_ECUFFT, RICK_ECUDA.  *out is set only on success. */
rick_status rick_plan_create(const rick_params *params, int64_t max_vis, rick_plan **out);

/* Release a plan (NULL is accepted).  The caller must make sure that no work
 * enqueued with the plan is still pending (e.g. synchronise its streams); the
 * device as a whole is not synchronised. */
rick_status rick_plan_destroy(rick_plan *plan);

/* Sticky error of a plan (RICK_OK if none). */
rick_status rick_plan_last_error(const rick_plan *plan);

/* Change a plan's sky geometry -- fov and the w range (NaN, NaN: from the
 * data) -- without rebuilding it: the cuFFT plan, the taper table (which
 * depends only on n and the kernel) and the kernel-weight fits stay.  Lets a
 * resident plan serve jobs with different fields of view.  Host-only: calls
 * already enqueued keep the geometry they were enqueued with.  RICK_EINVAL if
 * the new geometry is invalid (the plan is then unchanged). */
rick_status rick_plan_set_geometry(rick_plan *plan, double fov, double w_min, double w_max);

/* Change a plan's gridding kernel -- kernel, support, kb_beta, gauss_sigma as
 * in rick_params -- without rebuilding it: the taper table and the
 * kernel-weight fits are recomputed (a few microseconds of device work on the
 * plan's own stream, waited for), the cuFFT plan stays.  Lets a resident plan
 * serve jobs with different kernels.  Work enqueued with the plan must be
 * complete (the taper table is rewritten).  RICK_EINVAL if the kernel is
 * invalid for the plan (e.g. support > tile); the plan is then unchanged. */
rick_status rick_plan_set_kernel(rick_plan *plan, int32_t kernel, int32_t support, double kb_beta,
                                 double gauss_sigma);

/* Change a plan's image side image_n (as in rick_params; 0: the grid side)
 * without rebuilding it: only the crop of the w-correction and its adjoint
 * change.  Host-only, like rick_plan_set_geometry.  RICK_EINVAL if invalid
 * (the plan is then unchanged). */
rick_status rick_plan_set_image_n(rick_plan *plan, int32_t image_n);

/* Change a plan's number of w-planes to n_w, at most the number it was
 * created with, without rebuilding it: lets a resident plan (and buffers sized
 * for its created count: rick_workspace_bytes, the planes, the fused work
 * buffer) serve jobs with fewer planes.  The later calls lay out the
 * workspace, planes and work buffer for n_w.  rick_fft_wplanes needs the
 * created count (its batched cuFFT plan transforms that many planes) and
 * returns RICK_EINVAL otherwise; the fused transform covers the rest.
 * Host-only, like rick_plan_set_geometry.  RICK_EINVAL if n_w is out of range
 * (the plan is then unchanged). */
rick_status rick_plan_set_planes(rick_plan *plan, int32_t n_w);

/* Kaiser-Bessel shape for a grid oversampling alpha = n / image_n (Beatty,
 * Nishimura & Pauly 2005): beta = pi sqrt((W/alpha)^2 (alpha - 1/2)^2 - 0.8),
 * which puts the first zero of the kernel's transform just beyond the first
 * alias of the image edge.  The default kb_beta (NaN) is this value for
 * alpha = 2.  Returns NaN if support < 2, alpha < 1 or the root's argument is
 * not positive. */
double rick_kb_beta(int32_t support, double alpha);

/* Poll limit of the binning's bounded device-side wait (the key pass waits on
 * an mbarrier for the bulk copies of its inputs into shared memory).  Past the
 * limit a block gives up: it leaves its inputs out, lets its copies land (a
 * second wait, always with the default limit) and returns, and the binning
 * reports n_binned = -1 (and must not be used).  The default,
 * RICK_WAIT_POLLS_DEFAULT, is far more than a copy ever needs; polls = 0 gives
 * up without polling, which makes the give-up path run, for testing it.  The
 * paper has no counterpart.  Host-only; affects calls enqueued afterwards.
 * RICK_EINVAL for a NULL plan. */
#define RICK_WAIT_POLLS_DEFAULT (1u << 24)
rick_status rick_plan_set_wait_limit(rick_plan *plan, uint32_t polls);

/* Number of library kernels this plan has enqueued since it was created
 * (cuFFT's kernels are not included), for launch accounting. */
rick_status rick_plan_launch_count(const rick_plan *plan, uint64_t *count);

/* Bytes of the binning workspace of a plan created with max_vis = n_vis
 * (bin_bytes; the workspace layout depends only on params and that capacity)
 * and of the planes buffer (plane_bytes = n_w n^2 8).  Either output may be
 * NULL.  rick_plan_fft_bytes gives the cuFFT work area a plan holds. */
rick_status rick_workspace_bytes(const rick_params *params, int64_t n_vis, size_t *bin_bytes,
                                 size_t *plane_bytes);
rick_status rick_plan_fft_bytes(const rick_plan *plan, size_t *fft_bytes);

/* Binning (§2, gridding sub-step 1: "an array ... for each slab", here per
 * (w-plane, uv-tile)).  For each visibility: grid coordinates
 * x = fma(u, fov, n/2), y = fma(v, fov, n/2) in FP64; centre cell
 * c = floor(x + 1/2) (odd W) or floor(x) (even W); footprint corner
 * a = c - h, h = (W-1)/2 (odd) or W/2 - 1 (even); dropped unless
 * 0 <= a and a + W - 1 <= n - 1 on both axes.  Closest w-plane (§2):
 * k = #{j = 1..n_w-1 : w >= fma(j, dw, w_min)}, dw = (w_max - w_min)/n_w
 * (k = 0 when dw == 0).  Each kept visibility becomes one record
 * {vis * weight, (x - c_x, y - c_y) as float32, corner (a_x, a_y)} stored in
 * bin order: key = ((k (n/T) + a_y/T) (n/T) + a_x/T) 4 + edge class
 * (0: footprint inside its tile, 1: reaches the east tile only, 2: east and
 * south, 3: south only).  Records of one bin are contiguous; their order
 * within a bin is unspecified.
 *   uvw_dev:    float64 [n_vis][3]
 *   vis_dev:    complex64 [n_vis] (interleaved float32 re, im)
 *   weight_dev: float32 [n_vis], or NULL for unit weights
 *   ws_dev:     workspace of rick_workspace_bytes(params, plan max_vis)
 *               bytes, 256-byte aligned; overwritten; the later calls of
 *               this binning (grid, wcorrect, wspread, degrid) read it
 *   stats_dev:  device rick_bin_stats, or NULL
 * uvw_dev and weight_dev aligned to 16 bytes let each block of the key pass
 * fetch its 1024 rows with one bulk (TMA) copy; 8-byte alignment is enough for
 * correctness.
 * Errors: RICK_EINVAL (NULL pointer, misalignment), RICK_ERANGE (n_vis >
 * max_vis or ws_bytes too small), RICK_ECUDA. */
rick_status rick_bin(rick_plan *plan, int64_t n_vis, const double *uvw_dev, const void *vis_dev,
                     const float *weight_dev, void *ws_dev, size_t ws_bytes,
                     rick_bin_stats *stats_dev, void *stream);

/* rick_bin for multi-channel input: visibilities in rows of
 * n_chan channels, as a measurement set stores them, with uvw given once per
 * row and a factor per channel -- the uvw of channel c of row r is
 * uvw_rows[r] * chan_scale[c], one FP64 product per coordinate (e.g. metres
 * times nu_c / c, or wavelengths at a reference frequency times nu_c / nu_0).
 * The result is exactly that of rick_bin on the expanded uvw
 * [n_rows n_chan][3]; the device reads 24 bytes of uvw per row instead of per
 * visibility.
 *   uvw_rows_dev:   float64 [n_rows][3]
 *   chan_scale_dev: float64 [n_chan]
 *   vis_dev, weight_dev: [n_rows][n_chan], channel fastest, as for rick_bin
 * Errors: as rick_bin; RICK_EINVAL for n_chan < 1; RICK_ERANGE if
 * n_rows n_chan > max_vis. */
rick_status rick_bin_channels(rick_plan *plan, int64_t n_rows, int32_t n_chan,
                              const double *uvw_rows_dev, const double *chan_scale_dev,
                              const void *vis_dev, const float *weight_dev, void *ws_dev,
                              size_t ws_bytes, rick_bin_stats *stats_dev, void *stream);

/* Correlations per visibility that rick_bin_rows / rick_image_host_rows take. */
#define RICK_MAX_CORR 4

/* rick_bin_channels for rows whose visibilities carry n_corr correlations (a
 * measurement set stores e.g. the XX and YY products of linear feeds; the
 * paper's LOFAR counts include two).  Each (row, channel) is gridded once, as
 * the weighted sum of its correlations: its record holds sum_c w_c V_c and its
 * weight is sum_c w_c, so the normalised image is the weighted mean of the
 * correlations (Stokes I for XX and YY) and equals, up to FP32 rounding, the
 * image of the set with each correlation as its own visibility at the same
 * uvw.  A correlation with weight 0 (flagged) drops out.
 *   vis_dev:    complex64 [n_rows][n_chan][n_corr], correlation fastest
 *   weight_dev: float32 [n_rows][n_chan][n_corr], or NULL: unit weight per
 *               correlation (a visibility then weighs n_corr)
 * The binning's visibilities are the (row, channel) pairs: rick_bin_values,
 * rick_degrid and rick_density_weights then take one value or weight per pair,
 * and the stats count pairs (sum_weight sums all correlation weights).
 * n_corr == 1 is rick_bin_channels.  Errors: as rick_bin_channels;
 * RICK_EINVAL for n_corr outside 1 ... RICK_MAX_CORR. */
rick_status rick_bin_rows(rick_plan *plan, int64_t n_rows, int32_t n_chan, int32_t n_corr,
                          const double *uvw_rows_dev, const double *chan_scale_dev,
                          const void *vis_dev, const float *weight_dev, void *ws_dev,
                          size_t ws_bytes, rick_bin_stats *stats_dev, void *stream);

/* Where the binning arrays sit inside a workspace (byte offsets from ws_dev),
 * for callers that read the binned records directly:
 *   offsets  uint32 [n_bins + 1]   bin b holds records [offsets[b], offsets[b+1])
 *   perm     uint32 [n_binned]     record r came from input visibility perm[r]
 *   rec      float32 [n_binned][4] (re, im) of vis * weight, x - c_x, y - c_y
 *   rec_cell uint32 [n_binned]     a_x | a_y << 16
 *   stats    rick_bin_stats        the last binning's stats
 * n_bins = 4 n_w (n/T)^2.  Host-only; enqueues nothing. */
typedef struct rick_bin_view {
    size_t offsets, perm, rec, rec_cell, stats;
    int64_t n_bins;
} rick_bin_view;
rick_status rick_bin_layout(const rick_plan *plan, rick_bin_view *out);

/* rick_bin for callers that cannot allocate device memory.  Some callers run
 * where allocation is not an option: a host program may hand a plug-in only
 * the buffers it owns, a real-time loop may forbid allocator calls (they can
 * block and synchronise the device), or memory may be carved up in advance
 * from a fixed budget.  This entry point computes exactly what rick_bin
 * computes and writes the same workspace regions that later calls read --
 * the header and stats, the per-visibility keys and corner cells (read by
 * rick_degrid and rick_density_weights), the records, the permutation, the
 * bin offsets and the work lists -- but keeps its temporaries (the
 * per-visibility ranks and fractional offsets, the histogram, the scan
 * temporaries and the weight-sum partials) in a fixed array compiled into the
 * library (about 11.6 MB, held on every GPU that loads the library until the
 * process exits) instead of in ws_dev's scratch regions.  It calls no
 * cudaMalloc, cudaFree or allocating library routine.
 * The paper has no counterpart; this is an interface convenience.
 *   Limits: n_vis <= 262144 and 4 n_w (n/T)^2 <= 131072 bins, else
 *   RICK_ERANGE.  Arguments as for rick_bin.
 *   The first call on a device looks up the array's device address (once per
 *   device, with that device current); make that first call before any stream
 *   capture.  Every call shares the one array: calls that overlap on the GPU
 *   (other streams, other threads, other plans) race and must be serialised. */
rick_status rick_bin_noalloc(rick_plan *plan, int64_t n_vis, const double *uvw_dev,
                             const void *vis_dev, const float *weight_dev, void *ws_dev,
                             size_t ws_bytes, rick_bin_stats *stats_dev, void *stream);

/* Replace the record values of an existing binning by vis * weight for new
 * visibilities at the same uvw (weight NULL: unit), and recompute the weight
 * sum.  Used to grid gradients through the same geometry. */
rick_status rick_bin_values(rick_plan *plan, const void *vis_dev, const float *weight_dev,
                            void *ws_dev, rick_bin_stats *stats_dev, void *stream);

/* Gridding (Eq. 3): planes[k][a_y + jy][a_x + jx] +=
 * vis w G(jx - h - fx) G(jy - h - fy) for every record, with the
 * checkerboard (-1)^(i+j) of the centred FFT folded in.  Every element of
 * planes_dev (complex64 [n_w][n][n]) is overwritten.  Each uv-tile is summed
 * in shared memory and written once (plain stores; tiles with more records
 * than one chunk add their chunk sums with float atomics).  The kernel
 * weights G are degree-8 polynomial fits per unit segment (FP64 fit at plan
 * creation, FP32 evaluation).  rick_grid and rick_degrid use a word of the
 * workspace header as a work counter: calls that share a workspace must not
 * overlap on the device. */
rick_status rick_grid(rick_plan *plan, void *ws_dev, void *planes_dev, void *stream);

/* rick_grid that adds into planes_dev instead of overwriting it: planes_dev
 * must already hold planes (a rick_grid result, or zeros) of the same plan
 * geometry and w range.  Gridding is linear in the records, so gridding the
 * chunks of a visibility set one after another -- rick_bin + rick_grid for
 * the first, rick_bin + rick_grid_accumulate for the rest, all binned with the
 * same w range -- gives the planes of the whole set (up to FP32 summation
 * order).  Tiles written by one work item are read, added to and written;
 * tiles of several work items add with float atomics. */
rick_status rick_grid_accumulate(rick_plan *plan, void *ws_dev, void *planes_dev, void *stream);

/* Per-plane 2D FFT (§2 step 3, §3.1): cuFFT complex64, unnormalised, in place,
 * batched over the n_w planes.  direction +1: inverse (e^{+2 pi i}), used for
 * imaging; -1: forward, used by degridding.  RICK_EINVAL for a plan whose
 * plane count rick_plan_set_planes changed. */
rick_status rick_fft_wplanes(rick_plan *plan, void *planes_dev, int32_t direction, void *stream);

/* w-correction and plane sum (§2 step 4, Eq. 2):
 * image[q][p] = Re( sum_k (-1)^(p+q) F_k[q][p] e^{2 pi i w_k (n - 1)} ) s(p,q),
 * w_k = fma(k + 1/2, dw, w_min), n - 1 = -(l^2+m^2) / (1 + sqrt(1 - l^2 - m^2)),
 * s = [n if RICK_N_CORRECT] [1/n if RICK_N_DIVIDE] [1/sum w if RICK_NORMALIZE]
 *     / (C(l) C(m)),  C the continuous transform of G (C == 1 for W == 1).
 * The phase w_k (n - 1) is formed in double-single arithmetic from FP64 inputs
 * (RICK_PHASE_FP32: plain FP32, for comparison).  p, q are grid-frame pixels;
 * only the central image_n x image_n are computed and written, to the m x m
 * image_dev.
 * ws_dev supplies the w range and weight sum of the last rick_bin. */
rick_status rick_wcorrect_stack(rick_plan *plan, const void *planes_dev, const void *ws_dev,
                                float *image_dev, uint32_t flags, void *stream);

/* rick_grid that writes only the uv-tiles that records reach (the tiles with
 * gridding work items in ws_dev); every other tile of planes_dev keeps what it
 * held.  For rick_fft_wcorrect with sparse = 1 and the same ws_dev, which reads
 * exactly those tiles: the planes then need no clearing, which on sparse uv
 * coverage is most of the 8 n_w n^2 bytes rick_grid writes. */
rick_status rick_grid_sparse(rick_plan *plan, void *ws_dev, void *planes_dev, void *stream);

/* rick_grid_sparse of n_jobs imaging jobs in one launch (§2 step 2, Eq. 3, for
 * each job): the work items (uv-tile, chunk of records) of every job's last
 * rick_bin form one list, which one persistent grid kernel works through.  For
 * serving many small jobs, whose own launches would each leave most of the GPU
 * idle.  plans[j], ws_dev[j], planes_dev[j]: job j's plan, the workspace of its
 * binning and its planes (each job its own workspace and planes).
 * 1 <= n_jobs <= RICK_GRID_BATCH_MAX (else RICK_ERANGE).  Every plan must have
 * the same support and tile and be on one device, with RICK_PREC_FP32 and
 * without RICK_OPT_DETERMINISTIC (else RICK_EINVAL).  Each job's planes then
 * hold what rick_grid_sparse would have written (the same sums, possibly added
 * in another order).  Enqueued on stream; the caller orders it after every
 * job's binning (and before what reads the planes).  A CUDA launch error marks
 * every plan of the batch with RICK_ECUDA.  Uses the first job's workspace
 * header as the batch's work counter. */
#define RICK_GRID_BATCH_MAX 16
rick_status rick_grid_sparse_batch(rick_plan *const *plans, void *const *ws_dev,
                                   void *const *planes_dev, int32_t n_jobs, void *stream);

/* Bytes of the fused transform's work buffer (rick_fft_wcorrect,
 * rick_wspread_fft) for plans of these parameters, without a plan: 0 where n is
 * outside 256 ... 8192.  Host-only; enqueues nothing.  RICK_EINVAL for invalid
 * parameters.  For sizing device memory before plans exist (the serving
 * admission). */
rick_status rick_fused_work_bytes(const rick_params *params, size_t *work_bytes);

/* Bytes of the work buffer of rick_fft_wcorrect for this plan.  Its layout,
 * each piece starting on a 256-byte boundary: uint8 tile flags [n_w][nt][nt]
 * (nt = n / tile; 1: the tile was read), uint8 tile-row flags [n_w][nt],
 * uint8 plane flags [n_w], 128-bit tile-row bit masks [n_w] and tile bit
 * masks [n_w][nt] (two uint64 each, for nt <= 128), then the row transforms, complex64
 * [n_w][image_n][n] (8 n_w image_n n bytes; image_n = n without a crop; at
 * n = 8192 the columns are stored in interleaved pairs, [n_w][image_n/2][n][2]).
 * RICK_EINVAL if n is outside 256 ... 8192, the sizes the fused transform
 * covers (use rick_fft_wplanes + rick_wcorrect_stack there). */
rick_status rick_fft_wcorrect_bytes(const rick_plan *plan, size_t *work_bytes);

/* The inverse FFT of every plane (§2 step 3) fused with the w-correction and
 * plane sum (§2 step 4, Eq. 2): the same image as rick_fft_wplanes(+1)
 * followed by rick_wcorrect_stack with the same flags, up to FP32 rounding
 * order, without transforming the planes in place (planes_dev is only read).
 * Two passes of 1D transforms: along u for the rows of tile-rows that hold
 * records, stored transposed in work_dev; then along v for each image column,
 * summing the planes into the image (the w-phase of each block of 8 planes
 * by Horner's rule from the block's exact first-plane phase).
 *   sparse = 1: only the tiles with gridding work items in ws_dev are read;
 *               all other tiles are taken as zero (planes_dev from rick_grid
 *               or rick_grid_sparse with this ws_dev).
 *   sparse = 0: every tile is read (planes accumulated over several binnings).
 * work_dev: device, 256-byte aligned, at least rick_fft_wcorrect_bytes; its
 * contents are scratch, and calls that share it must not overlap on the device.
 * ws_dev supplies the w range, the weight sum and (for sparse) the tiles.  RICK_EINVAL for an n outside 256 ... 8192, a short or
 * misaligned buffer or unknown flags. */
rick_status rick_fft_wcorrect(rick_plan *plan, const void *planes_dev, const void *ws_dev,
                              int32_t sparse, void *work_dev, size_t work_bytes,
                              float *image_dev, uint32_t flags, void *stream);

/* The adjoint of rick_fft_wcorrect for degridding: w-spreading (the transpose
 * of the w-correction, Eq. 2) fused with the forward FFT of every plane, the
 * adjoint of §2 steps 3-4.  planes[k] = forward 2D DFT (e^{-2 pi i}) of
 * image[q][p] s(p,q) (-1)^(p+q) e^{-2 pi i w_k (n - 1)} (zero outside the crop),
 * the same as rick_wspread followed by rick_fft_wplanes(-1) with the same flags,
 * up to FP32 rounding order -- but written only for the uv-tiles with gridding
 * work items in ws_dev, the only cells rick_degrid reads for that binning; the
 * other tiles of planes_dev keep what they held.  Two passes of 1D transforms
 * (along q per image column, then along p per row of the tile-rows with
 * records).  work_dev as for rick_fft_wcorrect (the two calls may share it; its
 * contents are scratch).  RICK_EINVAL for an n outside 256 ... 8192, a short or
 * misaligned buffer or unknown flags. */
rick_status rick_wspread_fft(rick_plan *plan, const float *image_dev, const void *ws_dev,
                             void *work_dev, size_t work_bytes, void *planes_dev, uint32_t flags,
                             void *stream);

/* Adjoint of rick_wcorrect_stack (same flags): for every plane k,
 * planes[k][q][p] = image[q][p] s(p,q) (-1)^(p+q) e^{-2 pi i w_k (n - 1)},
 * the m x m image zero-padded to the n x n grid frame (cells outside the
 * central crop are written as 0). */
rick_status rick_wspread(rick_plan *plan, const float *image_dev, const void *ws_dev,
                         void *planes_dev, uint32_t flags, void *stream);

/* Degridding, the adjoint of rick_grid: for every binned visibility m,
 * vis_out[m] = [weight[m]] sum_{jx,jy} G(jx-h-fx) G(jy-h-fy)
 *              (-1)^(i+j) planes[k][a_y+jy][a_x+jx],
 * written in input order; dropped visibilities get 0.
 *   weight_dev: float32 [n_vis] (the weights given to rick_bin) or NULL (none)
 *   vis_out_dev: complex64 [n_vis] */
rick_status rick_degrid(rick_plan *plan, void *ws_dev, const void *planes_dev,
                        const float *weight_dev, void *vis_out_dev, void *stream);

/* Imaging a visibility set held in HOST memory, streamed through the GPU in
 * chunks (§4: visibilities are read in sequential chunks; §3.2 counts the
 * offload to the GPU in the gridding time).  The set is cut into chunks of at
 * most the plan's max_vis visibilities.  A copy stream owned by the plan
 * moves the next chunks into a ring of RICK_STREAM_BUFS staging buffers while
 * `stream` bins chunk c and grids it into planes_dev.  Where the fused
 * transform covers n (256 ... 8192), each chunk writes only the uv-tiles its
 * records reach (overwriting those no earlier chunk reached, adding into the
 * others) and rick_fft_wcorrect then reads the tiles any chunk reached; else
 * rick_grid grids the first chunk, rick_grid_accumulate the later ones, and
 * rick_fft_wplanes and rick_wcorrect_stack run once.  The image is that of
 * rick_bin + rick_grid + rick_fft_wplanes + rick_wcorrect_stack over the whole
 * set, up to FP32 summation order; the weight sum and drop counts are totals
 * over the chunks, added in chunk order.
 * The w range is the plan's; if it is (NaN, NaN), the exact range of the
 * whole set: uvw is then first copied, in chunks, into a device-resident
 * array in the staging buffer, each chunk's range folded in as it lands, and
 * every chunk is binned with that range (so nothing is dropped that the
 * range-from-data binning keeps).  With a given range nothing of the set stays
 * resident, so the set may be larger than device memory.
 *   uvw_host, vis_host, weight_host: host arrays laid out as for rick_bin
 *               (weight NULL: unit weights).  Page-locked memory
 *               (cudaHostAlloc, cudaHostRegister) lets copies overlap compute;
 *               pageable memory is accepted and copied without overlap.  They
 *               must not change until the work is complete.
 *   ws_dev, ws_bytes:       workspace of rick_workspace_bytes(params, max_vis)
 *   stage_dev, stage_bytes: staging area of rick_stream_bytes(params, max_vis,
 *               n_vis) bytes, 256-byte aligned
 *   planes_dev: complex64 [n_w][n][n], scratch (with the fused transform, the
 *               tiles no record reaches keep what they held)
 *   image_dev:  float32 [m][m]; flags as for rick_wcorrect_stack
 *   stats_dev:  device rick_bin_stats of the whole set, or NULL
 * Work is enqueued on `stream` and on the plan's copy stream, which waits for
 * earlier work on `stream` before it touches the staging area; the call is
 * complete when `stream` is.  Afterwards ws_dev holds the last chunk's binning
 * with the whole set's stats.  Errors: RICK_EINVAL (NULL pointer,
 * misalignment), RICK_ERANGE (stage_bytes or ws_bytes too small, max_vis ==
 * 0 with n_vis > 0), RICK_ECUDA, RICK_ECUFFT. */
#define RICK_STREAM_BUFS 6
rick_status rick_stream_bytes(const rick_params *params, int64_t max_vis, int64_t n_vis,
                              size_t *bytes);
rick_status rick_image_host(rick_plan *plan, int64_t n_vis, const double *uvw_host,
                            const void *vis_host, const float *weight_host, void *ws_dev,
                            size_t ws_bytes, void *stage_dev, size_t stage_bytes,
                            void *planes_dev, float *image_dev, uint32_t flags,
                            rick_bin_stats *stats_dev, void *stream);

/* Imaging weights from the uv-cell density (the paper's §2 names
 * Briggs 1995 for the weighting).  The density D of a uv cell is the sum of the
 * natural weights of the kept visibilities whose centre cell c (the cell
 * nearest to (x, y), as in rick_bin) it is, over all w-planes.
 *   RICK_WEIGHT_UNIFORM: w' = w / D
 *   RICK_WEIGHT_BRIGGS:  w' = w / (1 + f^2 D),
 *                        f^2 = (5 10^-robust)^2 / (sum_cells D^2 / sum w)
 * Dropped visibilities get w' = 0.  The pass reads the corners and keys that
 * the last rick_bin / rick_bin_channels of these n_vis visibilities left in
 * ws_dev, and their weights weight_dev (NULL: unit, as given to the binning).
 * To image with the new weights, pass them to rick_bin_values, then grid as
 * usual.  D is accumulated in FP32 with float atomics (order unspecified),
 * sum D^2 in FP64.
 *   scratch_dev: rick_density_scratch_bytes(params) bytes, 256-byte aligned
 *   weight_out_dev: float32 [n_vis], input order
 * Errors: RICK_EINVAL (NULL pointer, misalignment, unknown scheme, robust not
 * finite), RICK_ERANGE (n_vis > max_vis, scratch too small). */
rick_status rick_density_scratch_bytes(const rick_params *params, size_t *bytes);
rick_status rick_density_weights(rick_plan *plan, int64_t n_vis, const float *weight_dev,
                                 void *ws_dev, int32_t scheme, double robust, void *scratch_dev,
                                 size_t scratch_bytes, float *weight_out_dev, void *stream);

/* rick_image_host for multi-channel input held in host memory: rows of n_chan
 * channels with uvw once per row and a factor per channel, as for
 * rick_bin_channels (1 <= n_chan <= 4096).  Chunks are whole rows, at most
 * the plan's max_vis visibilities each; the staging area is that of
 * rick_stream_bytes(params, max_vis, n_rows n_chan).  Only 24 bytes of uvw per
 * row cross to the device.  The image equals rick_image_host's on the expanded
 * uvw. */
rick_status rick_image_host_channels(rick_plan *plan, int64_t n_rows, int32_t n_chan,
                                     const double *uvw_rows_host, const double *chan_scale_host,
                                     const void *vis_host, const float *weight_host,
                                     void *ws_dev, size_t ws_bytes, void *stage_dev,
                                     size_t stage_bytes, void *planes_dev, float *image_dev,
                                     uint32_t flags, rick_bin_stats *stats_dev, void *stream);

/* rick_image_host_channels with n_corr correlations per visibility, folded as
 * in rick_bin_rows (vis_host, weight_host [n_rows][n_chan][n_corr]).  A chunk
 * holds at most max_vis values, i.e. max_vis / n_corr visibilities, so the
 * staging area of rick_stream_bytes(params, max_vis, n_rows n_chan) serves it. */
rick_status rick_image_host_rows(rick_plan *plan, int64_t n_rows, int32_t n_chan, int32_t n_corr,
                                 const double *uvw_rows_host, const double *chan_scale_host,
                                 const void *vis_host, const float *weight_host, void *ws_dev,
                                 size_t ws_bytes, void *stage_dev, size_t stage_bytes,
                                 void *planes_dev, float *image_dev, uint32_t flags,
                                 rick_bin_stats *stats_dev, void *stream);

/* Measured per-SM throughput of this GPU (the current device), for stating the
 * gridding and transform kernels against the on-chip units that bound them
 * (the shared-memory read-modify-writes of Eq. 3's accumulation, the FP32
 * arithmetic of the transforms).  The paper has no counterpart; this is a
 * measurement aid.  One CTA of 1024 threads per SM repeats the operation on
 * eight private words (or registers) per thread, conflict-free, timed with the
 * SM's cycle counter; *ops_per_clock_per_sm is the median over the SMs, in
 * operations per SM clock (FP32 FMAs for the two FMA kinds).  Synchronous: it
 * allocates a few KB with cudaMalloc and synchronises the device.
 * Errors: RICK_EINVAL (unknown kind, NULL output), RICK_ENOMEM, RICK_ECUDA. */
#define RICK_PROBE_SMEM_RMW 0        /* plain FP32 load-add-store of shared memory   */
#define RICK_PROBE_SMEM_ATOMIC_F32 1 /* FP32 atomic add to shared memory             */
#define RICK_PROBE_SMEM_ATOMIC_U32 2 /* 32-bit integer atomic add to shared memory   */
#define RICK_PROBE_SMEM_ATOMIC_U64 3 /* 64-bit integer atomic add to shared memory   */
#define RICK_PROBE_FFMA 4            /* FP32 fused multiply-add, one per instruction */
#define RICK_PROBE_FFMA2 5           /* FP32 fused multiply-add, two per instruction */
#define RICK_PROBE_SHFL 6            /* 32-bit warp shuffle (per lane)               */
#define RICK_PROBE_F2I 7             /* FP32 to int32 conversion, round to nearest    */
rick_status rick_probe_throughput(int32_t kind, double *ops_per_clock_per_sm);

#ifdef __cplusplus
}
#endif
#endif /* RICK_H */

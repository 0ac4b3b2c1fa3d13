/*
 * vista.h -- C ABI of libvista, GB300-native visibility stacking in the
 * Fourier domain (the hot path of ViSta, arxiv 2609.01897).
 *
 * For every source, row, channel and polarisation the library
 *   1. phase-shifts the visibility to the source position
 *      V' = V exp(+2 pi i nu_k tau / c),  tau = u l + v m + w (sqrt(1-l^2-m^2) - 1)
 *      (paper Eq. 2; the sign makes a point source at (l, m) real), and grids
 *      it with the stored baseline, or with the baseline rotated to the
 *      stacking position (Eq. 1, vista_add_source_reproject),
 *   2. maps the observed channel to the rest frame, nu_rest = nu_obs (1+z)
 *      (Eq. 1's frequency scaling), spreading it over the output bins of a
 *      common rest lattice with the channel-overlap weights of Eqs. 3-4,
 *   3. accumulates sum W w_kj V', sum W w_kj, sum W w_kj |V|^2 and a count into
 *      a cube [nv][nu][nrest][npol] of uv cells x rest channels x pol planes.
 * vista_regrid_rows() gives the paper's own per-row output (Eq. 3) instead.
 *
 * Conventions shared by every call
 *   - Every call returns VISTA_OK (0) or a negative VISTA_E_* status.  A
 *     failing call leaves the handle as it was.  vista_last_error() gives a
 *     one-line reason.
 *   - A handle is used by one host thread at a time.
 *   - Device work is asynchronous on the stream given at open; vista_read_cube(),
 *     vista_get_stats(), vista_regrid_rows(), vista_contsub() and
 *     vista_close() wait for it.
 *   - Sizes are element counts, not bytes.
 */
#ifndef VISTA_H
#define VISTA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define VISTA_ABI_VERSION 6   /* 2: vista_add_source_reproject, vista_regrid_rows;
                                 3: vista_contsub, vista_set_wave_bytes, vista_get_waves;
                                 4: vista_get_h2d_bytes;
                                 5: vista_read_cube_async, vista_wait_readback;
                                 6: vista_read_cube_sparse */
#define VISTA_MAX_BINS 4      /* rest bins one input channel may touch */
#define VISTA_MAX_POL 4

enum {
    VISTA_OK = 0,
    VISTA_E_ARG = -1,      /* invalid argument or descriptor field */
    VISTA_E_STATE = -2,    /* call not valid in the handle's state, or unknown/closed handle */
    VISTA_E_NOMEM = -3,    /* host or device allocation failed */
    VISTA_E_CUDA = -4,     /* a CUDA runtime call failed */
    VISTA_E_RANGE = -5,    /* inputs exceed a supported size */
    VISTA_E_TIMEOUT = -6   /* a bounded device-side wait gave up (reported by read/stats) */
};
/* A call that fails on a CUDA runtime error (VISTA_E_NOMEM, VISTA_E_CUDA)
 * clears that error from the calling thread's CUDA state (cudaGetLastError)
 * before it returns: a failed allocation does not resurface in the caller's
 * later launch checks or in the next call.  The handle stays usable after
 * VISTA_E_NOMEM; free device memory and repeat the call. */

enum { VISTA_VIS_C64 = 0, VISTA_VIS_C128 = 1, VISTA_VIS_F16X2 = 2, VISTA_VIS_BF16X2 = 3 };
enum { VISTA_BIN_OVERLAP = 0, VISTA_BIN_NEAREST = 1 };
enum { VISTA_PREC_MIXED = 0, VISTA_PREC_FP64 = 1 };
enum { VISTA_MEM_DEVICE = 0, VISTA_MEM_HOST = 1 };

typedef struct vista_stack vista_stack;   /* opaque handle */

/* The output cube.
 *   nu, nv     uv cells along u and v; even, >= 2.  Cell iu holds
 *              floor(u_lambda / du) + nu/2 (and the same for v).
 *   nrest      rest-frame output channels, >= 1.
 *   npol       cube polarisation planes, 1..4.
 *   du, dv     uv cell size in wavelengths, > 0.
 *   rest_f0    lower edge of rest bin 0, Hz (used when rest_df > 0).
 *   rest_df    rest bin width, Hz; 0 selects the paper's rule (Sec. 3.1):
 *              the widest rest-frame input channel of the sources added
 *              before the first vista_run(), with the lattice centred on
 *              central_freq.  The lattice is fixed at the first run.
 *   central_freq  Hz, used only when rest_df == 0.
 *   bin_mode   VISTA_BIN_OVERLAP (Eqs. 3-4) or VISTA_BIN_NEAREST.
 *   precision  VISTA_PREC_MIXED: FP64 geometry and tables (the delay of
 *              each row kept as a float-float pair), FP32 per-visibility
 *              body, an FP32 cube whose entries are moved into an FP64 master
 *              cube at checkpoints spread over the drains and folded into it
 *              wholly after a run once 64 visibilities per cube entry have
 *              been stacked since the last fold (measured within 4.3e-6
 *              relative on every entry of a 3.8e11-visibility stack, and the
 *              same after stacking it twice); VISTA_PREC_FP64: the plain
 *              form, FP64 throughout with an FP64 cube.
 *   hermitian_fold  1: rows with v < 0 (or v == 0, u < 0) are negated and
 *              their shifted visibility conjugated before binning.
 *   stream     cudaStream_t for all device work (NULL = legacy default stream). */
typedef struct {
    int32_t nu, nv, nrest, npol;
    double du, dv;
    double rest_f0, rest_df;
    double central_freq;
    int32_t bin_mode, precision, hermitian_fold, reserved0;
    void *stream;
} vista_cube_desc;

/* One (source, spectral window).
 *   nrow, nchan, npol  nrow >= 0; nchan >= 1 (>= 2 in overlap mode, which
 *              needs a channel width); npol in {1, 2, 4}.
 *   uvw        [nrow][3] float64, metres.
 *   freqs      HOST [nchan] float64, observed channel centres in Hz, finite,
 *              > 0, strictly monotone (either direction).  Copied by the call.
 *   vis        [nrow][nchan][npol] complex values of type vis_type:
 *              C64 (2 x float32), C128 (2 x float64), F16X2 / BF16X2
 *              (2 x 16-bit, value = stored * vis_scale).  Base address
 *              aligned to the size of one channel's npol values, capped
 *              at 16 bytes.
 *   vis_scale  dequantisation scale of the 16-bit types (ignored otherwise).
 *   weights    [nrow][npol] float32, >= 0 (the MS WEIGHT column).
 *   flags      [nrow][nchan][npol] uint8, nonzero = flagged; NULL = none.
 *   pol_map    HOST [npol] int32: cube plane of each input pol, -1 = skip;
 *              NULL = identity (needs npol <= cube npol).  Copied by the call.
 *   l, m       direction cosines of the source relative to the phase
 *              centre, l^2 + m^2 < 1.
 *   z          redshift, > -1.
 *   mem        VISTA_MEM_DEVICE: uvw/vis/weights/flags are device pointers,
 *              borrowed: they must stay valid and unchanged until the stream
 *              work of the vista_run() that consumes them has completed.
 *              VISTA_MEM_HOST: they are host pointers (pinned memory gives
 *              asynchronous copies); vista_run() copies them to device
 *              buffers owned by the handle, in waves that overlap the
 *              stacking of the wave before, and returns without waiting:
 *              they must stay valid and unchanged until the run's stream
 *              work has completed (vista_read_cube(), vista_get_stats() or a
 *              stream synchronize). */
typedef struct {
    int64_t nrow;
    int32_t nchan, npol;
    const double *uvw;
    const double *freqs;
    const void *vis;
    int32_t vis_type;
    float vis_scale;
    const float *weights;
    const uint8_t *flags;
    const int32_t *pol_map;
    double l, m, z;
    int32_t mem, reserved0;
} vista_source_desc;

/* Counters over the visibilities of every channel that reaches the cube
 * (at least one rest bin inside [0, nrest)) and every mapped pol, summed
 * over all runs since open (or the last vista_zero_cube()). */
typedef struct {
    uint64_t n_vis;         /* visibilities read */
    uint64_t n_flagged;     /* of those, flagged */
    uint64_t n_dropped_uv;  /* unflagged, outside the uv grid */
    uint64_t n_stacked;     /* unflagged, accumulated into the cube */
    uint64_t n_reductions;  /* reductions into the cube issued by the mixed path (one per
                               cube entry update after on-chip pre-reduction); 0 for FP64 */
} vista_stats;

/* Launch shape of the mixed-precision path (0 fields = library default).
 *   rows_per_item   rows one warp walks through per work item (1..256; their
 *                   FP64 records are staged in shared memory).
 *   chans_per_lane  channels per lane in one item (item = 32 x this many
 *                   channels; 1, 2 or 4).
 *   warps_per_cta   warps per block of the stacking kernel.
 *   sort_rows       1: order rows by uv cell before stacking (fewer
 *                   global reductions), 0: stack in input order.
 *   prefetch_rows   visibility rows each warp keeps in flight (2, 4 or 8
 *                   with one channel per lane, 2 or 4 with two, 2 with
 *                   four). */
typedef struct {
    int32_t rows_per_item, chans_per_lane, warps_per_cta, sort_rows, prefetch_rows;
} vista_tuning;

/* Open a cube (zeroed) on the current CUDA device.  Allocates the cube.
 * Defined by Sec. 3.1 ("Architecture"): before the stacking loop the
 * pipeline computes one common output grid for all inputs, with the output
 * channel width the widest rest-frame input channel (rest_df = 0 here) and
 * the grid centred on central_freq; the cube is this library's form of that
 * common grid, extended by uv cells (the paper writes one spectral window per
 * input instead).
 * E_ARG on an invalid descriptor, E_NOMEM / E_CUDA on allocation failure.
 * On failure *out is set to NULL and vista_last_error(NULL) has the reason. */
int vista_open_stack(const vista_cube_desc *desc, vista_stack **out);

/* Queue one (source, spectral window) for the next vista_run().  Defined by
 * Sec. 3.1: each input is listed with its redshift z and sky position, and
 * the reader materialises its visibilities, flags, UVW coordinates and
 * per-channel frequencies (the DATA, FLAG, UVW columns and the SPECTRAL_WINDOW
 * table); here the position is the offset (l, m) of Eq. 2 and WEIGHT rides
 * along for the weighted sums.  Validates every host-visible field (sizes,
 * freqs, l, m, z, pol_map, pointer alignment); the contents of device arrays
 * are not inspected. */
int vista_add_source(vista_stack *h, const vista_source_desc *src);

/* Queue a window with the full re-projection of Eq. 1 (Sec. 3.2): the
 * window's phase centre is (ra0, dec0) and the stacking position (ra1, dec1),
 * radians, in one equatorial frame.  Otherwise as vista_add_source.
 *   - The phase shift of Eq. 2 uses (l, m) = the direction cosines of
 *     (ra1, dec1) seen from (ra0, dec0):
 *       l = cos dec1 sin(ra1 - ra0),
 *       m = sin dec1 cos dec0 - cos dec1 sin dec0 cos(ra1 - ra0);
 *     src->l and src->m are ignored.
 *   - The uv cells use the baseline expressed for the new phase centre,
 *     (u', v', w') = R (u, v, w) with R = M(ra1, dec1) M(ra0, dec0)^T and
 *     M(ra, dec) the rows (east, north, toward (ra, dec)) of the uvw frame;
 *     R is formed on the host in FP64, and u' = (R00 u + R01 v) + R02 w (the
 *     same for v') in FP64 with every product and sum rounded, so the cells
 *     follow the same FP64 rule as without re-projection.  The Hermitian fold
 *     (if on) tests the rotated (u', v').
 * E_ARG: non-finite angles, |dec| > pi/2, or a stacking position 90 degrees
 * or more from the phase centre; and every check of vista_add_source.  The
 * handle is unchanged on error.  Not available in vista_stack_noalloc. */
int vista_add_source_reproject(vista_stack *h, const vista_source_desc *src, double ra0, double dec0, double ra1,
                               double dec1);

/* The paper's per-row output (Eq. 3, Sec. 3.2): every row of one window
 * regridded onto the handle's rest lattice, as the rows of an output
 * measurement set (no uv cube).  For row r, output channel j, pol p:
 *   out_vis[r][j][p]  = sum_k V'(r,k,p) w_kj / sum_k w_kj   (complex64 as
 *                       float pairs; 0 where the sum of weights is 0),
 *   out_wsum[r][j][p] = sum_k w_kj,
 * over the unflagged channels k, with V' the shifted visibility of Eq. 2
 * (src->l, src->m) and w_kj the Eq. 4 weights (or the nearest bin, as the
 * handle's bin_mode).  out_uvw, if not NULL, gets uvw / (1 + z) ([nrow][3],
 * Eq. 1 with R = I).  The visibility weights are not used (Eq. 3 has none).
 * src must describe device arrays (mem = VISTA_MEM_DEVICE); the outputs are
 * device arrays of nrow x nrest x npol entries, owned by the caller.  Each
 * row's delay is formed in FP64 and kept as a float-float pair; each
 * contributor's phasor comes from a float-float phase (error below 5e-7 rad)
 * and the sums are FP32.  One thread per (row, output channel); synchronous
 * on the handle's stream.  The cube and the queue are not touched.
 * Alignment changes only the speed: complex64 vis with 2 or 4 pols on a
 * 16-byte boundary is read in vector loads, and with 2 or 4 pols, out_vis
 * on a 16-byte and out_wsum on a 16-byte (4 pols) or 8-byte (2 pols)
 * boundary are written in vector stores.
 * E_STATE: the lattice is not fixed yet (open with rest_df > 0, or run
 * first).  E_ARG: a host-visible field fails the checks of vista_add_source
 * (nchan >= 2 here). */
int vista_regrid_rows(vista_stack *h, const vista_source_desc *src, float *out_vis, float *out_wsum,
                      double *out_uvw);

/* Stack every queued source into the cube (additive across runs) and clear
 * the queue.  Defined by Sec. 3.2 ("C++/OpenMP Kernel"): per row and channel
 * the phase shift of Eq. 2, the rest-frame mapping of Eq. 1 and the
 * channel-overlap weights of Eqs. 3-4; all queued windows go to the device
 * together, as the N_batch measurement sets of one launch in Sec. 3.3 ("GPU
 * Acceleration").  Host planning happens here; device work is queued on the
 * stream and the call returns without waiting for it.  Host-memory windows
 * stream through two device staging slots in waves of about a quarter of
 * their bytes (64 MB to 2 GB): the copies of one wave, on four copy streams,
 * run while the wave before is stacked (the paper's read -> compute overlap,
 * Sec. 3.1 and 3.3).  E_STATE if nothing is queued,
 * E_RANGE if a channel would touch more than VISTA_MAX_BINS rest bins. */
int vista_run(vista_stack *h);

/* Staged bytes per wave of host-memory windows (vista_run()): 0 = the
 * library's rule (about a quarter of the run's host bytes, 64 MB to 2 GB);
 * smaller waves overlap more finely, each costs a round of kernel launches.
 * A window is never split: a window larger than the budget is a wave. */
int vista_set_wave_bytes(vista_stack *h, int64_t bytes);
/* The number of waves the last vista_run() streamed its host-memory windows
 * in (0: it had none). */
int vista_get_waves(vista_stack *h, int32_t *out);
/* The host-to-device bytes the last vista_run() copied for its host-memory
 * windows (0: none): uvw, weights, and the channels of vis and flags that
 * it reads -- a window's flags go as whole rows when they are whole 4-byte
 * words and at most four times the words read (or 16 MB in all), since a
 * copy of narrow rows runs far below the host link's rate. */
int vista_get_h2d_bytes(vista_stack *h, int64_t *out);

/* Wait for the stream, then copy the cube out.  The arrays are the two
 * sums of Eq. 3 per cube entry (numerator sum W w_kj V', denominator
 * sum W w_kj; their ratio is Eq. 3's V_out for that uv cell), with
 * sum W w_kj |V|^2 and the count of contributions beside them; normalising
 * is the caller's.  Any pointer may be NULL to skip that array.  Layout
 * [nv][nu][nrest][npol] (sum_wv with a trailing [2] = re, im).
 * dst_is_device: 1 = device pointers, 0 = host.  Returns E_TIMEOUT if a
 * device-side wait of an earlier run gave up. */
int vista_read_cube(vista_stack *h, float *sum_wv, float *sum_w, float *sum_wvv,
                    uint32_t *count, int dst_is_device);

/* As vista_read_cube() with float64 sums (exact copies of the FP64 cube of
 * VISTA_PREC_FP64; widened from FP32 for VISTA_PREC_MIXED). */
int vista_read_cube_f64(vista_stack *h, double *sum_wv, double *sum_w, double *sum_wvv,
                        uint32_t *count, int dst_is_device);

/* vista_read_cube() into HOST arrays without waiting (a library convention;
 * Eq. 3's sums as there): the cube as of the work queued so far is copied on
 * the handle's stream into a device snapshot, and the snapshot's copy to the
 * host arrays runs on a stream of its own, so it overlaps the runs queued
 * after this call (their host-to-device copies and kernels).  The host
 * arrays (pinned memory for an asynchronous copy) must stay valid and must
 * not be read until vista_wait_readback() returns.  A later call first lets
 * the previous copy finish before overwriting the snapshot; vista_read_cube()
 * and vista_close() wait for it.  FP32 sums; any pointer may be NULL to skip
 * that array (not all four).  Errors of the runs show in
 * vista_wait_readback(). */
int vista_read_cube_async(vista_stack *h, float *sum_wv, float *sum_w, float *sum_wvv, uint32_t *count);
/* Wait until the last vista_read_cube_async() copy has reached the host;
 * VISTA_OK at once when none is pending.  E_TIMEOUT if a device-side wait
 * of an earlier run gave up. */
int vista_wait_readback(vista_stack *h);

/* The cube's touched entries only (a library convention; Eq. 3's sums as
 * in vista_read_cube): the entries with count > 0, in entry order.  An
 * entry with count 0 received no contribution and holds zero sums, so they
 * give the whole cube.  index[i] is the flat entry index
 * ((iv * nu + iu) * nrest + j) * npol + p of the i-th touched entry.  Its
 * FP32 sums and count go to sum_wv[2 i], sum_wv[2 i + 1], sum_w[i],
 * sum_wvv[i] and count[i], with the same values vista_read_cube gives.  Any
 * sums or count pointer may be NULL to skip that array.  dst_is_device:
 * 1 = device pointers, 0 = host.  *n_touched gets the number of touched
 * entries.  cap = 0 only counts them and writes nothing.  With
 * 0 < cap < *n_touched, nothing is written and the call returns E_RANGE.
 * Waits for the stream (as vista_read_cube) and returns after the copy.
 * E_ARG: n_touched NULL, cap < 0, or index NULL with cap > 0.  E_TIMEOUT:
 * as vista_read_cube. */
int vista_read_cube_sparse(vista_stack *h, int64_t cap, int64_t *index, float *sum_wv, float *sum_w,
                           float *sum_wvv, uint32_t *count, int64_t *n_touched, int dst_is_device);

/* Zero the cube and the counters (the lattice stays fixed). */
int vista_zero_cube(vista_stack *h);

/* Wait for the stream and copy the counters. */
int vista_get_stats(vista_stack *h, vista_stats *out);

/* The rest lattice in use (after the first run; E_STATE before it unless
 * the descriptor fixed rest_df). */
int vista_get_lattice(vista_stack *h, double *rest_f0, double *rest_df);

int vista_set_tuning(vista_stack *h, const vista_tuning *t);
int vista_get_tuning(vista_stack *h, vista_tuning *t);

/* Per-phase device time of vista_run(), measured with CUDA events recorded
 * on the handle's stream around each phase (the paper's compute_s timer,
 * Sec. 4.3, split by kernel).  Accumulated over runs while enabled. */
typedef struct {
    double prepass_ms;   /* FP64 per-row pre-pass (and row ordering) kernels */
    double stack_ms;     /* the stacking kernel(s) */
    double other_ms;     /* host-memory copies and zeroing inside runs */
    int64_t runs;        /* runs timed */
    int64_t launches;    /* kernels launched by those runs */
} vista_timing;

/* on = 1 enables event timing (and resets the totals), 0 disables it. */
int vista_enable_timing(vista_stack *h, int on);
/* Waits for the stream, then reports the totals since timing was enabled. */
int vista_get_timing(vista_stack *h, vista_timing *out);

/* Autotuner of the launch shape (mixed precision).  Times the queued source
 * set under up to `budget` candidate shapes (0 = all of a fixed list: rows
 * per item 32-96, one or two channels per lane, 2-8 warps per block, 2-8
 * rows in flight; the current shape first), `reps` runs each (0 = 2), by
 * the event-timed device work of vista_run(), and keeps the fastest as the
 * handle's tuning (also returned in *best, which may be NULL).  The trial
 * runs go into the cube, which is zeroed afterwards (with the counters), so
 * call it before stacking anything worth keeping; the queue is left as it
 * was.  The paper's own batching is fixed (Sec. 3.3); the shape is this
 * library's. */
int vista_autotune(vista_stack *h, int32_t budget, int32_t reps, vista_tuning *best);

/* CUDA-graph replay of a run's device work (on by default).  The device work
 * of a run (flag repacking copies, the row-ordering pre-pass and the stacking
 * launches: the paper's one batched launch per set of measurement sets,
 * Sec. 3.3) is captured in a graph the second time an unchanged source set
 * is run, and replayed, without host planning, while the set stays
 * unchanged: the same arrays (pointers), shapes, frequencies, positions,
 * redshifts, pol maps, tuning and lattice.  The contents of the arrays may
 * change between runs.  Runs with host-memory sources, and runs while timing
 * is enabled, are planned and launched directly.  on = 0 disables replay. */
int vista_enable_graphs(vista_stack *h, int on);
/* Number of runs replayed from a graph since the handle was opened. */
int vista_graph_runs(vista_stack *h, uint64_t *out);

/* Continuum subtraction over the rest axis (Sec. 3.4, "Post-processing":
 * the paper's first post-processing step, done there by CASA on the output
 * measurement set).  Waits for the stream, then for every uv cell and cube
 * plane fits a polynomial of degree d = min(order, |F| - 1) in the rest-channel
 * abscissa x_j = (2 j - (nrest - 1)) / nrest to the cell's spectrum
 * V_j = sum_wv_j / sum_w_j by weighted least squares (weights sum_w_j) over
 * F = { j : line_free[j] != 0 and sum_w_j > 0 }, and writes
 *   sum_wv_out[..][j][..] = sum_wv_j - sum_w_j p(x_j)
 * for every channel (no fit, and so no change, when F is empty).  The output
 * is again a sum (divide by sum_w for the continuum-subtracted spectrum);
 * sum_w, sum_w|V|^2 and the counts are unchanged and come from
 * vista_read_cube().  The cube itself is not modified.
 *   line_free   HOST [nrest] uint8, nonzero = free of line emission.
 *   order       0..3.
 *   sum_wv_out  [nv][nu][nrest][npol][2] float32 (re, im); device memory if
 *               dst_is_device, else host memory.
 * FP64 fit (moments reduced over each cell's channels, Cholesky solve).
 * E_ARG: null pointers or an order outside 0..3; E_TIMEOUT as
 * vista_read_cube(). */
int vista_contsub(vista_stack *h, const uint8_t *line_free, int32_t order, float *sum_wv_out,
                  int dst_is_device);

/* Wait for the stream, free every device and host resource, and forget the
 * handle; any later call with it returns E_STATE.  A library convention (the
 * paper has no counterpart). */
int vista_close(vista_stack *h);

/* One-line reason for the last failure on h (NULL: the calling thread's last
 * failure without a handle).  Valid until the next call on the same handle.
 * A library convention (the paper has no counterpart). */
const char *vista_last_error(const vista_stack *h);

int vista_abi_version(void);

/* ---- host-only planner entry points (no GPU needed) ---------------------
 * The FP64 tables the library builds, exposed for inspection and tests. */

/* Rest lattice of Sec. 3.1 for nsrc windows: width = max over windows and
 * channels of Delta nu_k (1+z), lower edge = central_freq - (nrest/2) width. */
int vista_plan_lattice(const double *const *freqs, const int32_t *nchan, const double *z,
                       int32_t nsrc, int32_t nrest, double central_freq,
                       double *rest_f0, double *rest_df);

/* Rest bins of every channel of one window (Eqs. 3-4, or nearest): for
 * channel k, bins j0[k] .. j0[k]+nb[k]-1 inside [0, nrest) carry the weights
 * w[k*VISTA_MAX_BINS + b]; nb[k] = 0 when none.  E_RANGE if a channel touches
 * more than VISTA_MAX_BINS bins. */
int vista_plan_channels(const double *freqs, int32_t nchan, double z, double rest_f0,
                        double rest_df, int32_t nrest, int32_t bin_mode,
                        int32_t *j0, int32_t *nb, double *w);

/* ---- debug exports of the device arithmetic -------------------------------
 * Run the mixed (or FP64) path's own phase and cell code for source `src`
 * (index among the sources of the last vista_run, in add order) and write,
 * for every row and every channel the path reads, the phasor exp(+2 pi i
 * nu_k tau / c) as [nrow][nchan][2] float64, or the cell (iu, iv) as
 * [nrow][nchan][2] int32 ((-1, -1) outside the grid).  Entries of channels
 * the path does not read are left untouched.  dst is a device pointer. */
int vista_debug_phasors(vista_stack *h, int32_t src, double *dst);
int vista_debug_cells(vista_stack *h, int32_t src, int32_t *dst);

/* The order in which the mixed path of the last run walked the rows of
 * window `src`: dst (device, [nrow] int32) receives row indices in
 * processing order.  Available when the last run launched a single
 * (vis type, chunk width, npol) class; E_STATE otherwise. */
int vista_debug_order(vista_stack *h, int32_t src, int32_t *dst);

/* ---- stacking without allocation -----------------------------------------
 * (No counterpart in the paper: a deployment convenience.)
 *
 * Some callers cannot call cudaMalloc: an application whose device memory is
 * all owned by another allocator (a framework that reserves the GPU up
 * front), or a pipeline that must not allocate once running because an
 * allocation can synchronise the device at an arbitrary moment.  This call
 * stacks one (source, window) with the mixed-precision path without
 * allocating anything: no handle, and every intermediate lives in one
 * fixed 8 MiB device array inside the library, reserved when the library
 * is loaded and kept by every GPU that loads it until the process exits.
 *
 *   cube    descriptor of the cube; rest_df > 0 is required (the lattice is
 *           the caller's), precision must be VISTA_PREC_MIXED; stream used.
 *   src     one window, device memory (mem = VISTA_MEM_DEVICE).
 *   cube4   caller's device array [nv][nu][nrest][npol][4] float:
 *           (sum W V'.re, sum W V'.im, sum W, sum W |V|^2), added to;
 *           16-byte aligned.
 *   count   caller's device array [nv][nu][nrest][npol] uint32, added to;
 *           8-byte aligned.
 *   A misaligned cube4 or count gives E_ARG before any device work.
 *
 * Returns after the work has finished.  E_RANGE when the window needs more
 * scratch than the array holds: about 52 bytes per row (a 32-byte row
 * record and the row ordering) plus 9 bytes per row and 32-channel chunk
 * (chunk cells, work list), plus the flags when they are not in whole
 * words, i.e. ~95 000 rows of a 120-channel window.  The first call on a device looks up
 * the array's device address, so make that first call before any stream
 * capture.  All calls share the array: calls whose device work overlaps
 * (other host threads, other streams) race on it and must not be made;
 * each call clears what must start at zero.  Errors: vista_last_error(NULL). */
int vista_stack_noalloc(const vista_cube_desc *cube, const vista_source_desc *src, float *cube4,
                        uint32_t *count);

#ifdef __cplusplus
}
#endif

#endif /* VISTA_H */

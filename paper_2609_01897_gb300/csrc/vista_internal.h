// Internal data layout shared by the libvista host code and its kernels.
#pragma once
#include <cstdint>

#include <cuda_runtime.h>

#include "vista.h"

namespace vista {

constexpr double C_LIGHT = 299792458.0;   // m/s
constexpr int MAX_LOCAL_KEYS = 4096;      // cell keys inside one stripe (shared-memory histogram)
constexpr int MAX_STRIPES = 4096;         // stripes of the cube (shared-memory running counts)
constexpr int SEG_ROWS = 2048;            // rows per segment of the row-order slot assignment

// Row-ordering stripes of a cube: S iv rows per stripe (sized so that a
// stripe's cube entries, ~20 B each, stay near 40 MB and resident in L2),
// at most MAX_STRIPES stripes, and a local cell key (iv % S) * nuk + (iu >>
// ushift) below MAX_LOCAL_KEYS.  Returns false if no such layout exists.
inline bool stripe_layout(int nu, int nv, int nrest, int npol, int *S_out, int *nst_out, int *ushift_out,
                          int *nuk_out)
{
    const double row_bytes = (double)nu * nrest * npol * 20.0;
    const int minS = (nv + MAX_STRIPES - 1) / MAX_STRIPES;
    if (minS > MAX_LOCAL_KEYS) return false;
    double s0 = 40e6 / row_bytes;
    s0 = s0 < 1.0 ? 1.0 : (s0 > nv ? nv : s0);
    int S = (int)s0 < minS ? minS : (int)s0;
    int ushift = 0, nuk = nu;
    while ((int64_t)S * nuk > MAX_LOCAL_KEYS) {
        if (S > minS) {
            const int fit = MAX_LOCAL_KEYS / nuk;
            S = fit < minS ? minS : (fit < S - 1 ? fit : S - 1);
        } else {
            ++ushift;
            nuk = (nu + (1 << ushift) - 1) >> ushift;
        }
    }
    *S_out = S;
    *nst_out = (nv + S - 1) / S;
    *ushift_out = ushift;
    *nuk_out = nuk;
    return true;
}

// Channels per 4-byte word of flags (npol bytes per channel): the channel
// ranges the mixed path reads start and end on multiples of this.
__host__ __device__ inline int32_t flag_align_channels(int32_t npol) { return npol >= 4 ? 1 : 4 / npol; }

// Flag rows of a window as the mixed path reads them: the flag array itself
// when it starts on a 4-byte boundary and its rows are whole words, else a
// copy of the channels read with the row pitch rounded up to a word.
inline bool flags_direct(const void *flags, int32_t nchan, int32_t npol)
{
    return ((uintptr_t)flags % 4) == 0 && ((int64_t)nchan * npol) % 4 == 0;
}
inline int64_t flag_pitch(int32_t nin, int32_t npol) { return ((int64_t)nin * npol + 3) / 4 * 4; }

// Cube geometry as the kernels see it.
struct CubeGeom {
    int32_t nu, nv, nrest, npol;
    double gu, gv;      // fl(1 / fl(c du)), fl(1 / fl(c dv))
    int32_t fold, pad;
};

// Per channel the path reads, mixed path (32 B).  su/sv are fl32(s_k);
// nuc_hi + nuc_lo = nu_k / c as a float-float pair (the phase is
// tau * nu_k / c); w0, w1 the first two Eq. 4 weights (a third or fourth,
// possible only for lattices narrower than a channel, is read from ChanD).
struct ChanF {
    float su, sv;
    int32_t j0, nb;
    float w0, w1;
    float nuc_hi, nuc_lo;
};

// Per channel, exact FP64 values (64 B): s_k = fl(nu_k gu) as the cell rule
// defines it, the channel centre, and the FP64 weights.
struct ChanD {
    double su, sv, nu;
    int32_t j0, nb;
    double w[4];
};

// One (source, window) as the kernels see it.
struct SrcDev {
    const double *uvw;      // the stored baselines: the delay of Eq. 2
    const double *guvw;     // the gridding baselines (stride 3, u and v read): uvw, or R uvw for a
                            // re-projected window (Eq. 1)
    const void *vis;        // element (row, k, p) at (row * vstride + k - kbase) * npol + p
    const float *wts;
    int64_t nrow;
    int32_t nchan, npol;
    int32_t vis_type;
    float vis_scale;
    double l, m, n1;        // n1 = sqrt(1 - l^2 - m^2) - 1
    double step_c;          // channel step / c (linear axes)
    int32_t k_lo, k_hi;     // channels [k_lo, k_hi) are read
    int32_t chan_off;       // table entry of channel k is chan_off + (k - k_lo)
    int32_t linear;         // 1: f_k = f_0 + k step (one recurrence step)
    int32_t plane[4];       // cube plane of each input pol, -1 = skip
    int32_t nchunk;         // work chunks along the channel axis
    int32_t vstride;        // channels per stored row (nchan, or k_hi - k_lo when staged)
    int32_t kbase;          // channel index of the first stored channel
    int32_t rot1;           // 1 + index of the window's R in RunArgs::rot (k_rotate fills guvw), 0 = none
    float key_su, key_sv;   // fl32(s_k) at the row-ordering reference channel
    int64_t rec_off;        // first row record of this window
    int64_t cell_off;       // first chunk-cell entry of this window ([chunk][row] inside)
    // flag byte of (row r, channel k, pol p): fbase[r * fpitch + (k - fk0) * npol + p];
    // fbase is 4-byte aligned and fpitch a multiple of 4 (null: no flags)
    const uint8_t *fbase;
    int64_t fpitch;
    int32_t fk0;
    int32_t pad3;
    int64_t pad4;
};
static_assert(sizeof(SrcDev) % 16 == 0, "SrcDev is copied in 16-byte units");

// Per-row record written by the mixed path's FP64 pre-pass (32 B), in
// processing order.
//   tau_hi + tau_lo  the delay tau (metres) as a float-float pair, so that
//                    tau * nu_k / c is formed to ~1e-14 relative in FP32
//   W[4]             the row's weights (>= 0), negated for a folded row: the
//                    sign conjugates the shifted visibility, |W| is the weight
//                    (the sign bit of W[0] marks the fold, also for W = 0)
//   row              the row index in the window's arrays
struct __align__(16) RowRec {
    float tau_hi, tau_lo;
    float W[4];
    uint32_t row, pad;
};
static_assert(sizeof(RowRec) == 32, "RowRec is read as two 16-byte words");

// uv cells of one (row, channel chunk), written by the pre-pass (8 B):
//   x  the cell iv * nu + iu at the chunk's first channel, -1 off the grid
//   y  CC_NOCHANGE: every channel of the chunk shares x;
//      CC_MIXED: the chunk needs the per-channel FP64 rule;
//      else bits 0-7 / 8-15: chunk-local channel at which iu / iv steps
//      (255 = never), bit 16 / 17: that step is -1 (else +1).
// The cell index of a row is monotone in frequency along each axis, so a
// chunk whose end channels differ by at most one cell per axis, both ends on
// the grid, steps at most once per axis; every other chunk is CC_MIXED
// (or, off the grid at both ends of one axis, x = -1 with CC_NOCHANGE).
constexpr int32_t CC_NOCHANGE = 0x0000ffff;
constexpr int32_t CC_MIXED = -1;

// One unit of stacking work: rows [q0, q1) (in processing order) of window
// w, channel chunk c, with the table positions its bulk copies start at.
struct __align__(16) Item {
    int32_t w, chunk, q0, q1;
    int32_t chf0, nch;          // first channel-table entry of the chunk, channels in it
    int64_t rec0;               // first row record
    int64_t cell0;              // first chunk-cell entry
    int64_t pad;
};
static_assert(sizeof(Item) == 48, "Item is copied in 16-byte units");

// Counters (device), see vista_stats.
struct DevStats {
    unsigned long long n_vis, n_flagged, n_dropped_uv, n_stacked, n_reductions;
};

struct LaunchCfg {
    int32_t rows_per_item;
    int32_t chans_per_lane;     // upper bound; each window uses the smallest that fits
    int32_t warps_per_cta;
    int32_t sort_rows;
    int32_t prefetch_rows;      // visibility rows in flight per warp (2, 4, 8)
};

// Row ordering of one launch class (device buffers, see vista_kernels.cu).
//   hist     [nwin][nstripe]    rows per (window, stripe)
//   qstart   [nwin][nstripe]    first processing position of each bucket
//   slot     [rows]             arrival slot of the row inside its bucket
//   key      [rows]             stripe << 13 | local cell key
//   tmp      [rows]             (local key << 32) | row, bucket-grouped
//   perm     [rows]             row of each processing position
//   ioff     [nbuckets + 1]     first work item of each bucket (stripe-major)
//   segcnt   [nseg][nstripe]    rows of each (segment of SEG_ROWS rows, stripe), then
//                               the segment's first slot in each bucket
//   seg_off  [nwin + 1]         cumulative segments per window
//   items    [max_items]        work list, stripe-major
//   ctr      [2]                item count, queue head
struct SortArgs {
    uint32_t *hist, *qstart, *slot, *key, *perm;
    int64_t *ioff;
    uint32_t *segcnt;
    const int64_t *seg_off;
    int64_t nseg_total;
    unsigned long long *tmp;
    Item *items;
    uint32_t *ctr;
    int64_t max_items;
    int32_t stripe_rows;        // iv rows per stripe
    int32_t nstripe;
    int32_t ushift, nuk;        // local key = (iv % stripe_rows) * nuk + (iu >> ushift)
    int32_t sorted;             // 0: identity order
    int32_t rows_per_item;
};

// Everything one mixed or FP64 launch class needs on the device.
struct RunArgs {
    const SrcDev *srcs;
    int32_t nsrc;
    int32_t cw;                 // channels per chunk (32 * NS) of this class
    const ChanF *chf;
    const ChanD *chd;
    RowRec *recs;
    int2 *ccells;               // chunk cells (+ 4 entries of padding for the bulk copies)
    const int64_t *row_off;     // [nsrc+1] cumulative rows
    int64_t nrows_total;
    const double *rot;          // 9 doubles (row-major R of Eq. 1) per re-projected window
    CubeGeom g;
    void *cube;                 // per entry: FP64 double[4], or float4 (mixed)
    double *cube_master;        // mixed with comp = 1: FP64 double[4] per entry, the sums moved
                                // out of the float4 entries at checkpoints (value = master + float4)
    int32_t comp;
    uint32_t *count;
    DevStats *stats;
    int32_t *err;
    SortArgs so;
};

// Kernel launchers (vista_kernels.cu).  Return a cudaError_t.
// Row ordering, records and work list of one mixed class (several kernels).
cudaError_t launch_prepare(const RunArgs &a, cudaStream_t st, int *nlaunch = nullptr);   // kernels launched
// Persistent stacking kernel of one mixed class; key = (vis_type << 16) |
// (chans_per_lane << 8) | npol, shared by every window of the class.
cudaError_t launch_mixed(const RunArgs &a, int key, int warps_per_cta, int prefetch, cudaStream_t st);
cudaError_t launch_fp64(const RunArgs &a, cudaStream_t st);
// The gridding baselines R (u, v, w) of the class's re-projected windows
// (a.rot non-null; one thread per row of the class), for the FP64 form.
cudaError_t launch_rotate(const RunArgs &a, cudaStream_t st);
// Mixed cube: move every FP32 partial into the FP64 master and clear it.
cudaError_t launch_fold(void *cube, double *master, int64_t n, cudaStream_t st);
cudaError_t launch_unpack(const void *cube, const double *master, const uint32_t *count, int fp64, int64_t n,
                          void *sum_wv, void *sum_w, void *sum_wvv, uint32_t *cnt_out,
                          int out_f64, cudaStream_t st);
// Sparse readback (the entries with count > 0, in entry order): per tile of
// 4096 entries the touched count (tile_cnt [ntile]), their exclusive scan
// (tile_off [ntile]) and the total (one int64 on the device); then each
// touched entry's index and sums at its position (positions >= cap are not
// written).
inline int64_t sparse_tiles(int64_t n) { return (n + 4095) / 4096; }
cudaError_t launch_sparse_count(const uint32_t *count, int64_t n, uint32_t *tile_cnt, int64_t *tile_off,
                                int64_t *total, cudaStream_t st);
cudaError_t launch_sparse_write(const void *cube, const double *master, const uint32_t *count, int fp64, int64_t n,
                                const int64_t *tile_off, int64_t cap, int64_t *index, float *sum_wv, float *sum_w,
                                float *sum_wvv, uint32_t *cnt_out, cudaStream_t st);
cudaError_t launch_debug(const RunArgs &a, int ns, int src, int fp64, double *ph, int32_t *cells,
                         cudaStream_t st);

}  // namespace vista

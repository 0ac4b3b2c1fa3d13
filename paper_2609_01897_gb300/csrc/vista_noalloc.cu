// vista_stack_noalloc(): stack one (source, window) into a caller-provided
// cube without allocating anything.
//
// Some callers cannot call cudaMalloc: code that runs inside an application
// whose device memory is entirely owned by another allocator (a framework
// that reserves the GPU up front), or a pipeline that must not allocate after
// start-up because an allocation can synchronise the device at an arbitrary
// moment.  For them this entry point keeps every intermediate (channel
// tables, row records, the row ordering, the work list, counters) in one
// file-scope device array of fixed size, reserved when the library is
// loaded and held by every GPU that loads it until the process exits.
//
// The array is shared by all calls: calls whose device work overlaps in
// time (two host threads, or two streams) race on it and must not be made.
// Everything that has to start at zero is cleared by each call.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "planner.h"
#include "vista_handle.h"

using namespace vista;

namespace {

constexpr size_t NOALLOC_SCRATCH_BYTES = (size_t)8 << 20;   // 8 MiB per device

__device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

std::mutex g_noalloc_mu;
void *g_noalloc_addr[256];   // per device ordinal; null until set up

// The device address of the scratch array on the current device.  In host
// code the array's name only stands in for it, so the address is looked up
// once per device, with that device current.
cudaError_t scratch_address(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 256) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return cudaSuccess;
}

inline size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

extern "C" int vista_stack_noalloc(const vista_cube_desc *c, const vista_source_desc *s, float *cube4,
                                   uint32_t *count)
{
    if (!c || !s || !cube4 || !count) return fail(nullptr, VISTA_E_ARG, "null argument");
    // the stacking kernel adds to the cube with 16-byte vector reductions and,
    // for a pol pair on an even plane pair, to the counts with 8-byte ones:
    // reject pointers those would fault on, before any device work
    if ((uintptr_t)cube4 % 16) return fail(nullptr, VISTA_E_ARG, "cube4 must be 16-byte aligned");
    if ((uintptr_t)count % 8) return fail(nullptr, VISTA_E_ARG, "count must be 8-byte aligned");
    if (c->nu < 2 || c->nv < 2 || (c->nu & 1) || (c->nv & 1) || c->nrest < 1 || c->npol < 1 ||
        c->npol > VISTA_MAX_POL)
        return fail(nullptr, VISTA_E_ARG, "bad cube shape");
    if (!(c->du > 0.0 && c->dv > 0.0 && std::isfinite(c->du) && std::isfinite(c->dv)))
        return fail(nullptr, VISTA_E_ARG, "du and dv must be finite and > 0");
    if (!(c->rest_df > 0.0 && std::isfinite(c->rest_df) && std::isfinite(c->rest_f0)))
        return fail(nullptr, VISTA_E_ARG, "the no-allocation call needs an explicit rest lattice (rest_df > 0)");
    if (c->precision != VISTA_PREC_MIXED) return fail(nullptr, VISTA_E_ARG, "mixed precision only");
    if (c->bin_mode != VISTA_BIN_OVERLAP && c->bin_mode != VISTA_BIN_NEAREST)
        return fail(nullptr, VISTA_E_ARG, "bad bin_mode");
    if ((int64_t)c->nu * c->nv > (int64_t)0x7fffffff) return fail(nullptr, VISTA_E_RANGE, "nu*nv too large");
    if (s->mem != VISTA_MEM_DEVICE) return fail(nullptr, VISTA_E_ARG, "device-memory windows only");
    if (s->nrow < 0 || s->nchan < 1 || (c->bin_mode == VISTA_BIN_OVERLAP && s->nchan < 2) ||
        (s->npol != 1 && s->npol != 2 && s->npol != 4) || !s->freqs)
        return fail(nullptr, VISTA_E_ARG, "bad window shape");
    if (s->vis_type < VISTA_VIS_C64 || s->vis_type > VISTA_VIS_BF16X2) return fail(nullptr, VISTA_E_ARG, "bad vis_type");
    if (!(std::isfinite(s->l) && std::isfinite(s->m) && s->l * s->l + s->m * s->m < 1.0 && std::isfinite(s->z) &&
          s->z > -1.0))
        return fail(nullptr, VISTA_E_ARG, "need l^2 + m^2 < 1 and z > -1");
    if (s->nrow > 0 && (!s->uvw || !s->vis || !s->weights)) return fail(nullptr, VISTA_E_ARG, "null window array");
    for (int32_t k = 0; k < s->nchan; ++k)
        if (!(std::isfinite(s->freqs[k]) && s->freqs[k] > 0.0)) return fail(nullptr, VISTA_E_ARG, "bad freqs");
    for (int32_t k = 1; k < s->nchan; ++k)
        if ((s->freqs[1] > s->freqs[0]) ? !(s->freqs[k] > s->freqs[k - 1]) : !(s->freqs[k] < s->freqs[k - 1]))
            return fail(nullptr, VISTA_E_ARG, "freqs must be strictly monotone");
    {
        const size_t ve = (s->vis_type == VISTA_VIS_C64 ? 8 : s->vis_type == VISTA_VIS_C128 ? 16 : 4) * (size_t)s->npol;
        if (s->nrow > 0 && ((uintptr_t)s->vis % std::min<size_t>(ve, 16) || (uintptr_t)s->uvw % 8 ||
                            (uintptr_t)s->weights % 4 || (s->flags && (uintptr_t)s->flags % (size_t)s->npol)))
            return fail(nullptr, VISTA_E_ARG, "misaligned window array");
    }
    int32_t planes[4] = {-1, -1, -1, -1};
    for (int p = 0; p < s->npol; ++p) {
        planes[p] = s->pol_map ? s->pol_map[p] : p;
        if (planes[p] < -1 || planes[p] >= c->npol) return fail(nullptr, VISTA_E_ARG, "pol_map outside the cube");
    }
    cudaStream_t st = (cudaStream_t)c->stream;

    // channel tables (the same FP64 planner the handle path uses)
    const int32_t n = s->nchan;
    std::vector<int32_t> j0((size_t)n), nb((size_t)n);
    std::vector<double> w((size_t)n * VISTA_MAX_BINS);
    int rc = channel_bins(s->freqs, n, s->z, c->rest_f0, c->rest_df, c->nrest, c->bin_mode, j0.data(), nb.data(),
                          w.data());
    if (rc != VISTA_OK) return fail(nullptr, rc, "channel planning failed");
    int32_t lo = -1, hi = -1, key_ch = 0;
    for (int32_t k = 0; k < n; ++k)
        if (nb[(size_t)k] > 0) {
            if (lo < 0) lo = k;
            hi = k + 1;
        }
    if (s->nrow == 0 || lo < 0) return VISTA_OK;   // nothing reaches the cube
    {
        // the range read starts and ends on whole words of flags (as vista_run)
        const int32_t al = flag_align_channels(s->npol);
        lo = lo / al * al;
        hi = std::min(n, (hi + al - 1) / al * al);
    }
    const double gu = 1.0 / (C_LIGHT * c->du), gv = 1.0 / (C_LIGHT * c->dv);
    const int32_t nin = hi - lo;
    std::vector<ChanF> chf((size_t)nin);
    std::vector<ChanD> chd((size_t)nin);
    double fbest = -1.0;
    for (int32_t k = lo; k < hi; ++k) {
        ChanD &d = chd[(size_t)(k - lo)];
        ChanF &f = chf[(size_t)(k - lo)];
        d.su = s->freqs[k] * gu;
        d.sv = s->freqs[k] * gv;
        d.nu = s->freqs[k];
        d.j0 = j0[(size_t)k];
        d.nb = nb[(size_t)k];
        f.su = (float)d.su;
        f.sv = (float)d.sv;
        f.j0 = d.j0;
        f.nb = d.nb;
        for (int b = 0; b < VISTA_MAX_BINS; ++b) d.w[b] = w[(size_t)k * VISTA_MAX_BINS + b];
        f.w0 = (float)d.w[0];
        f.w1 = (float)d.w[1];
        const double nuc = d.nu / C_LIGHT;
        f.nuc_hi = (float)nuc;
        f.nuc_lo = (float)(nuc - (double)f.nuc_hi);
        if (std::fabs(d.nu) > fbest) {
            fbest = std::fabs(d.nu);
            key_ch = k;
        }
    }
    double step = 0.0;
    const bool linear = linear_axis(s->freqs, n, &step);

    // row-ordering stripes (as for a handle of the same cube)
    int S = 1, nstripe = 1, ushift = 0, nuk = 1;
    if (!stripe_layout(c->nu, c->nv, c->nrest, c->npol, &S, &nstripe, &ushift, &nuk))
        return fail(nullptr, VISTA_E_RANGE, "cube too tall for the row ordering");
    const int R = 64, cw = 32;
    const int nchunk = (nin + cw - 1) / cw;
    const int64_t nrow = s->nrow;
    const int64_t max_items = (int64_t)nchunk * ((nrow + R - 1) / R + nstripe);

    // scratch layout; reject what does not fit
    size_t o = 0;
    const size_t o_src = o;
    o += al256(sizeof(SrcDev));
    const size_t o_off = o;
    o += al256(4 * sizeof(int64_t));
    const size_t o_chf = o;
    o += al256(sizeof(ChanF) * (size_t)nin);
    const size_t o_chd = o;
    o += al256(sizeof(ChanD) * (size_t)nin);
    const size_t o_rec = o;
    o += al256(sizeof(RowRec) * (size_t)nrow);
    const size_t o_cells = o;
    o += al256(sizeof(int2) * ((size_t)nrow * (size_t)nchunk + 4));


    const size_t o_hist = o;
    o += al256(4 * (size_t)nstripe);
    const size_t o_qs = o;
    o += al256(4 * (size_t)nstripe);
    const size_t o_ioff = o;
    o += al256(8 * ((size_t)nstripe + 1));
    const size_t o_segcnt = o;
    o += al256(4 * (size_t)((nrow + SEG_ROWS - 1) / SEG_ROWS) * (size_t)nstripe);
    const size_t o_slot = o;
    o += al256(4 * (size_t)nrow);
    const size_t o_key = o;
    o += al256(4 * (size_t)nrow);
    const size_t o_perm = o;
    o += al256(4 * (size_t)nrow);
    const size_t o_tmp = o;
    o += al256(8 * (size_t)nrow);
    const size_t o_items = o;
    o += al256(sizeof(Item) * (size_t)max_items);
    const size_t o_ctr = o;
    o += 256;
    const size_t o_stats = o;
    o += al256(sizeof(DevStats));
    const size_t o_err = o;
    o += 256;
    // flags the kernel cannot read in words are copied with a word-aligned pitch
    const bool repack = s->flags && !flags_direct(s->flags, n, s->npol);
    const int64_t fpitch = repack ? flag_pitch(nin, s->npol) : (int64_t)n * s->npol;
    const size_t o_flags = o;
    if (repack) o += al256((size_t)nrow * (size_t)fpitch);
    if (o > NOALLOC_SCRATCH_BYTES)
        return fail(nullptr, VISTA_E_RANGE, "window needs %zu bytes of scratch; the no-allocation call has %zu", o,
                    NOALLOC_SCRATCH_BYTES);

    void *base = nullptr;
    cudaError_t e = scratch_address(&base);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "scratch address");
    char *b = (char *)base;

    SrcDev d{};
    d.uvw = s->uvw;
    d.guvw = s->uvw;   // no re-projection here
    d.vis = s->vis;
    d.wts = s->weights;
    d.fbase = repack ? (const uint8_t *)(b + o_flags) : s->flags;
    d.fpitch = fpitch;
    d.fk0 = repack ? lo : 0;
    d.nrow = nrow;
    d.nchan = n;
    d.npol = s->npol;
    d.vis_type = s->vis_type;
    d.vis_scale = (s->vis_type == VISTA_VIS_F16X2 || s->vis_type == VISTA_VIS_BF16X2) ? s->vis_scale : 1.0f;
    d.l = s->l;
    d.m = s->m;
    d.n1 = std::sqrt(1.0 - s->l * s->l - s->m * s->m) - 1.0;
    d.step_c = step / C_LIGHT;
    d.k_lo = lo;
    d.k_hi = hi;
    d.chan_off = 0;
    d.linear = linear ? 1 : 0;
    for (int p = 0; p < 4; ++p) d.plane[p] = planes[p];
    d.nchunk = nchunk;
    d.vstride = n;
    d.kbase = 0;
    d.key_su = (float)(s->freqs[key_ch] * gu);
    d.key_sv = (float)(s->freqs[key_ch] * gv);
    d.rec_off = 0;
    d.cell_off = 0;
    const int64_t nseg = (nrow + SEG_ROWS - 1) / SEG_ROWS;
    // rows, row segments
    const int64_t roff[4] = {0, nrow, 0, nseg};

    // tables into scratch; counters and the error word start at zero
    e = cudaMemcpyAsync(b + o_src, &d, sizeof d, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b + o_off, roff, sizeof roff, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b + o_chf, chf.data(), sizeof(ChanF) * chf.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b + o_chd, chd.data(), sizeof(ChanD) * chd.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && repack)
        e = cudaMemcpy2DAsync(b + o_flags, (size_t)fpitch, s->flags + (size_t)lo * s->npol, (size_t)n * s->npol,
                              (size_t)nin * s->npol, (size_t)nrow, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(b + o_stats, 0, sizeof(DevStats), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(b + o_err, 0, sizeof(int32_t), st);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "scratch set-up");

    RunArgs a{};
    a.srcs = (const SrcDev *)(b + o_src);
    a.nsrc = 1;
    a.cw = cw;
    a.chf = (const ChanF *)(b + o_chf);
    a.chd = (const ChanD *)(b + o_chd);
    a.recs = (RowRec *)(b + o_rec);
    a.ccells = (int2 *)(b + o_cells);
    a.row_off = (const int64_t *)(b + o_off);
    a.so.seg_off = a.row_off + 2;
    a.so.nseg_total = nseg;
    a.nrows_total = nrow;
    a.g = CubeGeom{c->nu, c->nv, c->nrest, c->npol, gu, gv, c->hermitian_fold, 0};
    a.cube = cube4;
    a.cube_master = nullptr;
    a.comp = 0;   // the caller's cube: plain float4 sums
    a.count = count;
    a.stats = (DevStats *)(b + o_stats);
    a.err = (int32_t *)(b + o_err);
    a.so.hist = (uint32_t *)(b + o_hist);
    a.so.qstart = (uint32_t *)(b + o_qs);
    a.so.ioff = (int64_t *)(b + o_ioff);
    a.so.segcnt = (uint32_t *)(b + o_segcnt);
    a.so.slot = (uint32_t *)(b + o_slot);
    a.so.key = (uint32_t *)(b + o_key);
    a.so.perm = (uint32_t *)(b + o_perm);
    a.so.tmp = (unsigned long long *)(b + o_tmp);
    a.so.items = (Item *)(b + o_items);
    a.so.ctr = (uint32_t *)(b + o_ctr);
    a.so.max_items = max_items;
    a.so.stripe_rows = S;
    a.so.nstripe = nstripe;
    a.so.ushift = ushift;
    a.so.nuk = nuk;
    a.so.sorted = 1;
    a.so.rows_per_item = R;
    e = launch_prepare(a, st);
    // one channel per lane, four warps per block, two rows of visibilities in flight
    if (e == cudaSuccess) e = launch_mixed(a, (s->vis_type << 16) | (1 << 8) | s->npol, 4, 2, st);
    int32_t err = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&err, b + o_err, sizeof err, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "no-allocation stack");
    if (err != 0) return fail(nullptr, VISTA_E_TIMEOUT, "a device-side wait or check gave up (code %d)", err);
    return VISTA_OK;
}

// vista_run(): host planning and launch orchestration of one stacking pass.
//
//   1. the rest lattice (Sec. 3.1), fixed at the first run
//   2. per window: FP64 channel tables (Eqs. 3-4, the uv scale s_k), the
//      range of channels that reach the cube, the chunk width
//   3. launch classes: windows sharing one kernel instantiation
//   4. host-memory windows: only the channels that reach the cube are
//      copied (whole rows as one copy, else 2-D copies), into handle-owned
//      device buffers, in waves: the copies of one wave (on four copy
//      streams) run while the wave before is stacked, two staging slots
//      taking turns (the streaming pipeline of Sec. 3.1/3.3: read ->
//      compute overlapped)
//   5. per mixed class: row ordering + records + work list, then the
//      persistent stacking kernel; FP64 precision: the plain kernel
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "planner.h"
#include "vista_handle.h"

using namespace vista;

namespace {

struct Plan {
    int32_t k_lo = 0, k_hi = 0;
    int32_t key_ch = 0;       // in-cube channel with the largest |frequency|
    bool linear = true;
    double step = 0.0;
    std::vector<ChanF> chf;
    std::vector<ChanD> chd;
};

int plan_source(vista_stack *h, const SrcHost &s, double gu, double gv, Plan &pl)
{
    const int32_t n = s.d.nchan;
    std::vector<int32_t> j0((size_t)n), nb((size_t)n);
    std::vector<double> w((size_t)n * VISTA_MAX_BINS);
    const int rc = channel_bins(s.freqs.data(), n, s.d.z, h->f0, h->df, h->desc.nrest, h->desc.bin_mode,
                                j0.data(), nb.data(), w.data());
    if (rc == VISTA_E_RANGE)
        return fail(h, VISTA_E_RANGE, "a channel touches more than %d rest bins (rest_df too small)",
                    VISTA_MAX_BINS);
    if (rc != VISTA_OK) return fail(h, rc, "channel planning failed");
    int32_t lo = -1, hi = -1;
    for (int32_t k = 0; k < n; ++k)
        if (nb[(size_t)k] > 0) {
            if (lo < 0) lo = k;
            hi = k + 1;
        }
    if (lo < 0) lo = hi = 0;
    // The range read starts and ends on a multiple of a = 4 / gcd(npol, 4)
    // channels (the added channels have no rest bin), so that a chunk's flag
    // bytes are whole 4-byte words.
    const int32_t al = flag_align_channels(s.d.npol);
    if (hi > lo) {
        lo = lo / al * al;
        hi = std::min(n, (hi + al - 1) / al * al);
    }
    pl.k_lo = lo;
    pl.k_hi = hi;
    pl.linear = linear_axis(s.freqs.data(), n, &pl.step);
    pl.chf.resize((size_t)(hi - lo));
    pl.chd.resize((size_t)(hi - lo));
    double fbest = -1.0;
    for (int32_t k = lo; k < hi; ++k) {
        ChanD &d = pl.chd[(size_t)(k - lo)];
        ChanF &f = pl.chf[(size_t)(k - lo)];
        d.su = s.freqs[(size_t)k] * gu;
        d.sv = s.freqs[(size_t)k] * gv;
        d.nu = s.freqs[(size_t)k];
        d.j0 = j0[(size_t)k];
        d.nb = nb[(size_t)k];
        f.su = (float)d.su;
        f.sv = (float)d.sv;
        f.j0 = d.j0;
        f.nb = d.nb;
        for (int b = 0; b < VISTA_MAX_BINS; ++b) d.w[b] = w[(size_t)k * VISTA_MAX_BINS + b];
        f.w0 = (float)d.w[0];
        f.w1 = (float)d.w[1];
        const double nuc = d.nu / C_LIGHT;   // nu_k / c as a float-float pair
        f.nuc_hi = (float)nuc;
        f.nuc_lo = (float)(nuc - (double)f.nuc_hi);
        if (std::fabs(d.nu) > fbest) {
            fbest = std::fabs(d.nu);
            pl.key_ch = k;
        }
    }
    return VISTA_OK;
}

// A run's table uploads go through one half of the handle's pinned staging
// area: the half is reused two runs later, after its uploads have completed
// (an event), and the copies from it return without waiting for the stream.
// Without pinned memory to be had, the tables are copied from pageable
// memory (correct, but the call then waits for the stream).
struct Uploader {
    vista_stack *h;
    char *base = nullptr;
    size_t pos = 0;
    cudaError_t begin(size_t total)
    {
        const int x = h->pin_half;
        cudaError_t e = cudaSuccess;
        if (!h->pin_ev[x]) e = cudaEventCreateWithFlags(&h->pin_ev[x], cudaEventDisableTiming);
        else e = cudaEventSynchronize(h->pin_ev[x]);   // this half's uploads of two runs ago
        if (e == cudaSuccess && total > h->pin_cap[x]) {
            if (h->pin[x]) cudaFreeHost(h->pin[x]);
            h->pin[x] = nullptr;
            h->pin_cap[x] = 0;
            const size_t want = total + total / 8 + 4096;
            if (cudaHostAlloc(&h->pin[x], want, cudaHostAllocDefault) == cudaSuccess) {
                h->pin_cap[x] = want;
            } else {
                h->pin[x] = nullptr;
                (void)cudaGetLastError();   // no pinned memory: pageable copies below
            }
        }
        base = (char *)h->pin[x];
        pos = 0;
        return e;
    }
    template <typename T>
    cudaError_t put(DevBuf &b, const std::vector<T> &v)
    {
        const size_t bytes = v.size() * sizeof(T);
        cudaError_t e = b.ensure(bytes > 0 ? bytes : 16);
        if (e != cudaSuccess || bytes == 0) return e;
        if (!base) return cudaMemcpyAsync(b.p, v.data(), bytes, cudaMemcpyHostToDevice, h->stream);
        std::memcpy(base + pos, v.data(), bytes);
        e = cudaMemcpyAsync(b.p, base + pos, bytes, cudaMemcpyHostToDevice, h->stream);
        pos += (bytes + 255) & ~(size_t)255;
        return e;
    }
    cudaError_t end()
    {
        const cudaError_t e = cudaEventRecord(h->pin_ev[h->pin_half], h->stream);
        h->pin_half ^= 1;
        return e;
    }
};
template <typename T>
size_t upload_bytes(const std::vector<T> &v)
{
    return (v.size() * sizeof(T) + 255) & ~(size_t)255;
}

// Smallest channels-per-lane (1, 2, 4; at most cap) whose chunk holds nin
// channels; windows wider than 32*cap use several chunks.
int choose_ns(int nin, int cap)
{
    for (int ns = 1; ns <= cap; ns <<= 1)
        if (32 * ns >= nin) return ns;
    return cap;
}

inline size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

// Layout of the shared ordering buffer for one class.
struct SortLayout {
    size_t hist, qstart, ioff, segcnt, slot, key, perm, tmp, items, ctr, total;
};

SortLayout sort_layout(int64_t rows, int64_t nbuckets, int64_t max_items, int64_t nseg, int nstripe)
{
    SortLayout L{};
    size_t o = 0;
    L.hist = o;
    o += al256(4 * (size_t)nbuckets);
    L.qstart = o;
    o += al256(4 * (size_t)nbuckets);
    L.ioff = o;
    o += al256(8 * ((size_t)nbuckets + 1));
    L.segcnt = o;
    o += al256(4 * (size_t)nseg * (size_t)nstripe);
    L.slot = o;
    o += al256(4 * (size_t)rows);
    L.key = o;
    o += al256(4 * (size_t)rows);
    L.perm = o;
    o += al256(4 * (size_t)rows);
    L.tmp = o;
    o += al256(8 * (size_t)rows);
    L.items = o;
    o += al256(sizeof(Item) * (size_t)max_items);
    L.ctr = o;
    o += 256;
    L.total = o;
    return L;
}

// One launch class: the row-ordering pre-pass and the stacking kernel (or
// the FP64 kernel).
cudaError_t launch_class(vista_stack *h, const ClassRun &cr, cudaStream_t st)
{
    const bool fp64 = h->desc.precision == VISTA_PREC_FP64;
    const LaunchCfg cfg = h->cfg;
    cudaError_t e = cudaSuccess;
    {
        const RunArgs &a = cr.args;
        if (a.rot && fp64) {
            // gridding baselines of the re-projected windows (the mixed path
            // forms them in its pre-pass)
            const int sp = span_begin(h, 0);
            e = launch_rotate(a, st);
            span_end(h, sp);
            if (h->timing) h->tacc.launches += 1;
            if (e != cudaSuccess) return e;
        }
        if (fp64) {
            const int sp = span_begin(h, 1);
            e = launch_fp64(a, st);
            span_end(h, sp);
            if (h->timing) h->tacc.launches += 1;
        } else {
            int sp = span_begin(h, 0);
            int nk = 0;
            e = launch_prepare(a, st, &nk);
            span_end(h, sp);
            if (h->timing) h->tacc.launches += nk;
            if (e == cudaSuccess) {
                sp = span_begin(h, 1);
                e = launch_mixed(a, cr.key, cfg.warps_per_cta, cfg.prefetch_rows, st);
                span_end(h, sp);
                if (h->timing) h->tacc.launches += 1;
            }
        }
    }
    return e;
}

// The device work of a planned run without host-memory windows: flag
// repacking copies, then every launch class.  The same sequence is launched
// directly or captured in a graph.
cudaError_t device_pass(vista_stack *h, cudaStream_t st)
{
    cudaError_t e = cudaSuccess;
    for (const Copy2D &cp : h->copies) {
        e = cudaMemcpy2DAsync(cp.dst, cp.dpitch, cp.src, cp.spitch, cp.width, cp.height, cudaMemcpyDeviceToDevice,
                              st);
        if (e != cudaSuccess) return e;
    }
    for (const ClassRun &cr : h->classes)
        if ((e = launch_class(h, cr, st)) != cudaSuccess) return e;
    return cudaSuccess;
}

// A run with host-memory windows, streamed wave by wave: the copies of wave
// w go on the copy streams into staging slot w mod 2 once the wave that used
// the slot before has been stacked; the handle's stream waits for them and
// stacks the wave's classes.  So the copies of wave w + 1 overlap the
// stacking of wave w, and nothing waits on the host.
cudaError_t streamed_pass(vista_stack *h)
{
    // the copy streams first wait for work already queued (an earlier run
    // may still read the staging buffer)
    cudaError_t e = xfer_fork(h);
    for (int j = 0; j < 2 && e == cudaSuccess; ++j)
        if (!h->slot_ev[j]) e = cudaEventCreateWithFlags(&h->slot_ev[j], cudaEventDisableTiming);
    for (const Copy2D &cp : h->copies) {
        if (e != cudaSuccess) break;
        e = cudaMemcpy2DAsync(cp.dst, cp.dpitch, cp.src, cp.spitch, cp.width, cp.height, cudaMemcpyDeviceToDevice,
                              h->stream);
    }
    size_t ci = 0;
    for (int w = 0; w < h->nwaves && e == cudaSuccess; ++w) {
        const int slot = w & 1;
        for (int j = 0; j < NXFER && e == cudaSuccess && w >= 2; ++j)
            e = cudaStreamWaitEvent(h->xfer[j], h->slot_ev[slot], 0);
        int k = 0;
        for (const HostCopy &c : h->hcopies) {
            if (c.wave != w || e != cudaSuccess) continue;
            const cudaStream_t cs = h->xfer[k++ % NXFER];
            if (c.width == c.spitch && c.width == c.dpitch)
                e = cudaMemcpyAsync(c.dst, c.src, c.width * c.height, cudaMemcpyHostToDevice, cs);
            else
                e = cudaMemcpy2DAsync(c.dst, c.dpitch, c.src, c.spitch, c.width, c.height, cudaMemcpyHostToDevice, cs);
        }
        if (e == cudaSuccess) e = xfer_join(h);   // the stream waits for this wave's copies
        while (e == cudaSuccess && ci < h->classes.size() && h->classes[ci].wave == w)
            e = launch_class(h, h->classes[ci++], h->stream);
        if (e == cudaSuccess) e = cudaEventRecord(h->slot_ev[slot], h->stream);
    }
    return e;
}

// Everything the plan of a run depends on, as bytes: the cube and lattice,
// the launch configuration, and per window its arrays, shape, position,
// re-projection, redshift, pol map and frequencies (by digest).
template <typename T>
void put(std::vector<uint8_t> &v, const T &x)
{
    const uint8_t *p = reinterpret_cast<const uint8_t *>(&x);
    v.insert(v.end(), p, p + sizeof(T));
}
std::vector<uint8_t> run_signature(const vista_stack *h)
{
    std::vector<uint8_t> v;
    v.reserve(64 + h->pending.size() * 128);
    put(v, h->f0);
    put(v, h->df);
    put(v, h->cfg);
    put(v, h->pending.size());
    for (const SrcHost &s : h->pending) {
        put(v, s.d.nrow);
        put(v, s.d.nchan);
        put(v, s.d.npol);
        put(v, s.d.uvw);
        put(v, s.d.vis);
        put(v, s.d.vis_type);
        put(v, s.d.vis_scale);
        put(v, s.d.weights);
        put(v, s.d.flags);
        put(v, s.d.mem);
        put(v, s.d.l);
        put(v, s.d.m);
        put(v, s.d.z);
        put(v, s.freq_digest);
        put(v, s.has_rot);
        if (s.has_rot) put(v, s.rot);
        for (int32_t p : s.pol_map) put(v, p);
    }
    return v;
}

}  // namespace

// The mixed cube's FP32 partials are folded into the FP64 master once the
// visibilities stacked since the last fold reach FOLD_DEPTH per cube entry:
// an entry's FP32 sum then holds at most the contributions of one such
// interval (and, inside it, those since the entry's last checkpoint), so its
// rounding does not grow with the depth of the stack.  A fold reads the
// float4 cube once and the master entries of the touched entries (about
// 16 + 80 x touched / entries bytes per entry): at 64 visibilities per entry
// between folds, below 2 bytes per 9-byte visibility.
constexpr uint64_t FOLD_DEPTH = 64;

static cudaError_t after_run(vista_stack *h, uint64_t nvis)
{
    if (h->desc.precision == VISTA_PREC_FP64 || !h->cube_master) return cudaSuccess;
    h->nvis_since_fold += nvis;
    if (h->nvis_since_fold < FOLD_DEPTH * (uint64_t)h->nentries) return cudaSuccess;
    h->nvis_since_fold = 0;
    if (h->timing) h->tacc.launches += 1;
    return launch_fold(h->cube, h->cube_master, h->nentries, h->stream);
}

extern "C" int vista_run(vista_stack *h)
{
    if (!handle_live(h)) return fail(nullptr, VISTA_E_STATE, "unknown or closed handle");
    if (h->pending.empty()) return fail(h, VISTA_E_STATE, "vista_run with no queued source");
    const vista_cube_desc &c = h->desc;
    const bool fp64 = c.precision == VISTA_PREC_FP64;
    cudaError_t e;

    // 0. an unchanged source set replays the device pass from a graph (not
    //    while timing spans are recorded; host-memory windows never match)
    std::vector<uint8_t> sig = run_signature(h);
    if (h->graphs && !h->timing && h->plan_valid && sig == h->plan_sig) {
        if (!h->gexec) {
            if (!h->cap_stream && (e = cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking)) != cudaSuccess)
                return cuda_fail(h, e, "capture stream");
            cudaGraph_t graph = nullptr;
            e = cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                const cudaError_t e1 = device_pass(h, h->cap_stream);
                e = cudaStreamEndCapture(h->cap_stream, &graph);
                if (e1 != cudaSuccess) e = e1;
            }
            if (e == cudaSuccess) e = cudaGraphInstantiate(&h->gexec, graph, 0);
            if (graph) cudaGraphDestroy(graph);
            if (e != cudaSuccess) {
                h->gexec = nullptr;
                h->plan_valid = false;
                return cuda_fail(h, e, "graph capture of the device pass");
            }
        }
        if ((e = cudaGraphLaunch(h->gexec, h->stream)) != cudaSuccess) return cuda_fail(h, e, "graph launch");
        if ((e = after_run(h, h->plan_nvis)) != cudaSuccess) return cuda_fail(h, e, "cube fold");
        ++h->graph_launches;
        h->host_nvis += h->plan_nvis;
        h->last = std::move(h->pending);
        h->pending.clear();
        return VISTA_OK;
    }

    // 1. the rest lattice (fixed at the first run)
    double f0 = h->f0, df = h->df;
    if (!h->lattice_fixed) {
        double best = 0.0;
        for (const SrcHost &s : h->pending) {
            if (s.d.nchan < 2)
                return fail(h, VISTA_E_ARG, "the automatic rest lattice needs >= 2 channels per window");
            const double wdt = widest_rest_channel(s.freqs.data(), s.d.nchan, s.d.z);
            if (wdt > best) best = wdt;
        }
        if (!(best > 0.0)) return fail(h, VISTA_E_ARG, "automatic rest lattice: zero channel width");
        df = best;
        f0 = lattice_f0(c.central_freq, c.nrest, best);
    }
    const double saved_f0 = h->f0, saved_df = h->df;
    h->f0 = f0;
    h->df = df;

    // 2. channel tables
    const double gu = 1.0 / (C_LIGHT * c.du), gv = 1.0 / (C_LIGHT * c.dv);
    const int nsrc = (int)h->pending.size();
    std::vector<Plan> plans((size_t)nsrc);
    for (int i = 0; i < nsrc; ++i) {
        const int rc = plan_source(h, h->pending[(size_t)i], gu, gv, plans[(size_t)i]);
        if (rc != VISTA_OK) {
            h->f0 = saved_f0;
            h->df = saved_df;
            return rc;
        }
    }
    h->lattice_fixed = true;

    // 3. waves of host-memory windows (by staged bytes, about a quarter of
    //    them each, 64 MB to 2 GB), then the launch classes, wave by wave
    //    (windows with no row or no channel in the cube are skipped)
    // A host window's flags are staged as whole rows with one contiguous copy
    // when its rows are whole words and not much wider than the channels
    // read (or the whole array is small): a 2-D copy of narrow rows runs far
    // below the host link's rate.  The kernel then reads them at the
    // in-cube channel offset.
    auto full_flag_rows = [&](int i) {
        const SrcHost &s = h->pending[(size_t)i];
        const int32_t nin = plans[(size_t)i].k_hi - plans[(size_t)i].k_lo;
        const size_t row_in = (size_t)s.d.nchan * (size_t)s.d.npol, fp = (size_t)flag_pitch(nin, s.d.npol);
        return s.d.flags && row_in % 4 == 0 && (row_in <= 4 * fp || (size_t)s.d.nrow * row_in <= ((size_t)16 << 20));
    };
    auto staged_bytes = [&](int i) {
        const SrcHost &s = h->pending[(size_t)i];
        const size_t nr = (size_t)s.d.nrow;
        const int32_t nin = plans[(size_t)i].k_hi - plans[(size_t)i].k_lo;
        const size_t fbytes = !s.d.flags ? 0
                              : full_flag_rows(i) ? al256(nr * (size_t)s.d.nchan * (size_t)s.d.npol)
                                                  : al256(nr * (size_t)flag_pitch(nin, s.d.npol));
        return al256(nr * 24) + al256(nr * (size_t)nin * (size_t)s.d.npol * vis_elem_bytes(s.d.vis_type)) +
               al256(nr * 4 * (size_t)s.d.npol) + fbytes;
    };
    auto in_cube = [&](int i) {
        return h->pending[(size_t)i].d.nrow > 0 && plans[(size_t)i].k_hi > plans[(size_t)i].k_lo;
    };
    std::vector<int> wave_of((size_t)nsrc, 0);
    int nwaves = 0;
    size_t slot_bytes = 0;
    {
        size_t host_total = 0;
        for (int i = 0; i < nsrc; ++i)
            if (h->pending[(size_t)i].d.mem == VISTA_MEM_HOST && in_cube(i)) host_total += staged_bytes(i);
        const size_t budget = h->wave_bytes > 0 ? (size_t)h->wave_bytes
                                                : std::max((size_t)64 << 20, std::min((size_t)2 << 30, host_total / 4));
        size_t cur = 0;
        for (int i = 0; i < nsrc; ++i) {
            if (h->pending[(size_t)i].d.mem != VISTA_MEM_HOST || !in_cube(i)) continue;
            const size_t b = staged_bytes(i);
            if (nwaves == 0 || (cur > 0 && cur + b > budget)) {
                ++nwaves;
                cur = 0;
            }
            wave_of[(size_t)i] = nwaves - 1;
            cur += b;
            slot_bytes = std::max(slot_bytes, cur);
        }
    }
    const LaunchCfg cfg = h->cfg;
    std::vector<ClassRun> classes;
    std::vector<int> ns_of((size_t)nsrc, 1);
    for (int i = 0; i < nsrc; ++i) {
        const SrcHost &s = h->pending[(size_t)i];
        const Plan &pl = plans[(size_t)i];
        if (s.d.nrow == 0 || pl.k_hi <= pl.k_lo) continue;
        // four pols x four channels per lane does not fit the register budget
        const int cap = s.d.npol == 4 ? std::min(2, (int)cfg.chans_per_lane) : (int)cfg.chans_per_lane;
        const int ns = fp64 ? 1 : choose_ns(pl.k_hi - pl.k_lo, cap);
        ns_of[(size_t)i] = ns;
        const int key = fp64 ? 0 : ((s.d.vis_type << 16) | (ns << 8) | s.d.npol);
        const int wv = wave_of[(size_t)i];
        int ci = -1;
        for (size_t j = 0; j < classes.size(); ++j)
            if (classes[j].key == key && classes[j].wave == wv) ci = (int)j;
        if (ci < 0) {
            classes.emplace_back();
            classes.back().key = key;
            classes.back().ns = ns;
            classes.back().wave = wv;
            ci = (int)classes.size() - 1;
        }
        classes[(size_t)ci].members.push_back(i);
    }
    std::stable_sort(classes.begin(), classes.end(),
                     [](const ClassRun &x, const ClassRun &y) { return x.wave < y.wave; });
    std::vector<ChanF> chf;
    std::vector<ChanD> chd;
    std::vector<int32_t> chan_off((size_t)nsrc);
    for (int i = 0; i < nsrc; ++i) {
        chan_off[(size_t)i] = (int32_t)chf.size();
        chf.insert(chf.end(), plans[(size_t)i].chf.begin(), plans[(size_t)i].chf.end());
        chd.insert(chd.end(), plans[(size_t)i].chd.begin(), plans[(size_t)i].chd.end());
    }
    if (chf.size() > (size_t)0x7fffffff) return fail(h, VISTA_E_RANGE, "too many channels in one run");

    // 4. staging layout: two slots for the waves of host-memory windows (the
    //    channels read only), then the flags of device windows the mixed
    //    path cannot read in words
    auto repack_flags = [&](const SrcHost &s) {
        return !fp64 && s.d.mem == VISTA_MEM_DEVICE && s.d.flags && !flags_direct(s.d.flags, s.d.nchan, s.d.npol);
    };
    const size_t host_region = slot_bytes * (size_t)(nwaves >= 2 ? 2 : nwaves);
    size_t stage_bytes = host_region;
    for (const ClassRun &cr : classes)
        for (int i : cr.members) {
            const SrcHost &s = h->pending[(size_t)i];
            if (repack_flags(s)) {
                const int32_t nin = plans[(size_t)i].k_hi - plans[(size_t)i].k_lo;
                stage_bytes += al256((size_t)s.d.nrow * (size_t)flag_pitch(nin, s.d.npol));
            }
        }
    if (stage_bytes) {
        e = h->b_stage.ensure(stage_bytes);
        if (e != cudaSuccess) return cuda_fail(h, e, "staging allocation");
    }

    std::vector<SrcDev> sdev;
    std::vector<double> rots;   // 9 per re-projected window (SrcDev::rot1 - 1 indexes them)
    std::vector<char> cls_rot(classes.size(), 0);
    // gridding baselines of the re-projected windows (filled by k_rotate)
    int64_t rot_rows = 0, guvw_pos = 0;
    for (const SrcHost &s : h->pending)
        if (s.has_rot) rot_rows += s.d.nrow;
    if (rot_rows > 0 && (e = h->b_guvw.ensure((size_t)rot_rows * 24)) != cudaSuccess)
        return cuda_fail(h, e, "re-projection buffer allocation");
    std::vector<int64_t> offs;
    std::vector<size_t> cls_src0(classes.size()), cls_off0(classes.size());
    std::vector<SortLayout> layouts(classes.size());
    size_t sort_bytes = 0;
    int64_t rec_total = 0, cell_total = 0;
    uint64_t nvis_run = 0;
    std::vector<Copy2D> copies;
    std::vector<HostCopy> hcopies;
    std::vector<size_t> wave_pos((size_t)std::max(nwaves, 1), 0);   // next free byte of each wave's slot
    size_t stage_pos = host_region;                                  // the repacked flags follow the slots
    for (size_t ci = 0; ci < classes.size(); ++ci) {
        ClassRun &cr = classes[ci];
        const int cw = 32 * cr.ns;
        cls_src0[ci] = sdev.size();
        cls_off0[ci] = offs.size();
        const size_t m = cr.members.size();
        std::vector<int64_t> roff(m + 1, 0), soff(m + 1, 0);
        int64_t max_items = 0;
        for (size_t t = 0; t < m; ++t) {
            const int i = cr.members[t];
            const SrcHost &s = h->pending[(size_t)i];
            const Plan &pl = plans[(size_t)i];
            const int32_t nin = pl.k_hi - pl.k_lo;
            SrcDev d{};
            d.uvw = s.d.uvw;
            d.vis = s.d.vis;
            d.wts = s.d.weights;
            d.vstride = s.d.nchan;
            d.kbase = 0;
            d.fbase = s.d.flags;
            d.fpitch = (int64_t)s.d.nchan * s.d.npol;
            d.fk0 = 0;
            if (s.d.mem == VISTA_MEM_HOST) {
                // staged in its wave's slot; the copies are issued by streamed_pass
                const int wv = wave_of[(size_t)i];
                const size_t nr = (size_t)s.d.nrow, P = (size_t)s.d.npol;
                const size_t esz = vis_elem_bytes(s.d.vis_type);
                const size_t nvv = nr * (size_t)nin * P;
                char *base = (char *)h->b_stage.p + (size_t)(wv & 1) * slot_bytes;
                size_t &pos = wave_pos[(size_t)wv];
                char *p_uvw = base + pos;
                pos += al256(nr * 24);
                char *p_vis = base + pos;
                pos += al256(nvv * esz);
                char *p_w = base + pos;
                pos += al256(nr * 4 * P);
                char *p_f = nullptr;
                const size_t row_in = (size_t)s.d.nchan * P, row_out = (size_t)nin * P;
                const bool whole = full_flag_rows(i);
                const size_t fp = whole ? row_in : (size_t)flag_pitch(nin, s.d.npol);
                if (s.d.flags) {
                    p_f = base + pos;
                    pos += al256(nr * fp);
                }
                hcopies.push_back(HostCopy{wv, p_uvw, nr * 24, s.d.uvw, nr * 24, nr * 24, 1});
                hcopies.push_back(HostCopy{wv, p_vis, row_out * esz, (const char *)s.d.vis + (size_t)pl.k_lo * P * esz,
                                           row_in * esz, row_out * esz, nr});
                hcopies.push_back(HostCopy{wv, p_w, nr * 4 * P, s.d.weights, nr * 4 * P, nr * 4 * P, 1});
                if (p_f && whole)
                    hcopies.push_back(HostCopy{wv, p_f, nr * row_in, s.d.flags, nr * row_in, nr * row_in, 1});
                else if (p_f)
                    hcopies.push_back(HostCopy{wv, p_f, fp, s.d.flags + (size_t)pl.k_lo * P, row_in, row_out, nr});
                d.uvw = (const double *)p_uvw;
                d.vis = p_vis;
                d.wts = (const float *)p_w;
                d.vstride = nin;
                d.kbase = pl.k_lo;
                d.fbase = (const uint8_t *)p_f;
                d.fpitch = (int64_t)fp;
                d.fk0 = whole ? 0 : pl.k_lo;
            } else if (repack_flags(s)) {
                const size_t nr = (size_t)s.d.nrow, P = (size_t)s.d.npol;
                const size_t fp = (size_t)flag_pitch(nin, s.d.npol);
                char *p_f = (char *)h->b_stage.p + stage_pos;
                stage_pos += al256(nr * fp);
                copies.push_back(Copy2D{p_f, fp, s.d.flags + (size_t)pl.k_lo * P, (size_t)s.d.nchan * P,
                                        (size_t)nin * P, nr});
                d.fbase = (const uint8_t *)p_f;
                d.fpitch = (int64_t)fp;
                d.fk0 = pl.k_lo;
            }
            d.nrow = s.d.nrow;
            d.nchan = s.d.nchan;
            d.npol = s.d.npol;
            d.vis_type = s.d.vis_type;
            d.vis_scale = (s.d.vis_type == VISTA_VIS_F16X2 || s.d.vis_type == VISTA_VIS_BF16X2) ? s.d.vis_scale : 1.0f;
            d.l = s.d.l;
            d.m = s.d.m;
            d.n1 = std::sqrt(1.0 - s.d.l * s.d.l - s.d.m * s.d.m) - 1.0;
            d.step_c = pl.step / C_LIGHT;
            d.k_lo = pl.k_lo;
            d.k_hi = pl.k_hi;
            d.chan_off = chan_off[(size_t)i];
            d.linear = pl.linear ? 1 : 0;
            for (int p = 0; p < 4; ++p) d.plane[p] = p < s.d.npol ? s.pol_map[(size_t)p] : -1;
            d.nchunk = (nin + cw - 1) / cw;
            d.key_su = (float)(s.freqs[(size_t)pl.key_ch] * gu);
            d.key_sv = (float)(s.freqs[(size_t)pl.key_ch] * gv);
            d.rec_off = rec_total;
            d.cell_off = cell_total;
            if (!fp64) {
                rec_total += d.nrow;
                cell_total += d.nrow * d.nchunk;
            }
            {
                int64_t nread = 0, npm = 0;
                for (const ChanF &f : pl.chf) nread += f.nb > 0;
                for (int p = 0; p < s.d.npol; ++p) npm += s.pol_map[(size_t)p] >= 0;
                nvis_run += (uint64_t)(d.nrow * nread * npm);
            }
            roff[t + 1] = roff[t] + d.nrow;
            soff[t + 1] = soff[t] + (fp64 ? 0 : (d.nrow + SEG_ROWS - 1) / SEG_ROWS);
            max_items += (int64_t)d.nchunk * ((d.nrow + cfg.rows_per_item - 1) / cfg.rows_per_item + h->nstripe);
            d.guvw = d.uvw;
            if (s.has_rot) {
                d.rot1 = (int32_t)(rots.size() / 9) + 1;
                rots.insert(rots.end(), s.rot, s.rot + 9);
                d.guvw = (const double *)h->b_guvw.p + 3 * guvw_pos;
                guvw_pos += d.nrow;
                cls_rot[ci] = 1;
            }
            sdev.push_back(d);
        }
        offs.insert(offs.end(), roff.begin(), roff.end());
        offs.insert(offs.end(), soff.begin(), soff.end());
        cr.args.so.nseg_total = soff[m];
        cr.args.nsrc = (int32_t)m;
        cr.args.cw = cw;
        cr.args.nrows_total = roff[m];
        const int nst = cfg.sort_rows ? h->nstripe : 1;
        layouts[ci] = sort_layout(roff[m], (int64_t)m * nst, max_items, soff[m], nst);
        cr.args.so.max_items = max_items;
        sort_bytes = std::max(sort_bytes, layouts[ci].total);
    }

    // uploads and buffers
    Uploader up{h};
    if ((e = up.begin(upload_bytes(sdev) + upload_bytes(chf) + upload_bytes(chd) + upload_bytes(offs) +
                      upload_bytes(rots))) != cudaSuccess)
        return cuda_fail(h, e, "pinned staging of the tables");
    if ((e = up.put(h->b_srcs, sdev)) != cudaSuccess) return cuda_fail(h, e, "source table upload");
    if ((e = up.put(h->b_chf, chf)) != cudaSuccess) return cuda_fail(h, e, "channel table upload");
    if ((e = up.put(h->b_chd, chd)) != cudaSuccess) return cuda_fail(h, e, "channel table upload");
    if ((e = up.put(h->b_off, offs)) != cudaSuccess) return cuda_fail(h, e, "offset table upload");
    if (!rots.empty() && (e = up.put(h->b_rot, rots)) != cudaSuccess)
        return cuda_fail(h, e, "re-projection table upload");
    if ((e = up.end()) != cudaSuccess) return cuda_fail(h, e, "pinned staging of the tables");
    if (!fp64) {
        if ((e = h->b_recs.ensure((size_t)(rec_total > 0 ? rec_total : 1) * sizeof(RowRec))) != cudaSuccess)
            return cuda_fail(h, e, "row record allocation");
        // padding: the bulk copy of an item's chunk cells starts and ends on
        // 16-byte boundaries, up to one entry past the last
        if ((e = h->b_cells.ensure((size_t)(cell_total + 4) * sizeof(int2))) != cudaSuccess)
            return cuda_fail(h, e, "chunk cell allocation");
        if ((e = h->b_sort.ensure(sort_bytes > 0 ? sort_bytes : 256)) != cudaSuccess)
            return cuda_fail(h, e, "ordering buffer allocation");
    }

    // 5. launch arguments, then the device pass
    const CubeGeom g{c.nu, c.nv, c.nrest, c.npol, gu, gv, c.hermitian_fold, 0};
    for (size_t ci = 0; ci < classes.size(); ++ci) {
        ClassRun &cr = classes[ci];
        RunArgs &a = cr.args;
        a.srcs = (const SrcDev *)h->b_srcs.p + cls_src0[ci];
        a.chf = (const ChanF *)h->b_chf.p;
        a.chd = (const ChanD *)h->b_chd.p;
        a.recs = (RowRec *)h->b_recs.p;
        a.rot = cls_rot[ci] ? (const double *)h->b_rot.p : nullptr;
        a.ccells = (int2 *)h->b_cells.p;
        a.row_off = (const int64_t *)h->b_off.p + cls_off0[ci];
        a.so.seg_off = a.row_off + cr.members.size() + 1;
        a.g = g;
        a.cube = h->cube;
        a.cube_master = h->cube_master;
        a.comp = h->cube_master ? 1 : 0;
        a.count = h->count;
        a.stats = h->stats;
        a.err = h->err;
        if (!fp64) {
            SortArgs &so = a.so;
            const SortLayout &L = layouts[ci];
            char *b = (char *)h->b_sort.p;
            so.hist = (uint32_t *)(b + L.hist);
            so.qstart = (uint32_t *)(b + L.qstart);
            so.ioff = (int64_t *)(b + L.ioff);
            so.segcnt = (uint32_t *)(b + L.segcnt);
            so.slot = (uint32_t *)(b + L.slot);
            so.key = (uint32_t *)(b + L.key);
            so.perm = (uint32_t *)(b + L.perm);
            so.tmp = (unsigned long long *)(b + L.tmp);
            so.items = (Item *)(b + L.items);
            so.ctr = (uint32_t *)(b + L.ctr);
            so.sorted = cfg.sort_rows;
            so.stripe_rows = cfg.sort_rows ? h->stripe_rows : c.nv;
            so.nstripe = cfg.sort_rows ? h->nstripe : 1;
            so.ushift = h->ushift;
            so.nuk = h->nuk;
            so.rows_per_item = cfg.rows_per_item;
        }
    }
    h->classes = std::move(classes);
    h->copies = std::move(copies);
    h->hcopies = std::move(hcopies);
    h->nwaves = nwaves;
    bool any_host = false;
    for (const SrcHost &s : h->pending) any_host |= s.d.mem == VISTA_MEM_HOST;
    // host-memory windows: streamed wave by wave (their arrays must stay valid
    // until this stream work completes); otherwise the device pass at once
    if ((e = (nwaves > 0 ? streamed_pass(h) : device_pass(h, h->stream))) != cudaSuccess) {
        h->plan_valid = false;
        return cuda_fail(h, e, "kernel launch or host-to-device copy");
    }
    if ((e = after_run(h, nvis_run)) != cudaSuccess) {
        h->plan_valid = false;
        return cuda_fail(h, e, "cube fold");
    }
    if (h->timing) h->tacc.runs += 1;
    h->host_nvis += nvis_run;
    // the device tables now hold this source set's plan: an unchanged set is
    // replayed from a graph of the device pass next time
    drop_graph(h);
    h->plan_valid = !any_host;
    h->plan_sig = run_signature(h);   // with the lattice as now fixed
    h->plan_nvis = nvis_run;
    h->last = std::move(h->pending);
    h->pending.clear();
    return VISTA_OK;
}

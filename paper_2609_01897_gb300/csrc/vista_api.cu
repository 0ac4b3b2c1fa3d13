// libvista C ABI: handle life cycle, validation, readback, counters, timing
// and debug exports (vista_run lives in vista_run.cu).  The contract of
// every call is in include/vista.h.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <set>

#include "vista_handle.h"

using namespace vista;

namespace {

thread_local std::string g_err;
std::mutex g_mu;
std::set<const vista_stack *> g_live;

bool is_fin(double x) { return std::isfinite(x); }

#define CHECK_HANDLE(h)                                                                \
    do {                                                                               \
        if (!handle_live(h)) return fail(nullptr, VISTA_E_STATE, "unknown or closed handle"); \
    } while (0)

// Row-ordering stripes: a few iv rows of the cube whose FP32 entries fit in
// about 40 MB, so the cube region a stripe's work touches stays in L2; the
// cell key inside a stripe must fit the shared-memory histogram.
int stripe_geometry(vista_stack *h)
{
    const vista_cube_desc &d = h->desc;
    int S = 1, nst = 1, ushift = 0, nuk = 1;
    if (!stripe_layout(d.nu, d.nv, d.nrest, d.npol, &S, &nst, &ushift, &nuk)) return VISTA_E_RANGE;
    h->stripe_rows = S;
    h->nstripe = nst;
    h->ushift = ushift;
    h->nuk = nuk;
    return VISTA_OK;
}

}  // namespace

namespace vista {

bool handle_live(const vista_stack *h)
{
    std::lock_guard<std::mutex> lk(g_mu);
    return h && g_live.count(h) != 0;
}

int fail(vista_stack *h, int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (h)
        h->msg = buf;
    else
        g_err = buf;
    return code;
}

int cuda_fail(vista_stack *h, cudaError_t e, const char *what)
{
    // a failed allocation or launch also leaves its code as the thread's last
    // CUDA error; cleared here, so that it cannot surface later in the
    // caller's own launch checks or in this library's next call (a sticky
    // error that ruined the context stays whatever this does)
    (void)cudaGetLastError();
    return fail(h, e == cudaErrorMemoryAllocation ? VISTA_E_NOMEM : VISTA_E_CUDA, "%s: %s", what,
                cudaGetErrorString(e));
}

int device_fail(vista_stack *h, int32_t code)
{
    if (code == 1) return fail(h, VISTA_E_TIMEOUT, "a device-side wait gave up (code 1)");
    return fail(h, VISTA_E_STATE, "a device-side check failed (code %d)", code);
}

static cudaEvent_t take_event(vista_stack *h)
{
    if (!h->ev_pool.empty()) {
        cudaEvent_t e = h->ev_pool.back();
        h->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

int span_begin(vista_stack *h, int kind)
{
    if (!h->timing) return -1;
    cudaEvent_t a = take_event(h), b = take_event(h);
    if (!a || !b) return -1;
    cudaEventRecord(a, h->stream);
    h->spans.push_back({a, b, kind});
    return (int)h->spans.size() - 1;
}

void span_end(vista_stack *h, int id)
{
    if (id >= 0) cudaEventRecord(h->spans[(size_t)id].b, h->stream);
}

uint64_t freq_digest(const double *f, size_t n)
{
    // FNV-1a's xor-multiply step on whole 64-bit words, four independent
    // lanes (no serial chain through every byte): each step is a bijection of
    // the lane state, so a single changed word always changes the digest
    uint64_t h[4] = {1469598103934665603ull, 0x9e3779b97f4a7c15ull, 0xc2b2ae3d27d4eb4full, 0x165667b19e3779f9ull};
    for (size_t i = 0; i < n; ++i) {
        uint64_t w;
        std::memcpy(&w, f + i, sizeof w);
        h[i & 3] = (h[i & 3] ^ w) * 1099511628211ull;
    }
    uint64_t d = n;
    for (int k = 0; k < 4; ++k) d = (d ^ h[k] ^ (h[k] >> 29)) * 0xbf58476d1ce4e5b9ull;
    return d;
}

cudaError_t xfer_fork(vista_stack *h)
{
    cudaError_t e = cudaSuccess;
    for (int j = 0; j < NXFER && e == cudaSuccess; ++j)
        if (!h->xfer[j]) e = cudaStreamCreateWithFlags(&h->xfer[j], cudaStreamNonBlocking);
    for (int j = 0; j <= NXFER && e == cudaSuccess; ++j)
        if (!h->xfer_ev[j]) e = cudaEventCreateWithFlags(&h->xfer_ev[j], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(h->xfer_ev[NXFER], h->stream);
    for (int j = 0; j < NXFER && e == cudaSuccess; ++j) e = cudaStreamWaitEvent(h->xfer[j], h->xfer_ev[NXFER], 0);
    return e;
}

cudaError_t xfer_join(vista_stack *h)
{
    cudaError_t e = cudaSuccess;
    for (int j = 0; j < NXFER && e == cudaSuccess; ++j) {
        e = cudaEventRecord(h->xfer_ev[j], h->xfer[j]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(h->stream, h->xfer_ev[j], 0);
    }
    return e;
}

void drop_graph(vista_stack *h)
{
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    h->gexec = nullptr;
}

size_t vis_elem_bytes(int vt)
{
    switch (vt) {
    case VISTA_VIS_C64: return 8;
    case VISTA_VIS_C128: return 16;
    default: return 4;
    }
}

}  // namespace vista

// ------------------------------------------------------------------ open

extern "C" int vista_abi_version(void) { return VISTA_ABI_VERSION; }

extern "C" int vista_open_stack(const vista_cube_desc *d, vista_stack **out)
{
    if (out) *out = nullptr;
    if (!d || !out) return fail(nullptr, VISTA_E_ARG, "null descriptor or output pointer");
    if (d->nu < 2 || d->nv < 2 || (d->nu & 1) || (d->nv & 1))
        return fail(nullptr, VISTA_E_ARG, "nu and nv must be even and >= 2 (got %d, %d)", d->nu, d->nv);
    if (d->nrest < 1) return fail(nullptr, VISTA_E_ARG, "nrest must be >= 1");
    if (d->npol < 1 || d->npol > VISTA_MAX_POL) return fail(nullptr, VISTA_E_ARG, "npol must be 1..4");
    if (!(d->du > 0.0) || !(d->dv > 0.0) || !is_fin(d->du) || !is_fin(d->dv))
        return fail(nullptr, VISTA_E_ARG, "du and dv must be finite and > 0");
    if (!(d->rest_df >= 0.0) || !is_fin(d->rest_df))
        return fail(nullptr, VISTA_E_ARG, "rest_df must be finite and >= 0");
    if (d->rest_df > 0.0 && !is_fin(d->rest_f0)) return fail(nullptr, VISTA_E_ARG, "rest_f0 must be finite");
    if (d->rest_df == 0.0 && !(is_fin(d->central_freq) && d->central_freq > 0.0))
        return fail(nullptr, VISTA_E_ARG, "central_freq must be finite and > 0 when rest_df == 0");
    if (d->bin_mode != VISTA_BIN_OVERLAP && d->bin_mode != VISTA_BIN_NEAREST)
        return fail(nullptr, VISTA_E_ARG, "bad bin_mode %d", d->bin_mode);
    if (d->precision != VISTA_PREC_MIXED && d->precision != VISTA_PREC_FP64)
        return fail(nullptr, VISTA_E_ARG, "bad precision %d", d->precision);
    if (d->hermitian_fold != 0 && d->hermitian_fold != 1)
        return fail(nullptr, VISTA_E_ARG, "hermitian_fold must be 0 or 1");
    const int64_t ncell = (int64_t)d->nu * d->nv;
    if (ncell > (int64_t)0x7fffffff) return fail(nullptr, VISTA_E_RANGE, "nu*nv exceeds 2^31-1");
    const int64_t n = ncell * d->nrest * d->npol;

    vista_stack *h = new (std::nothrow) vista_stack();
    if (!h) return fail(nullptr, VISTA_E_NOMEM, "host allocation failed");
    h->desc = *d;
    h->stream = (cudaStream_t)d->stream;
    h->nentries = n;
    if (d->rest_df > 0.0) {
        h->lattice_fixed = true;
        h->f0 = d->rest_f0;
        h->df = d->rest_df;
    }
    if (stripe_geometry(h) != VISTA_OK) {
        delete h;
        return fail(nullptr, VISTA_E_RANGE, "cube too tall for the row ordering");
    }
    cudaError_t e = cudaGetDevice(&h->device);
    const bool fp64c = d->precision == VISTA_PREC_FP64;
    const size_t esz = fp64c ? 32 : 16;   // double[4] (FP64) or float4 (mixed, plus an FP64 master cube)
    if (e == cudaSuccess) e = cudaMalloc(&h->cube, (size_t)n * esz);
    if (e == cudaSuccess) e = cudaMalloc((void **)&h->count, (size_t)n * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMalloc((void **)&h->stats, sizeof(DevStats));
    if (e == cudaSuccess) e = cudaMalloc((void **)&h->err, sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMemsetAsync(h->cube, 0, (size_t)n * esz, h->stream);
    if (e == cudaSuccess && !fp64c) e = cudaMalloc((void **)&h->cube_master, (size_t)n * 32);
    if (e == cudaSuccess && !fp64c) e = cudaMemsetAsync(h->cube_master, 0, (size_t)n * 32, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->count, 0, (size_t)n * sizeof(uint32_t), h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->stats, 0, sizeof(DevStats), h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->err, 0, sizeof(int32_t), h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
        const int rc = cuda_fail(nullptr, e, "cube allocation");
        cudaFree(h->cube);
        cudaFree(h->cube_master);
        cudaFree(h->count);
        cudaFree(h->stats);
        cudaFree(h->err);
        delete h;
        return rc;
    }
    {
        std::lock_guard<std::mutex> lk(g_mu);
        g_live.insert(h);
    }
    *out = h;
    return VISTA_OK;
}

// ------------------------------------------------------------- add source

namespace {

// Validation and queueing shared by the two add calls; rot: the window's
// re-projection (row-major 3 x 3), or null.
int add_source_impl(vista_stack *h, const vista_source_desc *s, const double *rot)
{
    if (!s) return fail(h, VISTA_E_ARG, "null source descriptor");
    const vista_cube_desc &c = h->desc;
    if (s->nrow < 0) return fail(h, VISTA_E_ARG, "nrow must be >= 0");
    if (s->nrow > (int64_t)0x7fffffff) return fail(h, VISTA_E_RANGE, "nrow exceeds 2^31-1");
    if (s->nchan < 1) return fail(h, VISTA_E_ARG, "nchan must be >= 1");
    if (c.bin_mode == VISTA_BIN_OVERLAP && s->nchan < 2)
        return fail(h, VISTA_E_ARG, "overlap binning needs >= 2 channels (channel width from centred differences)");
    if (s->npol != 1 && s->npol != 2 && s->npol != 4) return fail(h, VISTA_E_ARG, "npol must be 1, 2 or 4");
    if (s->vis_type < VISTA_VIS_C64 || s->vis_type > VISTA_VIS_BF16X2)
        return fail(h, VISTA_E_ARG, "bad vis_type %d", s->vis_type);
    if ((s->vis_type == VISTA_VIS_F16X2 || s->vis_type == VISTA_VIS_BF16X2) &&
        !(std::isfinite(s->vis_scale) && s->vis_scale > 0.0f))
        return fail(h, VISTA_E_ARG, "vis_scale must be finite and > 0 for 16-bit visibilities");
    if (s->mem != VISTA_MEM_DEVICE && s->mem != VISTA_MEM_HOST) return fail(h, VISTA_E_ARG, "bad mem %d", s->mem);
    if (!s->freqs) return fail(h, VISTA_E_ARG, "freqs is NULL");
    if (s->nrow > 0 && (!s->uvw || !s->vis || !s->weights))
        return fail(h, VISTA_E_ARG, "uvw, vis and weights must be non-NULL when nrow > 0");
    if (!(is_fin(s->l) && is_fin(s->m) && s->l * s->l + s->m * s->m < 1.0))
        return fail(h, VISTA_E_ARG, "need finite l, m with l^2 + m^2 < 1");
    if (!(is_fin(s->z) && s->z > -1.0)) return fail(h, VISTA_E_ARG, "need finite z > -1");
    if ((int64_t)s->nrow * s->nchan > ((int64_t)1 << 40)) return fail(h, VISTA_E_RANGE, "window too large");
    for (int32_t k = 0; k < s->nchan; ++k) {
        const double f = s->freqs[k];
        if (!(is_fin(f) && f > 0.0)) return fail(h, VISTA_E_ARG, "freqs[%d] is not finite and > 0", k);
    }
    if (s->nchan >= 2) {
        const bool up = s->freqs[1] > s->freqs[0];
        for (int32_t k = 1; k < s->nchan; ++k) {
            const bool ok = up ? s->freqs[k] > s->freqs[k - 1] : s->freqs[k] < s->freqs[k - 1];
            if (!ok) return fail(h, VISTA_E_ARG, "freqs must be strictly monotone (index %d)", k);
        }
    }
    SrcHost sh;
    sh.d = *s;
    sh.freqs.assign(s->freqs, s->freqs + s->nchan);
    sh.freq_digest = freq_digest(sh.freqs.data(), sh.freqs.size());
    sh.pol_map.resize((size_t)s->npol);
    for (int p = 0; p < s->npol; ++p) {
        const int32_t q = s->pol_map ? s->pol_map[p] : p;
        if (q < -1 || q >= c.npol)
            return fail(h, VISTA_E_ARG, "pol %d maps to plane %d outside [-1, %d)", p, q, c.npol);
        sh.pol_map[(size_t)p] = q;
    }
    if (s->mem == VISTA_MEM_DEVICE && s->nrow > 0) {
        const size_t ve = vis_elem_bytes(s->vis_type) * (size_t)s->npol;
        const size_t va = ve < 16 ? ve : 16;
        if ((uintptr_t)s->vis % va) return fail(h, VISTA_E_ARG, "vis must be %zu-byte aligned", va);
        if ((uintptr_t)s->uvw % 8) return fail(h, VISTA_E_ARG, "uvw must be 8-byte aligned");
        if ((uintptr_t)s->weights % 4) return fail(h, VISTA_E_ARG, "weights must be 4-byte aligned");
        if (s->flags && ((uintptr_t)s->flags % (size_t)s->npol))
            return fail(h, VISTA_E_ARG, "flags must be %d-byte aligned", s->npol);
    }
    sh.d.freqs = nullptr;
    sh.d.pol_map = nullptr;
    if (rot) {
        sh.has_rot = true;
        std::memcpy(sh.rot, rot, sizeof sh.rot);
    }
    h->pending.push_back(std::move(sh));
    return VISTA_OK;
}

// Eq. 1's frames: the rows of M(ra, dec) are the unit vectors u (east),
// v (north) and w (toward (ra, dec)) in equatorial coordinates.
void uvw_frame(double ra, double dec, double M[3][3])
{
    M[0][0] = -std::sin(ra);
    M[0][1] = std::cos(ra);
    M[0][2] = 0.0;
    M[1][0] = -std::sin(dec) * std::cos(ra);
    M[1][1] = -std::sin(dec) * std::sin(ra);
    M[1][2] = std::cos(dec);
    M[2][0] = std::cos(dec) * std::cos(ra);
    M[2][1] = std::cos(dec) * std::sin(ra);
    M[2][2] = std::sin(dec);
}

}  // namespace

extern "C" int vista_add_source(vista_stack *h, const vista_source_desc *s)
{
    CHECK_HANDLE(h);
    return add_source_impl(h, s, nullptr);
}

extern "C" int vista_add_source_reproject(vista_stack *h, const vista_source_desc *s, double ra0, double dec0,
                                          double ra1, double dec1)
{
    CHECK_HANDLE(h);
    if (!s) return fail(h, VISTA_E_ARG, "null source descriptor");
    const double half_pi = 1.5707963267948966;
    if (!(is_fin(ra0) && is_fin(ra1) && is_fin(dec0) && is_fin(dec1)))
        return fail(h, VISTA_E_ARG, "phase centre and stacking position must be finite");
    if (std::fabs(dec0) > half_pi || std::fabs(dec1) > half_pi)
        return fail(h, VISTA_E_ARG, "declinations must lie in [-pi/2, pi/2]");
    // R = M(ra1, dec1) M(ra0, dec0)^T, each entry summed in order (Eq. 1)
    double M0[3][3], M1[3][3], R[9];
    uvw_frame(ra0, dec0, M0);
    uvw_frame(ra1, dec1, M1);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) R[3 * i + j] = M1[i][0] * M0[j][0] + M1[i][1] * M0[j][1] + M1[i][2] * M0[j][2];
    // the shift's direction cosines: the stacking position seen from the phase centre
    const double da = ra1 - ra0;
    vista_source_desc d = *s;
    d.l = std::cos(dec1) * std::sin(da);
    d.m = std::sin(dec1) * std::cos(dec0) - std::cos(dec1) * std::sin(dec0) * std::cos(da);
    if (!(d.l * d.l + d.m * d.m < 1.0 && R[8] > 0.0))
        return fail(h, VISTA_E_ARG, "the stacking position must lie less than 90 degrees from the phase centre");
    return add_source_impl(h, &d, R);
}

// --------------------------------------------------------------- readback

namespace {

// Wait for a readback still copying out of b_unpack.
cudaError_t finish_readback(vista_stack *h)
{
    if (!h->rb_pending) return cudaSuccess;
    h->rb_pending = false;
    return cudaEventSynchronize(h->rb_done);
}

int read_common(vista_stack *h, void *sum_wv, void *sum_w, void *sum_wvv, uint32_t *count, int dst_dev,
                int out_f64)
{
    cudaError_t e = finish_readback(h);
    if (e != cudaSuccess) return cuda_fail(h, e, "earlier readback");
    e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "stream synchronize");
    int32_t err = 0;
    e = cudaMemcpy(&err, h->err, sizeof err, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(h, e, "error word read");
    if (err != 0) return device_fail(h, err);
    const int fp64 = h->desc.precision == VISTA_PREC_FP64;
    const int64_t n = h->nentries;
    const size_t fe = out_f64 ? 8 : 4;
    if (dst_dev) {
        e = launch_unpack(h->cube, h->cube_master, h->count, fp64, n, sum_wv, sum_w, sum_wvv, count, out_f64,
                          h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "cube unpack");
        return VISTA_OK;
    }
    // host destination: unpack into a device scratch area, then copy
    const size_t b_wv = sum_wv ? (size_t)n * 2 * fe : 0, b_w = sum_w ? (size_t)n * fe : 0,
                 b_vv = sum_wvv ? (size_t)n * fe : 0, b_c = count ? (size_t)n * 4 : 0;
    e = h->b_unpack.ensure(b_wv + b_w + b_vv + b_c + 64);
    if (e != cudaSuccess) return cuda_fail(h, e, "readback scratch allocation");
    char *p = (char *)h->b_unpack.p;
    char *d_wv = sum_wv ? p : nullptr;
    char *d_w = sum_w ? p + b_wv : nullptr;
    char *d_vv = sum_wvv ? p + b_wv + b_w : nullptr;
    uint32_t *d_c = count ? (uint32_t *)(p + b_wv + b_w + b_vv) : nullptr;
    e = launch_unpack(h->cube, h->cube_master, h->count, fp64, n, d_wv, d_w, d_vv, d_c, out_f64, h->stream);
    // the four arrays go back on the copy streams, in parallel
    if (e == cudaSuccess) e = xfer_fork(h);
    if (e == cudaSuccess && sum_wv) e = cudaMemcpyAsync(sum_wv, d_wv, b_wv, cudaMemcpyDeviceToHost, h->xfer[0]);
    if (e == cudaSuccess && sum_w) e = cudaMemcpyAsync(sum_w, d_w, b_w, cudaMemcpyDeviceToHost, h->xfer[1]);
    if (e == cudaSuccess && sum_wvv) e = cudaMemcpyAsync(sum_wvv, d_vv, b_vv, cudaMemcpyDeviceToHost, h->xfer[2]);
    if (e == cudaSuccess && count) e = cudaMemcpyAsync(count, d_c, b_c, cudaMemcpyDeviceToHost, h->xfer[3]);
    if (e == cudaSuccess) e = xfer_join(h);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "cube readback");
    return VISTA_OK;
}

}  // namespace

extern "C" int vista_read_cube(vista_stack *h, float *sum_wv, float *sum_w, float *sum_wvv, uint32_t *count,
                               int dst_is_device)
{
    CHECK_HANDLE(h);
    return read_common(h, sum_wv, sum_w, sum_wvv, count, dst_is_device, 0);
}

extern "C" int vista_read_cube_f64(vista_stack *h, double *sum_wv, double *sum_w, double *sum_wvv,
                                   uint32_t *count, int dst_is_device)
{
    CHECK_HANDLE(h);
    return read_common(h, sum_wv, sum_w, sum_wvv, count, dst_is_device, 1);
}

extern "C" int vista_read_cube_async(vista_stack *h, float *sum_wv, float *sum_w, float *sum_wvv, uint32_t *count)
{
    CHECK_HANDLE(h);
    if (!sum_wv && !sum_w && !sum_wvv && !count) return fail(h, VISTA_E_ARG, "no output array");
    cudaError_t e = cudaSuccess;
    if (!h->rb_stream) e = cudaStreamCreateWithFlags(&h->rb_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess && !h->rb_ready) e = cudaEventCreateWithFlags(&h->rb_ready, cudaEventDisableTiming);
    if (e == cudaSuccess && !h->rb_done) e = cudaEventCreateWithFlags(&h->rb_done, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_fail(h, e, "readback stream");
    const int fp64 = h->desc.precision == VISTA_PREC_FP64;
    const int64_t n = h->nentries;
    const size_t b_wv = sum_wv ? (size_t)n * 8 : 0, b_w = sum_w ? (size_t)n * 4 : 0,
                 b_vv = sum_wvv ? (size_t)n * 4 : 0, b_c = count ? (size_t)n * 4 : 0;
    const size_t need = b_wv + b_w + b_vv + b_c + 64;
    // a larger scratch area replaces the one the previous copy may still read
    if (need > h->b_unpack.cap && (e = finish_readback(h)) != cudaSuccess)
        return cuda_fail(h, e, "earlier readback");
    if ((e = h->b_unpack.ensure(need)) != cudaSuccess) return cuda_fail(h, e, "readback scratch allocation");
    char *p = (char *)h->b_unpack.p;
    char *d_wv = sum_wv ? p : nullptr;
    char *d_w = sum_w ? p + b_wv : nullptr;
    char *d_vv = sum_wvv ? p + b_wv + b_w : nullptr;
    uint32_t *d_c = count ? (uint32_t *)(p + b_wv + b_w + b_vv) : nullptr;
    // the snapshot waits for the previous copy out of the scratch area, then
    // follows the runs queued so far on the handle's stream
    if (h->rb_pending) e = cudaStreamWaitEvent(h->stream, h->rb_done, 0);
    if (e == cudaSuccess)
        e = launch_unpack(h->cube, h->cube_master, h->count, fp64, n, d_wv, d_w, d_vv, d_c, 0, h->stream);
    if (e == cudaSuccess) e = cudaEventRecord(h->rb_ready, h->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->rb_stream, h->rb_ready, 0);
    if (e == cudaSuccess && sum_wv) e = cudaMemcpyAsync(sum_wv, d_wv, b_wv, cudaMemcpyDeviceToHost, h->rb_stream);
    if (e == cudaSuccess && sum_w) e = cudaMemcpyAsync(sum_w, d_w, b_w, cudaMemcpyDeviceToHost, h->rb_stream);
    if (e == cudaSuccess && sum_wvv) e = cudaMemcpyAsync(sum_wvv, d_vv, b_vv, cudaMemcpyDeviceToHost, h->rb_stream);
    if (e == cudaSuccess && count) e = cudaMemcpyAsync(count, d_c, b_c, cudaMemcpyDeviceToHost, h->rb_stream);
    if (e == cudaSuccess) e = cudaEventRecord(h->rb_done, h->rb_stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "cube readback");
    h->rb_pending = true;
    return VISTA_OK;
}

extern "C" int vista_wait_readback(vista_stack *h)
{
    CHECK_HANDLE(h);
    const bool was = h->rb_pending;
    cudaError_t e = finish_readback(h);
    if (e != cudaSuccess) return cuda_fail(h, e, "readback");
    if (!was) return VISTA_OK;
    // the runs before the snapshot have completed: their error word
    int32_t err = 0;
    e = cudaMemcpyAsync(&err, h->err, sizeof err, cudaMemcpyDeviceToHost, h->rb_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->rb_stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "error word read");
    if (err != 0) return device_fail(h, err);
    return VISTA_OK;
}

extern "C" int vista_read_cube_sparse(vista_stack *h, int64_t cap, int64_t *index, float *sum_wv, float *sum_w,
                                      float *sum_wvv, uint32_t *count, int64_t *n_touched, int dst_is_device)
{
    CHECK_HANDLE(h);
    if (!n_touched) return fail(h, VISTA_E_ARG, "null n_touched");
    if (cap < 0) return fail(h, VISTA_E_ARG, "cap must be >= 0");
    if (cap > 0 && !index) return fail(h, VISTA_E_ARG, "null index with cap > 0");
    cudaError_t e = finish_readback(h);
    if (e != cudaSuccess) return cuda_fail(h, e, "earlier readback");
    e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "stream synchronize");
    int32_t err = 0;
    e = cudaMemcpy(&err, h->err, sizeof err, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(h, e, "error word read");
    if (err != 0) return device_fail(h, err);
    const int fp64 = h->desc.precision == VISTA_PREC_FP64;
    const int64_t n = h->nentries, ntile = sparse_tiles(n);
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    // scratch: tile counts | tile offsets | total (the touched entries of a
    // host destination go through the dense readback's scratch, free here)
    const size_t o_off = al((size_t)ntile * 4), o_tot = o_off + al((size_t)ntile * 8), o_end = o_tot + 256;
    if ((e = h->b_sparse.ensure(o_end)) != cudaSuccess) return cuda_fail(h, e, "sparse readback scratch");
    char *b = (char *)h->b_sparse.p;
    e = launch_sparse_count(h->count, n, (uint32_t *)b, (int64_t *)(b + o_off), (int64_t *)(b + o_tot), h->stream);
    int64_t total = 0;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&total, b + o_tot, sizeof total, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "sparse readback count");
    *n_touched = total;
    if (cap == 0) return VISTA_OK;   // the count only
    if (total > cap)
        return fail(h, VISTA_E_RANGE, "the cube has %lld touched entries, more than cap = %lld", (long long)total,
                    (long long)cap);
    if (dst_is_device) {
        e = launch_sparse_write(h->cube, h->cube_master, h->count, fp64, n, (const int64_t *)(b + o_off), cap, index,
                                sum_wv, sum_w, sum_wvv, count, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "sparse readback");
        return VISTA_OK;
    }
    // host destination: the touched entries into the scratch, then one copy per array
    const size_t t = (size_t)total;
    const size_t o_wv = al(t * 8), o_w = o_wv + al(t * 8), o_vv = o_w + al(t * 4), o_c = o_vv + al(t * 4),
                 need = o_c + al(t * 4);
    if ((e = h->b_unpack.ensure(need)) != cudaSuccess) return cuda_fail(h, e, "readback scratch allocation");
    char *u = (char *)h->b_unpack.p;
    e = launch_sparse_write(h->cube, h->cube_master, h->count, fp64, n, (const int64_t *)(b + o_off), cap,
                            (int64_t *)u, sum_wv ? (float *)(u + o_wv) : nullptr, sum_w ? (float *)(u + o_w) : nullptr,
                            sum_wvv ? (float *)(u + o_vv) : nullptr, count ? (uint32_t *)(u + o_c) : nullptr,
                            h->stream);
    if (e == cudaSuccess && t > 0) e = xfer_fork(h);
    if (e == cudaSuccess && t > 0) {
        e = cudaMemcpyAsync(index, u, t * 8, cudaMemcpyDeviceToHost, h->xfer[0]);
        if (e == cudaSuccess && sum_wv) e = cudaMemcpyAsync(sum_wv, u + o_wv, t * 8, cudaMemcpyDeviceToHost, h->xfer[1]);
        if (e == cudaSuccess && sum_w) e = cudaMemcpyAsync(sum_w, u + o_w, t * 4, cudaMemcpyDeviceToHost, h->xfer[2]);
        if (e == cudaSuccess && sum_wvv) e = cudaMemcpyAsync(sum_wvv, u + o_vv, t * 4, cudaMemcpyDeviceToHost, h->xfer[3]);
        if (e == cudaSuccess && count) e = cudaMemcpyAsync(count, u + o_c, t * 4, cudaMemcpyDeviceToHost, h->xfer[0]);
        if (e == cudaSuccess) e = xfer_join(h);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "sparse readback");
    return VISTA_OK;
}

extern "C" int vista_set_wave_bytes(vista_stack *h, int64_t bytes)
{
    CHECK_HANDLE(h);
    if (bytes < 0) return fail(h, VISTA_E_ARG, "wave bytes must be >= 0");
    h->wave_bytes = bytes;
    return VISTA_OK;
}

extern "C" int vista_get_waves(vista_stack *h, int32_t *out)
{
    CHECK_HANDLE(h);
    if (!out) return fail(h, VISTA_E_ARG, "null output");
    *out = h->nwaves;
    return VISTA_OK;
}

extern "C" int vista_get_h2d_bytes(vista_stack *h, int64_t *out)
{
    CHECK_HANDLE(h);
    if (!out) return fail(h, VISTA_E_ARG, "null output");
    int64_t n = 0;
    for (const HostCopy &c : h->hcopies) n += (int64_t)(c.width * c.height);
    *out = n;
    return VISTA_OK;
}

extern "C" int vista_zero_cube(vista_stack *h)
{
    CHECK_HANDLE(h);
    const size_t esz = h->desc.precision == VISTA_PREC_FP64 ? 32 : 16;
    cudaError_t e = cudaMemsetAsync(h->cube, 0, (size_t)h->nentries * esz, h->stream);
    if (e == cudaSuccess && h->cube_master)
        e = cudaMemsetAsync(h->cube_master, 0, (size_t)h->nentries * 32, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->count, 0, (size_t)h->nentries * 4, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->stats, 0, sizeof(DevStats), h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "cube zeroing");
    h->host_nvis = 0;
    h->nvis_since_fold = 0;
    return VISTA_OK;
}

extern "C" int vista_get_stats(vista_stack *h, vista_stats *out)
{
    CHECK_HANDLE(h);
    if (!out) return fail(h, VISTA_E_ARG, "null output");
    DevStats s;
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e == cudaSuccess) e = cudaMemcpy(&s, h->stats, sizeof s, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(h, e, "stats readback");
    // the kernels count flagged and off-grid visibilities; how many they read
    // is known from the channel tables
    out->n_vis = h->host_nvis;
    out->n_flagged = s.n_flagged;
    out->n_dropped_uv = s.n_dropped_uv;
    out->n_stacked = h->host_nvis - s.n_flagged - s.n_dropped_uv;
    out->n_reductions = s.n_reductions;
    return VISTA_OK;
}

extern "C" int vista_get_lattice(vista_stack *h, double *rest_f0, double *rest_df)
{
    CHECK_HANDLE(h);
    if (!rest_f0 || !rest_df) return fail(h, VISTA_E_ARG, "null output");
    if (!h->lattice_fixed) return fail(h, VISTA_E_STATE, "the automatic lattice is fixed at the first run");
    *rest_f0 = h->f0;
    *rest_df = h->df;
    return VISTA_OK;
}

extern "C" int vista_set_tuning(vista_stack *h, const vista_tuning *t)
{
    CHECK_HANDLE(h);
    if (!t) return fail(h, VISTA_E_ARG, "null tuning");
    LaunchCfg c = h->cfg;
    if (t->rows_per_item) {
        if (t->rows_per_item < 1 || t->rows_per_item > 256)
            return fail(h, VISTA_E_ARG, "rows_per_item must be in [1, 256]");
        c.rows_per_item = t->rows_per_item;
    }
    if (t->chans_per_lane) {
        if (t->chans_per_lane != 1 && t->chans_per_lane != 2 && t->chans_per_lane != 4)
            return fail(h, VISTA_E_ARG, "chans_per_lane must be 1, 2 or 4");
        c.chans_per_lane = t->chans_per_lane;
    }
    if (t->warps_per_cta) {
        if (t->warps_per_cta != 1 && t->warps_per_cta != 2 && t->warps_per_cta != 4 && t->warps_per_cta != 8)
            return fail(h, VISTA_E_ARG, "warps_per_cta must be 1, 2, 4 or 8");
        c.warps_per_cta = t->warps_per_cta;
    }
    if (t->sort_rows < 0 || t->sort_rows > 1) return fail(h, VISTA_E_ARG, "sort_rows must be 0 or 1");
    c.sort_rows = t->sort_rows;
    if (t->prefetch_rows) {
        if (t->prefetch_rows != 2 && t->prefetch_rows != 4 && t->prefetch_rows != 8)
            return fail(h, VISTA_E_ARG, "prefetch_rows must be 2, 4 or 8");
        c.prefetch_rows = t->prefetch_rows;
    }
    h->cfg = c;
    drop_graph(h);
    h->plan_valid = false;
    return VISTA_OK;
}

extern "C" int vista_get_tuning(vista_stack *h, vista_tuning *t)
{
    CHECK_HANDLE(h);
    if (!t) return fail(h, VISTA_E_ARG, "null output");
    t->rows_per_item = h->cfg.rows_per_item;
    t->chans_per_lane = h->cfg.chans_per_lane;
    t->warps_per_cta = h->cfg.warps_per_cta;
    t->sort_rows = h->cfg.sort_rows;
    t->prefetch_rows = h->cfg.prefetch_rows;
    return VISTA_OK;
}

extern "C" int vista_enable_timing(vista_stack *h, int on)
{
    CHECK_HANDLE(h);
    if (on != 0 && on != 1) return fail(h, VISTA_E_ARG, "on must be 0 or 1");
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "stream synchronize");
    for (auto &s : h->spans) {
        h->ev_pool.push_back(s.a);
        h->ev_pool.push_back(s.b);
    }
    h->spans.clear();
    h->tacc = vista_timing{};
    h->timing = on != 0;
    return VISTA_OK;
}

extern "C" int vista_get_timing(vista_stack *h, vista_timing *out)
{
    CHECK_HANDLE(h);
    if (!out) return fail(h, VISTA_E_ARG, "null output");
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "stream synchronize");
    for (auto &s : h->spans) {
        float ms = 0.f;
        e = cudaEventElapsedTime(&ms, s.a, s.b);
        if (e != cudaSuccess) return cuda_fail(h, e, "event timing");
        (s.kind == 0 ? h->tacc.prepass_ms : s.kind == 1 ? h->tacc.stack_ms : h->tacc.other_ms) += ms;
        h->ev_pool.push_back(s.a);
        h->ev_pool.push_back(s.b);
    }
    h->spans.clear();
    *out = h->tacc;
    return VISTA_OK;
}

extern "C" int vista_enable_graphs(vista_stack *h, int on)
{
    CHECK_HANDLE(h);
    if (on != 0 && on != 1) return fail(h, VISTA_E_ARG, "on must be 0 or 1");
    h->graphs = on != 0;
    if (!h->graphs) drop_graph(h);
    return VISTA_OK;
}

extern "C" int vista_graph_runs(vista_stack *h, uint64_t *out)
{
    CHECK_HANDLE(h);
    if (!out) return fail(h, VISTA_E_ARG, "null output");
    *out = h->graph_launches;
    return VISTA_OK;
}

extern "C" int vista_close(vista_stack *h)
{
    CHECK_HANDLE(h);
    {
        std::lock_guard<std::mutex> lk(g_mu);
        g_live.erase(h);
    }
    cudaStreamSynchronize(h->stream);
    for (auto &s : h->spans) {
        cudaEventDestroy(s.a);
        cudaEventDestroy(s.b);
    }
    for (cudaEvent_t ev : h->ev_pool) cudaEventDestroy(ev);
    drop_graph(h);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    for (int j = 0; j < NXFER; ++j)
        if (h->xfer[j]) {
            cudaStreamSynchronize(h->xfer[j]);
            cudaStreamDestroy(h->xfer[j]);
        }
    for (int j = 0; j <= NXFER; ++j)
        if (h->xfer_ev[j]) cudaEventDestroy(h->xfer_ev[j]);
    for (int j = 0; j < 2; ++j)
        if (h->slot_ev[j]) cudaEventDestroy(h->slot_ev[j]);
    if (h->rb_stream) {
        cudaStreamSynchronize(h->rb_stream);
        cudaStreamDestroy(h->rb_stream);
    }
    for (int j = 0; j < 2; ++j) {
        if (h->pin_ev[j]) cudaEventDestroy(h->pin_ev[j]);
        if (h->pin[j]) cudaFreeHost(h->pin[j]);
    }
    if (h->rb_ready) cudaEventDestroy(h->rb_ready);
    if (h->rb_done) cudaEventDestroy(h->rb_done);
    cudaFree(h->cube);
    cudaFree(h->cube_master);
    cudaFree(h->count);
    cudaFree(h->stats);
    cudaFree(h->err);
    h->b_srcs.release();
    h->b_chf.release();
    h->b_chd.release();
    h->b_recs.release();
    h->b_cells.release();
    h->b_off.release();
    h->b_stage.release();
    h->b_unpack.release();
    h->b_sort.release();
    h->b_rot.release();
    h->b_guvw.release();
    h->b_regrid.release();
    h->b_contsub.release();
    h->b_sparse.release();
    delete h;
    return VISTA_OK;
}

extern "C" const char *vista_last_error(const vista_stack *h)
{
    if (h && handle_live(h)) return h->msg.c_str();
    return g_err.c_str();
}

// ------------------------------------------------------------------- debug

namespace {

int debug_common(vista_stack *h, int32_t src, double *ph, int32_t *cells)
{
    if (src < 0 || (size_t)src >= h->last.size()) return fail(h, VISTA_E_ARG, "no source %d in the last run", src);
    for (const ClassRun &cr : h->classes) {
        for (size_t t = 0; t < cr.members.size(); ++t) {
            if (cr.members[t] != src) continue;
            cudaError_t e = launch_debug(cr.args, cr.ns, (int)t, h->desc.precision == VISTA_PREC_FP64, ph, cells,
                                         h->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
            if (e != cudaSuccess) return cuda_fail(h, e, "debug export");
            return VISTA_OK;
        }
    }
    return VISTA_OK;   // a window with no row or no channel in the cube: nothing is read
}

}  // namespace

extern "C" int vista_debug_phasors(vista_stack *h, int32_t src, double *dst)
{
    CHECK_HANDLE(h);
    if (!dst) return fail(h, VISTA_E_ARG, "null output");
    return debug_common(h, src, dst, nullptr);
}

extern "C" int vista_debug_cells(vista_stack *h, int32_t src, int32_t *dst)
{
    CHECK_HANDLE(h);
    if (!dst) return fail(h, VISTA_E_ARG, "null output");
    return debug_common(h, src, nullptr, dst);
}

extern "C" int vista_debug_order(vista_stack *h, int32_t src, int32_t *dst)
{
    CHECK_HANDLE(h);
    if (!dst) return fail(h, VISTA_E_ARG, "null output");
    if (h->desc.precision != VISTA_PREC_MIXED || h->classes.size() != 1)
        return fail(h, VISTA_E_STATE, "the processing order is kept for single-class mixed runs only");
    const ClassRun &cr = h->classes[0];
    for (size_t t = 0; t < cr.members.size(); ++t) {
        if (cr.members[t] != src) continue;
        int64_t off[2];
        cudaError_t e = cudaMemcpy(off, cr.args.row_off + t, sizeof off, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess)
            e = cudaMemcpy(dst, cr.args.so.perm + off[0], sizeof(int32_t) * (size_t)(off[1] - off[0]),
                           cudaMemcpyDeviceToDevice);
        if (e != cudaSuccess) return cuda_fail(h, e, "order export");
        return VISTA_OK;
    }
    return fail(h, VISTA_E_ARG, "window %d has no row in the cube", src);
}

// The paper's per-row output (Eq. 3): every row of one window regridded onto
// the rest lattice, V_out(j) = sum_k V'(k) w_kj / sum_k w_kj over unflagged
// channels, with V' the shifted visibility of Eq. 2 and w_kj the Eq. 4
// weights.  The contributing channels of each output channel are listed on
// the host (a compressed row table built from the FP64 planner's bins).  A
// first kernel forms each row's delay in FP64 and keeps it as a float-float
// pair; then one thread per (row, output channel) forms each contributor's
// phasor as the stacking kernel does (float-float product tau nu_k / c,
// reduced mod 1 turn, __sincosf: below 5e-7 rad) and sums in FP32 (a few
// terms per output channel).  For complex64 with 2 or 4 pols on 16-byte
// aligned arrays a channel's pols and their flags come in vector loads.
#include <cmath>
#include <vector>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "planner.h"
#include "vista_device.cuh"
#include "vista_handle.h"

namespace vista {
namespace {

struct RegridArgs {
    const double *uvw;
    const void *vis;
    const uint8_t *flags;
    const float2 *nuc;      // [nchan] nu_k / c as a float-float pair (1/m)
    const int32_t *start;   // [nrest + 1] first contributor of each output channel
    const int32_t *chan;    // contributing channel
    const float *w;         // its Eq. 4 weight
    float2 *tau;            // [nrow] the row's delay (m) as a float-float pair
    float *out_vis;         // [nrow][nrest][npol][2]
    float *out_wsum;        // [nrow][nrest][npol]
    double *out_uvw;        // [nrow][3] or null
    int64_t nrow;
    int32_t nchan, npol, nrest, vis_type;
    int32_t vec;            // complex64 with 2 or 4 pols, 16-byte aligned: a channel's pols in vector loads
    int32_t vout;           // 2 or 4 pols, outputs 16-byte (wsum of 2 pols: 8-byte) aligned: vector stores
    float vis_scale;
    double l, m, n1, inv_zf;
};

__device__ __forceinline__ float2 load_vis(const RegridArgs &a, int64_t i)
{
    switch (a.vis_type) {
    case VISTA_VIS_C128: {
        const double2 v = reinterpret_cast<const double2 *>(a.vis)[i];
        return make_float2((float)v.x, (float)v.y);
    }
    case VISTA_VIS_C64: return reinterpret_cast<const float2 *>(a.vis)[i];
    case VISTA_VIS_F16X2: {
        const __half2 v = reinterpret_cast<const __half2 *>(a.vis)[i];
        return make_float2(__low2float(v) * a.vis_scale, __high2float(v) * a.vis_scale);
    }
    default: {
        const __nv_bfloat162 v = reinterpret_cast<const __nv_bfloat162 *>(a.vis)[i];
        return make_float2(__low2float(v) * a.vis_scale, __high2float(v) * a.vis_scale);
    }
    }
}

// One thread per row: the Eq. 2 delay in FP64, kept as a float-float pair,
// and the rest-frame baseline (Eq. 1 with R = I) if asked for.
__global__ void __launch_bounds__(256) k_regrid_tau(RegridArgs a)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= a.nrow) return;
    const double *x = a.uvw + 3 * r;
    float hi, lo;
    split_ff(x[0] * a.l + x[1] * a.m + x[2] * a.n1, hi, lo);
    a.tau[r] = make_float2(hi, lo);
    if (a.out_uvw)
        for (int c = 0; c < 3; ++c) a.out_uvw[3 * r + c] = x[c] * a.inv_zf;
}

// One channel's P visibilities (and their flag bytes, 0 = unflagged) with
// vector loads: complex64 pols of a channel are 8 P contiguous, 16-byte
// aligned bytes, their flags 4 (P = 4) or 2 (P = 2) aligned bytes.
template <int P>
__device__ __forceinline__ void load_channel_c64(const RegridArgs &a, int64_t i0, float2 (&v)[4], uint32_t &fl)
{
    const float4 *q = reinterpret_cast<const float4 *>(reinterpret_cast<const float2 *>(a.vis) + i0);
    const float4 x = q[0];
    v[0] = make_float2(x.x, x.y);
    v[1] = make_float2(x.z, x.w);
    if constexpr (P == 4) {
        const float4 y = q[1];
        v[2] = make_float2(y.x, y.y);
        v[3] = make_float2(y.z, y.w);
        fl = a.flags ? *reinterpret_cast<const uint32_t *>(a.flags + i0) : 0u;
    } else {
        fl = a.flags ? (uint32_t)*reinterpret_cast<const uint16_t *>(a.flags + i0) : 0u;
    }
}

__global__ void __launch_bounds__(256) k_regrid(RegridArgs a)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= a.nrow * a.nrest) return;
    const int64_t r = t / a.nrest;
    const int j = (int)(t - r * a.nrest);
    const float2 tau = a.tau[r];
    float sr[4] = {0, 0, 0, 0}, si[4] = {0, 0, 0, 0}, sw[4] = {0, 0, 0, 0};
    for (int e = a.start[j]; e < a.start[j + 1]; ++e) {
        const int k = a.chan[e];
        const float w = a.w[e];
        const float2 nuc = a.nuc[k];
        const float2 ph = shift_phasor(tau.x, tau.y, nuc.x, nuc.y);
        const int64_t i0 = (r * a.nchan + k) * a.npol;
        if (a.vec) {
            float2 v[4];
            uint32_t fl;
            if (a.npol == 4) load_channel_c64<4>(a, i0, v, fl);
            else load_channel_c64<2>(a, i0, v, fl);
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                if (p >= a.npol || ((fl >> (8 * p)) & 0xffu)) continue;
                sr[p] = __fmaf_rn(w, v[p].x * ph.x - v[p].y * ph.y, sr[p]);
                si[p] = __fmaf_rn(w, v[p].x * ph.y + v[p].y * ph.x, si[p]);
                sw[p] += w;
            }
            continue;
        }
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            if (p >= a.npol) break;
            const int64_t i = i0 + p;
            if (a.flags && a.flags[i]) continue;
            const float2 v = load_vis(a, i);
            sr[p] = __fmaf_rn(w, v.x * ph.x - v.y * ph.y, sr[p]);
            si[p] = __fmaf_rn(w, v.x * ph.y + v.y * ph.x, si[p]);
            sw[p] += w;
        }
    }
    float ov[8];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const bool any = sw[p] > 0.0f;
        ov[2 * p] = any ? sr[p] / sw[p] : 0.0f;
        ov[2 * p + 1] = any ? si[p] / sw[p] : 0.0f;
    }
    const int64_t o = (r * a.nrest + j) * a.npol;
    if (a.vout) {
        // a thread's outputs are contiguous: whole 16-byte stores rather
        // than one 4-byte store per value (each of those spans 32 sectors
        // across the warp)
        float4 *dv = reinterpret_cast<float4 *>(a.out_vis + 2 * o);
        dv[0] = make_float4(ov[0], ov[1], ov[2], ov[3]);
        if (a.npol == 4) {
            dv[1] = make_float4(ov[4], ov[5], ov[6], ov[7]);
            *reinterpret_cast<float4 *>(a.out_wsum + o) = make_float4(sw[0], sw[1], sw[2], sw[3]);
        } else {
            *reinterpret_cast<float2 *>(a.out_wsum + o) = make_float2(sw[0], sw[1]);
        }
        return;
    }
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        if (p >= a.npol) break;
        a.out_vis[2 * (o + p)] = ov[2 * p];
        a.out_vis[2 * (o + p) + 1] = ov[2 * p + 1];
        a.out_wsum[o + p] = sw[p];
    }
}

}  // namespace
}  // namespace vista

using namespace vista;

extern "C" int vista_regrid_rows(vista_stack *h, const vista_source_desc *s, float *out_vis, float *out_wsum,
                                 double *out_uvw)
{
    if (!handle_live(h)) return fail(nullptr, VISTA_E_STATE, "unknown or closed handle");
    if (!s || !out_vis || !out_wsum) return fail(h, VISTA_E_ARG, "null descriptor or output");
    if (!h->lattice_fixed)
        return fail(h, VISTA_E_STATE, "the rest lattice is not fixed yet (give rest_df at open, or run first)");
    if (s->mem != VISTA_MEM_DEVICE) return fail(h, VISTA_E_ARG, "vista_regrid_rows reads device arrays only");
    if (s->nrow < 0 || s->nchan < 2) return fail(h, VISTA_E_ARG, "need nrow >= 0 and nchan >= 2");
    if (s->npol != 1 && s->npol != 2 && s->npol != 4) return fail(h, VISTA_E_ARG, "npol must be 1, 2 or 4");
    if (s->vis_type < VISTA_VIS_C64 || s->vis_type > VISTA_VIS_BF16X2)
        return fail(h, VISTA_E_ARG, "bad vis_type %d", s->vis_type);
    if (!s->freqs || (s->nrow > 0 && (!s->uvw || !s->vis)))
        return fail(h, VISTA_E_ARG, "freqs, uvw and vis must be non-NULL");
    if (!(std::isfinite(s->l) && std::isfinite(s->m) && s->l * s->l + s->m * s->m < 1.0))
        return fail(h, VISTA_E_ARG, "need finite l, m with l^2 + m^2 < 1");
    if (!(std::isfinite(s->z) && s->z > -1.0)) return fail(h, VISTA_E_ARG, "need finite z > -1");
    const int32_t n = s->nchan, nrest = h->desc.nrest;
    for (int32_t k = 0; k < n; ++k)
        if (!(std::isfinite(s->freqs[k]) && s->freqs[k] > 0.0))
            return fail(h, VISTA_E_ARG, "freqs[%d] is not finite and > 0", k);
    const bool up = s->freqs[1] > s->freqs[0];
    for (int32_t k = 1; k < n; ++k)
        if (up ? !(s->freqs[k] > s->freqs[k - 1]) : !(s->freqs[k] < s->freqs[k - 1]))
            return fail(h, VISTA_E_ARG, "freqs must be strictly monotone (index %d)", k);
    if (s->nrow == 0) return VISTA_OK;

    // contributors of each output channel (Eq. 4), from the FP64 planner
    std::vector<int32_t> j0((size_t)n), nb((size_t)n);
    std::vector<double> wk((size_t)n * VISTA_MAX_BINS);
    const int rc = channel_bins(s->freqs, n, s->z, h->f0, h->df, nrest, h->desc.bin_mode, j0.data(), nb.data(),
                                wk.data());
    if (rc != VISTA_OK) return fail(h, rc, "channel planning failed");
    std::vector<int32_t> start((size_t)nrest + 1, 0);
    for (int32_t k = 0; k < n; ++k)
        for (int b = 0; b < nb[(size_t)k]; ++b) ++start[(size_t)j0[(size_t)k] + b + 1];
    for (int32_t j = 0; j < nrest; ++j) start[(size_t)j + 1] += start[(size_t)j];
    const size_t nnz = (size_t)start[(size_t)nrest];
    std::vector<int32_t> chan(nnz > 0 ? nnz : 1), fill(start.begin(), start.end() - 1);
    std::vector<float> w(nnz > 0 ? nnz : 1);
    for (int32_t k = 0; k < n; ++k)
        for (int b = 0; b < nb[(size_t)k]; ++b) {
            const int32_t e = fill[(size_t)j0[(size_t)k] + b]++;
            chan[(size_t)e] = k;
            w[(size_t)e] = (float)wk[(size_t)k * VISTA_MAX_BINS + b];
        }

    // nu_k / c of every channel as a float-float pair
    std::vector<float2> nuc((size_t)n);
    for (int32_t k = 0; k < n; ++k) {
        const double x = s->freqs[k] / C_LIGHT;
        nuc[(size_t)k].x = (float)x;
        nuc[(size_t)k].y = (float)(x - (double)nuc[(size_t)k].x);
    }

    // one device buffer: nu/c | start | chan | w | per-row delays
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    const size_t o_f = 0, o_s = al(sizeof(float2) * (size_t)n), o_c = o_s + al(sizeof(int32_t) * start.size()),
                 o_w = o_c + al(sizeof(int32_t) * chan.size()), o_t = o_w + al(sizeof(float) * w.size()),
                 total = o_t + al(sizeof(float2) * (size_t)s->nrow);
    cudaError_t e = h->b_regrid.ensure(total);
    if (e != cudaSuccess) return cuda_fail(h, e, "regrid table allocation");
    char *b = (char *)h->b_regrid.p;
    e = cudaMemcpyAsync(b + o_f, nuc.data(), sizeof(float2) * (size_t)n, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b + o_s, start.data(), sizeof(int32_t) * start.size(), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b + o_c, chan.data(), sizeof(int32_t) * chan.size(), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b + o_w, w.data(), sizeof(float) * w.size(), cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "regrid table upload");

    RegridArgs a{};
    a.uvw = s->uvw;
    a.vis = s->vis;
    a.flags = s->flags;
    a.nuc = (const float2 *)(b + o_f);
    a.start = (const int32_t *)(b + o_s);
    a.chan = (const int32_t *)(b + o_c);
    a.w = (const float *)(b + o_w);
    a.tau = (float2 *)(b + o_t);
    a.out_vis = out_vis;
    a.out_wsum = out_wsum;
    a.out_uvw = out_uvw;
    a.nrow = s->nrow;
    a.nchan = n;
    a.npol = s->npol;
    a.nrest = nrest;
    a.vis_type = s->vis_type;
    a.vis_scale = (s->vis_type == VISTA_VIS_F16X2 || s->vis_type == VISTA_VIS_BF16X2) ? s->vis_scale : 1.0f;
    a.vec = s->vis_type == VISTA_VIS_C64 && (s->npol == 2 || s->npol == 4) && ((uintptr_t)s->vis % 16) == 0 &&
            (!s->flags || ((uintptr_t)s->flags % (uintptr_t)s->npol) == 0);
    a.vout = (s->npol == 2 || s->npol == 4) && ((uintptr_t)out_vis % 16) == 0 &&
             ((uintptr_t)out_wsum % (uintptr_t)(s->npol == 4 ? 16 : 8)) == 0;
    a.l = s->l;
    a.m = s->m;
    a.n1 = std::sqrt(1.0 - s->l * s->l - s->m * s->m) - 1.0;
    a.inv_zf = 1.0 / (1.0 + s->z);
    const int64_t threads = s->nrow * (int64_t)nrest;
    k_regrid_tau<<<(unsigned)((s->nrow + 255) / 256), 256, 0, h->stream>>>(a);
    e = cudaGetLastError();
    if (e == cudaSuccess) k_regrid<<<(unsigned)((threads + 255) / 256), 256, 0, h->stream>>>(a);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "regrid kernel");
    return VISTA_OK;
}

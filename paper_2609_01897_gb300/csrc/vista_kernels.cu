// libvista kernels for sm_103a: the visibility-stacking hot path.
//
//   prepass_mixed   FP64 per (row, chunk): delay tau, phase seed turns,
//                   recurrence stride, folded uvw -> RowRec (paper Eq. 2, and
//                   the phasor recurrence of Sec. 3.2)
//   stack_mixed     warp per work item (one window, a run of rows, 32 x NS
//                   channels, lane = channel): FP32 phasor, guarded-FP32 uv
//                   cell (exact against the FP64 rule), rest bins from the
//                   FP64 channel table (Eqs. 3-4), per-lane running sums
//                   over consecutive rows that share a cell, vector
//                   reductions into the FP32 cube
//   stack_fp64      the plain form: thread per (window, row), FP64
//                   recurrence, FP64 cells, FP64 atomics into an FP64 cube
//   unpack          cube -> caller arrays
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "vista_internal.h"

namespace vista {

// ---------------------------------------------------------------- helpers

// Largest s with off[s] <= x (off non-decreasing, off[0] = 0).
__device__ __forceinline__ int find_owner(const int64_t *__restrict__ off, int n, int64_t x)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (__ldg(off + mid) <= x)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// exp(2 pi i t) for t in turns; t is first reduced to [-0.5, 0.5] (exact
// for |t| < 2^22) so that sincospif sees its most accurate argument range.
__device__ __forceinline__ float2 turns_to_phasor(float t)
{
    t = __fsub_rn(t, rintf(t));
    float s, c;
    sincospif(2.0f * t, &s, &c);
    return make_float2(c, s);
}

// Seed phasor of channel c0 + lane of one row: t0 + frac(lane*dhi) + lane*dlo.
// lane*dhi is exact (dhi has <= 19 significant bits, lane < 32).
__device__ __forceinline__ float2 lane_seed(const RowRec &rec, int lane)
{
    float a = (float)lane * rec.dhi;
    a = __fsub_rn(a, floorf(a));
    float t = __fadd_rn(__fadd_rn(rec.t0, a), (float)lane * rec.dlo);
    return turns_to_phasor(t);
}

// One axis of the uv cell: floor(fl64(coord * s_k)) + n/2, or -1 outside
// [0, n).  Decided in FP32 when fl32(c32 * s32) is at least 2^-21 |x| away
// from an integer (the FP32 product differs from the FP64 one by at most
// 3 * 2^-24 |x|), else by the exact FP64 product.
__device__ __forceinline__ int axis_cell(float c32, float s32, const double *coord64, bool neg,
                                         const double *s64, int n)
{
    float x = __fmul_rn(c32, s32);
    float d = __fmaf_rn(fabsf(x), 4.76837158203125e-07f, 1e-30f);
    float fa = floorf(__fsub_rn(x, d)), fb = floorf(__fadd_rn(x, d));
    float fx;
    if (fa == fb) {
        fx = fa;
    } else {
        double c = *coord64;
        if (neg) c = -c;
        fx = (float)floor(__dmul_rn(c, *s64));
    }
    float h = (float)(n >> 1);
    if (!(fx >= -h && fx < h)) return -1;
    return (int)fx + (n >> 1);
}

__device__ __forceinline__ int axis_cell64(double c, double s, int n)
{
    double x = __dmul_rn(c, s);
    double h = (double)(n >> 1);
    if (!(x >= -h && x < h)) return -1;
    return (int)floor(x) + (n >> 1);
}

// ----------------------------------------------------------- vis loaders

template <int P, int VT>
struct VisLoad;

template <int P>
struct VisLoad<P, VISTA_VIS_C64> {
    static __device__ __forceinline__ void load(const void *base, int64_t idx, float scale, float2 (&v)[P])
    {
        (void)scale;
        const float2 *p = reinterpret_cast<const float2 *>(base) + idx * P;
        if constexpr (P == 1) {
            v[0] = __ldg(p);
        } else if constexpr (P == 2) {
            float4 q = __ldg(reinterpret_cast<const float4 *>(p));
            v[0] = make_float2(q.x, q.y);
            v[1] = make_float2(q.z, q.w);
        } else {
            float4 q0 = __ldg(reinterpret_cast<const float4 *>(p));
            float4 q1 = __ldg(reinterpret_cast<const float4 *>(p) + 1);
            v[0] = make_float2(q0.x, q0.y);
            v[1] = make_float2(q0.z, q0.w);
            v[2] = make_float2(q1.x, q1.y);
            v[3] = make_float2(q1.z, q1.w);
        }
    }
};

template <int P>
struct VisLoad<P, VISTA_VIS_C128> {
    static __device__ __forceinline__ void load(const void *base, int64_t idx, float scale, float2 (&v)[P])
    {
        (void)scale;
        const double2 *p = reinterpret_cast<const double2 *>(base) + idx * P;
#pragma unroll
        for (int i = 0; i < P; ++i) {
            double2 q = __ldg(p + i);
            v[i] = make_float2((float)q.x, (float)q.y);
        }
    }
};


template <int P>
struct VisLoad<P, VISTA_VIS_F16X2> {
    static __device__ __forceinline__ float2 cvt(uint32_t b, float scale)
    {
        __half2 h = *reinterpret_cast<__half2 *>(&b);
        float2 f = __half22float2(h);
        return make_float2(f.x * scale, f.y * scale);
    }
    static __device__ __forceinline__ void load(const void *base, int64_t idx, float scale, float2 (&v)[P])
    {
        const uint32_t *p = reinterpret_cast<const uint32_t *>(base) + idx * P;
        if constexpr (P == 1) {
            v[0] = cvt(__ldg(p), scale);
        } else if constexpr (P == 2) {
            uint2 q = __ldg(reinterpret_cast<const uint2 *>(p));
            v[0] = cvt(q.x, scale);
            v[1] = cvt(q.y, scale);
        } else {
            uint4 q = __ldg(reinterpret_cast<const uint4 *>(p));
            v[0] = cvt(q.x, scale);
            v[1] = cvt(q.y, scale);
            v[2] = cvt(q.z, scale);
            v[3] = cvt(q.w, scale);
        }
    }
};

template <int P>
struct VisLoad<P, VISTA_VIS_BF16X2> {
    static __device__ __forceinline__ float2 cvt(uint32_t b, float scale)
    {
        // bf16 -> f32 is a 16-bit shift
        float re = __uint_as_float(b << 16), im = __uint_as_float(b & 0xffff0000u);
        return make_float2(re * scale, im * scale);
    }
    static __device__ __forceinline__ void load(const void *base, int64_t idx, float scale, float2 (&v)[P])
    {
        const uint32_t *p = reinterpret_cast<const uint32_t *>(base) + idx * P;
        if constexpr (P == 1) {
            v[0] = cvt(__ldg(p), scale);
        } else if constexpr (P == 2) {
            uint2 q = __ldg(reinterpret_cast<const uint2 *>(p));
            v[0] = cvt(q.x, scale);
            v[1] = cvt(q.y, scale);
        } else {
            uint4 q = __ldg(reinterpret_cast<const uint4 *>(p));
            v[0] = cvt(q.x, scale);
            v[1] = cvt(q.y, scale);
            v[2] = cvt(q.z, scale);
            v[3] = cvt(q.w, scale);
        }
    }
};

template <int P>
__device__ __forceinline__ uint32_t load_flags(const uint8_t *flags, int64_t idx)
{
    if (!flags) return 0u;
    const uint8_t *p = flags + idx * P;
    if constexpr (P == 1) return (uint32_t)__ldg(p);
    else if constexpr (P == 2) return (uint32_t)__ldg(reinterpret_cast<const uint16_t *>(p));
    else return __ldg(reinterpret_cast<const uint32_t *>(p));
}

// ---------------------------------------------------------------- prepass

__global__ void __launch_bounds__(256) prepass_mixed(RunArgs a, int cw)
{
    int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= a.nrows_total) return;
    int s = find_owner(a.row_off, a.nsrc, gid);
    const SrcDev &S = a.srcs[s];
    int64_t r = gid - a.row_off[s];
    const double *uvw = S.uvw + 3 * r;
    double u = uvw[0], v = uvw[1], w = uvw[2];
    bool fold = a.g.fold && (v < 0.0 || (v == 0.0 && u < 0.0));
    double tau = u * S.l + v * S.m + w * S.n1;
    RowRec rec;
    rec.u = (float)(fold ? -u : u);
    rec.v = (float)(fold ? -v : v);
    rec.rowf = (uint32_t)r | (fold ? 0x80000000u : 0u);
#pragma unroll
    for (int p = 0; p < 4; ++p) rec.W[p] = p < S.npol ? S.wts[r * S.npol + p] : 0.0f;
    if (S.linear) {
        double D = tau * S.step_c;
        D -= floor(D);
        double Dhi = floor(D * 524288.0) * (1.0 / 524288.0);
        rec.dhi = (float)Dhi;
        rec.dlo = (float)(D - Dhi);
        double D32 = 32.0 * D;
        D32 -= floor(D32);
        float2 st = turns_to_phasor((float)D32);
        rec.sre = st.x;
        rec.sim = st.y;
    } else {
        rec.dhi = __int_as_float(__double2hiint(tau));
        rec.dlo = __int_as_float(__double2loint(tau));
        rec.sre = 1.0f;
        rec.sim = 0.0f;
    }
    const ChanD *cd = a.chd + S.chan_off;
    RowRec *out = a.recs + S.rec_off + r;
    for (int c = 0; c < S.nchunk; ++c) {
        double t = tau * (cd[c * cw].nu * (1.0 / C_LIGHT));
        t -= floor(t);
        rec.t0 = (float)t;
        out[(int64_t)c * S.nrow] = rec;
    }
}

// ------------------------------------------------------------ stack_mixed

template <int P, int VT, int NS>
__global__ void __launch_bounds__(256) stack_mixed(RunArgs a, int rows_per_item)
{
    const int lane = threadIdx.x & 31;
    const int64_t item = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (item >= a.nitems_total) return;
    const int s = find_owner(a.item_off, a.nsrc, item);
    const SrcDev &S = a.srcs[s];
    const int64_t nrow = S.nrow;
    const int64_t ntile = (nrow + rows_per_item - 1) / rows_per_item;
    const int64_t li = item - a.item_off[s];
    const int chunk = (int)(li / ntile);
    const int64_t i0 = (li % ntile) * rows_per_item;
    const int64_t i1 = min(nrow, i0 + rows_per_item);
    const int c0 = S.k_lo + chunk * 32 * NS;
    const int nchan = S.nchan, npol_c = a.g.npol, nrest = a.g.nrest;
    const bool linear = S.linear != 0;
    const void *vis = S.vis;
    const uint8_t *flags = S.flags;
    const float vscale = S.vis_scale;

    int plane[P];
#pragma unroll
    for (int p = 0; p < P; ++p) plane[p] = S.plane[p];

    // channel slots of this lane
    float su[NS], sv[NS], wb[NS][4];
    int j0[NS], nb[NS], kk[NS];
#pragma unroll
    for (int q = 0; q < NS; ++q) {
        kk[q] = c0 + q * 32 + lane;
        nb[q] = 0;
        j0[q] = 0;
        su[q] = sv[q] = 0.f;
#pragma unroll
        for (int b = 0; b < 4; ++b) wb[q][b] = 0.f;
        if (kk[q] < S.k_hi) {
            const ChanF cf = a.chf[S.chan_off + (kk[q] - S.k_lo)];
            su[q] = cf.su;
            sv[q] = cf.sv;
            j0[q] = cf.j0;
            nb[q] = cf.nb;
#pragma unroll
            for (int b = 0; b < 4; ++b) wb[q][b] = cf.w[b];
        }
    }

    int cell[NS];
    float4 acc[NS][P];
    uint32_t cnt[NS][P];
#pragma unroll
    for (int q = 0; q < NS; ++q) {
        cell[q] = -1;
#pragma unroll
        for (int p = 0; p < P; ++p) {
            acc[q][p] = make_float4(0.f, 0.f, 0.f, 0.f);
            cnt[q][p] = 0;
        }
    }
    uint32_t n_vis = 0, n_flag = 0, n_duv = 0, n_stk = 0;
    float4 *cube4 = reinterpret_cast<float4 *>(a.cube);

    auto flush = [&](int q) {
        if (cell[q] < 0) return;
#pragma unroll
        for (int p = 0; p < P; ++p) {
            if (cnt[q][p] == 0) continue;
            const size_t base = ((size_t)cell[q] * nrest + j0[q]) * npol_c + plane[p];
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                if (b < nb[q]) {
                    const float ww = wb[q][b];
                    atomicAdd(cube4 + base + (size_t)b * npol_c,
                              make_float4(ww * acc[q][p].x, ww * acc[q][p].y, ww * acc[q][p].z,
                                          ww * acc[q][p].w));
                    atomicAdd(a.count + base + (size_t)b * npol_c, cnt[q][p]);
                }
            }
            acc[q][p] = make_float4(0.f, 0.f, 0.f, 0.f);
            cnt[q][p] = 0;
        }
    };

    const RowRec *recs = a.recs + S.rec_off + (int64_t)chunk * nrow;
    for (int64_t i = i0; i < i1; ++i) {
        const RowRec rec = recs[i];
        const int64_t row = (int64_t)(rec.rowf & 0x7fffffffu);
        const bool fold = (rec.rowf >> 31) != 0;
        float2 ph;
        double tau = 0.0;
        if (linear) {
            ph = lane_seed(rec, lane);
        } else {
            tau = __hiloint2double(__float_as_int(rec.dhi), __float_as_int(rec.dlo));
        }
        const float2 stp = make_float2(rec.sre, rec.sim);
#pragma unroll
        for (int q = 0; q < NS; ++q) {
            if (!linear && kk[q] < S.k_hi) {
                double t = tau * (a.chd[S.chan_off + (kk[q] - S.k_lo)].nu * (1.0 / C_LIGHT));
                t -= floor(t);
                ph = turns_to_phasor((float)t);
            }
            if (nb[q] > 0) {
                const int iu = axis_cell(rec.u, su[q], S.uvw + 3 * row, fold,
                                         &a.chd[S.chan_off + (kk[q] - S.k_lo)].su, a.g.nu);
                const int iv = axis_cell(rec.v, sv[q], S.uvw + 3 * row + 1, fold,
                                         &a.chd[S.chan_off + (kk[q] - S.k_lo)].sv, a.g.nv);
                const int cid = (iu >= 0 && iv >= 0) ? iv * a.g.nu + iu : -1;
                const int64_t vidx = row * nchan + kk[q];
                float2 V[P];
                VisLoad<P, VT>::load(vis, vidx, vscale, V);
                const uint32_t fl = load_flags<P>(flags, vidx);
                if (cid != cell[q]) {
                    flush(q);
                    cell[q] = cid;
                }
#pragma unroll
                for (int p = 0; p < P; ++p) {
                    if (plane[p] < 0) continue;
                    const bool f = ((fl >> (8 * p)) & 0xffu) != 0;
                    ++n_vis;
                    if (f) {
                        ++n_flag;
                        continue;
                    }
                    if (cid < 0) {
                        ++n_duv;
                        continue;
                    }
                    ++n_stk;
                    float2 vs = cmul(V[p], ph);
                    if (fold) vs.y = -vs.y;
                    const float W = rec.W[p];
                    const float a2 = V[p].x * V[p].x + V[p].y * V[p].y;
                    acc[q][p].x += W * vs.x;
                    acc[q][p].y += W * vs.y;
                    acc[q][p].z += W;
                    acc[q][p].w += W * a2;
                    cnt[q][p] += 1;
                }
            }
            if (linear) ph = cmul(ph, stp);
        }
    }
#pragma unroll
    for (int q = 0; q < NS; ++q) flush(q);

    // counters: warp sum, one atomic per counter per item
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        n_vis += __shfl_xor_sync(0xffffffffu, n_vis, o);
        n_flag += __shfl_xor_sync(0xffffffffu, n_flag, o);
        n_duv += __shfl_xor_sync(0xffffffffu, n_duv, o);
        n_stk += __shfl_xor_sync(0xffffffffu, n_stk, o);
    }
    if (lane == 0) {
        if (n_vis) atomicAdd(&a.stats->n_vis, (unsigned long long)n_vis);
        if (n_flag) atomicAdd(&a.stats->n_flagged, (unsigned long long)n_flag);
        if (n_duv) atomicAdd(&a.stats->n_dropped_uv, (unsigned long long)n_duv);
        if (n_stk) atomicAdd(&a.stats->n_stacked, (unsigned long long)n_stk);
    }
}

// Debug export: the same seed/recurrence/cell code as stack_mixed, writing
// the phasor and the cell of every (row, channel) of one window.
template <int NS>
__global__ void debug_mixed(RunArgs a, int src, double *ph_out, int32_t *cell_out)
{
    const int lane = threadIdx.x & 31;
    const SrcDev &S = a.srcs[src];
    const int64_t nrow = S.nrow;
    const int64_t task = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (task >= nrow * S.nchunk) return;
    const int chunk = (int)(task / nrow);
    const int64_t i = task % nrow;
    const int c0 = S.k_lo + chunk * 32 * NS;
    const RowRec rec = a.recs[S.rec_off + (int64_t)chunk * nrow + i];
    const int64_t row = (int64_t)(rec.rowf & 0x7fffffffu);
    const bool fold = (rec.rowf >> 31) != 0;
    const bool linear = S.linear != 0;
    float2 ph = make_float2(1.f, 0.f);
    double tau = 0.0;
    if (linear) ph = lane_seed(rec, lane);
    else tau = __hiloint2double(__float_as_int(rec.dhi), __float_as_int(rec.dlo));
    const float2 stp = make_float2(rec.sre, rec.sim);
#pragma unroll
    for (int q = 0; q < NS; ++q) {
        const int k = c0 + q * 32 + lane;
        if (k < S.k_hi) {
            const ChanD *cd = a.chd + S.chan_off + (k - S.k_lo);
            const ChanF cf = a.chf[S.chan_off + (k - S.k_lo)];
            if (!linear) {
                double t = tau * (cd->nu * (1.0 / C_LIGHT));
                t -= floor(t);
                ph = turns_to_phasor((float)t);
            }
            const int iu = axis_cell(rec.u, cf.su, S.uvw + 3 * row, fold, &cd->su, a.g.nu);
            const int iv = axis_cell(rec.v, cf.sv, S.uvw + 3 * row + 1, fold, &cd->sv, a.g.nv);
            const int64_t o = row * S.nchan + k;
            if (ph_out) {
                ph_out[2 * o] = (double)ph.x;
                ph_out[2 * o + 1] = (double)ph.y;
            }
            if (cell_out) {
                const bool ok = iu >= 0 && iv >= 0;
                cell_out[2 * o] = ok ? iu : -1;
                cell_out[2 * o + 1] = ok ? iv : -1;
            }
        }
        if (linear) ph = cmul(ph, stp);
    }
}

// ------------------------------------------------------------- stack_fp64

__device__ __forceinline__ double2 turns_to_phasor64(double t)
{
    double s, c;
    sincospi(2.0 * t, &s, &c);
    return make_double2(c, s);
}

__device__ __forceinline__ double2 cmul64(double2 a, double2 b)
{
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

template <bool EXPORT>
__global__ void __launch_bounds__(128) stack_fp64(RunArgs a, int only_src, double *ph_out, int32_t *cell_out)
{
    int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= a.nrows_total) return;
    const int s = find_owner(a.row_off, a.nsrc, gid);
    if (EXPORT && s != only_src) return;
    const SrcDev &S = a.srcs[s];
    const int64_t r = gid - a.row_off[s];
    const double *uvw = S.uvw + 3 * r;
    double u = uvw[0], v = uvw[1], w = uvw[2];
    const bool fold = a.g.fold && (v < 0.0 || (v == 0.0 && u < 0.0));
    const double tau = u * S.l + v * S.m + w * S.n1;
    if (fold) {
        u = -u;
        v = -v;
    }
    const int npol = S.npol, nrest = a.g.nrest, npol_c = a.g.npol;
    double W[4];
    for (int p = 0; p < 4; ++p) W[p] = p < npol ? (double)S.wts[r * npol + p] : 0.0;
    const ChanD *cd = a.chd + S.chan_off;
    double2 ph = make_double2(1.0, 0.0), stp = make_double2(1.0, 0.0);
    if (S.linear && S.k_hi > S.k_lo) {
        double t = tau * (cd[0].nu * (1.0 / C_LIGHT));
        ph = turns_to_phasor64(t - floor(t));
        double d = tau * S.step_c;
        stp = turns_to_phasor64(d - floor(d));
    }
    double *cube = reinterpret_cast<double *>(a.cube);
    unsigned long long n_vis = 0, n_flag = 0, n_duv = 0, n_stk = 0;
    for (int k = S.k_lo; k < S.k_hi; ++k) {
        const ChanD c = cd[k - S.k_lo];
        if (!S.linear) {
            double t = tau * (c.nu * (1.0 / C_LIGHT));
            ph = turns_to_phasor64(t - floor(t));
        }
        if (c.nb > 0) {
            const int iu = axis_cell64(u, c.su, a.g.nu);
            const int iv = axis_cell64(v, c.sv, a.g.nv);
            const bool inuv = iu >= 0 && iv >= 0;
            if (EXPORT) {
                const int64_t o = r * S.nchan + k;
                if (ph_out) {
                    ph_out[2 * o] = ph.x;
                    ph_out[2 * o + 1] = ph.y;
                }
                if (cell_out) {
                    cell_out[2 * o] = inuv ? iu : -1;
                    cell_out[2 * o + 1] = inuv ? iv : -1;
                }
            } else {
                const int64_t vi = (r * S.nchan + k) * npol;
                for (int p = 0; p < npol; ++p) {
                    const int q = S.plane[p];
                    if (q < 0) continue;
                    ++n_vis;
                    if (S.flags && S.flags[vi + p]) {
                        ++n_flag;
                        continue;
                    }
                    if (!inuv) {
                        ++n_duv;
                        continue;
                    }
                    ++n_stk;
                    double vr, vim;
                    if (S.vis_type == VISTA_VIS_C128) {
                        const double2 z2 = reinterpret_cast<const double2 *>(S.vis)[vi + p];
                        vr = z2.x;
                        vim = z2.y;
                    } else if (S.vis_type == VISTA_VIS_C64) {
                        const float2 z2 = reinterpret_cast<const float2 *>(S.vis)[vi + p];
                        vr = z2.x;
                        vim = z2.y;
                    } else if (S.vis_type == VISTA_VIS_F16X2) {
                        const __half2 h = reinterpret_cast<const __half2 *>(S.vis)[vi + p];
                        vr = (double)__low2float(h) * (double)S.vis_scale;
                        vim = (double)__high2float(h) * (double)S.vis_scale;
                    } else {
                        const __nv_bfloat162 h = reinterpret_cast<const __nv_bfloat162 *>(S.vis)[vi + p];
                        vr = (double)__low2float(h) * (double)S.vis_scale;
                        vim = (double)__high2float(h) * (double)S.vis_scale;
                    }
                    double sr = vr * ph.x - vim * ph.y;
                    double si = vr * ph.y + vim * ph.x;
                    if (fold) si = -si;
                    const double a2 = vr * vr + vim * vim;
                    const size_t base = (((size_t)(iv * a.g.nu + iu) * nrest + c.j0) * npol_c + q);
                    for (int b = 0; b < c.nb; ++b) {
                        const double ww = W[p] * c.w[b];
                        double *e = cube + 4 * (base + (size_t)b * npol_c);
                        atomicAdd(e + 0, ww * sr);
                        atomicAdd(e + 1, ww * si);
                        atomicAdd(e + 2, ww);
                        atomicAdd(e + 3, ww * a2);
                        atomicAdd(a.count + base + (size_t)b * npol_c, 1u);
                    }
                }
            }
        }
        if (S.linear) ph = cmul64(ph, stp);
    }
    if (!EXPORT) {
        if (n_vis) atomicAdd(&a.stats->n_vis, n_vis);
        if (n_flag) atomicAdd(&a.stats->n_flagged, n_flag);
        if (n_duv) atomicAdd(&a.stats->n_dropped_uv, n_duv);
        if (n_stk) atomicAdd(&a.stats->n_stacked, n_stk);
    }
}

// ------------------------------------------------------------------ unpack

__global__ void unpack_kernel(const void *cube, const uint32_t *count, int fp64, int64_t n,
                              void *sum_wv, void *sum_w, void *sum_wvv, uint32_t *cnt_out, int out_f64)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double e[4];
        if (fp64) {
            const double *c = reinterpret_cast<const double *>(cube) + 4 * i;
            e[0] = c[0];
            e[1] = c[1];
            e[2] = c[2];
            e[3] = c[3];
        } else {
            const float4 c = reinterpret_cast<const float4 *>(cube)[i];
            e[0] = c.x;
            e[1] = c.y;
            e[2] = c.z;
            e[3] = c.w;
        }
        if (out_f64) {
            if (sum_wv) {
                reinterpret_cast<double *>(sum_wv)[2 * i] = e[0];
                reinterpret_cast<double *>(sum_wv)[2 * i + 1] = e[1];
            }
            if (sum_w) reinterpret_cast<double *>(sum_w)[i] = e[2];
            if (sum_wvv) reinterpret_cast<double *>(sum_wvv)[i] = e[3];
        } else {
            if (sum_wv) {
                reinterpret_cast<float *>(sum_wv)[2 * i] = (float)e[0];
                reinterpret_cast<float *>(sum_wv)[2 * i + 1] = (float)e[1];
            }
            if (sum_w) reinterpret_cast<float *>(sum_w)[i] = (float)e[2];
            if (sum_wvv) reinterpret_cast<float *>(sum_wvv)[i] = (float)e[3];
        }
        if (cnt_out) cnt_out[i] = count[i];
    }
}

// --------------------------------------------------------------- launchers

template <int P, int VT>
static cudaError_t launch_mixed_p(const RunArgs &a, const LaunchCfg &c, cudaStream_t st)
{
    const int wpb = c.warps_per_cta;
    const int64_t blocks = (a.nitems_total + wpb - 1) / wpb;
    if (blocks == 0) return cudaSuccess;
    switch (c.chans_per_lane) {
    case 1: stack_mixed<P, VT, 1><<<(unsigned)blocks, wpb * 32, 0, st>>>(a, c.rows_per_item); break;
    case 2: stack_mixed<P, VT, 2><<<(unsigned)blocks, wpb * 32, 0, st>>>(a, c.rows_per_item); break;
    case 4: stack_mixed<P, VT, 4><<<(unsigned)blocks, wpb * 32, 0, st>>>(a, c.rows_per_item); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <int VT>
static cudaError_t launch_mixed_vt(const RunArgs &a, const LaunchCfg &c, int npol, cudaStream_t st)
{
    switch (npol) {
    case 1: return launch_mixed_p<1, VT>(a, c, st);
    case 2: return launch_mixed_p<2, VT>(a, c, st);
    case 4: return launch_mixed_p<4, VT>(a, c, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_prepass(const RunArgs &a, const LaunchCfg &c, cudaStream_t st)
{
    if (a.nrows_total == 0) return cudaSuccess;
    const int64_t blocks = (a.nrows_total + 255) / 256;
    prepass_mixed<<<(unsigned)blocks, 256, 0, st>>>(a, 32 * c.chans_per_lane);
    return cudaGetLastError();
}

cudaError_t launch_mixed(const RunArgs &a, const LaunchCfg &c, int npol_vt, cudaStream_t st)
{
    // npol_vt packs (vis_type << 8) | npol: one (type, npol) class per launch.
    const int npol = npol_vt & 0xff, vt = npol_vt >> 8;
    switch (vt) {
    case VISTA_VIS_C64: return launch_mixed_vt<VISTA_VIS_C64>(a, c, npol, st);
    case VISTA_VIS_C128: return launch_mixed_vt<VISTA_VIS_C128>(a, c, npol, st);
    case VISTA_VIS_F16X2: return launch_mixed_vt<VISTA_VIS_F16X2>(a, c, npol, st);
    case VISTA_VIS_BF16X2: return launch_mixed_vt<VISTA_VIS_BF16X2>(a, c, npol, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_fp64(const RunArgs &a, cudaStream_t st)
{
    if (a.nrows_total == 0) return cudaSuccess;
    const int64_t blocks = (a.nrows_total + 127) / 128;
    stack_fp64<false><<<(unsigned)blocks, 128, 0, st>>>(a, -1, nullptr, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_unpack(const void *cube, const uint32_t *count, int fp64, int64_t n, void *sum_wv,
                          void *sum_w, void *sum_wvv, uint32_t *cnt_out, int out_f64, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    unpack_kernel<<<(unsigned)blocks, 256, 0, st>>>(cube, count, fp64, n, sum_wv, sum_w, sum_wvv, cnt_out,
                                                     out_f64);
    return cudaGetLastError();
}

cudaError_t launch_debug(const RunArgs &a, const LaunchCfg &c, int src, int fp64, double *ph,
                         int32_t *cells, cudaStream_t st)
{
    if (fp64) {
        if (a.nrows_total == 0) return cudaSuccess;
        const int64_t blocks = (a.nrows_total + 127) / 128;
        stack_fp64<true><<<(unsigned)blocks, 128, 0, st>>>(a, src, ph, cells);
        return cudaGetLastError();
    }
    SrcDev S;
    cudaError_t e = cudaMemcpyAsync(&S, a.srcs + src, sizeof(S), cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return e;
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    const int64_t tasks = S.nrow * S.nchunk;
    if (tasks == 0) return cudaSuccess;
    const int64_t blocks = (tasks + 3) / 4;
    switch (c.chans_per_lane) {
    case 1: debug_mixed<1><<<(unsigned)blocks, 128, 0, st>>>(a, src, ph, cells); break;
    case 2: debug_mixed<2><<<(unsigned)blocks, 128, 0, st>>>(a, src, ph, cells); break;
    case 4: debug_mixed<4><<<(unsigned)blocks, 128, 0, st>>>(a, src, ph, cells); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace vista

// Device helpers shared by the libvista kernels: work-list lookups, FP32
// phasors, the guarded uv-cell rule and the visibility / flag loaders.
#pragma once
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

// ---- TMA bulk copies into shared memory, completed on an mbarrier ----

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

// 1-D bulk copy global -> shared (16-byte aligned addresses, size a multiple of 16).
__device__ __forceinline__ void tma_load_1d(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: gives up after ~2^24 polls (seconds), records the failure in
// the error word and returns false; never traps and never spins forever.
constexpr int32_t ERR_WAIT_TIMEOUT = 1;
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, int32_t *err)
{
    for (uint32_t i = 0; i < (1u << 24); ++i)
        if (mbar_try_wait(bar, parity)) return true;
    atomicExch(err, ERR_WAIT_TIMEOUT);
    return false;
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// exp(2 pi i t) for a reduced turn count |t| <= 1/2 (|2 pi t| <= pi).
// CUDA's __sincosf has an absolute error of at most 2^-21.41 on [-pi, pi]
// (CUDA C Programming Guide, intrinsic functions), i.e. a phase error below
// 5e-7 rad, inside the 1e-5 rad budget, in two special-function-unit
// instructions.
__device__ __forceinline__ float2 turns_to_phasor(float t)
{
    float s, c;
    __sincosf(__fmul_rn(t, 6.28318530717958648f), &s, &c);
    return make_float2(c, s);
}

// exp(+2 pi i tau nu_k / c) from tau and nu_k / c given as float-float
// pairs.  The product is formed as p + e + x: p = fl(tau_hi nuc_hi), e its
// exact rounding error (one FMA), x the cross terms; tau_lo nuc_lo is below
// 2^-48 of the product and dropped.  p minus its nearest integer is exact, so
// the turns reach turns_to_phasor reduced, with an error of about 2^-25 turn
// (2e-7 rad) for phases up to 2^23 turns.
__device__ __forceinline__ float2 shift_phasor(float tau_hi, float tau_lo, float nuc_hi, float nuc_lo)
{
    const float p = __fmul_rn(tau_hi, nuc_hi);
    const float e = __fmaf_rn(tau_hi, nuc_hi, -p);
    const float x = __fmaf_rn(tau_hi, nuc_lo, __fmaf_rn(tau_lo, nuc_hi, e));
    const float r = __fsub_rn(p, rintf(p));
    return turns_to_phasor(__fadd_rn(r, x));
}

// Split a double into a float-float pair hi + lo.
__device__ __host__ __forceinline__ void split_ff(double x, float &hi, float &lo)
{
    hi = (float)x;
    lo = (float)(x - (double)hi);
}

// One axis of the uv cell: floor(fl64(coord * s_k)) + n/2, or -1 outside
// [0, n).  Decided in FP32 when fl32(c32 * s32) is at least 2^-21 |x| away
// from an integer (the FP32 product differs from the FP64 one by at most
// 3 * 2^-24 |x|), else by the exact FP64 product.
// The exact FP64 product, out of line so that the compiler cannot hoist it
// (and its FP64 work) out of the rarely taken branch below.
static __device__ __noinline__ float exact_floor_product(const double *coord64, bool neg, const double *s64)
{
    double c = *coord64;
    if (neg) c = -c;
    return (float)floor(__dmul_rn(c, *s64));
}

// floor(fl64(coord * s_k)) as a float (exact; see axis_cell).
__device__ __forceinline__ float axis_floor(float c32, float s32, const double *coord64, bool neg,
                                            const double *s64)
{
    float x = __fmul_rn(c32, s32);
    float d = __fmaf_rn(fabsf(x), 4.76837158203125e-07f, 1e-30f);
    float fa = floorf(__fsub_rn(x, d)), fb = floorf(__fadd_rn(x, d));
    float fx = fa;
    if (__builtin_expect(fa != fb, 0)) fx = exact_floor_product(coord64, neg, s64);
    return fx;
}

__device__ __forceinline__ int axis_cell(float c32, float s32, const double *coord64, bool neg,
                                         const double *s64, int n)
{
    const float fx = axis_floor(c32, s32, coord64, neg, s64);
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

// Eq. 1: the gridding coordinates (u', v') = the first two rows of R (u, v, w)
// of one row of a re-projected window, each product and sum rounded in the
// order written (no FMA, as the oracle), so that the FP64 cell rule applied
// to them is exact.  Stored at g[0], g[1] (g[2], w', is not needed: the delay
// uses the stored baseline); returned as well.
__device__ __forceinline__ double2 rotate_row(const double *R, const double *x, double *g)
{
    const double a = x[0], b = x[1], c = x[2];
    const double u = __dadd_rn(__dadd_rn(__dmul_rn(R[0], a), __dmul_rn(R[1], b)), __dmul_rn(R[2], c));
    const double v = __dadd_rn(__dadd_rn(__dmul_rn(R[3], a), __dmul_rn(R[4], b)), __dmul_rn(R[5], c));
    g[0] = u;
    g[1] = v;
    return make_double2(u, v);
}

// The cell iv * nu + iu of channel `cd` of one row by the FP64 rule, -1 off
// the grid (the fall-back of CC_MIXED chunks; out of line, rarely run).
static __device__ __noinline__ int cell_exact(const double *uvw, int64_t row, bool fold, const ChanD *cd, int nu,
                                              int nv)
{
    double u = uvw[3 * row], v = uvw[3 * row + 1];
    if (fold) {
        u = -u;
        v = -v;
    }
    const int iu = axis_cell64(u, cd->su, nu), iv = axis_cell64(v, cd->sv, nv);
    return (iu >= 0 && iv >= 0) ? iv * nu + iu : -1;
}

// Cell of chunk-local channel kk from a chunk-cell entry that is neither
// CC_NOCHANGE nor CC_MIXED.
__device__ __forceinline__ int chunk_cell_step(int2 cc, int kk, int nu)
{
    const uint32_t m = (uint32_t)cc.y;
    int c = cc.x;
    if (kk >= (int)(m & 0xffu)) c += (m & 0x10000u) ? -1 : 1;
    if (kk >= (int)((m >> 8) & 0xffu)) c += (m & 0x20000u) ? -nu : nu;
    return c;
}

// ----------------------------------------------------------- vis loaders

template <int P, int VT>
struct VisLoad;

template <int P>
struct VisLoad<P, VISTA_VIS_C64> {
    static constexpr int kBytes = 8;   // bytes per complex value
    static __device__ __forceinline__ void load(const void *base, int64_t idx, float scale, float2 (&v)[P])
    {
        (void)scale;
        const float2 *p = reinterpret_cast<const float2 *>(base) + idx * P;
        if constexpr (P == 1) {
            v[0] = __ldcs(p);
        } else if constexpr (P == 2) {
            float4 q = __ldcs(reinterpret_cast<const float4 *>(p));
            v[0] = make_float2(q.x, q.y);
            v[1] = make_float2(q.z, q.w);
        } else {
            float4 q0 = __ldcs(reinterpret_cast<const float4 *>(p));
            float4 q1 = __ldcs(reinterpret_cast<const float4 *>(p) + 1);
            v[0] = make_float2(q0.x, q0.y);
            v[1] = make_float2(q0.z, q0.w);
            v[2] = make_float2(q1.x, q1.y);
            v[3] = make_float2(q1.z, q1.w);
        }
    }
};

template <int P>
struct VisLoad<P, VISTA_VIS_C128> {
    static constexpr int kBytes = 16;
    static __device__ __forceinline__ void load(const void *base, int64_t idx, float scale, float2 (&v)[P])
    {
        (void)scale;
        const double2 *p = reinterpret_cast<const double2 *>(base) + idx * P;
#pragma unroll
        for (int i = 0; i < P; ++i) {
            double2 q = __ldcs(p + i);
            v[i] = make_float2((float)q.x, (float)q.y);
        }
    }
};


template <int P>
struct VisLoad<P, VISTA_VIS_F16X2> {
    static constexpr int kBytes = 4;
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
            v[0] = cvt(__ldcs(p), scale);
        } else if constexpr (P == 2) {
            uint2 q = __ldcs(reinterpret_cast<const uint2 *>(p));
            v[0] = cvt(q.x, scale);
            v[1] = cvt(q.y, scale);
        } else {
            uint4 q = __ldcs(reinterpret_cast<const uint4 *>(p));
            v[0] = cvt(q.x, scale);
            v[1] = cvt(q.y, scale);
            v[2] = cvt(q.z, scale);
            v[3] = cvt(q.w, scale);
        }
    }
};

template <int P>
struct VisLoad<P, VISTA_VIS_BF16X2> {
    static constexpr int kBytes = 4;
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
            v[0] = cvt(__ldcs(p), scale);
        } else if constexpr (P == 2) {
            uint2 q = __ldcs(reinterpret_cast<const uint2 *>(p));
            v[0] = cvt(q.x, scale);
            v[1] = cvt(q.y, scale);
        } else {
            uint4 q = __ldcs(reinterpret_cast<const uint4 *>(p));
            v[0] = cvt(q.x, scale);
            v[1] = cvt(q.y, scale);
            v[2] = cvt(q.z, scale);
            v[3] = cvt(q.w, scale);
        }
    }
};

// ---- asynchronous copies of one lane's visibilities into shared memory ----

__device__ __forceinline__ void cp_async_16(uint32_t dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_8(uint32_t dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_4(uint32_t dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// One lane's P values of one (row, channel): kLaneBytes bytes, naturally
// aligned (a multiple of the element size), copied by cp.async in 16-, 8- or
// 4-byte pieces and decoded from shared memory.
template <int P, int VT>
struct VisAsync {
    static constexpr int kLaneBytes = P * VisLoad<P, VT>::kBytes;
    static __device__ __forceinline__ void copy(uint32_t dst, const void *src)
    {
        const char *s = reinterpret_cast<const char *>(src);
        if constexpr (kLaneBytes % 16 == 0) {
#pragma unroll
            for (int i = 0; i < kLaneBytes / 16; ++i) cp_async_16(dst + 16 * i, s + 16 * i);
        } else if constexpr (kLaneBytes == 8) {
            cp_async_8(dst, s);
        } else {
            static_assert(kLaneBytes == 4, "lane bytes");
            cp_async_4(dst, s);
        }
    }
    static __device__ __forceinline__ void decode(const void *sm, float scale, float2 (&v)[P])
    {
        if constexpr (VT == VISTA_VIS_C64) {
            const float2 *q = reinterpret_cast<const float2 *>(sm);
#pragma unroll
            for (int i = 0; i < P; ++i) v[i] = q[i];
        } else if constexpr (VT == VISTA_VIS_C128) {
            const double2 *q = reinterpret_cast<const double2 *>(sm);
#pragma unroll
            for (int i = 0; i < P; ++i) v[i] = make_float2((float)q[i].x, (float)q[i].y);
        } else {
            const uint32_t *q = reinterpret_cast<const uint32_t *>(sm);
#pragma unroll
            for (int i = 0; i < P; ++i) v[i] = VisLoad<P, VT>::cvt(q[i], scale);
        }
    }
};

}  // namespace vista

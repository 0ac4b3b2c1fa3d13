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

// exp(2 pi i t) for t in turns, for |t| < 2^21.
//
// Own evaluation (textbook quadrant reduction + Taylor series): x = 4t is
// split into the nearest integer q (quadrant) and r in [-1/2, 1/2]
// (exact: Sterbenz), theta = r pi/2 in [-pi/4, pi/4], then
//   sin theta = theta (1 - theta^2/3! + theta^4/5! - theta^6/7! + theta^8/9!)
//   cos theta = 1 - theta^2/2! + theta^4/4! - theta^6/6! + theta^8/8!
// whose truncation errors on |theta| <= pi/4 are below 2e-9 and 3e-8, and
// finally exp(i (q pi/2 + theta)) by rotating (cos, sin) q quarter turns.
// The phase error is a few 1e-8 rad, far inside the 1e-5 rad budget.
__device__ __forceinline__ float2 turns_to_phasor(float t)
{
    const float x = 4.0f * t;                 // exact
    const float q = rintf(x);
    const float r = __fsub_rn(x, q);          // exact, |r| <= 1/2
    const float th = r * 1.57079632679489662f;
    const float t2 = th * th;
    float s = __fmaf_rn(t2, 2.75573192e-06f, -1.98412698e-04f);   // 1/9!, -1/7!
    s = __fmaf_rn(t2, s, 8.33333333e-03f);                          // 1/5!
    s = __fmaf_rn(t2, s, -1.66666667e-01f);                         // -1/3!
    s = __fmaf_rn(t2 * th, s, th);
    float c = __fmaf_rn(t2, 2.48015873e-05f, -1.38888889e-03f);    // 1/8!, -1/6!
    c = __fmaf_rn(t2, c, 4.16666667e-02f);                          // 1/4!
    c = __fmaf_rn(t2, c, -0.5f);
    c = __fmaf_rn(t2, c, 1.0f);
    const int qi = ((int)q) & 3;
    const float cs = (qi & 1) ? s : c, sn = (qi & 1) ? c : s;
    return make_float2((qi == 1 || qi == 2) ? -cs : cs, (qi >= 2) ? -sn : sn);
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

template <int P>
__device__ __forceinline__ uint32_t load_flags(const uint8_t *flags, int64_t idx)
{
    if (!flags) return 0u;
    const uint8_t *p = flags + idx * P;
    if constexpr (P == 1) return (uint32_t)__ldcs(p);
    else if constexpr (P == 2) return (uint32_t)__ldcs(reinterpret_cast<const uint16_t *>(p));
    else return __ldcs(reinterpret_cast<const uint32_t *>(p));
}

}  // namespace vista

// vista_contsub(): continuum subtraction over the rest axis of the cube.
//
// The paper names continuum subtraction as the first post-processing step of
// the stacked output (Sec. 3.4); here it is the uv-plane form of that step.
// For every uv cell and cube plane, a polynomial of degree
// d = min(order, |F| - 1) in x_j = (2 j - (nrest - 1)) / nrest is fitted by
// weighted least squares to the cell's spectrum V_j = sum_wv_j / sum_w_j
// over F = { j : line_free[j] and sum_w_j > 0 } (weights sum_w_j), and
//   out_j = sum_wv_j - sum_w_j p(x_j)
// is written for every j.  With V_j sum_w_j = sum_wv_j the normal equations
// need only the cube's sums:
//   A_kl = sum_F sum_w_j x_j^(k+l),   b_k = sum_F x_j^k sum_wv_j.
//
// One warp per uv cell when the plane count divides 32 (lanes over the
// cell's (channel, plane) entries, so every load is contiguous; lane L keeps
// plane L mod npol), else one warp per (cell, plane).  A first pass
// accumulates the moments, the lanes of one plane reduce them, every lane
// solves its plane's (d+1) x (d+1) system by Cholesky in FP64, and a second
// pass writes the output.  The per-entry work avoids GB300's slow FP64 pipe:
// each FP64 value (the master sums, or the FP64 cube) is split into a pair
// of floats by integer operations on its bit fields, the moments are
// accumulated as compensated FP32 sums (hi + lo, about 2^-44 relative), and
// the output is formed in FP32 (the output is a float; its error is about
// 2^-23 of |sum_wv| + |sum_w p|).  Memory bound: the entries are read twice
// (with thousands of cells in flight, the second time from DRAM as well)
// and the output written once.
#include "vista_handle.h"

using namespace vista;

namespace {

constexpr int MAX_ORDER = 3;

// The entry's (sum_wv.re, sum_wv.im, sum_w) in FP64: the FP64 cube, or the
// mixed path's FP32 partial plus its FP64 master.
__device__ __forceinline__ double3 entry_sums(const void *cube, const double *master, int fp64, int64_t e)
{
    if (fp64) {
        const double *c = reinterpret_cast<const double *>(cube) + 4 * e;
        return make_double3(c[0], c[1], c[2]);
    }
    const float4 f = reinterpret_cast<const float4 *>(cube)[e];
    double3 r = make_double3(f.x, f.y, f.z);
    if (master) {
        const double *m = master + 4 * e;
        r.x += m[0];
        r.y += m[1];
        r.z += m[2];
    }
    return r;
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// The fitted polynomial's coefficients (lowest power first) from the
// moments M[n] = sum_F w x^n and the right-hand sides B[k] = sum_F x^k wv:
// degree d = min(ORDER, nfit - 1), Cholesky of the normal matrix in FP64
// (positive definite: d + 1 <= nfit distinct abscissae, positive weights),
// then the two triangular solves per part; all zero when nothing is fitted.
template <int ORDER>
__device__ __forceinline__ void solve_fit(const double (&M)[2 * ORDER + 1], const double (&Br)[ORDER + 1],
                                          const double (&Bi)[ORDER + 1], int nfit, double (&cr)[ORDER + 1],
                                          double (&ci)[ORDER + 1])
{
    constexpr int NB = ORDER + 1;
#pragma unroll
    for (int k = 0; k < NB; ++k) cr[k] = ci[k] = 0.0;
    const int d = nfit < 1 ? -1 : (nfit - 1 < ORDER ? nfit - 1 : ORDER);
    if (d >= 0) {
        double L[NB][NB];
#pragma unroll
        for (int r = 0; r < NB; ++r)
#pragma unroll
            for (int c = 0; c < NB; ++c) L[r][c] = 0.0;
#pragma unroll
        for (int r = 0; r < NB; ++r) {
            if (r > d) break;
#pragma unroll
            for (int c = 0; c <= r; ++c) {
                double v = M[r + c];
#pragma unroll
                for (int k = 0; k < c; ++k) v -= L[r][k] * L[c][k];
                L[r][c] = (r == c) ? sqrt(v) : v / L[c][c];
            }
        }
        double yr[NB], yi[NB];
#pragma unroll
        for (int r = 0; r < NB; ++r) {
            if (r > d) break;
            double vr = Br[r], vi = Bi[r];
#pragma unroll
            for (int k = 0; k < r; ++k) {
                vr -= L[r][k] * yr[k];
                vi -= L[r][k] * yi[k];
            }
            yr[r] = vr / L[r][r];
            yi[r] = vi / L[r][r];
        }
#pragma unroll
        for (int r = NB - 1; r >= 0; --r) {
            if (r > d) continue;
            double vr = yr[r], vi = yi[r];
#pragma unroll
            for (int k = r + 1; k < NB; ++k) {
                if (k > d) break;
                vr -= L[k][r] * cr[k];
                vi -= L[k][r] * ci[k];
            }
            cr[r] = vr / L[r][r];
            ci[r] = vi / L[r][r];
        }
    }

}

// A double as hi + lo, two floats: hi is the double truncated to 24
// significant bits, lo the remaining 29 bits rounded to a float (so hi + lo
// is the double to about 2^-47 relative, less where lo falls below the
// normal floats).  Integer and FP32 operations only.  Magnitudes outside
// [2^-126, 2^128) give (0, 0): zero, and values far below any sum of
// weights or visibilities (no sum reaches the upper end).
__device__ __forceinline__ float2 split_double(double d)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(d);
    const int e = (int)((b >> 52) & 0x7ff);
    if (e < 897 || e > 1150) return make_float2(0.f, 0.f);
    const unsigned sign = (unsigned)(b >> 63) << 31;
    const unsigned hi_bits = sign | ((unsigned)(e - 896) << 23) | (unsigned)((b >> 29) & 0x7fffffu);
    // the low 29 mantissa bits times 2^-52 (exact), times 2^(e - 1023)
    const float lo = (__uint2float_rn((unsigned)(b & 0x1fffffffu)) * 0x1p-52f) * __int_as_float((e - 896) << 23);
    return make_float2(__uint_as_float(hi_bits), sign ? -lo : lo);
}

// Compensated accumulation: (s, c) += x with the rounding error of each
// addition (TwoSum) kept in c.
__device__ __forceinline__ void acc2(float &s, float &c, float x)
{
    const float t = s + x, z = t - s;
    c += (s - (t - z)) + (x - z);
    s = t;
}

// Float-pair (hi, lo) arithmetic, about 2^-44 relative.
__device__ __forceinline__ float2 ff_norm(float h, float l)   // |h| >= |l| (Fast2Sum)
{
    const float s = h + l;
    return make_float2(s, l - (s - h));
}
__device__ __forceinline__ float2 ff_add(float2 a, float2 b)
{
    const float s = a.x + b.x, z = s - a.x;
    const float e = ((a.x - (s - z)) + (b.x - z)) + (a.y + b.y);
    return ff_norm(s, e);
}
__device__ __forceinline__ float2 ff_mul(float2 a, float2 b)
{
    const float h = a.x * b.x;
    return ff_norm(h, __fmaf_rn(a.x, b.x, -h) + (a.x * b.y + a.y * b.x));
}
__device__ __forceinline__ float2 ff_of(double d)   // once per fit: FP64 conversions
{
    const float h = (float)d;
    return make_float2(h, (float)(d - (double)h));
}

// The entry's (sum_wv.re, sum_wv.im, sum_w) as float pairs (hi, lo).
struct EntryFF {
    float2 x, y, z;
};
__device__ __forceinline__ float2 add_ff(float2 a, float b)   // (a.x + a.y) + b as a pair
{
    const float t = a.x + b, z = t - a.x;
    const float err = (a.x - (t - z)) + (b - z);
    const float lo = a.y + err, hi = t + lo;
    return make_float2(hi, lo - (hi - t));
}
__device__ __forceinline__ EntryFF entry_ff(const void *cube, const double *master, int fp64, int64_t e)
{
    EntryFF r;
    if (fp64) {
        const double *c = reinterpret_cast<const double *>(cube) + 4 * e;
        r.x = split_double(c[0]);
        r.y = split_double(c[1]);
        r.z = split_double(c[2]);
        return r;
    }
    const float4 f = reinterpret_cast<const float4 *>(cube)[e];
    if (master) {
        const double2 m01 = *reinterpret_cast<const double2 *>(master + 4 * e);
        const double m2 = master[4 * e + 2];
        r.x = add_ff(split_double(m01.x), f.x);
        r.y = add_ff(split_double(m01.y), f.y);
        r.z = add_ff(split_double(m2), f.z);
    } else {
        r.x = make_float2(f.x, 0.f);
        r.y = make_float2(f.y, 0.f);
        r.z = make_float2(f.z, 0.f);
    }
    return r;
}

// x_j = (2 j - (nrest - 1)) / nrest as a float pair, from 1 / nrest as a
// float pair inv (the numerator is exact in FP32, |2 j - (nrest - 1)| < 2^24,
// and its product with inv.x exact by FMA).
__device__ __forceinline__ float2 absc_ff(int j, int nrest, float2 inv)
{
    const float a = (float)(2 * j - (nrest - 1));
    const float h = a * inv.x;
    return make_float2(h, __fmaf_rn(a, inv.x, -h) + a * inv.y);
}

// The moments of one plane's fit set as compensated float-pair sums, entry
// by entry: sum t x^n (n = 0 .. 2 ORDER) with t = sum_w, and sum v x^k
// (k = 0 .. ORDER) with v = sum_wv (re and im); t, v, x and every power as
// float pairs (products to about 2^-44).
template <int ORDER>
struct MomentsFF {
    static constexpr int NM = 2 * ORDER + 1, NB = ORDER + 1;
    float Ms[NM], Mc[NM], Brs[NB], Brc[NB], Bis[NB], Bic[NB];
    __device__ __forceinline__ void zero()
    {
#pragma unroll
        for (int k = 0; k < NM; ++k) Ms[k] = Mc[k] = 0.f;
#pragma unroll
        for (int k = 0; k < NB; ++k) Brs[k] = Brc[k] = Bis[k] = Bic[k] = 0.f;
    }
    __device__ __forceinline__ void add(const EntryFF &v, float2 x)
    {
        float th = v.z.x, tl = v.z.y;
#pragma unroll
        for (int k = 0; k < NM; ++k) {
            acc2(Ms[k], Mc[k], th);
            Mc[k] += tl;
            const float ph = th * x.x;
            tl = __fmaf_rn(th, x.x, -ph) + (th * x.y + tl * x.x);
            th = ph;
        }
        float rh = v.x.x, rl = v.x.y, ih = v.y.x, il = v.y.y;
#pragma unroll
        for (int k = 0; k < NB; ++k) {
            acc2(Brs[k], Brc[k], rh);
            Brc[k] += rl;
            acc2(Bis[k], Bic[k], ih);
            Bic[k] += il;
            const float pr = rh * x.x, pi = ih * x.x;
            rl = __fmaf_rn(rh, x.x, -pr) + (rh * x.y + rl * x.x);
            il = __fmaf_rn(ih, x.x, -pi) + (ih * x.y + il * x.x);
            rh = pr;
            ih = pi;
        }
    }
    __device__ __forceinline__ void to_double(double (&M)[NM], double (&Br)[NB], double (&Bi)[NB]) const
    {
#pragma unroll
        for (int k = 0; k < NM; ++k) M[k] = (double)Ms[k] + (double)Mc[k];
#pragma unroll
        for (int k = 0; k < NB; ++k) {
            Br[k] = (double)Brs[k] + (double)Brc[k];
            Bi[k] = (double)Bis[k] + (double)Bic[k];
        }
    }
};

// The same moments in FP64 from an entry's FP64 sums (the refit of an
// ill-conditioned plane).
template <int ORDER>
__device__ __forceinline__ void add_moments_fp64(const double3 &v, double x, double (&Md)[2 * ORDER + 1],
                                                 double (&Brd)[ORDER + 1], double (&Bid)[ORDER + 1])
{
    double t = v.z, xr = v.x, xi = v.y;
#pragma unroll
    for (int k = 0; k < 2 * ORDER + 1; ++k) {
        Md[k] += t;
        t *= x;
    }
#pragma unroll
    for (int k = 0; k < ORDER + 1; ++k) {
        Brd[k] += xr;
        Bid[k] += xi;
        xr *= x;
        xi *= x;
    }
}

// One output entry, sum_wv - sum_w p(x): p by Horner in float-pair
// arithmetic from its float-pair coefficients (a nearly interpolating fit
// has large coefficients whose terms cancel, so single floats would not do).
template <int NB>
__device__ __forceinline__ float2 subtract_fit(const EntryFF &v, float2 x, const float2 (&fr)[NB],
                                               const float2 (&fi)[NB])
{
    float2 pr = fr[NB - 1], pi = fi[NB - 1];
#pragma unroll
    for (int k = NB - 2; k >= 0; --k) {
        pr = ff_add(ff_mul(pr, x), fr[k]);
        pi = ff_add(ff_mul(pi, x), fi[k]);
    }
    const float2 neg_w = make_float2(-v.z.x, -v.z.y);
    const float2 orr = ff_add(v.x, ff_mul(neg_w, pr)), oi = ff_add(v.y, ff_mul(neg_w, pi));
    return make_float2(orr.x + orr.y, oi.x + oi.y);
}

// Warp per cell (npol divides 32): lane L handles entries L, L + 32, ... of
// the cell ([nrest][npol], so plane L mod npol); x_j = (2 j - (nrest - 1)) *
// (1 / nrest) with 1 / nrest as a float pair inv (exact products by FMA).
template <int ORDER>
__global__ void __launch_bounds__(256) k_contsub_cell(const void *cube, const double *master, int fp64,
                                                      const uint8_t *line_free, int64_t ncell, int nrest, int npol,
                                                      float2 inv, float2 *out)
{
    constexpr int NM = 2 * ORDER + 1;
    constexpr int NB = ORDER + 1;
    const int lane = threadIdx.x & 31;
    const int64_t cell = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (cell >= ncell) return;   // whole warps
    const int64_t e0 = cell * nrest * npol;
    const int nent = nrest * npol;
    MomentsFF<ORDER> mo;
    mo.zero();
    int nfit = 0;
    float xmin = 2.f, xmax = -2.f;
    for (int f = lane; f < nent; f += 32) {
        const int j = f / npol;
        if (!line_free[j]) continue;
        const EntryFF v = entry_ff(cube, master, fp64, e0 + f);
        if (!(v.z.x > 0.f)) continue;
        ++nfit;
        const float2 x = absc_ff(j, nrest, inv);
        xmin = fminf(xmin, x.x);
        xmax = fmaxf(xmax, x.x);
        mo.add(v, x);
    }
    // sums over the lanes of this lane's plane, in FP64
    double M[NM], Br[NB], Bi[NB];
    mo.to_double(M, Br, Bi);
    for (int o = 16; o >= npol; o >>= 1) {
        nfit += __shfl_xor_sync(0xffffffffu, nfit, o);
        xmin = fminf(xmin, __shfl_xor_sync(0xffffffffu, xmin, o));
        xmax = fmaxf(xmax, __shfl_xor_sync(0xffffffffu, xmax, o));
#pragma unroll
        for (int k = 0; k < NM; ++k) M[k] += __shfl_xor_sync(0xffffffffu, M[k], o);
#pragma unroll
        for (int k = 0; k < NB; ++k) {
            Br[k] += __shfl_xor_sync(0xffffffffu, Br[k], o);
            Bi[k] += __shfl_xor_sync(0xffffffffu, Bi[k], o);
        }
    }
    // A quadratic or cubic fit over few or clustered channels is too ill
    // conditioned (its normal matrix up to ~1e10) for the float-pair moments:
    // such a plane's moments are accumulated again in FP64 (few terms).
    const bool refine = ORDER >= 2 && nfit > 0 && (xmax - xmin < 0.5f || nfit < 4 * NB);
    if (__any_sync(0xffffffffu, refine)) {
        double Md[NM], Brd[NB], Bid[NB];
#pragma unroll
        for (int k = 0; k < NM; ++k) Md[k] = 0.0;
#pragma unroll
        for (int k = 0; k < NB; ++k) Brd[k] = Bid[k] = 0.0;
        const double inv_n = 1.0 / (double)nrest;
        for (int f = lane; refine && f < nent; f += 32) {
            const int j = f / npol;
            if (!line_free[j]) continue;
            const double3 v = entry_sums(cube, master, fp64, e0 + f);
            if (!(v.z > 0.0)) continue;
            add_moments_fp64<ORDER>(v, (double)(2 * j - (nrest - 1)) * inv_n, Md, Brd, Bid);
        }
        for (int o = 16; o >= npol; o >>= 1) {
#pragma unroll
            for (int k = 0; k < NM; ++k) Md[k] += __shfl_xor_sync(0xffffffffu, Md[k], o);
#pragma unroll
            for (int k = 0; k < NB; ++k) {
                Brd[k] += __shfl_xor_sync(0xffffffffu, Brd[k], o);
                Bid[k] += __shfl_xor_sync(0xffffffffu, Bid[k], o);
            }
        }
        if (refine) {
#pragma unroll
            for (int k = 0; k < NM; ++k) M[k] = Md[k];
#pragma unroll
            for (int k = 0; k < NB; ++k) {
                Br[k] = Brd[k];
                Bi[k] = Bid[k];
            }
        }
    }
    double cr[NB], ci[NB];
    solve_fit<ORDER>(M, Br, Bi, nfit, cr, ci);
    float2 fr[NB], fi[NB];   // the coefficients as float pairs
#pragma unroll
    for (int k = 0; k < NB; ++k) {
        fr[k] = ff_of(cr[k]);
        fi[k] = ff_of(ci[k]);
    }
    for (int f = lane; f < nent; f += 32) {
        const int j = f / npol;
        out[e0 + f] = subtract_fit<NB>(entry_ff(cube, master, fp64, e0 + f), absc_ff(j, nrest, inv), fr, fi);
    }
}

template <int ORDER>
__global__ void __launch_bounds__(256) k_contsub(const void *cube, const double *master, int fp64,
                                                 const uint8_t *line_free, int64_t ncell, int nrest, int npol,
                                                 float2 *out)
{
    constexpr int NM = 2 * ORDER + 1;   // moments sum w x^n, n = 0 .. 2 ORDER
    constexpr int NB = ORDER + 1;       // right-hand sides sum x^k wv
    const int lane = threadIdx.x & 31;
    const int64_t task = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (task >= ncell * npol) return;   // whole warps
    const int64_t cell = task / npol;
    const int pl = (int)(task % npol);
    const double inv_n = 1.0 / (double)nrest;
    auto entry = [&](int j) { return (cell * nrest + j) * npol + pl; };
    auto absc = [&](int j) { return (double)(2 * j - (nrest - 1)) * inv_n; };

    double M[NM], Br[NB], Bi[NB];
#pragma unroll
    for (int k = 0; k < NM; ++k) M[k] = 0.0;
#pragma unroll
    for (int k = 0; k < NB; ++k) Br[k] = Bi[k] = 0.0;
    int nfit = 0;
    for (int j = lane; j < nrest; j += 32) {
        if (!line_free[j]) continue;
        const double3 s = entry_sums(cube, master, fp64, entry(j));
        if (!(s.z > 0.0)) continue;
        ++nfit;
        const double x = absc(j);
        double t = s.z;
#pragma unroll
        for (int k = 0; k < NM; ++k) {
            M[k] += t;
            t *= x;
        }
        double xr = s.x, xi = s.y;
#pragma unroll
        for (int k = 0; k < NB; ++k) {
            Br[k] += xr;
            Bi[k] += xi;
            xr *= x;
            xi *= x;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nfit += __shfl_xor_sync(0xffffffffu, nfit, o);
#pragma unroll
    for (int k = 0; k < NM; ++k) M[k] = warp_sum(M[k]);
#pragma unroll
    for (int k = 0; k < NB; ++k) {
        Br[k] = warp_sum(Br[k]);
        Bi[k] = warp_sum(Bi[k]);
    }

    // coefficients of p (lowest power first); none when nothing is fitted
    double cr[NB], ci[NB];
    solve_fit<ORDER>(M, Br, Bi, nfit, cr, ci);

    for (int j = lane; j < nrest; j += 32) {
        const int64_t e = entry(j);
        const double3 s = entry_sums(cube, master, fp64, e);
        const double x = absc(j);
        double pr = 0.0, pi = 0.0;
#pragma unroll
        for (int k = NB - 1; k >= 0; --k) {
            pr = pr * x + cr[k];
            pi = pi * x + ci[k];
        }
        out[e] = make_float2((float)(s.x - s.z * pr), (float)(s.y - s.z * pi));
    }
}

cudaError_t launch_contsub(const vista_stack *h, const uint8_t *line_free, int order, float2 *out, cudaStream_t st)
{
    const int64_t ncell = (int64_t)h->desc.nu * h->desc.nv;
    const int fp64 = h->desc.precision == VISTA_PREC_FP64;
    const double *m = fp64 ? nullptr : h->cube_master;
    const int nrest = h->desc.nrest, npol = h->desc.npol;
    if (32 % npol == 0) {
        // a warp per cell; 1 / nrest as a float pair
        const double r = 1.0 / (double)nrest;
        const float2 inv = make_float2((float)r, (float)(r - (double)(float)r));
        const unsigned cb = (unsigned)((ncell * 32 + 255) / 256);
        switch (order) {
        case 0: k_contsub_cell<0><<<cb, 256, 0, st>>>(h->cube, m, fp64, line_free, ncell, nrest, npol, inv, out); break;
        case 1: k_contsub_cell<1><<<cb, 256, 0, st>>>(h->cube, m, fp64, line_free, ncell, nrest, npol, inv, out); break;
        case 2: k_contsub_cell<2><<<cb, 256, 0, st>>>(h->cube, m, fp64, line_free, ncell, nrest, npol, inv, out); break;
        case 3: k_contsub_cell<3><<<cb, 256, 0, st>>>(h->cube, m, fp64, line_free, ncell, nrest, npol, inv, out); break;
        default: return cudaErrorInvalidValue;
        }
        return cudaGetLastError();
    }
    const int64_t warps = ncell * h->desc.npol;
    const unsigned blocks = (unsigned)((warps * 32 + 255) / 256);
    switch (order) {
    case 0: k_contsub<0><<<blocks, 256, 0, st>>>(h->cube, m, fp64, line_free, ncell, h->desc.nrest, h->desc.npol, out); break;
    case 1: k_contsub<1><<<blocks, 256, 0, st>>>(h->cube, m, fp64, line_free, ncell, h->desc.nrest, h->desc.npol, out); break;
    case 2: k_contsub<2><<<blocks, 256, 0, st>>>(h->cube, m, fp64, line_free, ncell, h->desc.nrest, h->desc.npol, out); break;
    case 3: k_contsub<3><<<blocks, 256, 0, st>>>(h->cube, m, fp64, line_free, ncell, h->desc.nrest, h->desc.npol, out); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace

extern "C" int vista_contsub(vista_stack *h, const uint8_t *line_free, int32_t order, float *sum_wv_out,
                             int dst_is_device)
{
    if (!handle_live(h)) return fail(nullptr, VISTA_E_STATE, "unknown or closed handle");
    if (!line_free || !sum_wv_out) return fail(h, VISTA_E_ARG, "null line_free or output");
    if (order < 0 || order > MAX_ORDER) return fail(h, VISTA_E_ARG, "order must be 0..%d", MAX_ORDER);
    const int nrest = h->desc.nrest;
    const size_t n_out = (size_t)h->nentries * sizeof(float2);
    const size_t lf_bytes = ((size_t)nrest + 255) & ~(size_t)255;
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "stream synchronize");
    int32_t err = 0;
    e = cudaMemcpy(&err, h->err, sizeof err, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(h, e, "error word read");
    if (err != 0) return device_fail(h, err);
    // the mask (and, for a host destination, the output) in a handle buffer
    e = h->b_contsub.ensure(lf_bytes + (dst_is_device ? 0 : n_out));
    if (e != cudaSuccess) return cuda_fail(h, e, "continuum subtraction buffer");
    uint8_t *d_lf = (uint8_t *)h->b_contsub.p;
    float2 *d_out = dst_is_device ? reinterpret_cast<float2 *>(sum_wv_out)
                                  : reinterpret_cast<float2 *>((char *)h->b_contsub.p + lf_bytes);
    e = cudaMemcpyAsync(d_lf, line_free, (size_t)nrest, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = launch_contsub(h, d_lf, order, d_out, h->stream);
    if (e == cudaSuccess && !dst_is_device)
        e = cudaMemcpyAsync(sum_wv_out, d_out, n_out, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "continuum subtraction");
    return VISTA_OK;
}

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
// One warp per (cell, plane), lanes over the rest channels: a first pass
// accumulates the moments in FP64 and reduces them over the warp, every
// lane solves the (d+1) x (d+1) system by Cholesky in FP64, and a second
// pass writes the output.  Memory bound: the entry's sums are read twice
// (the second time mostly from L2) and the output written once.
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
#pragma unroll
    for (int k = 0; k < NB; ++k) cr[k] = ci[k] = 0.0;
    const int d = nfit < 1 ? -1 : (nfit - 1 < ORDER ? nfit - 1 : ORDER);
    if (d >= 0) {
        // Cholesky of A (positive definite: d + 1 <= nfit distinct abscissae,
        // positive weights), then the two triangular solves per part
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
    const int64_t warps = ncell * h->desc.npol;
    const unsigned blocks = (unsigned)((warps * 32 + 255) / 256);
    const int fp64 = h->desc.precision == VISTA_PREC_FP64;
    const double *m = fp64 ? nullptr : h->cube_master;
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

// libvista stacking kernels for sm_103a.
//
//   (the mixed-precision stacking kernel is in vista_stack.cu)
//   stack_fp64    the plain form: thread per (window, row), FP64 phasor
//                 recurrence, FP64 cells, FP64 atomics into an FP64 cube
//   debug_mixed   the mixed path's own phasor and cell code, exported
//   unpack        cube -> caller arrays
#include "vista_device.cuh"

namespace vista {

// Debug export: the same phasor and cell code as stack_mixed, writing the
// phasor and the cell of every (row, channel) of one window.
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
    const RowRec rec = a.recs[S.rec_off + i];
    const int2 cc = a.ccells[S.cell_off + (int64_t)chunk * nrow + i];
    const int64_t row = rec.row;
    const bool fold = signbit(rec.W[0]);
#pragma unroll
    for (int q = 0; q < NS; ++q) {
        const int kk = q * 32 + lane, k = c0 + kk;
        if (k < S.k_hi) {
            const ChanD *cd = a.chd + S.chan_off + (k - S.k_lo);
            const ChanF cf = a.chf[S.chan_off + (k - S.k_lo)];
            const float2 ph = shift_phasor(rec.tau_hi, rec.tau_lo, cf.nuc_hi, cf.nuc_lo);
            // same cell path as the stacking kernel
            int cid;
            if (cc.y == CC_NOCHANGE)
                cid = cc.x;
            else if (cc.y != CC_MIXED)
                cid = chunk_cell_step(cc, kk, a.g.nu);
            else
                cid = cell_exact(S.guvw, row, fold, cd, a.g.nu, a.g.nv);
            const int iu = cid < 0 ? -1 : cid % a.g.nu, iv = cid < 0 ? -1 : cid / a.g.nu;
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
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= a.nrows_total) return;
    const int s = find_owner(a.row_off, a.nsrc, gid);
    if (EXPORT && s != only_src) return;
    const SrcDev &S = a.srcs[s];
    const int64_t r = gid - a.row_off[s];
    const double *uvw = S.uvw + 3 * r;     // the stored baseline: the delay of Eq. 2
    const double tau = uvw[0] * S.l + uvw[1] * S.m + uvw[2] * S.n1;
    double u = S.guvw[3 * r], v = S.guvw[3 * r + 1];   // the gridding baseline (Eq. 1)
    const bool fold = a.g.fold && (v < 0.0 || (v == 0.0 && u < 0.0));
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
        const double t = tau * (cd[0].nu * (1.0 / C_LIGHT));
        ph = turns_to_phasor64(t - floor(t));
        const double d = tau * S.step_c;
        stp = turns_to_phasor64(d - floor(d));
    }
    double *cube = reinterpret_cast<double *>(a.cube);
    unsigned long long n_vis = 0, n_flag = 0, n_duv = 0, n_stk = 0;
    for (int k = S.k_lo; k < S.k_hi; ++k) {
        const ChanD c = cd[k - S.k_lo];
        if (!S.linear) {
            const double t = tau * (c.nu * (1.0 / C_LIGHT));
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
                const int64_t vi = (r * S.vstride + (k - S.kbase)) * npol;
                for (int p = 0; p < npol; ++p) {
                    const int q = S.plane[p];
                    if (q < 0) continue;
                    ++n_vis;
                    if (S.fbase && S.fbase[r * S.fpitch + (int64_t)(k - S.fk0) * npol + p]) {
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
                    const double sr = vr * ph.x - vim * ph.y;
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

__global__ void unpack_kernel(const void *cube, const double *master, const uint32_t *count, int fp64, int64_t n,
                              void *sum_wv, void *sum_w, void *sum_wvv, uint32_t *cnt_out, int out_f64)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double e[4];
        if (fp64) {
            const double *c = reinterpret_cast<const double *>(cube) + 4 * i;
            e[0] = c[0];
            e[1] = c[1];
            e[2] = c[2];
            e[3] = c[3];
        } else {
            // the float4 sums since the last checkpoint plus the FP64 master sums
            const float4 c = reinterpret_cast<const float4 *>(cube)[i];
            e[0] = c.x;
            e[1] = c.y;
            e[2] = c.z;
            e[3] = c.w;
            if (master) {
                const double *m = master + 4 * i;
                e[0] += m[0];
                e[1] += m[1];
                e[2] += m[2];
                e[3] += m[3];
            }
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

cudaError_t launch_fp64(const RunArgs &a, cudaStream_t st)
{
    if (a.nrows_total == 0) return cudaSuccess;
    const int64_t blocks = (a.nrows_total + 127) / 128;
    stack_fp64<false><<<(unsigned)blocks, 128, 0, st>>>(a, -1, nullptr, nullptr);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ fold

// Every nonzero FP32 entry of the mixed cube is added to its FP64 master
// entry and cleared (the exact widening of each component), so the FP32
// partials start again from zero.  Nothing else touches the cube meanwhile
// (the handle's stream orders it after the run's stacking).
__global__ void fold_kernel(float4 *cube, double *master, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float4 c = cube[i];
        if (c.x != 0.f || c.y != 0.f || c.z != 0.f || c.w != 0.f) {
            double *m = master + 4 * i;
            m[0] += (double)c.x;
            m[1] += (double)c.y;
            m[2] += (double)c.z;
            m[3] += (double)c.w;
            cube[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
}

cudaError_t launch_fold(void *cube, double *master, int64_t n, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    fold_kernel<<<(unsigned)blocks, 256, 0, st>>>(reinterpret_cast<float4 *>(cube), master, n);
    return cudaGetLastError();
}

cudaError_t launch_unpack(const void *cube, const double *master, const uint32_t *count, int fp64, int64_t n,
                          void *sum_wv, void *sum_w, void *sum_wvv, uint32_t *cnt_out, int out_f64, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    unpack_kernel<<<(unsigned)blocks, 256, 0, st>>>(cube, master, count, fp64, n, sum_wv, sum_w, sum_wvv, cnt_out,
                                                    out_f64);
    return cudaGetLastError();
}

cudaError_t launch_debug(const RunArgs &a, int ns, int src, int fp64, double *ph, int32_t *cells, cudaStream_t st)
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
    switch (ns) {
    case 1: debug_mixed<1><<<(unsigned)blocks, 128, 0, st>>>(a, src, ph, cells); break;
    case 2: debug_mixed<2><<<(unsigned)blocks, 128, 0, st>>>(a, src, ph, cells); break;
    case 4: debug_mixed<4><<<(unsigned)blocks, 128, 0, st>>>(a, src, ph, cells); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace vista

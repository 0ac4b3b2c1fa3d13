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

// Entry i's four sums (re and im of sum wV, sum w, sum w|V|^2) in FP64: the
// FP64 cube, or the mixed cube's float4 sums since the last checkpoint plus
// its FP64 master sums.
__device__ __forceinline__ void entry_value(const void *cube, const double *master, int fp64, int64_t i,
                                            double (&e)[4])
{
    if (fp64) {
        const double *c = reinterpret_cast<const double *>(cube) + 4 * i;
        e[0] = c[0];
        e[1] = c[1];
        e[2] = c[2];
        e[3] = c[3];
        return;
    }
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

__global__ void unpack_kernel(const void *cube, const double *master, const uint32_t *count, int fp64, int64_t n,
                              void *sum_wv, void *sum_w, void *sum_wvv, uint32_t *cnt_out, int out_f64)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double e[4];
        entry_value(cube, master, fp64, i, e);
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

// Sparse readback: the entries with count > 0, in entry order, in three
// passes over tiles of SPARSE_TILE consecutive entries (thread t of a block
// reads entries t, t + 256, ... of its tile, so every load is coalesced):
// the touched entries of each tile; one block's exclusive scan of the tile
// counts, with the total at the end; and each tile's touched entries
// written from its offset on, in entry order (a ballot per warp and a count
// per warp in shared memory per round of 256 entries).
constexpr int SPARSE_THREADS = 256, SPARSE_ROUNDS = 16, SPARSE_TILE = SPARSE_THREADS * SPARSE_ROUNDS;
constexpr int SPARSE_WARPS = SPARSE_THREADS / 32, SCAN_THREADS = 1024;
static_assert(SPARSE_TILE == 4096, "sparse_tiles() counts tiles of 4096 entries");

__global__ void __launch_bounds__(SPARSE_THREADS) sparse_count_kernel(const uint32_t *count, int64_t n,
                                                                      uint32_t *tile_cnt)
{
    __shared__ int ws[SPARSE_WARPS];
    const int64_t base = (int64_t)blockIdx.x * SPARSE_TILE;
    int c = 0;
    for (int k = 0; k < SPARSE_ROUNDS; ++k) {
        const int64_t i = base + (int64_t)k * SPARSE_THREADS + threadIdx.x;
        c += (i < n && count[i] != 0u) ? 1 : 0;
    }
    c = __reduce_add_sync(0xffffffffu, c);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < SPARSE_WARPS; ++w) t += ws[w];
        tile_cnt[blockIdx.x] = (uint32_t)t;
    }
}

// One block of SCAN_THREADS: thread t sums a contiguous run of tiles, the
// block scans those sums (warp shuffles, then the warps' totals), and each
// thread writes its tiles' offsets; the last thread writes the total.
__global__ void __launch_bounds__(SCAN_THREADS) sparse_scan_kernel(const uint32_t *tile_cnt, int64_t ntile,
                                                                   int64_t *tile_off, int64_t *total)
{
    __shared__ long long wtot[SCAN_THREADS / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t per = (ntile + SCAN_THREADS - 1) / SCAN_THREADS;
    const int64_t t0 = min((int64_t)threadIdx.x * per, ntile), t1 = min(t0 + per, ntile);
    long long s = 0;
    for (int64_t t = t0; t < t1; ++t) s += tile_cnt[t];
    long long x = s;   // inclusive scan over the warp
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wtot[wid] = x;
    __syncthreads();
    long long before = 0;
    for (int w = 0; w < wid; ++w) before += wtot[w];
    long long off = before + x - s;   // exclusive
    for (int64_t t = t0; t < t1; ++t) {
        tile_off[t] = off;
        off += tile_cnt[t];
    }
    if (threadIdx.x == SCAN_THREADS - 1) *total = before + x;
}

__global__ void __launch_bounds__(SPARSE_THREADS) sparse_write_kernel(const void *cube, const double *master,
                                                                      const uint32_t *count, int fp64, int64_t n,
                                                                      const int64_t *tile_off, int64_t cap,
                                                                      int64_t *idx_out, float *sum_wv, float *sum_w,
                                                                      float *sum_wvv, uint32_t *cnt_out)
{
    __shared__ int ws[SPARSE_WARPS];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t base = (int64_t)blockIdx.x * SPARSE_TILE;
    int64_t pos = tile_off[blockIdx.x];
    for (int k = 0; k < SPARSE_ROUNDS; ++k) {
        const int64_t i = base + (int64_t)k * SPARSE_THREADS + threadIdx.x;
        const uint32_t c = i < n ? count[i] : 0u;
        const unsigned bal = __ballot_sync(0xffffffffu, c != 0u);
        if (lane == 0) ws[wid] = __popc(bal);
        __syncthreads();
        int before = 0, all = 0;
        for (int w = 0; w < SPARSE_WARPS; ++w) {
            before += w < wid ? ws[w] : 0;
            all += ws[w];
        }
        if (c != 0u) {
            const int64_t q = pos + before + __popc(bal & ((1u << lane) - 1u));
            if (q < cap) {
                double e[4];
                entry_value(cube, master, fp64, i, e);
                idx_out[q] = i;
                if (sum_wv) {
                    sum_wv[2 * q] = (float)e[0];
                    sum_wv[2 * q + 1] = (float)e[1];
                }
                if (sum_w) sum_w[q] = (float)e[2];
                if (sum_wvv) sum_wvv[q] = (float)e[3];
                if (cnt_out) cnt_out[q] = c;
            }
        }
        pos += all;
        __syncthreads();   // ws is written again in the next round
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

cudaError_t launch_sparse_count(const uint32_t *count, int64_t n, uint32_t *tile_cnt, int64_t *tile_off,
                                int64_t *total, cudaStream_t st)
{
    const int64_t ntile = sparse_tiles(n);
    if (ntile == 0) return cudaMemsetAsync(total, 0, sizeof(int64_t), st);
    sparse_count_kernel<<<(unsigned)ntile, SPARSE_THREADS, 0, st>>>(count, n, tile_cnt);
    sparse_scan_kernel<<<1, SCAN_THREADS, 0, st>>>(tile_cnt, ntile, tile_off, total);
    return cudaGetLastError();
}

cudaError_t launch_sparse_write(const void *cube, const double *master, const uint32_t *count, int fp64, int64_t n,
                                const int64_t *tile_off, int64_t cap, int64_t *index, float *sum_wv, float *sum_w,
                                float *sum_wvv, uint32_t *cnt_out, cudaStream_t st)
{
    const int64_t ntile = sparse_tiles(n);
    if (ntile == 0 || cap == 0) return cudaSuccess;
    sparse_write_kernel<<<(unsigned)ntile, SPARSE_THREADS, 0, st>>>(cube, master, count, fp64, n, tile_off, cap, index,
                                                                   sum_wv, sum_w, sum_wvv, cnt_out);
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

// Row ordering, per-row FP64 records and the work list of the mixed path.
//
// Rows of each window are put in uv-cell order so that the stacking kernel's
// per-lane running sums absorb consecutive rows that share a cell, and the
// work list walks the cube stripe by stripe (a stripe = a few iv rows of the
// cube, sized to stay resident in L2) across all windows.
//
//   k_keys         cell of every row at the window's highest in-cube
//                  frequency -> (stripe, local cell key); per-bucket arrival
//                  slots with warp-aggregated atomics
//   k_scan         one block: per-window bucket offsets, and the work list in
//                  stripe-major order (item = rows of one bucket x one chunk)
//   k_scatter      rows grouped by bucket
//   k_bucket_sort  one block per bucket: counting sort by local cell key
//   k_records      FP64 delay, phase seeds and recurrence stride of every
//                  (row, chunk), written in processing order (paper Eq. 2 and
//                  the phasor recurrence of Sec. 3.2)
#include "vista_device.cuh"

namespace vista {

__global__ void __launch_bounds__(256) k_keys(RunArgs a)
{
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= a.nrows_total) return;
    const SortArgs &so = a.so;
    const int w = find_owner(a.row_off, a.nsrc, g);
    const SrcDev &S = a.srcs[w];
    const int64_t r = g - a.row_off[w];
    uint32_t stripe = 0, L = 0, slot;
    if (so.sorted) {
        if (S.k_hi > S.k_lo) {
            double u = S.uvw[3 * r], v = S.uvw[3 * r + 1];
            if (a.g.fold && (v < 0.0 || (v == 0.0 && u < 0.0))) {
                u = -u;
                v = -v;
            }
            float x = floorf((float)u * S.key_su) + (float)(a.g.nu >> 1);
            float y = floorf((float)v * S.key_sv) + (float)(a.g.nv >> 1);
            x = fminf(fmaxf(x, 0.0f), (float)(a.g.nu - 1));   // NaN -> 0
            y = fminf(fmaxf(y, 0.0f), (float)(a.g.nv - 1));
            const int iu = (int)x, iv = (int)y;
            stripe = (uint32_t)(iv / so.stripe_rows);
            L = (uint32_t)((iv % so.stripe_rows) * so.nuk + (iu >> so.ushift));
        }
        const uint32_t b = (uint32_t)w * so.nstripe + stripe;
        const unsigned act = __activemask();
        const unsigned peers = __match_any_sync(act, b);
        const int lane = threadIdx.x & 31;
        const int leader = __ffs(peers) - 1;
        const uint32_t rank = __popc(peers & ((1u << lane) - 1u));
        uint32_t base = 0;
        if (lane == leader) base = atomicAdd(&so.hist[b], (uint32_t)__popc(peers));
        base = __shfl_sync(peers, base, leader);
        slot = base + rank;
    } else {
        slot = (uint32_t)r;
        if (r == 0) so.hist[w] = (uint32_t)S.nrow;
    }
    so.slot[g] = slot;
    so.key[g] = (stripe << 13) | L;
}

// One block of 1024 threads.
__global__ void __launch_bounds__(1024) k_scan(RunArgs a)
{
    const SortArgs &so = a.so;
    const int nw = a.nsrc, ns = so.nstripe, R = so.rows_per_item;
    for (int w = threadIdx.x; w < nw; w += blockDim.x) {
        uint32_t acc = 0;
        for (int s = 0; s < ns; ++s) {
            so.qstart[(size_t)w * ns + s] = acc;
            acc += so.hist[(size_t)w * ns + s];
        }
    }
    __syncthreads();
    // work list in stripe-major order: bucket i = s * nw + w
    const int64_t nb = (int64_t)nw * ns;
    const int64_t per = (nb + blockDim.x - 1) / blockDim.x;
    const int64_t i0 = min(nb, (int64_t)threadIdx.x * per), i1 = min(nb, i0 + per);
    int64_t local = 0;
    for (int64_t i = i0; i < i1; ++i) {
        const int s = (int)(i / nw), w = (int)(i % nw);
        const int64_t n = so.hist[(size_t)w * ns + s];
        local += ((n + R - 1) / R) * a.srcs[w].nchunk;
    }
    __shared__ long long part[1024];
    part[threadIdx.x] = local;
    __syncthreads();
    for (int off = 1; off < (int)blockDim.x; off <<= 1) {
        long long v = threadIdx.x >= (unsigned)off ? part[threadIdx.x - off] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    int64_t pos = part[threadIdx.x] - local;
    const int64_t total = part[blockDim.x - 1];
    for (int64_t i = i0; i < i1; ++i) {
        const int s = (int)(i / nw), w = (int)(i % nw);
        const int64_t n = so.hist[(size_t)w * ns + s];
        const int64_t q = so.qstart[(size_t)w * ns + s];
        const int nch = a.srcs[w].nchunk;
        for (int64_t t = 0; t * R < n; ++t) {
            for (int c = 0; c < nch; ++c) {
                if (pos < so.max_items) {
                    Item it;
                    it.w = w;
                    it.chunk = c;
                    it.q0 = (int32_t)(q + t * R);
                    it.q1 = (int32_t)min(q + n, q + (t + 1) * R);
                    so.items[pos] = it;
                }
                ++pos;
            }
        }
    }
    if (threadIdx.x == 0) {
        if (total > so.max_items) atomicExch(a.err, 2);   // host sizing bug: never expected
        so.ctr[0] = (uint32_t)min(total, so.max_items);
        so.ctr[1] = 0u;
    }
}

__global__ void __launch_bounds__(256) k_scatter(RunArgs a)
{
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= a.nrows_total) return;
    const SortArgs &so = a.so;
    const int w = find_owner(a.row_off, a.nsrc, g);
    const uint32_t r = (uint32_t)(g - a.row_off[w]);
    const uint32_t key = so.key[g];
    const uint32_t s = key >> 13, L = key & 0x1fffu;
    const int64_t q = (int64_t)so.qstart[(size_t)w * so.nstripe + s] + so.slot[g];
    so.tmp[a.row_off[w] + q] = ((unsigned long long)L << 32) | r;
}

// One block per (window, stripe) bucket.
__global__ void __launch_bounds__(256) k_bucket_sort(RunArgs a)
{
    const SortArgs &so = a.so;
    const int64_t b = blockIdx.x;
    const int w = (int)(b / so.nstripe);
    const uint32_t n = so.hist[b];
    if (n == 0) return;
    const int64_t base = a.row_off[w] + so.qstart[b];
    if (!so.sorted || n == 1) {
        for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) so.perm[base + i] = (uint32_t)so.tmp[base + i];
        return;
    }
    __shared__ uint32_t sh[MAX_LOCAL_KEYS];
    __shared__ uint32_t start[MAX_LOCAL_KEYS];
    __shared__ uint32_t part[256];
    const int nk = so.stripe_rows * so.nuk;
    for (int i = threadIdx.x; i < nk; i += blockDim.x) sh[i] = 0;
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) atomicAdd(&sh[(uint32_t)(so.tmp[base + i] >> 32)], 1u);
    __syncthreads();
    // exclusive scan of sh[0, nk): contiguous slices per thread
    const int per = (nk + blockDim.x - 1) / blockDim.x;
    const int k0 = min(nk, (int)threadIdx.x * per), k1 = min(nk, k0 + per);
    uint32_t loc = 0;
    for (int k = k0; k < k1; ++k) loc += sh[k];
    part[threadIdx.x] = loc;
    __syncthreads();
    for (int off = 1; off < (int)blockDim.x; off <<= 1) {
        uint32_t v = threadIdx.x >= (unsigned)off ? part[threadIdx.x - off] : 0u;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    uint32_t run = part[threadIdx.x] - loc;
    for (int k = k0; k < k1; ++k) {
        const uint32_t c = sh[k];
        sh[k] = run;
        start[k] = run;
        run += c;
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
        const unsigned long long t = so.tmp[base + i];
        const uint32_t pos = atomicAdd(&sh[(uint32_t)(t >> 32)], 1u);
        so.perm[base + pos] = (uint32_t)t;
    }
    __syncthreads();
    // Rows that share a cell key arrive in arbitrary (atomic) order; order
    // each such group by row index.  Rows of one baseline are then
    // consecutive in time, so at the other channels of the window the cell
    // changes at most once inside the group instead of alternating.
    // A warp per group: rank of each row = rows of the group with a smaller
    // index (indices are distinct), written to tmp, then copied back.
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int k = warp; k < nk; k += nwarps) {
        const uint32_t s0 = start[k], cnt = sh[k] - s0;
        if (cnt < 2) continue;
        const uint32_t *g = so.perm + base + s0;
        for (uint32_t i = lane; i < cnt; i += 32) {
            const uint32_t ri = g[i];
            uint32_t rank = 0;
            for (uint32_t j = 0; j < cnt; ++j) rank += g[j] < ri;
            so.tmp[base + s0 + rank] = ri;
        }
    }
    __syncthreads();
    for (int k = warp; k < nk; k += nwarps) {
        const uint32_t s0 = start[k], cnt = sh[k] - s0;
        if (cnt < 2) continue;
        for (uint32_t i = lane; i < cnt; i += 32) so.perm[base + s0 + i] = (uint32_t)so.tmp[base + s0 + i];
    }
}

__global__ void __launch_bounds__(256) k_records(RunArgs a)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.nrows_total) return;
    const int w = find_owner(a.row_off, a.nsrc, p);
    const SrcDev &S = a.srcs[w];
    const int64_t q = p - a.row_off[w];
    const int64_t r = a.so.perm[p];
    const double *uvw = S.uvw + 3 * r;
    const double u = uvw[0], v = uvw[1], wz = uvw[2];
    const bool fold = a.g.fold && (v < 0.0 || (v == 0.0 && u < 0.0));
    const double tau = u * S.l + v * S.m + wz * S.n1;
    RowRec rec;
    split_ff(tau, rec.tau_hi, rec.tau_lo);
    rec.u = (float)(fold ? -u : u);
    rec.v = (float)(fold ? -v : v);
    rec.rowf = (uint32_t)r | (fold ? 0x80000000u : 0u);
#pragma unroll
    for (int k = 0; k < 4; ++k) rec.W[k] = k < S.npol ? S.wts[r * S.npol + k] : 0.0f;
    // The cell index is monotone in frequency along a row, so equal cells at a
    // chunk's two end channels hold for every channel between them.
    const ChanD *cd = a.chd + S.chan_off;
    const ChanF *cf = a.chf + S.chan_off;
    const int nin = S.k_hi - S.k_lo;
#pragma unroll
    for (int c = 0; c < REC_CELLS; ++c) {
        int info = CELL_MIXED;
        if (c < S.nchunk) {
            const int e0 = c * a.cw, e1 = min(nin, (c + 1) * a.cw) - 1;
            const float fu0 = axis_floor(rec.u, cf[e0].su, uvw, fold, &cd[e0].su);
            const float fu1 = axis_floor(rec.u, cf[e1].su, uvw, fold, &cd[e1].su);
            const float fv0 = axis_floor(rec.v, cf[e0].sv, uvw + 1, fold, &cd[e0].sv);
            const float fv1 = axis_floor(rec.v, cf[e1].sv, uvw + 1, fold, &cd[e1].sv);
            if (fu0 == fu1 && fv0 == fv1) {
                const float hu = (float)(a.g.nu >> 1), hv = (float)(a.g.nv >> 1);
                const bool in = fu0 >= -hu && fu0 < hu && fv0 >= -hv && fv0 < hv;
                info = in ? ((int)fv0 + (a.g.nv >> 1)) * a.g.nu + ((int)fu0 + (a.g.nu >> 1)) : -1;
            }
        }
        rec.cell[c] = info;
    }
    a.recs[S.rec_off + q] = rec;
}

cudaError_t launch_prepare(const RunArgs &a, cudaStream_t st)
{
    const SortArgs &so = a.so;
    cudaError_t e = cudaMemsetAsync(so.hist, 0, sizeof(uint32_t) * (size_t)a.nsrc * so.nstripe, st);
    if (e != cudaSuccess) return e;
    const unsigned rb = (unsigned)((a.nrows_total + 255) / 256);
    if (rb) k_keys<<<rb, 256, 0, st>>>(a);
    k_scan<<<1, 1024, 0, st>>>(a);
    if (rb) k_scatter<<<rb, 256, 0, st>>>(a);
    const int64_t nbuckets = (int64_t)a.nsrc * so.nstripe;
    if (rb && nbuckets) k_bucket_sort<<<(unsigned)nbuckets, 256, 0, st>>>(a);
    if (rb) k_records<<<rb, 256, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace vista

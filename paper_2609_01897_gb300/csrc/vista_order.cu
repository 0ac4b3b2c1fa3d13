// Row ordering, per-row FP64 records and the work list of the mixed path.
//
// Rows of each window are put in uv-cell order so that the stacking kernel's
// per-lane running sums absorb consecutive rows that share a cell, and the
// work list walks the cube stripe by stripe (a stripe = a few iv rows of the
// cube, sized to stay resident in L2) across all windows.
//
//   k_keys         cell of every row at the window's highest in-cube
//                  frequency -> (stripe, local cell key); stripe counts per
//                  segment of rows
//   k_segscan      segment offsets inside each (window, stripe) bucket
//   k_slots        each row's slot in its bucket, in row order
//   k_scan         one block: per-window bucket offsets, per-bucket work-list
//                  offsets in stripe-major order (item = rows of one bucket x
//                  one chunk)
//   k_items        the work list, one thread per item
//   k_scatter      rows grouped by bucket
//   k_bucket_sort  one block per bucket: stable counting sort by local cell
//                  key (the rows of one key stay in row order)
//   k_records      per row, in processing order: the FP64 delay of Eq. 2 as
//                  a float-float pair and the (fold-signed) weights
//   k_cells        per (row, channel chunk): the chunk's uv cells
#include "vista_device.cuh"

namespace vista {

// Row-order slots in (window, stripe) buckets, three passes over segments of
// SEG_ROWS rows: keys and per-segment stripe counts, an exclusive scan of the
// counts over each window's segments, then each segment's slots in row order
// (ranks within a warp from a match, warps in turn against running counts in
// shared memory).  Rows that share a bucket thus keep their row order.
constexpr uint32_t NO_BUCKET = 0xffffffffu;

struct SegRange {
    int w;
    int64_t g0, r0, r1;   // first global row of the window, rows [r0, r1) of the segment
};
__device__ __forceinline__ SegRange seg_range(const RunArgs &a, int64_t seg)
{
    SegRange sr;
    sr.w = find_owner(a.so.seg_off, a.nsrc, seg);
    sr.g0 = a.row_off[sr.w];
    sr.r0 = (seg - a.so.seg_off[sr.w]) * SEG_ROWS;
    const int64_t n = a.srcs[sr.w].nrow;
    sr.r1 = sr.r0 + SEG_ROWS < n ? sr.r0 + SEG_ROWS : n;
    return sr;
}

// Pass 1: the cell of every row at the window's highest in-cube frequency ->
// (stripe, local cell key), and the stripe counts of the segment.
__global__ void __launch_bounds__(256) k_keys(RunArgs a)
{
    __shared__ uint32_t cnt[MAX_STRIPES];
    const SortArgs &so = a.so;
    const int64_t seg = blockIdx.x;
    const SegRange sr = seg_range(a, seg);
    const SrcDev &S = a.srcs[sr.w];
    if (!so.sorted) {
        for (int64_t r = sr.r0 + threadIdx.x; r < sr.r1; r += blockDim.x) {
            so.slot[sr.g0 + r] = (uint32_t)r;
            so.key[sr.g0 + r] = 0u;
        }
        if (threadIdx.x == 0 && sr.r0 == 0) so.hist[sr.w] = (uint32_t)S.nrow;
        return;
    }
    for (int k = threadIdx.x; k < so.nstripe; k += blockDim.x) cnt[k] = 0u;
    __syncthreads();
    for (int64_t r = sr.r0 + threadIdx.x; r < sr.r1; r += blockDim.x) {
        uint32_t stripe = 0, L = 0;
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
        so.key[sr.g0 + r] = (stripe << 13) | L;
        atomicAdd(&cnt[stripe], 1u);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < so.nstripe; k += blockDim.x) so.segcnt[seg * so.nstripe + k] = cnt[k];
}

// Pass 2: one thread per (window, stripe): the segments' first slots and the
// bucket's row count.
__global__ void __launch_bounds__(256) k_segscan(RunArgs a)
{
    const SortArgs &so = a.so;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (!so.sorted || t >= (int64_t)a.nsrc * so.nstripe) return;
    const int w = (int)(t / so.nstripe), k = (int)(t % so.nstripe);
    uint32_t run = 0;
    for (int64_t seg = so.seg_off[w]; seg < so.seg_off[w + 1]; ++seg) {
        uint32_t *c = so.segcnt + seg * so.nstripe + k;
        const uint32_t n = *c;
        *c = run;
        run += n;
    }
    so.hist[t] = run;
}

// Pass 3: each segment's slots in row order.
__global__ void __launch_bounds__(256) k_slots(RunArgs a)
{
    __shared__ uint32_t run[MAX_STRIPES];
    const SortArgs &so = a.so;
    if (!so.sorted) return;
    const int64_t seg = blockIdx.x;
    const SegRange sr = seg_range(a, seg);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int k = threadIdx.x; k < so.nstripe; k += blockDim.x) run[k] = so.segcnt[seg * so.nstripe + k];
    __syncthreads();
    for (int64_t c = sr.r0; c < sr.r1; c += blockDim.x) {
        const int64_t r = c + threadIdx.x;
        const uint32_t stripe = r < sr.r1 ? so.key[sr.g0 + r] >> 13 : NO_BUCKET;
        const unsigned peers = __match_any_sync(0xffffffffu, stripe);
        const int leader = __ffs(peers) - 1;
        const uint32_t rank = __popc(peers & ((1u << lane) - 1u));
        uint32_t slot = 0;
        for (int wi = 0; wi < nwarps; ++wi) {
            if (warp == wi) {
                uint32_t base = 0;
                if (lane == leader && stripe != NO_BUCKET) {
                    base = run[stripe];
                    run[stripe] = base + (uint32_t)__popc(peers);
                }
                slot = __shfl_sync(peers, base, leader) + rank;
            }
            __syncthreads();
        }
        if (r < sr.r1) so.slot[sr.g0 + r] = slot;
    }
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
        so.ioff[i] = pos;
        const int s = (int)(i / nw), w = (int)(i % nw);
        const int64_t n = so.hist[(size_t)w * ns + s];
        pos += ((n + R - 1) / R) * a.srcs[w].nchunk;
    }
    if (threadIdx.x == 0) so.ioff[nb] = total;
    if (threadIdx.x == 0) {
        if (total > so.max_items) atomicExch(a.err, 2);   // host sizing bug: never expected
        so.ctr[0] = (uint32_t)min(total, so.max_items);
        so.ctr[1] = 0u;
    }
}

// One thread per work item: bucket i (stripe-major) holds items
// [ioff[i], ioff[i+1]), rows in groups of rows_per_item, each group split
// into the window's channel chunks.
__global__ void __launch_bounds__(256) k_items(RunArgs a)
{
    const SortArgs &so = a.so;
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nb = (int64_t)a.nsrc * so.nstripe;
    if (p >= so.ioff[nb] || p >= so.max_items) return;
    const int i = find_owner(so.ioff, (int)nb, p);
    const int nw = a.nsrc, R = so.rows_per_item;
    const int st = i / nw, w = i % nw;
    const SrcDev &S = a.srcs[w];
    const int64_t local = p - so.ioff[i];
    const int c = (int)(local % S.nchunk);
    const int64_t t = local / S.nchunk;
    const int64_t n = so.hist[(size_t)w * so.nstripe + st];
    const int64_t q = so.qstart[(size_t)w * so.nstripe + st];
    const int nin = S.k_hi - S.k_lo;
    Item it;
    it.w = w;
    it.chunk = c;
    it.q0 = (int32_t)(q + t * R);
    it.q1 = (int32_t)min(q + n, q + (t + 1) * R);
    it.chf0 = S.chan_off + c * a.cw;
    it.nch = min(a.cw, nin - c * a.cw);
    it.rec0 = S.rec_off + it.q0;
    it.cell0 = S.cell_off + (int64_t)c * S.nrow + it.q0;
    it.pad = 0;
    so.items[p] = it;
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
        run += c;
    }
    __syncthreads();
    // Stable scatter: the bucket's rows arrive in row order (k_keys), and
    // keep it within each local key, so that rows of one baseline stay
    // consecutive in time and, at the window's other channels, a group's
    // cell changes at most once instead of alternating.
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (uint32_t c0 = 0; c0 < n; c0 += blockDim.x) {
        const uint32_t i = c0 + threadIdx.x;
        const bool valid = i < n;
        const unsigned long long t = valid ? so.tmp[base + i] : 0ull;
        const uint32_t L = valid ? (uint32_t)(t >> 32) : NO_BUCKET;
        const unsigned peers = __match_any_sync(0xffffffffu, L);
        const int leader = __ffs(peers) - 1;
        const uint32_t rank = __popc(peers & ((1u << lane) - 1u));
        uint32_t pos = 0;
        for (int wi = 0; wi < nwarps; ++wi) {
            if (warp == wi) {
                uint32_t b0 = 0;
                if (lane == leader && valid) {
                    b0 = sh[L];
                    sh[L] = b0 + (uint32_t)__popc(peers);
                }
                pos = __shfl_sync(peers, b0, leader) + rank;
            }
            __syncthreads();
        }
        if (valid) so.perm[base + pos] = (uint32_t)t;
    }
}

// First chunk-local channel in (lo, hi] whose floor(coord * s) differs from
// f_lo (the cell is monotone in frequency; hi is known to differ).
__device__ int axis_step(float c32, const ChanF *cf, const ChanD *cd, int e0, int lo, int hi, const double *coord64,
                         bool neg, bool v_axis, float f_lo)
{
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        const float f = v_axis ? axis_floor(c32, cf[e0 + mid].sv, coord64, neg, &cd[e0 + mid].sv)
                               : axis_floor(c32, cf[e0 + mid].su, coord64, neg, &cd[e0 + mid].su);
        if (f == f_lo)
            lo = mid;
        else
            hi = mid;
    }
    return hi;
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
    rec.row = (uint32_t)r;
    rec.pad = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float wk = k < S.npol ? S.wts[r * S.npol + k] : 0.0f;
        rec.W[k] = fold ? -wk : wk;
    }
    a.recs[S.rec_off + q] = rec;
}

// Chunk cells: one thread per (row, channel chunk) entry, laid out [chunk][row]
// per window (rows in processing order).  The cell index is monotone in
// frequency along each axis, so the cells at a chunk's two end channels
// bound every channel between.
__global__ void __launch_bounds__(256) k_cells(RunArgs a)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.ncells_total) return;
    const int w = find_owner(a.cell_cum, a.nsrc, p);
    const SrcDev &S = a.srcs[w];
    const int64_t loc = p - a.cell_cum[w];
    const int c = (int)(loc / S.nrow);
    const int64_t q = loc - (int64_t)c * S.nrow;
    const int64_t r = a.so.perm[a.row_off[w] + q];
    const double *uvw = S.uvw + 3 * r;
    const double u = uvw[0], v = uvw[1];
    const bool fold = a.g.fold && (v < 0.0 || (v == 0.0 && u < 0.0));
    const float uf = (float)(fold ? -u : u), vf = (float)(fold ? -v : v);
    const ChanD *cd = a.chd + S.chan_off;
    const ChanF *cf = a.chf + S.chan_off;
    const int nin = S.k_hi - S.k_lo;
    const float hu = (float)(a.g.nu >> 1), hv = (float)(a.g.nv >> 1);
    const int e0 = c * a.cw, last = min(nin, e0 + a.cw) - 1 - e0;
    const float fu0 = axis_floor(uf, cf[e0].su, uvw, fold, &cd[e0].su);
    const float fu1 = axis_floor(uf, cf[e0 + last].su, uvw, fold, &cd[e0 + last].su);
    const float fv0 = axis_floor(vf, cf[e0].sv, uvw + 1, fold, &cd[e0].sv);
    const float fv1 = axis_floor(vf, cf[e0 + last].sv, uvw + 1, fold, &cd[e0 + last].sv);
    // both ends off the grid on the same side of one axis: off throughout
    const bool offu = (fu0 < -hu && fu1 < -hu) || (fu0 >= hu && fu1 >= hu);
    const bool offv = (fv0 < -hv && fv1 < -hv) || (fv0 >= hv && fv1 >= hv);
    const bool in = fu0 >= -hu && fu0 < hu && fu1 >= -hu && fu1 < hu && fv0 >= -hv && fv0 < hv &&
                    fv1 >= -hv && fv1 < hv;
    int2 cc;
    if (offu || offv) {
        cc = make_int2(-1, CC_NOCHANGE);
    } else if (!in || fabsf(fu1 - fu0) > 1.0f || fabsf(fv1 - fv0) > 1.0f) {
        cc = make_int2(-1, CC_MIXED);
    } else {
        uint32_t m = CC_NOCHANGE;
        if (fu1 != fu0) {
            const int b = axis_step(uf, cf, cd, e0, 0, last, uvw, fold, false, fu0);
            m = (m & ~0xffu) | (uint32_t)b | (fu1 < fu0 ? 0x10000u : 0u);
        }
        if (fv1 != fv0) {
            const int b = axis_step(vf, cf, cd, e0, 0, last, uvw + 1, fold, true, fv0);
            m = (m & ~0xff00u) | ((uint32_t)b << 8) | (fv1 < fv0 ? 0x20000u : 0u);
        }
        cc = make_int2(((int)fv0 + (a.g.nv >> 1)) * a.g.nu + ((int)fu0 + (a.g.nu >> 1)), (int)m);
    }
    a.ccells[S.cell_off + loc] = cc;
}

cudaError_t launch_prepare(const RunArgs &a, cudaStream_t st)
{
    const SortArgs &so = a.so;
    cudaError_t e = cudaMemsetAsync(so.hist, 0, sizeof(uint32_t) * (size_t)a.nsrc * so.nstripe, st);
    if (e != cudaSuccess) return e;
    const unsigned rb = (unsigned)((a.nrows_total + 255) / 256);
    if (so.nseg_total > 0) {
        k_keys<<<(unsigned)so.nseg_total, 256, 0, st>>>(a);
        const int64_t nb = (int64_t)a.nsrc * so.nstripe;
        k_segscan<<<(unsigned)((nb + 255) / 256), 256, 0, st>>>(a);
        k_slots<<<(unsigned)so.nseg_total, 256, 0, st>>>(a);
    }
    k_scan<<<1, 1024, 0, st>>>(a);
    if (so.max_items > 0) k_items<<<(unsigned)((so.max_items + 255) / 256), 256, 0, st>>>(a);
    if (rb) k_scatter<<<rb, 256, 0, st>>>(a);
    const int64_t nbuckets = (int64_t)a.nsrc * so.nstripe;
    if (rb && nbuckets) k_bucket_sort<<<(unsigned)nbuckets, 256, 0, st>>>(a);
    if (rb) k_records<<<rb, 256, 0, st>>>(a);
    if (a.ncells_total > 0) k_cells<<<(unsigned)((a.ncells_total + 255) / 256), 256, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace vista

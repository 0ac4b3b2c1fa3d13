// Row ordering, per-row FP64 records and the work list of the mixed path.
//
// Rows of each window are put in uv-cell order so that the stacking kernel's
// per-lane running sums absorb consecutive rows that share a cell, and the
// work list walks the cube stripe by stripe (a stripe = a few iv rows of the
// cube, sized to stay resident in L2) across all windows.
//
//   k_keys         cell of every row at the window's highest in-cube
//                  frequency -> (stripe, local cell key); stripe counts per
//                  segment of rows; a re-projected window's gridding
//                  baselines R (u, v, w) (Eq. 1)
//   k_segscan      segment offsets inside each (window, stripe) bucket (a
//                  warp scan per bucket)
//   k_slots        each row's slot in its bucket, in row order
//   k_scan         one block: per-window bucket offsets, per-bucket work-list
//                  offsets in stripe-major order (item = rows of one bucket x
//                  one chunk)
//   k_items        the work list, one thread per item
//   k_scatter      rows grouped by bucket
//   k_bucket_sort  one block per bucket: stable counting sort by local cell
//                  key (the rows of one key stay in row order), one
//                  contiguous part of the bucket per warp
//   k_rows         per row, in processing order: the FP64 delay of Eq. 2 as
//                  a float-float pair, the (fold-signed) weights, and the
//                  uv cells of each of the window's channel chunks
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
    // a re-projected window's gridding baselines are written here (Eq. 1)
    const double *R = S.rot1 ? a.rot + 9 * (int64_t)(S.rot1 - 1) : nullptr;
    double *G = R ? const_cast<double *>(S.guvw) : nullptr;
    if (!so.sorted) {
        for (int64_t r = sr.r0 + threadIdx.x; r < sr.r1; r += blockDim.x) {
            so.slot[sr.g0 + r] = (uint32_t)r;
            so.key[sr.g0 + r] = 0u;
            if (G) rotate_row(R, S.uvw + 3 * r, G + 3 * r);
        }
        if (threadIdx.x == 0 && sr.r0 == 0) so.hist[sr.w] = (uint32_t)S.nrow;
        return;
    }
    for (int k = threadIdx.x; k < so.nstripe; k += blockDim.x) cnt[k] = 0u;
    __syncthreads();
    for (int64_t r = sr.r0 + threadIdx.x; r < sr.r1; r += blockDim.x) {
        uint32_t stripe = 0, L = 0;
        if (S.k_hi > S.k_lo) {
            double u, v;
            if (G) {
                const double2 g = rotate_row(R, S.uvw + 3 * r, G + 3 * r);
                u = g.x;
                v = g.y;
            } else {
                u = S.uvw[3 * r];
                v = S.uvw[3 * r + 1];
            }
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

// Pass 2: one warp per (window, stripe): the segments' first slots (an
// exclusive scan of the counts over the window's segments, 32 at a time)
// and the bucket's row count.
__global__ void __launch_bounds__(256) k_segscan(RunArgs a)
{
    const SortArgs &so = a.so;
    const int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (!so.sorted || t >= (int64_t)a.nsrc * so.nstripe) return;   // whole warps
    const int w = (int)(t / so.nstripe), k = (int)(t % so.nstripe);
    const int64_t s1 = so.seg_off[w + 1];
    uint32_t run = 0;
    for (int64_t s0 = so.seg_off[w]; s0 < s1; s0 += 32) {
        const int64_t seg = s0 + lane;
        uint32_t *c = so.segcnt + seg * so.nstripe + k;
        const uint32_t n = seg < s1 ? *c : 0u;
        uint32_t incl = n;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (seg < s1) *c = run + incl - n;
        run += __shfl_sync(0xffffffffu, incl, 31);
    }
    if (lane == 0) so.hist[t] = run;
}

// Pass 3: each segment's slots in row order.  Warp w of W takes the
// contiguous w-th part of the segment, counts its stripes into its own
// shared-memory row, the counts become offsets (the segment's first slots
// plus the earlier warps' counts), and the warp assigns its rows in order.
// Dynamic shared memory: W x nstripe words.
__global__ void __launch_bounds__(256) k_slots(RunArgs a)
{
    extern __shared__ uint32_t dsm[];
    const SortArgs &so = a.so;
    if (!so.sorted) return;
    const int64_t seg = blockIdx.x;
    const SegRange sr = seg_range(a, seg);
    const int ns = so.nstripe;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    uint32_t *cnt = dsm + (size_t)warp * ns;
    for (int i = threadIdx.x; i < nwarps * ns; i += blockDim.x) dsm[i] = 0u;
    __syncthreads();
    const int64_t nr = sr.r1 - sr.r0;
    const int64_t p0 = sr.r0 + nr * warp / nwarps, p1 = sr.r0 + nr * (warp + 1) / nwarps;
    for (int64_t c = p0; c < p1; c += 32) {
        const int64_t r = c + lane;
        const uint32_t stripe = r < p1 ? so.key[sr.g0 + r] >> 13 : NO_BUCKET;
        const unsigned peers = __match_any_sync(0xffffffffu, stripe);
        if (stripe != NO_BUCKET && lane == __ffs(peers) - 1) cnt[stripe] += (uint32_t)__popc(peers);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < ns; k += blockDim.x) {
        uint32_t run = so.segcnt[seg * ns + k];
        for (int v = 0; v < nwarps; ++v) {
            const uint32_t c = dsm[(size_t)v * ns + k];
            dsm[(size_t)v * ns + k] = run;
            run += c;
        }
    }
    __syncthreads();
    for (int64_t c = p0; c < p1; c += 32) {
        const int64_t r = c + lane;
        const uint32_t stripe = r < p1 ? so.key[sr.g0 + r] >> 13 : NO_BUCKET;
        const unsigned peers = __match_any_sync(0xffffffffu, stripe);
        const int leader = __ffs(peers) - 1;
        uint32_t b0 = 0;
        if (stripe != NO_BUCKET && lane == leader) {
            b0 = cnt[stripe];
            cnt[stripe] = b0 + (uint32_t)__popc(peers);
        }
        const uint32_t slot = __shfl_sync(0xffffffffu, b0, leader) + (uint32_t)__popc(peers & ((1u << lane) - 1u));
        if (r < p1) so.slot[sr.g0 + r] = slot;
    }
}

// Warps per block for a per-warp table of nk words in shared memory
// (tables + extra tables of nk words kept within 96 KB).
static int table_warps(int nk, int extra)
{
    int nw = (int)(96 * 1024 / (4 * (int64_t)(nk > 0 ? nk : 1))) - extra;
    return nw < 1 ? 1 : (nw > 8 ? 8 : nw);
}

// Launch a kernel that takes dynamic shared memory above the 48 KB default.
template <typename K>
static cudaError_t allow_smem(K kern, size_t smem)
{
    if (smem <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
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

// One block per (window, stripe) bucket: a stable counting sort of the
// bucket's rows by local cell key.  The rows arrive in row order (k_slots)
// and keep it within each key, so that rows of one baseline stay
// consecutive in time and, at the window's other channels, a group's cell
// changes at most once instead of alternating.  Warp w of W takes the
// contiguous w-th part of the bucket: it counts its keys into its own
// shared-memory row (no block barrier per 32 rows), the counts become
// offsets (key-major, then warp), and the warp scatters its part in order.
// Dynamic shared memory: (W + 1) x nk words.
__global__ void __launch_bounds__(256) k_bucket_sort(RunArgs a)
{
    extern __shared__ uint32_t dsm[];
    __shared__ uint32_t part[256];
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
    const int nk = so.stripe_rows * so.nuk;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    uint32_t *cnt = dsm + (size_t)warp * nk;        // this warp's counts, then its offsets
    uint32_t *tot = dsm + (size_t)nwarps * nk;      // per key: all warps' counts, then the key's start
    for (int i = threadIdx.x; i < (nwarps + 1) * nk; i += blockDim.x) dsm[i] = 0u;
    __syncthreads();
    const uint32_t r0 = (uint32_t)((uint64_t)n * warp / nwarps), r1 = (uint32_t)((uint64_t)n * (warp + 1) / nwarps);
    for (uint32_t c0 = r0; c0 < r1; c0 += 32) {
        const uint32_t i = c0 + lane;
        const uint32_t L = i < r1 ? (uint32_t)(so.tmp[base + i] >> 32) : NO_BUCKET;
        const unsigned peers = __match_any_sync(0xffffffffu, L);
        if (L != NO_BUCKET && lane == __ffs(peers) - 1) cnt[L] += (uint32_t)__popc(peers);
    }
    __syncthreads();
    // per key: exclusive prefix over the warps, and the key's total
    for (int k = threadIdx.x; k < nk; k += blockDim.x) {
        uint32_t run = 0;
        for (int v = 0; v < nwarps; ++v) {
            const uint32_t c = dsm[(size_t)v * nk + k];
            dsm[(size_t)v * nk + k] = run;
            run += c;
        }
        tot[k] = run;
    }
    __syncthreads();
    // exclusive scan of the totals over the keys: contiguous slices per thread
    const int per = (nk + blockDim.x - 1) / blockDim.x;
    const int k0 = min(nk, (int)threadIdx.x * per), k1 = min(nk, k0 + per);
    uint32_t loc = 0;
    for (int k = k0; k < k1; ++k) loc += tot[k];
    part[threadIdx.x] = loc;
    __syncthreads();
    for (int off = 1; off < (int)blockDim.x; off <<= 1) {
        const uint32_t v = threadIdx.x >= (unsigned)off ? part[threadIdx.x - off] : 0u;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    uint32_t run = part[threadIdx.x] - loc;
    for (int k = k0; k < k1; ++k) {
        const uint32_t c = tot[k];
        tot[k] = run;
        run += c;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < nk; k += blockDim.x) {
        const uint32_t st = tot[k];
        for (int v = 0; v < nwarps; ++v) dsm[(size_t)v * nk + k] += st;
    }
    __syncthreads();
    // each warp scatters its part in row order
    for (uint32_t c0 = r0; c0 < r1; c0 += 32) {
        const uint32_t i = c0 + lane;
        const bool valid = i < r1;
        const unsigned long long t = valid ? so.tmp[base + i] : 0ull;
        const uint32_t L = valid ? (uint32_t)(t >> 32) : NO_BUCKET;
        const unsigned peers = __match_any_sync(0xffffffffu, L);
        const int leader = __ffs(peers) - 1;
        uint32_t b0 = 0;
        if (valid && lane == leader) {
            b0 = cnt[L];
            cnt[L] = b0 + (uint32_t)__popc(peers);
        }
        const uint32_t pos = __shfl_sync(0xffffffffu, b0, leader) + (uint32_t)__popc(peers & ((1u << lane) - 1u));
        if (valid) so.perm[base + pos] = (uint32_t)t;
    }
}

// The cell scales (su, sv) of channel k of a window's table (read-only).
__device__ __forceinline__ float2 chan_scales(const ChanF *cf, int k)
{
    return __ldg(reinterpret_cast<const float2 *>(cf + k));
}

// The scales of a chunk's first and last channel: all a chunk's entry needs
// unless its cell changes inside it.
struct ChunkEnds {
    float2 s0, s1;
};
__device__ __forceinline__ ChunkEnds chunk_ends(const RunArgs &a, const ChanF *cf, int nin, int c)
{
    const int e0 = c * a.cw, last = min(nin, e0 + a.cw) - 1 - e0;
    return ChunkEnds{chan_scales(cf, e0), chan_scales(cf, e0 + last)};
}

// First chunk-local channel in (lo, hi] whose floor(coord * s) differs from
// f_lo; f_hi = the floor at hi (different), x_lo, x_hi = fl32(coord * s) at
// lo and hi.  The cell is monotone in frequency.  The scales are close to
// linear in the channel index across a chunk, so the crossing is first
// estimated by linear interpolation and the floors at the estimate and the
// channel before it are evaluated (two loads issued together); they either
// settle the answer or narrow the bisection that follows, so the result is
// the exact first differing channel whatever the estimate.
__device__ int axis_step(float c32, const ChanF *cf, const ChanD *cd, int e0, int lo, int hi, const double *coord64,
                         bool neg, bool v_axis, float f_lo, float f_hi, float x_lo, float x_hi)
{
    auto f_at = [&](int k) {
        const float2 sc = chan_scales(cf, e0 + k);
        return axis_floor(c32, v_axis ? sc.y : sc.x, coord64, neg, v_axis ? &cd[e0 + k].sv : &cd[e0 + k].su);
    };
    if (hi - lo > 1) {
        const float B = f_hi > f_lo ? f_lo + 1.0f : f_lo;   // the value coord * s crosses
        const float dx = x_hi - x_lo, span = (float)(hi - lo);
        int k = (lo + hi + 1) >> 1;
        if (dx != 0.0f) {
            const float t = (B - x_lo) / dx * span;
            if (t > 0.0f && t < span) k = lo + (int)ceilf(t);   // a NaN fails both tests
        }
        k = min(max(k, lo + 1), hi);
        const float fk = f_at(k), fm = f_at(k - 1);   // k - 1 >= lo, where the floor is f_lo
        if (fk == f_lo)
            lo = k;
        else if (fm == f_lo)
            return k;
        else
            hi = k - 1;
    }
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (f_at(mid) == f_lo)
            lo = mid;
        else
            hi = mid;
    }
    return hi;
}

// The chunk-cell entry of chunk c of one row (coordinates uf, vf after the
// fold; uvw the row's FP64 coordinates for the exact fall-backs; ce the
// scales at the chunk's two end channels).  The cell index is monotone in
// frequency along each axis, so the cells at a chunk's two end channels
// bound every channel between.
__device__ int2 chunk_cell(const RunArgs &a, const SrcDev &S, const ChanF *cf, const ChanD *cd, int c, float uf,
                           float vf, const double *uvw, bool fold, const ChunkEnds &ce)
{
    const int nin = S.k_hi - S.k_lo;
    const float hu = (float)(a.g.nu >> 1), hv = (float)(a.g.nv >> 1);
    const int e0 = c * a.cw, last = min(nin, e0 + a.cw) - 1 - e0;
    const float fu0 = axis_floor(uf, ce.s0.x, uvw, fold, &cd[e0].su);
    const float fu1 = axis_floor(uf, ce.s1.x, uvw, fold, &cd[e0 + last].su);
    const float fv0 = axis_floor(vf, ce.s0.y, uvw + 1, fold, &cd[e0].sv);
    const float fv1 = axis_floor(vf, ce.s1.y, uvw + 1, fold, &cd[e0 + last].sv);
    // both ends off the grid on the same side of one axis: off throughout
    const bool offu = (fu0 < -hu && fu1 < -hu) || (fu0 >= hu && fu1 >= hu);
    const bool offv = (fv0 < -hv && fv1 < -hv) || (fv0 >= hv && fv1 >= hv);
    const bool in = fu0 >= -hu && fu0 < hu && fu1 >= -hu && fu1 < hu && fv0 >= -hv && fv0 < hv &&
                    fv1 >= -hv && fv1 < hv;
    if (offu || offv) return make_int2(-1, CC_NOCHANGE);
    if (!in || fabsf(fu1 - fu0) > 1.0f || fabsf(fv1 - fv0) > 1.0f) return make_int2(-1, CC_MIXED);
    uint32_t m = CC_NOCHANGE;
    if (fu1 != fu0) {
        const int b = axis_step(uf, cf, cd, e0, 0, last, uvw, fold, false, fu0, fu1, __fmul_rn(uf, ce.s0.x),
                                __fmul_rn(uf, ce.s1.x));
        m = (m & ~0xffu) | (uint32_t)b | (fu1 < fu0 ? 0x10000u : 0u);
    }
    if (fv1 != fv0) {
        const int b = axis_step(vf, cf, cd, e0, 0, last, uvw + 1, fold, true, fv0, fv1, __fmul_rn(vf, ce.s0.y),
                                __fmul_rn(vf, ce.s1.y));
        m = (m & ~0xff00u) | ((uint32_t)b << 8) | (fv1 < fv0 ? 0x20000u : 0u);
    }
    return make_int2(((int)fv0 + (a.g.nv >> 1)) * a.g.nu + ((int)fu0 + (a.g.nu >> 1)), (int)m);
}

// One thread per row, in processing order: the row record (the FP64 delay
// of Eq. 2 as a float-float pair, the fold-signed weights, the row index)
// and the chunk-cell entries of all the window's chunks, laid out
// [chunk][row] per window so that an item's entries are contiguous.  The
// row's coordinates are read once for both.  The window's channel table is
// read from L2 (the tables of the windows a block's rows span do not stay
// in L1), so the end scales of chunk c + 1 are loaded before chunk c's entry
// is formed: one load latency per chunk overlaps the previous chunk's work.
__global__ void __launch_bounds__(256) k_rows(RunArgs a)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.nrows_total) return;
    const int w = find_owner(a.row_off, a.nsrc, p);
    const SrcDev &S = a.srcs[w];
    const int64_t q = p - a.row_off[w];
    const int64_t r = a.so.perm[p];
    const double *uvw = S.uvw + 3 * r;     // the stored baseline: the delay of Eq. 2
    const double *guvw = S.guvw + 3 * r;   // the gridding baseline (rotated for a re-projected window)
    const double tau = uvw[0] * S.l + uvw[1] * S.m + uvw[2] * S.n1;
    const double u = guvw[0], v = guvw[1];
    const bool fold = a.g.fold && (v < 0.0 || (v == 0.0 && u < 0.0));
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

    const float uf = (float)(fold ? -u : u), vf = (float)(fold ? -v : v);
    const ChanD *cd = a.chd + S.chan_off;
    const ChanF *cf = a.chf + S.chan_off;
    int2 *out = a.ccells + S.cell_off + q;
    const int nchunk = S.nchunk, nin = S.k_hi - S.k_lo;
    if (nchunk <= 0) return;
    ChunkEnds nx = chunk_ends(a, cf, nin, 0);
    for (int c = 0; c < nchunk; ++c) {
        const ChunkEnds ce = nx;
        if (c + 1 < nchunk) nx = chunk_ends(a, cf, nin, c + 1);
        out[(int64_t)c * S.nrow] = chunk_cell(a, S, cf, cd, c, uf, vf, guvw, fold, ce);
    }
}

// Re-projected windows (Eq. 1): their gridding baselines R (u, v, w) (see
// rotate_row), one thread per row.  The mixed path forms them in k_keys,
// which reads every row anyway; this kernel serves the plain FP64 form.
__global__ void __launch_bounds__(256) k_rotate(RunArgs a)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.nrows_total) return;
    const int w = find_owner(a.row_off, a.nsrc, p);
    const SrcDev &S = a.srcs[w];
    if (!S.rot1) return;
    const int64_t r = p - a.row_off[w];
    rotate_row(a.rot + 9 * (int64_t)(S.rot1 - 1), S.uvw + 3 * r, const_cast<double *>(S.guvw) + 3 * r);
}

cudaError_t launch_rotate(const RunArgs &a, cudaStream_t st)
{
    if (!a.rot || a.nrows_total == 0) return cudaSuccess;
    k_rotate<<<(unsigned)((a.nrows_total + 255) / 256), 256, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_prepare(const RunArgs &a, cudaStream_t st, int *nlaunch)
{
    const SortArgs &so = a.so;
    int n = 0;
    cudaError_t e = cudaMemsetAsync(so.hist, 0, sizeof(uint32_t) * (size_t)a.nsrc * so.nstripe, st);
    if (e != cudaSuccess) return e;
    const unsigned rb = (unsigned)((a.nrows_total + 255) / 256);
    if (so.nseg_total > 0) {
        k_keys<<<(unsigned)so.nseg_total, 256, 0, st>>>(a);
        const int64_t nb = (int64_t)a.nsrc * so.nstripe;
        k_segscan<<<(unsigned)((nb * 32 + 255) / 256), 256, 0, st>>>(a);
        const int nws = table_warps(so.nstripe, 0);
        const size_t smem_s = (size_t)nws * so.nstripe * sizeof(uint32_t);
        const cudaError_t ea = allow_smem(k_slots, smem_s);
        if (ea != cudaSuccess) return ea;
        k_slots<<<(unsigned)so.nseg_total, 32 * nws, smem_s, st>>>(a);
        n += 3;
    }
    k_scan<<<1, 1024, 0, st>>>(a);
    ++n;
    if (so.max_items > 0) {
        k_items<<<(unsigned)((so.max_items + 255) / 256), 256, 0, st>>>(a);
        ++n;
    }
    if (rb) {
        k_scatter<<<rb, 256, 0, st>>>(a);
        ++n;
    }
    const int64_t nbuckets = (int64_t)a.nsrc * so.nstripe;
    if (rb && nbuckets) {
        const int nk = so.stripe_rows * so.nuk, nw = table_warps(nk, 1);
        const size_t smem = (size_t)(nw + 1) * nk * sizeof(uint32_t);
        const cudaError_t ea = allow_smem(k_bucket_sort, smem);
        if (ea != cudaSuccess) return ea;
        k_bucket_sort<<<(unsigned)nbuckets, 32 * nw, smem, st>>>(a);
        ++n;
    }
    if (rb) {
        k_rows<<<rb, 256, 0, st>>>(a);
        ++n;
    }
    if (nlaunch) *nlaunch = n;
    return cudaGetLastError();
}

}  // namespace vista

// The mixed-precision stacking kernel (sm_103a).
//
// Persistent: every warp pops work items (one window, up to rows_per_item
// rows in uv-cell order, a chunk of 32 x NS channels, lane = channel) from a
// queue in stripe-major order.  Per warp, the FP64 row records of the next
// item are fetched into shared memory by a TMA bulk copy (completing on an
// mbarrier) while the current item is processed; inside an item the
// visibility and flag loads run D rows ahead of the arithmetic.
//
// Per (row, channel): FP32 phasor from the record's FP64-reduced seed and
// the lane recurrence (Sec. 3.2), guarded-FP32 uv cell that is bit-exact
// against the FP64 cell rule, rest bins and Eq. 4 weights from the FP64
// channel table.  Per lane, running sums over consecutive rows that share a
// uv cell stay in registers and are flushed as one float4 reduction per
// (cell, rest bin, pol) and one count reduction (one u64 for a pol pair).
#include "vista_device.cuh"

namespace vista {

constexpr int RB_MAX = 256;   // largest item (rows) the shared-memory buffers hold

template <int P, int VT, int NS, int D>
__global__ void __launch_bounds__(256) stack_mixed(RunArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const int RB = a.so.rows_per_item;
    RowRec *rbuf = reinterpret_cast<RowRec *>(smem) + (size_t)wid * 2 * RB;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + (size_t)nwarp * 2 * RB * sizeof(RowRec)) + 2 * wid;
    if (lane == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        mbar_init_fence();
    }
    __syncwarp();

    const uint32_t nitems = a.so.ctr[0];
    const int npol_c = a.g.npol, nrest = a.g.nrest;
    float4 *cube4 = reinterpret_cast<float4 *>(a.cube);
    uint32_t n_vis = 0, n_flag = 0, n_duv = 0, n_stk = 0, n_red = 0;
    uint32_t phase = 0;   // bit s: parity of the next completion of slot s

    auto pop = [&]() -> uint32_t {
        uint32_t it = 0;
        if (lane == 0) it = atomicAdd(&a.so.ctr[1], 1u);
        return __shfl_sync(0xffffffffu, it, 0);
    };
    // Fetch the records of item `it` into slot s (lane 0 issues the copy).
    auto issue = [&](int s, uint32_t it) -> Item {
        const Item item = a.so.items[it];
        const SrcDev &S = a.srcs[item.w];
        if (lane == 0) {
            const RowRec *src = a.recs + S.rec_off + (int64_t)item.chunk * S.nrow + item.q0;
            const uint32_t bytes = (uint32_t)(item.q1 - item.q0) * (uint32_t)sizeof(RowRec);
            fence_proxy_async();
            mbar_expect_tx(&bars[s], bytes);
            tma_load_1d(rbuf + (size_t)s * RB, src, bytes, &bars[s]);
        }
        return item;
    };

    uint32_t it_next = pop();
    Item nxt{};
    if (it_next < nitems) nxt = issue(0, it_next);
    int s = 0;
    while (it_next < nitems) {
        const Item item = nxt;
        const int cs = s;
        __syncwarp();
        it_next = pop();
        if (it_next < nitems) nxt = issue(cs ^ 1, it_next);
        if (!mbar_wait_bounded(&bars[cs], (phase >> cs) & 1u, a.err)) {
            // give the other slot's copy a bounded chance to land, then stop
            if (it_next < nitems) mbar_wait_bounded(&bars[cs ^ 1], (phase >> (cs ^ 1)) & 1u, a.err);
            break;
        }
        phase ^= 1u << cs;
        const RowRec *rb = rbuf + (size_t)cs * RB;

        // ---- process one item ----
        const SrcDev &S = a.srcs[item.w];
        const int c0 = S.k_lo + item.chunk * 32 * NS;
        const bool linear = S.linear != 0;
        const void *vis = S.vis;
        const uint8_t *flags = S.flags;
        const float vscale = S.vis_scale;
        const int64_t vstride = S.vstride, kbase = S.kbase;
        int plane[P];
#pragma unroll
        for (int p = 0; p < P; ++p) plane[p] = S.plane[p];
        const bool pack2 = (P == 2) && plane[0] >= 0 && plane[1] == plane[0] + 1 && !(plane[0] & 1) &&
                           !(npol_c & 1);

        // per channel slot: fl32(s_k), first bin | bin count << 28, first two weights
        // (a third or fourth bin, possible only for user lattices narrower than
        // a channel, reads its weight from the table)
        float su[NS], sv[NS], wb[NS][2];
        int jn[NS];
#pragma unroll
        for (int q = 0; q < NS; ++q) {
            const int k = c0 + q * 32 + lane;
            jn[q] = 0;
            su[q] = sv[q] = 0.f;
            wb[q][0] = wb[q][1] = 0.f;
            if (k < S.k_hi) {
                const ChanF cf = a.chf[S.chan_off + (k - S.k_lo)];
                su[q] = cf.su;
                sv[q] = cf.sv;
                jn[q] = cf.j0 | (cf.nb << 28);
                wb[q][0] = cf.w[0];
                wb[q][1] = cf.w[1];
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
        auto flush = [&](int q) {
            if (cell[q] < 0) return;
            const int nbq = jn[q] >> 28;
            const size_t base = ((size_t)cell[q] * nrest + (jn[q] & 0x0fffffff)) * npol_c;
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                if (b < nbq) {
                    const float ww =
                        b < 2 ? wb[q][b] : a.chf[S.chan_off + (c0 + q * 32 + lane - S.k_lo)].w[b];
                    const size_t e = base + (size_t)b * npol_c;
#pragma unroll
                    for (int p = 0; p < P; ++p) {
                        if (cnt[q][p] == 0) continue;
                        atomicAdd(cube4 + e + plane[p], make_float4(ww * acc[q][p].x, ww * acc[q][p].y,
                                                                    ww * acc[q][p].z, ww * acc[q][p].w));
                        ++n_red;
                        if (!pack2) {
                            atomicAdd(a.count + e + plane[p], cnt[q][p]);
                            ++n_red;
                        }
                    }
                    if (pack2 && (cnt[q][0] | cnt[q][P - 1])) {
                        atomicAdd(reinterpret_cast<unsigned long long *>(a.count + e + plane[0]),
                                  (unsigned long long)cnt[q][0] | ((unsigned long long)cnt[q][P - 1] << 32));
                        ++n_red;
                    }
                }
            }
#pragma unroll
            for (int p = 0; p < P; ++p) {
                acc[q][p] = make_float4(0.f, 0.f, 0.f, 0.f);
                cnt[q][p] = 0;
            }
        };

        // visibility / flag ring, D rows ahead
        const int n = item.q1 - item.q0;
        float2 RV[D][NS][P];
        uint32_t RF[D][NS];
        auto fetch = [&](int d, int i) {
            const int64_t row = (int64_t)(rb[i].rowf & 0x7fffffffu);
#pragma unroll
            for (int q = 0; q < NS; ++q) {
                RF[d][q] = 0;
                if (jn[q] >> 28) {
                    const int64_t vidx = row * vstride + (c0 + q * 32 + lane - kbase);
                    VisLoad<P, VT>::load(vis, vidx, vscale, RV[d][q]);
                    RF[d][q] = load_flags<P>(flags, vidx);
                }
            }
        };
#pragma unroll
        for (int d = 0; d < D; ++d)
            if (d < n) fetch(d, d);

        for (int i0 = 0; i0 < n; i0 += D) {
#pragma unroll
            for (int d = 0; d < D; ++d) {
                const int i = i0 + d;
                if (i >= n) break;
                float2 V[NS][P];
                uint32_t F[NS];
#pragma unroll
                for (int q = 0; q < NS; ++q) {
                    F[q] = RF[d][q];
#pragma unroll
                    for (int p = 0; p < P; ++p) V[q][p] = RV[d][q][p];
                }
                if (i + D < n) fetch(d, i + D);

                const RowRec &rec = rb[i];
                const uint32_t rowf = rec.rowf;
                const int64_t row = (int64_t)(rowf & 0x7fffffffu);
                const bool fold = (rowf >> 31) != 0;
                const float ru = rec.u, rv = rec.v;
                float2 ph = make_float2(1.f, 0.f);
                double tau = 0.0;
                if (linear)
                    ph = lane_seed(rec, lane);
                else
                    tau = __hiloint2double(__float_as_int(rec.dhi), __float_as_int(rec.dlo));
                const float2 stp = make_float2(rec.sre, rec.sim);
                float W[P];
#pragma unroll
                for (int p = 0; p < P; ++p) W[p] = rec.W[p];
#pragma unroll
                for (int q = 0; q < NS; ++q) {
                    const int k = c0 + q * 32 + lane;
                    if (!linear && k < S.k_hi) {
                        double t = tau * (a.chd[S.chan_off + (k - S.k_lo)].nu * (1.0 / C_LIGHT));
                        t -= floor(t);
                        ph = turns_to_phasor((float)t);
                    }
                    if (jn[q] >> 28) {
                        const ChanD *cd = a.chd + S.chan_off + (k - S.k_lo);
                        const int iu = axis_cell(ru, su[q], S.uvw + 3 * row, fold, &cd->su, a.g.nu);
                        const int iv = axis_cell(rv, sv[q], S.uvw + 3 * row + 1, fold, &cd->sv, a.g.nv);
                        const int cid = (iu >= 0 && iv >= 0) ? iv * a.g.nu + iu : -1;
                        if (cid != cell[q]) {
                            flush(q);
                            cell[q] = cid;
                        }
#pragma unroll
                        for (int p = 0; p < P; ++p) {
                            if (plane[p] < 0) continue;
                            const bool f = ((F[q] >> (8 * p)) & 0xffu) != 0;
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
                            float2 vs = cmul(V[q][p], ph);
                            if (fold) vs.y = -vs.y;
                            const float a2 = V[q][p].x * V[q][p].x + V[q][p].y * V[q][p].y;
                            acc[q][p].x += W[p] * vs.x;
                            acc[q][p].y += W[p] * vs.y;
                            acc[q][p].z += W[p];
                            acc[q][p].w += W[p] * a2;
                            cnt[q][p] += 1;
                        }
                    }
                    if (linear) ph = cmul(ph, stp);
                }
            }
        }
#pragma unroll
        for (int q = 0; q < NS; ++q) flush(q);
        s ^= 1;
    }

    // counters: warp sum, one atomic per counter per warp
    unsigned long long c5[5] = {n_vis, n_flag, n_duv, n_stk, n_red};
#pragma unroll
    for (int k = 0; k < 5; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c5[k] += __shfl_xor_sync(0xffffffffu, c5[k], o);
    if (lane == 0) {
        if (c5[0]) atomicAdd(&a.stats->n_vis, c5[0]);
        if (c5[1]) atomicAdd(&a.stats->n_flagged, c5[1]);
        if (c5[2]) atomicAdd(&a.stats->n_dropped_uv, c5[2]);
        if (c5[3]) atomicAdd(&a.stats->n_stacked, c5[3]);
        if (c5[4]) atomicAdd(&a.stats->n_reductions, c5[4]);
    }
}

// --------------------------------------------------------------- launchers

static int sm_count()
{
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

template <typename K>
static cudaError_t launch_persistent(K kern, const RunArgs &a, int wpc, cudaStream_t st)
{
    const int rb = a.so.rows_per_item;
    if (rb < 1 || rb > RB_MAX) return cudaErrorInvalidValue;
    const size_t smem = (size_t)wpc * (2 * (size_t)rb * sizeof(RowRec) + 2 * sizeof(uint64_t));
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, wpc * 32, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    kern<<<per_sm * sm_count(), wpc * 32, smem, st>>>(a);
    return cudaGetLastError();
}

template <int P, int VT>
static cudaError_t launch_mixed_p(const RunArgs &a, int ns, int wpc, cudaStream_t st)
{
    switch (ns) {
    // prefetch depth D: as many rows ahead as the register budget allows
    case 1: return launch_persistent(stack_mixed<P, VT, 1, (P <= 2 ? 4 : 2)>, a, wpc, st);
    case 2: return launch_persistent(stack_mixed<P, VT, 2, (P <= 2 ? 2 : 1)>, a, wpc, st);
    case 4: return launch_persistent(stack_mixed<P, VT, 4, 1>, a, wpc, st);
    default: return cudaErrorInvalidValue;
    }
}

template <int VT>
static cudaError_t launch_mixed_vt(const RunArgs &a, int ns, int npol, int wpc, cudaStream_t st)
{
    switch (npol) {
    case 1: return launch_mixed_p<1, VT>(a, ns, wpc, st);
    case 2: return launch_mixed_p<2, VT>(a, ns, wpc, st);
    case 4: return launch_mixed_p<4, VT>(a, ns, wpc, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_mixed(const RunArgs &a, int key, int wpc, cudaStream_t st)
{
    const int npol = key & 0xff, ns = (key >> 8) & 0xff, vt = key >> 16;
    switch (vt) {
    case VISTA_VIS_C64: return launch_mixed_vt<VISTA_VIS_C64>(a, ns, npol, wpc, st);
    case VISTA_VIS_C128: return launch_mixed_vt<VISTA_VIS_C128>(a, ns, npol, wpc, st);
    case VISTA_VIS_F16X2: return launch_mixed_vt<VISTA_VIS_F16X2>(a, ns, npol, wpc, st);
    case VISTA_VIS_BF16X2: return launch_mixed_vt<VISTA_VIS_BF16X2>(a, ns, npol, wpc, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace vista

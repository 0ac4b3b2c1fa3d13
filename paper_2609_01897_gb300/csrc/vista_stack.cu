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

// Running sums of one channel slot for one uv cell, written to the cube.
// Out of line: after row ordering it runs once per several rows, and keeping
// it out of the unrolled row loop keeps the loop small.
// Everything one flush needs, passed by value: taking the address of the
// live running sums would move them out of registers for the whole loop.
template <int P>
struct FlushArgs {
    float4 acc[P];
    uint32_t cnt[P];
    int plane[P];
    int cell, jn;
    float w0, w1;
    const float *wtab;
    bool pack2;
};

template <int P>
static __device__ __noinline__ uint32_t flush_slot(const RunArgs &a, const FlushArgs<P> f)
{
    const float4 *acc = f.acc;
    const uint32_t *cnt = f.cnt;
    const int *plane = f.plane;
    const int cell = f.cell, jn = f.jn;
    const float w0 = f.w0, w1 = f.w1;
    const float *wtab = f.wtab;
    const bool pack2 = f.pack2;
    const int npol_c = a.g.npol;
    const int nbq = jn >> 28;
    float4 *cube4 = reinterpret_cast<float4 *>(a.cube);
    const size_t base = ((size_t)cell * a.g.nrest + (jn & 0x0fffffff)) * npol_c;
    uint32_t nred = 0;
    for (int b = 0; b < nbq; ++b) {
        const float ww = b == 0 ? w0 : b == 1 ? w1 : wtab[b];
        const size_t e = base + (size_t)b * npol_c;
        for (int p = 0; p < P; ++p) {
            if (cnt[p] == 0) continue;
            atomicAdd(cube4 + e + plane[p], make_float4(ww * acc[p].x, ww * acc[p].y, ww * acc[p].z, ww * acc[p].w));
            ++nred;
            if (!pack2) {
                atomicAdd(a.count + e + plane[p], cnt[p]);
                ++nred;
            }
        }
        if (pack2 && (cnt[0] | cnt[P - 1])) {
            atomicAdd(reinterpret_cast<unsigned long long *>(a.count + e + plane[0]),
                      (unsigned long long)cnt[0] | ((unsigned long long)cnt[P - 1] << 32));
            ++nred;
        }
    }
    return nred;
}

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
    uint32_t n_flag = 0, n_duv = 0, n_red = 0;
    uint32_t phase = 0;   // bit s: parity of the next completion of slot s

    auto pop = [&]() -> uint32_t {
        uint32_t it = 0;
        if (lane == 0) it = atomicAdd(&a.so.ctr[1], 1u);
        return __shfl_sync(0xffffffffu, it, 0);
    };
    // Fetch the records of item `it` into slot s (lane 0 issues the copy).
    auto issue = [&](int s, uint32_t it) -> Item {
        const Item item = a.so.items[it];
        if (lane == 0) {
            const SrcDev &S = a.srcs[item.w];
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

        // ---- one item ----
        // window fields in registers (the cube reductions below could alias
        // global memory, so references into the table would be re-read)
        struct WinRegs {
            const void *vis;
            const uint8_t *flags;
            const double *uvw;
            int64_t vstride, kbase;
            float vis_scale;
            int32_t k_lo, k_hi, chan_off, linear;
        } S;
        {
            const SrcDev &G = a.srcs[item.w];
            S.vis = G.vis;
            S.flags = G.flags;
            S.uvw = G.uvw;
            S.vstride = G.vstride;
            S.kbase = G.kbase;
            S.vis_scale = G.vis_scale;
            S.k_lo = G.k_lo;
            S.k_hi = G.k_hi;
            S.chan_off = G.chan_off;
            S.linear = G.linear;
        }
        const int c0 = S.k_lo + item.chunk * 32 * NS;
        const bool linear = S.linear != 0;
        int plane[P];
#pragma unroll
        for (int p = 0; p < P; ++p) plane[p] = a.srcs[item.w].plane[p];
        const bool pack2 = (P == 2) && plane[0] >= 0 && plane[1] == plane[0] + 1 && !(plane[0] & 1) &&
                           !(a.g.npol & 1);

        // per channel slot: fl32(s_k), first bin | bin count << 28, first two weights
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
            uint32_t any = 0;
#pragma unroll
            for (int p = 0; p < P; ++p) any |= cnt[q][p];
            if (cell[q] >= 0 && any) {
                FlushArgs<P> fa;
#pragma unroll
                for (int p = 0; p < P; ++p) {
                    fa.acc[p] = acc[q][p];
                    fa.cnt[p] = cnt[q][p];
                    fa.plane[p] = plane[p];
                }
                fa.cell = cell[q];
                fa.jn = jn[q];
                fa.w0 = wb[q][0];
                fa.w1 = wb[q][1];
                fa.wtab = a.chf[S.chan_off + (c0 + q * 32 + lane - S.k_lo)].w;
                fa.pack2 = pack2;
                n_red += flush_slot<P>(a, fa);
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
                    const int64_t vidx = row * S.vstride + (c0 + q * 32 + lane - S.kbase);
                    VisLoad<P, VT>::load(S.vis, vidx, S.vis_scale, RV[d][q]);
                    RF[d][q] = load_flags<P>(S.flags, vidx);
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
                float2 ph = make_float2(1.f, 0.f);
                if (linear) ph = lane_seed(rec, lane);
#pragma unroll
                for (int q = 0; q < NS; ++q) {
                    const int k = c0 + q * 32 + lane;
                    if (!linear && k < S.k_hi) {
                        const double tau = __hiloint2double(__float_as_int(rec.dhi), __float_as_int(rec.dlo));
                        double t = tau * (a.chd[S.chan_off + (k - S.k_lo)].nu * (1.0 / C_LIGHT));
                        t -= floor(t);
                        ph = turns_to_phasor((float)t);
                    }
                    if (jn[q] >> 28) {
                        const ChanD *cd = a.chd + S.chan_off + (k - S.k_lo);
                        const int iu = axis_cell(rec.u, su[q], S.uvw + 3 * row, fold, &cd->su, a.g.nu);
                        const int iv = axis_cell(rec.v, sv[q], S.uvw + 3 * row + 1, fold, &cd->sv, a.g.nv);
                        const int cid = (iu >= 0 && iv >= 0) ? iv * a.g.nu + iu : -1;
                        if (cid != cell[q]) {
                            flush(q);
                            cell[q] = cid;
                        }
#pragma unroll
                        for (int p = 0; p < P; ++p) {
                            if (plane[p] < 0) continue;
                            if ((F[q] >> (8 * p)) & 0xffu) {
                                ++n_flag;
                                continue;
                            }
                            if (cid < 0) {
                                ++n_duv;
                                continue;
                            }
                            float2 vs = cmul(V[q][p], ph);
                            if (fold) vs.y = -vs.y;
                            const float W = rec.W[p];
                            const float a2 = V[q][p].x * V[q][p].x + V[q][p].y * V[q][p].y;
                            acc[q][p].x += W * vs.x;
                            acc[q][p].y += W * vs.y;
                            acc[q][p].z += W;
                            acc[q][p].w += W * a2;
                            cnt[q][p] += 1;
                        }
                    }
                    if (linear && q + 1 < NS) ph = cmul(ph, make_float2(rec.sre, rec.sim));
                }
            }
        }
#pragma unroll
        for (int q = 0; q < NS; ++q) flush(q);
        s ^= 1;
    }

    // counters (the visibilities read are counted on the host from the
    // channel tables): warp sum, one atomic per counter per warp
    unsigned long long c3[3] = {n_flag, n_duv, n_red};
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c3[k] += __shfl_xor_sync(0xffffffffu, c3[k], o);
    if (lane == 0) {
        if (c3[0]) atomicAdd(&a.stats->n_flagged, c3[0]);
        if (c3[1]) atomicAdd(&a.stats->n_dropped_uv, c3[1]);
        if (c3[2]) atomicAdd(&a.stats->n_reductions, c3[2]);
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

// Prefetch depth D (rows of visibilities in flight per warp): deeper rings
// hide more HBM latency but cost registers; the common storage types get a
// choice, the rest one depth per channels-per-lane.
template <int P, int VT>
static cudaError_t launch_mixed_p(const RunArgs &a, int ns, int pf, int wpc, cudaStream_t st)
{
    constexpr bool choice = VT != VISTA_VIS_C128 && P <= 2;
    switch (ns) {
    case 1:
        if constexpr (choice) {
            if (pf >= 8) return launch_persistent(stack_mixed<P, VT, 1, 8>, a, wpc, st);
            if (pf >= 4) return launch_persistent(stack_mixed<P, VT, 1, 4>, a, wpc, st);
        }
        return launch_persistent(stack_mixed<P, VT, 1, 2>, a, wpc, st);
    case 2:
        if constexpr (choice) {
            if (pf >= 4) return launch_persistent(stack_mixed<P, VT, 2, 4>, a, wpc, st);
        }
        return launch_persistent(stack_mixed<P, VT, 2, (P <= 2 ? 2 : 1)>, a, wpc, st);
    case 4: return launch_persistent(stack_mixed<P, VT, 4, 1>, a, wpc, st);
    default: return cudaErrorInvalidValue;
    }
}

template <int VT>
static cudaError_t launch_mixed_vt(const RunArgs &a, int ns, int pf, int npol, int wpc, cudaStream_t st)
{
    switch (npol) {
    case 1: return launch_mixed_p<1, VT>(a, ns, pf, wpc, st);
    case 2: return launch_mixed_p<2, VT>(a, ns, pf, wpc, st);
    case 4: return launch_mixed_p<4, VT>(a, ns, pf, wpc, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_mixed(const RunArgs &a, int key, int wpc, int prefetch, cudaStream_t st)
{
    const int npol = key & 0xff, ns = (key >> 8) & 0xff, vt = key >> 16;
    switch (vt) {
    case VISTA_VIS_C64: return launch_mixed_vt<VISTA_VIS_C64>(a, ns, prefetch, npol, wpc, st);
    case VISTA_VIS_C128: return launch_mixed_vt<VISTA_VIS_C128>(a, ns, prefetch, npol, wpc, st);
    case VISTA_VIS_F16X2: return launch_mixed_vt<VISTA_VIS_F16X2>(a, ns, prefetch, npol, wpc, st);
    case VISTA_VIS_BF16X2: return launch_mixed_vt<VISTA_VIS_BF16X2>(a, ns, prefetch, npol, wpc, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace vista

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
// uv cell stay in registers.  When a lane's cell changes, its finished run
// is appended to a per-warp staging area in shared memory (slots from a warp
// ballot, no divergent branch); the warp drains the staging area together,
// one lane per run, as float4 reductions per (cell, rest bin, pol) and one
// count reduction per (cell, rest bin) (one u64 for a pol pair).
#include "vista_device.cuh"

namespace vista {

constexpr int RB_MAX = 256;     // largest item (rows) the shared-memory buffers hold
constexpr int KMAX_THREADS = 256;   // blocks of at most 8 warps
constexpr int STAGE_CAP = 96;   // staged runs per warp

// One finished run of one channel slot.
template <int P>
struct __align__(16) Staged {
    int cell;         // iv * nu + iu
    int chf;          // channel-table entry (rest bins and weights)
    uint32_t cnt[P];
    float4 acc[P];    // sum W V'.re, sum W V'.im, sum W, sum W |V|^2
};

template <int P>
__host__ __device__ constexpr size_t warp_smem_bytes(int rb)
{
    return 2 * (size_t)rb * sizeof(RowRec) + STAGE_CAP * sizeof(Staged<P>) + 2 * sizeof(uint64_t);
}

template <int P, int VT, int NS, int D>
__global__ void __launch_bounds__(KMAX_THREADS) stack_mixed(RunArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int RB = a.so.rows_per_item;
    unsigned char *wsm = smem + (size_t)wid * warp_smem_bytes<P>(RB);
    RowRec *rbuf = reinterpret_cast<RowRec *>(wsm);
    Staged<P> *stage = reinterpret_cast<Staged<P> *>(wsm + 2 * (size_t)RB * sizeof(RowRec));
    uint64_t *bars = reinterpret_cast<uint64_t *>(wsm + 2 * (size_t)RB * sizeof(RowRec) +
                                                  STAGE_CAP * sizeof(Staged<P>));
    if (lane == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        mbar_init_fence();
    }
    __syncwarp();

    const uint32_t nitems = a.so.ctr[0];
    const int npol_c = a.g.npol, nrest = a.g.nrest;
    const unsigned lt_mask = (1u << lane) - 1u;
    float4 *cube4 = reinterpret_cast<float4 *>(a.cube);
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
            const RowRec *src = a.recs + S.rec_off + item.q0;
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
        // window fields in registers (the cube reductions could alias global
        // memory, so references into the table would be re-read)
        const void *vis;
        const uint8_t *flags;
        const double *uvw;
        int64_t vstride;
        float vscale;
        int k_lo, k_hi, chan_off;
        int plane[P];
        {
            const SrcDev &G = a.srcs[item.w];
            vis = G.vis;
            flags = G.flags;
            uvw = G.uvw;
            vstride = G.vstride;
            vscale = G.vis_scale;
            k_lo = G.k_lo;
            k_hi = G.k_hi;
            chan_off = G.chan_off;
            const int c0g = G.k_lo + item.chunk * 32 * NS;
            vis = reinterpret_cast<const char *>(G.vis) +
                  (int64_t)(c0g + lane - G.kbase) * P * (int64_t)VisLoad<P, VT>::kBytes;
            if (flags) flags += (int64_t)(c0g + lane - G.kbase) * P;
#pragma unroll
            for (int p = 0; p < P; ++p) plane[p] = G.plane[p];
        }
        const int c0 = k_lo + item.chunk * 32 * NS;
        const bool pack2 = (P == 2) && plane[0] >= 0 && plane[1] == plane[0] + 1 && !(plane[0] & 1) && !(npol_c & 1);

        // per channel slot: fl32(s_k), nu_k / c as float-float, and whether the
        // channel has a rest bin
        float su[NS], sv[NS], nh[NS], nl[NS];
        bool act[NS];
#pragma unroll
        for (int q = 0; q < NS; ++q) {
            const int k = c0 + q * 32 + lane;
            act[q] = false;
            su[q] = sv[q] = nh[q] = nl[q] = 0.f;
            if (k < k_hi) {
                const ChanF cf = a.chf[chan_off + (k - k_lo)];
                su[q] = cf.su;
                sv[q] = cf.sv;
                nh[q] = cf.nuc_hi;
                nl[q] = cf.nuc_lo;
                act[q] = cf.nb > 0;
            }
        }
        const int cslot = item.chunk < REC_CELLS ? item.chunk : -1;
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
        int nstaged = 0;

        // Stage lane runs that end here (`fl`): convergent, slots by ballot.
        // The caller drains whenever fewer than 32 slots are free, so the
        // index below stays inside the buffer; the check records a breach
        // instead of writing out of bounds.
        auto stage_runs = [&](int q, bool fl) {
            const unsigned bal = __ballot_sync(0xffffffffu, fl);
            const int slot = nstaged + __popc(bal & lt_mask);
            if (fl && slot >= STAGE_CAP) atomicExch(a.err, 3);
            if (fl && slot < STAGE_CAP) {
                Staged<P> &st = stage[slot];
                st.cell = cell[q];
                st.chf = chan_off + (c0 + q * 32 + lane - k_lo);
#pragma unroll
                for (int p = 0; p < P; ++p) {
                    st.cnt[p] = cnt[q][p];
                    st.acc[p] = acc[q][p];
                }
            }
            nstaged += __popc(bal);
        };
        // All lanes write the staged runs to the cube, one run per lane.
        auto drain = [&]() {
            __syncwarp();
            for (int e = lane; e < nstaged; e += 32) {
                const Staged<P> &st = stage[e];
                const ChanF cf = a.chf[st.chf];
                const size_t base = ((size_t)st.cell * nrest + cf.j0) * npol_c;
                for (int b = 0; b < cf.nb; ++b) {
                    const float ww = b == 0 ? cf.w0 : b == 1 ? cf.w1 : (float)a.chd[st.chf].w[b];
                    const size_t e2 = base + (size_t)b * npol_c;
#pragma unroll
                    for (int p = 0; p < P; ++p) {
                        if (st.cnt[p] == 0) continue;
                        const float4 v = st.acc[p];
                        atomicAdd(cube4 + e2 + plane[p], make_float4(ww * v.x, ww * v.y, ww * v.z, ww * v.w));
                        ++n_red;
                        if (!pack2) {
                            atomicAdd(a.count + e2 + plane[p], st.cnt[p]);
                            ++n_red;
                        }
                    }
                    if (pack2 && (st.cnt[0] | st.cnt[P - 1])) {
                        atomicAdd(reinterpret_cast<unsigned long long *>(a.count + e2 + plane[0]),
                                  (unsigned long long)st.cnt[0] | ((unsigned long long)st.cnt[P - 1] << 32));
                        ++n_red;
                    }
                }
            }
            __syncwarp();
            nstaged = 0;
        };

        // visibility / flag ring, D rows ahead
        const int n = item.q1 - item.q0;
        float2 RV[D][NS][P];
        uint32_t RF[D][NS];
        auto fetch = [&](int d, int i) {
            const int64_t row = (int64_t)(rb[i].rowf & 0x7fffffffu);
            const int64_t off = row * vstride;
#pragma unroll
            for (int q = 0; q < NS; ++q) {
                RF[d][q] = 0;
                if (act[q]) {
                    VisLoad<P, VT>::load(vis, off + q * 32, vscale, RV[d][q]);
                    RF[d][q] = load_flags<P>(flags, off + q * 32);
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
                const float th = rec.tau_hi, tl = rec.tau_lo;
                // the chunk's shared cell, if the pre-pass found one
                const int cinfo = cslot >= 0 ? rec.cell[cslot] : CELL_MIXED;
#pragma unroll
                for (int q = 0; q < NS; ++q) {
                    const int k = c0 + q * 32 + lane;
                    const float2 ph = shift_phasor(th, tl, nh[q], nl[q]);
                    int cid = cell[q];
                    if (act[q]) {
                        if (cinfo != CELL_MIXED) {
                            cid = cinfo;
                        } else {
                            const ChanD *cd = a.chd + chan_off + (k - k_lo);
                            const int iu = axis_cell(rec.u, su[q], uvw + 3 * row, fold, &cd->su, a.g.nu);
                            const int iv = axis_cell(rec.v, sv[q], uvw + 3 * row + 1, fold, &cd->sv, a.g.nv);
                            cid = (iu >= 0 && iv >= 0) ? iv * a.g.nu + iu : -1;
                        }
                    }
                    const bool newcell = cid != cell[q];
                    uint32_t any = 0;
#pragma unroll
                    for (int p = 0; p < P; ++p) any |= cnt[q][p];
                    stage_runs(q, newcell && cell[q] >= 0 && any != 0);
                    if (nstaged > STAGE_CAP - 32) drain();
                    if (newcell) {
                        cell[q] = cid;
#pragma unroll
                        for (int p = 0; p < P; ++p) {
                            acc[q][p] = make_float4(0.f, 0.f, 0.f, 0.f);
                            cnt[q][p] = 0;
                        }
                    }
                    if (act[q]) {
#pragma unroll
                        for (int p = 0; p < P; ++p) {
                            // short predicated bodies instead of branches
                            const bool pl = plane[p] >= 0;
                            const bool f = ((F[q] >> (8 * p)) & 0xffu) != 0;
                            const bool use = pl && !f && cid >= 0;
                            n_flag += (pl && f) ? 1u : 0u;
                            n_duv += (pl && !f && cid < 0) ? 1u : 0u;
                            float2 vs = cmul(V[q][p], ph);
                            vs.y = fold ? -vs.y : vs.y;
                            const float W = rec.W[p];
                            const float a2 = V[q][p].x * V[q][p].x + V[q][p].y * V[q][p].y;
                            if (use) {
                                acc[q][p].x += W * vs.x;
                                acc[q][p].y += W * vs.y;
                                acc[q][p].z += W;
                                acc[q][p].w += W * a2;
                                cnt[q][p] += 1;
                            }
                        }
                    }
                }
            }
        }
#pragma unroll
        for (int q = 0; q < NS; ++q) {
            uint32_t any = 0;
#pragma unroll
            for (int p = 0; p < P; ++p) any |= cnt[q][p];
            stage_runs(q, cell[q] >= 0 && any != 0);
            if (nstaged > STAGE_CAP - 32) drain();
        }
        drain();
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

template <int P, typename K>
static cudaError_t launch_persistent(K kern, const RunArgs &a, int wpc, cudaStream_t st)
{
    const int rb = a.so.rows_per_item;
    if (rb < 1 || rb > RB_MAX) return cudaErrorInvalidValue;
    static int smem_max = 0;
    if (smem_max == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    }
    // fewer warps per block when their staging buffers would not fit
    if (wpc * 32 > KMAX_THREADS) wpc = KMAX_THREADS / 32;
    while (wpc > 1 && (size_t)wpc * warp_smem_bytes<P>(rb) > (size_t)smem_max) wpc >>= 1;
    const size_t smem = (size_t)wpc * warp_smem_bytes<P>(rb);
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
            if (pf >= 8) return launch_persistent<P>(stack_mixed<P, VT, 1, 8>, a, wpc, st);
            if (pf >= 4) return launch_persistent<P>(stack_mixed<P, VT, 1, 4>, a, wpc, st);
        }
        return launch_persistent<P>(stack_mixed<P, VT, 1, 2>, a, wpc, st);
    case 2:
        if constexpr (choice) {
            if (pf >= 4) return launch_persistent<P>(stack_mixed<P, VT, 2, 4>, a, wpc, st);
        }
        return launch_persistent<P>(stack_mixed<P, VT, 2, (P <= 2 ? 2 : 1)>, a, wpc, st);
    case 4: return launch_persistent<P>(stack_mixed<P, VT, 4, 1>, a, wpc, st);
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

// The mixed-precision stacking kernel (sm_103a).  Each visibility type's
// instantiations are compiled in a translation unit of their own
// (vista_stack_<type>.cu, built in parallel); vista_stack.cu dispatches.
//
// Persistent: warp g of G takes work items g, g + G, g + 2G, ... of a list
// in stripe-major order (item = one window, up to rows_per_item rows in
// uv-cell order, a chunk of 32 x NS channels, lane = channel).  While a warp
// processes an item, TMA bulk copies (one mbarrier per slot) bring the next
// item's row records, chunk cells, window header, channel table and work-list
// entries into the other shared-memory slot, so an item starts without a
// global round trip.  Inside an item the visibilities and flags of the next
// D - 1 rows are in flight into a shared-memory ring (cp.async), so the row
// loop waits on no synchronous global load.  Each lane copies the 4-byte flag
// word that holds its flags (a chunk's flags start on a word, see
// flag_align_channels) and, when a lane's values are at most 16 bytes, its
// own values.  Wider values (four pols, or complex128) are copied in 16-byte
// pieces with piece i of lane L at byte 512 i + 16 L of the row's channel
// slot, so that every cp.async instruction of the warp reads 512 contiguous
// bytes (a lane copying its own 32 bytes as two pieces would make each
// instruction read half of every 32-byte sector, and fetch each sector from
// L2 twice); the warp then synchronises before a row's values are read and
// before their ring slot is refilled.
//
// Per (row, channel): the FP32 phasor of Eq. 2 from the record's float-float
// delay and the channel's float-float nu_k / c, the uv cell from the chunk's
// cell entry (exact: computed by the pre-pass with the FP64 rule), rest bins
// and Eq. 4 weights from the FP64 channel table.  Per lane, running sums
// over consecutive rows that share a uv cell stay in registers.  When a
// lane's cell changes, its finished run goes to a per-warp circular staging
// area in shared memory (slots from a warp ballot); once 32 runs wait the
// warp drains them together (between rows, from one place in the code, so
// the drain is compiled once), one lane per run, as float4 reductions per
// (cell, rest bin, pol) and one count reduction per (cell, rest bin) (one
// u64 for a pol pair).  Runs off the grid only feed the dropped counter.
#pragma once
#include <climits>

#include "vista_device.cuh"

namespace vista {

constexpr int RB_MAX = 256;         // largest item (rows) the shared-memory buffers hold
constexpr int KMAX_THREADS = 256;   // blocks of at most 8 warps
// staged runs per warp (circular; a power of two): at most 31 wait before a
// row, which may stage 32 per channel slot
template <int NS>
__host__ __device__ constexpr int stage_cap() { return NS == 1 ? 64 : NS == 2 ? 128 : 256; }
constexpr uint32_t CKPT_EVERY = 8;     // valid runs of a lane between checkpoint choices (a power of two)
constexpr uint32_t SERVICE_EVERY = 4;  // 1 / probability that a drain exchanges the chosen entries (a power of two)
constexpr int NO_RUN = INT_MIN;     // lane holds no run

// What a window without flags reads as its flags (every row: pitch 0).
__device__ __align__(16) uint8_t g_zero_flags[512];

// One finished run of one channel slot.
template <int P>
struct __align__(16) Staged {
    int cell;         // iv * nu + iu, -1 off the grid
    int kk;           // chunk-local channel
    uint32_t cnt[P];
    float4 acc[P];    // sum W V'.re, sum W V'.im, sum W, sum W |V|^2
};

// A shared-memory channel-table entry as two 16-byte loads (a 32-byte stride
// read in 4-byte pieces conflicts eight ways).
__device__ __forceinline__ ChanF load_chanf(const ChanF *p)
{
    const int4 a = *reinterpret_cast<const int4 *>(p);
    const float4 b = *reinterpret_cast<const float4 *>(reinterpret_cast<const char *>(p) + 16);
    ChanF c;
    c.su = __int_as_float(a.x);
    c.sv = __int_as_float(a.y);
    c.j0 = a.z;
    c.nb = a.w;
    c.w0 = b.x;
    c.w1 = b.y;
    c.nuc_hi = b.z;
    c.nuc_lo = b.w;
    return c;
}

// A 32-bit integer hash (C. Wellons' "lowbias32" finaliser): which drains
// exchange the lanes' chosen checkpoint entries.
__device__ __forceinline__ uint32_t mix32(uint32_t x)
{
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

// Weight of a third or fourth rest bin (lattices narrower than a channel;
// out of line so that its FP64 conversion is not hoisted into every drain).
static __device__ __noinline__ float far_bin_weight(const ChanD *cd, int b) { return (float)cd->w[b]; }

// A float as a double, exactly, by moving its IEEE-754 fields (integer
// instructions; the FP64 unit converts slowly).  Zero and subnormal inputs
// give zero (below 1.2e-38), infinities and NaNs do not occur in the sums.
__device__ __forceinline__ double widen(float x)
{
    const uint32_t b = __float_as_uint(x);
    const uint32_t e = (b >> 23) & 0xffu;
    if (e == 0u) return 0.0;
    const uint32_t hi = (b & 0x80000000u) | ((e + 896u) << 20) | ((b & 0x7fffffu) >> 3);
    return __hiloint2double((int)hi, (int)(b << 29));
}

// Chunk-cell entries per slot: an item's rows plus the entries that round
// its bulk copy out to 16-byte boundaries.
__host__ __device__ constexpr int cc_slot_entries(int rb) { return (rb + 3) & ~1; }

// One item slot in shared memory (filled by bulk copies).
template <int P, int NS>
__host__ __device__ constexpr size_t slot_bytes(int rb)
{
    return 2 * sizeof(Item) + sizeof(SrcDev) + 32 * NS * sizeof(ChanF) + (size_t)rb * sizeof(RowRec) +
           (size_t)cc_slot_entries(rb) * sizeof(int2);
}

// Per-warp shared memory: two item slots, the D-row visibility and flag
// rings, the staging area and two mbarriers.
template <int P, int VT, int NS, int D>
__host__ __device__ constexpr size_t warp_smem_bytes(int rb)
{
    return 2 * slot_bytes<P, NS>(rb) + (size_t)D * NS * 32 * (VisAsync<P, VT>::kLaneBytes + 4) +
           stage_cap<NS>() * sizeof(Staged<P>) + 2 * sizeof(uint64_t);
}

// Views of one slot.
template <int NS>
struct Slot {
    Item *self, *next;   // this item, the item after it (same warp)
    SrcDev *hdr;
    ChanF *chf;
    RowRec *rec;
    int2 *cells;
    __device__ Slot(unsigned char *base, int rb)
    {
        self = reinterpret_cast<Item *>(base);
        next = self + 1;
        hdr = reinterpret_cast<SrcDev *>(next + 1);
        chf = reinterpret_cast<ChanF *>(hdr + 1);
        rec = reinterpret_cast<RowRec *>(chf + 32 * NS);
        cells = reinterpret_cast<int2 *>(rec + rb);
    }
};

template <int P, int VT, int NS, int D>
__global__ void __launch_bounds__(KMAX_THREADS) stack_mixed(RunArgs a)
{
    static_assert(D >= 2 && (D & (D - 1)) == 0, "ring depth: a power of two");
    using VA = VisAsync<P, VT>;
    constexpr int LB = VA::kLaneBytes;
    constexpr int FWD = 32 * NS;                // flag words of one (row, chunk): one per lane and slot
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int RB = a.so.rows_per_item;
    unsigned char *wsm = smem + (size_t)wid * warp_smem_bytes<P, VT, NS, D>(RB);
    auto slot_at = [&](int s) { return Slot<NS>(wsm + (size_t)s * slot_bytes<P, NS>(RB), RB); };
    unsigned char *vring = wsm + 2 * slot_bytes<P, NS>(RB);
    unsigned char *fring = vring + (size_t)D * NS * 32 * LB;
    Staged<P> *stage = reinterpret_cast<Staged<P> *>(fring + (size_t)D * FWD * 4);
    uint64_t *bars = reinterpret_cast<uint64_t *>(stage + stage_cap<NS>());
    if (lane == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        mbar_init_fence();
    }
    __syncwarp();
    const uint32_t vring_lane = smem_addr(vring) + (uint32_t)lane * LB;
    const uint32_t vring_base = smem_addr(vring);
    const unsigned char *vring_lane_p = vring + lane * LB;
    const uint32_t fring_lane = smem_addr(vring) + (uint32_t)(D * NS * 32 * LB) + 4u * (uint32_t)lane;

    const uint32_t nitems = a.so.ctr[0];
    const uint32_t G = gridDim.x * (blockDim.x >> 5);
    const uint32_t gw = blockIdx.x * (blockDim.x >> 5) + wid;
    const int npol_c = a.g.npol, nrest = a.g.nrest, gnu = a.g.nu, gnv = a.g.nv;
    const bool comp = a.comp != 0;
    const unsigned lt_mask = (1u << lane) - 1u;
    float4 *cube4 = reinterpret_cast<float4 *>(a.cube);
    // visibilities read, stacked (unflagged, on the grid) and dropped off the
    // grid; flagged = read - stacked - dropped
    uint32_t n_read = 0, n_ok = 0, n_duv = 0, n_red = 0;
    // drains of this warp (hashed: the schedule of checkpoint exchanges)
    uint32_t n_drains = gw << 16;
    // valid runs this lane drained (offset: lanes choose at different times)
    // and the entry chosen at its last choice, not yet exchanged (-1: none)
    uint32_t n_runs = lane * 37u;
    int64_t ck_e = -1;
    // the lane's pending checkpoint: FP32 sums taken out of the cube, to be
    // added to the master entry ck_dst
    float4 ck_took = make_float4(0.f, 0.f, 0.f, 0.f);
    double *ck_dst = nullptr;
    auto flush_ckpt = [&]() {
        if (ck_dst) {
            atomicAdd(ck_dst, widen(ck_took.x));
            atomicAdd(ck_dst + 1, widen(ck_took.y));
            atomicAdd(ck_dst + 2, widen(ck_took.z));
            atomicAdd(ck_dst + 3, widen(ck_took.w));
            n_red += 4;
            ck_dst = nullptr;
        }
    };
    // warp sums of the counters, one atomic per counter per warp (at the
    // end, or early if a lane's count nears 2^32)
    auto flush_counters = [&]() {
        unsigned long long c3[3] = {(unsigned long long)n_read - n_ok - n_duv, n_duv, n_red};
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) c3[k] += __shfl_xor_sync(0xffffffffu, c3[k], o);
        if (lane == 0) {
            if (c3[0]) atomicAdd(&a.stats->n_flagged, c3[0]);
            if (c3[1]) atomicAdd(&a.stats->n_dropped_uv, c3[1]);
            if (c3[2]) atomicAdd(&a.stats->n_reductions, c3[2]);
        }
        n_read = n_ok = n_duv = n_red = 0;
    };
    uint32_t phase = 0;   // bit s: parity of the next completion of slot s

    // Lane 0: bulk copies of item `it` (its entry `item`) into slot s,
    // together with the entry of the warp's following item `itn`, if any.
    auto issue = [&](int s, uint32_t it, const Item &item, uint32_t itn) {
        const Slot<NS> S = slot_at(s);
        const int n = item.q1 - item.q0;
        const int64_t e0a = item.cell0 & ~(int64_t)1;
        const uint32_t ncc = (uint32_t)((item.cell0 + n - e0a + 1) & ~(int64_t)1);
        const uint32_t b_items = (uint32_t)sizeof(Item) * (itn < nitems ? 2u : 1u);
        const uint32_t b_chf = (uint32_t)item.nch * (uint32_t)sizeof(ChanF);
        const uint32_t b_rec = (uint32_t)n * (uint32_t)sizeof(RowRec), b_cc = ncc * (uint32_t)sizeof(int2);
        fence_proxy_async();
        mbar_expect_tx(&bars[s], b_items + (uint32_t)sizeof(SrcDev) + b_chf + b_rec + b_cc);
        tma_load_1d(S.self, a.so.items + it, (uint32_t)sizeof(Item), &bars[s]);
        if (itn < nitems) tma_load_1d(S.next, a.so.items + itn, (uint32_t)sizeof(Item), &bars[s]);
        tma_load_1d(S.hdr, a.srcs + item.w, (uint32_t)sizeof(SrcDev), &bars[s]);
        tma_load_1d(S.chf, a.chf + item.chf0, b_chf, &bars[s]);
        tma_load_1d(S.rec, a.recs + item.rec0, b_rec, &bars[s]);
        tma_load_1d(S.cells, a.ccells + e0a, b_cc, &bars[s]);
    };

    uint32_t it = gw;
    if (lane == 0 && it < nitems) {
        const Item first = a.so.items[it];
        issue(0, it, first, it + G);
    }
    int s = 0;
    for (; it < nitems; it += G, s ^= 1) {
        const int cs = s;
        __syncwarp();
        if (!mbar_wait_bounded(&bars[cs], (phase >> cs) & 1u, a.err)) {
            // the copy in flight gets one more bounded wait before the warp stops
            mbar_wait_bounded(&bars[cs], (phase >> cs) & 1u, a.err);
            break;
        }
        phase ^= 1u << cs;
        const Slot<NS> S = slot_at(cs);
        // the next item's copies run while this one is processed
        if (lane == 0 && it + G < nitems) issue(cs ^ 1, it + G, *S.next, it + 2 * G);

        // ---- one item ----
        // window fields in registers (the cube reductions could alias global
        // memory, so reads through pointers would be repeated)
        const RowRec *rb = S.rec;
        const ChanF *ctab = S.chf;
        const int2 *cb;
        const unsigned char *vis0;   // the chunk's first channel of row 0
        uint32_t vrow_bytes;         // visibility bytes per row
        const uint8_t *fw0;          // the flag word holding this lane's slot-0 flags in row 0
        uint32_t frow_bytes;         // flag bytes per row (0: no flags, all zero)
        const double *uvw;
        float vscale;
        int nch, chf0, n;
        int plane[P];
        {
            const SrcDev &H = *S.hdr;
            const Item &I = *S.self;
            uvw = H.guvw;   // the gridding baselines (the per-channel cell fall-back)
            vscale = H.vis_scale;
            nch = I.nch;
            chf0 = I.chf0;
            n = I.q1 - I.q0;
            const int64_t c0 = (int64_t)(H.k_lo + I.chunk * 32 * NS - H.kbase);
            vis0 = reinterpret_cast<const unsigned char *>(H.vis) + c0 * LB;
            vrow_bytes = (uint32_t)(H.vstride * LB);
            const int fl0 = (min(lane, I.nch - 1) * P) & ~3;
            if (H.fbase) {
                fw0 = H.fbase + (int64_t)(H.k_lo + I.chunk * 32 * NS - H.fk0) * P + fl0;
                frow_bytes = (uint32_t)H.fpitch;
            } else {
                fw0 = g_zero_flags + fl0;
                frow_bytes = 0;
            }
#pragma unroll
            for (int p = 0; p < P; ++p) plane[p] = H.plane[p];
            cb = S.cells + (I.cell0 & 1);
        }
        // pol pairs (2k, 2k + 1) whose count entries are adjacent and 8-byte
        // aligned take one u64 reduction for both counts
        constexpr int NPK = P >= 2 ? P / 2 : 1;
        bool pk[NPK];
#pragma unroll
        for (int k = 0; k < NPK; ++k)
            pk[k] = P >= 2 && plane[2 * k] >= 0 && plane[2 * k + 1] == plane[2 * k] + 1 && !(plane[2 * k] & 1) &&
                    !(npol_c & 1);
        int npl = 0;
#pragma unroll
        for (int p = 0; p < P; ++p) npl += plane[p] >= 0;

        // per channel slot: nu_k / c as float-float, whether the channel has
        // a rest bin, and the lane's byte offsets (lanes past the chunk's last
        // channel read that channel: always inside the row)
        float nh[NS], nl[NS];
        bool act[NS];
        int kv[NS], fo[NS], fsh[NS];
        // wide values: the row offsets of the 16-byte pieces this lane copies
        // (pieces past the chunk's last channel re-read that channel's bytes)
        constexpr int NPC = LB >= 32 ? LB / 16 : 1;
        int gv[NS][NPC];
#pragma unroll
        for (int q = 0; q < NS; ++q) {
            const int kk = q * 32 + lane, kc = min(kk, nch - 1);
            const ChanF cf = load_chanf(ctab + kc);
            nh[q] = cf.nuc_hi;
            nl[q] = cf.nuc_lo;
            act[q] = kk < nch && cf.nb > 0;
            kv[q] = kc * LB;
            fo[q] = ((kc * P) & ~3) - ((min(lane, nch - 1) * P) & ~3);
            fsh[q] = 8 * ((kc * P) & 3);
#pragma unroll
            for (int i = 0; i < NPC; ++i) {
                const int g = 512 * i + 16 * lane, ch = q * 32 + g / LB;
                gv[q][i] = ch < nch ? q * 32 * LB + g : (nch - 1) * LB + g % LB;
            }
            if (act[q]) n_read += (uint32_t)(n * npl);
        }

        // the cell of channel slot q in row i (NO_RUN for a lane without a
        // channel); chunk entries are shared by the warp, so the branches are
        // taken by all lanes alike
        auto lane_cell = [&](int q, int2 cc, int i) -> int {
            int cid;
            if (__all_sync(0xffffffffu, cc.y == CC_NOCHANGE)) {
                cid = cc.x;
            } else if (__all_sync(0xffffffffu, cc.y != CC_MIXED)) {
                cid = chunk_cell_step(cc, q * 32 + lane, gnu);
            } else {
                cid = NO_RUN;
                if (act[q]) {
                    const float4 r0 = *reinterpret_cast<const float4 *>(&rb[i]);
                    cid = cell_exact(uvw, rb[i].row, signbit(r0.z), a.chd + chf0 + q * 32 + lane, gnu,
                                     gnv);
                }
            }
            return act[q] ? cid : NO_RUN;
        };

        int cell[NS];
        float4 acc[NS][P];
        uint32_t cnt[NS][P];
        {
            const int2 cc0 = cb[0];
#pragma unroll
            for (int q = 0; q < NS; ++q) {
                cell[q] = lane_cell(q, cc0, 0);
#pragma unroll
                for (int p = 0; p < P; ++p) {
                    acc[q][p] = make_float4(0.f, 0.f, 0.f, 0.f);
                    cnt[q][p] = 0;
                }
            }
        }
        uint32_t head = 0, count = 0;   // circular staging area

        // The warp writes min(count, 32) staged runs to the cube, one per lane:
        // a float4 reduction per (cell, rest bin, pol) and the counts.  With
        // checkpoints (comp), at every CKPT_EVERY-th valid run it drains, a lane
        // chooses one entry of that run (cycling through its bins and pols);
        // in one drain in SERVICE_EVERY (drawn by a hash of the warp's drain
        // counter, so the same for all lanes) the lanes holding a choice move
        // the chosen entry's FP32 sums into the FP64 master cube together:
        // 16-byte atomic exchange with zero, and the FP64 reductions of the
        // value taken at the lane's next exchange (or at the end), so no drain
        // waits on a returned value.  An entry's FP32 sum thus holds only the
        // runs since its last checkpoint, about CKPT_EVERY x (entries per run).
        // The choice is per lane and per run: the same choice made by all lanes
        // at the same drain checkpoints the cube's deepest entries less often
        // (measured on the batched stack: 1.7e-5 against 9e-6 relative error).
        auto drain = [&]() {
            __syncwarp();
            // warp-uniform, so that the exchange code runs once for all lanes
            // rather than for a few lanes in most drains
            const bool service = comp && (mix32(++n_drains) & (SERVICE_EVERY - 1)) == 0;
            if ((uint32_t)lane < count) {
                const Staged<P> st = stage[(head + lane) & (stage_cap<NS>() - 1)];
                uint32_t tot = 0;
#pragma unroll
                for (int p = 0; p < P; ++p) tot += plane[p] >= 0 ? st.cnt[p] : 0u;
                if (st.cell < 0) {
                    n_duv += tot;
                } else {
                    n_ok += tot;
                    const ChanF ct = load_chanf(ctab + st.kk);
                    const int nb = ct.nb;
                    const size_t base = ((size_t)st.cell * nrest + ct.j0) * npol_c;
                    for (int b = 0; b < nb; ++b) {
                        const float ww = b == 0 ? ct.w0 : b == 1 ? ct.w1 : far_bin_weight(a.chd + chf0 + st.kk, b);
                        const size_t e2 = base + (size_t)b * npol_c;
#pragma unroll
                        for (int p = 0; p < P; ++p) {
                            if (plane[p] < 0 || st.cnt[p] == 0) continue;
                            const float4 v = st.acc[p];
                            atomicAdd(cube4 + e2 + plane[p], make_float4(ww * v.x, ww * v.y, ww * v.z, ww * v.w));
                            ++n_red;
                            if (!(P >= 2 && pk[p / 2])) {
                                atomicAdd(a.count + e2 + plane[p], st.cnt[p]);
                                ++n_red;
                            }
                        }
#pragma unroll
                        for (int k = 0; k < (P >= 2 ? P / 2 : 0); ++k) {
                            if (pk[k] && (st.cnt[2 * k] | st.cnt[2 * k + 1])) {
                                atomicAdd(reinterpret_cast<unsigned long long *>(a.count + e2 + plane[2 * k]),
                                          (unsigned long long)st.cnt[2 * k] |
                                              ((unsigned long long)st.cnt[2 * k + 1] << 32));
                                ++n_red;
                            }
                        }
                    }
                    if (comp && ((++n_runs & (CKPT_EVERY - 1)) == 0)) {
                        // choose one entry of this run (cycling through its bins and pols)
                        const uint32_t pick = n_runs / CKPT_EVERY;
                        const int b = (int)(pick / P) % (nb < 2 ? nb : 2), pp = (int)(pick % P);
                        int pl = -1;
#pragma unroll
                        for (int p = 0; p < P; ++p)   // static indices (no local-memory copy)
                            if (p == pp && plane[p] >= 0 && st.cnt[p] != 0) pl = plane[p];
                        if (pl >= 0) ck_e = (int64_t)(base + (size_t)b * npol_c + pl);
                    }
                }
            }
            if (service && ck_e >= 0) {
                // complete the lane's previous exchange, whose value has long
                // arrived, then take the chosen entry's FP32 sums
                flush_ckpt();
                ck_took = atomicExch(cube4 + ck_e, make_float4(0.f, 0.f, 0.f, 0.f));
                ck_dst = a.cube_master + 4 * ck_e;
                ck_e = -1;
                ++n_red;
            }
            __syncwarp();
            const uint32_t k = count < 32u ? count : 32u;
            head += k;
            count -= k;
        };
        // A lane whose cell changes stages its finished run and starts a new
        // one (staging only: the warp drains between rows, see below).
        auto next_cell = [&](int q, int cid) {
            const bool fl = cid != cell[q];
            const unsigned bal = __ballot_sync(0xffffffffu, fl);
            if (bal) {
                if (fl) {
                    Staged<P> &st = stage[(head + count + __popc(bal & lt_mask)) & (stage_cap<NS>() - 1)];
                    st.cell = cell[q];
                    st.kk = q * 32 + lane;
#pragma unroll
                    for (int p = 0; p < P; ++p) {
                        st.cnt[p] = cnt[q][p];
                        st.acc[p] = acc[q][p];
                    }
                    cell[q] = cid;
#pragma unroll
                    for (int p = 0; p < P; ++p) {
                        acc[q][p] = make_float4(0.f, 0.f, 0.f, 0.f);
                        cnt[q][p] = 0;
                    }
                }
                count += __popc(bal);
            }
        };

        // D-row rings of visibilities and flags, filled by cp.async (one
        // commit group per row); row i sits in slot i mod D.  Each lane copies
        // its own values and the flag word holding its flags (inside the row).
        auto fetch = [&](int d, int i) {
            const uint32_t row = rb[i].row;
            const unsigned char *vrow = vis0 + (uint64_t)row * vrow_bytes;
#pragma unroll
            for (int q = 0; q < NS; ++q) {
                if constexpr (LB >= 32) {
#pragma unroll
                    for (int i = 0; i < NPC; ++i)
                        cp_async_16(vring_base + (uint32_t)((d * NS + q) * 32 * LB + 512 * i + 16 * lane),
                                    vrow + gv[q][i]);
                } else {
                    VA::copy(vring_lane + (uint32_t)((d * NS + q) * 32 * LB), vrow + kv[q]);
                }
            }
            const uint8_t *frow = fw0 + (uint64_t)row * frow_bytes;
#pragma unroll
            for (int q = 0; q < NS; ++q) cp_async_4(fring_lane + (uint32_t)(d * FWD * 4 + 128 * q), frow + fo[q]);
        };
        auto body = [&](int i, int d) {
            const float4 r0 = *reinterpret_cast<const float4 *>(&rb[i]);   // tau_hi, tau_lo, W0, W1
            float W[P];
            W[0] = r0.z;
            if constexpr (P > 1) W[1] = r0.w;
            if constexpr (P > 2) {
                const float2 r1 = *reinterpret_cast<const float2 *>(&rb[i].W[2]);
                W[2] = r1.x;
                W[3] = r1.y;
            }
            const int2 cc = cb[i];
#pragma unroll
            for (int q = 0; q < NS; ++q) {
                float2 V[P];
                VA::decode(vring_lane_p + (size_t)(d * NS + q) * 32 * LB, vscale, V);
                const uint32_t F = *reinterpret_cast<const uint32_t *>(fring + d * FWD * 4 + (q * 32 + lane) * 4) >> fsh[q];
                const float2 ph = shift_phasor(r0.x, r0.y, nh[q], nl[q]);
                next_cell(q, lane_cell(q, cc, i));
#pragma unroll
                for (int p = 0; p < P; ++p) {
                    const bool ok = ((F >> (8 * p)) & 0xffu) == 0;
                    const float2 v = V[p];
                    const float re = v.x * ph.x - v.y * ph.y;
                    const float im = v.x * ph.y + v.y * ph.x;
                    const float a2 = v.x * v.x + v.y * v.y;
                    const float Ws = W[p], Wa = fabsf(Ws);   // the sign conjugates folded rows
                    acc[q][p].x = ok ? __fmaf_rn(Wa, re, acc[q][p].x) : acc[q][p].x;
                    acc[q][p].y = ok ? __fmaf_rn(Ws, im, acc[q][p].y) : acc[q][p].y;
                    acc[q][p].z = ok ? acc[q][p].z + Wa : acc[q][p].z;
                    acc[q][p].w = ok ? __fmaf_rn(Wa, a2, acc[q][p].w) : acc[q][p].w;
                    cnt[q][p] += ok ? 1u : 0u;
                }
            }
        };

#pragma unroll
        for (int d = 0; d < D - 1; ++d) {
            fetch(d, min(d, n - 1));
            cp_async_commit();
        }
        // Rows are processed while fewer than 32 runs wait; then the warp
        // drains (one drain in the code: the loop comes back to it at the
        // item's end, when the runs still open are staged too, once fewer
        // than 32 wait, so at most 31 + 32 NS are ever staged).
        int i = 0;
        bool open = true;
#pragma unroll 1
        for (;;) {
#pragma unroll 1
            while (i < n && count < 32u) {
                if constexpr (LB >= 32) __syncwarp();   // every lane is done with the slot refilled next
                fetch((i + D - 1) & (D - 1), min(i + D - 1, n - 1));
                cp_async_commit();
                cp_async_wait<D - 1>();
                if constexpr (LB >= 32) __syncwarp();   // the row's pieces were copied by other lanes
                body(i, i & (D - 1));
                ++i;
            }
            if (open && i >= n && count < 32u) {   // room for one more run per lane and slot
                cp_async_wait<0>();
#pragma unroll
                for (int q = 0; q < NS; ++q) next_cell(q, NO_RUN);
                open = false;
            }
            if (count == 0u) break;
            drain();
        }
        if (__any_sync(0xffffffffu, (n_read | n_ok | n_duv | n_red) >= 0x40000000u)) flush_counters();
    }

    flush_ckpt();
    // counters (the visibilities read are also counted on the host from the
    // channel tables)
    flush_counters();
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

template <int P, int VT, int NS, int D>
static cudaError_t launch_persistent(const RunArgs &a, int wpc, cudaStream_t st)
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
    auto kern = stack_mixed<P, VT, NS, D>;
    const size_t wsm = warp_smem_bytes<P, VT, NS, D>(rb);
    if (wpc * 32 > KMAX_THREADS) wpc = KMAX_THREADS / 32;
    while (wpc > 1 && (size_t)wpc * wsm > (size_t)smem_max) wpc >>= 1;
    const size_t smem = (size_t)wpc * wsm;
    if (smem > (size_t)smem_max) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, wpc * 32, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    kern<<<per_sm * sm_count(), wpc * 32, smem, st>>>(a);
    return cudaGetLastError();
}

// Ring depth D (rows of visibilities in flight per warp): the ring lives in
// shared memory, so depth costs only its flag registers and code size.  One
// channel per lane takes D = 2, 4 or 8 (prefetch_rows), two take 2 or 4,
// four take 2.
template <int P, int VT>
static cudaError_t launch_mixed_p(const RunArgs &a, int ns, int pf, int wpc, cudaStream_t st)
{
    switch (ns) {
    case 1:
        if (pf >= 8) return launch_persistent<P, VT, 1, 8>(a, wpc, st);
        if (pf >= 4) return launch_persistent<P, VT, 1, 4>(a, wpc, st);
        return launch_persistent<P, VT, 1, 2>(a, wpc, st);
    case 2:
        if (pf >= 4) return launch_persistent<P, VT, 2, 4>(a, wpc, st);
        return launch_persistent<P, VT, 2, 2>(a, wpc, st);
    case 4: return launch_persistent<P, VT, 4, 2>(a, wpc, st);
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

// One visibility type's launchers (vista_stack_<type>.cu).
cudaError_t launch_mixed_c64(const RunArgs &a, int ns, int pf, int npol, int wpc, cudaStream_t st);
cudaError_t launch_mixed_c128(const RunArgs &a, int ns, int pf, int npol, int wpc, cudaStream_t st);
cudaError_t launch_mixed_f16(const RunArgs &a, int ns, int pf, int npol, int wpc, cudaStream_t st);
cudaError_t launch_mixed_bf16(const RunArgs &a, int ns, int pf, int npol, int wpc, cudaStream_t st);

}  // namespace vista

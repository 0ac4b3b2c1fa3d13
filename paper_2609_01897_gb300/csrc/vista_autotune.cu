// vista_autotune(): choose the stacking launch shape for a queued source set
// by timing it.
//
// Each candidate launch shape (rows per work item, channels per lane, warps
// per block, visibility rows in flight) runs the queued set with event timing
// of the device pass (row-ordering pre-pass + stacking kernels); the fastest
// of `reps` runs per candidate counts.  The handle keeps the winner.  The
// trial runs accumulate into the handle's cube, which is zeroed afterwards,
// and the queue is left as it was, for the caller's own vista_run().
#include <algorithm>
#include <vector>

#include "vista_handle.h"

using namespace vista;

namespace {

// Candidate shapes, most promising first (the budget keeps a prefix).
std::vector<LaunchCfg> candidates(const LaunchCfg &cur)
{
    std::vector<LaunchCfg> c;
    auto add = [&](int rows, int cpl, int wpc, int pf) {
        for (const LaunchCfg &x : c)
            if (x.rows_per_item == rows && x.chans_per_lane == cpl && x.warps_per_cta == wpc && x.prefetch_rows == pf)
                return;
        c.push_back(LaunchCfg{rows, cpl, wpc, cur.sort_rows, pf});
    };
    add(cur.rows_per_item, cur.chans_per_lane, cur.warps_per_cta, cur.prefetch_rows);
    const int rows[] = {64, 48, 32, 96};
    const int pfs[] = {4, 2, 8};
    for (int cpl : {1, 2})
        for (int pf : pfs)
            for (int r : rows) add(r, cpl, 4, pf);
    for (int r : rows) add(r, 1, 2, 4);
    for (int r : rows) add(r, 1, 8, 4);
    return c;
}

}  // namespace

extern "C" int vista_autotune(vista_stack *h, int32_t budget, int32_t reps, vista_tuning *best)
{
    if (!handle_live(h)) return fail(nullptr, VISTA_E_STATE, "unknown or closed handle");
    if (h->pending.empty()) return fail(h, VISTA_E_STATE, "vista_autotune with no queued source");
    if (h->desc.precision != VISTA_PREC_MIXED) return fail(h, VISTA_E_ARG, "the launch shape tunes the mixed path only");
    if (budget < 0 || reps < 0) return fail(h, VISTA_E_ARG, "budget and reps must be >= 0");
    if (reps == 0) reps = 2;
    const std::vector<SrcHost> queued = h->pending;
    const LaunchCfg start = h->cfg;
    const bool timing_was = h->timing;
    std::vector<LaunchCfg> cand = candidates(start);
    if (budget > 0 && (size_t)budget < cand.size()) cand.resize((size_t)budget);

    double best_ms = -1.0;
    LaunchCfg win = start;
    int rc = VISTA_OK;
    for (const LaunchCfg &c : cand) {
        h->cfg = c;
        double t = -1.0;
        for (int r = 0; r < reps && rc == VISTA_OK; ++r) {
            h->pending = queued;
            rc = vista_enable_timing(h, 1);
            if (rc == VISTA_OK) rc = vista_run(h);
            vista_timing tm{};
            if (rc == VISTA_OK) rc = vista_get_timing(h, &tm);
            if (rc != VISTA_OK) break;
            const double ms = tm.prepass_ms + tm.stack_ms;
            if (t < 0.0 || ms < t) t = ms;
        }
        if (rc != VISTA_OK) break;
        if (best_ms < 0.0 || t < best_ms) {
            best_ms = t;
            win = c;
        }
    }
    // restore the handle: the winning shape, the queue, a zero cube, timing as before
    h->cfg = rc == VISTA_OK ? win : start;
    h->pending = queued;
    drop_graph(h);
    h->plan_valid = false;
    const int rz = vista_zero_cube(h);
    vista_enable_timing(h, timing_was ? 1 : 0);
    if (rc != VISTA_OK) return rc;
    if (rz != VISTA_OK) return rz;
    if (best) {
        best->rows_per_item = win.rows_per_item;
        best->chans_per_lane = win.chans_per_lane;
        best->warps_per_cta = win.warps_per_cta;
        best->sort_rows = win.sort_rows;
        best->prefetch_rows = win.prefetch_rows;
    }
    return VISTA_OK;
}

// The libvista handle and the small host utilities the ABI translation
// units share.
#pragma once
#include <cstdarg>
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "vista.h"
#include "vista_internal.h"

namespace vista {

// A growable device buffer (grows by reallocation, never shrinks).
struct DevBuf {
    void *p = nullptr;
    size_t cap = 0;
    cudaError_t ensure(size_t bytes)
    {
        if (bytes <= cap) return cudaSuccess;
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
        const size_t want = bytes + bytes / 8 + 256;   // headroom against regrowth
        cudaError_t e = cudaMalloc(&p, want);
        if (e == cudaSuccess) cap = want;
        else (void)cudaGetLastError();   // the failure is returned, not left pending
        return e;
    }
    void release()
    {
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
    }
};

struct SrcHost {
    vista_source_desc d;
    std::vector<double> freqs;
    std::vector<int32_t> pol_map;   // npol entries (identity filled in)
    uint64_t freq_digest = 0;       // digest of the frequencies (freq_digest())
    bool has_rot = false;           // re-projected (Eq. 1): cells from rot (u, v, w)
    double rot[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
};

// A device-to-device 2-D copy of a run's device pass (flag repacking).
struct Copy2D {
    void *dst;
    size_t dpitch;
    const void *src;
    size_t spitch, width, height;
};

// A host-to-device copy of a host-memory window's array (whole rows as one
// copy when the pitches allow, else a 2-D copy), into the staging slot of
// its wave.
struct HostCopy {
    int wave;
    void *dst;
    size_t dpitch;
    const void *src;
    size_t spitch, width, height;
};

// One launch class of a run: windows that share the kernel instantiation.
struct ClassRun {
    int key = 0;                    // mixed: (vis_type << 16) | (NS << 8) | npol
    int ns = 1;
    int wave = 0;                   // host-memory runs: the wave of windows the class belongs to
    RunArgs args{};
    std::vector<int> members;       // run-order index of each window
};

struct Span {
    cudaEvent_t a, b;
    int kind;   // 0 prepass, 1 stack, 2 other
};

}  // namespace vista

struct vista_stack {
    vista_cube_desc desc{};
    cudaStream_t stream = nullptr;
    int device = 0;
    bool lattice_fixed = false;
    double f0 = 0.0, df = 0.0;
    std::vector<vista::SrcHost> pending, last;
    void *cube = nullptr;
    double *cube_master = nullptr;   // mixed: FP64 sums moved out of the float4 cube at checkpoints
    uint32_t *count = nullptr;
    int64_t nentries = 0;
    vista::DevStats *stats = nullptr;
    uint64_t host_nvis = 0;   // visibilities read, counted from the channel tables at each run
    uint64_t nvis_since_fold = 0;   // mixed: visibilities stacked since the FP32 partials were last folded
    int32_t *err = nullptr;
    vista::DevBuf b_srcs, b_chf, b_chd, b_recs, b_cells, b_off, b_stage, b_unpack, b_sort, b_rot, b_guvw, b_regrid,
        b_contsub, b_sparse;
    std::vector<vista::ClassRun> classes;
    std::vector<vista::Copy2D> copies;   // device copies of the last planned run
    std::vector<vista::HostCopy> hcopies;   // host-memory windows of the last run, by wave
    int nwaves = 0;                      // waves of host-memory windows of the last run (0: none)
    int64_t wave_bytes = 0;              // staged bytes per wave (0: the library's rule)
    cudaEvent_t slot_ev[2] = {};         // a staging slot's wave has been stacked
    // readback without waiting (vista_read_cube_async): the snapshot in
    // b_unpack is ready (rb_ready), its copy to the host is done (rb_done)
    // pinned host staging of a run's table uploads, two halves used by
    // alternate runs (a copy from pageable memory would wait for the stream,
    // so planning the next run would wait for this one's device work)
    void *pin[2] = {};
    size_t pin_cap[2] = {};
    cudaEvent_t pin_ev[2] = {};
    int pin_half = 0;
    cudaStream_t rb_stream = nullptr;
    cudaEvent_t rb_ready = nullptr, rb_done = nullptr;
    bool rb_pending = false;
    vista::LaunchCfg cfg{64, 1, 4, 1, 4};
    // CUDA-graph replay of the device pass while the source set is unchanged
    bool graphs = true;
    bool plan_valid = false;             // device tables hold the plan of `plan_sig`
    std::vector<uint8_t> plan_sig;
    uint64_t plan_nvis = 0;
    cudaStream_t cap_stream = nullptr;   // capture stream (handle-owned)
    // host<->device copies spread over several streams (copy engines run in
    // parallel), forked from and joined back into `stream`
    cudaStream_t xfer[4] = {};
    cudaEvent_t xfer_ev[5] = {};
    cudaGraphExec_t gexec = nullptr;
    uint64_t graph_launches = 0;
    // stripe geometry of the row ordering (depends on the cube only)
    int32_t stripe_rows = 1, nstripe = 1, ushift = 0, nuk = 1;
    std::string msg;
    bool timing = false;
    std::vector<vista::Span> spans;
    std::vector<cudaEvent_t> ev_pool;
    vista_timing tacc{};
};

namespace vista {

bool handle_live(const vista_stack *h);
int fail(vista_stack *h, int code, const char *fmt, ...) __attribute__((format(printf, 3, 4)));
int cuda_fail(vista_stack *h, cudaError_t e, const char *what);
// A nonzero device error word as a status: 1 a bounded wait gave up
// (E_TIMEOUT), other codes an internal sizing check (E_STATE).
int device_fail(vista_stack *h, int32_t code);
int span_begin(vista_stack *h, int kind);
void span_end(vista_stack *h, int id);
size_t vis_elem_bytes(int vt);
uint64_t freq_digest(const double *f, size_t n);   // change detection of a frequency axis
void drop_graph(vista_stack *h);
constexpr int NXFER = 4;
cudaError_t xfer_fork(vista_stack *h);   // copy streams wait for the work queued on h->stream
cudaError_t xfer_join(vista_stack *h);   // h->stream waits for the copies queued on them

}  // namespace vista

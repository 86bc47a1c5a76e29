// hb_handle.h -- the hb_graph handle (internal: shared by the C-ABI
// implementation and the batched / served forms).
#pragma once

#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "hb_internal.cuh"
#include "hyperball.h"

namespace hb {

// A named range on the host timeline of NVIDIA's profilers (NVTX), for the
// life of the object; costs a check and nothing else when no profiler is
// attached.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// Device allocations owned by a handle, freed together.
struct DevMem {
    std::vector<void *> blocks;
    size_t bytes = 0;
    cudaError_t err = cudaSuccess;
    // With a pool, allocations are stream-ordered on `stream` from that pool
    // (no device-wide synchronisation on free).
    cudaMemPool_t pool = nullptr;
    cudaStream_t stream = nullptr;
    template <class T>
    T *alloc(size_t count) {
        if (err != cudaSuccess) return nullptr;
        void *p = nullptr;
        size_t sz = count * sizeof(T);
        if (sz == 0) sz = 16;
        err = pool ? cudaMallocFromPoolAsync(&p, sz, pool, stream) : cudaMalloc(&p, sz);
        if (err != cudaSuccess) { cudaGetLastError(); return nullptr; }
        blocks.push_back(p);
        bytes += sz;
        return static_cast<T *>(p);
    }
    void free_one(void *p) {
        if (pool) cudaFreeAsync(p, stream);
        else cudaFree(p);
    }
    void release(void *p) {
        for (size_t i = 0; i < blocks.size(); ++i)
            if (blocks[i] == p) { free_one(p); blocks.erase(blocks.begin() + (long)i); return; }
    }
    void free_all() {
        for (void *p : blocks) free_one(p);
        blocks.clear();
    }
};

// The library's device memory pool for the current device (created on
// first use; null if the device cannot make one, and callers then fall
// back to cudaMalloc).  Handles allocate from it in stream order, and
// memory they free stays in it for the next handle until
// hb_trim_memory() returns it: creating and destroying handles costs no
// device-wide synchronisation and no page mapping after the first time.
cudaMemPool_t library_pool();
// Stream-ordered temporary allocation from the library pool (the default
// pool of the device if there is none); free with cudaFreeAsync.
cudaError_t tmp_alloc(void **p, size_t bytes, cudaStream_t s);
template <class T>
cudaError_t tmp_alloc(T **p, size_t bytes, cudaStream_t s) {
    return tmp_alloc(reinterpret_cast<void **>(p), bytes, s);
}

// Host-side services of hb_api.cu used by the other translation units.
hb_status create_handle64(const int64_t *offsets, const int32_t *targets, int64_t n, int64_t m,
                          int log2m, uint64_t seed, const hb_options *opt, hb_graph **out);
// Bring the handle's host bookkeeping (t, convergence) up to date with its
// device counters after kernels launched outside hb_step.
hb_status sync_host_state(hb_graph *g);
// Per-run state: its size, its allocation, and a new run (instance) that
// borrows the read-only set-up of a template handle.
size_t run_bytes(const hb_graph *g);
hb_status setup_run(hb_graph *g);
// The instance's run state comes from `pool` (stream-ordered on s) when
// given, and it reads its counters through `ctr_host` (pinned, owned by the
// caller) when given.
hb_status make_instance(const hb_graph *tmpl, uint64_t seed, cudaStream_t s, hb_graph **out,
                        cudaMemPool_t pool = nullptr, Counters *ctr_host = nullptr);
// Free the per-run state of a handle that serves only as a template.
void drop_run_state(hb_graph *g);
// Re-size the light degree classes of a handle (autotuner).
hb_status retune(hb_graph *g, int aps);
// Candidate class sizings the autotuners try.
constexpr int kTuneAps[] = {1, 2, 4, 8, 16, 32, 64, 128};
// The autotuner times each candidate over the first iterations (most of a
// run's work: the dense ones), up to the fixpoint.
constexpr int kTuneIters = 8;
// Candidate sizes (MiB of counters) of the hot range the autotuner tries:
// for the one-pass gather with L2 priorities, and for the two-phase gather.
constexpr int64_t kTuneHintMiB[] = {32, 64, 96, 128};
constexpr int64_t kTuneHotMiB[] = {64, 128, 192};
// HB_FRONTIER_AUTO pushes when the arcs to push are at most this fraction
// of m (hb_set_frontier_switch changes it per handle).
constexpr double kFrontierSwitch = 0.25;
// Handles made by hb_create, hb_create32 and hb_create_runs with at least
// this many arcs build their reverse lists on a second stream while the
// first iterations, which gather, run (hb_step makes the handle's stream
// wait for them before the first iteration that may push).
constexpr int64_t kDeferReverseArcs = (int64_t)1 << 20;

}  // namespace hb

using namespace hb;

struct hb_graph {
    int64_t n = 0, m = 0;
    int b = 4;
    Layout y{};
    uint64_t seed = 0;
    hb_options opt{};
    cudaStream_t s = nullptr;
    bool fp32 = false, relabel = true, broken = false;
    bool push_union = false;   // frontier iterations push changed counters (reverse CSR)
    int step_grid = 0;
    DevMem mem;
    int64_t *off = nullptr;
    int32_t *tgt = nullptr;
    int64_t *roff = nullptr;
    int32_t *rtgt = nullptr;
    int32_t *perm = nullptr, *inv = nullptr;
    bool own_tgt = true;           // tgt is the library's copy (its lists may be reordered)
    int32_t *hcnt = nullptr;       // two-phase gather: hot arcs at the head of each list
    uint32_t hcnt_hot = 0;         // the hot range hcnt and the list order were made for
    unsigned long long *indeg = nullptr;   // create time only: in-degree of each caller node
    int64_t *wfirst = nullptr;     // Sec. 6: first replica item of each caller node (n+1), or null
    double *disc = nullptr;        // Sec. 7: discounted accumulator (n), or null
    double *ftab = nullptr;        // its discount table
    int gb = 4;                    // log2 of one run's registers (b = gb + lruns: the row)
    int lruns = 0;                 // log2 of the runs per row (hb_create_runs), 0 otherwise
    uint64_t *run_seeds = nullptr; // their seeds (device)
    std::vector<int32_t> run_last; // per run: last iteration in which it changed (-1: none)
    bool track_nf = false;         // HB_NEIGHBOURHOOD: N(t) after every iteration
    bool packed = false;           // HB_PACKED_REGISTERS: rows of 3p/4 bytes, six bits per register
    bool defer_reverse = false;    // reverse lists may be built on rev_s (public creates)
    bool rev_pending = false;      // rev_s may still be writing rtgt; s has not waited for rev_ev
    cudaStream_t rev_s = nullptr;
    cudaEvent_t rev_ev = nullptr;  // recorded on rev_s once rtgt is complete
    double *nf_part = nullptr;     // block partials of the estimate sum
    std::vector<double> nf;        // N(0), N(1), ... of the current run
    Counters *ctr = nullptr;
    Counters *ctr_host = nullptr;
    int64_t seg_count[kSegs] = {0};
    int64_t n_pos = 0;
    int64_t heavy_total = 0;
    StepArgs a{};
    // host bookkeeping
    int32_t t = 0;
    bool converged = false;
    int64_t last_changed = 0, last_nodes = 0, last_arcs = 0, total_arcs = 0;
    int32_t last_sparse = 0;
    int launches = 0;
    bool profile = false;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    int64_t kernel_launches = 0;
    double kernel_ms = 0.0, kernel_bytes = 0.0;
    int64_t push_launches = 0;
    double push_ms = 0.0, push_bytes = 0.0;

    bool own_ctr_host = true;

    ~hb_graph() {
        if (rev_s) cudaStreamSynchronize(rev_s);   // nothing of it outlives the buffers
        if (rev_s) cudaStreamDestroy(rev_s);
        if (rev_ev) cudaEventDestroy(rev_ev);
        for (cudaEvent_t &x : ev)
            if (x) cudaEventDestroy(x);
        if (ctr_host && own_ctr_host) cudaFreeHost(ctr_host);
        mem.free_all();
    }
};

// Bytes of one node's row of counters: p registers, one byte each, or six
// bits each with HB_PACKED_REGISTERS.
inline int64_t row_bytes(const hb_graph *g) {
    const int64_t P = (int64_t)1 << g->b;
    return g->packed ? 3 * P / 4 : P;
}

// Order the handle's stream after the reverse lists' build, if it may still
// run: before anything that reads the reverse lists or rewrites the targets.
inline void wait_reverse(hb_graph *g) {
    if (!g->rev_pending) return;
    cudaStreamWaitEvent(g->s, g->rev_ev, 0);
    g->rev_pending = false;
}

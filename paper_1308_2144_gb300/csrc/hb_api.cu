// hb_api.cu -- the C ABI of include/hyperball.h: argument checks, device
// memory, the create-time pipeline (upload, validate, transpose, degree
// relabelling, reverse CSR, plans, init) and the host side of iterations.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "hb_handle.h"

using namespace hb;

namespace {

thread_local std::string g_err;

hb_status fail(hb_status st, const std::string &msg) {
    g_err = msg;
    return st;
}

hb_status cuda_fail(cudaError_t e, const char *what) {
    return fail(HB_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

bool is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// alpha_p of Flajolet, Fusy, Gandouet & Meunier (2007), the constant of
// Sec. 4.1's size() (Algorithm 1).
double hll_alpha(int p) {
    switch (p) {
        case 16: return 0.673;
        case 32: return 0.697;
        case 64: return 0.709;
        default: return 0.7213 / (1.0 + 1.079 / (double)p);
    }
}

}  // namespace

namespace hb {

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_pool_mu;
cudaMemPool_t g_pools[kMaxDevices] = {};
bool g_pool_tried[kMaxDevices] = {};
}  // namespace

cudaMemPool_t library_pool() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return nullptr;
    }
    std::lock_guard<std::mutex> lock(g_pool_mu);
    if (!g_pool_tried[dev]) {
        g_pool_tried[dev] = true;
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        if (cudaMemPoolCreate(&pool, &props) == cudaSuccess) {
            // keep freed memory for the next handle (hb_trim_memory returns it)
            uint64_t keep = UINT64_MAX;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
            g_pools[dev] = pool;
        } else {
            cudaGetLastError();
        }
    }
    return g_pools[dev];
}

cudaError_t tmp_alloc(void **p, size_t bytes, cudaStream_t s) {
    cudaMemPool_t pool = library_pool();
    return pool ? cudaMallocFromPoolAsync(p, bytes, pool, s) : cudaMallocAsync(p, bytes, s);
}

double hll_alpha_of(int p) { return hll_alpha(p); }
void set_last_error(const char *msg) { g_err = msg ? msg : ""; }
}  // namespace hb

namespace {

void default_opts(hb_options *o) {
    o->flags = 0;
    o->frontier = HB_FRONTIER_AUTO;
    o->max_steps = 1 << 20;
    o->stream = nullptr;
    o->arcs_per_slot = 0;
    o->hot_nodes = 0;
    o->hot_passes = 1;
    o->frontier_switch = 0.0;
}

// The class sizing an options block asks for (0: the default); false if it
// is not one of the candidates.
bool sizing_of(const hb_options &o, int *aps) {
    *aps = o.arcs_per_slot ? o.arcs_per_slot : kArcsPerSlot;
    for (int c : kTuneAps)
        if (c == *aps) return true;
    return false;
}

// The hot range of the two-phase gather for a request of hot_nodes (0:
// one pass): clipped to n; handles of several runs per row gather in one
// pass.
uint32_t hot_window(const hb_graph *g, int64_t hot_nodes) {
    if (g->lruns || hot_nodes <= 0) return 0u;
    return (uint32_t)(hot_nodes < g->n ? hot_nodes : g->n);
}

// Put the hot range of the gather in place.  One pass (passes = 1): the
// gather reads counters [0, hot) with the normal L2 priority and the others
// with evict-first.  Two passes: with the library's own copy of the
// targets, every node's list is reordered hot targets first (once per hot
// range) and the passes split each list at hcnt[v]; with the caller's
// borrowed targets each pass tests every arc.
hb_status apply_hot(hb_graph *g, int64_t hot_nodes, int passes) {
    const uint32_t hot = hot_window(g, hot_nodes);
    g->a.hot = hot;
    g->a.two_pass = passes == 2 ? 1 : 0;
    g->a.hcnt = nullptr;
    if (hot == 0 || passes != 2 || !g->own_tgt) return HB_OK;
    if (g->hcnt_hot != hot) {
        if (!g->hcnt) {
            g->hcnt = g->mem.alloc<int32_t>((size_t)(g->n > 0 ? g->n : 1));
            if (!g->hcnt) return fail(HB_ERR_OOM, "out of device memory (hot counts)");
        }
        g->hcnt_hot = 0;
        wait_reverse(g);   // the reverse lists' build reads the lists reordered here
        cudaError_t e = partition_hot(g->off, g->tgt, g->n, g->m, hot, g->hcnt, g->s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(g->s);
        if (e != cudaSuccess) {
            g->a.hot = 0;
            return e == cudaErrorMemoryAllocation ? fail(HB_ERR_OOM, "out of device memory (hot partition)")
                                                   : cuda_fail(e, "hot partition");
        }
        g->hcnt_hot = hot;
    }
    g->a.hcnt = g->hcnt;
    return HB_OK;
}

// Copy `bytes` from a host or device source into device memory.
cudaError_t to_device(void *dst, const void *src, size_t bytes, cudaStream_t s) {
    if (bytes == 0) return cudaSuccess;
    return cudaMemcpyAsync(dst, src, bytes, is_device_ptr(src) ? cudaMemcpyDeviceToDevice
                                                               : cudaMemcpyHostToDevice, s);
}

// Host targets to the device in chunks on s, each chunk checked against
// [0, n) (and its in-arcs counted into indeg, when not null) on a second
// stream as soon as it has arrived, so that the checks run under the copy;
// s waits for the checks at the end.
cudaError_t upload_checked(int32_t *dst, const int32_t *src, int64_t m, int64_t n, unsigned long long *err,
                           unsigned long long *indeg, cudaStream_t s) {
    constexpr int K = 8;
    cudaStream_t side = nullptr;
    cudaEvent_t ev[K + 1] = {};
    cudaError_t e = cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking);
    for (int k = 0; e == cudaSuccess && k <= K; ++k) e = cudaEventCreateWithFlags(&ev[k], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(ev[K], s);   // the buffers' allocation and clearing
    if (e == cudaSuccess) e = cudaStreamWaitEvent(side, ev[K], 0);
    const int64_t step = (m + K - 1) / K;
    for (int k = 0; e == cudaSuccess && k < K; ++k) {
        const int64_t c0 = k * step, c1 = c0 + step < m ? c0 + step : m;
        if (c0 >= c1) break;
        e = cudaMemcpyAsync(dst + c0, src + c0, sizeof(int32_t) * (c1 - c0), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaEventRecord(ev[k], s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(side, ev[k], 0);
        if (e == cudaSuccess) e = check_targets(dst + c0, c1 - c0, n, err, indeg, side);
    }
    if (e == cudaSuccess) e = cudaEventRecord(ev[K], side);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev[K], 0);
    if (e != cudaSuccess && side) cudaStreamSynchronize(side);   // nothing of it outlives the buffers
    for (cudaEvent_t x : ev)
        if (x) cudaEventDestroy(x);
    if (side) cudaStreamDestroy(side);
    return e;
}
// Targets from host memory at least this long are uploaded by upload_checked.
constexpr int64_t kCheckedUploadMin = (int64_t)1 << 23;

// Deliver a device result into a caller buffer (host or device).
cudaError_t to_caller(void *dst, const void *src, size_t bytes, cudaStream_t s) {
    if (bytes == 0 || !dst) return cudaSuccess;
    return cudaMemcpyAsync(dst, src, bytes, is_device_ptr(dst) ? cudaMemcpyDeviceToDevice
                                                               : cudaMemcpyDeviceToHost, s);
}

// Shared set-up of a graph for one log2m, once the scanned CSR (g->off,
// g->tgt) is in place: degree segments, heavy chunks, reverse CSR,
// estimator tables, the dense plan and the launch shape.  Everything here
// is read-only during iterations, so several runs (different seeds) can
// share it.
hb_status setup_shared(hb_graph *g) {
    cudaStream_t s = g->s;
    const int64_t n = g->n, m = g->m;
    const int P = 1 << g->b;     // bytes of a row
    const int Pe = 1 << g->gb;   // registers of one run: the estimator's p
    cudaError_t e = count_degree_segments(g->off, n, g->y, g->seg_count, s);
    if (e != cudaSuccess) return cuda_fail(e, "degree segments");
    int64_t seg_begin[kSegs];
    int64_t run = 0;
    for (int k = 0; k < kSegs; ++k) { seg_begin[k] = run; run += g->seg_count[k]; }
    g->n_pos = run;
    e = heavy_chunk_total(g->off, n, g->y, &g->heavy_total, s);
    if (e != cudaSuccess) return cuda_fail(e, "heavy chunks");

    const bool want_reverse = g->opt.frontier == HB_FRONTIER_AUTO || g->opt.frontier == HB_FRONTIER_PUSH;
    DevMem &M = g->mem;
    if (want_reverse) {
        g->roff = M.alloc<int64_t>(n + 1);
        g->rtgt = M.alloc<int32_t>(m);
        if (M.err != cudaSuccess) return fail(HB_ERR_OOM, "out of device memory (reverse CSR)");
        // large graphs of single-graph handles: the targets' scatter on a
        // second stream, under the first (gathered) iterations
        bool defer = g->defer_reverse && m >= kDeferReverseArcs;
        if (defer && !g->rev_s &&
            (cudaStreamCreateWithFlags(&g->rev_s, cudaStreamNonBlocking) != cudaSuccess ||
             cudaEventCreateWithFlags(&g->rev_ev, cudaEventDisableTiming) != cudaSuccess)) {
            cudaGetLastError();
            defer = false;
        }
        cudaStream_t xs = defer ? g->rev_s : nullptr;
        cudaEvent_t xe = defer ? g->rev_ev : nullptr;
        e = g->indeg ? transpose_csr_counted(g->off, g->tgt, n, m, g->indeg, g->perm, g->roff, g->rtgt, s, xs, xe)
                     : transpose_csr(g->off, g->tgt, n, m, g->roff, g->rtgt, s, xs, xe);
        if (e != cudaSuccess) return cuda_fail(e, "reverse CSR");
        g->rev_pending = defer;
    }
    StepArgs &a = g->a;
    a = StepArgs{};
    a.off = g->off;
    a.tgt = g->tgt;
    a.roff = g->roff;
    a.rtgt = g->rtgt;
    a.has_reverse = want_reverse ? 1 : 0;
    a.packed = g->packed ? 1 : 0;
    g->push_union = want_reverse && (g->opt.flags & HB_PULL_GATHER) == 0;
    a.push_union = g->push_union ? 1 : 0;
    a.plan_dense = M.alloc<Plan>(1);
    a.owner_dense = M.alloc<int32_t>(g->heavy_total);
    a.cstart_dense = M.alloc<int64_t>(g->seg_count[0] + 1);
    double *lc64 = M.alloc<double>(Pe + 1);
    float *lc32 = M.alloc<float>(Pe + 1);
    a.lc64 = lc64;
    a.lc32 = lc32;
    int32_t *dense_list = nullptr;
    if (!g->relabel) dense_list = M.alloc<int32_t>(g->n_pos);
    if (g->track_nf) g->nf_part = M.alloc<double>(kNfBlocks);
    if (M.err != cudaSuccess) return fail(HB_ERR_OOM, "out of device memory (HyperBall tables)");

    const double alpha = hll_alpha(Pe);
    a.c64 = std::ldexp(alpha * (double)Pe * (double)Pe, 64 - g->gb);
    a.c32 = (float)a.c64;
    // small-range switch: raw estimate <= 5p/2  <=>  X >= alpha 2^64 * 2/5
    const unsigned __int128 Y = (unsigned __int128)std::ldexp(alpha, 64);
    a.thr_x = (unsigned long long)((2 * Y + 4) / 5);
    a.n = n;
    a.n_pos = g->n_pos;
    a.m = m;
    for (int k = 0; k < kSegs; ++k) {
        a.seg_begin[k] = seg_begin[k];
        a.seg_lo[k] = g->y.lo[k];
        a.seg_hi[k] = g->y.hi[k];
    }
    a.b = g->b;
    a.gb = g->gb;
    a.lruns = g->lruns;
    a.run_seeds = g->run_seeds;
    a.aps = g->y.aps;
    a.frontier = g->opt.frontier;
    a.sparse_frac = g->opt.frontier_switch > 0.0 ? g->opt.frontier_switch : kFrontierSwitch;
    a.hot = 0;   // the hot range is put in place after set-up (apply_hot)
    if (dense_list) {
        int64_t *sb_dev = M.alloc<int64_t>(kSegs);
        unsigned long long *fill = M.alloc<unsigned long long>(kSegs);
        if (M.err != cudaSuccess) return fail(HB_ERR_OOM, "out of device memory (dense list)");
        e = cudaMemcpyAsync(sb_dev, seg_begin, sizeof(seg_begin), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = build_dense_list(g->off, n, g->y, sb_dev, dense_list, fill, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "dense list");
        M.release(sb_dev);
        M.release(fill);
    }
    a.dense_list = dense_list;
    e = launch_lc_tables(lc64, lc32, Pe, s);
    if (e != cudaSuccess) return cuda_fail(e, "estimator tables");
    e = launch_dense_plan(a, g->y, g->seg_count, const_cast<Plan *>(a.plan_dense),
                          const_cast<int32_t *>(a.owner_dense), const_cast<int64_t *>(a.cstart_dense), s);
    if (e != cudaSuccess) return cuda_fail(e, "dense plan");
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    g->step_grid = sms * (g->lruns ? runs_step_blocks_per_sm(g->b, g->fp32) : step_blocks_per_sm(g->b, g->fp32));
    return HB_OK;
}

hb_status init_state(hb_graph *g, uint64_t seed);

}  // namespace

namespace hb {

// Bytes of the per-run state of a graph (counters, accumulators, flags,
// lists, frontier plan, heavy-chunk scratch), carved from one allocation.
size_t run_bytes(const hb_graph *g) {
    const int64_t n = g->n, m = g->m, P = (int64_t)1 << g->b;
    const int64_t big_cap = (m / kBigRdeg + 1) < n ? (m / kBigRdeg + 1) : (n > 0 ? n : 1);
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    size_t b = 0;
    const int64_t nr = n << g->lruns;   // (node, run) pairs
    b += 2 * up((size_t)n * row_bytes(g));
    b += 2 * up(sizeof(double) * nr);
    b += up((g->fp32 ? sizeof(float) : sizeof(double)) * nr);
    b += up((size_t)n);
    b += up(sizeof(uint32_t) * ((n + 31) / 32 + 1));
    b += 2 * up(sizeof(int32_t) * n) + 2 * up(sizeof(int32_t) * big_cap);
    b += up(sizeof(int32_t) * g->n_pos);
    b += up(sizeof(Plan)) + up(sizeof(int32_t) * g->heavy_total) + up(sizeof(int64_t) * (g->seg_count[0] + 1));
    b += up((size_t)g->heavy_total * P) + up(sizeof(uint32_t) * (g->seg_count[0] + 1));
    b += up(sizeof(Counters));
    return b;
}

// Per-run state of a graph whose shared set-up (g->a's shared fields) is
// done: one device allocation, carved.
hb_status setup_run(hb_graph *g) {
    const int64_t n = g->n, m = g->m, P = (int64_t)1 << g->b;
    const int64_t big_cap = (m / kBigRdeg + 1) < n ? (m / kBigRdeg + 1) : (n > 0 ? n : 1);
    const size_t total = run_bytes(g);
    uint8_t *base = g->mem.alloc<uint8_t>(total);
    if (!base) return fail(HB_ERR_OOM, "out of device memory (HyperBall state: " + std::to_string(total) + " bytes)");
    size_t off = 0;
    auto take = [&](size_t bytes) { uint8_t *p = base + off; off += (bytes + 255) & ~(size_t)255; return p; };
    StepArgs &a = g->a;
    a.regs[0] = take((size_t)n * row_bytes(g));
    a.regs[1] = take((size_t)n * row_bytes(g));
    const int64_t nr = n << g->lruns;
    a.sumd = reinterpret_cast<double *>(take(sizeof(double) * nr));
    a.harm = reinterpret_cast<double *>(take(sizeof(double) * nr));
    a.ecache = take((g->fp32 ? sizeof(float) : sizeof(double)) * nr);
    a.changed = take((size_t)n);
    a.mustbits = reinterpret_cast<uint32_t *>(take(sizeof(uint32_t) * ((n + 31) / 32 + 1)));
    a.clist[0] = reinterpret_cast<int32_t *>(take(sizeof(int32_t) * n));
    a.clist[1] = reinterpret_cast<int32_t *>(take(sizeof(int32_t) * n));
    a.biglist[0] = reinterpret_cast<int32_t *>(take(sizeof(int32_t) * big_cap));
    a.biglist[1] = reinterpret_cast<int32_t *>(take(sizeof(int32_t) * big_cap));
    a.slist = reinterpret_cast<int32_t *>(take(sizeof(int32_t) * g->n_pos));
    a.plan_sparse = reinterpret_cast<Plan *>(take(sizeof(Plan)));
    a.owner_sparse = reinterpret_cast<int32_t *>(take(sizeof(int32_t) * g->heavy_total));
    a.cstart_sparse = reinterpret_cast<int64_t *>(take(sizeof(int64_t) * (g->seg_count[0] + 1)));
    a.partial = take((size_t)g->heavy_total * P);
    a.arrive = reinterpret_cast<uint32_t *>(take(sizeof(uint32_t) * (g->seg_count[0] + 1)));
    g->ctr = reinterpret_cast<Counters *>(take(sizeof(Counters)));
    a.ctr = g->ctr;
    if (!g->ctr_host && cudaMallocHost(&g->ctr_host, sizeof(Counters)) != cudaSuccess)
        return fail(HB_ERR_OOM, "out of pinned host memory");
    cudaError_t e = cudaMemsetAsync(a.arrive, 0, sizeof(uint32_t) * (g->seg_count[0] + 1), g->s);
    if (e == cudaSuccess) e = cudaMemsetAsync(a.changed, 0, (size_t)(n > 0 ? n : 1), g->s);
    if (e != cudaSuccess) return cuda_fail(e, "run state");
    return HB_OK;
}

void drop_run_state(hb_graph *g) {
    if (g->a.regs[0]) g->mem.release(g->a.regs[0]);   // the carved per-run block starts there
    StepArgs &a = g->a;
    a.regs[0] = a.regs[1] = nullptr;
    a.sumd = a.harm = nullptr;
    a.ecache = nullptr;
    a.changed = nullptr;
    a.mustbits = nullptr;
    a.clist[0] = a.clist[1] = a.biglist[0] = a.biglist[1] = a.slist = nullptr;
    a.plan_sparse = nullptr;
    a.owner_sparse = nullptr;
    a.cstart_sparse = nullptr;
    a.partial = nullptr;
    a.arrive = nullptr;
    a.ctr = g->ctr = nullptr;
}

// Re-size the light degree classes (arcs per slot), keeping every read-only
// array that does not depend on it: segments, the dense list of an
// unrelabelled graph and the dense plan are rebuilt.
hb_status retune(hb_graph *g, int aps) {
    cudaStream_t s = g->s;
    const int64_t n = g->n;
    g->y = make_layout(g->b, aps);
    cudaError_t e = count_degree_segments(g->off, n, g->y, g->seg_count, s);
    if (e != cudaSuccess) return cuda_fail(e, "degree segments");
    int64_t seg_begin[kSegs], run = 0;
    for (int k = 0; k < kSegs; ++k) { seg_begin[k] = run; run += g->seg_count[k]; }
    StepArgs &a = g->a;
    for (int k = 0; k < kSegs; ++k) {
        a.seg_begin[k] = seg_begin[k];
        a.seg_lo[k] = g->y.lo[k];
        a.seg_hi[k] = g->y.hi[k];
    }
    a.aps = aps;
    if (a.dense_list) {
        int64_t *sb_dev = nullptr;
        unsigned long long *fill = nullptr;
        e = tmp_alloc(&sb_dev, sizeof(seg_begin), s);
        if (e == cudaSuccess) e = tmp_alloc(&fill, sizeof(unsigned long long) * kSegs, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(sb_dev, seg_begin, sizeof(seg_begin), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess)
            e = build_dense_list(g->off, n, g->y, sb_dev, const_cast<int32_t *>(a.dense_list), fill, s);
        cudaFreeAsync(sb_dev, s);
        cudaFreeAsync(fill, s);
        if (e != cudaSuccess) return cuda_fail(e, "dense list");
    }
    e = launch_dense_plan(a, g->y, g->seg_count, const_cast<Plan *>(a.plan_dense),
                          const_cast<int32_t *>(a.owner_dense), const_cast<int64_t *>(a.cstart_dense), s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "dense plan");
    return HB_OK;
}

// A new run on the shared set-up of `tmpl` (same graph and log2m): the
// instance borrows the template's read-only arrays, owns only its per-run
// state, and starts from the counters of `seed`.
hb_status make_instance(const hb_graph *tmpl, uint64_t seed, cudaStream_t s, hb_graph **out,
                        cudaMemPool_t pool, Counters *ctr_host) {
    hb_graph *g = new hb_graph();
    g->mem.pool = pool ? pool : library_pool();
    g->mem.stream = s;
    if (ctr_host) {
        g->ctr_host = ctr_host;
        g->own_ctr_host = false;
    }
    g->n = tmpl->n; g->m = tmpl->m; g->b = tmpl->b; g->y = tmpl->y;
    g->gb = tmpl->gb; g->lruns = tmpl->lruns; g->run_seeds = tmpl->run_seeds;
    g->opt = tmpl->opt;
    g->s = s;
    g->fp32 = tmpl->fp32; g->relabel = tmpl->relabel; g->push_union = tmpl->push_union;
    g->step_grid = tmpl->step_grid;
    g->off = tmpl->off; g->tgt = tmpl->tgt; g->roff = tmpl->roff; g->rtgt = tmpl->rtgt;
    g->perm = tmpl->perm; g->inv = tmpl->inv;
    for (int k = 0; k < kSegs; ++k) g->seg_count[k] = tmpl->seg_count[k];
    g->n_pos = tmpl->n_pos;
    g->heavy_total = tmpl->heavy_total;
    g->a = tmpl->a;
    g->a.disc = nullptr;   // weights and discounts belong to single-graph handles
    g->a.ftab = nullptr;
    g->a.flen = 0;
    hb_status st = setup_run(g);
    if (st == HB_OK) st = init_state(g, seed);
    if (st != HB_OK) { delete g; return st; }
    *out = g;
    return HB_OK;
}

}  // namespace hb

namespace {

hb_status finish_setup(hb_graph *g) {
    hb_status st = setup_shared(g);
    return st == HB_OK ? setup_run(g) : st;
}

hb_status init_state(hb_graph *g, uint64_t seed) {
    NvtxRange nv("init");
    g->seed = seed;
    cudaError_t e = launch_init(g->a, g->perm, seed, g->fp32, g->s, g->wfirst);
    g->launches += g->n > 0 ? 2 : 1;
    if (e == cudaSuccess && g->track_nf) {
        e = launch_estimate_sum(g->a.ecache, g->fp32, g->n, g->nf_part, g->ctr, g->s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(g->ctr_host, g->ctr, sizeof(Counters), cudaMemcpyDeviceToHost, g->s);
        g->launches += 2;
    }
    g->kernel_launches = 0;
    g->kernel_ms = g->kernel_bytes = 0.0;
    g->push_launches = 0;
    g->push_ms = g->push_bytes = 0.0;
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->s);
    if (e != cudaSuccess) return cuda_fail(e, "init");
    g->t = 0;
    g->converged = false;
    g->last_changed = g->last_nodes = g->last_arcs = g->total_arcs = 0;
    g->last_sparse = 0;
    g->nf.clear();
    if (g->track_nf) g->nf.push_back(g->ctr_host->nsum);
    g->run_last.assign(g->lruns ? (size_t)1 << g->lruns : 0, -1);
    return HB_OK;
}

// lruns > 0: 2^lruns runs of one graph per row (hb_create_runs), run r
// hashed with seeds[r] (host or device memory).  defer_reverse: the
// handle's own iterations may start before its reverse lists are complete
// (single-graph handles; templates of batches and servers are complete on
// return).
template <class OffT>
hb_status create_impl(const OffT *offsets, const int32_t *targets, int64_t n, int64_t m, int log2m,
                      uint64_t seed, const hb_options *opt, hb_graph **out, int lruns = 0,
                      const uint64_t *seeds = nullptr, bool defer_reverse = false) {
    if (!out) return fail(HB_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (log2m < kMinLog2m || log2m > kMaxLog2m)
        return fail(HB_ERR_INVALID, "log2m must lie in [4, 12]");
    if (n < 0 || n >= (int64_t)1 << 31) return fail(HB_ERR_INVALID, "n must lie in [0, 2^31)");
    if (m < 0 || (sizeof(OffT) == 4 && m >= (int64_t)1 << 31))
        return fail(HB_ERR_INVALID, "m out of range for the offset type");
    if (!offsets) return fail(HB_ERR_INVALID, "offsets is NULL");
    if (m > 0 && !targets) return fail(HB_ERR_INVALID, "targets is NULL");
    hb_options o;
    if (opt) o = *opt; else default_opts(&o);
    if (o.max_steps <= 0) o.max_steps = 1 << 20;
    if (o.frontier < HB_FRONTIER_AUTO || o.frontier > HB_FRONTIER_OFF)
        return fail(HB_ERR_INVALID, "unknown frontier policy");
    int aps = 0;
    if (!sizing_of(o, &aps)) return fail(HB_ERR_INVALID, "arcs_per_slot must be 0 or a power of two from 1 to 128");
    if (o.hot_nodes < 0) return fail(HB_ERR_INVALID, "hot_nodes must be >= 0");
    if (o.hot_passes < 0 || o.hot_passes > 2) return fail(HB_ERR_INVALID, "hot_passes must be 0, 1 or 2");
    if (!(o.frontier_switch >= 0.0) || !std::isfinite(o.frontier_switch))
        return fail(HB_ERR_INVALID, "frontier_switch must be 0 (the default) or a finite positive fraction");
    if (o.flags & HB_PACKED_REGISTERS) {
        if (o.frontier != HB_FRONTIER_OFF)
            return fail(HB_ERR_INVALID, "HB_PACKED_REGISTERS needs the frontier policy HB_FRONTIER_OFF");
        if (lruns) return fail(HB_ERR_INVALID, "HB_PACKED_REGISTERS is for handles of one run");
        if (o.hot_nodes) return fail(HB_ERR_INVALID, "HB_PACKED_REGISTERS takes no hot range");
    }
    cudaError_t e = cudaFree(nullptr);   // make sure a context exists
    if (e != cudaSuccess) return cuda_fail(e, "CUDA context");

    hb_graph *g = new hb_graph();
    g->n = n;
    g->m = m;
    g->b = log2m + lruns;
    g->gb = log2m;
    g->lruns = lruns;
    g->y = make_layout(g->b, aps);
    g->opt = o;
    g->s = static_cast<cudaStream_t>(o.stream);
    g->fp32 = (o.flags & HB_FP32_ESTIMATE) != 0;
    g->relabel = (o.flags & HB_NO_RELABEL) == 0;
    g->profile = (o.flags & HB_PROFILE) != 0;
    g->track_nf = (o.flags & HB_NEIGHBOURHOOD) != 0;
    g->defer_reverse = defer_reverse;
    g->packed = (o.flags & HB_PACKED_REGISTERS) != 0;
    if (g->profile) {
        for (cudaEvent_t &x : g->ev)
            if (cudaEventCreate(&x) != cudaSuccess) {
                delete g;
                return fail(HB_ERR_CUDA, "cannot create profiling events");
            }
    }
    cudaStream_t s = g->s;
    DevMem &M = g->mem;
    M.pool = library_pool();
    M.stream = s;
    if (lruns) {
        g->run_seeds = M.alloc<uint64_t>((size_t)1 << lruns);
        if (!g->run_seeds) { delete g; return fail(HB_ERR_OOM, "out of device memory (run seeds)"); }
        e = to_device(g->run_seeds, seeds, sizeof(uint64_t) << lruns, s);
        if (e != cudaSuccess) { delete g; return cuda_fail(e, "run seeds"); }
    }

    NvtxRange nv_create("hb_create");
    // 1. input CSR on the device (int64 offsets), the targets checked as
    // they arrive; when the graph given is the one scanned, the degree
    // sort's key (every node's in-degree) is counted by the same pass
    const bool borrow = (o.flags & HB_BORROW_DEVICE_PTRS) != 0;
    const bool off_dev = is_device_ptr(offsets), tgt_dev = m == 0 || is_device_ptr(targets);
    const bool pre_count = g->relabel && (o.flags & HB_TRANSPOSE) == 0 && n > 0 && m > 0;
    unsigned long long *err_dev = M.alloc<unsigned long long>(1);
    if (pre_count) g->indeg = M.alloc<unsigned long long>(n);
    if (M.err != cudaSuccess) { delete g; return fail(HB_ERR_OOM, "out of device memory"); }
    cudaMemsetAsync(err_dev, 0, sizeof(unsigned long long), s);
    if (pre_count) cudaMemsetAsync(g->indeg, 0, sizeof(unsigned long long) * n, s);
    bool checked = false;
    int64_t *in_off = nullptr;
    int32_t *in_tgt = nullptr;
    bool own_in_off = true, own_in_tgt = true;
    if (sizeof(OffT) == 8 && borrow && off_dev) {
        in_off = const_cast<int64_t *>(reinterpret_cast<const int64_t *>(offsets));
        own_in_off = false;
    } else {
        in_off = M.alloc<int64_t>(n + 1);
        if (sizeof(OffT) == 4) {
            int32_t *tmp = M.alloc<int32_t>(n + 1);
            if (M.err == cudaSuccess) {
                e = to_device(tmp, offsets, sizeof(int32_t) * (n + 1), s);
                if (e == cudaSuccess) e = widen_offsets(tmp, in_off, n + 1, s);
                M.release(tmp);
            }
        } else if (M.err == cudaSuccess) {
            e = to_device(in_off, offsets, sizeof(int64_t) * (n + 1), s);
        }
    }
    if (borrow && tgt_dev) {
        in_tgt = const_cast<int32_t *>(targets);
        own_in_tgt = false;
    } else {
        in_tgt = M.alloc<int32_t>(m);
        if (M.err == cudaSuccess && e == cudaSuccess) {
            if (!tgt_dev && m >= kCheckedUploadMin) {
                e = upload_checked(in_tgt, targets, m, n, err_dev, g->indeg, s);
                checked = true;
            } else {
                e = to_device(in_tgt, targets, sizeof(int32_t) * m, s);
            }
        }
    }
    if (M.err != cudaSuccess) { delete g; return fail(HB_ERR_OOM, "out of device memory (graph)"); }
    if (e != cudaSuccess) { delete g; return cuda_fail(e, "graph upload"); }

    // 2. validation
    unsigned long long err_host = 0;
    {
        NvtxRange nv("validate");
        e = validate_offsets(in_off, n, m, err_dev, s);
        if (e == cudaSuccess && !checked) e = check_targets(in_tgt, m, n, err_dev, g->indeg, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&err_host, err_dev, sizeof(err_host), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    M.release(err_dev);
    if (e != cudaSuccess) { delete g; return cuda_fail(e, "validation"); }
    if (err_host) {
        delete g;
        std::string why;
        if (err_host & 1) why += " offsets[0] != 0;";
        if (err_host & 2) why += " offsets[n] != m;";
        if (err_host & 4) why += " offsets decrease;";
        if (err_host & 8) why += " a target lies outside [0, n);";
        return fail(HB_ERR_INVALID, "malformed CSR:" + why);
    }

    // 3. transpose on request (Sec. 5: the in-centralities scan G^T)
    if (o.flags & HB_TRANSPOSE) {
        int64_t *toff = M.alloc<int64_t>(n + 1);
        int32_t *ttgt = M.alloc<int32_t>(m);
        if (M.err != cudaSuccess) { delete g; return fail(HB_ERR_OOM, "out of device memory (transpose)"); }
        e = transpose_csr(in_off, in_tgt, n, m, toff, ttgt, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) { delete g; return cuda_fail(e, "transpose"); }
        if (own_in_off) M.release(in_off);
        if (own_in_tgt) M.release(in_tgt);
        in_off = toff; in_tgt = ttgt; own_in_off = own_in_tgt = true;
    }

    // 4. degree-sorted relabelling
    if (g->relabel) {
        NvtxRange nv("relabel");
        g->perm = M.alloc<int32_t>(n);
        g->inv = M.alloc<int32_t>(n);
        int64_t *noff = M.alloc<int64_t>(n + 1);
        int32_t *ntgt = M.alloc<int32_t>(m);
        if (!g->indeg) g->indeg = M.alloc<unsigned long long>(n);
        if (M.err != cudaSuccess) { delete g; return fail(HB_ERR_OOM, "out of device memory (relabel)"); }
        e = degree_sort_counted(in_off, in_tgt, n, m, g->perm, g->inv, g->indeg, pre_count, s);
        if (e == cudaSuccess) e = relabel_csr(in_off, in_tgt, n, m, g->perm, g->inv, noff, ntgt, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) { delete g; return cuda_fail(e, "relabel"); }
        if (own_in_off) M.release(in_off);
        if (own_in_tgt) M.release(in_tgt);
        g->off = noff;
        g->tgt = ntgt;
    } else {
        g->off = in_off;
        g->tgt = in_tgt;
        g->own_tgt = own_in_tgt;
    }

    hb_status st;
    {
        NvtxRange nv("setup");
        st = finish_setup(g);
    }
    if (st == HB_OK && o.hot_nodes > 0) st = apply_hot(g, o.hot_nodes, o.hot_passes);
    if (g->indeg) M.release(g->indeg);
    g->indeg = nullptr;
    if (st == HB_OK) st = init_state(g, seed);
    if (st != HB_OK) { delete g; return st; }
    *out = g;
    return HB_OK;
}

}  // namespace

namespace hb {

hb_status create_handle64(const int64_t *offsets, const int32_t *targets, int64_t n, int64_t m,
                          int log2m, uint64_t seed, const hb_options *opt, hb_graph **out) {
    return create_impl<int64_t>(offsets, targets, n, m, log2m, seed, opt, out);
}

hb_status sync_host_state(hb_graph *g) {
    cudaError_t e = cudaMemcpyAsync(g->ctr_host, g->ctr, sizeof(Counters), cudaMemcpyDeviceToHost, g->s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->s);
    if (e != cudaSuccess) return cuda_fail(e, "device counters");
    g->t = g->ctr_host->steps_done;
    g->converged = g->ctr_host->converged != 0;
    g->last_changed = (int64_t)g->ctr_host->n_changed;
    return HB_OK;
}

}  // namespace hb

namespace {

// Temporary device buffers of a call on handle g: from the library pool, on
// the handle's stream (freed into the pool when the call returns).
DevMem scratch(const hb_graph *g) {
    DevMem d;
    d.pool = library_pool();
    d.stream = g->s;
    return d;
}

hb_status check(hb_graph *g) {
    if (!g) return fail(HB_ERR_INVALID, "handle is NULL");
    if (g->broken) return fail(HB_ERR_STATE, "handle unusable after a CUDA error");
    return HB_OK;
}

const uint8_t *current_regs(hb_graph *g) { return g->a.regs[g->t & 1]; }

// Whether the next iteration may push (and so read the reverse lists): the
// test that starts every iteration on the device, made here on the counters
// of the iteration before, with a margin so that the answer errs towards
// yes.  The first iteration of a computation always gathers.
bool may_push(const hb_graph *g) {
    if (g->t == 0) return false;
    if (g->a.frontier == HB_FRONTIER_PUSH) return true;
    if (g->a.frontier != HB_FRONTIER_AUTO) return false;
    return (double)g->ctr_host->push_arcs <= g->a.sparse_frac * (double)g->m * (1.0 + 1e-9) + 1.0;
}

}  // namespace

extern "C" {

void hb_default_options(hb_options *opt) {
    if (opt) default_opts(opt);
}

hb_status hb_create(const int64_t *offsets, const int32_t *targets, int64_t n, int64_t m, int log2m,
                    uint64_t seed, const hb_options *opt, hb_graph **out) {
    g_err.clear();
    return create_impl<int64_t>(offsets, targets, n, m, log2m, seed, opt, out, 0, nullptr, true);
}

hb_status hb_create32(const int32_t *offsets, const int32_t *targets, int64_t n, int64_t m, int log2m,
                      uint64_t seed, const hb_options *opt, hb_graph **out) {
    g_err.clear();
    return create_impl<int32_t>(offsets, targets, n, m, log2m, seed, opt, out, 0, nullptr, true);
}

hb_status hb_step(hb_graph *g, int64_t *n_changed) {
    hb_status st = check(g);
    if (st != HB_OK) return st;
    NvtxRange nv("hb_step");
    if (g->rev_pending && may_push(g)) wait_reverse(g);
    cudaError_t e = launch_iteration(g->a, g->y, g->fp32, g->step_grid, g->s, g->profile ? g->ev : nullptr,
                                     &g->launches);
    if (e == cudaSuccess && g->track_nf) {
        e = launch_estimate_sum(g->a.ecache, g->fp32, g->n, g->nf_part, g->ctr, g->s);
        g->launches += 2;
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(g->ctr_host, g->ctr, sizeof(Counters), cudaMemcpyDeviceToHost, g->s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->s);
    if (e != cudaSuccess) {
        g->broken = true;
        return cuda_fail(e, "step");
    }
    const Counters &c = *g->ctr_host;
    if (c.err) {
        g->broken = true;
        std::string why = "a device-side check failed during the step:";
        if (c.err & kErrCasBound) why += " the pushed union's compare-and-swap loop reached its bound;";
        if (c.err & kErrTarget) why += " an arc target lies outside [0, n) (debug build check);";
        return fail(HB_ERR_STATE, why);
    }
    g->t = c.steps_done;
    g->last_changed = (int64_t)c.n_changed;
    g->last_sparse = c.mode;
    if (g->track_nf) g->nf.push_back(c.nsum);
    for (size_t r = 0; r < g->run_last.size(); ++r)
        if ((c.run_mask >> r) & 1ULL) g->run_last[r] = c.steps_done - 1;
    if (c.mode == 1) {
        int64_t nodes = 0;
        for (int k = 0; k < kSegs; ++k) nodes += (int64_t)c.fill[k];
        g->last_nodes = nodes;
        g->last_arcs = (int64_t)c.arcs;
    } else {
        g->last_nodes = g->n_pos;
        g->last_arcs = g->m;
    }
    g->total_arcs += g->last_arcs;
    if (c.n_changed == 0) g->converged = true;
    const bool pushed = c.mode == 1 && g->push_union;
    if (g->profile && pushed) {
        // pushed union: P arcs into the C' nodes changed last time, K nodes
        // recomputed, C changed
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, g->ev[2], g->ev[3]) == cudaSuccess) {
            const double p = (double)(1 << g->b);
            const double esz = g->fp32 ? 4.0 : 8.0;
            g->push_ms += ms;
            g->push_launches += 1;
            g->push_bytes += (double)c.arcs * (4.0 + 2.0 * p) + (double)c.prev_list_len * (8.0 + p) +
                             (double)g->last_nodes * (5.0 + 3.0 * p) +
                             (double)c.n_changed * (4.0 + 32.0 + 2.0 * esz);
        }
    } else if (g->profile) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, g->ev[0], g->ev[1]) == cudaSuccess) {
            const double p = (double)row_bytes(g);   // bytes of a counter
            const double esz = g->fp32 ? 4.0 : 8.0;
            g->kernel_ms += ms;
            g->kernel_launches += 1;
            g->kernel_bytes += (double)g->last_arcs * (4.0 + p) +
                               (double)g->last_nodes * (8.0 + 2.0 * p + 1.0 + (c.mode == 1 ? 4.0 : 0.0)) +
                               (double)c.n_changed * (4.0 + 32.0 + 2.0 * esz);
        }
    }
    if (n_changed) *n_changed = (int64_t)c.n_changed;
    return HB_OK;
}

hb_status hb_run_to_fixpoint(hb_graph *g, int32_t *steps) {
    hb_status st = check(g);
    if (st != HB_OK) return st;
    NvtxRange nv("hb_run_to_fixpoint");
    while (!g->converged && g->t < g->opt.max_steps) {
        st = hb_step(g, nullptr);
        if (st != HB_OK) return st;
    }
    if (steps) *steps = g->t;
    if (!g->converged) return fail(HB_ERR_NOT_CONVERGED, "max_steps reached before the fixpoint");
    return HB_OK;
}

hb_status hb_get_centralities(hb_graph *g, double *closeness, double *harmonic, double *lin,
                              double *reachable) {
    hb_status st = check(g);
    if (st != HB_OK) return st;
    if (g->lruns) return fail(HB_ERR_STATE, "a handle of several runs: use hb_get_run_centralities");
    NvtxRange nv("hb_get_centralities");
    const int64_t n = g->n;
    double *outs[4] = {closeness, harmonic, lin, reachable};
    bool host[4] = {false, false, false, false};
    bool any_host = false;
    for (int k = 0; k < 4; ++k) {
        host[k] = outs[k] && !is_device_ptr(outs[k]);
        any_host |= host[k];
    }
    cudaError_t e = cudaSuccess;
    if (!any_host) {
        // device outputs: written in the caller's order by one launch
        e = launch_finalize(g->a, current_regs(g), g->inv, g->fp32, 0, n, outs[0], outs[1], outs[2], outs[3],
                            g->s);
        if (n > 0) g->launches += 1;
        if (e == cudaSuccess) e = cudaStreamSynchronize(g->s);
        if (e != cudaSuccess) return cuda_fail(e, "centralities");
        return HB_OK;
    }
    // host outputs: chunks of nodes computed into two alternating staging
    // buffers on the handle's stream and copied out on a second stream, so
    // the copies of one chunk overlap the computation of the next
    const int64_t chunk = std::min<int64_t>(n, (int64_t)1 << 24);
    DevMem tmp = scratch(g);
    double *stage[4][2] = {};
    for (int k = 0; k < 4; ++k)
        if (host[k]) {
            stage[k][0] = tmp.alloc<double>(chunk > 0 ? chunk : 1);
            stage[k][1] = tmp.alloc<double>(chunk > 0 ? chunk : 1);
        }
    if (tmp.err != cudaSuccess) { tmp.free_all(); return fail(HB_ERR_OOM, "out of device memory"); }
    cudaStream_t cs = nullptr;
    cudaEvent_t ev_k[2] = {nullptr, nullptr}, ev_c[2] = {nullptr, nullptr};
    e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
        e = cudaEventCreateWithFlags(&ev_k[i], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_c[i], cudaEventDisableTiming);
    }
    for (int64_t c = 0, u0 = 0; u0 < n && e == cudaSuccess; ++c, u0 += chunk) {
        const int slot = (int)(c & 1);
        const int64_t cnt = std::min(chunk, n - u0);
        if (c >= 2) e = cudaStreamWaitEvent(g->s, ev_c[slot], 0);   // the slot's last copies are done
        double *dst[4];
        for (int k = 0; k < 4; ++k) dst[k] = !outs[k] ? nullptr : host[k] ? stage[k][slot] : outs[k] + u0;
        if (e == cudaSuccess)
            e = launch_finalize(g->a, current_regs(g), g->inv, g->fp32, u0, cnt, dst[0], dst[1], dst[2], dst[3],
                                g->s);
        g->launches += 1;
        if (e == cudaSuccess) e = cudaEventRecord(ev_k[slot], g->s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ev_k[slot], 0);
        for (int k = 0; k < 4 && e == cudaSuccess; ++k)
            if (host[k])
                e = cudaMemcpyAsync(outs[k] + u0, stage[k][slot], sizeof(double) * cnt, cudaMemcpyDeviceToHost, cs);
        if (e == cudaSuccess) e = cudaEventRecord(ev_c[slot], cs);
    }
    // the staging buffers go back to the pool on the handle's stream once
    // the copies that read them are done
    if (cs && e == cudaSuccess && n > 0) e = cudaStreamWaitEvent(g->s, ev_c[((n - 1) / chunk) & 1], 0);
    if (cs) {
        const cudaError_t f = cudaStreamSynchronize(cs);
        if (e == cudaSuccess) e = f;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->s);
    tmp.free_all();
    for (int i = 0; i < 2; ++i) {
        if (ev_k[i]) cudaEventDestroy(ev_k[i]);
        if (ev_c[i]) cudaEventDestroy(ev_c[i]);
    }
    if (cs) cudaStreamDestroy(cs);
    if (e != cudaSuccess) return cuda_fail(e, "centralities");
    return HB_OK;
}

hb_status hb_get_accumulators(hb_graph *g, double *sumd, double *harm) {
    hb_status st = check(g);
    if (st != HB_OK) return st;
    if (g->lruns) return fail(HB_ERR_STATE, "a handle of several runs: use hb_get_run_accumulators");
    const int64_t n = g->n;
    double *outs[2] = {sumd, harm};
    const double *src[2] = {g->a.sumd, g->a.harm};
    DevMem tmp = scratch(g);
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
        if (!outs[k]) continue;
        double *d = is_device_ptr(outs[k]) ? outs[k] : tmp.alloc<double>(n);
        if (!d) { tmp.free_all(); return fail(HB_ERR_OOM, "out of device memory"); }
        e = launch_gather_f64(src[k], g->inv, n, d, g->s);
        if (e == cudaSuccess && d != outs[k]) e = to_caller(outs[k], d, sizeof(double) * n, g->s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->s);
    tmp.free_all();
    if (e != cudaSuccess) return cuda_fail(e, "accumulators");
    return HB_OK;
}

hb_status hb_get_registers(hb_graph *g, uint8_t *out) {
    hb_status st = check(g);
    if (st != HB_OK) return st;
    const size_t bytes = (size_t)g->n << g->b;
    if (bytes == 0) return HB_OK;
    if (!out) return fail(HB_ERR_INVALID, "out is NULL");
    DevMem tmp = scratch(g);
    uint8_t *d = is_device_ptr(out) ? out : tmp.alloc<uint8_t>(bytes);
    if (!d) { tmp.free_all(); return fail(HB_ERR_OOM, "out of device memory"); }
    cudaError_t e = launch_gather_rows(current_regs(g), g->inv, g->n, 1 << g->b, d, g->s, g->packed);
    if (e == cudaSuccess && d != out) e = to_caller(out, d, bytes, g->s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->s);
    tmp.free_all();
    if (e != cudaSuccess) return cuda_fail(e, "registers");
    return HB_OK;
}

hb_status hb_get_frontier(hb_graph *g, uint8_t *changed, uint8_t *must_check) {
    hb_status st = check(g);
    if (st != HB_OK) return st;
    const int64_t n = g->n;
    DevMem tmp = scratch(g);
    uint8_t *dc = changed ? (is_device_ptr(changed) ? changed : tmp.alloc<uint8_t>(n)) : nullptr;
    uint8_t *dm = must_check ? (is_device_ptr(must_check) ? must_check : tmp.alloc<uint8_t>(n)) : nullptr;
    if (tmp.err != cudaSuccess) { tmp.free_all(); return fail(HB_ERR_OOM, "out of device memory"); }
    cudaError_t e = launch_frontier_out(g->a, g->inv, dc, dm, g->s);
    if (e == cudaSuccess && dc && dc != changed) e = to_caller(changed, dc, n, g->s);
    if (e == cudaSuccess && dm && dm != must_check) e = to_caller(must_check, dm, n, g->s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->s);
    tmp.free_all();
    if (e != cudaSuccess) return cuda_fail(e, "frontier");
    return HB_OK;
}

hb_status hb_get_info(hb_graph *g, hb_info *info) {
    if (!g || !info) return fail(HB_ERR_INVALID, "NULL argument");
    info->n = g->n;
    info->m = g->m;
    info->log2m = g->b;
    info->t = g->t;
    info->last_changed = g->last_changed;
    info->last_nodes = g->last_nodes;
    info->last_arcs = g->last_arcs;
    info->total_arcs = g->total_arcs;
    info->last_sparse = g->last_sparse;
    info->converged = g->converged ? 1 : 0;
    info->device_bytes = (int64_t)g->mem.bytes;
    info->launches = g->launches;
    info->kernel_launches = g->kernel_launches;
    info->kernel_ms = g->kernel_ms;
    info->kernel_bytes = g->kernel_bytes;
    info->packed = g->packed ? 1 : 0;
    info->frontier_switch = g->a.sparse_frac;
    info->push_launches = g->push_launches;
    info->push_ms = g->push_ms;
    info->push_bytes = g->push_bytes;
    info->arcs_per_slot = g->y.aps;
    info->hot_nodes = (int32_t)g->a.hot;
    info->hot_passes = g->a.two_pass ? 2 : 1;
    return HB_OK;
}

hb_status hb_set_class_sizing(hb_graph *g, int32_t arcs_per_slot) {
    hb_status st = check(g);
    if (st != HB_OK) return st;
    bool ok = false;
    for (int c : kTuneAps) ok |= c == arcs_per_slot;
    if (!ok) return fail(HB_ERR_INVALID, "arcs_per_slot must be a power of two from 1 to 128");
    st = retune(g, arcs_per_slot);
    return st == HB_OK ? init_state(g, g->seed) : st;
}

hb_status hb_tune(hb_graph *g, int32_t *arcs_per_slot) {
    hb_status st = check(g);
    if (st != HB_OK) return st;
    const uint64_t seed = g->seed;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return fail(HB_ERR_CUDA, "tuning events");
    // every candidate twice, in ascending then descending order, keeping
    // its faster time: a drift of the clocks during tuning then favours no
    // end of the list
    constexpr int nc = sizeof(kTuneAps) / sizeof(kTuneAps[0]);
    float cand_ms[nc];
    for (float &x : cand_ms) x = 1e30f;
    for (int pass = 0; pass < 2 * nc && st == HB_OK; ++pass) {
        const int ci = pass < nc ? pass : 2 * nc - 1 - pass;
        st = retune(g, kTuneAps[ci]);
        if (st == HB_OK) st = init_state(g, seed);
        if (st != HB_OK) break;
        cudaEventRecord(e0, g->s);
        for (int i = 0; i < kTuneIters && st == HB_OK && !g->converged; ++i) st = hb_step(g, nullptr);
        cudaEventRecord(e1, g->s);
        float ms = 0.f;
        if (st == HB_OK && cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess &&
            ms < cand_ms[ci])
            cand_ms[ci] = ms;
    }
    int best = g->y.aps;
    float best_ms = 1e30f;
    for (int ci = 0; ci < nc; ++ci)
        if (cand_ms[ci] < best_ms) {
            best_ms = cand_ms[ci];
            best = kTuneAps[ci];
        }
    if (st == HB_OK) st = retune(g, best);
    // then the hot range of the two-phase gather, with that sizing: one
    // pass, or hot counters filling each candidate share of L2 (single-run
    // handles whose counters do not fit in L2 alone)
    int dev = 0, l2 = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev);
    const int64_t row = (int64_t)1 << g->b;
    if (st == HB_OK && !g->lruns && !g->packed && g->n * row > (int64_t)l2) {
        // candidates: one pass without a hot range (the sizing above); one
        // pass with L2 priorities, each hot range with 1 and 2 times the
        // sizing; two passes, each hot range with 1, 2 and 4 times it (each
        // pass gathers only part of every list)
        struct Cand { uint32_t hot; int aps, passes; };
        std::vector<Cand> cands{{0u, best, 1}};
        const int aps_max = kTuneAps[sizeof(kTuneAps) / sizeof(kTuneAps[0]) - 1];
        auto add = [&](int64_t mb, int passes) {
            const int64_t h = (mb << 20) / row;
            if (h >= g->n) return;
            for (int f = 1; f <= (passes == 1 ? 2 : 4); f *= 2)
                if (best * f <= aps_max) cands.push_back({(uint32_t)h, best * f, passes});
        };
        for (int64_t mb : kTuneHintMiB) add(mb, 1);
        for (int64_t mb : kTuneHotMiB) add(mb, 2);
        const int nh = (int)cands.size();
        std::vector<float> hot_ms(nh, 1e30f);
        for (int pass = 0; pass < 2 * nh && st == HB_OK; ++pass) {
            const int ci = pass < nh ? pass : 2 * nh - 1 - pass;
            if (g->y.aps != cands[ci].aps) st = retune(g, cands[ci].aps);
            if (st == HB_OK) st = apply_hot(g, cands[ci].hot, cands[ci].passes);
            if (st == HB_OK) st = init_state(g, seed);
            if (st != HB_OK) break;
            cudaEventRecord(e0, g->s);
            for (int i = 0; i < kTuneIters && st == HB_OK && !g->converged; ++i) st = hb_step(g, nullptr);
            cudaEventRecord(e1, g->s);
            float ms = 0.f;
            if (st == HB_OK && cudaEventSynchronize(e1) == cudaSuccess &&
                cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms < hot_ms[ci])
                hot_ms[ci] = ms;
        }
        int bi = 0;
        for (int ci = 1; ci < nh; ++ci)
            if (hot_ms[ci] < hot_ms[bi]) bi = ci;
        best = cands[bi].aps;
        if (st == HB_OK && g->y.aps != best) st = retune(g, best);
        if (st == HB_OK) st = apply_hot(g, cands[bi].hot, cands[bi].passes);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != HB_OK) return st;
    st = init_state(g, seed);
    if (st == HB_OK && arcs_per_slot) *arcs_per_slot = best;
    return st;
}

hb_status hb_set_hot_nodes(hb_graph *g, int32_t hot_nodes, int32_t passes) {
    hb_status st = check(g);
    if (st != HB_OK) return st;
    if (hot_nodes < 0) return fail(HB_ERR_INVALID, "hot_nodes must be >= 0");
    if (passes < 1 || passes > 2) return fail(HB_ERR_INVALID, "passes must be 1 or 2");
    if (g->lruns && hot_nodes > 0)
        return fail(HB_ERR_INVALID, "handles of several runs per row take no hot range");
    if (g->packed && hot_nodes > 0)
        return fail(HB_ERR_STATE, "handles with HB_PACKED_REGISTERS take no hot range");
    return apply_hot(g, hot_nodes, passes);
}

hb_status hb_set_frontier_switch(hb_graph *g, double push_frac) {
    hb_status st = check(g);
    if (st != HB_OK) return st;
    if (!(push_frac > 0.0) || !std::isfinite(push_frac))
        return fail(HB_ERR_INVALID, "push_frac must be a finite positive fraction");
    g->opt.frontier_switch = push_frac;
    g->a.sparse_frac = push_frac;
    return HB_OK;
}

hb_status hb_reset(hb_graph *g, uint64_t seed) {
    hb_status st = check(g);
    if (st != HB_OK) return st;
    return init_state(g, seed);
}

hb_status hb_set_weights(hb_graph *g, const int64_t *weights) {
    hb_status st = check(g);
    if (st != HB_OK) return st;
    if (g->packed) return fail(HB_ERR_STATE, "handles with HB_PACKED_REGISTERS take no node weights");
    DevMem &M = g->mem;
    if (!weights) {
        if (g->wfirst) M.release(g->wfirst);
        g->wfirst = nullptr;
        return init_state(g, g->seed);
    }
    const int64_t n = g->n;
    DevMem tmp = scratch(g);
    int64_t *w = nullptr;
    cudaError_t e = cudaSuccess;
    if (is_device_ptr(weights)) {
        w = const_cast<int64_t *>(weights);
    } else {
        w = tmp.alloc<int64_t>(n);
        if (w) e = to_device(w, weights, sizeof(int64_t) * n, g->s);
    }
    unsigned long long *err = tmp.alloc<unsigned long long>(1);
    int64_t *wf = M.alloc<int64_t>(n + 1);
    if (!w || !err || !wf) {
        tmp.free_all();
        if (wf) M.release(wf);
        return fail(HB_ERR_OOM, "out of device memory (weights)");
    }
    unsigned long long err_host = 0;
    if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(unsigned long long), g->s);
    if (e == cudaSuccess) e = replica_starts(w, n, wf, err, g->s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&err_host, err, sizeof(err_host), cudaMemcpyDeviceToHost, g->s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->s);
    tmp.free_all();
    if (e != cudaSuccess) {
        M.release(wf);
        return cuda_fail(e, "weights");
    }
    if (err_host) {
        M.release(wf);
        return fail(HB_ERR_INVALID, "every weight must lie in [0, 2^31)");
    }
    if (g->wfirst) M.release(g->wfirst);
    g->wfirst = wf;
    return init_state(g, g->seed);
}

hb_status hb_set_discount(hb_graph *g, const double *f, int32_t len) {
    hb_status st = check(g);
    if (st != HB_OK) return st;
    if (len < 0) return fail(HB_ERR_INVALID, "len must be >= 0");
    if (len > 0 && !f) return fail(HB_ERR_INVALID, "f is NULL");
    DevMem &M = g->mem;
    StepArgs &a = g->a;
    if (g->ftab) M.release(g->ftab);
    g->ftab = nullptr;
    if (len == 0) {
        if (g->disc) M.release(g->disc);
        g->disc = nullptr;
        a.disc = nullptr;
        a.ftab = nullptr;
        a.flen = 0;
        return init_state(g, g->seed);
    }
    if (!g->disc) g->disc = M.alloc<double>(g->n << g->lruns);   // one per (node, run)
    g->ftab = M.alloc<double>(len);
    if (!g->disc || !g->ftab) {
        if (g->disc) M.release(g->disc);
        if (g->ftab) M.release(g->ftab);
        g->disc = g->ftab = nullptr;
        a.disc = nullptr;
        a.ftab = nullptr;
        a.flen = 0;
        return fail(HB_ERR_OOM, "out of device memory (discount)");
    }
    cudaError_t e = to_device(g->ftab, f, sizeof(double) * len, g->s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->s);
    if (e != cudaSuccess) return cuda_fail(e, "discount table");
    a.disc = g->disc;
    a.ftab = g->ftab;
    a.flen = len;
    return init_state(g, g->seed);
}

hb_status hb_get_discounted(hb_graph *g, double *out) {
    hb_status st = check(g);
    if (st != HB_OK) return st;
    if (!g->a.disc) return fail(HB_ERR_STATE, "no discount function set (hb_set_discount)");
    if (g->lruns) return fail(HB_ERR_STATE, "a handle of several runs: use hb_get_run_discounted");
    if (g->n > 0 && !out) return fail(HB_ERR_INVALID, "out is NULL");
    const int64_t n = g->n;
    DevMem tmp = scratch(g);
    double *d = is_device_ptr(out) ? out : tmp.alloc<double>(n);
    if (!d) { tmp.free_all(); return fail(HB_ERR_OOM, "out of device memory"); }
    cudaError_t e = launch_gather_f64(g->a.disc, g->inv, n, d, g->s);
    if (e == cudaSuccess && d != out) e = to_caller(out, d, sizeof(double) * n, g->s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->s);
    tmp.free_all();
    if (e != cudaSuccess) return cuda_fail(e, "discounted accumulator");
    return HB_OK;
}

hb_status hb_get_neighbourhood(hb_graph *g, double *out, int32_t cap, int32_t *len) {
    hb_status st = check(g);
    if (st != HB_OK) return st;
    if (!g->track_nf) return fail(HB_ERR_STATE, "the handle was created without HB_NEIGHBOURHOOD");
    if (cap < 0 || (cap > 0 && !out)) return fail(HB_ERR_INVALID, "out is NULL or cap < 0");
    const int32_t k = (int32_t)g->nf.size();
    for (int32_t i = 0; i < k && i < cap; ++i) out[i] = g->nf[i];
    if (len) *len = k;
    return HB_OK;
}

hb_status hb_create_runs(const int64_t *offsets, const int32_t *targets, int64_t n, int64_t m, int log2m,
                         int32_t runs, const uint64_t *seeds, const hb_options *opt, hb_graph **out) {
    g_err.clear();
    if (!out) return fail(HB_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (!seeds) return fail(HB_ERR_INVALID, "seeds is NULL");
    int lr = 0;
    while (lr < 7 && (1 << lr) < runs) ++lr;
    if (runs < 2 || runs > 64 || (1 << lr) != runs)
        return fail(HB_ERR_INVALID, "runs must be a power of two from 2 to 64");
    if (log2m < kMinLog2m || log2m > 9) return fail(HB_ERR_INVALID, "log2m must lie in [4, 9] for several runs");
    if (log2m + lr > kMaxLog2m) return fail(HB_ERR_INVALID, "runs * 2^log2m must not exceed 4096 bytes");
    if (opt && (opt->flags & HB_NEIGHBOURHOOD))
        return fail(HB_ERR_INVALID, "HB_NEIGHBOURHOOD needs a handle of one run");
    return create_impl<int64_t>(offsets, targets, n, m, log2m, seeds[0], opt, out, lr, seeds, true);
}

namespace {
hb_status check_runs(hb_graph *g) {
    hb_status st = check(g);
    if (st != HB_OK) return st;
    if (!g->lruns) return fail(HB_ERR_STATE, "not a handle of several runs (hb_create_runs)");
    return HB_OK;
}
}  // namespace

hb_status hb_get_run_steps(hb_graph *g, int32_t *steps) {
    hb_status st = check_runs(g);
    if (st != HB_OK) return st;
    if (!steps) return fail(HB_ERR_INVALID, "steps is NULL");
    // run r's fixpoint came one iteration after its last change (Sec. 4.2);
    // until then it has run every iteration so far
    for (size_t r = 0; r < g->run_last.size(); ++r) {
        const int32_t fix = g->run_last[r] + 2;
        steps[r] = fix < g->t ? fix : g->t;
    }
    return HB_OK;
}

hb_status hb_get_run_centralities(hb_graph *g, int32_t run, double *closeness, double *harmonic,
                                  double *lin, double *reachable) {
    hb_status st = check_runs(g);
    if (st != HB_OK) return st;
    if (run < 0 || run >= (1 << g->lruns)) return fail(HB_ERR_INVALID, "run out of range");
    const int64_t n = g->n;
    double *outs[4] = {closeness, harmonic, lin, reachable};
    double *dev[4] = {nullptr, nullptr, nullptr, nullptr};
    DevMem tmp = scratch(g);
    for (int k = 0; k < 4; ++k)
        if (outs[k]) dev[k] = is_device_ptr(outs[k]) ? outs[k] : tmp.alloc<double>(n);
    if (tmp.err != cudaSuccess) { tmp.free_all(); return fail(HB_ERR_OOM, "out of device memory"); }
    cudaError_t e = launch_runs_centralities(g->a, current_regs(g), g->perm, g->fp32, run, dev[0], dev[1],
                                             dev[2], dev[3], g->s);
    for (int k = 0; k < 4 && e == cudaSuccess; ++k)
        if (outs[k] && dev[k] != outs[k]) e = to_caller(outs[k], dev[k], sizeof(double) * n, g->s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->s);
    tmp.free_all();
    if (e != cudaSuccess) return cuda_fail(e, "run centralities");
    return HB_OK;
}

hb_status hb_get_run_accumulators(hb_graph *g, int32_t run, double *sumd, double *harm) {
    hb_status st = check_runs(g);
    if (st != HB_OK) return st;
    if (run < 0 || run >= (1 << g->lruns)) return fail(HB_ERR_INVALID, "run out of range");
    const int64_t n = g->n;
    double *outs[2] = {sumd, harm};
    const double *src[2] = {g->a.sumd, g->a.harm};
    DevMem tmp = scratch(g);
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
        if (!outs[k]) continue;
        double *d = is_device_ptr(outs[k]) ? outs[k] : tmp.alloc<double>(n);
        if (!d) { tmp.free_all(); return fail(HB_ERR_OOM, "out of device memory"); }
        e = launch_gather_strided(src[k], g->inv, n, g->lruns, run, d, g->s);
        if (e == cudaSuccess && d != outs[k]) e = to_caller(outs[k], d, sizeof(double) * n, g->s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->s);
    tmp.free_all();
    if (e != cudaSuccess) return cuda_fail(e, "run accumulators");
    return HB_OK;
}

hb_status hb_get_run_discounted(hb_graph *g, int32_t run, double *out) {
    hb_status st = check_runs(g);
    if (st != HB_OK) return st;
    if (run < 0 || run >= (1 << g->lruns)) return fail(HB_ERR_INVALID, "run out of range");
    if (!g->a.disc) return fail(HB_ERR_STATE, "no discount function set (hb_set_discount)");
    if (g->n > 0 && !out) return fail(HB_ERR_INVALID, "out is NULL");
    const int64_t n = g->n;
    DevMem tmp = scratch(g);
    double *d = is_device_ptr(out) ? out : tmp.alloc<double>(n);
    if (!d) { tmp.free_all(); return fail(HB_ERR_OOM, "out of device memory"); }
    cudaError_t e = launch_gather_strided(g->a.disc, g->inv, n, g->lruns, run, d, g->s);
    if (e == cudaSuccess && d != out) e = to_caller(out, d, sizeof(double) * n, g->s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->s);
    tmp.free_all();
    if (e != cudaSuccess) return cuda_fail(e, "run discounted accumulator");
    return HB_OK;
}

hb_status hb_get_run_stats(hb_graph *g, int32_t which, double *mean, double *sd) {
    hb_status st = check_runs(g);
    if (st != HB_OK) return st;
    if (which < 0 || which > 4) return fail(HB_ERR_INVALID, "which must lie in [0, 4]");
    if (which == 4 && !g->a.disc) return fail(HB_ERR_STATE, "no discount function set (hb_set_discount)");
    const int64_t n = g->n;
    DevMem tmp = scratch(g);
    double *dm = mean ? (is_device_ptr(mean) ? mean : tmp.alloc<double>(n)) : nullptr;
    double *ds = sd ? (is_device_ptr(sd) ? sd : tmp.alloc<double>(n)) : nullptr;
    if (tmp.err != cudaSuccess) { tmp.free_all(); return fail(HB_ERR_OOM, "out of device memory"); }
    cudaError_t e = launch_runs_stats(g->a, current_regs(g), g->perm, g->fp32, which, dm, ds, g->s);
    if (e == cudaSuccess && mean && dm != mean) e = to_caller(mean, dm, sizeof(double) * n, g->s);
    if (e == cudaSuccess && sd && ds != sd) e = to_caller(sd, ds, sizeof(double) * n, g->s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->s);
    tmp.free_all();
    if (e != cudaSuccess) return cuda_fail(e, "run statistics");
    return HB_OK;
}

// ------------------------------------------------------------ checkpoint --

namespace {
constexpr uint64_t kMagic = 0x32304c4c41425948ULL;   // "HYBALL02"

struct SaveHeader {
    uint64_t magic;
    int64_t n, m;
    int32_t b, fp32, relabel, t;
    uint64_t seed;
    int32_t converged, frontier;
    int64_t total_arcs;
    int32_t weighted, flen;   // Sec. 6 replica starts and Sec. 7 discount follow when set
    int32_t nf_len, pad;      // recorded neighbourhood function values follow when set
};

bool write_dev(FILE *f, const void *dev, size_t bytes, cudaStream_t s) {
    std::vector<char> buf(bytes);
    if (bytes && cudaMemcpyAsync(buf.data(), dev, bytes, cudaMemcpyDeviceToHost, s) != cudaSuccess) return false;
    if (cudaStreamSynchronize(s) != cudaSuccess) return false;
    return fwrite(buf.data(), 1, bytes, f) == bytes;
}

bool read_dev(FILE *f, void *dev, size_t bytes, cudaStream_t s) {
    std::vector<char> buf(bytes);
    if (fread(buf.data(), 1, bytes, f) != bytes) return false;
    if (bytes && cudaMemcpyAsync(dev, buf.data(), bytes, cudaMemcpyHostToDevice, s) != cudaSuccess) return false;
    return cudaStreamSynchronize(s) == cudaSuccess;
}
}  // namespace

hb_status hb_save(hb_graph *g, const char *path) {
    hb_status st = check(g);
    if (st != HB_OK) return st;
    if (g->lruns) return fail(HB_ERR_STATE, "checkpoints need a handle of one run");
    if (g->packed) return fail(HB_ERR_STATE, "checkpoints hold byte registers, not HB_PACKED_REGISTERS");
    if (!path) return fail(HB_ERR_INVALID, "path is NULL");
    FILE *f = fopen(path, "wb");
    if (!f) return fail(HB_ERR_INVALID, std::string("cannot open ") + path);
    SaveHeader h{kMagic, g->n, g->m, g->b, g->fp32, g->relabel, g->t, g->seed,
                 g->converged, g->opt.frontier, g->total_arcs, g->wfirst ? 1 : 0, g->a.flen,
                 g->track_nf ? (int32_t)g->nf.size() : -1, 0};
    const size_t P = (size_t)1 << g->b;
    const size_t n = (size_t)g->n;
    bool ok = fwrite(&h, sizeof(h), 1, f) == 1;
    ok = ok && write_dev(f, g->off, sizeof(int64_t) * (n + 1), g->s);
    ok = ok && write_dev(f, g->tgt, sizeof(int32_t) * g->m, g->s);
    if (g->relabel) {
        ok = ok && write_dev(f, g->perm, sizeof(int32_t) * n, g->s);
        ok = ok && write_dev(f, g->inv, sizeof(int32_t) * n, g->s);
    }
    ok = ok && write_dev(f, current_regs(g), n * P, g->s);
    ok = ok && write_dev(f, g->a.sumd, sizeof(double) * n, g->s);
    ok = ok && write_dev(f, g->a.harm, sizeof(double) * n, g->s);
    ok = ok && write_dev(f, g->a.ecache, (g->fp32 ? sizeof(float) : sizeof(double)) * n, g->s);
    ok = ok && write_dev(f, g->a.changed, n, g->s);
    ok = ok && write_dev(f, g->ctr, sizeof(Counters), g->s);
    Counters c{};
    if (ok) ok = cudaMemcpy(&c, g->ctr, sizeof(c), cudaMemcpyDeviceToHost) == cudaSuccess;
    // the last iteration's changed lists drive the next frontier
    const int last = (g->t + 1) & 1;
    ok = ok && write_dev(f, g->a.clist[last], sizeof(int32_t) * c.list_len, g->s);
    ok = ok && write_dev(f, g->a.biglist[last], sizeof(int32_t) * c.n_big, g->s);
    if (g->wfirst) ok = ok && write_dev(f, g->wfirst, sizeof(int64_t) * (n + 1), g->s);
    if (g->a.flen) {
        ok = ok && write_dev(f, g->ftab, sizeof(double) * g->a.flen, g->s);
        ok = ok && write_dev(f, g->disc, sizeof(double) * n, g->s);
    }
    if (g->track_nf && !g->nf.empty())
        ok = ok && fwrite(g->nf.data(), sizeof(double), g->nf.size(), f) == g->nf.size();
    fclose(f);
    if (!ok) return fail(HB_ERR_CUDA, "checkpoint write failed");
    return HB_OK;
}

hb_status hb_load(const char *path, const hb_options *opt, hb_graph **out) {
    g_err.clear();
    if (!path || !out) return fail(HB_ERR_INVALID, "NULL argument");
    *out = nullptr;
    FILE *f = fopen(path, "rb");
    if (!f) return fail(HB_ERR_INVALID, std::string("cannot open ") + path);
    SaveHeader h{};
    if (fread(&h, sizeof(h), 1, f) != 1 || h.magic != kMagic) {
        fclose(f);
        return fail(HB_ERR_INVALID, "not a HyperBall checkpoint");
    }
    hb_options o;
    if (opt) o = *opt; else default_opts(&o);
    if (o.max_steps <= 0) o.max_steps = 1 << 20;
    int aps = 0;
    if (!sizing_of(o, &aps)) {
        fclose(f);
        return fail(HB_ERR_INVALID, "arcs_per_slot must be 0 or a power of two from 1 to 128");
    }
    if (o.flags & HB_PACKED_REGISTERS) {
        fclose(f);
        return fail(HB_ERR_INVALID, "checkpoints hold byte registers, not HB_PACKED_REGISTERS");
    }
    cudaFree(nullptr);
    hb_graph *g = new hb_graph();
    g->n = h.n; g->m = h.m; g->b = h.b; g->gb = h.b; g->y = make_layout(h.b, aps);
    g->opt = o;
    g->opt.frontier = h.frontier;
    g->s = static_cast<cudaStream_t>(o.stream);
    g->mem.pool = library_pool();
    g->mem.stream = g->s;
    g->fp32 = h.fp32 != 0;
    g->relabel = h.relabel != 0;
    g->track_nf = h.nf_len >= 0;
    const size_t P = (size_t)1 << g->b, n = (size_t)g->n;
    DevMem &M = g->mem;
    g->off = M.alloc<int64_t>(n + 1);
    g->tgt = M.alloc<int32_t>(g->m);
    if (g->relabel) { g->perm = M.alloc<int32_t>(n); g->inv = M.alloc<int32_t>(n); }
    bool ok = M.err == cudaSuccess;
    ok = ok && read_dev(f, g->off, sizeof(int64_t) * (n + 1), g->s);
    ok = ok && read_dev(f, g->tgt, sizeof(int32_t) * g->m, g->s);
    if (ok && g->relabel) {
        ok = read_dev(f, g->perm, sizeof(int32_t) * n, g->s) && read_dev(f, g->inv, sizeof(int32_t) * n, g->s);
    }
    if (!ok) { fclose(f); delete g; return fail(HB_ERR_INVALID, "truncated checkpoint or no memory"); }
    hb_status st = finish_setup(g);
    if (st == HB_OK && o.hot_nodes > 0) st = apply_hot(g, o.hot_nodes, o.hot_passes);
    if (st == HB_OK) st = init_state(g, h.seed);
    if (st != HB_OK) { fclose(f); delete g; return st; }
    // restore the state of iteration t: counters into both buffers
    g->t = h.t;
    g->converged = h.converged != 0;
    g->total_arcs = h.total_arcs;
    ok = read_dev(f, g->a.regs[h.t & 1], n * P, g->s);
    if (ok && n * P) ok = cudaMemcpy(g->a.regs[(h.t + 1) & 1], g->a.regs[h.t & 1], n * P,
                                     cudaMemcpyDeviceToDevice) == cudaSuccess;
    ok = ok && read_dev(f, g->a.sumd, sizeof(double) * n, g->s);
    ok = ok && read_dev(f, g->a.harm, sizeof(double) * n, g->s);
    ok = ok && read_dev(f, g->a.ecache, (g->fp32 ? sizeof(float) : sizeof(double)) * n, g->s);
    ok = ok && read_dev(f, g->a.changed, n, g->s);
    ok = ok && read_dev(f, g->ctr, sizeof(Counters), g->s);
    Counters c{};
    if (ok) ok = cudaMemcpy(&c, g->ctr, sizeof(c), cudaMemcpyDeviceToHost) == cudaSuccess;
    const int last = (h.t + 1) & 1;
    ok = ok && read_dev(f, g->a.clist[last], sizeof(int32_t) * c.list_len, g->s);
    ok = ok && read_dev(f, g->a.biglist[last], sizeof(int32_t) * c.n_big, g->s);
    if (ok && h.weighted) {
        g->wfirst = M.alloc<int64_t>(n + 1);
        ok = g->wfirst && read_dev(f, g->wfirst, sizeof(int64_t) * (n + 1), g->s);
    }
    if (ok && h.flen > 0) {
        g->ftab = M.alloc<double>(h.flen);
        g->disc = M.alloc<double>(n);
        ok = g->ftab && g->disc && read_dev(f, g->ftab, sizeof(double) * h.flen, g->s) &&
             read_dev(f, g->disc, sizeof(double) * n, g->s);
        g->a.disc = g->disc;
        g->a.ftab = g->ftab;
        g->a.flen = h.flen;
    }
    if (ok && h.nf_len >= 0) {
        g->nf.assign((size_t)h.nf_len, 0.0);
        ok = fread(g->nf.data(), sizeof(double), (size_t)h.nf_len, f) == (size_t)h.nf_len;
    }
    fclose(f);
    if (!ok) { delete g; return fail(HB_ERR_INVALID, "truncated checkpoint"); }
    *out = g;
    return HB_OK;
}

void hb_destroy(hb_graph *g) {
    if (!g) return;
    wait_reverse(g);
    if (g->s) cudaStreamSynchronize(g->s);
    else cudaDeviceSynchronize();
    delete g;
}

hb_status hb_set_l2_fetch_bytes(int32_t bytes, int32_t *previous) {
    if (bytes != 0 && bytes != 32 && bytes != 64 && bytes != 128)
        return fail(HB_ERR_INVALID, "the L2 fetch granularity must be 32, 64 or 128 bytes (0: unchanged)");
    size_t cur = 0;
    cudaError_t e = cudaDeviceGetLimit(&cur, cudaLimitMaxL2FetchGranularity);
    if (e != cudaSuccess) return cuda_fail(e, "L2 fetch granularity");
    if (previous) *previous = (int32_t)cur;
    if (bytes) {
        e = cudaDeviceSetLimit(cudaLimitMaxL2FetchGranularity, (size_t)bytes);
        if (e != cudaSuccess) return cuda_fail(e, "L2 fetch granularity");
    }
    return HB_OK;
}

hb_status hb_trim_memory(void) {
    std::lock_guard<std::mutex> lock(g_pool_mu);
    for (int d = 0; d < kMaxDevices; ++d) {
        if (!g_pools[d]) continue;
        const cudaError_t e = cudaMemPoolTrimTo(g_pools[d], 0);
        if (e != cudaSuccess) return cuda_fail(e, "trim");
    }
    return HB_OK;
}

const char *hb_last_error(void) { return g_err.c_str(); }

const char *hb_version(void) { return "hyperball-gb300 0.1 (sm_103a)"; }

}  // extern "C"

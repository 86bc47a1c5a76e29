// hb_batch.cu -- the batched form: many independent HyperBall problems
// (graphs of uneven size, each with its own log2m, seed, iteration index
// and frontier) advanced together.  Every kernel of an iteration covers
// all graphs in one launch: work items of all graphs form one index space
// (per-graph prefix sums), a warp looks its graph up by binary search and
// runs the same per-node code as the single-graph kernels.  The iteration
// is captured once into a CUDA graph; a run to every fixpoint is one graph
// launch whose conditional while node repeats the iteration on the device
// until no graph is active or the iteration cap is reached.
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "hb_handle.h"
#include "hb_step_dev.cuh"

namespace hb {

namespace {

using namespace dev;

constexpr int kMaxBatch = 4096;
constexpr int kMode_Idle = 2;

struct BatchCtl {
    int32_t n_active;
    int32_t iterations;
    int32_t max_steps;
    int32_t k;
    unsigned long long total_arcs;
};

struct BatchArrays {
    const StepArgs *args;          // [k]
    int64_t *item_prefix;          // [9][k+1] work items of the running iteration, per log2m
    int64_t *list_prefix;          // [k+1] previous changed lists (push marking)
    int64_t *big_prefix;           // [k+1] previous many-predecessor lists
    int64_t *push_prefix;          // [k+1] pushed union: warp items of 32 previous changed nodes
    int64_t *pbig_prefix;          // [k+1] pushed union: previous many-predecessor lists
    int64_t *copy_prefix;          // [k+1] copy-forward elements
    int64_t *word_prefix;          // [k+1] must-check bitmap words to clear
    const int64_t *tile_prefix;    // [k+1] 256-node tiles (static)
    int64_t *graph_arcs;           // [k] arcs scanned per graph since init
    int32_t *done;                 // [k] 1 once the graph has converged
    BatchCtl *ctl;
    int k;
    int use_cond;
    unsigned log2m_mask;           // bit b-4 set: some graph has log2m b
    cudaGraphConditionalHandle cond;
};

__device__ __forceinline__ int find_graph(const int64_t *prefix, int k, int64_t i) {
    int lo = 0, hi = k;   // prefix[lo] <= i < prefix[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (prefix[mid] <= i) lo = mid; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ int logsmax_of(int b) { return 5 - ((b - 4) < 5 ? (b - 4) : 5); }

// Exclusive prefix over graphs of a per-graph value, by one block.
template <class F>
__device__ void graph_prefix(int k, int64_t *out, F value) {
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < k; base += blockDim.x) {
        const int g = base + threadIdx.x;
        const int64_t v = g < k ? value(g) : 0;
        int64_t ex;
        const int64_t tot = block_excl_scan(v, ex);
        if (g < k) out[g] = carry + ex;
        __syncthreads();
        if (threadIdx.x == 0) carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) out[k] = carry;
    __syncthreads();
}

__global__ void batch_begin_kernel(BatchArrays B) {
    for (int g = threadIdx.x; g < B.k; g += blockDim.x) {
        const StepArgs &a = B.args[g];
        Counters *c = a.ctr;
        if (c->converged) {
            c->t = c->steps_done;
            c->n_changed = 0; c->list_len = 0; c->push_arcs = 0; c->n_big = 0; c->arcs = 0;
            for (int s = 0; s < kSegs; ++s) c->fill[s] = 0;
            c->mode = kMode_Idle;
        } else {
            begin_one(a);
        }
    }
    __syncthreads();
    auto push_ok = [&](int g) {
        const StepArgs &a = B.args[g];
        return a.ctr->mode == 1 && a.has_reverse && a.frontier != HB_FRONTIER_PULL && !a.push_union;
    };
    auto pushed = [&](int g) {
        const StepArgs &a = B.args[g];
        return a.ctr->mode == 1 && a.push_union;
    };
    graph_prefix(B.k, B.push_prefix, [&](int g) {
        return pushed(g) ? ((int64_t)B.args[g].ctr->prev_list_len + 31) / 32 : 0; });
    graph_prefix(B.k, B.pbig_prefix, [&](int g) {
        return pushed(g) ? (int64_t)B.args[g].ctr->prev_big : 0; });
    graph_prefix(B.k, B.list_prefix, [&](int g) {
        return push_ok(g) ? (int64_t)B.args[g].ctr->prev_list_len : 0; });
    graph_prefix(B.k, B.big_prefix, [&](int g) {
        return push_ok(g) ? (int64_t)B.args[g].ctr->prev_big : 0; });
    graph_prefix(B.k, B.copy_prefix, [&](int g) {
        const StepArgs &a = B.args[g];
        return a.ctr->mode == 1 ? (int64_t)a.ctr->prev_list_len << (a.b - 4) : 0; });
    graph_prefix(B.k, B.word_prefix, [&](int g) {
        const StepArgs &a = B.args[g];
        return a.ctr->mode == 1 ? (a.n + 31) / 32 : 0; });
}

__global__ void batch_clear_bits_kernel(BatchArrays B) {
    const int64_t total = B.word_prefix[B.k];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int g = find_graph(B.word_prefix, B.k, i);
        B.args[g].mustbits[i - B.word_prefix[g]] = 0u;
    }
}

__global__ void batch_mark_push_kernel(BatchArrays B) {
    const int lane = threadIdx.x & 31;
    const int64_t total = B.list_prefix[B.k];
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = gw; i < total; i += nw) {
        const int g = find_graph(B.list_prefix, B.k, i);
        const StepArgs &a = B.args[g];
        const int t = a.ctr->t;
        const int32_t w = a.clist[(t + 1) & 1][i - B.list_prefix[g]];
        if (a.roff[w + 1] - a.roff[w] > kBigRdeg) continue;
        push_warp(a, w, lane);
    }
    // nodes with many predecessors: one block each
    const int64_t nbig = B.big_prefix[B.k];
    const int wid = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int64_t q = blockIdx.x; q < nbig; q += gridDim.x) {
        const int g = find_graph(B.big_prefix, B.k, q);
        const StepArgs &a = B.args[g];
        const int t = a.ctr->t;
        const int32_t w = a.biglist[(t + 1) & 1][q - B.big_prefix[g]];
        const int64_t r0 = a.roff[w], r1 = a.roff[w + 1];
        for (int64_t j0 = r0 + 32 * wid; j0 < r1; j0 += 32 * nwarps) {
            const int64_t j = j0 + lane;
            mark_append(a, j < r1 ? a.rtgt[j] : -1, lane);
        }
    }
}

// Pushed union of the graphs in a pushed frontier iteration: a warp per 32
// changed nodes, a block per node with many predecessors.
__global__ void __launch_bounds__(kStepThreads, 4) batch_push_union_kernel(BatchArrays B) {
    const int lane = threadIdx.x & 31;
    const int64_t total = B.push_prefix[B.k];
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = gw; i < total; i += nw) {
        const int g = find_graph(B.push_prefix, B.k, i);
        const StepArgs &a = B.args[g];
        const int t = a.ctr->t;
        push_union_item(a, reinterpret_cast<const uint4 *>(a.regs[t & 1]),
                        reinterpret_cast<uint4 *>(a.regs[(t + 1) & 1]), a.clist[(t + 1) & 1],
                        (int64_t)a.ctr->prev_list_len, (i - B.push_prefix[g]) * 32, a.b - 4, lane);
    }
    const int64_t nbig = B.pbig_prefix[B.k];
    const int wid = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int64_t q = blockIdx.x; q < nbig; q += gridDim.x) {
        const int g = find_graph(B.pbig_prefix, B.k, q);
        const StepArgs &a = B.args[g];
        const int t = a.ctr->t;
        push_union_big(a, reinterpret_cast<const uint4 *>(a.regs[t & 1]),
                       reinterpret_cast<uint4 *>(a.regs[(t + 1) & 1]),
                       a.biglist[(t + 1) & 1][q - B.pbig_prefix[g]], wid, nwarps, a.b - 4, lane);
    }
}

__global__ void batch_copy_forward_kernel(BatchArrays B) {
    const int64_t total = B.copy_prefix[B.k];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int g = find_graph(B.copy_prefix, B.k, i);
        const StepArgs &a = B.args[g];
        copy_forward_one(a, a.ctr->t, i - B.copy_prefix[g]);
    }
}

// One block per graph: the work plan of graphs in frontier mode.
__global__ void batch_plan_kernel(BatchArrays B) {
    for (int g = blockIdx.x; g < B.k; g += gridDim.x) {
        const StepArgs &a = B.args[g];
        if (a.ctr->mode != 1 || a.push_union) continue;   // pushed iterations need no gather plan
        PlanParams pp{};
        const int ls = logsmax_of(a.b);
        pp.chunk = 64LL << ls;
        pp.nlight = ls + 1;
        pp.dense = 0;
        plan_block(a, pp, a.plan_sparse, a.owner_sparse, a.cstart_sparse);
        __syncthreads();
    }
}

// Work-item prefixes, one per log2m present: graphs of other log2m count 0.
__global__ void batch_items_kernel(BatchArrays B) {
    for (int lb = kMinLog2m; lb <= kMaxLog2m; ++lb) {
        if (!((B.log2m_mask >> (lb - kMinLog2m)) & 1u)) continue;
        graph_prefix(B.k, B.item_prefix + (size_t)(lb - kMinLog2m) * (B.k + 1), [&](int g) -> int64_t {
            const StepArgs &a = B.args[g];
            const int mode = a.ctr->mode;
            if (mode == kMode_Idle || a.b != lb) return 0;
            if (mode == 1 && a.push_union) {   // tail items of 32/L marked nodes
                int64_t nodes = 0;
                for (int s = 0; s < kSegs; ++s) nodes += (int64_t)a.ctr->fill[s];
                const int npw = 32 >> ((lb - 4) < 5 ? (lb - 4) : 5);
                return (nodes + npw - 1) / npw;
            }
            return mode == 1 ? a.plan_sparse->items : a.plan_dense->items;
        });
    }
}

// Work item `it` of one graph (the body of the single-graph step kernel's
// loop, with the plan read from memory).
template <int LOG2P, bool F32>
__device__ __forceinline__ void batch_item(const StepArgs &a, int64_t it, int t, bool sparse,
                                           double rdist64, float rdist32,
                                           const unsigned long long *pow2, bool prefetch,
                                           unsigned long long *cnt) {
    using C = Cfg<LOG2P>;
    const Plan *pl = sparse ? a.plan_sparse : a.plan_dense;
    const int32_t *list = sparse ? a.slist : a.dense_list;
    const uint8_t *cur = a.regs[t & 1];
    uint8_t *nxt = a.regs[(t + 1) & 1];
    int32_t *clist = a.clist[t & 1];
    int32_t *biglist = a.biglist[t & 1];
    const int64_t hch = pl->heavy_chunks;
    if (it < hch) {
        heavy_item<LOG2P, F32>(a, cur, nxt, t, it, sparse ? a.owner_sparse : a.owner_dense,
                               sparse ? a.cstart_sparse : a.cstart_dense, list, clist, biglist, sparse,
                               cnt, rdist64, rdist32, pow2);
        return;
    }
    const int64_t li = it - hch;
    int j = 0;
#pragma unroll
    for (int q = 1; q < C::NLIGHT; ++q)
        if (li >= pl->item_begin[q]) j = q;
    const int64_t seg0 = a.seg_begin[j + 1];
    const int64_t pos0 = seg0 + ((li - pl->item_begin[j]) << j);
    light_item<LOG2P, F32>(a, cur, nxt, t, pos0, seg0 + pl->count[j + 1], C::LOGSMAX - j, list, clist,
                           biglist, sparse, cnt, rdist64, rdist32, pow2, prefetch);
}

// The gather kernel over the items of every graph with log2m = LOG2P (one
// instantiation per log2m keeps its register budget that of the
// single-graph kernel).
template <int LOG2P, bool F32>
__global__ void __launch_bounds__(kStepThreads, Cfg<LOG2P>::CPL >= 4 ? 3 : 4)
    batch_step_kernel(BatchArrays B) {
    extern __shared__ int64_t s_prefix[];                 // [k+1]
    __shared__ unsigned long long s_pow2[64];
    __shared__ unsigned long long s_cnt[kStepThreads / 32];
    const int64_t *prefix = B.item_prefix + (size_t)(LOG2P - kMinLog2m) * (B.k + 1);
    for (int i = threadIdx.x; i <= B.k; i += blockDim.x) s_prefix[i] = prefix[i];
    if (threadIdx.x < 64) {
        const int M = threadIdx.x, sh = 64 - LOG2P;
        s_pow2[M] = (M == 0 || M > sh) ? 0ULL : 1ULL << (sh - M);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) s_cnt[wid] = 0;
    __syncthreads();
    const int64_t total = s_prefix[B.k];
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    int cur_g = -1, t = 0;
    bool sparse = false, prefetch = false, pushed = false;
    double rd64 = 1.0;
    float rd32 = 1.0f;
    for (int64_t it = gw; it < total; it += nw) {
        const int g = find_graph(s_prefix, B.k, it);
        const StepArgs &a = B.args[g];
        if (g != cur_g) {
            if (cur_g >= 0 && lane == 0 && s_cnt[wid]) {
                atomicAdd(&B.args[cur_g].ctr->n_changed, s_cnt[wid]);
                s_cnt[wid] = 0;
            }
            cur_g = g;
            const Counters *c = a.ctr;
            t = c->t;
            sparse = c->mode == 1;
            pushed = sparse && a.push_union;
            prefetch = !sparse && (t == 0 || 4 * (int64_t)c->prev_changed > a.n_pos);
            rd64 = 1.0 / (double)(t + 1);
            rd32 = 1.0f / (float)(t + 1);
        }
        __syncwarp();
        if (pushed)
            union_tail_item<LOG2P, F32>(a, t, (it - s_prefix[g]) * (32 / Cfg<LOG2P>::L), &s_cnt[wid], rd64,
                                        rd32, s_pow2);
        else
            batch_item<LOG2P, F32>(a, it - s_prefix[g], t, sparse, rd64, rd32, s_pow2, prefetch, &s_cnt[wid]);
    }
    __syncwarp();
    if (cur_g >= 0 && lane == 0 && s_cnt[wid]) atomicAdd(&B.args[cur_g].ctr->n_changed, s_cnt[wid]);
}

template <bool F32>
const void *batch_step_ptr(int lb) {
    switch (lb) {
#define HB_CASE(LB) case LB: return reinterpret_cast<const void *>(&batch_step_kernel<LB, F32>);
        HB_CASE(4) HB_CASE(5) HB_CASE(6) HB_CASE(7) HB_CASE(8) HB_CASE(9) HB_CASE(10) HB_CASE(11) HB_CASE(12)
#undef HB_CASE
        default: return nullptr;
    }
}

template <bool F32>
void launch_batch_step(int lb, int grid, size_t smem, cudaStream_t s, const BatchArrays &B) {
    switch (lb) {
#define HB_CASE(LB) case LB: batch_step_kernel<LB, F32><<<grid, kStepThreads, smem, s>>>(B); break;
        HB_CASE(4) HB_CASE(5) HB_CASE(6) HB_CASE(7) HB_CASE(8) HB_CASE(9) HB_CASE(10) HB_CASE(11) HB_CASE(12)
#undef HB_CASE
        default: break;
    }
}

// Changed-list compaction for graphs that ran a dense iteration.
__global__ void __launch_bounds__(256) batch_compact_kernel(BatchArrays B) {
    const int64_t total = B.tile_prefix[B.k];
    for (int64_t tile = blockIdx.x; tile < total; tile += gridDim.x) {
        const int g = find_graph(B.tile_prefix, B.k, tile);
        const StepArgs &a = B.args[g];
        if (a.ctr->mode != 0 || a.frontier == HB_FRONTIER_OFF) continue;
        compact_tile(a, a.ctr->t, (tile - B.tile_prefix[g]) * 256);
    }
}

__global__ void batch_end_kernel(BatchArrays B) {
    __shared__ int active;
    __shared__ unsigned long long arcs;
    if (threadIdx.x == 0) { active = 0; arcs = 0; }
    __syncthreads();
    for (int g = threadIdx.x; g < B.k; g += blockDim.x) {
        const StepArgs &a = B.args[g];
        Counters *c = a.ctr;
        if (c->mode != kMode_Idle) {
            end_one(a);
            const int64_t scanned = c->mode == 1 ? (int64_t)c->arcs : a.m;
            B.graph_arcs[g] += scanned;
            atomicAdd(&arcs, (unsigned long long)scanned);
        }
        if (!c->converged) atomicAdd(&active, 1);
        B.done[g] = c->converged ? 1 : 0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        BatchCtl *ctl = B.ctl;
        ctl->n_active = active;
        ctl->iterations += 1;
        ctl->total_arcs += arcs;
        if (B.use_cond)
            cudaGraphSetConditional(B.cond, (active > 0 && ctl->iterations < ctl->max_steps) ? 1u : 0u);
    }
}

// Sec. 5 (multiple runs): per node u of the caller's order, the mean and
// the empirical (sample, k-1) standard deviation over the k graphs of the
// batch of one centrality (which: 0 closeness, 1 harmonic, 2 Lin,
// 3 reachable), in two passes over the runs.  Graph r maps u to its own
// node index through invs[r] (null: identity) and reads its current
// counters (buffer of its completed-iteration parity).
template <bool F32>
__device__ __forceinline__ double run_value(const StepArgs &a, const int32_t *inv, int64_t u, int which) {
    const int64_t v = inv ? (int64_t)inv[u] : u;
    double c[4];
    node_centralities<F32>(a, a.regs[a.ctr->steps_done & 1], v, c);
    return c[which];
}

template <bool F32>
__global__ void run_stats_kernel(const StepArgs *args, const int32_t *const *invs, int k, int64_t n,
                                 int which, double *mean, double *sd) {
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n;
         u += (int64_t)gridDim.x * blockDim.x) {
        double sum = 0.0;
        for (int r = 0; r < k; ++r) sum += run_value<F32>(args[r], invs[r], u, which);
        const double mu = sum / (double)k;
        double q = 0.0;
        for (int r = 0; r < k; ++r) {
            const double d = run_value<F32>(args[r], invs[r], u, which) - mu;
            q += d * d;
        }
        if (mean) mean[u] = mu;
        if (sd) sd[u] = k > 1 ? sqrt(q / (double)(k - 1)) : 0.0;
    }
}

}  // namespace

}  // namespace hb

using namespace hb;

struct hb_batch {
    int k = 0;
    std::vector<hb_graph *> graphs;
    bool fp32 = false;
    bool own_stream = false;
    cudaStream_t s = nullptr;
    int step_grid = 0;
    int aux_grid = 0;
    DevMem mem;
    BatchArrays B{};
    BatchCtl *ctl_host = nullptr;
    cudaGraphExec_t step_exec = nullptr;
    cudaGraphExec_t run_exec = nullptr;
    cudaGraph_t step_graph = nullptr;
    cudaGraph_t run_graph = nullptr;
    int32_t max_steps = 1 << 20;
    unsigned log2m_mask = 0;
    int lb_grid[kMaxLog2m + 1] = {0};
    cudaStream_t side[kMaxLog2m + 1] = {nullptr};
    cudaEvent_t ev_fork = nullptr, ev_join[kMaxLog2m + 1] = {nullptr};

    ~hb_batch() {
        for (int i = 0; i <= kMaxLog2m; ++i) {
            if (side[i]) cudaStreamDestroy(side[i]);
            if (ev_join[i]) cudaEventDestroy(ev_join[i]);
        }
        if (ev_fork) cudaEventDestroy(ev_fork);
        if (step_exec) cudaGraphExecDestroy(step_exec);
        if (run_exec) cudaGraphExecDestroy(run_exec);
        if (step_graph) cudaGraphDestroy(step_graph);
        if (run_graph) cudaGraphDestroy(run_graph);
        // instances before the graph whose arrays they share
        for (size_t i = graphs.size(); i-- > 0;) hb_destroy(graphs[i]);
        if (ctl_host) cudaFreeHost(ctl_host);
        mem.free_all();
        if (own_stream && s) cudaStreamDestroy(s);
    }
};

namespace {

hb_status bfail(hb_status st, const std::string &m) {
    set_last_error(m.c_str());
    return st;
}

// The kernels of one batched iteration, enqueued on b->s (captured).
cudaError_t enqueue_iteration(hb_batch *b, const BatchArrays &B) {
    cudaStream_t s = b->s;
    batch_begin_kernel<<<1, 1024, 0, s>>>(B);
    batch_clear_bits_kernel<<<b->aux_grid, 256, 0, s>>>(B);
    batch_mark_push_kernel<<<b->step_grid, kStepThreads, 0, s>>>(B);
    batch_push_union_kernel<<<b->step_grid, kStepThreads, 0, s>>>(B);
    batch_copy_forward_kernel<<<b->aux_grid, 256, 0, s>>>(B);
    batch_plan_kernel<<<b->k < 65535 ? b->k : 65535, 1024, 0, s>>>(B);
    batch_items_kernel<<<1, 1024, 0, s>>>(B);
    const size_t smem = sizeof(int64_t) * (size_t)(B.k + 1);
    // one gather kernel per log2m present, as parallel branches
    cudaEventRecord(b->ev_fork, s);
    for (int lb = kMinLog2m; lb <= kMaxLog2m; ++lb) {
        if (!((b->log2m_mask >> (lb - kMinLog2m)) & 1u)) continue;
        cudaStreamWaitEvent(b->side[lb], b->ev_fork, 0);
        if (b->fp32) launch_batch_step<true>(lb, b->lb_grid[lb], smem, b->side[lb], B);
        else launch_batch_step<false>(lb, b->lb_grid[lb], smem, b->side[lb], B);
        cudaEventRecord(b->ev_join[lb], b->side[lb]);
        cudaStreamWaitEvent(s, b->ev_join[lb], 0);
    }
    batch_compact_kernel<<<b->aux_grid, 256, 0, s>>>(B);
    batch_end_kernel<<<1, 1024, 0, s>>>(B);
    return cudaGetLastError();
}

hb_status build_graphs(hb_batch *b) {
    cudaError_t e = cudaStreamBeginCapture(b->s, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        BatchArrays B = b->B;
        B.use_cond = 0;
        e = enqueue_iteration(b, B);
        cudaError_t e2 = cudaStreamEndCapture(b->s, &b->step_graph);
        if (e == cudaSuccess) e = e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->step_exec, b->step_graph, 0);
    if (e != cudaSuccess) return bfail(HB_ERR_CUDA, std::string("batch iteration graph: ") + cudaGetErrorString(e));

    // run to every fixpoint: while (active && iterations < cap) { iteration }
    e = cudaGraphCreate(&b->run_graph, 0);
    cudaGraphConditionalHandle cond;
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&cond, b->run_graph, 1, cudaGraphCondAssignDefault);
    cudaGraphNodeParams cp = {};
    cudaGraphNode_t node;
    if (e == cudaSuccess) {
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = cond;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        e = cudaGraphAddNode(&node, b->run_graph, nullptr, nullptr, 0, &cp);
    }
    if (e == cudaSuccess) {
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        e = cudaStreamBeginCaptureToGraph(b->s, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            BatchArrays B = b->B;
            B.use_cond = 1;
            B.cond = cond;
            e = enqueue_iteration(b, B);
            cudaGraph_t out = nullptr;
            cudaError_t e2 = cudaStreamEndCapture(b->s, &out);
            if (e == cudaSuccess) e = e2;
        }
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->run_exec, b->run_graph, 0);
    if (e != cudaSuccess) return bfail(HB_ERR_CUDA, std::string("batch loop graph: ") + cudaGetErrorString(e));
    return HB_OK;
}

hb_status reset_ctl(hb_batch *b) {
    BatchCtl c{};
    c.k = b->k;
    c.max_steps = b->max_steps;
    cudaError_t e = cudaMemcpyAsync(b->B.ctl, &c, sizeof(c), cudaMemcpyHostToDevice, b->s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->B.graph_arcs, 0, sizeof(int64_t) * b->k, b->s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->s);
    if (e != cudaSuccess) return bfail(HB_ERR_CUDA, std::string("batch reset: ") + cudaGetErrorString(e));
    return HB_OK;
}

hb_status read_ctl(hb_batch *b) {
    cudaError_t e = cudaMemcpyAsync(b->ctl_host, b->B.ctl, sizeof(BatchCtl), cudaMemcpyDeviceToHost, b->s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->s);
    if (e != cudaSuccess) return bfail(HB_ERR_CUDA, std::string("batch: ") + cudaGetErrorString(e));
    return HB_OK;
}

// Device arrays, launch shape and captured graphs of a batch of k slots.
hb_status batch_setup(hb_batch *b, const std::vector<StepArgs> &hargs, const std::vector<int64_t> &tiles) {
    const int k = b->k;
    DevMem &M = b->mem;
    StepArgs *args = M.alloc<StepArgs>(k);
    int64_t *pref = M.alloc<int64_t>((size_t)17 * (k + 1));
    int64_t *garcs = M.alloc<int64_t>(k);
    int32_t *done = M.alloc<int32_t>(k);
    BatchCtl *ctl = M.alloc<BatchCtl>(1);
    if (M.err != cudaSuccess || (!b->ctl_host && cudaMallocHost(&b->ctl_host, sizeof(BatchCtl)) != cudaSuccess))
        return bfail(HB_ERR_OOM, "out of memory (batch arrays)");
    cudaError_t e = cudaMemcpyAsync(args, hargs.data(), sizeof(StepArgs) * k, cudaMemcpyHostToDevice, b->s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(pref + 5 * (k + 1), tiles.data(), sizeof(int64_t) * (k + 1), cudaMemcpyHostToDevice, b->s);
    if (e == cudaSuccess) e = cudaMemsetAsync(done, 0, sizeof(int32_t) * k, b->s);
    if (e != cudaSuccess) return bfail(HB_ERR_CUDA, "batch upload");
    BatchArrays &B = b->B;
    B.args = args;
    B.item_prefix = pref + 6 * (k + 1);   // 9 arrays, one per log2m (6 .. 14)
    B.push_prefix = pref + 15 * (k + 1);
    B.pbig_prefix = pref + 16 * (k + 1);
    B.list_prefix = pref + (k + 1);
    B.big_prefix = pref + 2 * (k + 1);
    B.copy_prefix = pref + 3 * (k + 1);
    B.word_prefix = pref + 4 * (k + 1);
    B.tile_prefix = pref + 5 * (k + 1);
    B.log2m_mask = b->log2m_mask;
    B.graph_arcs = garcs;
    B.done = done;
    B.ctl = ctl;
    B.k = k;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t smem = sizeof(int64_t) * (size_t)(k + 1);
    if (cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) != cudaSuccess)
        return bfail(HB_ERR_CUDA, "batch events");
    for (int lb = kMinLog2m; lb <= kMaxLog2m; ++lb) {
        if (!((b->log2m_mask >> (lb - kMinLog2m)) & 1u)) continue;
        const void *fn = b->fp32 ? batch_step_ptr<true>(lb) : batch_step_ptr<false>(lb);
        if (smem > 48 * 1024) cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int per = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, kStepThreads, smem);
        b->lb_grid[lb] = sms * (per > 0 ? per : 1);
        if (cudaStreamCreateWithFlags(&b->side[lb], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&b->ev_join[lb], cudaEventDisableTiming) != cudaSuccess)
            return bfail(HB_ERR_CUDA, "batch streams");
    }
    b->step_grid = sms * 6;
    b->aux_grid = sms * 8;
    hb_status st = reset_ctl(b);
    if (st == HB_OK) st = build_graphs(b);
    return st;
}

// A batch of k slots with the options' stream (or its own), before its
// graphs are added.
hb_status new_batch(int k, const hb_options *opt, hb_options *o, hb_batch **out) {
    if (opt) *o = *opt; else hb_default_options(o);
    if (o->max_steps <= 0) o->max_steps = 1 << 20;
    if (o->frontier == HB_FRONTIER_PULL) o->frontier = HB_FRONTIER_AUTO;
    o->flags &= ~(uint32_t)HB_PROFILE;
    if (o->flags & HB_PACKED_REGISTERS) return bfail(HB_ERR_INVALID, "batches hold byte registers, not HB_PACKED_REGISTERS");
    hb_batch *b = new hb_batch();
    b->k = k;
    b->fp32 = (o->flags & HB_FP32_ESTIMATE) != 0;
    b->max_steps = o->max_steps;
    if (o->stream) {
        b->s = static_cast<cudaStream_t>(o->stream);
    } else {
        if (cudaStreamCreateWithFlags(&b->s, cudaStreamNonBlocking) != cudaSuccess) {
            delete b;
            return bfail(HB_ERR_CUDA, "cannot create the batch stream");
        }
        b->own_stream = true;
    }
    o->stream = b->s;
    *out = b;
    return HB_OK;
}

// Per-graph arguments, tiles and captured graphs once every graph is in.
hb_status finish_batch(hb_batch *b) {
    const int k = b->k;
    std::vector<StepArgs> hargs(k);
    std::vector<int64_t> tiles(k + 1, 0);
    for (int i = 0; i < k; ++i) {
        hargs[i] = b->graphs[i]->a;
        tiles[i + 1] = tiles[i] + (b->graphs[i]->n + 255) / 256;
        b->log2m_mask |= 1u << (b->graphs[i]->b - kMinLog2m);
    }
    return batch_setup(b, hargs, tiles);
}

}  // namespace

extern "C" {

hb_status hb_batch_create(int k, const hb_graph_desc *gs, const hb_options *opt, hb_batch **out) {
    set_last_error("");
    if (!out) return bfail(HB_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (k < 1 || k > kMaxBatch) return bfail(HB_ERR_INVALID, "k must lie in [1, 4096]");
    if (!gs) return bfail(HB_ERR_INVALID, "gs is NULL");
    hb_options o;
    hb_batch *b = nullptr;
    hb_status st0 = new_batch(k, opt, &o, &b);
    if (st0 != HB_OK) return st0;
    for (int i = 0; i < k; ++i) {
        hb_graph *g = nullptr;
        hb_status st = create_handle64(gs[i].offsets, gs[i].targets, gs[i].n, gs[i].m, gs[i].log2m,
                                       gs[i].seed, &o, &g);
        if (st != HB_OK) {
            std::string msg = std::string("graph ") + std::to_string(i) + ": " + hb_last_error();
            delete b;
            return bfail(st, msg);
        }
        b->graphs.push_back(g);
    }
    hb_status st = finish_batch(b);
    if (st != HB_OK) { delete b; return st; }
    *out = b;
    return HB_OK;
}

hb_status hb_batch_create_runs(const int64_t *offsets, const int32_t *targets, int64_t n, int64_t m,
                               int log2m, int runs, const uint64_t *seeds, const hb_options *opt,
                               hb_batch **out) {
    set_last_error("");
    if (!out) return bfail(HB_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (runs < 1 || runs > kMaxBatch) return bfail(HB_ERR_INVALID, "runs must lie in [1, 4096]");
    if (!seeds) return bfail(HB_ERR_INVALID, "seeds is NULL");
    hb_options o;
    hb_batch *b = nullptr;
    hb_status st = new_batch(runs, opt, &o, &b);
    if (st != HB_OK) return st;
    hb_graph *tmpl = nullptr;
    st = create_handle64(offsets, targets, n, m, log2m, seeds[0], &o, &tmpl);
    if (st != HB_OK) { delete b; return st; }
    b->graphs.push_back(tmpl);
    // the other runs share the first one's graph, layout and tables
    for (int r = 1; r < runs; ++r) {
        hb_graph *g = nullptr;
        st = make_instance(tmpl, seeds[r], b->s, &g);
        if (st != HB_OK) { delete b; return st; }
        b->graphs.push_back(g);
    }
    st = finish_batch(b);
    if (st != HB_OK) { delete b; return st; }
    *out = b;
    return HB_OK;
}

hb_status hb_batch_get_run_stats(hb_batch *b, int32_t which, double *mean, double *sd) {
    if (!b) return bfail(HB_ERR_INVALID, "batch is NULL");
    if (which < 0 || which > 3) return bfail(HB_ERR_INVALID, "which must lie in [0, 3]");
    const int64_t n = b->graphs[0]->n;
    for (hb_graph *g : b->graphs)
        if (g->n != n) return bfail(HB_ERR_INVALID, "run statistics need graphs of one node count");
    if (n > 0 && !mean && !sd) return bfail(HB_ERR_INVALID, "mean and sd are both NULL");
    DevMem tmp;
    std::vector<const int32_t *> inv_h(b->k);
    for (int i = 0; i < b->k; ++i) inv_h[i] = b->graphs[i]->inv;
    auto dev_or_tmp = [&](double *p) -> double * {
        if (!p) return nullptr;
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, p) == cudaSuccess &&
            (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged))
            return p;
        cudaGetLastError();
        return tmp.alloc<double>(n);
    };
    double *dm = dev_or_tmp(mean), *ds = dev_or_tmp(sd);
    const int32_t **invs = tmp.alloc<const int32_t *>(b->k);
    if (tmp.err != cudaSuccess) { tmp.free_all(); return bfail(HB_ERR_OOM, "out of device memory"); }
    cudaError_t e = cudaMemcpyAsync(invs, inv_h.data(), sizeof(const int32_t *) * b->k,
                                    cudaMemcpyHostToDevice, b->s);
    if (e == cudaSuccess && n > 0) {
        if (b->fp32)
            run_stats_kernel<true><<<grid_for(n, 256), 256, 0, b->s>>>(b->B.args, invs, b->k, n, which, dm, ds);
        else
            run_stats_kernel<false><<<grid_for(n, 256), 256, 0, b->s>>>(b->B.args, invs, b->k, n, which, dm, ds);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && mean && dm != mean)
        e = cudaMemcpyAsync(mean, dm, sizeof(double) * n, cudaMemcpyDeviceToHost, b->s);
    if (e == cudaSuccess && sd && ds != sd)
        e = cudaMemcpyAsync(sd, ds, sizeof(double) * n, cudaMemcpyDeviceToHost, b->s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->s);
    tmp.free_all();
    if (e != cudaSuccess) return bfail(HB_ERR_CUDA, std::string("run statistics: ") + cudaGetErrorString(e));
    return HB_OK;
}

hb_status hb_batch_step(hb_batch *b, int32_t *n_active) {
    if (!b) return bfail(HB_ERR_INVALID, "batch is NULL");
    NvtxRange nv("hb_batch_step");
    cudaError_t e = cudaGraphLaunch(b->step_exec, b->s);
    if (e != cudaSuccess) return bfail(HB_ERR_CUDA, std::string("batch step: ") + cudaGetErrorString(e));
    hb_status st = read_ctl(b);
    if (st != HB_OK) return st;
    if (n_active) *n_active = b->ctl_host->n_active;
    return HB_OK;
}

hb_status hb_batch_run(hb_batch *b, int32_t *iterations) {
    if (!b) return bfail(HB_ERR_INVALID, "batch is NULL");
    NvtxRange nv("hb_batch_run");
    cudaError_t e = cudaGraphLaunch(b->run_exec, b->s);
    if (e != cudaSuccess) return bfail(HB_ERR_CUDA, std::string("batch run: ") + cudaGetErrorString(e));
    hb_status st = read_ctl(b);
    if (st != HB_OK) return st;
    if (iterations) *iterations = b->ctl_host->iterations;
    if (b->ctl_host->n_active > 0)
        return bfail(HB_ERR_NOT_CONVERGED, "the iteration cap was reached before every graph converged");
    return HB_OK;
}

hb_status hb_batch_reset(hb_batch *b, const uint64_t *seeds) {
    if (!b) return bfail(HB_ERR_INVALID, "batch is NULL");
    for (int i = 0; i < b->k; ++i) {
        hb_graph *g = b->graphs[i];
        hb_status st = hb_reset(g, seeds ? seeds[i] : g->seed);
        if (st != HB_OK) return st;
    }
    return reset_ctl(b);
}

static hb_status graph_of(hb_batch *b, int i, hb_graph **g) {
    if (!b) return bfail(HB_ERR_INVALID, "batch is NULL");
    if (i < 0 || i >= b->k) return bfail(HB_ERR_INVALID, "graph index out of range");
    *g = b->graphs[i];
    return sync_host_state(*g);
}

hb_status hb_batch_get_centralities(hb_batch *b, int i, double *closeness, double *harmonic,
                                    double *lin, double *reachable) {
    hb_graph *g;
    hb_status st = graph_of(b, i, &g);
    return st != HB_OK ? st : hb_get_centralities(g, closeness, harmonic, lin, reachable);
}

hb_status hb_batch_get_registers(hb_batch *b, int i, uint8_t *out) {
    hb_graph *g;
    hb_status st = graph_of(b, i, &g);
    return st != HB_OK ? st : hb_get_registers(g, out);
}

hb_status hb_batch_get_accumulators(hb_batch *b, int i, double *sumd, double *harm) {
    hb_graph *g;
    hb_status st = graph_of(b, i, &g);
    return st != HB_OK ? st : hb_get_accumulators(g, sumd, harm);
}

hb_status hb_batch_get_info(hb_batch *b, int i, hb_info *info) {
    hb_graph *g;
    hb_status st = graph_of(b, i, &g);
    if (st != HB_OK) return st;
    st = hb_get_info(g, info);
    if (st != HB_OK) return st;
    int64_t arcs = 0;
    cudaError_t e = cudaMemcpy(&arcs, b->B.graph_arcs + i, sizeof(arcs), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return bfail(HB_ERR_CUDA, "batch info");
    info->total_arcs = arcs;
    return HB_OK;
}

hb_status hb_batch_tune(hb_batch *b, int32_t *arcs_per_slot) {
    if (!b) return bfail(HB_ERR_INVALID, "batch is NULL");
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return bfail(HB_ERR_CUDA, "tuning events");
    auto apply = [&](int aps) -> hb_status {
        std::vector<StepArgs> hargs(b->k);
        for (int i = 0; i < b->k; ++i) {
            hb_graph *g = b->graphs[i];
            hb_status st = retune(g, aps);
            if (st == HB_OK) st = hb_reset(g, g->seed);
            if (st != HB_OK) return st;
            hargs[i] = g->a;
        }
        cudaError_t e = cudaMemcpyAsync(const_cast<StepArgs *>(b->B.args), hargs.data(), sizeof(StepArgs) * b->k,
                                        cudaMemcpyHostToDevice, b->s);
        if (e != cudaSuccess) return bfail(HB_ERR_CUDA, "batch tune upload");
        return reset_ctl(b);
    };
    // as hb_tune: every candidate twice, ascending then descending
    constexpr int nc = sizeof(kTuneAps) / sizeof(kTuneAps[0]);
    float cand_ms[nc];
    for (float &x : cand_ms) x = 1e30f;
    hb_status st = HB_OK;
    for (int pass = 0; pass < 2 * nc; ++pass) {
        const int ci = pass < nc ? pass : 2 * nc - 1 - pass;
        st = apply(kTuneAps[ci]);
        if (st != HB_OK) break;
        cudaEventRecord(e0, b->s);
        for (int i = 0; i < kTuneIters; ++i) cudaGraphLaunch(b->step_exec, b->s);
        cudaEventRecord(e1, b->s);
        float ms = 0.f;
        if (cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess &&
            ms < cand_ms[ci])
            cand_ms[ci] = ms;
    }
    int best = kArcsPerSlot;
    float best_ms = 1e30f;
    for (int ci = 0; ci < nc; ++ci)
        if (cand_ms[ci] < best_ms) {
            best_ms = cand_ms[ci];
            best = kTuneAps[ci];
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st == HB_OK) st = apply(best);
    if (st == HB_OK && arcs_per_slot) *arcs_per_slot = best;
    return st;
}

hb_status hb_batch_get_totals(hb_batch *b, int32_t *iterations, int32_t *n_active, int64_t *arcs) {
    if (!b) return bfail(HB_ERR_INVALID, "batch is NULL");
    hb_status st = read_ctl(b);
    if (st != HB_OK) return st;
    if (iterations) *iterations = b->ctl_host->iterations;
    if (n_active) *n_active = b->ctl_host->n_active;
    if (arcs) *arcs = (int64_t)b->ctl_host->total_arcs;
    return HB_OK;
}

void hb_batch_destroy(hb_batch *b) {
    if (!b) return;
    if (b->s) cudaStreamSynchronize(b->s);
    delete b;
}

}  // extern "C"

// ------------------------------------------------------------------ serving --
// A request loop over the batched kernels: a fixed number of slots, each
// holding one running request (graph from the server's pool, log2m, seed)
// with its counters resident on the device.  Between iterations, queued
// requests are admitted into free slots while device memory allows, and
// requests whose counters stopped changing are finalised, copied to the
// host and their memory freed; all running requests advance in the same
// launches (continuous batching).

#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>

namespace {

struct ServeReq {
    int graph = 0, log2m = 4;
    uint64_t seed = 0;
    int state = HB_REQ_QUEUED;
    double t_submit = 0, t_admit = 0, t_done = 0;
    hb_graph *inst = nullptr;
    int slot = -1;
    int32_t steps = 0;
    int64_t arcs = 0;
    hb_status err = HB_OK;
    int64_t n = 0;
    double *dres = nullptr;   // device: closeness, harmonic, lin, reachable (n each)
    bool cancel = false;      // running: retire at the next iteration boundary
    bool large = false;       // its graph has at least large_arcs arcs
};

struct PoolGraph {
    int64_t *off = nullptr;
    int32_t *tgt = nullptr;
    int64_t n = 0, m = 0;
    std::map<int, hb_graph *> tmpl;   // per log2m: relabelled CSR, reverse CSR, plans
};

}  // namespace

struct hb_server {
    hb_server_options opt{};
    hb_batch *batch = nullptr;
    DevMem mem;
    cudaMemPool_t pool = nullptr;       // per-request state and results, stream-ordered
    Counters *ctr_host = nullptr;       // pinned counter block shared by the server's instances
    cudaStream_t copy_stream = nullptr; // result copies to the client
    Counters *null_ctr = nullptr;
    std::vector<StepArgs> slot_args;
    std::vector<int64_t> slot_req;
    std::vector<int64_t> tiles;
    std::vector<PoolGraph> graphs;
    std::map<int64_t, ServeReq> reqs;
    std::deque<int64_t> queue;
    int64_t next_id = 1;
    std::mutex mu;
    std::condition_variable cv, done_cv;
    std::thread th;
    bool stop = false;
    std::chrono::steady_clock::time_point t0;
    int64_t iterations = 0, total_arcs = 0, completed = 0;
    double busy_s = 0;
    std::string fatal;

    double now() const {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    ~hb_server() {
        {
            std::lock_guard<std::mutex> lk(mu);
            stop = true;
        }
        cv.notify_all();
        if (th.joinable()) th.join();
        cudaStream_t s = batch ? batch->s : nullptr;
        for (auto &kv : reqs) {
            if (kv.second.inst) hb_destroy(kv.second.inst);
            if (kv.second.dres) cudaFreeAsync(kv.second.dres, s);
        }
        for (auto &pg : graphs)
            for (auto &kv : pg.tmpl) hb_destroy(kv.second);
        if (s) cudaStreamSynchronize(s);
        if (copy_stream) { cudaStreamSynchronize(copy_stream); cudaStreamDestroy(copy_stream); }
        delete batch;
        mem.free_all();
        if (pool) cudaMemPoolDestroy(pool);
        if (ctr_host) cudaFreeHost(ctr_host);
    }
};

namespace {

StepArgs null_slot(hb_server *S, int slot) {
    StepArgs a{};
    a.ctr = S->null_ctr + slot;
    a.b = 4;
    a.frontier = HB_FRONTIER_OFF;
    return a;
}

// Put the slot's arguments (and the node tiles of every slot) on the device.
cudaError_t publish_slots(hb_server *S) {
    hb_batch *b = S->batch;
    const int k = b->k;
    S->tiles.assign(k + 1, 0);
    for (int i = 0; i < k; ++i) S->tiles[i + 1] = S->tiles[i] + (S->slot_args[i].n + 255) / 256;
    cudaError_t e = cudaMemcpyAsync(const_cast<StepArgs *>(b->B.args), S->slot_args.data(),
                                    sizeof(StepArgs) * k, cudaMemcpyHostToDevice, b->s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(const_cast<int64_t *>(b->B.tile_prefix), S->tiles.data(), sizeof(int64_t) * (k + 1),
                            cudaMemcpyHostToDevice, b->s);
    return e;
}

void serve_loop(hb_server *S) {
    hb_batch *b = S->batch;
    const int k = b->k;
    std::vector<int32_t> done(k);
    std::vector<int64_t> garcs(k);
    std::vector<ServeReq *> running_req(k, nullptr);
    std::vector<char> fresh(k, 0);
    for (;;) {
        bool changed = false;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            // admission: FIFO, into free slots, while device memory allows;
            // with a large-request limit, large requests beyond it stay
            // queued (in order) and the requests behind them go first
            bool trimmed = false;
            int large_running = 0;
            if (S->opt.large_slots > 0)
                for (int q = 0; q < k; ++q)
                    if (S->slot_req[q] >= 0 && S->reqs[S->slot_req[q]].large) ++large_running;
            for (int slot = 0; slot < k && !S->queue.empty(); ++slot) {
                if (S->slot_req[slot] >= 0) continue;
                auto qit = S->queue.begin();
                if (S->opt.large_slots > 0 && large_running >= S->opt.large_slots)
                    while (qit != S->queue.end() && S->reqs[*qit].large) ++qit;
                if (qit == S->queue.end()) break;
                const int64_t id = *qit;
                ServeReq &r = S->reqs[id];
                hb_graph *tmpl = S->graphs[r.graph].tmpl[r.log2m];
                // admission by device memory: free memory plus what the
                // server's pool holds but does not use
                size_t free_b = 0, total_b = 0, reserved = 0, used = 0;
                cudaMemGetInfo(&free_b, &total_b);
                cudaMemPoolGetAttribute(S->pool, cudaMemPoolAttrReservedMemCurrent, &reserved);
                cudaMemPoolGetAttribute(S->pool, cudaMemPoolAttrUsedMemCurrent, &used);
                const int64_t avail = (int64_t)free_b + (int64_t)(reserved - used);
                const int64_t need = (int64_t)run_bytes(tmpl) + 32 * tmpl->n + 4096;
                bool any_running = false;
                for (int q = 0; q < k; ++q) any_running |= S->slot_req[q] >= 0;
                if (need + S->opt.reserve_bytes > (int64_t)total_b ||
                    (trimmed && !any_running && avail < need + S->opt.reserve_bytes)) {
                    // can never fit, or does not fit while none of the
                    // server's requests holds memory: refuse it
                    qit = S->queue.erase(qit);
                    r.state = HB_REQ_FAILED;
                    r.err = HB_ERR_OOM;
                    r.t_done = S->now();
                    S->done_cv.notify_all();
                    --slot;
                    continue;
                }
                if (avail < need + S->opt.reserve_bytes) {
                    // memory cached by the library's own pool (freed by
                    // handles destroyed earlier) goes back to the device first
                    cudaMemPool_t lib = library_pool();
                    size_t lres = 0, lused = 0;
                    if (!trimmed && lib &&
                        cudaMemPoolGetAttribute(lib, cudaMemPoolAttrReservedMemCurrent, &lres) == cudaSuccess &&
                        cudaMemPoolGetAttribute(lib, cudaMemPoolAttrUsedMemCurrent, &lused) == cudaSuccess &&
                        lres > lused && avail + (int64_t)(lres - lused) >= need + S->opt.reserve_bytes) {
                        cudaStreamSynchronize(b->s);
                        cudaMemPoolTrimTo(lib, lused);
                        trimmed = true;   // once per admission pass
                        --slot;
                        continue;
                    }
                    if (!trimmed && !any_running) {   // refused above on the next look
                        trimmed = true;
                        --slot;
                        continue;
                    }
                    break;
                }
                qit = S->queue.erase(qit);
                lk.unlock();
                hb_graph *inst = nullptr;
                hb_status st = make_instance(tmpl, r.seed, b->s, &inst, S->pool, S->ctr_host);
                lk.lock();
                if (st != HB_OK) {
                    r.state = HB_REQ_FAILED;
                    r.err = st;
                    r.t_done = S->now();
                    S->done_cv.notify_all();
                    --slot;
                    continue;
                }
                if (r.large) ++large_running;
                r.inst = inst;
                r.slot = slot;
                r.state = HB_REQ_RUNNING;
                r.t_admit = S->now();
                S->slot_req[slot] = id;
                S->slot_args[slot] = inst->a;
                running_req[slot] = &r;
                fresh[slot] = 1;
                changed = true;
            }
            bool running = false;
            for (int slot = 0; slot < k; ++slot) running |= S->slot_req[slot] >= 0;
            if (!running) {
                if (S->stop) return;
                S->cv.wait(lk);
                continue;
            }
        }
        const double t_start = S->now();
        NvtxRange nv("serve iteration");
        cudaError_t e = cudaSuccess;
        if (changed) {
            e = publish_slots(S);
            for (int slot = 0; slot < k && e == cudaSuccess; ++slot)
                if (fresh[slot]) {
                    e = cudaMemsetAsync(b->B.graph_arcs + slot, 0, sizeof(int64_t), b->s);
                    fresh[slot] = 0;
                }
        }
        if (e == cudaSuccess) e = cudaGraphLaunch(b->step_exec, b->s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(done.data(), b->B.done, sizeof(int32_t) * k, cudaMemcpyDeviceToHost, b->s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(garcs.data(), b->B.graph_arcs, sizeof(int64_t) * k, cudaMemcpyDeviceToHost, b->s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->s);
        if (e != cudaSuccess) {
            std::lock_guard<std::mutex> lk(S->mu);
            S->fatal = cudaGetErrorString(e);
            for (auto &kv : S->reqs)
                if (kv.second.state == HB_REQ_RUNNING || kv.second.state == HB_REQ_QUEUED) {
                    kv.second.state = HB_REQ_FAILED;
                    kv.second.err = HB_ERR_CUDA;
                }
            S->done_cv.notify_all();
            return;
        }
        ++S->iterations;
        bool freed = false;
        for (int slot = 0; slot < k; ++slot) {
            if (!running_req[slot]) continue;
            ServeReq &r = *running_req[slot];
            r.steps += 1;
            const bool capped = r.steps >= S->opt.max_steps;
            bool cancel;
            {
                std::lock_guard<std::mutex> lk(S->mu);
                cancel = r.cancel;
            }
            if (cancel) {
                // retired without results; the other slots are untouched
                hb_destroy(r.inst);
                std::lock_guard<std::mutex> lk(S->mu);
                r.inst = nullptr;
                r.slot = -1;
                r.err = HB_ERR_STATE;
                r.state = HB_REQ_CANCELLED;
                r.t_done = S->now();
                S->slot_req[slot] = -1;
                S->slot_args[slot] = null_slot(S, slot);
                running_req[slot] = nullptr;
                freed = true;
                S->done_cv.notify_all();
                continue;
            }
            if (!done[slot] && !capped) continue;
            hb_graph *inst = r.inst;
            hb_status st = sync_host_state(inst);
            // results stay on the device until the client takes them; the
            // counters and the rest of the run state are freed now
            double *dres = nullptr;
            if (st == HB_OK && cudaMallocFromPoolAsync(reinterpret_cast<void **>(&dres),
                                                       sizeof(double) * 4 * (size_t)(inst->n > 0 ? inst->n : 1),
                                                       S->pool, b->s) != cudaSuccess) {
                cudaGetLastError();
                dres = nullptr;
                st = HB_ERR_OOM;
            }
            const size_t nn = (size_t)inst->n;
            if (st == HB_OK)
                st = hb_get_centralities(inst, dres, dres + nn, dres + 2 * nn, dres + 3 * nn);
            r.steps = inst->t;
            r.arcs = garcs[slot];
            r.n = inst->n;
            hb_destroy(inst);
            if (st != HB_OK && dres) { cudaFreeAsync(dres, b->s); dres = nullptr; }
            r.dres = dres;
            std::lock_guard<std::mutex> lk(S->mu);
            r.inst = nullptr;
            r.slot = -1;
            r.err = st != HB_OK ? st : (done[slot] ? HB_OK : HB_ERR_NOT_CONVERGED);
            r.state = r.err == HB_OK ? HB_REQ_DONE : HB_REQ_FAILED;
            r.t_done = S->now();
            S->total_arcs += r.arcs;
            S->completed += 1;
            S->slot_req[slot] = -1;
            S->slot_args[slot] = null_slot(S, slot);
            running_req[slot] = nullptr;
            freed = true;
            S->done_cv.notify_all();
        }
        if (freed) publish_slots(S);
        std::lock_guard<std::mutex> lk(S->mu);
        S->busy_s += S->now() - t_start;
    }
}

hb_status sfail(hb_status st, const std::string &m) {
    set_last_error(m.c_str());
    return st;
}

}  // namespace

extern "C" {

void hb_server_default_options(hb_server_options *o) {
    if (!o) return;
    o->slots = 32;
    o->flags = 0;
    o->max_steps = 1 << 16;
    o->reserve_bytes = (int64_t)4 << 30;
    o->large_arcs = (int64_t)1 << 25;
    o->large_slots = 0;
}

hb_status hb_server_create(const hb_server_options *opt, hb_server **out) {
    set_last_error("");
    if (!out) return sfail(HB_ERR_INVALID, "out is NULL");
    *out = nullptr;
    hb_server_options o;
    if (opt) o = *opt; else hb_server_default_options(&o);
    if (o.slots < 1 || o.slots > kMaxBatch) return sfail(HB_ERR_INVALID, "slots must lie in [1, 4096]");
    if (o.max_steps <= 0) o.max_steps = 1 << 16;
    if (o.reserve_bytes < 0) o.reserve_bytes = 0;
    if (o.large_slots < 0 || o.large_arcs < 0) return sfail(HB_ERR_INVALID, "large_slots and large_arcs must be >= 0");
    if (o.flags & HB_PACKED_REGISTERS) return sfail(HB_ERR_INVALID, "servers hold byte registers, not HB_PACKED_REGISTERS");
    cudaFree(nullptr);
    hb_server *S = new hb_server();
    S->opt = o;
    S->t0 = std::chrono::steady_clock::now();
    hb_batch *b = new hb_batch();
    S->batch = b;
    b->k = o.slots;
    b->fp32 = (o.flags & HB_FP32_ESTIMATE) != 0;
    b->max_steps = 1 << 30;
    b->log2m_mask = (1u << (kMaxLog2m - kMinLog2m + 1)) - 1;   // requests may use any log2m
    if (cudaStreamCreateWithFlags(&b->s, cudaStreamNonBlocking) != cudaSuccess) {
        delete S;
        return sfail(HB_ERR_CUDA, "cannot create the server stream");
    }
    b->own_stream = true;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    uint64_t keep = UINT64_MAX;
    if (cudaMemPoolCreate(&S->pool, &props) != cudaSuccess ||
        cudaMemPoolSetAttribute(S->pool, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess ||
        cudaMallocHost(&S->ctr_host, sizeof(Counters)) != cudaSuccess ||
        cudaStreamCreateWithFlags(&S->copy_stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete S;
        return sfail(HB_ERR_CUDA, "server memory pool or streams");
    }
    S->null_ctr = S->mem.alloc<Counters>(o.slots);
    if (!S->null_ctr) { delete S; return sfail(HB_ERR_OOM, "out of device memory"); }
    std::vector<Counters> nc(o.slots);
    for (auto &c : nc) { std::memset(&c, 0, sizeof(c)); c.converged = 1; }
    if (cudaMemcpy(S->null_ctr, nc.data(), sizeof(Counters) * o.slots, cudaMemcpyHostToDevice) != cudaSuccess) {
        delete S;
        return sfail(HB_ERR_CUDA, "server set-up");
    }
    S->slot_args.resize(o.slots);
    S->slot_req.assign(o.slots, -1);
    for (int i = 0; i < o.slots; ++i) S->slot_args[i] = null_slot(S, i);
    std::vector<int64_t> tiles(o.slots + 1, 0);
    hb_status st = batch_setup(b, S->slot_args, tiles);
    if (st != HB_OK) { delete S; return st; }
    S->th = std::thread(serve_loop, S);
    *out = S;
    return HB_OK;
}

hb_status hb_server_add_graph(hb_server *S, const int64_t *offsets, const int32_t *targets, int64_t n,
                              int64_t m, const int32_t *log2ms, int n_log2m, int32_t *graph_id) {
    if (!S || !graph_id || !log2ms || n_log2m < 1) return sfail(HB_ERR_INVALID, "NULL argument");
    hb_options o;
    hb_default_options(&o);
    o.flags = (S->opt.flags & HB_FP32_ESTIMATE) | HB_BORROW_DEVICE_PTRS;
    o.stream = nullptr;
    PoolGraph pg;
    pg.n = n;
    pg.m = m;
    // the pool keeps its own device copy of the CSR
    pg.off = S->mem.alloc<int64_t>(n + 1);
    pg.tgt = S->mem.alloc<int32_t>(m);
    if (S->mem.err != cudaSuccess) return sfail(HB_ERR_OOM, "out of device memory (pool graph)");
    cudaError_t e = cudaMemcpy(pg.off, offsets, sizeof(int64_t) * (n + 1), cudaMemcpyDefault);
    if (e == cudaSuccess && m > 0) e = cudaMemcpy(pg.tgt, targets, sizeof(int32_t) * m, cudaMemcpyDefault);
    if (e != cudaSuccess) return sfail(HB_ERR_CUDA, std::string("pool upload: ") + cudaGetErrorString(e));
    for (int i = 0; i < n_log2m; ++i) {
        hb_graph *t = nullptr;
        hb_status st = create_handle64(pg.off, pg.tgt, n, m, log2ms[i], 0, &o, &t);
        if (st != HB_OK) {
            for (auto &kv : pg.tmpl) hb_destroy(kv.second);
            return st;
        }
        drop_run_state(t);
        pg.tmpl[log2ms[i]] = t;
    }
    std::lock_guard<std::mutex> lk(S->mu);
    S->graphs.push_back(std::move(pg));
    *graph_id = (int32_t)S->graphs.size() - 1;
    return HB_OK;
}

hb_status hb_server_submit(hb_server *S, int32_t graph_id, int32_t log2m, uint64_t seed, int64_t *request_id) {
    if (!S || !request_id) return sfail(HB_ERR_INVALID, "NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    if (!S->fatal.empty()) return sfail(HB_ERR_STATE, "server stopped after a CUDA error: " + S->fatal);
    if (graph_id < 0 || graph_id >= (int32_t)S->graphs.size()) return sfail(HB_ERR_INVALID, "unknown graph id");
    if (!S->graphs[graph_id].tmpl.count(log2m))
        return sfail(HB_ERR_INVALID, "log2m not prepared for this graph (hb_server_add_graph)");
    const int64_t id = S->next_id++;
    ServeReq &r = S->reqs[id];
    r.graph = graph_id;
    r.log2m = log2m;
    r.seed = seed;
    r.large = S->graphs[graph_id].m >= S->opt.large_arcs;
    r.t_submit = S->now();
    S->queue.push_back(id);
    *request_id = id;
    S->cv.notify_all();
    return HB_OK;
}

hb_status hb_server_wait(hb_server *S, int64_t request_id, double timeout_s, hb_request_info *info) {
    if (!S) return sfail(HB_ERR_INVALID, "server is NULL");
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(request_id);
    if (it == S->reqs.end()) return sfail(HB_ERR_INVALID, "unknown request");
    ServeReq &r = it->second;
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
    while (r.state == HB_REQ_QUEUED || r.state == HB_REQ_RUNNING) {
        if (timeout_s >= 0 && S->done_cv.wait_until(lk, deadline) == std::cv_status::timeout &&
            (r.state == HB_REQ_QUEUED || r.state == HB_REQ_RUNNING))
            break;
        if (timeout_s < 0) S->done_cv.wait(lk);
    }
    if (info) {
        info->state = r.state;
        info->steps = r.steps;
        info->arcs = r.arcs;
        info->submit_s = r.t_submit;
        info->admit_s = r.t_admit;
        info->done_s = r.t_done;
    }
    if (r.state == HB_REQ_QUEUED || r.state == HB_REQ_RUNNING) return sfail(HB_ERR_TIMEOUT, "request not finished");
    if (r.state == HB_REQ_CANCELLED) return sfail(HB_ERR_STATE, "request cancelled");
    if (r.state == HB_REQ_FAILED)
        return sfail(r.err, r.err == HB_ERR_OOM ? "request refused: its device memory cannot be had"
                                                : "request failed");
    return HB_OK;
}

hb_status hb_server_cancel(hb_server *S, int64_t request_id) {
    if (!S) return sfail(HB_ERR_INVALID, "server is NULL");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(request_id);
    if (it == S->reqs.end()) return sfail(HB_ERR_INVALID, "unknown request");
    ServeReq &r = it->second;
    if (r.state == HB_REQ_QUEUED) {
        for (auto q = S->queue.begin(); q != S->queue.end(); ++q)
            if (*q == request_id) { S->queue.erase(q); break; }
        r.state = HB_REQ_CANCELLED;
        r.err = HB_ERR_STATE;
        r.t_done = S->now();
        S->done_cv.notify_all();
        return HB_OK;
    }
    if (r.state == HB_REQ_RUNNING) {
        r.cancel = true;
        return HB_OK;
    }
    return sfail(HB_ERR_STATE, "request already finished");
}

hb_status hb_server_take(hb_server *S, int64_t request_id, double *closeness, double *harmonic, double *lin,
                         double *reachable) {
    if (!S) return sfail(HB_ERR_INVALID, "server is NULL");
    double *dres = nullptr;
    int64_t n = 0;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        auto it = S->reqs.find(request_id);
        if (it == S->reqs.end()) return sfail(HB_ERR_INVALID, "unknown request");
        ServeReq &r = it->second;
        if (r.state == HB_REQ_FAILED || r.state == HB_REQ_CANCELLED) {
            if (r.dres) cudaFreeAsync(r.dres, S->copy_stream);
            S->reqs.erase(it);
            return sfail(HB_ERR_STATE, "request failed or cancelled; forgotten");
        }
        if (r.state != HB_REQ_DONE) return sfail(HB_ERR_STATE, "request not done");
        dres = r.dres;
        n = r.n;
        S->reqs.erase(it);
    }
    // copied outside the lock, so the server loop keeps running meanwhile
    double *dst[4] = {closeness, harmonic, lin, reachable};
    cudaError_t e = cudaSuccess;
    for (int q = 0; q < 4 && e == cudaSuccess; ++q)
        if (dst[q] && n > 0)
            e = cudaMemcpyAsync(dst[q], dres + (size_t)q * n, sizeof(double) * n, cudaMemcpyDefault, S->copy_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(S->copy_stream);
    cudaFreeAsync(dres, S->copy_stream);
    if (e != cudaSuccess) return sfail(HB_ERR_CUDA, std::string("result copy: ") + cudaGetErrorString(e));
    return HB_OK;
}

hb_status hb_server_stats(hb_server *S, int64_t *completed, int64_t *iterations, int64_t *arcs,
                          double *busy_s, double *clock_s) {
    if (!S) return sfail(HB_ERR_INVALID, "server is NULL");
    std::lock_guard<std::mutex> lk(S->mu);
    if (completed) *completed = S->completed;
    if (iterations) *iterations = S->iterations;
    if (arcs) *arcs = S->total_arcs;
    if (busy_s) *busy_s = S->busy_s;
    if (clock_s) *clock_s = S->now();
    return HB_OK;
}

void hb_server_destroy(hb_server *S) { delete S; }

}  // extern "C"

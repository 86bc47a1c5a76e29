// hb_step.cu -- the HyperBall iteration on the device (Sec. 4.2,
// Algorithm 2, with the Sec. 5 accumulators and modification tracking).
//
// One iteration is a fixed launch sequence whose sizes live in device
// memory, so the host never needs to know them:
//   step_begin      choose dense (every node) or sparse (frontier) mode
//   mark_push/pull  sparse: set the must-check bitmap and list the nodes
//                   that have a changed successor, grouped by degree class
//   copy_forward    sparse: nodes that changed last time but are not
//                   recomputed now get their counter copied into the
//                   write buffer (double buffering replaces the paper's
//                   update file)
//   plan            sparse: map listed nodes onto warp items
//   step_kernel     gather + register-wise max (union), changed test,
//                   estimator and accumulators for changed nodes
//   step_end        count the iteration, record convergence
#include <map>
#include <mutex>

#include "hb_step_dev.cuh"

namespace hb {

namespace {

using namespace dev;

// ---------------------------------------------------------- estimator --

__global__ void lc_tables_kernel(double *lc64, float *lc32, int P) {
    for (int V = threadIdx.x + blockIdx.x * blockDim.x; V <= P; V += blockDim.x * gridDim.x) {
        double e = 0.0;
        if (V > 0) e = __dmul_rn((double)P, log(__ddiv_rn((double)P, (double)V)));
        lc64[V] = e;
        lc32[V] = (float)e;
    }
}

// ------------------------------------------------ neighbourhood function --

// Each block sums a fixed strided set of nodes, then a fixed tree in
// shared memory; one block then sums the block partials the same way.
__device__ __forceinline__ double block_tree_sum(double x, double *sh) {
    sh[threadIdx.x] = x;
    __syncthreads();
    for (int w = blockDim.x >> 1; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    return sh[0];
}

template <bool F32>
__global__ void __launch_bounds__(256) estimate_partials_kernel(const void *ecache, int64_t n, double *part) {
    __shared__ double sh[256];
    double x = 0.0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        x += F32 ? (double)static_cast<const float *>(ecache)[v] : static_cast<const double *>(ecache)[v];
    const double tot = block_tree_sum(x, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) estimate_total_kernel(const double *part, int np, Counters *ctr) {
    __shared__ double sh[1024];
    const double tot = block_tree_sum((int)threadIdx.x < np ? part[threadIdx.x] : 0.0, sh);
    if (threadIdx.x == 0) ctr->nsum = tot;
}

// ---------------------------------------------------------------- init --

// Algorithm 2, first loop: add(c[v], v) into an empty counter, in both
// buffers (the second buffer then already holds c_0 for nodes that are
// never recomputed).  packed: 16-register chunks written as 12 bytes.
__global__ void init_rows_kernel(uint8_t *r0, uint8_t *r1, const int32_t *perm, int64_t n, int b,
                                 uint64_t seed, int packed) {
    const int CH = (1 << b) >> 4;
    const int64_t total = n * CH;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < total;
         k += (int64_t)gridDim.x * blockDim.x) {
        int64_t v = k / CH;
        int c = (int)(k - v * CH);
        uint64_t orig = perm ? (uint64_t)perm[v] : (uint64_t)v;
        uint32_t idx, rho;
        hash_to_register(splitmix64(seed, orig), b, idx, rho);
        uint32_t w[4] = {0u, 0u, 0u, 0u};
        if ((int)(idx >> 4) == c) w[(idx >> 2) & 3] = rho << (8 * (idx & 3));
        uint4 val = make_uint4(w[0], w[1], w[2], w[3]);
        if (packed) {
            uint32_t q0, q1, q2;
            pack_chunk(val, q0, q1, q2);
            uint32_t *d0 = reinterpret_cast<uint32_t *>(r0) + 3 * k;
            uint32_t *d1 = reinterpret_cast<uint32_t *>(r1) + 3 * k;
            d0[0] = q0; d0[1] = q1; d0[2] = q2;
            d1[0] = q0; d1[1] = q1; d1[2] = q2;
        } else {
            reinterpret_cast<uint4 *>(r0)[k] = val;
            reinterpret_cast<uint4 *>(r1)[k] = val;
        }
    }
}

template <bool F32>
__global__ void init_nodes_kernel(StepArgs a, const int32_t *perm, uint64_t seed) {
    const int P = 1 << a.b;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < a.n;
         v += (int64_t)gridDim.x * blockDim.x) {
        uint64_t orig = perm ? (uint64_t)perm[v] : (uint64_t)v;
        uint32_t idx, rho;
        hash_to_register(splitmix64(seed, orig), a.b, idx, rho);
        uint32_t V = (uint32_t)P - 1;
        unsigned long long S = 1ULL << (64 - a.b - (int)rho);
        if (F32) static_cast<float *>(a.ecache)[v] = estimate32(V, S, P, a.b, a.c32, a.thr_x, a.lc32);
        else static_cast<double *>(a.ecache)[v] = estimate64(V, S, P, a.b, a.c64, a.thr_x, a.lc64);
        a.sumd[v] = 0.0;
        a.harm[v] = 0.0;
        if (a.disc) a.disc[v] = 0.0;
        a.changed[v] = 0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) reset_counters(a.ctr);
}

// Sec. 6: integer node weights simulated by replicas.  The replicas of the
// caller's node u are the items wfirst[u] .. wfirst[u+1]-1 (numbered
// consecutively in the caller's node order, so unit weights give the items
// 0..n-1 of the unweighted init); each is hashed like a node id and added
// to u's empty counter, which is then written to both buffers.  One thread
// per node: its row is written by no other thread.
template <bool F32>
__global__ void init_weighted_kernel(StepArgs a, const int32_t *perm, const int64_t *wfirst,
                                     uint64_t seed) {
    const int P = 1 << a.b;
    const int CH = P >> 4;
    const uint4 z = make_uint4(0u, 0u, 0u, 0u);
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < a.n;
         v += (int64_t)gridDim.x * blockDim.x) {
        const int64_t u = perm ? (int64_t)perm[v] : v;
        uint8_t *r0 = a.regs[0] + v * P;
        uint4 *r1 = reinterpret_cast<uint4 *>(a.regs[1] + v * P);
        for (int c = 0; c < CH; ++c) reinterpret_cast<uint4 *>(r0)[c] = z;
        for (int64_t item = wfirst[u]; item < wfirst[u + 1]; ++item) {
            uint32_t idx, rho;
            hash_to_register(splitmix64(seed, (uint64_t)item), a.b, idx, rho);
            if (r0[idx] < rho) r0[idx] = (uint8_t)rho;
        }
        uint32_t V = 0;
        unsigned long long S = 0;
        for (int c = 0; c < CH; ++c) {
            const uint4 x = reinterpret_cast<const uint4 *>(r0)[c];
            r1[c] = x;
            chunk_sums(x, a.b, V, S);
        }
        if (F32) static_cast<float *>(a.ecache)[v] = estimate32(V, S, P, a.b, a.c32, a.thr_x, a.lc32);
        else static_cast<double *>(a.ecache)[v] = estimate64(V, S, P, a.b, a.c64, a.thr_x, a.lc64);
        a.sumd[v] = 0.0;
        a.harm[v] = 0.0;
        if (a.disc) a.disc[v] = 0.0;
        a.changed[v] = 0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) reset_counters(a.ctr);
}

// -------------------------------------------------------- step control --

__global__ void step_begin_kernel(StepArgs a) { begin_one(a); }

__global__ void step_end_kernel(StepArgs a) { end_one(a); }

__global__ void clear_bits_kernel(StepArgs a, int64_t words) {
    if (a.ctr->mode != 1) return;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < words;
         i += (int64_t)gridDim.x * blockDim.x)
        a.mustbits[i] = 0u;
}

// ----------------------------------------------------- frontier marking --

// Push: every node changed in the last iteration marks its predecessors.
__global__ void mark_push_kernel(StepArgs a) {
    const Counters *c = a.ctr;
    if (c->mode != 1 || a.frontier == HB_FRONTIER_PULL) return;
    const int t = c->t;
    const int32_t *prev = a.clist[(t + 1) & 1];
    const int32_t *bigp = a.biglist[(t + 1) & 1];
    const int64_t np = (int64_t)c->prev_list_len, nb = (int64_t)c->prev_big;
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = gw; i < np; i += nw) {
        const int32_t w = prev[i];
        if (a.roff[w + 1] - a.roff[w] > kBigRdeg) continue;
        push_warp(a, w, lane);
    }
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    const int64_t wbase = gw * 32;
    for (int64_t q = 0; q < nb; ++q) {
        const int32_t w = bigp[q];
        const int64_t r0 = a.roff[w], r1 = a.roff[w + 1];
        for (int64_t j0 = r0 + wbase; j0 < r1; j0 += nthreads) {
            int64_t j = j0 + lane;
            mark_append(a, j < r1 ? a.rtgt[j] : -1, lane);
        }
    }
}

// Pull: every node with a changed successor marks itself (no reverse CSR).
__global__ void mark_pull_kernel(StepArgs a) {
    const Counters *c = a.ctr;
    if (c->mode != 1 || a.frontier != HB_FRONTIER_PULL) return;
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t v = gw; v < a.n; v += nw) {
        const int64_t e0 = a.off[v], e1 = a.off[v + 1];
        bool hit = false;
        for (int64_t j0 = e0; j0 < e1 && !hit; j0 += 32) {
            int64_t j = j0 + lane;
            bool h = j < e1 && a.changed[a.tgt[j]];
            hit = __any_sync(FULL, h);
        }
        mark_append(a, (hit && lane == 0) ? (int32_t)v : -1, lane);
    }
}

// Sparse mode: clear last iteration's changed flags and copy forward the
// counters of nodes that changed then but are not recomputed now.
__global__ void copy_forward_kernel(StepArgs a) {
    const Counters *c = a.ctr;
    if (c->mode != 1) return;
    const int t = c->t;
    const int64_t total = (int64_t)c->prev_list_len << (a.b - 4);
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < total;
         k += (int64_t)gridDim.x * blockDim.x)
        copy_forward_one(a, t, k);
}

// -------------------------------------------------------------- planning --

// One block.  Items: first the chunks of heavy nodes (chunk starts by a
// block scan, then the chunk -> node map), then each light class packs
// 2^j nodes per warp item.
__global__ void plan_kernel(StepArgs a, PlanParams pp, Plan *plan, int32_t *owner, int64_t *cstart) {
    if (!pp.dense && a.push_union) return;   // pushed frontier iterations need no gather plan
    plan_block(a, pp, plan, owner, cstart);
}

__global__ void heavy_total_kernel(const int64_t *off, int64_t n, int64_t heavy, int64_t chunk,
                                   unsigned long long *tot) {
    unsigned long long s = 0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        int64_t d = off[v + 1] - off[v];
        if (d > heavy) s += (unsigned long long)((d + chunk - 1) / chunk);
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(tot, s);
}

// ------------------------------------------------------------ the step --

template <int LOG2P, bool F32>
__global__ void __launch_bounds__(kStepThreads, Cfg<LOG2P>::CPL >= 4 ? 3 : HB_MIN_BLOCKS)
    step_kernel(StepArgs a) {
    step_body<LOG2P, F32, false>(a);
}

// The one-pass gather with L2 priorities: counters of nodes below a.hint
// are read with the normal eviction priority, the others with evict-first.
// Built for one block fewer per SM than step_kernel, so that the two cache
// policies fit in registers without spilling.
#ifndef HB_HINT_MIN_BLOCKS
#define HB_HINT_MIN_BLOCKS 4
#endif
template <int LOG2P, bool F32>
__global__ void __launch_bounds__(kStepThreads, Cfg<LOG2P>::CPL >= 4 ? 3 : HB_HINT_MIN_BLOCKS)
    step_kernel_hint(StepArgs a) {
    step_body<LOG2P, F32, false, false, true>(a);
}

// Packed registers (six bits each, rows of 3p/4 bytes): the plain gather
// on packed rows, dense iterations only.  Built for one block fewer per SM
// than step_kernel: the unpacking of the arcs in flight needs the registers.
#ifndef HB_PACKED_MIN_BLOCKS
#define HB_PACKED_MIN_BLOCKS 4
#endif
template <int LOG2P, bool F32>
__global__ void __launch_bounds__(kStepThreads, Cfg<LOG2P>::CPL >= 4 ? 3 : HB_PACKED_MIN_BLOCKS)
    step_kernel_packed(StepArgs a) {
    step_body<LOG2P, F32, false, false, false, true>(a);
}

// The same gather in two passes (a.pass = 1, then 2): dense iterations
// first gather the arcs into the hot counters [0, a.hot), then the others.
template <int LOG2P, bool F32>
__global__ void __launch_bounds__(kStepThreads, Cfg<LOG2P>::CPL >= 4 ? 3 : HB_MIN_BLOCKS)
    step_kernel_two_pass(StepArgs a) {
    step_body<LOG2P, F32, false, true>(a);
}

// ------------------------------------------------ pushed frontier union --

// Frontier iteration with the reverse CSR: the counter of every node that
// changed in the last iteration is folded into each predecessor's write
// buffer counter, and the predecessor is marked for recomputation (the
// frontier of Sec. 5.1, as mark_push does): a warp per 32 changed nodes
// (push_union_item), the nodes with many predecessors by the whole grid.
__global__ void __launch_bounds__(kStepThreads, 4) push_union_kernel(StepArgs a) {
    const Counters *c = a.ctr;
    if (c->mode != 1 || !a.push_union) return;
    const int t = c->t;
    const uint4 *cur4 = reinterpret_cast<const uint4 *>(a.regs[t & 1]);
    uint4 *nxt4 = reinterpret_cast<uint4 *>(a.regs[(t + 1) & 1]);
    const int32_t *prev = a.clist[(t + 1) & 1];
    const int32_t *bigp = a.biglist[(t + 1) & 1];
    const int64_t np = (int64_t)c->prev_list_len, nb = (int64_t)c->prev_big;
    const int logCH = a.b - 4;
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t base = gw * 32; base < np; base += nw * 32)
        push_union_item(a, cur4, nxt4, prev, np, base, logCH, lane);
    for (int64_t q = 0; q < nb; ++q) push_union_big(a, cur4, nxt4, bigp[q], gw, nw, logCH, lane);
}

// The per-node tail of a pushed frontier iteration over the marked nodes.
template <int LOG2P, bool F32>
__global__ void __launch_bounds__(kStepThreads) union_tail_kernel(StepArgs a) {
    tail_body<LOG2P, F32, false>(a);
}

// After a dense iteration (frontier kept): list the changed nodes, their
// predecessor count and the ones with many predecessors.
__global__ void __launch_bounds__(256) compact_changed_kernel(StepArgs a) {
    if (a.ctr->mode != 0) return;
    const int t = a.ctr->t;
    for (int64_t base = (int64_t)blockIdx.x * 2048; base < a.n; base += (int64_t)gridDim.x * 2048)
        compact_tile_wide(a, t, base);
}

// --------------------------------------------------------------- outputs --

// Centralities of the caller's nodes u0 .. u0+count-1, written to out[k][u -
// u0] in the caller's order: each thread reads its node's row and
// accumulators at the internal index inv[u] (scattered 32-byte reads) and
// writes contiguously (scattered 8-byte writes would each rewrite a sector).
template <bool F32>
__global__ void finalize_kernel(StepArgs a, const uint8_t *regs, const int32_t *inv, int64_t u0, int64_t count,
                                double *closeness, double *harmonic, double *lin, double *reachable) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t u = u0 + i;
        const int64_t v = inv ? (int64_t)inv[u] : u;
        double c[4];
        node_centralities<F32>(a, regs, v, c);
        if (closeness) closeness[i] = c[0];
        if (harmonic) harmonic[i] = c[1];
        if (lin) lin[i] = c[2];
        if (reachable) reachable[i] = c[3];
    }
}

// Rows in the caller's order, one byte per register (packed rows are
// unpacked on the way).
__global__ void gather_rows_kernel(const uint8_t *regs, const int32_t *inv, int64_t n, int CH,
                                   uint8_t *out, int packed) {
    const int64_t total = n * CH;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < total;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t u = k / CH;
        const int c = (int)(k - u * CH);
        const int64_t v = inv ? (int64_t)inv[u] : u;
        reinterpret_cast<uint4 *>(out)[k] = packed ? ld_packed(regs + 12 * (v * CH + c), 0)
                                                   : reinterpret_cast<const uint4 *>(regs)[v * CH + c];
    }
}

__global__ void gather_f64_kernel(const double *src, const int32_t *inv, int64_t n, double *out) {
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n;
         u += (int64_t)gridDim.x * blockDim.x)
        out[u] = src[inv ? (int64_t)inv[u] : u];
}

// changed[u] for the caller's node u; must[u] = some successor changed
// (by definition, pulled over the scanned arcs).
__global__ void frontier_out_kernel(StepArgs a, const int32_t *inv, uint8_t *changed, uint8_t *must) {
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < a.n;
         u += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = inv ? (int64_t)inv[u] : u;
        if (changed) changed[u] = a.changed[v];
        if (must) {
            uint8_t mk = 0;
            for (int64_t e = a.off[v]; e < a.off[v + 1]; ++e)
                if (a.changed[a.tgt[e]]) { mk = 1; break; }
            must[u] = mk;
        }
    }
}

template <bool F32>
const void *step_kernel_ptr(int log2m) {
    switch (log2m) {
#define HB_CASE(B) case B: return reinterpret_cast<const void *>(&step_kernel<B, F32>);
        HB_CASE(4) HB_CASE(5) HB_CASE(6) HB_CASE(7) HB_CASE(8) HB_CASE(9) HB_CASE(10) HB_CASE(11)
        HB_CASE(12)
#undef HB_CASE
        default: return nullptr;
    }
}

template <bool F32>
const void *hint_kernel_ptr(int log2m) {
    switch (log2m) {
#define HB_CASE(B) case B: return reinterpret_cast<const void *>(&step_kernel_hint<B, F32>);
        HB_CASE(4) HB_CASE(5) HB_CASE(6) HB_CASE(7) HB_CASE(8) HB_CASE(9) HB_CASE(10) HB_CASE(11)
        HB_CASE(12)
#undef HB_CASE
        default: return nullptr;
    }
}

template <bool F32>
const void *packed_kernel_ptr(int log2m) {
    switch (log2m) {
#define HB_CASE(B) case B: return reinterpret_cast<const void *>(&step_kernel_packed<B, F32>);
        HB_CASE(4) HB_CASE(5) HB_CASE(6) HB_CASE(7) HB_CASE(8) HB_CASE(9) HB_CASE(10) HB_CASE(11)
        HB_CASE(12)
#undef HB_CASE
        default: return nullptr;
    }
}

// Resident blocks per SM of a kernel, looked up once per kernel.
int blocks_per_sm_of(const void *k) {
    static std::mutex mu;
    static std::map<const void *, int> cache;
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(k);
    if (it != cache.end()) return it->second;
    int blocks = 0;
    if (!k || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k, kStepThreads, 0) != cudaSuccess) {
        cudaGetLastError();
        blocks = 4;
    }
    if (blocks < 1) blocks = 1;
    cache[k] = blocks;
    return blocks;
}

template <bool F32>
cudaError_t launch_step_t(const StepArgs &a_in, int log2m, int grid, cudaStream_t s) {
    StepArgs a = a_in;
    if (a.packed) {
        // packed rows: the packed kernel's own occupancy over the same SMs
        const int per = blocks_per_sm_of(step_kernel_ptr<F32>(log2m));
        const int per_p = blocks_per_sm_of(packed_kernel_ptr<F32>(log2m));
        const int g = (grid / per) * per_p;
        switch (log2m) {
#define HB_CASE(B) case B: step_kernel_packed<B, F32><<<g, kStepThreads, 0, s>>>(a); break;
            HB_CASE(4) HB_CASE(5) HB_CASE(6) HB_CASE(7) HB_CASE(8) HB_CASE(9) HB_CASE(10) HB_CASE(11)
            HB_CASE(12)
#undef HB_CASE
            default: return cudaErrorInvalidValue;
        }
        return cudaGetLastError();
    }
    if (a.hot > 0 && !a.two_pass) {
        // one pass with L2 priorities: the grid of the hint kernel's own
        // occupancy over the same SMs
        a.hint = a.hot;
        const int per = blocks_per_sm_of(step_kernel_ptr<F32>(log2m));
        const int per_h = blocks_per_sm_of(hint_kernel_ptr<F32>(log2m));
        const int g = (grid / per) * per_h;
        switch (log2m) {
#define HB_CASE(B) case B: step_kernel_hint<B, F32><<<g, kStepThreads, 0, s>>>(a); break;
            HB_CASE(4) HB_CASE(5) HB_CASE(6) HB_CASE(7) HB_CASE(8) HB_CASE(9) HB_CASE(10) HB_CASE(11)
            HB_CASE(12)
#undef HB_CASE
            default: return cudaErrorInvalidValue;
        }
        return cudaGetLastError();
    }
    if (a.hot > 0) {
        // two launches: pass 1 (hot counters; dense iterations only), pass 2
        StepArgs a1 = a, a2 = a;
        a1.pass = 1;
        a2.pass = 2;
        switch (log2m) {
#define HB_CASE(B)                                                        \
    case B:                                                               \
        step_kernel_two_pass<B, F32><<<grid, kStepThreads, 0, s>>>(a1);   \
        step_kernel_two_pass<B, F32><<<grid, kStepThreads, 0, s>>>(a2);   \
        break;
            HB_CASE(4) HB_CASE(5) HB_CASE(6) HB_CASE(7) HB_CASE(8) HB_CASE(9) HB_CASE(10) HB_CASE(11)
            HB_CASE(12)
#undef HB_CASE
            default: return cudaErrorInvalidValue;
        }
        return cudaGetLastError();
    }
    switch (log2m) {
#define HB_CASE(B) case B: step_kernel<B, F32><<<grid, kStepThreads, 0, s>>>(a); break;
        HB_CASE(4) HB_CASE(5) HB_CASE(6) HB_CASE(7) HB_CASE(8) HB_CASE(9) HB_CASE(10) HB_CASE(11)
        HB_CASE(12)
#undef HB_CASE
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <bool F32>
cudaError_t launch_union_tail_t(const StepArgs &a, int log2m, int grid, cudaStream_t s) {
    switch (log2m) {
#define HB_CASE(B) case B: union_tail_kernel<B, F32><<<grid, kStepThreads, 0, s>>>(a); break;
        HB_CASE(4) HB_CASE(5) HB_CASE(6) HB_CASE(7) HB_CASE(8) HB_CASE(9) HB_CASE(10) HB_CASE(11)
        HB_CASE(12)
#undef HB_CASE
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace

int step_blocks_per_sm(int log2m, bool fp32) {
    const void *k = fp32 ? step_kernel_ptr<true>(log2m) : step_kernel_ptr<false>(log2m);
    int blocks = 0;
    if (!k || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k, kStepThreads, 0) != cudaSuccess)
        return 4;
    return blocks > 0 ? blocks : 1;
}

cudaError_t launch_step_kernel(const StepArgs &a, int log2m, bool fp32, int grid, cudaStream_t s) {
    return fp32 ? launch_step_t<true>(a, log2m, grid, s) : launch_step_t<false>(a, log2m, grid, s);
}

cudaError_t launch_lc_tables(double *lc64, float *lc32, int P, cudaStream_t s) {
    lc_tables_kernel<<<(P + 256) / 256, 256, 0, s>>>(lc64, lc32, P);
    return cudaGetLastError();
}

cudaError_t heavy_chunk_total(const int64_t *off, int64_t n, const Layout &y, int64_t *total_host,
                              cudaStream_t s) {
    unsigned long long *tot = nullptr;
    cudaError_t e = cudaMallocAsync(&tot, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    cudaMemsetAsync(tot, 0, sizeof(unsigned long long), s);
    if (n > 0) heavy_total_kernel<<<grid_for(n, 256), 256, 0, s>>>(off, n, y.heavy, y.chunk, tot);
    unsigned long long h = 0;
    cudaMemcpyAsync(&h, tot, sizeof(h), cudaMemcpyDeviceToHost, s);
    e = cudaStreamSynchronize(s);
    cudaFreeAsync(tot, s);
    *total_host = (int64_t)h;
    return e;
}

cudaError_t launch_init(const StepArgs &a, const int32_t *perm, uint64_t seed, bool fp32,
                        cudaStream_t s, const int64_t *wfirst) {
    const int CH = (1 << a.b) >> 4;
    if (a.lruns) return launch_runs_init(a, perm, fp32, s, wfirst);
    if (wfirst) {
        if (fp32) init_weighted_kernel<true><<<grid_for(a.n, 128), 128, 0, s>>>(a, perm, wfirst, seed);
        else init_weighted_kernel<false><<<grid_for(a.n, 128), 128, 0, s>>>(a, perm, wfirst, seed);
        return cudaGetLastError();
    }
    if (a.n > 0)
        init_rows_kernel<<<grid_for(a.n * CH, 256), 256, 0, s>>>(a.regs[0], a.regs[1], perm, a.n,
                                                                a.b, seed, a.packed);
    if (fp32) init_nodes_kernel<true><<<grid_for(a.n, 256), 256, 0, s>>>(a, perm, seed);
    else init_nodes_kernel<false><<<grid_for(a.n, 256), 256, 0, s>>>(a, perm, seed);
    return cudaGetLastError();
}

cudaError_t launch_estimate_sum(const void *ecache, bool fp32, int64_t n, double *part, Counters *ctr,
                                cudaStream_t s) {
    if (fp32) estimate_partials_kernel<true><<<kNfBlocks, 256, 0, s>>>(ecache, n, part);
    else estimate_partials_kernel<false><<<kNfBlocks, 256, 0, s>>>(ecache, n, part);
    estimate_total_kernel<<<1, 1024, 0, s>>>(part, kNfBlocks, ctr);
    return cudaGetLastError();
}

cudaError_t launch_dense_plan(const StepArgs &a, const Layout &y, const int64_t *seg_count,
                              Plan *plan, int32_t *owner, int64_t *cstart, cudaStream_t s) {
    PlanParams pp{};
    for (int k = 0; k < kSegs; ++k) pp.count[k] = seg_count[k];
    pp.chunk = y.chunk;
    pp.nlight = y.nlight;
    pp.dense = 1;
    plan_kernel<<<1, 1024, 0, s>>>(a, pp, plan, owner, cstart);
    return cudaGetLastError();
}

cudaError_t launch_iteration(const StepArgs &a, const Layout &y, bool fp32, int step_grid,
                             cudaStream_t s, const cudaEvent_t *ev, int *launches) {
    int k = 0;
    step_begin_kernel<<<1, 1, 0, s>>>(a);
    ++k;
    if (a.frontier != HB_FRONTIER_OFF) {
        const int64_t words = (a.n + 31) / 32;
        clear_bits_kernel<<<grid_for(words, 256), 256, 0, s>>>(a, words);
        if (a.frontier == HB_FRONTIER_PULL)
            mark_pull_kernel<<<step_grid, kStepThreads, 0, s>>>(a);
        else if (a.has_reverse && !a.push_union)
            mark_push_kernel<<<step_grid, kStepThreads, 0, s>>>(a);
        if (a.push_union) {
            // marks and pushes in one pass (frontier iterations only)
            if (ev) cudaEventRecord(ev[2], s);
            push_union_kernel<<<step_grid, kStepThreads, 0, s>>>(a);
        }
        copy_forward_kernel<<<step_grid, kStepThreads, 0, s>>>(a);
        PlanParams pp{};
        pp.chunk = y.chunk;
        pp.nlight = y.nlight;
        pp.dense = 0;
        plan_kernel<<<1, 1024, 0, s>>>(a, pp, a.plan_sparse, a.owner_sparse, a.cstart_sparse);
        k += (a.frontier == HB_FRONTIER_PULL || a.has_reverse) ? 4 : 3;
        if (a.push_union) ++k;   // push_union in place of mark_push, plus the tail below
    }
    if (ev) cudaEventRecord(ev[0], s);
    cudaError_t e = a.lruns ? launch_runs_step(a, y.log2m, fp32, step_grid, s)
                  : fp32    ? launch_step_t<true>(a, y.log2m, step_grid, s)
                            : launch_step_t<false>(a, y.log2m, step_grid, s);
    if (e != cudaSuccess) return e;
    if (a.hot > 0 && a.two_pass && !a.lruns) ++k;   // the two-phase gather's second launch
    if (ev) cudaEventRecord(ev[1], s);
    if (a.push_union) {
        e = a.lruns ? launch_runs_tail(a, y.log2m, fp32, step_grid, s)
          : fp32    ? launch_union_tail_t<true>(a, y.log2m, step_grid, s)
                    : launch_union_tail_t<false>(a, y.log2m, step_grid, s);
        if (e != cudaSuccess) return e;
        if (ev) cudaEventRecord(ev[3], s);
    }
    if (a.frontier != HB_FRONTIER_OFF) {
        compact_changed_kernel<<<grid_for((a.n + 7) / 8, 256), 256, 0, s>>>(a);
        ++k;
    }
    step_end_kernel<<<1, 1, 0, s>>>(a);
    k += 2;
    if (launches) *launches += k;
    return cudaGetLastError();
}

cudaError_t launch_finalize(const StepArgs &a, const uint8_t *regs, const int32_t *inv, bool fp32, int64_t u0,
                            int64_t count, double *closeness, double *harmonic, double *lin, double *reachable,
                            cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    if (fp32)
        finalize_kernel<true><<<grid_for(count, 256), 256, 0, s>>>(a, regs, inv, u0, count, closeness, harmonic,
                                                                   lin, reachable);
    else
        finalize_kernel<false><<<grid_for(count, 256), 256, 0, s>>>(a, regs, inv, u0, count, closeness, harmonic,
                                                                    lin, reachable);
    return cudaGetLastError();
}

cudaError_t launch_gather_rows(const uint8_t *regs, const int32_t *inv, int64_t n, int P,
                               uint8_t *out, cudaStream_t s, bool packed) {
    const int CH = P >> 4;
    if (n > 0) gather_rows_kernel<<<grid_for(n * CH, 256), 256, 0, s>>>(regs, inv, n, CH, out, packed ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_gather_f64(const double *src, const int32_t *inv, int64_t n, double *out,
                              cudaStream_t s) {
    if (n > 0) gather_f64_kernel<<<grid_for(n, 256), 256, 0, s>>>(src, inv, n, out);
    return cudaGetLastError();
}

cudaError_t launch_frontier_out(const StepArgs &a, const int32_t *inv, uint8_t *changed,
                                uint8_t *must, cudaStream_t s) {
    if (a.n > 0) frontier_out_kernel<<<grid_for(a.n, 256), 256, 0, s>>>(a, inv, changed, must);
    return cudaGetLastError();
}

}  // namespace hb

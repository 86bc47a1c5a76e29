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
#include "hb_internal.cuh"

#include "hyperball.h"

// Arcs in flight per lane when a lane holds one 16-byte chunk of a counter,
// and the minimum resident blocks the step kernel is compiled for.
#ifndef HB_UNROLL
#define HB_UNROLL 8
#endif
#ifndef HB_MIN_BLOCKS
#define HB_MIN_BLOCKS 6
#endif

namespace hb {

namespace {

constexpr unsigned FULL = 0xffffffffu;

// ---------------------------------------------------------- estimator --

__global__ void lc_tables_kernel(double *lc64, float *lc32, int P) {
    for (int V = threadIdx.x + blockIdx.x * blockDim.x; V <= P; V += blockDim.x * gridDim.x) {
        double e = 0.0;
        if (V > 0) e = __dmul_rn((double)P, log(__ddiv_rn((double)P, (double)V)));
        lc64[V] = e;
        lc32[V] = (float)e;
    }
}

// ---------------------------------------------------------------- init --

// Algorithm 2, first loop: add(c[v], v) into an empty counter, in both
// buffers (the second buffer then already holds c_0 for nodes that are
// never recomputed).
__global__ void init_rows_kernel(uint8_t *r0, uint8_t *r1, const int32_t *perm, int64_t n, int b,
                                 uint64_t seed) {
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
        reinterpret_cast<uint4 *>(r0)[k] = val;
        reinterpret_cast<uint4 *>(r1)[k] = val;
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
        a.changed[v] = 0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        Counters *c = a.ctr;
        c->n_changed = 0; c->list_len = 0; c->push_arcs = 0; c->n_big = 0; c->arcs = 0;
        for (int s = 0; s < kSegs; ++s) c->fill[s] = 0;
        c->prev_changed = 0; c->prev_list_len = 0; c->prev_push_arcs = 0; c->prev_big = 0;
        c->mode = 0; c->t = 0; c->steps_done = 0; c->converged = 0; c->err = 0;
    }
}

// -------------------------------------------------------- step control --

__global__ void step_begin_kernel(StepArgs a) {
    Counters *c = a.ctr;
    const int t = c->steps_done;
    c->t = t;
    c->prev_changed = c->n_changed;
    c->prev_list_len = c->list_len;
    c->prev_push_arcs = c->push_arcs;
    c->prev_big = c->n_big;
    c->n_changed = 0; c->list_len = 0; c->push_arcs = 0; c->n_big = 0; c->arcs = 0;
    for (int s = 0; s < kSegs; ++s) c->fill[s] = 0;
    int sparse = 0;
    if (t > 0) {
        if (a.frontier == HB_FRONTIER_PULL) sparse = 1;
        else if (a.frontier == HB_FRONTIER_PUSH) sparse = a.has_reverse;
        else if (a.frontier == HB_FRONTIER_AUTO)
            sparse = a.has_reverse && (double)c->prev_push_arcs <= a.sparse_frac * (double)a.m;
    }
    c->mode = sparse;
}

__global__ void step_end_kernel(StepArgs a) {
    Counters *c = a.ctr;
    c->steps_done = c->t + 1;
    if (c->n_changed == 0) c->converged = 1;
}

__global__ void clear_bits_kernel(StepArgs a, int64_t words) {
    if (a.ctr->mode != 1) return;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < words;
         i += (int64_t)gridDim.x * blockDim.x)
        a.mustbits[i] = 0u;
}

// ----------------------------------------------------- frontier marking --

__device__ __forceinline__ int segment_of(const StepArgs &a, int64_t d) {
#pragma unroll
    for (int s = 0; s < kSegs; ++s)
        if (d >= a.seg_lo[s] && d <= a.seg_hi[s]) return s;
    return -1;
}

// Called by all 32 lanes; u < 0 for lanes with nothing to mark.  Sets the
// must-check bit of u and, if it was clear, appends u to its degree
// segment of the sparse list.
__device__ __forceinline__ void mark_append(const StepArgs &a, int32_t u, int lane) {
    int key = -1;
    int64_t d = 0;
    if (u >= 0) {
        unsigned bit = 1u << (u & 31);
        unsigned old = atomicOr(&a.mustbits[u >> 5], bit);
        if (!(old & bit)) {
            d = a.off[u + 1] - a.off[u];
            key = segment_of(a, d);
        }
    }
    unsigned peers = __match_any_sync(FULL, key);
    int leader = __ffs(peers) - 1;
    unsigned long long base = 0;
    if (key >= 0 && lane == leader)
        base = atomicAdd(&a.ctr->fill[key], (unsigned long long)__popc(peers));
    base = __shfl_sync(FULL, base, leader);
    if (key >= 0) a.slist[a.seg_begin[key] + (int64_t)base + __popc(peers & lanemask_lt())] = u;
    unsigned long long dd = key >= 0 ? (unsigned long long)d : 0ULL;
#pragma unroll
    for (int o = 16; o; o >>= 1) dd += __shfl_xor_sync(FULL, dd, o);
    if (lane == 0 && dd) atomicAdd(&a.ctr->arcs, dd);
}

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
        const int64_t r0 = a.roff[w], r1 = a.roff[w + 1];
        if (r1 - r0 > kBigRdeg) continue;
        for (int64_t j0 = r0; j0 < r1; j0 += 32) {
            int64_t j = j0 + lane;
            mark_append(a, j < r1 ? a.rtgt[j] : -1, lane);
        }
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
    const int32_t *prev = a.clist[(t + 1) & 1];
    const uint8_t *cur = a.regs[t & 1];
    uint8_t *nxt = a.regs[(t + 1) & 1];
    const int CH = (1 << a.b) >> 4;
    const int logCH = a.b - 4;
    const int64_t total = (int64_t)c->prev_list_len << logCH;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < total;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = k >> logCH;
        const int ch = (int)(k & (CH - 1));
        const int32_t w = prev[i];
        if (ch == 0) a.changed[w] = 0;
        if (!((a.mustbits[w >> 5] >> (w & 31)) & 1u)) {
            const int64_t o = ((int64_t)w << logCH) + ch;
            reinterpret_cast<uint4 *>(nxt)[o] = reinterpret_cast<const uint4 *>(cur)[o];
        }
    }
}

// -------------------------------------------------------------- planning --

struct PlanParams {
    int64_t count[kSegs];   // dense: segment sizes
    int64_t chunk;
    int32_t nlight;
    int32_t dense;
};

// One block.  Items: first the chunks of heavy nodes (chunk starts by a
// block scan, then the chunk -> node map), then each light class packs
// 2^j nodes per warp item.
__global__ void plan_kernel(StepArgs a, PlanParams pp, Plan *plan, int32_t *owner, int64_t *cstart) {
    if (!pp.dense && a.ctr->mode != 1) return;
    __shared__ int64_t carry;
    int64_t cnt[kSegs];
    for (int s = 0; s < kSegs; ++s) cnt[s] = pp.dense ? pp.count[s] : (int64_t)a.ctr->fill[s];
    const int32_t *list = pp.dense ? a.dense_list : a.slist;
    const int64_t h = cnt[0];
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < h; base += blockDim.x) {
        const int64_t i = base + threadIdx.x;
        int64_t c = 0;
        if (i < h) {
            const int64_t pos = a.seg_begin[0] + i;
            const int64_t v = list ? list[pos] : pos;
            const int64_t d = a.off[v + 1] - a.off[v];
            c = (d + pp.chunk - 1) / pp.chunk;
        }
        int64_t ex;
        const int64_t tot = block_excl_scan(c, ex);
        if (i < h) cstart[i] = carry + ex;
        __syncthreads();
        if (threadIdx.x == 0) carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) cstart[h] = carry;
    __syncthreads();
    for (int64_t i = threadIdx.x; i < h; i += blockDim.x)
        for (int64_t q = cstart[i]; q < cstart[i + 1]; ++q) owner[q] = (int32_t)i;
    if (threadIdx.x == 0) {
        int64_t run = 0, nodes = 0;
        for (int s = 0; s < kSegs; ++s) { plan->count[s] = cnt[s]; nodes += cnt[s]; }
        for (int j = 0; j < kSegs - 1; ++j) {
            plan->item_begin[j] = run;
            if (j < pp.nlight) run += (cnt[j + 1] + (1LL << j) - 1) >> j;
        }
        plan->item_begin[kSegs - 1] = run;
        plan->heavy_chunks = carry;
        plan->items = carry + run;
        plan->nodes = nodes;
        plan->arcs = pp.dense ? a.m : (int64_t)a.ctr->arcs;
    }
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

// Gather the counters of arcs e, e+S, ... < eend (S = 2^logS) into acc
// (this lane's chunks), U arcs in flight per lane; full groups of U arcs
// run without bounds checks.
template <int LOG2P>
__device__ __forceinline__ void gather_arcs(const int32_t *__restrict__ tgt,
                                            const uint8_t *__restrict__ cur, int64_t e,
                                            int64_t eend, int logS, int cl,
                                            uint4 (&acc)[Cfg<LOG2P>::CPL]) {
    using C = Cfg<LOG2P>;
    constexpr int U = C::CPL >= 8 ? 1 : (C::CPL == 4 ? 2 : (C::CPL == 2 ? 4 : HB_UNROLL));
    if (e >= eend) return;
    const int cnt = (int)((eend - e + (1LL << logS) - 1) >> logS);
    const int32_t *tp = tgt + e;
    const uint8_t *base = cur + cl * 16;
    int j = 0;
    for (; j + U <= cnt; j += U) {
        int32_t w[U];
#pragma unroll
        for (int u = 0; u < U; ++u) w[u] = ld_stream(tp + ((j + u) << logS));
        uint4 g[U][C::CPL];
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int c = 0; c < C::CPL; ++c)
                g[u][c] = ld_counter(base + (size_t)(uint32_t)w[u] * C::P + c * C::L * 16);
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int c = 0; c < C::CPL; ++c) acc[c] = vmax16(acc[c], g[u][c]);
    }
    if (j < cnt) {
        const uint4 z = make_uint4(0u, 0u, 0u, 0u);
        int32_t w[U];
#pragma unroll
        for (int u = 0; u < U; ++u) w[u] = j + u < cnt ? ld_stream(tp + ((j + u) << logS)) : -1;
        uint4 g[U][C::CPL];
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int c = 0; c < C::CPL; ++c)
                g[u][c] = w[u] >= 0 ? ld_counter(base + (size_t)(uint32_t)w[u] * C::P + c * C::L * 16) : z;
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int c = 0; c < C::CPL; ++c) acc[c] = vmax16(acc[c], g[u][c]);
    }
}

// Per-node tail, called by all 32 lanes.  acc holds the union of the
// successors' counters (this lane's chunks; every slot of the team holds
// the same).  Folds in the node's own counter, writes it to the write
// buffer, sets the changed flag, and for changed nodes evaluates size()
// and updates the accumulators (Sec. 5), appending the node to the changed
// list.
template <int LOG2P, bool F32>
__device__ __forceinline__ void node_epilogue(const StepArgs &a, const uint8_t *__restrict__ cur,
                                              uint8_t *__restrict__ nxt, int t, int64_t v,
                                              bool active, uint4 (&acc)[Cfg<LOG2P>::CPL], int cl,
                                              int tl, int team, int logT, int32_t *clist,
                                              int32_t *biglist, bool sparse,
                                              unsigned long long *s_changed, double rdist64,
                                              float rdist32, const unsigned long long *pow2) {
    using C = Cfg<LOG2P>;
    const int lane = threadIdx.x & 31;
    bool diff = false;
    if (active) {
        const uint8_t *own = cur + v * C::P + cl * 16;
#pragma unroll
        for (int c = 0; c < C::CPL; ++c) {
            const uint4 o = ld_counter(own + c * C::L * 16);
            const uint4 nv = vmax16(acc[c], o);
            diff |= ne16(nv, o);
            acc[c] = nv;
        }
    }
    const unsigned bal = __ballot_sync(FULL, diff);
    const unsigned tmask = logT == 5 ? FULL : (((1u << (1 << logT)) - 1u) << (team << logT));
    const bool ch = (bal & tmask) != 0u;
    if (active && tl < C::L) {
        uint8_t *dst = nxt + v * C::P + cl * 16;
#pragma unroll
        for (int c = 0; c < C::CPL; ++c) *reinterpret_cast<uint4 *>(dst + c * C::L * 16) = acc[c];
    }
    const bool leader = active && tl == 0;
    if (leader) a.changed[v] = ch ? 1 : 0;
    const unsigned lb = __ballot_sync(FULL, leader && ch);
    if (lb == 0u) return;

    // size() of the new counter: zero count and fixed-point sum, reduced
    // over the chunk lanes of the team.
    uint32_t V = 0;
    unsigned long long S = 0;
#pragma unroll
    for (int c = 0; c < C::CPL; ++c) chunk_sums_tab(acc[c], pow2, V, S);
#pragma unroll
    for (int o = 1; o < C::L; o <<= 1) {
        V += __shfl_xor_sync(FULL, V, o);
        S += __shfl_xor_sync(FULL, S, o);
    }
    if (leader && ch) {
        // Sec. 5: the new layer sits at distance t+1
        if (F32) {
            float *ec = static_cast<float *>(a.ecache);
            const float E = estimate32(V, S, C::P, a.b, a.c32, a.thr_x, a.lc32);
            const float d = __fsub_rn(E, ec[v]);
            ec[v] = E;
            a.sumd[v] = __fma_rn((double)(t + 1), (double)d, a.sumd[v]);   // exact product
            a.harm[v] = __dadd_rn(a.harm[v], (double)__fmul_rn(d, rdist32));
        } else {
            double *ec = static_cast<double *>(a.ecache);
            const double E = estimate64(V, S, C::P, a.b, a.c64, a.thr_x, a.lc64);
            const double d = __dsub_rn(E, ec[v]);
            ec[v] = E;
            a.sumd[v] = __fma_rn((double)(t + 1), d, a.sumd[v]);
            a.harm[v] = __fma_rn(d, rdist64, a.harm[v]);
        }
    }
    if (lane == 0) atomicAdd(s_changed, (unsigned long long)__popc(lb));
    if (!sparse) return;   // dense iterations: the changed list is compacted afterwards
    // frontier iterations change few nodes: append them right away
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(&a.ctr->list_len, (unsigned long long)__popc(lb));
    base = __shfl_sync(FULL, base, 0);
    if (leader && ch) clist[base + __popc(lb & lanemask_lt())] = (int32_t)v;
    if (a.has_reverse) {
        const int64_t rd = (leader && ch) ? a.roff[v + 1] - a.roff[v] : 0;
        unsigned long long s = (unsigned long long)rd;
#pragma unroll
        for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
        if (lane == 0 && s) atomicAdd(&a.ctr->push_arcs, s);
        const unsigned bb = __ballot_sync(FULL, rd > kBigRdeg);
        if (bb) {
            unsigned long long bbase = 0;
            if (lane == 0) bbase = atomicAdd(&a.ctr->n_big, (unsigned long long)__popc(bb));
            bbase = __shfl_sync(FULL, bbase, 0);
            if (rd > kBigRdeg) biglist[bbase + __popc(bb & lanemask_lt())] = (int32_t)v;
        }
    }
}

template <int LOG2P, bool F32>
__device__ __forceinline__ void light_item(const StepArgs &a, const uint8_t *__restrict__ cur,
                                           uint8_t *__restrict__ nxt, int t, int64_t pos0,
                                           int64_t pos_end, int logS, const int32_t *list,
                                           int32_t *clist, int32_t *biglist, bool sparse,
                                           unsigned long long *s_changed, double rdist64,
                                           float rdist32, const unsigned long long *pow2) {
    using C = Cfg<LOG2P>;
    const int lane = threadIdx.x & 31;
    const int logT = C::LOGL + logS;
    const int team = lane >> logT;
    const int tl = lane & ((1 << logT) - 1);
    const int cl = tl & (C::L - 1);
    const int slot = tl >> C::LOGL;
    const int64_t pos = pos0 + team;
    const bool active = pos < pos_end;
    int64_t v = 0, e0 = 0, e1 = 0;
    if (active) {
        v = list ? (int64_t)list[pos] : pos;
        e0 = a.off[v];
        e1 = a.off[v + 1];
    }
    uint4 acc[C::CPL];
#pragma unroll
    for (int c = 0; c < C::CPL; ++c) acc[c] = make_uint4(0u, 0u, 0u, 0u);
    gather_arcs<LOG2P>(a.tgt, cur, e0 + slot, e1, logS, cl, acc);
    for (int o = C::L; o < (1 << logT); o <<= 1)
#pragma unroll
        for (int c = 0; c < C::CPL; ++c) acc[c] = vmax16(acc[c], shfl_xor16(acc[c], o));
    node_epilogue<LOG2P, F32>(a, cur, nxt, t, v, active, acc, cl, tl, team, logT, clist, biglist,
                              sparse, s_changed, rdist64, rdist32, pow2);
}

// One chunk of a heavy node, by a whole warp.  Each chunk leaves its
// partial union in scratch; the last chunk to arrive combines them and
// finishes the node.
template <int LOG2P, bool F32>
__device__ __forceinline__ void heavy_item(const StepArgs &a, const uint8_t *__restrict__ cur,
                                           uint8_t *__restrict__ nxt, int t, int64_t it,
                                           const int32_t *owner, const int64_t *cstart,
                                           const int32_t *list, int32_t *clist, int32_t *biglist,
                                           bool sparse, unsigned long long *s_changed,
                                           double rdist64, float rdist32,
                                           const unsigned long long *pow2) {
    using C = Cfg<LOG2P>;
    const int lane = threadIdx.x & 31;
    const int cl = lane & (C::L - 1);
    const int slot = lane >> C::LOGL;
    const int32_t hp = owner[it];
    const int64_t c0 = cstart[hp];
    const int64_t nch = cstart[hp + 1] - c0;
    const int64_t k = it - c0;
    const int64_t pos = a.seg_begin[0] + hp;
    const int64_t v = list ? (int64_t)list[pos] : pos;
    const int64_t a1 = a.off[v + 1];
    const int64_t e0 = a.off[v] + k * C::CHUNK;
    const int64_t e1 = e0 + C::CHUNK < a1 ? e0 + C::CHUNK : a1;
    uint4 acc[C::CPL];
#pragma unroll
    for (int c = 0; c < C::CPL; ++c) acc[c] = make_uint4(0u, 0u, 0u, 0u);
    gather_arcs<LOG2P>(a.tgt, cur, e0 + slot, e1, C::LOGSMAX, cl, acc);
#pragma unroll
    for (int o = C::L; o < 32; o <<= 1)
#pragma unroll
        for (int c = 0; c < C::CPL; ++c) acc[c] = vmax16(acc[c], shfl_xor16(acc[c], o));
    if (nch > 1) {
        if (slot == 0) {
            uint8_t *dst = a.partial + it * C::P + cl * 16;
#pragma unroll
            for (int c = 0; c < C::CPL; ++c) __stcg(reinterpret_cast<uint4 *>(dst + c * C::L * 16), acc[c]);
        }
        __threadfence();
        __syncwarp();
        unsigned last = 0;
        if (lane == 0) last = atomicAdd(&a.arrive[hp], 1u) == (unsigned)(nch - 1) ? 1u : 0u;
        last = __shfl_sync(FULL, last, 0);
        if (!last) return;
        if (lane == 0) a.arrive[hp] = 0u;
        __threadfence();
#pragma unroll
        for (int c = 0; c < C::CPL; ++c) acc[c] = make_uint4(0u, 0u, 0u, 0u);
        for (int64_t q = slot; q < nch; q += C::SMAX) {
            const uint8_t *src = a.partial + (c0 + q) * C::P + cl * 16;
#pragma unroll
            for (int c = 0; c < C::CPL; ++c)
                acc[c] = vmax16(acc[c], __ldcg(reinterpret_cast<const uint4 *>(src + c * C::L * 16)));
        }
#pragma unroll
        for (int o = C::L; o < 32; o <<= 1)
#pragma unroll
            for (int c = 0; c < C::CPL; ++c) acc[c] = vmax16(acc[c], shfl_xor16(acc[c], o));
    }
    node_epilogue<LOG2P, F32>(a, cur, nxt, t, v, true, acc, cl, lane, 0, 5, clist, biglist, sparse,
                              s_changed, rdist64, rdist32, pow2);
}

template <int LOG2P, bool F32>
__global__ void __launch_bounds__(kStepThreads, Cfg<LOG2P>::CPL >= 4 ? 3 : HB_MIN_BLOCKS)
    step_kernel(StepArgs a) {
    using C = Cfg<LOG2P>;
    const Counters *ctr = a.ctr;
    const int t = ctr->t;
    const bool sparse = ctr->mode == 1;
    const Plan *pl = sparse ? a.plan_sparse : a.plan_dense;
    const int32_t *list = sparse ? a.slist : a.dense_list;
    const int32_t *owner = sparse ? a.owner_sparse : a.owner_dense;
    const int64_t *cstart = sparse ? a.cstart_sparse : a.cstart_dense;
    const uint8_t *cur = a.regs[t & 1];
    uint8_t *nxt = a.regs[(t + 1) & 1];
    int32_t *clist = a.clist[t & 1];
    int32_t *biglist = a.biglist[t & 1];
    const int64_t items = pl->items;
    const int64_t hch = pl->heavy_chunks;
    int64_t ib[C::NLIGHT + 1], cnt[C::NLIGHT];
#pragma unroll
    for (int j = 0; j <= C::NLIGHT; ++j) ib[j] = pl->item_begin[j];
#pragma unroll
    for (int j = 0; j < C::NLIGHT; ++j) cnt[j] = pl->count[j + 1];
    __shared__ unsigned long long s_changed;
    __shared__ unsigned long long s_pow2[64];
    const double rdist64 = 1.0 / (double)(t + 1);
    const float rdist32 = 1.0f / (float)(t + 1);
    if (threadIdx.x == 0) s_changed = 0;
    if (threadIdx.x < 64) {
        const int M = threadIdx.x, sh = 64 - a.b;
        s_pow2[M] = (M == 0 || M > sh) ? 0ULL : 1ULL << (sh - M);
    }
    __syncthreads();
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t it = gw; it < items; it += nw) {
        if (it < hch) {
            heavy_item<LOG2P, F32>(a, cur, nxt, t, it, owner, cstart, list, clist, biglist, sparse,
                                   &s_changed, rdist64, rdist32, s_pow2);
        } else {
            const int64_t li = it - hch;
            int j = 0;
            int64_t ibj = ib[0], cntj = cnt[0], seg0 = a.seg_begin[1];
#pragma unroll
            for (int q = 1; q < C::NLIGHT; ++q)
                if (li >= ib[q]) { j = q; ibj = ib[q]; cntj = cnt[q]; seg0 = a.seg_begin[q + 1]; }
            const int64_t pos0 = seg0 + ((li - ibj) << j);
            light_item<LOG2P, F32>(a, cur, nxt, t, pos0, seg0 + cntj, C::LOGSMAX - j, list,
                                   clist, biglist, sparse, &s_changed, rdist64, rdist32, s_pow2);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && s_changed) atomicAdd(&a.ctr->n_changed, s_changed);
}

// After a dense iteration (frontier kept): list the changed nodes, their
// predecessor count and the ones with many predecessors.  One global atomic
// per block; the list order does not matter.
__global__ void __launch_bounds__(256) compact_changed_kernel(StepArgs a) {
    const Counters *c = a.ctr;
    if (c->mode != 0) return;
    const int t = c->t;
    int32_t *clist = a.clist[t & 1];
    int32_t *biglist = a.biglist[t & 1];
    __shared__ unsigned wcnt[8], wbig[8];
    __shared__ unsigned long long sbase, bbase, spush;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < a.n; base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = base + threadIdx.x;
        const bool ch = v < a.n && a.changed[v];
        int64_t rd = 0;
        if (ch && a.has_reverse) rd = a.roff[v + 1] - a.roff[v];
        const bool big = rd > kBigRdeg;
        const unsigned bc = __ballot_sync(FULL, ch), bb = __ballot_sync(FULL, big);
        unsigned long long ps = (unsigned long long)rd;
#pragma unroll
        for (int o = 16; o; o >>= 1) ps += __shfl_xor_sync(FULL, ps, o);
        if (threadIdx.x == 0) spush = 0;
        if (lane == 0) { wcnt[wid] = __popc(bc); wbig[wid] = __popc(bb); }
        __syncthreads();
        if (lane == 0 && ps) atomicAdd(&spush, ps);
        if (threadIdx.x == 0) {
            unsigned tot = 0, totb = 0;
            for (int w = 0; w < 8; ++w) { tot += wcnt[w]; totb += wbig[w]; }
            sbase = tot ? atomicAdd(&a.ctr->list_len, (unsigned long long)tot) : 0;
            bbase = totb ? atomicAdd(&a.ctr->n_big, (unsigned long long)totb) : 0;
        }
        __syncthreads();
        unsigned off = 0, offb = 0;
        for (int w = 0; w < wid; ++w) { off += wcnt[w]; offb += wbig[w]; }
        if (ch) clist[sbase + off + __popc(bc & lanemask_lt())] = (int32_t)v;
        if (big) biglist[bbase + offb + __popc(bb & lanemask_lt())] = (int32_t)v;
        if (threadIdx.x == 0 && spush) atomicAdd(&a.ctr->push_arcs, spush);
        __syncthreads();
    }
}

// --------------------------------------------------------------- outputs --

template <bool F32>
__global__ void finalize_kernel(StepArgs a, const uint8_t *regs, const int32_t *perm, double *closeness,
                                double *harmonic, double *lin, double *reachable) {
    const int P = 1 << a.b;
    const int CH = P >> 4;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < a.n;
         v += (int64_t)gridDim.x * blockDim.x) {
        uint32_t V = 0;
        unsigned long long S = 0;
        const uint4 *row = reinterpret_cast<const uint4 *>(regs + v * P);
        for (int c = 0; c < CH; ++c) chunk_sums(row[c], a.b, V, S);
        double r;
        if (F32) r = (double)estimate32(V, S, P, a.b, a.c32, a.thr_x, a.lc32);
        else r = estimate64(V, S, P, a.b, a.c64, a.thr_x, a.lc64);
        const double s = a.sumd[v];
        const int64_t o = perm ? (int64_t)perm[v] : v;
        if (reachable) reachable[o] = r;
        if (closeness) closeness[o] = s > 0.0 ? __ddiv_rn(1.0, s) : 0.0;
        if (lin) lin[o] = s > 0.0 ? __ddiv_rn(__dmul_rn(r, r), s) : 1.0;
        if (harmonic) harmonic[o] = a.harm[v];
    }
}

__global__ void gather_rows_kernel(const uint8_t *regs, const int32_t *inv, int64_t n, int CH,
                                   uint8_t *out) {
    const int64_t total = n * CH;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < total;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t u = k / CH;
        const int c = (int)(k - u * CH);
        const int64_t v = inv ? (int64_t)inv[u] : u;
        reinterpret_cast<uint4 *>(out)[k] = reinterpret_cast<const uint4 *>(regs)[v * CH + c];
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

int grid_for(int64_t work, int threads) {
    int64_t g = (work + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > 152 * 32) g = 152 * 32;
    return (int)g;
}

template <bool F32>
cudaError_t launch_step_t(const StepArgs &a, int log2m, int grid, cudaStream_t s) {
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
const void *step_kernel_ptr(int log2m) {
    switch (log2m) {
#define HB_CASE(B) case B: return reinterpret_cast<const void *>(&step_kernel<B, F32>);
        HB_CASE(4) HB_CASE(5) HB_CASE(6) HB_CASE(7) HB_CASE(8) HB_CASE(9) HB_CASE(10) HB_CASE(11)
        HB_CASE(12)
#undef HB_CASE
        default: return nullptr;
    }
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
                        cudaStream_t s) {
    const int CH = (1 << a.b) >> 4;
    if (a.n > 0)
        init_rows_kernel<<<grid_for(a.n * CH, 256), 256, 0, s>>>(a.regs[0], a.regs[1], perm, a.n,
                                                                a.b, seed);
    if (fp32) init_nodes_kernel<true><<<grid_for(a.n, 256), 256, 0, s>>>(a, perm, seed);
    else init_nodes_kernel<false><<<grid_for(a.n, 256), 256, 0, s>>>(a, perm, seed);
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
                             cudaStream_t s, cudaEvent_t ev_before, cudaEvent_t ev_after,
                             int *launches) {
    int k = 0;
    step_begin_kernel<<<1, 1, 0, s>>>(a);
    ++k;
    if (a.frontier != HB_FRONTIER_OFF) {
        const int64_t words = (a.n + 31) / 32;
        clear_bits_kernel<<<grid_for(words, 256), 256, 0, s>>>(a, words);
        if (a.frontier == HB_FRONTIER_PULL)
            mark_pull_kernel<<<step_grid, kStepThreads, 0, s>>>(a);
        else if (a.has_reverse)
            mark_push_kernel<<<step_grid, kStepThreads, 0, s>>>(a);
        copy_forward_kernel<<<step_grid, kStepThreads, 0, s>>>(a);
        PlanParams pp{};
        pp.chunk = y.chunk;
        pp.nlight = y.nlight;
        pp.dense = 0;
        plan_kernel<<<1, 1024, 0, s>>>(a, pp, a.plan_sparse, a.owner_sparse, a.cstart_sparse);
        k += (a.frontier == HB_FRONTIER_PULL || a.has_reverse) ? 4 : 3;
    }
    if (ev_before) cudaEventRecord(ev_before, s);
    cudaError_t e = fp32 ? launch_step_t<true>(a, y.log2m, step_grid, s)
                         : launch_step_t<false>(a, y.log2m, step_grid, s);
    if (e != cudaSuccess) return e;
    if (ev_after) cudaEventRecord(ev_after, s);
    if (a.frontier != HB_FRONTIER_OFF) {
        compact_changed_kernel<<<grid_for(a.n, 256), 256, 0, s>>>(a);
        ++k;
    }
    step_end_kernel<<<1, 1, 0, s>>>(a);
    k += 2;
    if (launches) *launches += k;
    return cudaGetLastError();
}

cudaError_t launch_finalize(const StepArgs &a, const uint8_t *regs, const int32_t *perm, bool fp32,
                            double *closeness, double *harmonic, double *lin, double *reachable,
                            cudaStream_t s) {
    if (a.n == 0) return cudaSuccess;
    if (fp32)
        finalize_kernel<true><<<grid_for(a.n, 256), 256, 0, s>>>(a, regs, perm, closeness, harmonic,
                                                                 lin, reachable);
    else
        finalize_kernel<false><<<grid_for(a.n, 256), 256, 0, s>>>(a, regs, perm, closeness, harmonic,
                                                                  lin, reachable);
    return cudaGetLastError();
}

cudaError_t launch_gather_rows(const uint8_t *regs, const int32_t *inv, int64_t n, int P,
                               uint8_t *out, cudaStream_t s) {
    const int CH = P >> 4;
    if (n > 0) gather_rows_kernel<<<grid_for(n * CH, 256), 256, 0, s>>>(regs, inv, n, CH, out);
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

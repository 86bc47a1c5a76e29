// hb_step_dev.cuh -- device-side pieces of one HyperBall iteration shared by
// the single-graph kernels (hb_step.cu) and the batched kernels (hb_batch.cu):
// frontier marking, the gather + register-wise max of a node's successors,
// and the per-node tail (own counter, changed flag, estimator, accumulators).
#pragma once

#include "hb_internal.cuh"
#include "hyperball.h"

// Arcs in flight per lane when a lane holds one 16-byte chunk of a counter,
// and the minimum resident blocks the step kernel is compiled for.
#ifndef HB_UNROLL
#define HB_UNROLL 8
#endif
// Targets staged in shared memory (1) or read from global memory by each
// lane (0), and arcs in flight per lane in the staged gather.
#ifndef HB_STAGE
#define HB_STAGE 0
#endif
#ifndef HB_STAGED_UNROLL
#define HB_STAGED_UNROLL 4
#endif
#ifndef HB_MIN_BLOCKS
#define HB_MIN_BLOCKS 5
#endif
// Streaming stores for data the next iteration reads only after it has
// left L2.
#ifndef HB_STREAM_STORES
#define HB_STREAM_STORES 1
#endif
// Debug builds (libhyperball_debug.so, HB_DEBUG=1) check every arc target
// against [0, n) before its counter is read: a target outside sets
// kErrTarget in the device error word and its arc is skipped.
#ifndef HB_DEBUG
#define HB_DEBUG 0
#endif

namespace hb {
namespace dev {

constexpr unsigned FULL = 0xffffffffu;

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
    if (a.push_union) return;   // arcs are then counted where they are pushed
    unsigned long long dd = key >= 0 ? (unsigned long long)d : 0ULL;
#pragma unroll
    for (int o = 16; o; o >>= 1) dd += __shfl_xor_sync(FULL, dd, o);
    if (lane == 0 && dd) atomicAdd(&a.ctr->arcs, dd);
}

// A successor's counter chunk.  HINT (the one-pass gather with L2
// priorities): counters of nodes below `hint` (the most gathered ones
// after the degree relabelling) are read with the normal L2 eviction
// priority and all others with evict-first and without allocating in L1,
// so that the lines of the cold counters, each read by one or two arcs per
// iteration, leave L2 before the lines of the hot ones and take no L1
// space from them.
// HB_HINT_COLD_NO_L1 = 0 builds let the cold lines allocate in L1 (one
// load instruction with a per-lane policy instead of two predicated ones).
#ifndef HB_HINT_COLD_NO_L1
#define HB_HINT_COLD_NO_L1 1
#endif
template <bool HINT>
__device__ __forceinline__ uint4 ld_counter_h(const uint8_t *p, uint32_t w, uint32_t hint) {
    if constexpr (HINT) {
        uint64_t pn, pf;
        asm("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(pn));
        asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pf));
        uint4 r;
#if HB_HINT_COLD_NO_L1
        if (w < hint)
            asm("ld.global.nc.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
                : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
                : "l"(p), "l"(pn));
        else
            asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
                : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
                : "l"(p), "l"(pf));
#else
        const uint64_t pol = w < hint ? pn : pf;
        asm("ld.global.nc.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
            : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
            : "l"(p), "l"(pol));
#endif
        return r;
    } else {
        (void)w;
        (void)hint;
        return ld_counter(p);
    }
}

// An arc's target, checked against [0, n) in debug builds (-1 if outside).
__device__ __forceinline__ int32_t arc_target(const int32_t *p, int64_t n, unsigned long long *err) {
    const int32_t w = ld_stream(p);
#if HB_DEBUG
    if ((uint64_t)(uint32_t)w >= (uint64_t)n) {
        atomicOr(err, kErrTarget);
        return -1;
    }
#endif
    return w;
}

// Gather the counters of arcs e, e+S, ... < eend (S = 2^logS) into acc
// (this lane's chunks), U arcs in flight per lane; full groups of U arcs
// run without bounds checks (targets were validated at creation; debug
// builds check them here).  n and err serve the debug check only.  WIN:
// only targets w with w - wlo < wspan (unsigned) are gathered, the others
// are skipped (the two-phase gather below).  PK: counters packed six bits
// per register, rows of 3p/4 bytes (chunk k of a row at byte 12 k).
template <int LOG2P, int UMAX, bool WIN = false, bool HINT = false, bool PK = false>
__device__ __forceinline__ void gather_arcs(const int32_t *__restrict__ tgt,
                                            const uint8_t *__restrict__ cur, int64_t e,
                                            int64_t eend, int logS, int cl,
                                            uint4 (&acc)[Cfg<LOG2P>::CPL], int64_t n,
                                            unsigned long long *err, uint32_t wlo = 0u,
                                            uint32_t wspan = 0u, uint32_t hint = 0xffffffffu) {
    using C = Cfg<LOG2P>;
    constexpr int U0 = C::CPL >= 8 ? 1 : (C::CPL == 4 ? 2 : (C::CPL == 2 ? 4 : HB_UNROLL));
    constexpr int U = U0 < UMAX ? U0 : UMAX;
    if (e >= eend) return;
    const int cnt = (int)((eend - e + (1LL << logS) - 1) >> logS);
    const int32_t *tp = tgt + e;
    const uint8_t *base = cur + cl * 16;
    // chunk c of target w's counter (this lane's chunks)
    auto chunk = [&](int32_t w, int c) -> uint4 {
        if constexpr (PK && C::CH == 1)
            return ld_packed_pair(cur, (int64_t)(uint32_t)w);
        else if constexpr (PK)
            return ld_packed(cur + (size_t)(uint32_t)w * (3 * C::P / 4), cl + c * C::L);
        else
            return ld_counter_h<HINT>(base + (size_t)(uint32_t)w * C::P + c * C::L * 16, (uint32_t)w, hint);
    };
    int j = 0;
    for (; j + U <= cnt; j += U) {
        int32_t w[U];
#pragma unroll
        for (int u = 0; u < U; ++u) w[u] = arc_target(tp + ((j + u) << logS), n, err);
        uint4 g[U][C::CPL];
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int c = 0; c < C::CPL; ++c)
#if HB_DEBUG
                g[u][c] = (w[u] >= 0 && (!WIN || (uint32_t)w[u] - wlo < wspan))
                              ? chunk(w[u], c)
                              : make_uint4(0u, 0u, 0u, 0u);
#else
                g[u][c] = (!WIN || (uint32_t)w[u] - wlo < wspan)
                              ? chunk(w[u], c)
                              : make_uint4(0u, 0u, 0u, 0u);
#endif
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int c = 0; c < C::CPL; ++c) acc[c] = vmax16(acc[c], g[u][c]);
    }
    if (j < cnt) {
        const uint4 z = make_uint4(0u, 0u, 0u, 0u);
        int32_t w[U];
#pragma unroll
        for (int u = 0; u < U; ++u) w[u] = j + u < cnt ? arc_target(tp + ((j + u) << logS), n, err) : -1;
        uint4 g[U][C::CPL];
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int c = 0; c < C::CPL; ++c)
                g[u][c] = (w[u] >= 0 && (!WIN || (uint32_t)w[u] - wlo < wspan))
                              ? chunk(w[u], c)
                              : z;
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int c = 0; c < C::CPL; ++c) acc[c] = vmax16(acc[c], g[u][c]);
    }
}

// ------------------------------------------- targets staged in shared memory --
// In dense iterations of a relabelled graph a warp item's nodes are
// consecutive ids, so their arcs are one contiguous range of the target
// array.  The warp copies that range, kTile targets at a time, into its
// shared-memory tile with coalesced 16-byte loads (32 lanes read 512
// contiguous bytes per instruction), and each lane then reads its arcs'
// targets from the tile: one L1 request per 128 targets instead of one per
// arc and lane, and the gathers no longer wait on a global load of their
// target.
constexpr int kTile = 512;                 // targets per warp tile
constexpr int kWarpsPerBlock = kStepThreads / 32;

// Copy targets [cb, ce) (cb a multiple of 4, ce <= cb + kTile, rounded up
// to a multiple of 4 as far as targets exist, < m) into tile; called by
// the whole warp, followed by __syncwarp.
__device__ __forceinline__ void load_tile(int32_t *tile, const int32_t *__restrict__ tgt, int64_t cb,
                                          int64_t ce, int64_t m, int lane) {
    const int nq = (int)((ce - cb + 3) >> 2);
    for (int q = lane; q < nq; q += 32) {
        const int64_t e = cb + 4 * q;
        if (e + 4 <= m) {
            reinterpret_cast<int4 *>(tile)[q] = __ldcs(reinterpret_cast<const int4 *>(tgt + e));
        } else {
            for (int i = 0; i < 4; ++i)
                if (e + i < m) tile[4 * q + i] = ld_stream(tgt + e + i);
        }
    }
}

// As gather_arcs, for arcs e, e+S, ... < eend that all lie in the tile
// holding targets [cb, cb + kTile).
template <int LOG2P, int UMAX, bool WIN = false>
__device__ __forceinline__ void gather_staged(const int32_t *tile, int64_t cb,
                                              const uint8_t *__restrict__ cur, int64_t e, int64_t eend,
                                              int logS, int cl, uint4 (&acc)[Cfg<LOG2P>::CPL], int64_t n,
                                              unsigned long long *err, uint32_t wlo, uint32_t wspan) {
    using C = Cfg<LOG2P>;
    constexpr int U0 = C::CPL >= 8 ? 1 : (C::CPL == 4 ? 2 : (C::CPL == 2 ? 4 : HB_STAGED_UNROLL));
    constexpr int U = U0 < UMAX ? U0 : UMAX;
    if (e >= eend) return;
    const int cnt = (int)((eend - e + (1LL << logS) - 1) >> logS);
    const int32_t *tp = tile + (e - cb);
    const uint8_t *base = cur + cl * 16;
    const uint4 z = make_uint4(0u, 0u, 0u, 0u);
    for (int j = 0; j < cnt; j += U) {
        int32_t w[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            w[u] = j + u < cnt ? tp[(j + u) << logS] : -1;
#if HB_DEBUG
            if (w[u] >= 0 && (uint64_t)(uint32_t)w[u] >= (uint64_t)n) {
                atomicOr(err, kErrTarget);
                w[u] = -1;
            }
#endif
        }
        uint4 g[U][C::CPL];
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int c = 0; c < C::CPL; ++c)
                g[u][c] = (w[u] >= 0 && (!WIN || (uint32_t)w[u] - wlo < wspan))
                              ? ld_counter(base + (size_t)(uint32_t)w[u] * C::P + c * C::L * 16)
                              : z;
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int c = 0; c < C::CPL; ++c) acc[c] = vmax16(acc[c], g[u][c]);
    }
}

// The arcs e0, e0+S, ... < e1 of one lane, gathered tile by tile over the
// warp's contiguous arc range [A0, A1) (which contains [e0, e1)).  Called
// by the whole warp.
template <int LOG2P, int UMAX, bool WIN = false>
__device__ __forceinline__ void gather_range_staged(int32_t *tile, const int32_t *__restrict__ tgt, int64_t m,
                                                    const uint8_t *__restrict__ cur, int64_t A0, int64_t A1,
                                                    int64_t e0, int64_t e1, int logS, int cl,
                                                    uint4 (&acc)[Cfg<LOG2P>::CPL], int64_t n,
                                                    unsigned long long *err, uint32_t wlo, uint32_t wspan) {
    const int lane = threadIdx.x & 31;
    const int64_t S = 1LL << logS;
    for (int64_t cb = A0 & ~(int64_t)3; cb < A1; cb += kTile) {
        __syncwarp();
        load_tile(tile, tgt, cb, cb + kTile < A1 ? cb + kTile : A1, m, lane);
        __syncwarp();
        const int64_t ce = cb + kTile < e1 ? cb + kTile : e1;
        int64_t e = e0;
        if (e < cb) e += ((cb - e + S - 1) >> logS) << logS;
        if (e < ce) gather_staged<LOG2P, UMAX, WIN>(tile, cb, cur, e, ce, logS, cl, acc, n, err, wlo, wspan);
    }
}

// Pull the node's accumulators and cached estimate into L2 while its
// successors are gathered (used when most nodes are expected to change).
__device__ __forceinline__ void prefetch_accumulators(const StepArgs &a, int64_t v, bool f32) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(a.sumd + v));
    asm volatile("prefetch.global.L2 [%0];" ::"l"(a.harm + v));
    if (f32) asm volatile("prefetch.global.L2 [%0];" ::"l"(static_cast<float *>(a.ecache) + v));
    else asm volatile("prefetch.global.L2 [%0];" ::"l"(static_cast<double *>(a.ecache) + v));
    if (a.disc) asm volatile("prefetch.global.L2 [%0];" ::"l"(a.disc + v));
}

// f(t+1), the discount of the layer that iteration t adds (Sec. 7).
__device__ __forceinline__ double discount_of(const StepArgs &a, int t) {
    return t < a.flen ? a.ftab[t] : 0.0;
}

// Per-node tail, called by all 32 lanes.  acc holds the union of the
// successors' counters (this lane's chunks; every slot of the team holds
// the same).  Folds in the node's own counter, writes it to the write
// buffer, sets the changed flag, and for changed nodes evaluates size()
// and updates the accumulators (Sec. 5), appending the node to the changed
// list.  PK: rows packed six bits per register.
template <int LOG2P, bool F32, bool PK = false>
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
            const uint4 o = PK ? ld_packed(cur + v * (3 * C::P / 4), cl + c * C::L)
                               : ld_counter(own + c * C::L * 16);
            const uint4 nv = vmax16(acc[c], o);
            diff |= ne16(nv, o);
            acc[c] = nv;
        }
    }
    const unsigned bal = __ballot_sync(FULL, diff);
    const unsigned tmask = logT == 5 ? FULL : (((1u << (1 << logT)) - 1u) << (team << logT));
    const bool ch = (bal & tmask) != 0u;
    if (PK && active && tl < C::L) {
#pragma unroll
        for (int c = 0; c < C::CPL; ++c) st_packed(nxt + v * (3 * C::P / 4), cl + c * C::L, acc[c]);
    } else if (active && tl < C::L) {
        uint8_t *dst = nxt + v * C::P + cl * 16;
#pragma unroll
        for (int c = 0; c < C::CPL; ++c) {
#if HB_STREAM_STORES
            __stcs(reinterpret_cast<uint4 *>(dst + c * C::L * 16), acc[c]);
#else
            *reinterpret_cast<uint4 *>(dst + c * C::L * 16) = acc[c];
#endif
        }
    }
    const bool leader = active && tl == 0;
    // The accumulator loads go out together, before any store of this
    // node: the three arrays may alias as far as the compiler knows, so a
    // load placed after a store would wait a full round trip for it.
    double s_old = 0.0, h_old = 0.0, e_old = 0.0, q_old = 0.0;
    if (leader && ch) {
        s_old = a.sumd[v];
        h_old = a.harm[v];
        e_old = F32 ? (double)static_cast<const float *>(a.ecache)[v]
                    : static_cast<const double *>(a.ecache)[v];
        if (a.disc) q_old = a.disc[v];
    }
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
            const float E = estimate32(V, S, C::P, a.b, a.c32, a.thr_x, a.lc32);
            const float d = __fsub_rn(E, (float)e_old);
            static_cast<float *>(a.ecache)[v] = E;
            a.sumd[v] = __fma_rn((double)(t + 1), (double)d, s_old);   // exact product
            a.harm[v] = __dadd_rn(h_old, (double)__fmul_rn(d, rdist32));
            if (a.disc) a.disc[v] = __fma_rn(discount_of(a, t), (double)d, q_old);
        } else {
            const double E = estimate64(V, S, C::P, a.b, a.c64, a.thr_x, a.lc64);
            const double d = __dsub_rn(E, e_old);
            static_cast<double *>(a.ecache)[v] = E;
            a.sumd[v] = __fma_rn((double)(t + 1), d, s_old);
            a.harm[v] = __fma_rn(d, rdist64, h_old);
            if (a.disc) a.disc[v] = __fma_rn(discount_of(a, t), d, q_old);
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

// Per-node tail for rows that hold 2^lruns runs of p = 2^gb registers each
// (hb_create_runs).  Run r owns bytes [r p, (r+1) p) of the row; the
// register-wise max never mixes bytes, so the row's union is every run's
// union at once.  The row write, changed flag and changed lists are those
// of node_epilogue (a node changed if any of its runs did).  Then every run
// whose registers changed gets its own size(), delta and Sec. 5
// accumulators at index v * runs + r, and sets bit r of the iteration's run
// mask (s_changed[1]); s_changed[0] counts changed nodes.
template <int LOG2P, bool F32>
__device__ __forceinline__ void node_epilogue_wide(const StepArgs &a, const uint8_t *__restrict__ cur,
                                                   uint8_t *__restrict__ nxt, int t, int64_t v,
                                                   bool active, uint4 (&acc)[Cfg<LOG2P>::CPL], int cl,
                                                   int tl, int team, int logT, int32_t *clist,
                                                   int32_t *biglist, bool sparse,
                                                   unsigned long long *s_changed, double rdist64,
                                                   float rdist32, const unsigned long long *pow2) {
    using C = Cfg<LOG2P>;
    const int lane = threadIdx.x & 31;
    bool cd[C::CPL];
    bool diff = false;
#pragma unroll
    for (int c = 0; c < C::CPL; ++c) cd[c] = false;
    if (active) {
        const uint8_t *own = cur + v * C::P + cl * 16;
#pragma unroll
        for (int c = 0; c < C::CPL; ++c) {
            const uint4 o = ld_counter(own + c * C::L * 16);
            const uint4 nv = vmax16(acc[c], o);
            cd[c] = ne16(nv, o);
            diff |= cd[c];
            acc[c] = nv;
        }
    }
    const unsigned bal = __ballot_sync(FULL, diff);
    const unsigned tmask = logT == 5 ? FULL : (((1u << (1 << logT)) - 1u) << (team << logT));
    const bool ch = (bal & tmask) != 0u;
    if (active && tl < C::L) {
        uint8_t *dst = nxt + v * C::P + cl * 16;
#pragma unroll
        for (int c = 0; c < C::CPL; ++c) __stcs(reinterpret_cast<uint4 *>(dst + c * C::L * 16), acc[c]);
    }
    const bool leader = active && tl == 0;
    if (leader) a.changed[v] = ch ? 1 : 0;
    const unsigned lb = __ballot_sync(FULL, leader && ch);
    if (lb == 0u) return;

    // A run's Gc = p/16 chunks sit in Gc consecutive chunk lanes (Gc <= L):
    // chunk k of lane cl is chunk cl + k L of the row.  Sum each chunk's
    // zero count and fixed-point sum over the run's lanes; the lane holding
    // the run's first chunk finishes the run.
    const int lg = a.gb - 4;
    const int P = 1 << a.gb;
    unsigned long long rmask = 0;
#pragma unroll
    for (int c = 0; c < C::CPL; ++c) {
        uint32_t V = 0;
        unsigned long long S = 0;
        chunk_sums_tab(acc[c], pow2, V, S);
        unsigned g = cd[c] ? 1u : 0u;
        for (int o = 1; o < (1 << lg); o <<= 1) {
            V += __shfl_xor_sync(FULL, V, o);
            S += __shfl_xor_sync(FULL, S, o);
            g |= __shfl_xor_sync(FULL, g, o);
        }
        const int r = (cl + c * C::L) >> lg;
        if (active && ch && g && tl < C::L && (cl & ((1 << lg) - 1)) == 0) {
            const int64_t q = (v << a.lruns) + r;
            const double s_old = a.sumd[q], h_old = a.harm[q];
            const double q_old = a.disc ? a.disc[q] : 0.0;
            // Sec. 5: the new layer sits at distance t+1
            if (F32) {
                const float e_old = static_cast<const float *>(a.ecache)[q];
                const float E = estimate32(V, S, P, a.gb, a.c32, a.thr_x, a.lc32);
                const float d = __fsub_rn(E, e_old);
                static_cast<float *>(a.ecache)[q] = E;
                a.sumd[q] = __fma_rn((double)(t + 1), (double)d, s_old);
                a.harm[q] = __dadd_rn(h_old, (double)__fmul_rn(d, rdist32));
                if (a.disc) a.disc[q] = __fma_rn(discount_of(a, t), (double)d, q_old);
            } else {
                const double e_old = static_cast<const double *>(a.ecache)[q];
                const double E = estimate64(V, S, P, a.gb, a.c64, a.thr_x, a.lc64);
                const double d = __dsub_rn(E, e_old);
                static_cast<double *>(a.ecache)[q] = E;
                a.sumd[q] = __fma_rn((double)(t + 1), d, s_old);
                a.harm[q] = __fma_rn(d, rdist64, h_old);
                if (a.disc) a.disc[q] = __fma_rn(discount_of(a, t), d, q_old);
            }
            rmask |= 1ULL << r;
        }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) rmask |= __shfl_xor_sync(FULL, rmask, o);
    if (lane == 0) {
        atomicAdd(s_changed, (unsigned long long)__popc(lb));
        if (rmask) atomicOr(s_changed + 1, rmask);
    }
    if (!sparse) return;   // dense iterations: the changed list is compacted afterwards
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(&a.ctr->list_len, (unsigned long long)__popc(lb));
    base = __shfl_sync(FULL, base, 0);
    if (leader && ch) clist[base + __popc(lb & lanemask_lt())] = (int32_t)v;
    if (a.has_reverse) {
        const int64_t rd = (leader && ch) ? a.roff[v + 1] - a.roff[v] : 0;
        unsigned long long sr = (unsigned long long)rd;
#pragma unroll
        for (int o = 16; o; o >>= 1) sr += __shfl_xor_sync(FULL, sr, o);
        if (lane == 0 && sr) atomicAdd(&a.ctr->push_arcs, sr);
        const unsigned bb = __ballot_sync(FULL, rd > kBigRdeg);
        if (bb) {
            unsigned long long bbase = 0;
            if (lane == 0) bbase = atomicAdd(&a.ctr->n_big, (unsigned long long)__popc(bb));
            bbase = __shfl_sync(FULL, bbase, 0);
            if (rd > kBigRdeg) biglist[bbase + __popc(bb & lanemask_lt())] = (int32_t)v;
        }
    }
}

// The tail of one node: node_epilogue, or node_epilogue_wide for rows of
// several runs.
template <int LOG2P, bool F32, bool WIDE, bool PK = false>
__device__ __forceinline__ void node_tail(const StepArgs &a, const uint8_t *__restrict__ cur,
                                          uint8_t *__restrict__ nxt, int t, int64_t v, bool active,
                                          uint4 (&acc)[Cfg<LOG2P>::CPL], int cl, int tl, int team,
                                          int logT, int32_t *clist, int32_t *biglist, bool sparse,
                                          unsigned long long *s_changed, double rdist64, float rdist32,
                                          const unsigned long long *pow2) {
    if constexpr (WIDE)
        node_epilogue_wide<LOG2P, F32>(a, cur, nxt, t, v, active, acc, cl, tl, team, logT, clist, biglist,
                                       sparse, s_changed, rdist64, rdist32, pow2);
    else
        node_epilogue<LOG2P, F32, PK>(a, cur, nxt, t, v, active, acc, cl, tl, team, logT, clist, biglist,
                                      sparse, s_changed, rdist64, rdist32, pow2);
}

// The two-phase gather of a dense iteration (StepArgs::hot > 0): a first
// launch (pass 1) gathers only the arcs into the hot counters [0, hot) and
// leaves each node's partial union in its write-buffer row; a second
// launch (pass 2) gathers the other arcs, folds that partial in and runs the
// per-node tail.  The register-wise max is associative and commutative, so
// the union is the same as one pass over all arcs; only the order in which
// the counters are read changes, so that while pass 1 runs the random
// reads touch a set of counters small enough to stay in L2.
struct Window {
    uint32_t lo, span;   // targets w with w - lo < span (unsigned) are gathered
    int pass;            // 0: one pass over all arcs; 1, 2: the passes above
};

// Pass 1: the partial union of a node goes to its write-buffer row.
template <int LOG2P>
__device__ __forceinline__ void store_partial(uint8_t *__restrict__ nxt, int64_t v, int cl,
                                              const uint4 (&acc)[Cfg<LOG2P>::CPL]) {
    using C = Cfg<LOG2P>;
    uint8_t *dst = nxt + v * C::P + cl * 16;
#pragma unroll
    for (int c = 0; c < C::CPL; ++c) __stcs(reinterpret_cast<uint4 *>(dst + c * C::L * 16), acc[c]);
}

// Pass 2: fold in the partial union pass 1 left in the write-buffer row.
template <int LOG2P>
__device__ __forceinline__ void fold_partial(const uint8_t *__restrict__ nxt, int64_t v, int cl,
                                             uint4 (&acc)[Cfg<LOG2P>::CPL]) {
    using C = Cfg<LOG2P>;
    const uint8_t *src = nxt + v * C::P + cl * 16;
#pragma unroll
    for (int c = 0; c < C::CPL; ++c)
        acc[c] = vmax16(acc[c], __ldcs(reinterpret_cast<const uint4 *>(src + c * C::L * 16)));
}

template <int LOG2P, bool F32, bool WIDE = false, bool WIN = false, bool HINT = false, bool PK = false>
__device__ __forceinline__ void light_item(const StepArgs &a, const uint8_t *__restrict__ cur,
                                           uint8_t *__restrict__ nxt, int t, int64_t pos0,
                                           int64_t pos_end, int logS, const int32_t *list,
                                           int32_t *clist, int32_t *biglist, bool sparse,
                                           unsigned long long *s_changed, double rdist64,
                                           float rdist32, const unsigned long long *pow2,
                                           bool prefetch, Window win = Window{0u, 0u, 0},
                                           int32_t *tile = nullptr) {
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
        if (WIN && win.pass != 0 && a.hcnt) {
            // partitioned lists: the hot targets are the node's first hcnt[v] arcs
            const int64_t sp = e0 + a.hcnt[v];
            if (win.pass == 1) e1 = sp;
            else e0 = sp;
        }
        if (prefetch && tl == 0) prefetch_accumulators(a, v, F32);
    }
    uint4 acc[C::CPL];
#pragma unroll
    for (int c = 0; c < C::CPL; ++c) acc[c] = make_uint4(0u, 0u, 0u, 0u);
    const uint32_t wlo = win.lo, wspan = win.span;
    if (tile) {
        // consecutive nodes pos0 .. : their arcs are one contiguous range
        const int64_t plast = pos0 + (32 >> logT) < pos_end ? pos0 + (32 >> logT) : pos_end;
        const int64_t A0 = a.off[pos0], A1 = a.off[plast];
        if (a.aps <= 2)
            gather_range_staged<LOG2P, 2, WIN>(tile, a.tgt, a.m, cur, A0, A1, e0 + slot, e1, logS, cl, acc, a.n,
                                               &a.ctr->err, wlo, wspan);
        else if (a.aps <= 4 && logS != C::LOGSMAX)
            gather_range_staged<LOG2P, 4, WIN>(tile, a.tgt, a.m, cur, A0, A1, e0 + slot, e1, logS, cl, acc, a.n,
                                               &a.ctr->err, wlo, wspan);
        else
            gather_range_staged<LOG2P, 64, WIN>(tile, a.tgt, a.m, cur, A0, A1, e0 + slot, e1, logS, cl, acc,
                                                a.n, &a.ctr->err, wlo, wspan);
    } else if (logS == C::LOGSMAX)
        gather_arcs<LOG2P, 64, WIN, HINT, PK>(a.tgt, cur, e0 + slot, e1, logS, cl, acc, a.n, &a.ctr->err, wlo,
                                              wspan, a.hint);
    else if (a.aps <= 2)
        gather_arcs<LOG2P, 2, WIN, HINT, PK>(a.tgt, cur, e0 + slot, e1, logS, cl, acc, a.n, &a.ctr->err, wlo,
                                             wspan, a.hint);
    else if (a.aps <= 4)
        gather_arcs<LOG2P, 4, WIN, HINT, PK>(a.tgt, cur, e0 + slot, e1, logS, cl, acc, a.n, &a.ctr->err, wlo,
                                             wspan, a.hint);
    else
        gather_arcs<LOG2P, 64, WIN, HINT, PK>(a.tgt, cur, e0 + slot, e1, logS, cl, acc, a.n, &a.ctr->err, wlo,
                                              wspan, a.hint);
    for (int o = C::L; o < (1 << logT); o <<= 1)
#pragma unroll
        for (int c = 0; c < C::CPL; ++c) acc[c] = vmax16(acc[c], shfl_xor16(acc[c], o));
    if (WIN && win.pass == 1) {
        if (active && tl < C::L) store_partial<LOG2P>(nxt, v, cl, acc);
        return;
    }
    if (WIN && win.pass == 2 && active) fold_partial<LOG2P>(nxt, v, cl, acc);
    node_tail<LOG2P, F32, WIDE, PK>(a, cur, nxt, t, v, active, acc, cl, tl, team, logT, clist, biglist,
                                    sparse, s_changed, rdist64, rdist32, pow2);
}

// One chunk of a heavy node, by a whole warp.  Each chunk leaves its
// partial union in scratch; the last chunk to arrive combines them and
// finishes the node.  The partial unions stay one byte per register.
template <int LOG2P, bool F32, bool WIDE = false, bool WIN = false, bool HINT = false, bool PK = false>
__device__ __forceinline__ void heavy_item(const StepArgs &a, const uint8_t *__restrict__ cur,
                                           uint8_t *__restrict__ nxt, int t, int64_t it,
                                           const int32_t *owner, const int64_t *cstart,
                                           const int32_t *list, int32_t *clist, int32_t *biglist,
                                           bool sparse, unsigned long long *s_changed,
                                           double rdist64, float rdist32,
                                           const unsigned long long *pow2,
                                           Window win = Window{0u, 0u, 0}, int32_t *tile = nullptr) {
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
    int64_t e0 = a.off[v] + k * C::CHUNK;
    int64_t e1 = e0 + C::CHUNK < a1 ? e0 + C::CHUNK : a1;
    if (WIN && win.pass != 0 && a.hcnt) {
        // partitioned lists: this pass takes the chunk's part of the node's
        // first hcnt[v] arcs (pass 1) or of the rest (pass 2)
        const int64_t sp = a.off[v] + a.hcnt[v];
        if (win.pass == 1) e1 = e1 < sp ? e1 : sp;
        else e0 = e0 > sp ? e0 : sp;
        if (e1 < e0) e1 = e0;
    }
    uint4 acc[C::CPL];
#pragma unroll
    for (int c = 0; c < C::CPL; ++c) acc[c] = make_uint4(0u, 0u, 0u, 0u);
    if (tile)
        gather_range_staged<LOG2P, 64, WIN>(tile, a.tgt, a.m, cur, e0, e1, e0 + slot, e1, C::LOGSMAX, cl, acc,
                                            a.n, &a.ctr->err, win.lo, win.span);
    else
        gather_arcs<LOG2P, 64, WIN, HINT, PK>(a.tgt, cur, e0 + slot, e1, C::LOGSMAX, cl, acc, a.n, &a.ctr->err,
                                              win.lo, win.span, a.hint);
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
    if (WIN && win.pass == 1) {
        if (slot == 0) store_partial<LOG2P>(nxt, v, cl, acc);
        return;
    }
    if (WIN && win.pass == 2) fold_partial<LOG2P>(nxt, v, cl, acc);
    node_tail<LOG2P, F32, WIDE, PK>(a, cur, nxt, t, v, true, acc, cl, lane, 0, 5, clist, biglist, sparse,
                                    s_changed, rdist64, rdist32, pow2);
}

// Start of an iteration for one graph: shift this iteration's counters
// into the "previous" slots and choose dense or sparse (frontier) mode.
__device__ __forceinline__ void begin_one(const StepArgs &a) {
    Counters *c = a.ctr;
    const int t = c->steps_done;
    c->t = t;
    c->prev_changed = c->n_changed;
    c->prev_list_len = c->list_len;
    c->prev_push_arcs = c->push_arcs;
    c->prev_big = c->n_big;
    c->n_changed = 0; c->list_len = 0; c->push_arcs = 0; c->n_big = 0; c->arcs = 0;
    c->run_mask = 0;
    for (int s = 0; s < kSegs; ++s) c->fill[s] = 0;
    int sparse = 0;
    if (t > 0) {
        if (a.frontier == HB_FRONTIER_PULL) sparse = 1;
        else if (a.frontier == HB_FRONTIER_PUSH) sparse = a.has_reverse;
        else if (a.frontier == HB_FRONTIER_AUTO)
            sparse = a.has_reverse && (double)c->prev_push_arcs <= a.sparse_frac * (double)a.m;
    }
    c->mode = sparse;
    // pushed frontier iterations examine exactly the arcs into last
    // iteration's changed nodes
    if (sparse && a.push_union) c->arcs = c->prev_push_arcs;
}

// End of an iteration: count it and record convergence (Sec. 4.2: stop
// after the first iteration that changes no counter).
__device__ __forceinline__ void end_one(const StepArgs &a) {
    Counters *c = a.ctr;
    c->steps_done = c->t + 1;
    if (c->n_changed == 0) c->converged = 1;
}

// Push marking by one warp: the predecessors of changed node w.
__device__ __forceinline__ void push_warp(const StepArgs &a, int32_t w, int lane) {
    const int64_t r0 = a.roff[w], r1 = a.roff[w + 1];
    for (int64_t j0 = r0; j0 < r1; j0 += 32) {
        const int64_t j = j0 + lane;
        mark_append(a, j < r1 ? a.rtgt[j] : -1, lane);
    }
}

// Copy-forward element k (node index k / CH of the previous changed list,
// chunk k % CH): clears the node's changed flag and, unless the node is
// recomputed in this iteration, copies that chunk of its counter into the
// write buffer.
__device__ __forceinline__ void copy_forward_one(const StepArgs &a, int t, int64_t k) {
    const int32_t *prev = a.clist[(t + 1) & 1];
    const uint8_t *cur = a.regs[t & 1];
    uint8_t *nxt = a.regs[(t + 1) & 1];
    const int logCH = a.b - 4;
    const int64_t i = k >> logCH;
    const int ch = (int)(k & ((1 << logCH) - 1));
    const int32_t w = prev[i];
    if (ch == 0) a.changed[w] = 0;
    if (!((a.mustbits[w >> 5] >> (w & 31)) & 1u)) {
        const int64_t o = ((int64_t)w << logCH) + ch;
        reinterpret_cast<uint4 *>(nxt)[o] = reinterpret_cast<const uint4 *>(cur)[o];
    }
}

// Pushed union (frontier iterations with the reverse CSR).  For t >= 1 a
// successor w that did not change in iteration t-1 has c_t[w] = c_{t-1}[w]
// <= c_t[v] register by register (Jacobi: c_t[v] already holds the max over
// v's successors at t-1), so it adds nothing to v's union.  The union of a
// recomputed node therefore needs only its successors that changed last
// time, which the reverse CSR of those nodes enumerates: each changed
// node's counter is folded into the write-buffer counter of each
// predecessor with a byte-wise atomic max.  The write buffer holds c_{t-1}
// before the iteration (<= c_t), and the per-node tail folds in c_t[v], so
// every recomputed node ends with exactly the union of Algorithm 2.
// One pair (w, v) by a team of G lanes, chunks tl, tl + G, ...; only words
// that would grow are written.
__device__ __forceinline__ void push_pair(const StepArgs &a, const uint4 *cur4, uint4 *nxt4, int32_t w,
                                          int32_t v, int logCH, int tl, int G) {
    const int CH = 1 << logCH;
    const uint4 *src = cur4 + ((int64_t)w << logCH);
    uint4 *dst = nxt4 + ((int64_t)v << logCH);
    for (int ch = tl; ch < CH; ch += G) {
        const uint4 x = __ldg(src + ch);
        const uint4 y = __ldcg(dst + ch);
        if (!ne16(vmax16(y, x), y)) continue;
        uint32_t *d32 = reinterpret_cast<uint32_t *>(dst + ch);
        if (bmax4(y.x, x.x) != y.x) atomic_bmax4(d32 + 0, x.x, &a.ctr->err);
        if (bmax4(y.y, x.y) != y.y) atomic_bmax4(d32 + 1, x.y, &a.ctr->err);
        if (bmax4(y.z, x.z) != y.z) atomic_bmax4(d32 + 2, x.z, &a.ctr->err);
        if (bmax4(y.w, x.w) != y.w) atomic_bmax4(d32 + 3, x.w, &a.ctr->err);
    }
}

// The changed nodes prev[base .. base + 32) of the last iteration (np in
// all): every pair (w, predecessor v) is pushed and v marked.  The pairs of
// the 32 nodes are spread over teams of G lanes (a warp scan of their
// predecessor counts, then a binary search over it by shuffles), so nodes
// with few predecessors leave no lane idle.  Nodes with more than kBigRdeg
// predecessors are skipped here (push_union_big).  Called by a whole warp.
__device__ __forceinline__ void push_union_item(const StepArgs &a, const uint4 *cur4, uint4 *nxt4,
                                                const int32_t *prev, int64_t np, int64_t base,
                                                int logCH, int lane) {
    const int logG = logCH < 5 ? logCH : 5;
    const int team = lane >> logG;
    const int tl = lane & ((1 << logG) - 1);
    const int ppw = 32 >> logG;   // pairs per warp pass
    const int64_t i = base + lane;
    int32_t w = 0;
    int64_t r0 = 0;
    int cnt = 0;   // predecessors, <= kBigRdeg
    if (i < np) {
        w = prev[i];
        r0 = a.roff[w];
        const int64_t rd = a.roff[w + 1] - r0;
        if (rd <= kBigRdeg) cnt = (int)rd;
    }
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += y;
    }
    const int total = __shfl_sync(FULL, incl, 31);
    const int excl = incl - cnt;
    for (int eb = 0; eb < total; eb += ppw) {
        const int e = eb + team;
        // owner: the first lane whose inclusive count exceeds e
        int q = 0;
#pragma unroll
        for (int s = 16; s; s >>= 1)
            if (__shfl_sync(FULL, incl, q + s - 1) <= e) q += s;
        const int32_t ow = __shfl_sync(FULL, w, q);
        const int64_t or0 = __shfl_sync(FULL, r0, q);
        const int oex = __shfl_sync(FULL, excl, q);
        int32_t v = -1;
        if (e < total) {
            v = a.rtgt[or0 + (e - oex)];
            push_pair(a, cur4, nxt4, ow, v, logCH, tl, 1 << logG);
        }
        mark_append(a, tl == 0 ? v : -1, lane);
    }
}

// The pairs of one changed node w with many predecessors, by warp wi of
// nwi warps.
__device__ __forceinline__ void push_union_big(const StepArgs &a, const uint4 *cur4, uint4 *nxt4,
                                               int32_t w, int64_t wi, int64_t nwi, int logCH, int lane) {
    const int logG = logCH < 5 ? logCH : 5;
    const int team = lane >> logG;
    const int tl = lane & ((1 << logG) - 1);
    const int ppw = 32 >> logG;
    const int64_t r0 = a.roff[w], rd = a.roff[w + 1] - r0;
    for (int64_t pb = wi * ppw; pb < rd; pb += nwi * ppw) {
        const int64_t e = pb + team;
        int32_t v = -1;
        if (e < rd) {
            v = a.rtgt[r0 + e];
            push_pair(a, cur4, nxt4, w, v, logCH, tl, 1 << logG);
        }
        mark_append(a, tl == 0 ? v : -1, lane);
    }
}

// Per-node tail of a pushed frontier iteration for the marked nodes at
// flat positions base .. base + 32/L of the sparse list (by degree
// segment): the pushed union is read back from the write buffer and goes
// through the same tail as a gathered node (own counter folded in,
// changed flag, estimator, accumulators, changed list).  One team of L
// lanes per node; called by a whole warp.
template <int LOG2P, bool F32, bool WIDE = false>
__device__ __forceinline__ void union_tail_item(const StepArgs &a, int t, int64_t base,
                                                unsigned long long *cnt, double rdist64, float rdist32,
                                                const unsigned long long *pow2) {
    using C = Cfg<LOG2P>;
    const Counters *ctr = a.ctr;
    const uint8_t *cur = a.regs[t & 1];
    uint8_t *nxt = a.regs[(t + 1) & 1];
    int64_t start[kSegs + 1];
    start[0] = 0;
#pragma unroll
    for (int s = 0; s < kSegs; ++s) start[s + 1] = start[s] + (int64_t)ctr->fill[s];
    const int lane = threadIdx.x & 31;
    const int team = lane >> C::LOGL;
    const int tl = lane & (C::L - 1);
    const int64_t i = base + team;
    const bool active = i < start[kSegs];
    int64_t v = 0;
    uint4 acc[C::CPL];
#pragma unroll
    for (int c = 0; c < C::CPL; ++c) acc[c] = make_uint4(0u, 0u, 0u, 0u);
    if (active) {
        int64_t pos = a.seg_begin[0] + i;
#pragma unroll
        for (int s = 1; s < kSegs; ++s)
            if (i >= start[s]) pos = a.seg_begin[s] + (i - start[s]);
        v = a.slist[pos];
        const uint4 *row = reinterpret_cast<const uint4 *>(nxt + v * C::P) + tl;
#pragma unroll
        for (int c = 0; c < C::CPL; ++c) acc[c] = __ldcg(row + c * C::L);
    }
    node_tail<LOG2P, F32, WIDE>(a, cur, nxt, t, v, active, acc, tl, tl, team, C::LOGL, a.clist[t & 1],
                                a.biglist[t & 1], true, cnt, rdist64, rdist32, pow2);
}

// The gather kernel's body: every work item of the iteration's plan (heavy
// chunks, then light items of each degree class), with the per-node tail
// of one run per row or, WIDE, of several runs per row.  PK: packed rows
// (dense iterations only, no staging).
template <int LOG2P, bool F32, bool WIDE, bool WIN = false, bool HINT = false, bool PK = false>
__device__ __forceinline__ void step_body(const StepArgs &a) {
    using C = Cfg<LOG2P>;
    const Counters *ctr = a.ctr;
    const int t = ctr->t;
    const bool sparse = ctr->mode == 1;
    // WIN: launch a.pass = 1 or 2 of the two-phase gather in dense
    // iterations; frontier iterations take one pass over all arcs, in the
    // pass-2 launch
    Window win{0u, 0xffffffffu, 0};
    if (WIN) {
        if (sparse) {
            if (a.pass == 1) return;
        } else if (a.hcnt) {
            // partitioned lists: each pass takes its own part of every list
            win = Window{0u, 0xffffffffu, a.pass == 1 ? 1 : 2};
        } else if (a.pass == 1) {
            win = Window{0u, a.hot, 1};
        } else {
            win = Window{a.hot, (uint32_t)a.n - a.hot, 2};
        }
    }
    const Plan *pl = sparse ? a.plan_sparse : a.plan_dense;
    const int32_t *list = sparse ? a.slist : a.dense_list;
    const int32_t *owner = sparse ? a.owner_sparse : a.owner_dense;
    const int64_t *cstart = sparse ? a.cstart_sparse : a.cstart_dense;
    const uint8_t *cur = a.regs[t & 1];
    uint8_t *nxt = a.regs[(t + 1) & 1];
    int32_t *clist = a.clist[t & 1];
    int32_t *biglist = a.biglist[t & 1];
    if (sparse && a.push_union) return;   // the pushed union does this iteration
    const int64_t items = pl->items;
    const int64_t hch = pl->heavy_chunks;
    int64_t ib[C::NLIGHT + 1], cnt[C::NLIGHT];
#pragma unroll
    for (int j = 0; j <= C::NLIGHT; ++j) ib[j] = pl->item_begin[j];
#pragma unroll
    for (int j = 0; j < C::NLIGHT; ++j) cnt[j] = pl->count[j + 1];
    __shared__ unsigned long long s_changed[2];   // changed nodes; WIDE: mask of changed runs
    __shared__ unsigned long long s_pow2[64];
    __shared__ int4 s_tile[kWarpsPerBlock][kTile / 4];
    // targets staged in shared memory when a warp item's nodes are
    // consecutive ids (no node list) and the target array is 16-byte aligned
    int32_t *tile = (HB_STAGE && !PK && list == nullptr && (reinterpret_cast<uintptr_t>(a.tgt) & 15) == 0)
                        ? reinterpret_cast<int32_t *>(s_tile[threadIdx.x >> 5])
                        : nullptr;
    const double rdist64 = 1.0 / (double)(t + 1);
    const float rdist32 = 1.0f / (float)(t + 1);
    // most nodes change in the first iterations: fetch their accumulators early
    const bool prefetch = !sparse && win.pass != 1 && (t == 0 || 4 * (int64_t)ctr->prev_changed > a.n_pos);
    if (threadIdx.x < 2) s_changed[threadIdx.x] = 0;
    if (threadIdx.x < 64) {
        const int M = threadIdx.x, sh = 64 - (WIDE ? a.gb : a.b);
        s_pow2[M] = (M == 0 || M > sh) ? 0ULL : 1ULL << (sh - M);
    }
    __syncthreads();
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t it = gw; it < items; it += nw) {
        if (it < hch) {
            heavy_item<LOG2P, F32, WIDE, WIN, HINT, PK>(a, cur, nxt, t, it, owner, cstart, list, clist, biglist,
                                                        sparse, s_changed, rdist64, rdist32, s_pow2, win, tile);
        } else {
            const int64_t li = it - hch;
            int j = 0;
            int64_t ibj = ib[0], cntj = cnt[0], seg0 = a.seg_begin[1];
#pragma unroll
            for (int q = 1; q < C::NLIGHT; ++q)
                if (li >= ib[q]) { j = q; ibj = ib[q]; cntj = cnt[q]; seg0 = a.seg_begin[q + 1]; }
            const int64_t pos0 = seg0 + ((li - ibj) << j);
            light_item<LOG2P, F32, WIDE, WIN, HINT, PK>(a, cur, nxt, t, pos0, seg0 + cntj, C::LOGSMAX - j, list,
                                                        clist, biglist, sparse, s_changed, rdist64, rdist32,
                                                        s_pow2, prefetch && !WIDE, win, tile);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && s_changed[0]) atomicAdd(&a.ctr->n_changed, s_changed[0]);
    if (WIDE && threadIdx.x == 0 && s_changed[1]) atomicOr(&a.ctr->run_mask, s_changed[1]);
}

// The pushed-union tail kernel's body: the per-node tail over the nodes
// marked in a pushed frontier iteration.
template <int LOG2P, bool F32, bool WIDE>
__device__ __forceinline__ void tail_body(const StepArgs &a) {
    using C = Cfg<LOG2P>;
    const Counters *ctr = a.ctr;
    if (ctr->mode != 1 || !a.push_union) return;
    const int t = ctr->t;
    int64_t total = 0;
#pragma unroll
    for (int s = 0; s < kSegs; ++s) total += (int64_t)ctr->fill[s];
    __shared__ unsigned long long s_changed[2];
    __shared__ unsigned long long s_pow2[64];
    const double rdist64 = 1.0 / (double)(t + 1);
    const float rdist32 = 1.0f / (float)(t + 1);
    if (threadIdx.x < 2) s_changed[threadIdx.x] = 0;
    if (threadIdx.x < 64) {
        const int M = threadIdx.x, sh = 64 - (WIDE ? a.gb : a.b);
        s_pow2[M] = (M == 0 || M > sh) ? 0ULL : 1ULL << (sh - M);
    }
    __syncthreads();
    constexpr int NPW = 32 / C::L;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t base = gw * NPW; base < total; base += nw * NPW)
        union_tail_item<LOG2P, F32, WIDE>(a, t, base, s_changed, rdist64, rdist32, s_pow2);
    __syncthreads();
    if (threadIdx.x == 0 && s_changed[0]) atomicAdd(&a.ctr->n_changed, s_changed[0]);
    if (WIDE && threadIdx.x == 0 && s_changed[1]) atomicOr(&a.ctr->run_mask, s_changed[1]);
}

__device__ __forceinline__ void reset_counters(Counters *c) {
    c->n_changed = 0; c->list_len = 0; c->push_arcs = 0; c->n_big = 0; c->arcs = 0;
    for (int s = 0; s < kSegs; ++s) c->fill[s] = 0;
    c->prev_changed = 0; c->prev_list_len = 0; c->prev_push_arcs = 0; c->prev_big = 0;
    c->mode = 0; c->t = 0; c->steps_done = 0; c->converged = 0; c->err = 0;
    c->nsum = 0.0; c->run_mask = 0;
}

struct PlanParams {
    int64_t count[kSegs];   // dense: segment sizes
    int64_t chunk;
    int32_t nlight;
    int32_t dense;
};

// Work plan of one graph, by one whole block.  Items: first the chunks of
// heavy nodes (chunk starts by a block scan, then the chunk -> node map),
// then each light class packs 2^j nodes per warp item.
__device__ __forceinline__ void plan_block(const StepArgs &a, const PlanParams &pp, Plan *plan,
                                           int32_t *owner, int64_t *cstart) {
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

// Changed-list compaction of the 256 nodes from `base`, by one block of 256
// threads: one global atomic per block; the list order does not matter.
__device__ __forceinline__ void compact_tile(const StepArgs &a, int t, int64_t base) {
    int32_t *clist = a.clist[t & 1];
    int32_t *biglist = a.biglist[t & 1];
    __shared__ unsigned wcnt[8], wbig[8];
    __shared__ unsigned long long sbase, bbase, spush;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
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

// The same compaction over the 2048 nodes from `base` (base a multiple of
// 8), eight consecutive nodes per thread: one 8-byte load of their flags,
// one block scan of the packed counts (changed nodes in the low half, nodes
// with many predecessors in the high half) and one global atomic per list
// per tile.  Called by one block of 256 threads.
__device__ __forceinline__ void compact_tile_wide(const StepArgs &a, int t, int64_t base) {
    int32_t *clist = a.clist[t & 1];
    int32_t *biglist = a.biglist[t & 1];
    __shared__ unsigned long long sbase, bbase;
    const int lane = threadIdx.x & 31;
    const int64_t v0 = base + 8 * (int64_t)threadIdx.x;
    uint32_t flags = 0;   // bit i: node v0 + i changed
    if (v0 + 8 <= a.n) {
        const uint2 x = *reinterpret_cast<const uint2 *>(a.changed + v0);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            flags |= (((x.x >> (8 * i)) & 0xffu) ? 1u : 0u) << i;
            flags |= (((x.y >> (8 * i)) & 0xffu) ? 1u : 0u) << (4 + i);
        }
    } else {
        for (int i = 0; i < 8; ++i)
            if (v0 + i < a.n && a.changed[v0 + i]) flags |= 1u << i;
    }
    uint32_t bigs = 0;
    unsigned long long ps = 0;
    if (flags && a.has_reverse) {
        int64_t r = a.roff[v0 + __ffs(flags) - 1];
        for (int i = __ffs(flags) - 1; i < 8; ++i) {
            const int64_t r1 = (v0 + i < a.n) ? a.roff[v0 + i + 1] : r;
            if ((flags >> i) & 1u) {
                const int64_t rd = r1 - r;
                ps += (unsigned long long)rd;
                if (rd > kBigRdeg) bigs |= 1u << i;
            }
            r = r1;
        }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) ps += __shfl_xor_sync(FULL, ps, o);
    if (lane == 0 && ps) atomicAdd(&a.ctr->push_arcs, ps);
    int64_t excl;
    const int64_t packed = (int64_t)__popc(flags) + ((int64_t)__popc(bigs) << 32);
    const int64_t tot = block_excl_scan(packed, excl);
    if (threadIdx.x == 0) {
        const unsigned long long nc = (unsigned long long)(tot & 0xffffffffLL);
        const unsigned long long nb = (unsigned long long)(tot >> 32);
        sbase = nc ? atomicAdd(&a.ctr->list_len, nc) : 0;
        bbase = nb ? atomicAdd(&a.ctr->n_big, nb) : 0;
    }
    __syncthreads();
    unsigned long long cpos = sbase + (unsigned long long)(excl & 0xffffffffLL);
    unsigned long long bpos = bbase + (unsigned long long)(excl >> 32);
    for (int i = 0; i < 8; ++i) {
        if ((flags >> i) & 1u) clist[cpos++] = (int32_t)(v0 + i);
        if ((bigs >> i) & 1u) biglist[bpos++] = (int32_t)(v0 + i);
    }
    __syncthreads();
}

}  // namespace dev
}  // namespace hb

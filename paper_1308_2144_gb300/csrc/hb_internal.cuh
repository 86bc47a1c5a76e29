// hb_internal.cuh -- types and device helpers shared by the library's
// translation units.  Nothing here is part of the public C ABI.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace hb {

constexpr int kWarp = 32;
constexpr int kMaxLog2m = 12;
constexpr int kMinLog2m = 4;
constexpr int kSegs = 7;          // segment 0: heavy nodes; 1..6: light classes
constexpr int kArcsPerSlot = 16;  // default class sizing: about this many arcs per lane slot
constexpr int kStepThreads = 256;
constexpr int kBigRdeg = 1024;    // changed nodes with more predecessors are pushed grid-wide
// Bits of Counters::err, the device-side error word the host reads after
// every iteration (and turns into HB_ERR_STATE).
constexpr unsigned long long kErrCasBound = 2;  // the pushed union's CAS loop hit its bound
constexpr unsigned long long kErrTarget = 4;    // debug builds: an arc target outside [0, n)

// Per-p layout of a counter across the lanes of a warp.  A counter of P
// bytes is CH 16-byte chunks; L lanes ("chunk lanes") hold one arc's
// counter, CPL chunks each.  A team of T = L * S lanes works on one node,
// its S slots taking every S-th arc.
template <int LOG2P>
struct Cfg {
    static constexpr int P = 1 << LOG2P;
    static constexpr int CH = P / 16;
    static constexpr int LOGL = (LOG2P - 4) < 5 ? (LOG2P - 4) : 5;
    static constexpr int L = 1 << LOGL;
    static constexpr int CPL = CH / L;
    static constexpr int LOGSMAX = 5 - LOGL;      // a full warp has 2^LOGSMAX slots
    static constexpr int SMAX = 1 << LOGSMAX;
    static constexpr int NLIGHT = LOGSMAX + 1;    // light classes, slots SMAX, SMAX/2, ..., 1
    static constexpr int64_t CHUNK = 64 * SMAX;   // arcs per heavy-node chunk
    static constexpr int64_t HEAVY = 2 * CHUNK;   // degree above which a node is split
};

// Host-side copy of the same numbers for a runtime log2m.
struct Layout {
    int log2m, P, logL, L, logSmax, nlight, aps;
    int64_t chunk, heavy;
    // degree bounds of segment s: nodes with lo[s] <= deg <= hi[s]
    int64_t lo[kSegs], hi[kSegs];
};

// aps (arcs per slot, a power of two from 1 to 128) sizes the light degree
// classes: a node of degree d gets the smallest team whose slots each take
// at most aps arcs.  The autotuner picks it per graph.
inline Layout make_layout(int log2m, int aps = kArcsPerSlot) {
    Layout y{};
    y.log2m = log2m;
    y.aps = aps;
    y.P = 1 << log2m;
    y.logL = (log2m - 4) < 5 ? (log2m - 4) : 5;
    y.L = 1 << y.logL;
    y.logSmax = 5 - y.logL;
    y.nlight = y.logSmax + 1;
    y.chunk = 64LL << y.logSmax;
    y.heavy = 2 * y.chunk;
    y.lo[0] = y.heavy + 1;
    y.hi[0] = INT64_MAX;
    for (int j = 0; j < y.nlight; ++j) {
        int64_t s = 1LL << (y.logSmax - j);
        y.hi[j + 1] = (j == 0) ? y.heavy : aps * s;
        y.lo[j + 1] = (j == y.nlight - 1) ? 1 : aps * s / 2 + 1;
    }
    for (int s = y.nlight + 1; s < kSegs; ++s) { y.lo[s] = 1; y.hi[s] = 0; }
    return y;
}

// Work plan of one step: which nodes are recomputed and how they map onto
// warp items.  Segment s occupies list positions [seg_begin[s], seg_begin[s]
// + count[s]).  Items [0, heavy_chunks) are chunks of segment-0 nodes; then
// come the light segments, item_begin[j] .. item_begin[j+1]-1 for light
// class j (segment j+1).
struct Plan {
    int64_t count[kSegs];
    int64_t heavy_chunks;
    int64_t item_begin[kSegs];
    int64_t items;
    int64_t nodes;
    int64_t arcs;
};

// Device counters of the running step.  "cur" fields are produced by the
// step being executed, "prev" fields are those of the step before.
struct Counters {
    unsigned long long n_changed;      // nodes whose counter changed
    unsigned long long list_len;       // length of the changed list (built when a frontier is kept)
    unsigned long long push_arcs;      // sum of predecessor counts of changed nodes
    unsigned long long n_big;          // changed nodes with > kBigRdeg predecessors
    unsigned long long fill[kSegs];    // sparse list fill per segment
    unsigned long long arcs;           // arcs scanned by the sparse list
    unsigned long long prev_changed;
    unsigned long long prev_list_len;
    unsigned long long prev_push_arcs;
    unsigned long long prev_big;
    int32_t mode;                      // 0 = dense (all nodes), 1 = sparse (frontier list)
    int32_t t;                         // loop index of the step being run
    int32_t steps_done;                // iterations completed
    int32_t converged;
    unsigned long long err;            // nonzero: a device-side check failed
    double nsum;                       // sum of the nodes' cached estimates (neighbourhood function)
    unsigned long long run_mask;       // rows of several runs: bit r set if run r changed
};

// Everything the step kernels read, passed by value.  Buffers that
// alternate between iterations come in pairs indexed by the parity of the
// loop index t, which the kernels read from the device counters, so the
// same launch sequence serves every iteration (and can be captured once
// into a CUDA graph).
struct StepArgs {
    const int64_t *off;
    const int32_t *tgt;
    const int64_t *roff;          // reverse CSR offsets (may be null)
    const int32_t *rtgt;
    uint8_t *regs[2];             // counters: iteration t reads regs[t&1], writes regs[(t+1)&1]
    double *sumd;
    double *harm;
    double *disc;                 // Sec. 7 discounted accumulator (null: no discount)
    const double *ftab;           // discount table: f(d) = ftab[d-1] for d <= flen, else 0
    void *ecache;                 // double[n] (FP64 form) or float[n] (FP32 form)
    uint8_t *changed;             // 1 if the node changed in the last iteration
    uint32_t *mustbits;           // frontier bitmap of the running iteration
    int32_t *clist[2];            // changed nodes, appended by iteration t into clist[t&1]
    int32_t *biglist[2];          // changed nodes with many predecessors, same pairing
    const int32_t *dense_list;    // node of each dense position (null: position = node)
    int32_t *slist;               // sparse list, laid out by segment
    const Plan *plan_dense;
    Plan *plan_sparse;
    const int32_t *owner_dense;   // heavy chunk -> heavy index
    const int64_t *cstart_dense;  // heavy index -> first chunk
    int32_t *owner_sparse;
    int64_t *cstart_sparse;
    uint8_t *partial;             // per heavy chunk partial counter
    uint32_t *arrive;             // per heavy index arrival count
    Counters *ctr;
    const double *lc64;           // p ln(p/V), V = 0..p
    const float *lc32;
    double c64;                   // alpha_p p^2 2^(64-b)
    float c32;                    // the same as float
    unsigned long long thr_x;     // small-range switch in fixed point
    int64_t n;
    int64_t n_pos;                // nodes of nonzero degree
    int64_t m;
    int64_t seg_begin[kSegs];
    int64_t seg_lo[kSegs];
    int64_t seg_hi[kSegs];
    int32_t b;
    int32_t frontier;             // HB_FRONTIER_* policy
    int32_t has_reverse;          // roff/rtgt present
    int32_t aps;                  // class sizing (arcs per slot) of the layout
    int32_t push_union;           // frontier iterations push changed counters along reverse arcs
    int32_t flen;                 // entries of ftab
    int32_t gb;                   // log2 of one run's registers (= b unless rows hold several runs)
    int32_t lruns;                // log2 of the runs sharing each row (0: one run per row)
    const uint64_t *run_seeds;    // hash seed of each run of a row
    double sparse_frac;           // AUTO: push when the last push arcs <= sparse_frac * m
    uint32_t hot;                 // > 0: counters [0, hot) (the most gathered ones after the
                                  // degree relabelling) get the treatment two_pass selects
    int32_t pass;                 // which launch of the two-phase gather this is (1 or 2)
    int32_t two_pass;             // with hot > 0: 1 = the two-phase gather, 0 = one pass
                                  // reading counters [0, hot) with the normal L2 priority and
                                  // the others with evict-first
    uint32_t hint;                // set by the launcher of the one-pass gather: hot
    int32_t packed;               // counters packed six bits per register (rows of 3p/4 bytes)
    const int32_t *hcnt;          // two-phase gather: every node's targets below hot come
                                  // first, hcnt[v] of them (null: each arc tested in both passes)
};

// ------------------------------------------------------------ helpers --

// Blocks for a grid-stride loop over `work` items: enough to cover it, at
// most 32 resident blocks' worth per SM of the 152.
inline int grid_for(int64_t work, int threads) {
    int64_t g = (work + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > 152 * 32) g = 152 * 32;
    return (int)g;
}

// Byte-wise maximum of two words whose bytes are all below 128.  Register
// values never exceed 64 - b <= 60, so in t = a + 0x80808080 - b every byte
// is a_i + 128 - b_i, in [1, 255] (no carry crosses a byte), and its bit 7
// is set exactly when a_i >= b_i; prmt in sign-replicate mode (selector
// nibbles 8..B) spreads that bit over the byte, giving the select mask.
__device__ __forceinline__ uint32_t bmax4(uint32_t a, uint32_t b) {
    const uint32_t t = a + 0x80808080u - b;
    uint32_t m;
    asm("prmt.b32 %0, %1, 0, 0xBA98;" : "=r"(m) : "r"(t));
    return (a & m) | (b & ~m);
}

// *addr = bmax4(*addr, v) atomically.  Every byte of *addr only grows, so
// each failed compare-and-swap means another thread raised a byte: the
// loop ends after at most 4 x 64 retries; the bound below only guards
// against a broken invariant (it sets err and gives up).
__device__ __forceinline__ void atomic_bmax4(uint32_t *addr, uint32_t v, unsigned long long *err) {
    uint32_t old = __ldcg(addr);
    uint32_t nv = bmax4(old, v);
    for (int guard = 0; nv != old; ++guard) {
        const uint32_t seen = atomicCAS(addr, old, nv);
        if (seen == old) return;
        old = seen;
        nv = bmax4(old, v);
        if (guard == 1024) {
            atomicOr(err, kErrCasBound);
            return;
        }
    }
}

__device__ __forceinline__ uint4 vmax16(uint4 a, uint4 b) {
    return make_uint4(bmax4(a.x, b.x), bmax4(a.y, b.y), bmax4(a.z, b.z), bmax4(a.w, b.w));
}

__device__ __forceinline__ bool ne16(uint4 a, uint4 b) {
    return ((a.x ^ b.x) | (a.y ^ b.y) | (a.z ^ b.z) | (a.w ^ b.w)) != 0u;
}

__device__ __forceinline__ uint4 shfl_xor16(uint4 a, int o) {
    a.x = __shfl_xor_sync(0xffffffffu, a.x, o);
    a.y = __shfl_xor_sync(0xffffffffu, a.y, o);
    a.z = __shfl_xor_sync(0xffffffffu, a.z, o);
    a.w = __shfl_xor_sync(0xffffffffu, a.w, o);
    return a;
}

// Counter loads: the read buffer does not change during a step.
__device__ __forceinline__ uint4 ld_counter(const uint8_t *p) {
    return __ldg(reinterpret_cast<const uint4 *>(p));
}

// Packed registers (Sec. 4.1 register width): six bits per register, a
// chunk of 16 registers in 12 bytes (three words, 96 bits, register j at
// bits 6j .. 6j+5, least significant first), so a counter of p registers
// takes 3p/4 bytes.  Every register value (<= 64 - b <= 60) fits.  In
// registers a chunk is unpacked to the usual 16 bytes, one per register.
__device__ __forceinline__ uint32_t spread24(uint32_t x) {   // 4 fields of 6 bits -> 4 bytes
    return (x & 0x3Fu) | ((x << 2) & 0x3F00u) | ((x << 4) & 0x3F0000u) | ((x << 6) & 0x3F000000u);
}
__device__ __forceinline__ uint32_t gather24(uint32_t y) {   // 4 bytes (each < 64) -> 24 bits
    return (y & 0x3Fu) | ((y >> 2) & 0xFC0u) | ((y >> 4) & 0x3F000u) | ((y >> 6) & 0xFC0000u);
}
__device__ __forceinline__ uint4 unpack_chunk(uint32_t w0, uint32_t w1, uint32_t w2) {
    return make_uint4(spread24(w0 & 0xFFFFFFu), spread24(__funnelshift_r(w0, w1, 24) & 0xFFFFFFu),
                      spread24(__funnelshift_r(w1, w2, 16) & 0xFFFFFFu), spread24(w2 >> 8));
}
__device__ __forceinline__ void pack_chunk(uint4 c, uint32_t &w0, uint32_t &w1, uint32_t &w2) {
    const uint32_t x0 = gather24(c.x), x1 = gather24(c.y), x2 = gather24(c.z), x3 = gather24(c.w);
    w0 = x0 | (x1 << 24);
    w1 = (x1 >> 8) | (x2 << 16);
    w2 = (x2 >> 16) | (x3 << 8);
}
// Chunk k of the packed counter at row: 12 bytes from row + 12 k.
__device__ __forceinline__ uint4 ld_packed(const uint8_t *row, int k) {
    const uint32_t *q = reinterpret_cast<const uint32_t *>(row + 12 * k);
    return unpack_chunk(__ldg(q), __ldg(q + 1), __ldg(q + 2));
}
// Chunk g of a packed buffer (the buffer 8-byte aligned) with one 8-byte
// and one 4-byte load instead of three 4-byte ones: 12 g is a multiple of 8
// for even g, so there the first two words form an aligned 8-byte word, and
// for odd g the last two do.  The words are selected, not branched on, so
// lanes of either parity run the same instructions.  The gather uses it
// where a counter is a single chunk (p = 16); for wider counters the
// selects cost more than the load they save.
__device__ __forceinline__ uint4 ld_packed_pair(const uint8_t *base, int64_t g) {
    const uint32_t *q = reinterpret_cast<const uint32_t *>(base + 12 * g);
    const bool odd = (g & 1) != 0;
    const uint2 d = __ldg(reinterpret_cast<const uint2 *>(q + (odd ? 1 : 0)));
    const uint32_t x = __ldg(q + (odd ? 0 : 2));
    return unpack_chunk(odd ? x : d.x, odd ? d.x : d.y, odd ? d.y : x);
}
__device__ __forceinline__ void st_packed(uint8_t *row, int k, uint4 c) {
    uint32_t w0, w1, w2;
    pack_chunk(c, w0, w1, w2);
    uint32_t *q = reinterpret_cast<uint32_t *>(row + 12 * k);
    __stcs(q, w0);
    __stcs(q + 1, w1);
    __stcs(q + 2, w2);
}

// Targets are streamed once per step.
__device__ __forceinline__ int32_t ld_stream(const int32_t *p) { return __ldcs(p); }

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// SplitMix64 output number v+1 of a generator seeded with `seed`
// (Steele, Lea & Flood 2014): the node hash h of Sec. 4.1.
__host__ __device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t v) {
    uint64_t z = seed + (v + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

// Register index = top b bits; rho+ = leading zeros of the other 64-b bits
// plus one, capped at 64-b (Sec. 4.1, Algorithm 1).
__device__ __forceinline__ void hash_to_register(uint64_t x, int b, uint32_t &idx, uint32_t &rho) {
    idx = (uint32_t)(x >> (64 - b));
    uint64_t rest = x << b;
    uint32_t lz = rest == 0 ? 64u : (uint32_t)__clzll((long long)rest);
    uint32_t r = lz + 1;
    uint32_t cap = (uint32_t)(64 - b);
    rho = r < cap ? r : cap;
}

// Zero-register count and fixed-point sum of 2^(64-b-M) over the 16 bytes
// of one chunk.
__device__ __forceinline__ void chunk_sums(uint4 c, int b, uint32_t &V, unsigned long long &S) {
    const uint32_t w[4] = {c.x, c.y, c.z, c.w};
    const int sh = 64 - b;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            uint32_t M = (w[k] >> (8 * j)) & 0xffu;
            if (M == 0) V += 1;
            else S += 1ULL << (sh - (int)M);
        }
    }
}

// The same with the powers looked up in a 64-entry table (pow2[M] =
// 2^(64-b-M), pow2[0] = 0) and the zero bytes counted four at a time:
// byte + 0x7F has bit 7 set exactly when the byte is nonzero (bytes < 128).
__device__ __forceinline__ void chunk_sums_tab(uint4 c, const unsigned long long *pow2, uint32_t &V,
                                               unsigned long long &S) {
    const uint32_t w[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const uint32_t x = w[k];
        V += 4u - __popc((x + 0x7F7F7F7Fu) & 0x80808080u);
        S += pow2[x & 0xffu] + pow2[(x >> 8) & 0xffu] + pow2[(x >> 16) & 0xffu] + pow2[x >> 24];
    }
}

// Sec. 4.1 estimate from the zero-register count V and the fixed-point
// sum S = sum over nonzero registers of 2^(64-b-M).  X = V 2^(64-b) + S is
// the exact register sum scaled by 2^(64-b) (it fits in 64 bits unless the
// counter is empty, V = p, whose estimate is 0).  Small-range switch
// (linear counting p ln(p/V) when the raw estimate alpha_p p^2 / sum is
// <= 5p/2 and V > 0) is taken exactly on X: X >= thr_x.  The raw estimate
// is c64 / X with c64 = alpha_p p^2 2^(64-b), X converted once to double;
// the reciprocal comes from an FP32 seed refined by two Newton steps in
// FP64 (GB300 runs FP64 at a small fraction of its FP32 rate, so the
// correctly rounded division is avoided; the result is within 2 ulp).
__device__ __forceinline__ double estimate64(uint32_t V, unsigned long long S, int P, int b,
                                             double c64, unsigned long long thr_x,
                                             const double *lc64) {
    if (V == (uint32_t)P) return 0.0;
    const unsigned long long X = ((unsigned long long)V << (64 - b)) + S;
    if (V > 0 && X >= thr_x) return lc64[V];
    const double xd = __ull2double_rn(X);
    double r = (double)__frcp_rn(__ull2float_rn(X));
    double e = __fma_rn(-xd, r, 1.0);
    r = __fma_rn(r, e, r);
    e = __fma_rn(-xd, r, 1.0);
    r = __fma_rn(r, e, r);
    return __dmul_rn(c64, r);
}

// Precision form: the same switch on X, the estimate in FP32.
__device__ __forceinline__ float estimate32(uint32_t V, unsigned long long S, int P, int b,
                                            float c32, unsigned long long thr_x, const float *lc32) {
    if (V == (uint32_t)P) return 0.0f;
    const unsigned long long X = ((unsigned long long)V << (64 - b)) + S;
    if (V > 0 && X >= thr_x) return lc32[V];
    return __fmul_rn(c32, __frcp_rn(__ull2float_rn(X)));
}

// Sec. 3 centralities of node v (internal index) from its counter row in
// `regs` and its Sec. 5 accumulators, in the order closeness, harmonic,
// Lin, reachable:
//     reachable = size(c[v]); closeness = 1/sumd (0 if sumd = 0);
//     lin = reachable^2/sumd (1 if sumd = 0); harmonic = harm.
template <bool F32>
__device__ __forceinline__ void node_centralities(const StepArgs &a, const uint8_t *regs, int64_t v,
                                                  double out[4]) {
    const int P = 1 << a.b;
    const int CH = P >> 4;
    uint32_t V = 0;
    unsigned long long S = 0;
    if (a.packed) {
        const uint8_t *prow = regs + v * (3 * P / 4);
        for (int c = 0; c < CH; ++c) chunk_sums(ld_packed(prow, c), a.b, V, S);
    } else {
        const uint4 *row = reinterpret_cast<const uint4 *>(regs + v * P);
        for (int c = 0; c < CH; ++c) chunk_sums(row[c], a.b, V, S);
    }
    double r;
    if (F32) r = (double)estimate32(V, S, P, a.b, a.c32, a.thr_x, a.lc32);
    else r = estimate64(V, S, P, a.b, a.c64, a.thr_x, a.lc64);
    const double s = a.sumd[v];
    out[0] = s > 0.0 ? __ddiv_rn(1.0, s) : 0.0;
    out[1] = a.harm[v];
    out[2] = s > 0.0 ? __ddiv_rn(__dmul_rn(r, r), s) : 1.0;
    out[3] = r;
}

// Inclusive warp scan and exclusive block scan (one value per thread,
// blockDim a multiple of 32 up to 1024); the block scan returns the total.
__device__ __forceinline__ int64_t warp_incl_scan(int64_t x) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

__device__ __forceinline__ int64_t block_excl_scan(int64_t x, int64_t &excl) {
    __shared__ int64_t wsum[32];
    __shared__ int64_t wtotal;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    int64_t inc = warp_incl_scan(x);
    if (lane == 31) wsum[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        int64_t w = lane < nw ? wsum[lane] : 0;
        int64_t wi = warp_incl_scan(w);
        if (lane < nw) wsum[lane] = wi - w;
        if (lane == 31) wtotal = wi;
    }
    __syncthreads();
    excl = inc - x + wsum[wid];
    int64_t total = wtotal;
    __syncthreads();
    return total;
}

// ----------------------------------------------------------- launchers --
// (defined in hb_build.cu / hb_step.cu; all take the stream last)

cudaError_t scan_exclusive_i64(const int64_t *in, int64_t *out, int64_t N, cudaStream_t s);
// CSR checks (error bits 1 offsets[0] != 0, 2 offsets[n] != m, 4 offsets
// decrease, 8 a target outside [0, n)) in two parts, so that the target
// checks can follow an upload chunk by chunk: the offsets, and targets
// [0, len), which with indeg not null also add each target's in-arc there.
cudaError_t validate_offsets(const int64_t *off, int64_t n, int64_t m, unsigned long long *err_dev,
                             cudaStream_t s);
cudaError_t check_targets(const int32_t *tgt, int64_t len, int64_t n, unsigned long long *err_dev,
                          unsigned long long *indeg, cudaStream_t s);
cudaError_t widen_offsets(const int32_t *in, int64_t *out, int64_t count, cudaStream_t s);
// With scatter_s, the offsets are computed on s and the targets scattered
// on scatter_s after them; scatter_done is then recorded on scatter_s when
// the targets are in place.
cudaError_t transpose_csr(const int64_t *off, const int32_t *tgt, int64_t n, int64_t m,
                          int64_t *toff, int32_t *ttgt, cudaStream_t s, cudaStream_t scatter_s = nullptr,
                          cudaEvent_t scatter_done = nullptr);
// transpose_csr of a relabelled graph whose node v is the caller's perm[v]
// (perm null: the identity) and has in-degree indeg[perm[v]]; indeg null
// counts the in-arcs instead.
cudaError_t transpose_csr_counted(const int64_t *off, const int32_t *tgt, int64_t n, int64_t m,
                                  const unsigned long long *indeg, const int32_t *perm, int64_t *toff,
                                  int32_t *ttgt, cudaStream_t s, cudaStream_t scatter_s = nullptr,
                                  cudaEvent_t scatter_done = nullptr);
// Node order for the step kernel (perm: new -> caller's id, inv: its
// inverse).  indeg (n entries) holds the in-degree of each of the caller's
// nodes when counted is true, and receives it otherwise.
cudaError_t degree_sort_counted(const int64_t *off, const int32_t *tgt, int64_t n, int64_t m, int32_t *perm,
                                int32_t *inv, unsigned long long *indeg, bool counted, cudaStream_t s);
cudaError_t relabel_csr(const int64_t *off, const int32_t *tgt, int64_t n, int64_t m,
                        const int32_t *perm, const int32_t *inv, int64_t *noff, int32_t *ntgt,
                        cudaStream_t s);
cudaError_t count_degree_segments(const int64_t *off, int64_t n, const Layout &y,
                                  int64_t *seg_count_host, cudaStream_t s);
cudaError_t build_dense_list(const int64_t *off, int64_t n, const Layout &y,
                             const int64_t *seg_begin, int32_t *list, unsigned long long *fill,
                             cudaStream_t s);

// Two-phase gather: reorder every node's targets so that those below `hot`
// come first (within the node's own range), and hcnt[v] = their number.
cudaError_t partition_hot(const int64_t *off, int32_t *tgt, int64_t n, int64_t m, uint32_t hot, int32_t *hcnt,
                          cudaStream_t s);

cudaError_t heavy_chunk_total(const int64_t *off, int64_t n, const Layout &y, int64_t *total_host,
                              cudaStream_t s);
// Algorithm 2's first loop; with wfirst (Sec. 6), the counters of weighted
// nodes, whose replicas are the items wfirst[u] .. wfirst[u+1]-1.
cudaError_t launch_init(const StepArgs &a, const int32_t *perm, uint64_t seed, bool fp32,
                        cudaStream_t s, const int64_t *wfirst = nullptr);
// Rows of several runs (hb_create_runs): the gather with the per-run tail,
// the pushed-union tail, initial counters, and per-run readouts.  log2row
// is the row's log2 byte count (a.b); a.gb and a.lruns give the runs.
cudaError_t launch_runs_step(const StepArgs &a, int log2row, bool fp32, int grid, cudaStream_t s);
cudaError_t launch_runs_tail(const StepArgs &a, int log2row, bool fp32, int grid, cudaStream_t s);
cudaError_t launch_runs_init(const StepArgs &a, const int32_t *perm, bool fp32, cudaStream_t s,
                             const int64_t *wfirst = nullptr);
cudaError_t launch_runs_centralities(const StepArgs &a, const uint8_t *regs, const int32_t *perm, bool fp32,
                                     int run, double *closeness, double *harmonic, double *lin,
                                     double *reachable, cudaStream_t s);
cudaError_t launch_runs_stats(const StepArgs &a, const uint8_t *regs, const int32_t *perm, bool fp32,
                              int which, double *mean, double *sd, cudaStream_t s);
// out[u] = src[(inv[u] << lstride) + off] (inv may be null: identity).
cudaError_t launch_gather_strided(const double *src, const int32_t *inv, int64_t n, int lstride, int off,
                                  double *out, cudaStream_t s);
int runs_step_blocks_per_sm(int log2row, bool fp32);
// Neighbourhood function: the sum of the n cached estimates (float or
// double) into ctr->nsum, in a fixed order (grid kNfBlocks, partials in
// part[kNfBlocks]) so that the result does not vary between runs.
constexpr int kNfBlocks = 608;
cudaError_t launch_estimate_sum(const void *ecache, bool fp32, int64_t n, double *part, Counters *ctr,
                                cudaStream_t s);
// First replica item of every node: wfirst = exclusive prefix sums of the
// n weights w (device), n+1 entries; sets bit 1 of *err if a weight lies
// outside [0, 2^31).
cudaError_t replica_starts(const int64_t *w, int64_t n, int64_t *wfirst, unsigned long long *err,
                           cudaStream_t s);
cudaError_t launch_dense_plan(const StepArgs &a, const Layout &y, const int64_t *seg_count,
                              Plan *plan, int32_t *owner, int64_t *cstart, cudaStream_t s);
// One iteration: the whole launch sequence, sizes read on the device.
// With ev (four events): ev[0], ev[1] around the gather kernel, ev[2],
// ev[3] around the pushed union (when a.push_union).
cudaError_t launch_iteration(const StepArgs &a, const Layout &y, bool fp32, int step_grid,
                             cudaStream_t s, const cudaEvent_t *ev = nullptr,
                             int *launches = nullptr);
int step_blocks_per_sm(int log2m, bool fp32);
// The gather kernel alone (mode and t already set in the counters).
cudaError_t launch_step_kernel(const StepArgs &a, int log2m, bool fp32, int grid, cudaStream_t s);
// alpha_p of the estimator and the thread-local message of hb_last_error().
double hll_alpha_of(int p);
void set_last_error(const char *msg);
// Centralities of the caller's nodes [u0, u0 + count) into out[k][0 ..
// count) (any output may be null); inv maps a caller's node to its internal
// index (null: the identity).
cudaError_t launch_finalize(const StepArgs &a, const uint8_t *regs, const int32_t *inv, bool fp32, int64_t u0,
                            int64_t count, double *closeness, double *harmonic, double *lin, double *reachable,
                            cudaStream_t s);
// Rows of p = P registers in the caller's order, one byte per register
// (packed: the rows are held six bits per register).
cudaError_t launch_gather_rows(const uint8_t *regs, const int32_t *inv, int64_t n, int P,
                               uint8_t *out, cudaStream_t s, bool packed = false);
cudaError_t launch_gather_f64(const double *src, const int32_t *inv, int64_t n, double *out,
                              cudaStream_t s);
cudaError_t launch_frontier_out(const StepArgs &a, const int32_t *inv, uint8_t *changed,
                                uint8_t *must, cudaStream_t s);
cudaError_t launch_lc_tables(double *lc64, float *lc32, int P, cudaStream_t s);

}  // namespace hb

// hb_build.cu -- create-time device work: CSR validation, offset widening,
// exclusive scans, transposition (Sec. 5: HyperBall runs on G^T for the
// in-centralities), and the degree-sorted relabelling that lays nodes out
// for the step kernel (heavy nodes first, then light degree classes).
#include <cstdio>

#include "hb_handle.h"

namespace hb {

namespace {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

__global__ void scan_tile_sums(const int64_t *in, int64_t N, int64_t *sums) {
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    int64_t s = 0;
    for (int i = 0; i < kScanItems; ++i) {
        int64_t k = base + (int64_t)threadIdx.x * kScanItems + i;
        if (k < N) s += in[k];
    }
    int64_t ex;
    int64_t tot = block_excl_scan(s, ex);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void scan_tile_apply(const int64_t *in, int64_t *out, int64_t N, const int64_t *offs) {
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    int64_t v[kScanItems];
    int64_t s = 0;
    for (int i = 0; i < kScanItems; ++i) {
        int64_t k = base + (int64_t)threadIdx.x * kScanItems + i;
        v[i] = k < N ? in[k] : 0;
        s += v[i];
    }
    int64_t ex;
    block_excl_scan(s, ex);
    int64_t run = ex + (offs ? offs[blockIdx.x] : 0);
    for (int i = 0; i < kScanItems; ++i) {
        int64_t k = base + (int64_t)threadIdx.x * kScanItems + i;
        if (k < N) out[k] = run;
        run += v[i];
    }
}

// ------------------------------------------------------------ validate --

// Error bits: 1 offsets[0] != 0, 2 offsets[n] != m, 4 offsets decrease,
// 8 a target outside [0, n).
__global__ void validate_offsets_kernel(const int64_t *off, int64_t n, int64_t m, unsigned long long *err) {
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid == 0) {
        if (off[0] != 0) atomicOr(err, 1ULL);
        if (off[n] != m) atomicOr(err, 2ULL);
    }
    for (int64_t v = tid; v < n; v += (int64_t)gridDim.x * blockDim.x)
        if (off[v + 1] < off[v]) { atomicOr(err, 4ULL); break; }
}

// Targets tgt[0 .. len) against [0, n); with indeg, every target in range
// also adds one to its node's in-degree.
__global__ void check_targets_kernel(const int32_t *tgt, int64_t len, int64_t n, unsigned long long *err,
                                     unsigned long long *indeg) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < len;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t w = tgt[e];
        if (w < 0 || (int64_t)w >= n) { atomicOr(err, 8ULL); break; }
        if (indeg) atomicAdd(&indeg[w], 1ULL);
    }
}

__global__ void widen_kernel(const int32_t *in, int64_t *out, int64_t count) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (int64_t)in[i];
}

// ----------------------------------------------------------- transpose --

// Node u with off[u] <= e < off[u+1] (the last such u when degrees are 0).
__device__ __forceinline__ int64_t arc_source(const int64_t *off, int64_t n, int64_t e) {
    int64_t lo = 0, hi = n;   // off[lo] <= e < off[hi]
    while (hi - lo > 1) {
        int64_t mid = (lo + hi) >> 1;
        if (off[mid] <= e) lo = mid; else hi = mid;
    }
    return lo;
}

__global__ void count_targets(const int32_t *tgt, int64_t m, unsigned long long *cnt) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&cnt[tgt[e]], 1ULL);
}

// Arc passes that need each arc's source node work on tiles of kArcTile
// consecutive arcs.  tile_ends_kernel finds, for all tiles in parallel, the
// sources u0 of a tile's first arc and u1 of its last (a binary search over
// the offsets each); a block stages off[u0 .. u1] in shared memory, and
// every arc's source is then the last staged node whose offset is <= the
// arc (off[u1+1] lies beyond the tile).  A tile whose sources span more
// than kStageNodes nodes (runs of empty nodes) falls back to the search
// over all offsets.  Each thread takes kArcPer arcs of a tile and runs
// their dependent loads (and atomics) stage by stage, so that the loads of
// all its arcs are in flight together.
constexpr int kArcTile = 2048;
constexpr int kStageNodes = 2048;
constexpr int kArcThreads = 256;
constexpr int kArcPer = kArcTile / kArcThreads;

struct ArcTile {
    int64_t e0, e1, u0;
    int cnt;   // staged offsets (0: fall back)
};

__global__ void tile_ends_kernel(const int64_t *off, int64_t n, int64_t m, int64_t ntiles, int64_t *ends) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < ntiles;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e0 = t * kArcTile, e1 = e0 + kArcTile < m ? e0 + kArcTile : m;
        ends[2 * t] = arc_source(off, n, e0);
        ends[2 * t + 1] = arc_source(off, n, e1 - 1);
    }
}

__device__ __forceinline__ ArcTile stage_arc_tile(const int64_t *off, int64_t m, int64_t tile, const int64_t *ends,
                                                  int64_t *s_off) {
    const int64_t e0 = tile * kArcTile, e1 = e0 + kArcTile < m ? e0 + kArcTile : m;
    const int64_t u0 = ends[2 * tile], u1 = ends[2 * tile + 1];
    const int cnt = u1 - u0 + 1 <= kStageNodes ? (int)(u1 - u0 + 1) : 0;
    __syncthreads();   // the previous tile's readers are done with s_off
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) s_off[i] = off[u0 + i];
    __syncthreads();
    return ArcTile{e0, e1, u0, cnt};
}

// Source node of arc e of the tile, and its first arc off[u].
__device__ __forceinline__ int64_t tile_source(const ArcTile &t, const int64_t *s_off, const int64_t *off,
                                               int64_t n, int64_t e, int64_t &first) {
    if (t.cnt == 0) {
        const int64_t u = arc_source(off, n, e);
        first = off[u];
        return u;
    }
    int lo = 0, hi = t.cnt;   // s_off[lo] <= e < off[u0 + hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (s_off[mid] <= e) lo = mid; else hi = mid;
    }
    first = s_off[lo];
    return t.u0 + lo;
}

__global__ void __launch_bounds__(kArcThreads) scatter_transpose(const int64_t *off, const int32_t *tgt, int64_t n,
                                                                 int64_t m, const int64_t *ends,
                                                                 unsigned long long *cursor, int32_t *ttgt) {
    __shared__ int64_t s_off[kStageNodes];
    const int64_t ntiles = (m + kArcTile - 1) / kArcTile;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const ArcTile t = stage_arc_tile(off, m, tile, ends, s_off);
        int32_t w[kArcPer], u[kArcPer];
        unsigned long long pos[kArcPer];
#pragma unroll
        for (int q = 0; q < kArcPer; ++q) {
            const int64_t e = t.e0 + threadIdx.x + q * kArcThreads;
            if (e < t.e1) {
                int64_t first;
                w[q] = tgt[e];
                u[q] = (int32_t)tile_source(t, s_off, off, n, e, first);
            }
        }
#pragma unroll
        for (int q = 0; q < kArcPer; ++q)
            if (t.e0 + threadIdx.x + q * kArcThreads < t.e1) pos[q] = atomicAdd(&cursor[w[q]], 1ULL);
#pragma unroll
        for (int q = 0; q < kArcPer; ++q)
            if (t.e0 + threadIdx.x + q * kArcThreads < t.e1) ttgt[pos[q]] = u[q];
    }
}

// In-arc counts of the relabelled graph from the in-degrees of the
// caller's nodes: node v of the relabelled graph is the caller's perm[v].
__global__ void permuted_counts(const unsigned long long *indeg, const int32_t *perm, int64_t n,
                                unsigned long long *cnt) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x)
        cnt[v] = indeg[perm ? perm[v] : v];
    if (blockIdx.x == 0 && threadIdx.x == 0) cnt[n] = 0;
}

// -------------------------------------------------------- degree sort --
// Stable partition of nodes into descending degree buckets: quarter
// octaves of deg-1, so every power-of-two class bound is a bucket bound;
// degree-0 nodes last.

constexpr int kBuckets = 128;
constexpr int kPartThreads = 256;
constexpr int kPartRounds = 16;
constexpr int kPartTile = kPartThreads * kPartRounds;

__device__ __forceinline__ int degree_bucket(int64_t d) {
    if (d <= 0) return 120;
    uint64_t x = (uint64_t)(d - 1);
    int b;
    if (x < 8) b = (int)x;
    else {
        int k = 63 - __clzll((long long)x);
        int f = (int)((x >> (k - 2)) & 3);
        b = 8 + (k - 3) * 4 + f;
        if (b > 119) b = 119;
    }
    return 119 - b;   // larger degree, smaller key
}

__global__ void key_out_kernel(const int64_t *off, int64_t n, uint8_t *key) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x)
        key[v] = (uint8_t)degree_bucket(off[v + 1] - off[v]);
}

__global__ void key_in_kernel(const unsigned long long *indeg, int64_t n, uint8_t *key) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x)
        key[v] = (uint8_t)degree_bucket((int64_t)indeg[v]);
}

// Stable partition of the sequence src (identity if null) by key[node]:
// per-tile bucket counts, a scan, then an order-preserving scatter.
__global__ void part_count(const int32_t *src, const uint8_t *key, int64_t n, int64_t ntiles,
                           int64_t *counts) {
    __shared__ int hist[kBuckets];
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        for (int k = threadIdx.x; k < kBuckets; k += blockDim.x) hist[k] = 0;
        __syncthreads();
        for (int i = threadIdx.x; i < kPartTile; i += blockDim.x) {
            int64_t q = tile * kPartTile + i;
            if (q < n) atomicAdd(&hist[key[src ? src[q] : q]], 1);
        }
        __syncthreads();
        for (int k = threadIdx.x; k < kBuckets; k += blockDim.x) counts[(int64_t)k * ntiles + tile] = hist[k];
        __syncthreads();
    }
}

__global__ void part_scatter(const int32_t *src, const uint8_t *key, int64_t n, int64_t ntiles,
                             const int64_t *offs, int32_t *out, int32_t *inv) {
    __shared__ int64_t base[kBuckets];
    __shared__ int wcnt[kPartThreads / 32][kBuckets];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        for (int k = threadIdx.x; k < kBuckets; k += blockDim.x) base[k] = offs[(int64_t)k * ntiles + tile];
        __syncthreads();
        for (int r = 0; r < kPartRounds; ++r) {
            for (int k = threadIdx.x; k < (kPartThreads / 32) * kBuckets; k += blockDim.x)
                (&wcnt[0][0])[k] = 0;
            __syncthreads();
            const int64_t q = tile * kPartTile + (int64_t)r * kPartThreads + threadIdx.x;
            const bool valid = q < n;
            const int64_t v = valid ? (src ? (int64_t)src[q] : q) : 0;
            const int k = valid ? (int)key[v] : -1;
            const unsigned peers = __match_any_sync(0xffffffffu, k);
            const int rank = __popc(peers & lanemask_lt());
            if (valid && lane == __ffs(peers) - 1) wcnt[wid][k] = __popc(peers);
            __syncthreads();
            if (valid) {
                int64_t pos = base[k] + rank;
                for (int w = 0; w < wid; ++w) pos += wcnt[w][k];
                out[pos] = (int32_t)v;
                if (inv) inv[v] = (int32_t)pos;
            }
            __syncthreads();
            for (int kk = threadIdx.x; kk < kBuckets; kk += blockDim.x) {
                int sum = 0;
                for (int w = 0; w < kPartThreads / 32; ++w) sum += wcnt[w][kk];
                base[kk] += sum;
            }
            __syncthreads();
        }
    }
}

__global__ void permuted_degrees(const int64_t *off, const int32_t *perm, int64_t n, int64_t *deg) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        int64_t u = perm[v];
        deg[v] = off[u + 1] - off[u];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) deg[n] = 0;
}

// Arcs of the relabelled CSR in their own order: arc e of new node v (the
// caller's u = perm[v]) is u's arc e - noff[v], its target mapped by inv.
// The writes are sequential and each node's targets are read as one run.
__global__ void __launch_bounds__(kArcThreads) relabel_arcs(const int64_t *off, const int32_t *tgt, int64_t n,
                                                            int64_t m, const int32_t *perm, const int32_t *inv,
                                                            const int64_t *noff, const int64_t *ends, int32_t *ntgt) {
    __shared__ int64_t s_off[kStageNodes];
    const int64_t ntiles = (m + kArcTile - 1) / kArcTile;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const ArcTile t = stage_arc_tile(noff, m, tile, ends, s_off);
        int64_t v[kArcPer], at[kArcPer];
        int32_t x[kArcPer];
#pragma unroll
        for (int q = 0; q < kArcPer; ++q) {
            const int64_t e = t.e0 + threadIdx.x + q * kArcThreads;
            int64_t first = e;
            v[q] = e < t.e1 ? tile_source(t, s_off, noff, n, e, first) : 0;
            at[q] = e - first;   // the arc's rank in its node's list
        }
#pragma unroll
        for (int q = 0; q < kArcPer; ++q) v[q] = perm[v[q]];
#pragma unroll
        for (int q = 0; q < kArcPer; ++q)
            if (t.e0 + threadIdx.x + q * kArcThreads < t.e1) at[q] += off[v[q]];
#pragma unroll
        for (int q = 0; q < kArcPer; ++q)
            if (t.e0 + threadIdx.x + q * kArcThreads < t.e1) x[q] = __ldcs(tgt + at[q]);
#pragma unroll
        for (int q = 0; q < kArcPer; ++q) {
            const int64_t e = t.e0 + threadIdx.x + q * kArcThreads;
            if (e < t.e1) ntgt[e] = inv[x[q]];
        }
    }
}

// ------------------------------------------------------ degree segments --

struct SegBounds {
    int64_t lo[kSegs], hi[kSegs];
};

__device__ __forceinline__ int segment_of(int64_t d, const SegBounds &sb) {
    for (int s = 0; s < kSegs; ++s)
        if (d >= sb.lo[s] && d <= sb.hi[s]) return s;
    return -1;   // degree 0
}

// Nodes per degree segment.  After the degree relabelling a warp's 32
// nodes nearly always share a segment, so each warp adds its count with one
// shared-memory atomic per segment present (not 32 on one address).
__global__ void seg_count_kernel(const int64_t *off, int64_t n, SegBounds sb, unsigned long long *cnt) {
    __shared__ unsigned long long c[kSegs];
    if (threadIdx.x < kSegs) c[threadIdx.x] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    for (int64_t v0 = (int64_t)blockIdx.x * blockDim.x; v0 < n; v0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = v0 + threadIdx.x;
        const int s = v < n ? segment_of(off[v + 1] - off[v], sb) : -1;
        const unsigned peers = __match_any_sync(0xffffffffu, s);
        if (s >= 0 && lane == __ffs(peers) - 1) atomicAdd(&c[s], (unsigned long long)__popc(peers));
    }
    __syncthreads();
    if (threadIdx.x < kSegs && c[threadIdx.x]) atomicAdd(&cnt[threadIdx.x], c[threadIdx.x]);
}

__global__ void dense_list_kernel(const int64_t *off, int64_t n, SegBounds sb, const int64_t *seg_begin,
                                  int32_t *list, unsigned long long *fill) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        int s = segment_of(off[v + 1] - off[v], sb);
        if (s >= 0) {
            unsigned long long pos = atomicAdd(&fill[s], 1ULL);
            list[seg_begin[s] + (int64_t)pos] = (int32_t)v;
        }
    }
}

SegBounds bounds_of(const Layout &y) {
    SegBounds sb;
    for (int s = 0; s < kSegs; ++s) { sb.lo[s] = y.lo[s]; sb.hi[s] = y.hi[s]; }
    return sb;
}

}  // namespace

cudaError_t scan_exclusive_i64(const int64_t *in, int64_t *out, int64_t N, cudaStream_t s) {
    if (N <= 0) return cudaSuccess;
    int64_t tiles = (N + kScanTile - 1) / kScanTile;
    if (tiles == 1) {
        scan_tile_apply<<<1, kScanThreads, 0, s>>>(in, out, N, nullptr);
        return cudaGetLastError();
    }
    int64_t *sums = nullptr;
    cudaError_t e = tmp_alloc(&sums, sizeof(int64_t) * tiles * 2, s);
    if (e != cudaSuccess) return e;
    scan_tile_sums<<<(unsigned)tiles, kScanThreads, 0, s>>>(in, N, sums);
    e = scan_exclusive_i64(sums, sums + tiles, tiles, s);
    if (e == cudaSuccess) {
        scan_tile_apply<<<(unsigned)tiles, kScanThreads, 0, s>>>(in, out, N, sums + tiles);
        e = cudaGetLastError();
    }
    cudaFreeAsync(sums, s);
    return e;
}

cudaError_t validate_offsets(const int64_t *off, int64_t n, int64_t m, unsigned long long *err_dev,
                             cudaStream_t s) {
    validate_offsets_kernel<<<grid_for(n, 256), 256, 0, s>>>(off, n, m, err_dev);
    return cudaGetLastError();
}

cudaError_t check_targets(const int32_t *tgt, int64_t len, int64_t n, unsigned long long *err_dev,
                          unsigned long long *indeg, cudaStream_t s) {
    if (len > 0) check_targets_kernel<<<grid_for(len, 256), 256, 0, s>>>(tgt, len, n, err_dev, indeg);
    return cudaGetLastError();
}


namespace {
__global__ void weights_in_kernel(const int64_t *w, int64_t n, int64_t *tmp, unsigned long long *err) {
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u <= n;
         u += (int64_t)gridDim.x * blockDim.x) {
        int64_t x = u < n ? w[u] : 0;
        if (x < 0 || x >= ((int64_t)1 << 31)) {
            atomicOr(err, 1ULL);
            x = 0;
        }
        tmp[u] = x;
    }
}
}  // namespace

cudaError_t replica_starts(const int64_t *w, int64_t n, int64_t *wfirst, unsigned long long *err,
                           cudaStream_t s) {
    int64_t *tmp = nullptr;
    cudaError_t e = tmp_alloc(&tmp, sizeof(int64_t) * (n + 1), s);
    if (e != cudaSuccess) return e;
    weights_in_kernel<<<grid_for(n + 1, 256), 256, 0, s>>>(w, n, tmp, err);
    e = scan_exclusive_i64(tmp, wfirst, n + 1, s);
    cudaFreeAsync(tmp, s);
    return e;
}

cudaError_t widen_offsets(const int32_t *in, int64_t *out, int64_t count, cudaStream_t s) {
    widen_kernel<<<grid_for(count, 256), 256, 0, s>>>(in, out, count);
    return cudaGetLastError();
}

// Source nodes of the first and last arc of every kArcTile tile of the
// CSR (off, m arcs): 2 entries per tile, freed by the caller.
static cudaError_t tile_ends(const int64_t *off, int64_t n, int64_t m, int64_t **ends, cudaStream_t s,
                             bool default_pool = false) {
    const int64_t ntiles = (m + kArcTile - 1) / kArcTile;
    cudaError_t e = default_pool ? cudaMallocAsync(reinterpret_cast<void **>(ends), sizeof(int64_t) * 2 * ntiles, s)
                                 : tmp_alloc(ends, sizeof(int64_t) * 2 * ntiles, s);
    if (e != cudaSuccess) return e;
    tile_ends_kernel<<<grid_for(ntiles, 256), 256, 0, s>>>(off, n, m, ntiles, *ends);
    return cudaGetLastError();
}

cudaError_t transpose_csr_counted(const int64_t *off, const int32_t *tgt, int64_t n, int64_t m,
                                  const unsigned long long *indeg, const int32_t *perm, int64_t *toff,
                                  int32_t *ttgt, cudaStream_t s, cudaStream_t scatter_s,
                                  cudaEvent_t scatter_done) {
    // With the scatter on its own stream, the buffers it uses (and frees on
    // that stream) come from the device's default pool: a block freed there is
    // never handed to a later allocation of the library's pool on s, which
    // would make s wait for the scatter.
    const bool apart = scatter_s != nullptr;
    unsigned long long *cnt = nullptr;
    cudaError_t e = apart ? cudaMallocAsync(reinterpret_cast<void **>(&cnt), sizeof(unsigned long long) * (n + 1), s)
                          : tmp_alloc(&cnt, sizeof(unsigned long long) * (n + 1), s);
    if (e != cudaSuccess) return e;
    if (indeg) {
        permuted_counts<<<grid_for(n + 1, 256), 256, 0, s>>>(indeg, perm, n, cnt);
    } else {
        cudaMemsetAsync(cnt, 0, sizeof(unsigned long long) * (n + 1), s);
        if (m > 0) count_targets<<<grid_for(m, 256), 256, 0, s>>>(tgt, m, cnt);
    }
    e = scan_exclusive_i64(reinterpret_cast<int64_t *>(cnt), toff, n + 1, s);
    int64_t *ends = nullptr;
    if (e == cudaSuccess && m > 0) e = tile_ends(off, n, m, &ends, s, apart);
    cudaStream_t xs = s;   // the scatter's stream
    if (e == cudaSuccess && m > 0) {
        e = cudaMemcpyAsync(cnt, toff, sizeof(int64_t) * n, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess && scatter_s) {
            // the scatter on its own stream, ordered after everything above
            e = cudaEventRecord(scatter_done, s);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(scatter_s, scatter_done, 0);
            if (e == cudaSuccess) xs = scatter_s;
        }
        if (e == cudaSuccess) {
            const int64_t ntiles = (m + kArcTile - 1) / kArcTile;
            scatter_transpose<<<grid_for(ntiles * kArcThreads, kArcThreads), kArcThreads, 0, xs>>>(off, tgt, n, m,
                                                                                               ends, cnt, ttgt);
            e = cudaGetLastError();
        }
    }
    cudaFreeAsync(cnt, xs);
    if (ends) cudaFreeAsync(ends, xs);
    if (e == cudaSuccess && scatter_s) e = cudaEventRecord(scatter_done, xs);
    return e;
}

cudaError_t transpose_csr(const int64_t *off, const int32_t *tgt, int64_t n, int64_t m,
                          int64_t *toff, int32_t *ttgt, cudaStream_t s, cudaStream_t scatter_s,
                          cudaEvent_t scatter_done) {
    return transpose_csr_counted(off, tgt, n, m, nullptr, nullptr, toff, ttgt, s, scatter_s, scatter_done);
}

// Node order for the step kernel: out-degree buckets descending (so every
// degree class is a contiguous id range), and within a bucket in-degree
// buckets descending (the most gathered counters share L2 lines); two
// stable partitions, least significant key first.
cudaError_t degree_sort_counted(const int64_t *off, const int32_t *tgt, int64_t n, int64_t m, int32_t *perm,
                                int32_t *inv, unsigned long long *indeg, bool counted, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const int64_t ntiles = (n + kPartTile - 1) / kPartTile;
    int64_t *counts = nullptr;
    uint8_t *keys = nullptr;
    int32_t *perm1 = nullptr;
    cudaError_t e = tmp_alloc(&counts, sizeof(int64_t) * kBuckets * ntiles * 2, s);
    if (e == cudaSuccess) e = tmp_alloc(&keys, 2 * (size_t)n, s);
    if (e == cudaSuccess) e = tmp_alloc(&perm1, sizeof(int32_t) * n, s);
    if (e == cudaSuccess && !counted) {
        cudaMemsetAsync(indeg, 0, sizeof(unsigned long long) * n, s);
        if (m > 0) count_targets<<<grid_for(m, 256), 256, 0, s>>>(tgt, m, indeg);
    }
    if (e == cudaSuccess) {
        key_in_kernel<<<grid_for(n, 256), 256, 0, s>>>(indeg, n, keys);
        key_out_kernel<<<grid_for(n, 256), 256, 0, s>>>(off, n, keys + n);
        const int g = (int)(ntiles < 152 * 8 ? ntiles : 152 * 8);
        // pass 1: by in-degree bucket
        part_count<<<g, kPartThreads, 0, s>>>(nullptr, keys, n, ntiles, counts);
        e = scan_exclusive_i64(counts, counts + kBuckets * ntiles, kBuckets * ntiles, s);
        if (e == cudaSuccess)
            part_scatter<<<g, kPartThreads, 0, s>>>(nullptr, keys, n, ntiles, counts + kBuckets * ntiles,
                                                     perm1, nullptr);
        // pass 2 (stable): by out-degree bucket
        if (e == cudaSuccess) part_count<<<g, kPartThreads, 0, s>>>(perm1, keys + n, n, ntiles, counts);
        if (e == cudaSuccess) e = scan_exclusive_i64(counts, counts + kBuckets * ntiles, kBuckets * ntiles, s);
        if (e == cudaSuccess) {
            part_scatter<<<g, kPartThreads, 0, s>>>(perm1, keys + n, n, ntiles, counts + kBuckets * ntiles,
                                                     perm, inv);
            e = cudaGetLastError();
        }
    }
    cudaFreeAsync(counts, s);
    cudaFreeAsync(keys, s);
    cudaFreeAsync(perm1, s);
    return e;
}


cudaError_t relabel_csr(const int64_t *off, const int32_t *tgt, int64_t n, int64_t m,
                        const int32_t *perm, const int32_t *inv, int64_t *noff, int32_t *ntgt,
                        cudaStream_t s) {
    int64_t *deg = nullptr;
    cudaError_t e = tmp_alloc(&deg, sizeof(int64_t) * (n + 1), s);
    if (e != cudaSuccess) return e;
    permuted_degrees<<<grid_for(n + 1, 256), 256, 0, s>>>(off, perm, n, deg);
    e = scan_exclusive_i64(deg, noff, n + 1, s);
    int64_t *ends = nullptr;
    if (e == cudaSuccess && m > 0) e = tile_ends(noff, n, m, &ends, s);
    if (e == cudaSuccess && m > 0) {
        const int64_t ntiles = (m + kArcTile - 1) / kArcTile;
        relabel_arcs<<<grid_for(ntiles * kArcThreads, kArcThreads), kArcThreads, 0, s>>>(off, tgt, n, m, perm, inv,
                                                                                     noff, ends, ntgt);
        e = cudaGetLastError();
    }
    cudaFreeAsync(deg, s);
    if (ends) cudaFreeAsync(ends, s);
    return e;
}

cudaError_t count_degree_segments(const int64_t *off, int64_t n, const Layout &y,
                                  int64_t *seg_count_host, cudaStream_t s) {
    unsigned long long *cnt = nullptr;
    cudaError_t e = tmp_alloc(&cnt, sizeof(unsigned long long) * kSegs, s);
    if (e != cudaSuccess) return e;
    cudaMemsetAsync(cnt, 0, sizeof(unsigned long long) * kSegs, s);
    if (n > 0) seg_count_kernel<<<grid_for(n, 256), 256, 0, s>>>(off, n, bounds_of(y), cnt);
    unsigned long long h[kSegs];
    cudaMemcpyAsync(h, cnt, sizeof(h), cudaMemcpyDeviceToHost, s);
    e = cudaStreamSynchronize(s);
    cudaFreeAsync(cnt, s);
    for (int k = 0; k < kSegs; ++k) seg_count_host[k] = (int64_t)h[k];
    return e;
}

cudaError_t build_dense_list(const int64_t *off, int64_t n, const Layout &y,
                             const int64_t *seg_begin, int32_t *list, unsigned long long *fill,
                             cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(fill, 0, sizeof(unsigned long long) * kSegs, s);
    if (e != cudaSuccess) return e;
    if (n > 0) dense_list_kernel<<<grid_for(n, 256), 256, 0, s>>>(off, n, bounds_of(y), seg_begin, list, fill);
    return cudaGetLastError();
}

namespace {

// One warp per node: the node's targets below `hot` first, then the
// others (each group in its original order), written to out; hcnt[v]
// receives the size of the first group.  A node's arcs stay in its own
// range [off[v], off[v+1]), so the CSR is the same graph.
__global__ void partition_hot_kernel(const int64_t *__restrict__ off, const int32_t *__restrict__ tgt,
                                     int64_t n, uint32_t hot, int32_t *__restrict__ out, int32_t *hcnt) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    unsigned lt;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(lt));
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t v = gw; v < n; v += nw) {
        const int64_t e0 = off[v], e1 = off[v + 1];
        int64_t c = 0;
        for (int64_t j0 = e0; j0 < e1; j0 += 32) {
            const int64_t j = j0 + lane;
            c += __popc(__ballot_sync(FULL, j < e1 && (uint32_t)tgt[j] < hot));
        }
        int64_t hp = e0, cp = e0 + c;
        for (int64_t j0 = e0; j0 < e1; j0 += 32) {
            const int64_t j = j0 + lane;
            const bool valid = j < e1;
            const int32_t w = valid ? tgt[j] : 0;
            const bool h = valid && (uint32_t)w < hot;
            const unsigned bh = __ballot_sync(FULL, h), bc = __ballot_sync(FULL, valid && !h);
            if (h) out[hp + __popc(bh & lt)] = w;
            else if (valid) out[cp + __popc(bc & lt)] = w;
            hp += __popc(bh);
            cp += __popc(bc);
        }
        if (lane == 0) hcnt[v] = (int32_t)c;
    }
}

}  // namespace

cudaError_t partition_hot(const int64_t *off, int32_t *tgt, int64_t n, int64_t m, uint32_t hot, int32_t *hcnt,
                          cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    int32_t *tmp = nullptr;
    cudaError_t e = tmp_alloc(&tmp, sizeof(int32_t) * (size_t)(m > 0 ? m : 1), s);
    if (e != cudaSuccess) return e;
    partition_hot_kernel<<<grid_for(32 * n, 256), 256, 0, s>>>(off, tgt, n, hot, tmp, hcnt);
    e = cudaGetLastError();
    if (e == cudaSuccess && m > 0) e = cudaMemcpyAsync(tgt, tmp, sizeof(int32_t) * (size_t)m,
                                                       cudaMemcpyDeviceToDevice, s);
    const cudaError_t f = cudaFreeAsync(tmp, s);
    return e != cudaSuccess ? e : f;
}

}  // namespace hb

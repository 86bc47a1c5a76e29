// hb_runs.cu -- several HyperBall runs of one graph in one handle (Sec. 5:
// repeated runs with independent hash seeds, whose spread gives the
// empirical standard deviation of every estimate).
//
// Each node's row holds R = 2^lruns counters of p = 2^gb registers, run r
// in bytes [r p, (r+1) p) and hashed with its own seed.  The register-wise
// maximum of Algorithm 2 never mixes bytes, so one union over the row is
// every run's union, and the gather, the frontier, the pushed union and
// the copy-forward of the single-run path serve unchanged on rows of R p
// bytes: the targets are streamed once per iteration for all runs and each
// gathered row is R p contiguous bytes.  Only the initial counters, the
// per-node tail (one size() and one set of Sec. 5 accumulators per run,
// stored run-minor at v * R + r) and the readouts differ.
#include "hb_step_dev.cuh"

namespace hb {

namespace {

using namespace dev;

template <int LOG2P, bool F32>
__global__ void __launch_bounds__(kStepThreads, Cfg<LOG2P>::CPL >= 4 ? 3 : HB_MIN_BLOCKS)
    runs_step_kernel(StepArgs a) {
    step_body<LOG2P, F32, true>(a);
}

template <int LOG2P, bool F32>
__global__ void __launch_bounds__(kStepThreads) runs_tail_kernel(StepArgs a) {
    tail_body<LOG2P, F32, true>(a);
}

// Algorithm 2's first loop for every run: chunk c of node v belongs to run
// r = c / (p/16); add(c_r[v], v) with run r's seed, in both buffers.
__global__ void runs_init_rows_kernel(StepArgs a, const int32_t *perm) {
    const int CH = (1 << a.b) >> 4;
    const int lg = a.gb - 4;
    const int64_t total = a.n * CH;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < total;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = k / CH;
        const int c = (int)(k - v * CH);
        const int r = c >> lg;
        const uint64_t orig = perm ? (uint64_t)perm[v] : (uint64_t)v;
        uint32_t idx, rho;
        hash_to_register(splitmix64(a.run_seeds[r], orig), a.gb, idx, rho);
        uint32_t w[4] = {0u, 0u, 0u, 0u};
        if ((int)(idx >> 4) == (c & ((1 << lg) - 1))) w[(idx >> 2) & 3] = rho << (8 * (idx & 3));
        const uint4 val = make_uint4(w[0], w[1], w[2], w[3]);
        reinterpret_cast<uint4 *>(a.regs[0])[k] = val;
        reinterpret_cast<uint4 *>(a.regs[1])[k] = val;
    }
}

// Cached estimate and zero accumulators of every (node, run): the initial
// counter of a run has one nonzero register.
template <bool F32>
__global__ void runs_init_nodes_kernel(StepArgs a, const int32_t *perm) {
    const int P = 1 << a.gb;
    const int64_t total = a.n << a.lruns;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = q >> a.lruns;
        const int r = (int)(q & ((1 << a.lruns) - 1));
        const uint64_t orig = perm ? (uint64_t)perm[v] : (uint64_t)v;
        uint32_t idx, rho;
        hash_to_register(splitmix64(a.run_seeds[r], orig), a.gb, idx, rho);
        const uint32_t V = (uint32_t)P - 1;
        const unsigned long long S = 1ULL << (64 - a.gb - (int)rho);
        if (F32) static_cast<float *>(a.ecache)[q] = estimate32(V, S, P, a.gb, a.c32, a.thr_x, a.lc32);
        else static_cast<double *>(a.ecache)[q] = estimate64(V, S, P, a.gb, a.c64, a.thr_x, a.lc64);
        a.sumd[q] = 0.0;
        a.harm[q] = 0.0;
        if (a.disc) a.disc[q] = 0.0;
        if (r == 0) a.changed[v] = 0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) reset_counters(a.ctr);
}

// Sec. 6 for rows of several runs: run r of the caller's node u starts from
// the replicas wfirst[u] .. wfirst[u+1]-1 hashed with run r's seed.  One
// thread per (node, run) writes that run's p bytes of the row, in both
// buffers, and its cached estimate and zero accumulators.
template <bool F32>
__global__ void runs_init_weighted_kernel(StepArgs a, const int32_t *perm, const int64_t *wfirst) {
    const int P = 1 << a.gb;
    const int CH = P >> 4;
    const uint4 z = make_uint4(0u, 0u, 0u, 0u);
    const int64_t total = a.n << a.lruns;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = q >> a.lruns;
        const int r = (int)(q & ((1 << a.lruns) - 1));
        const int64_t u = perm ? (int64_t)perm[v] : v;
        uint8_t *g0 = a.regs[0] + (v << a.b) + (int64_t)r * P;
        uint4 *g1 = reinterpret_cast<uint4 *>(a.regs[1] + (v << a.b) + (int64_t)r * P);
        for (int c = 0; c < CH; ++c) reinterpret_cast<uint4 *>(g0)[c] = z;
        for (int64_t item = wfirst[u]; item < wfirst[u + 1]; ++item) {
            uint32_t idx, rho;
            hash_to_register(splitmix64(a.run_seeds[r], (uint64_t)item), a.gb, idx, rho);
            if (g0[idx] < rho) g0[idx] = (uint8_t)rho;
        }
        uint32_t V = 0;
        unsigned long long S = 0;
        for (int c = 0; c < CH; ++c) {
            const uint4 x = reinterpret_cast<const uint4 *>(g0)[c];
            g1[c] = x;
            chunk_sums(x, a.gb, V, S);
        }
        if (F32) static_cast<float *>(a.ecache)[q] = estimate32(V, S, P, a.gb, a.c32, a.thr_x, a.lc32);
        else static_cast<double *>(a.ecache)[q] = estimate64(V, S, P, a.gb, a.c64, a.thr_x, a.lc64);
        a.sumd[q] = 0.0;
        a.harm[q] = 0.0;
        if (a.disc) a.disc[q] = 0.0;
        if (r == 0) a.changed[v] = 0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) reset_counters(a.ctr);
}

// Sec. 3 centralities of run r of node v (internal index), as
// node_centralities for a single run: closeness, harmonic, Lin, reachable.
template <bool F32>
__device__ __forceinline__ void run_centralities(const StepArgs &a, const uint8_t *regs, int64_t v, int r,
                                                 double out[4]) {
    const int P = 1 << a.gb;
    const int CH = P >> 4;
    uint32_t V = 0;
    unsigned long long S = 0;
    const uint4 *row = reinterpret_cast<const uint4 *>(regs + (v << a.b) + (int64_t)r * P);
    for (int c = 0; c < CH; ++c) chunk_sums(row[c], a.gb, V, S);
    double e;
    if (F32) e = (double)estimate32(V, S, P, a.gb, a.c32, a.thr_x, a.lc32);
    else e = estimate64(V, S, P, a.gb, a.c64, a.thr_x, a.lc64);
    const int64_t q = (v << a.lruns) + r;
    const double s = a.sumd[q];
    out[0] = s > 0.0 ? __ddiv_rn(1.0, s) : 0.0;
    out[1] = a.harm[q];
    out[2] = s > 0.0 ? __ddiv_rn(__dmul_rn(e, e), s) : 1.0;
    out[3] = e;
}

template <bool F32>
__global__ void runs_centralities_kernel(StepArgs a, const uint8_t *regs, const int32_t *perm, int r,
                                         double *closeness, double *harmonic, double *lin,
                                         double *reachable) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < a.n;
         v += (int64_t)gridDim.x * blockDim.x) {
        double c[4];
        run_centralities<F32>(a, regs, v, r, c);
        const int64_t o = perm ? (int64_t)perm[v] : v;
        if (closeness) closeness[o] = c[0];
        if (harmonic) harmonic[o] = c[1];
        if (lin) lin[o] = c[2];
        if (reachable) reachable[o] = c[3];
    }
}

// Sec. 5: per node, the mean and the empirical (sample, R-1) standard
// deviation over the R runs of one centrality (which = 4: the Sec. 7
// discounted accumulator), in two passes.
template <bool F32>
__global__ void runs_stats_kernel(StepArgs a, const uint8_t *regs, const int32_t *perm, int which,
                                  double *mean, double *sd) {
    const int R = 1 << a.lruns;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < a.n;
         v += (int64_t)gridDim.x * blockDim.x) {
        double c[4], sum = 0.0;
        for (int r = 0; r < R; ++r) {
            if (which < 4) run_centralities<F32>(a, regs, v, r, c);
            sum += which < 4 ? c[which] : a.disc[(v << a.lruns) + r];
        }
        const double mu = sum / (double)R;
        double q = 0.0;
        for (int r = 0; r < R; ++r) {
            if (which < 4) run_centralities<F32>(a, regs, v, r, c);
            const double d = (which < 4 ? c[which] : a.disc[(v << a.lruns) + r]) - mu;
            q += d * d;
        }
        const int64_t o = perm ? (int64_t)perm[v] : v;
        if (mean) mean[o] = mu;
        if (sd) sd[o] = R > 1 ? sqrt(q / (double)(R - 1)) : 0.0;
    }
}

__global__ void gather_strided_kernel(const double *src, const int32_t *inv, int64_t n, int lstride, int off,
                                      double *out) {
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n;
         u += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = inv ? (int64_t)inv[u] : u;
        out[u] = src[(v << lstride) + off];
    }
}

template <bool F32>
const void *runs_step_ptr(int log2row) {
    switch (log2row) {
#define HB_CASE(B) case B: return reinterpret_cast<const void *>(&runs_step_kernel<B, F32>);
        HB_CASE(5) HB_CASE(6) HB_CASE(7) HB_CASE(8) HB_CASE(9) HB_CASE(10) HB_CASE(11) HB_CASE(12)
#undef HB_CASE
        default: return nullptr;
    }
}

template <bool F32>
cudaError_t runs_step_t(const StepArgs &a, int log2row, int grid, cudaStream_t s) {
    switch (log2row) {
#define HB_CASE(B) case B: runs_step_kernel<B, F32><<<grid, kStepThreads, 0, s>>>(a); break;
        HB_CASE(5) HB_CASE(6) HB_CASE(7) HB_CASE(8) HB_CASE(9) HB_CASE(10) HB_CASE(11) HB_CASE(12)
#undef HB_CASE
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <bool F32>
cudaError_t runs_tail_t(const StepArgs &a, int log2row, int grid, cudaStream_t s) {
    switch (log2row) {
#define HB_CASE(B) case B: runs_tail_kernel<B, F32><<<grid, kStepThreads, 0, s>>>(a); break;
        HB_CASE(5) HB_CASE(6) HB_CASE(7) HB_CASE(8) HB_CASE(9) HB_CASE(10) HB_CASE(11) HB_CASE(12)
#undef HB_CASE
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace

int runs_step_blocks_per_sm(int log2row, bool fp32) {
    const void *k = fp32 ? runs_step_ptr<true>(log2row) : runs_step_ptr<false>(log2row);
    int blocks = 0;
    if (!k || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k, kStepThreads, 0) != cudaSuccess)
        return 4;
    return blocks > 0 ? blocks : 1;
}

cudaError_t launch_runs_step(const StepArgs &a, int log2row, bool fp32, int grid, cudaStream_t s) {
    return fp32 ? runs_step_t<true>(a, log2row, grid, s) : runs_step_t<false>(a, log2row, grid, s);
}

cudaError_t launch_runs_tail(const StepArgs &a, int log2row, bool fp32, int grid, cudaStream_t s) {
    return fp32 ? runs_tail_t<true>(a, log2row, grid, s) : runs_tail_t<false>(a, log2row, grid, s);
}

cudaError_t launch_runs_init(const StepArgs &a, const int32_t *perm, bool fp32, cudaStream_t s,
                             const int64_t *wfirst) {
    if (wfirst) {
        const int64_t q = a.n << a.lruns;
        if (fp32) runs_init_weighted_kernel<true><<<grid_for(q, 128), 128, 0, s>>>(a, perm, wfirst);
        else runs_init_weighted_kernel<false><<<grid_for(q, 128), 128, 0, s>>>(a, perm, wfirst);
        return cudaGetLastError();
    }
    const int64_t chunks = a.n * ((1 << a.b) >> 4);
    if (a.n > 0) runs_init_rows_kernel<<<grid_for(chunks, 256), 256, 0, s>>>(a, perm);
    const int64_t q = a.n << a.lruns;
    if (fp32) runs_init_nodes_kernel<true><<<grid_for(q, 256), 256, 0, s>>>(a, perm);
    else runs_init_nodes_kernel<false><<<grid_for(q, 256), 256, 0, s>>>(a, perm);
    return cudaGetLastError();
}

cudaError_t launch_runs_centralities(const StepArgs &a, const uint8_t *regs, const int32_t *perm, bool fp32,
                                     int run, double *closeness, double *harmonic, double *lin,
                                     double *reachable, cudaStream_t s) {
    if (a.n == 0) return cudaSuccess;
    if (fp32)
        runs_centralities_kernel<true><<<grid_for(a.n, 256), 256, 0, s>>>(a, regs, perm, run, closeness,
                                                                          harmonic, lin, reachable);
    else
        runs_centralities_kernel<false><<<grid_for(a.n, 256), 256, 0, s>>>(a, regs, perm, run, closeness,
                                                                           harmonic, lin, reachable);
    return cudaGetLastError();
}

cudaError_t launch_runs_stats(const StepArgs &a, const uint8_t *regs, const int32_t *perm, bool fp32,
                              int which, double *mean, double *sd, cudaStream_t s) {
    if (a.n == 0) return cudaSuccess;
    if (fp32) runs_stats_kernel<true><<<grid_for(a.n, 256), 256, 0, s>>>(a, regs, perm, which, mean, sd);
    else runs_stats_kernel<false><<<grid_for(a.n, 256), 256, 0, s>>>(a, regs, perm, which, mean, sd);
    return cudaGetLastError();
}

cudaError_t launch_gather_strided(const double *src, const int32_t *inv, int64_t n, int lstride, int off,
                                  double *out, cudaStream_t s) {
    if (n > 0) gather_strided_kernel<<<grid_for(n, 256), 256, 0, s>>>(src, inv, n, lstride, off, out);
    return cudaGetLastError();
}

}  // namespace hb

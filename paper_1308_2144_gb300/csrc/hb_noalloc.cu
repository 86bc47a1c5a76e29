// hb_noalloc.cu -- one HyperBall iteration for callers that cannot
// allocate device memory (hb_step_noalloc in include/hyperball.h).
//
// Who needs it: code that runs inside another framework's memory pool or
// arena (where a cudaMalloc outside the pool breaks its accounting or is
// forbidden), services that freeze allocation after start-up so that no
// request can stall in or fail on the allocator, and hosts that hand this
// library device buffers but no allocator at all.  The caller passes every
// input and output; the temporary data of the iteration (degree lists,
// work plan, partial counters of split nodes, cached estimates, counters,
// estimator tables) lives in g_noalloc_scratch, one file-scope __device__
// array of HB_NOALLOC_SCRATCH_BYTES that every GPU loading the library
// holds until the process exits.  The paper has no counterpart.
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "hb_internal.cuh"
#include "hyperball.h"

namespace hb {

namespace {

constexpr size_t kScratchBytes = (size_t)HB_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

// In host code this name is only a stand-in for the array: its device
// address comes from cudaGetSymbolAddress (see scratch_of()).
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_setup_mu;
unsigned char *g_scratch_dev[kMaxDevices] = {nullptr};

struct Bounds {
    int64_t lo[kSegs], hi[kSegs];
};

__device__ __forceinline__ int seg_of(int64_t d, const Bounds &sb) {
    for (int s = 0; s < kSegs; ++s)
        if (d >= sb.lo[s] && d <= sb.hi[s]) return s;
    return -1;
}

// Nodes per degree segment and chunks of split (heavy) nodes.
__global__ void na_count_kernel(const int64_t *off, int64_t n, Bounds sb, int64_t heavy,
                                int64_t chunk, unsigned long long *cnt) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        const int64_t d = off[v + 1] - off[v];
        const int s = seg_of(d, sb);
        if (s >= 0) atomicAdd(&cnt[s], 1ULL);
        if (d > heavy) atomicAdd(&cnt[kSegs], (unsigned long long)((d + chunk - 1) / chunk));
    }
}

// size() of every current counter: the iteration subtracts it from the
// size of each counter that changes (Sec. 5).
__global__ void na_estimates_kernel(StepArgs a, const uint8_t *cur) {
    const int P = 1 << a.b;
    const int CH = P >> 4;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < a.n;
         v += (int64_t)gridDim.x * blockDim.x) {
        uint32_t V = 0;
        unsigned long long S = 0;
        const uint4 *row = reinterpret_cast<const uint4 *>(cur + v * P);
        for (int c = 0; c < CH; ++c) chunk_sums(row[c], a.b, V, S);
        static_cast<double *>(a.ecache)[v] = estimate64(V, S, P, a.b, a.c64, a.thr_x, a.lc64);
    }
}

int grid_of(int64_t work) {
    int64_t g = (work + 255) / 256;
    if (g < 1) g = 1;
    if (g > 152 * 32) g = 152 * 32;
    return (int)g;
}

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

hb_status fail(hb_status st, const std::string &msg) {
    set_last_error(msg.c_str());
    return st;
}

bool on_device(const void *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// True when the byte ranges [p, p + a) and [q, q + b) share a byte.
bool overlaps(const void *p, size_t a, const void *q, size_t b) {
    if (!p || !q || a == 0 || b == 0) return false;
    const uintptr_t x = reinterpret_cast<uintptr_t>(p), y = reinterpret_cast<uintptr_t>(q);
    return x < y + b && y < x + a;
}

// Device address of the scratch array on the current device, looked up
// once per device (with that device current).
cudaError_t scratch_of(unsigned char **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_dev[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_dev[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_scratch_dev[dev];
    return cudaSuccess;
}

}  // namespace

}  // namespace hb

using namespace hb;

extern "C" hb_status hb_step_noalloc(const int64_t *offsets, const int32_t *targets, int64_t n,
                                     int64_t m, int log2m, int32_t t, const uint8_t *cur,
                                     uint8_t *next, double *sumd, double *harm, uint8_t *changed,
                                     int64_t *n_changed, void *stream) {
    set_last_error("");
    if (log2m < kMinLog2m || log2m > kMaxLog2m) return fail(HB_ERR_INVALID, "log2m must lie in [4, 12]");
    if (n < 0 || n >= (int64_t)1 << 31) return fail(HB_ERR_INVALID, "n must lie in [0, 2^31)");
    if (m < 0) return fail(HB_ERR_INVALID, "m must be >= 0");
    if (t < 0) return fail(HB_ERR_INVALID, "t must be >= 0");
    if (!offsets || (m > 0 && !targets) ||
        (n > 0 && (!cur || !next || !sumd || !harm || !changed)))
        return fail(HB_ERR_INVALID, "a required pointer is NULL");
    const void *ptrs[] = {offsets, targets, cur, next, sumd, harm, changed};
    for (const void *p : ptrs)
        if (p && !on_device(p))
            return fail(HB_ERR_INVALID, "hb_step_noalloc takes device pointers only");
    {
        // Buffers the iteration writes may share no byte with any other
        // buffer: next must not alias cur (the gather would read counters
        // this iteration already raised), and a write into offsets, targets
        // or the other outputs would corrupt what the kernels still read.
        const int P0 = 1 << log2m;
        const size_t rb = (size_t)n * (size_t)P0;
        const struct { const void *p; size_t bytes; bool written; const char *name; } buf[] = {
            {offsets, sizeof(int64_t) * (size_t)(n + 1), false, "offsets"},
            {targets, sizeof(int32_t) * (size_t)m, false, "targets"},
            {cur, rb, false, "cur"},
            {next, rb, true, "next"},
            {sumd, sizeof(double) * (size_t)n, true, "sumd"},
            {harm, sizeof(double) * (size_t)n, true, "harm"},
            {changed, (size_t)n, true, "changed"}};
        const int nb = (int)(sizeof(buf) / sizeof(buf[0]));
        for (int i = 0; i < nb; ++i)
            for (int j = i + 1; j < nb; ++j)
                if ((buf[i].written || buf[j].written) &&
                    overlaps(buf[i].p, buf[i].bytes, buf[j].p, buf[j].bytes))
                    return fail(HB_ERR_INVALID, std::string("hb_step_noalloc: ") + buf[i].name + " and " +
                                                    buf[j].name + " overlap");
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned char *base = nullptr;
    cudaError_t e = scratch_of(&base);
    if (e != cudaSuccess) return fail(HB_ERR_CUDA, std::string("scratch set-up: ") + cudaGetErrorString(e));

    const Layout y = make_layout(log2m);
    const int P = 1 << log2m;
    // 1. the CSR checks of hb_create (offsets[0] = 0, offsets[n] = m,
    //    offsets never decrease, every target in [0, n)) into the word after
    //    the counts, and the degree segments and heavy chunks of the
    //    caller's CSR; both come back in one copy, before any gather runs.
    //    The count kernel reads only offsets[0 .. n], so it is safe on a
    //    malformed CSR too.
    unsigned long long *cnt = reinterpret_cast<unsigned long long *>(base);
    unsigned long long *csr_err = cnt + kSegs + 1;
    const size_t cnt_bytes = up256(sizeof(unsigned long long) * (kSegs + 2));
    Bounds sb;
    for (int k = 0; k < kSegs; ++k) { sb.lo[k] = y.lo[k]; sb.hi[k] = y.hi[k]; }
    unsigned long long hcnt[kSegs + 2];
    e = cudaMemsetAsync(cnt, 0, sizeof(hcnt), s);
    if (e == cudaSuccess) e = validate_offsets(offsets, n, m, csr_err, s);
    if (e == cudaSuccess) e = check_targets(targets, m, n, csr_err, nullptr, s);
    if (e == cudaSuccess && n > 0) {
        na_count_kernel<<<grid_of(n), 256, 0, s>>>(offsets, n, sb, y.heavy, y.chunk, cnt);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(hcnt, cnt, sizeof(hcnt), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(HB_ERR_CUDA, std::string("hb_step_noalloc: ") + cudaGetErrorString(e));
    if (const unsigned long long bad = hcnt[kSegs + 1]) {
        std::string why;
        if (bad & 1) why += " offsets[0] != 0;";
        if (bad & 2) why += " offsets[n] != m;";
        if (bad & 4) why += " offsets decrease;";
        if (bad & 8) why += " a target lies outside [0, n);";
        return fail(HB_ERR_INVALID, "malformed CSR:" + why);
    }
    int64_t seg_count[kSegs], seg_begin[kSegs], n_pos = 0;
    for (int k = 0; k < kSegs; ++k) { seg_count[k] = (int64_t)hcnt[k]; seg_begin[k] = n_pos; n_pos += seg_count[k]; }
    const int64_t heavy_nodes = seg_count[0];
    const int64_t chunks = (int64_t)hcnt[kSegs];

    // 2. carve the scratch array
    size_t off = cnt_bytes;
    auto take = [&](size_t bytes) { size_t at = off; off += up256(bytes); return base + at; };
    Counters *ctr = reinterpret_cast<Counters *>(take(sizeof(Counters)));
    Plan *plan = reinterpret_cast<Plan *>(take(sizeof(Plan)));
    int64_t *seg_begin_dev = reinterpret_cast<int64_t *>(take(sizeof(seg_begin)));
    unsigned long long *fill = reinterpret_cast<unsigned long long *>(take(sizeof(unsigned long long) * kSegs));
    double *lc64 = reinterpret_cast<double *>(take(sizeof(double) * (P + 1)));
    float *lc32 = reinterpret_cast<float *>(take(sizeof(float) * (P + 1)));
    int32_t *list = reinterpret_cast<int32_t *>(take(sizeof(int32_t) * (size_t)n_pos));
    double *ecache = reinterpret_cast<double *>(take(sizeof(double) * (size_t)n));
    int64_t *cstart = reinterpret_cast<int64_t *>(take(sizeof(int64_t) * (size_t)(heavy_nodes + 1)));
    int32_t *owner = reinterpret_cast<int32_t *>(take(sizeof(int32_t) * (size_t)chunks));
    uint8_t *partial = take((size_t)chunks * P);
    uint32_t *arrive = reinterpret_cast<uint32_t *>(take(sizeof(uint32_t) * (size_t)(heavy_nodes + 1)));
    if (off > kScratchBytes)
        return fail(HB_ERR_INVALID, "hb_step_noalloc: this graph needs " + std::to_string(off) +
                                        " bytes of scratch; the maximum is " +
                                        std::to_string(kScratchBytes) + " (HB_NOALLOC_SCRATCH_BYTES)");

    // 3. the iteration's arguments: dense mode, no frontier, caller's order
    StepArgs a{};
    a.off = offsets;
    a.tgt = targets;
    a.regs[t & 1] = const_cast<uint8_t *>(cur);
    a.regs[(t + 1) & 1] = next;
    a.sumd = sumd;
    a.harm = harm;
    a.ecache = ecache;
    a.changed = changed;
    a.dense_list = list;
    a.plan_dense = plan;
    a.plan_sparse = plan;
    a.owner_dense = owner;
    a.cstart_dense = cstart;
    a.owner_sparse = owner;
    a.cstart_sparse = cstart;
    a.partial = partial;
    a.arrive = arrive;
    a.ctr = ctr;
    a.lc64 = lc64;
    a.lc32 = lc32;
    const double alpha = hll_alpha_of(P);
    a.c64 = std::ldexp(alpha * (double)P * (double)P, 64 - log2m);
    a.c32 = (float)a.c64;
    const unsigned __int128 Y = (unsigned __int128)std::ldexp(alpha, 64);
    a.thr_x = (unsigned long long)((2 * Y + 4) / 5);
    a.n = n;
    a.n_pos = n_pos;
    a.m = m;
    for (int k = 0; k < kSegs; ++k) { a.seg_begin[k] = seg_begin[k]; a.seg_lo[k] = y.lo[k]; a.seg_hi[k] = y.hi[k]; }
    a.b = log2m;
    a.aps = y.aps;
    a.frontier = HB_FRONTIER_OFF;
    a.has_reverse = 0;

    // 4. everything that must start at zero or at a fixed value; the array
    //    keeps the previous call's contents otherwise
    Counters c0;
    std::memset(&c0, 0, sizeof(c0));
    c0.mode = 0;
    c0.t = t;
    c0.steps_done = t;
    e = cudaMemcpyAsync(ctr, &c0, sizeof(c0), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(arrive, 0, sizeof(uint32_t) * (size_t)(heavy_nodes + 1), s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(seg_begin_dev, seg_begin, sizeof(seg_begin), cudaMemcpyHostToDevice, s);
    // nodes without successors keep their counter and never change
    if (e == cudaSuccess && n > 0) e = cudaMemcpyAsync(next, cur, (size_t)n * P, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && n > 0) e = cudaMemsetAsync(changed, 0, (size_t)n, s);
    if (e == cudaSuccess) e = launch_lc_tables(lc64, lc32, P, s);
    if (e == cudaSuccess && n > 0) {
        na_estimates_kernel<<<grid_of(n), 256, 0, s>>>(a, cur);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = build_dense_list(offsets, n, y, seg_begin_dev, list, fill, s);
    if (e == cudaSuccess) e = launch_dense_plan(a, y, seg_count, plan, owner, cstart, s);
    int dev = 0, sms = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = launch_step_kernel(a, log2m, false, sms * step_blocks_per_sm(log2m, false), s);
    Counters done;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&done, ctr, sizeof(done), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(HB_ERR_CUDA, std::string("hb_step_noalloc: ") + cudaGetErrorString(e));
    if (done.err) {
        // the same device-side checks, and the same report, as hb_step
        std::string why = "a device-side check failed during the step:";
        if (done.err & kErrCasBound) why += " the pushed union's compare-and-swap loop reached its bound;";
        if (done.err & kErrTarget) why += " an arc target lies outside [0, n) (debug build check);";
        return fail(HB_ERR_STATE, why);
    }
    if (n_changed) *n_changed = (int64_t)done.n_changed;
    return HB_OK;
}

/*
 * hyperball.h -- C ABI of the GB300 HyperBall library.
 *
 * HyperBall (Boldi & Vigna, "In-Core Computation of Geometric Centralities
 * with HyperBall", arXiv:1308.2144) keeps one HyperLogLog counter of
 * p = 2^log2m one-byte registers per node.  Each iteration sets every
 * counter to the register-wise maximum of itself and its successors'
 * counters (Sec. 4.2, Algorithm 2) and folds the change of each counter's
 * size estimate into three per-node accumulators (Sec. 5); iterations stop
 * after the first one that leaves every counter unchanged (Sec. 4.2).
 * Closeness, Lin and harmonic centrality and the coreachable-set size
 * follow (Sec. 3).
 *
 * Conventions for every call:
 *   - Graphs are CSR: the successors of node v are
 *     targets[offsets[v] .. offsets[v+1]-1]; offsets has n+1 entries with
 *     offsets[0] = 0 and offsets[n] = m, non-decreasing; every target lies
 *     in [0, n).  Self-loops and repeated arcs are accepted (union is
 *     idempotent).  n must be below 2^31.
 *   - The graph given is the one scanned: a node's counter collects its
 *     successors.  The paper's (in-)centralities are distances *to* a node,
 *     so pass the transpose G^T, or pass G with HB_TRANSPOSE (Sec. 5).
 *   - Pointers may be host or device memory; the library tells them apart
 *     with cudaPointerGetAttributes.  Inputs are copied unless
 *     HB_BORROW_DEVICE_PTRS is set, in which case device inputs must stay
 *     valid and unchanged until hb_destroy.  Outputs may be host or device
 *     memory of the stated size; the call returns when they are written.
 *   - The library owns every buffer it allocates (registers, flags,
 *     accumulators) and frees them in hb_destroy (into its memory pool:
 *     see hb_trim_memory).
 *   - All device work runs on the stream in hb_options (NULL = the legacy
 *     default stream).  A handle must not be used by two threads at once;
 *     distinct handles are independent.
 *   - Every call returns an hb_status.  On failure hb_last_error() gives a
 *     message (thread-local).  A failed call leaves the handle as it was,
 *     except HB_ERR_CUDA during a step, after which the handle is marked
 *     unusable (HB_ERR_STATE on later calls).
 */
#ifndef HYPERBALL_H
#define HYPERBALL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HB_OK = 0,
    HB_ERR_INVALID = -1,        /* bad argument or malformed graph */
    HB_ERR_OOM = -2,            /* device allocation failed */
    HB_ERR_CUDA = -3,           /* a CUDA call failed */
    HB_ERR_NOT_CONVERGED = -4,  /* max_steps iterations ran, state still valid */
    HB_ERR_TIMEOUT = -5,        /* a bounded device-side wait gave up */
    HB_ERR_STATE = -6           /* handle unusable or call out of order */
} hb_status;

/* hb_options.flags */
#define HB_TRANSPOSE          0x1u  /* scan G^T: the library transposes the CSR on the device */
#define HB_BORROW_DEVICE_PTRS 0x2u  /* device inputs are used in place, not copied */
#define HB_FP32_ESTIMATE      0x4u  /* precision form: FP32 estimates and deltas, FP64 accumulators */
#define HB_NO_RELABEL         0x8u  /* keep the caller's node order on the device (no degree sort) */
#define HB_PROFILE            0x10u /* time the gather kernel of every iteration with CUDA events */
#define HB_PULL_GATHER        0x20u /* frontier iterations gather every successor of the nodes they
                                       recompute, instead of pushing last iteration's changed
                                       counters along the reverse CSR (results are the same) */
#define HB_NEIGHBOURHOOD      0x40u /* record the neighbourhood function N(t) after every iteration
                                       (hb_get_neighbourhood) */
#define HB_PACKED_REGISTERS   0x80u /* hold each register in six bits, not a byte (Sec. 4.1: a
                                       register needs about log2 log2 n bits; every value the
                                       method produces, at most 64 - log2m, fits): a counter
                                       takes 3p/4 bytes, 16 registers in 12 bytes, register j
                                       at bits 6j .. 6j+5 of the counter read as one
                                       little-endian bit string.  Results are identical to
                                       byte registers.  Needs HB_FRONTIER_OFF; not with
                                       hot_nodes, hb_set_hot_nodes, hb_set_weights, hb_save,
                                       hb_create_runs, the batched or served forms
                                       (HB_ERR_INVALID, or HB_ERR_STATE on a handle). */

/* hb_options.frontier: how the nodes to recompute are chosen each step
 * (Sec. 5 / 5.1 modification tracking).  Results never depend on it. */
#define HB_FRONTIER_AUTO 0  /* push from changed nodes when that is cheaper than a full scan */
#define HB_FRONTIER_PULL 1  /* each node checks its successors' changed flags */
#define HB_FRONTIER_PUSH 2  /* changed nodes mark their predecessors (needs the reverse CSR) */
#define HB_FRONTIER_OFF  3  /* recompute every node at every step */

typedef struct {
    uint32_t flags;      /* HB_* flags above */
    int32_t frontier;    /* HB_FRONTIER_* */
    int32_t max_steps;   /* iteration cap for hb_run_to_fixpoint; <= 0 means 1<<20 */
    void *stream;        /* cudaStream_t, or NULL */
    int32_t arcs_per_slot; /* class sizing of the gather from creation (as hb_set_class_sizing:
                              a power of two from 1 to 128), for callers who know it from an
                              earlier hb_tune; 0 = the default, 16.  Results never depend on it. */
    int32_t hot_nodes;   /* hot range of the gather from creation (as hb_set_hot_nodes),
                            for callers who know it from an earlier hb_tune; 0 = none.
                            Results never depend on it. */
    int32_t hot_passes;  /* how the hot range is used: 1 (or 0) one pass with L2
                            priorities, 2 the two-phase gather (as hb_set_hot_nodes) */
    double frontier_switch; /* HB_FRONTIER_AUTO's switch from creation (as
                               hb_set_frontier_switch); 0 = the default, 0.25.
                               Results never depend on it. */
} hb_options;

typedef struct hb_graph hb_graph;   /* opaque handle */

/* Per-handle counters, for measurement and tests. */
typedef struct {
    int64_t n, m;                /* nodes and arcs of the scanned graph */
    int32_t log2m;               /* b: p = 2^b registers per counter */
    int32_t t;                   /* iterations executed so far */
    int64_t last_changed;        /* nodes whose counter changed in the last iteration */
    int64_t last_nodes;          /* nodes recomputed in the last iteration */
    int64_t last_arcs;           /* arcs scanned in the last iteration (arc-updates) */
    int64_t total_arcs;          /* arcs scanned since the counters were initialised */
    int32_t last_sparse;         /* 1 if the last iteration used the changed-node frontier */
    int32_t converged;           /* 1 once an iteration changed nothing */
    int64_t device_bytes;        /* bytes of device memory the handle holds */
    int64_t launches;            /* kernels launched by the handle since its creation */
    int64_t kernel_launches;     /* HB_PROFILE: gather-kernel launches timed since the last reset */
    double kernel_ms;            /* HB_PROFILE: their summed duration (CUDA events, same stream) */
    double kernel_bytes;         /* HB_PROFILE: their summed algorithmic bytes (see below) */
    int64_t push_launches;       /* HB_PROFILE: pushed frontier iterations timed since the last reset */
    double push_ms;              /* HB_PROFILE: their summed duration (push + per-node tail) */
    double push_bytes;           /* HB_PROFILE: their summed algorithmic bytes (see below) */
    int32_t arcs_per_slot;       /* the gather's class sizing (hb_set_class_sizing, hb_tune) */
    int32_t hot_nodes;           /* hot range of the gather, 0 = none (hb_set_hot_nodes,
                                    hb_tune) */
    int32_t hot_passes;          /* 1: one pass with L2 priorities; 2: the two-phase gather */
    int32_t packed;              /* 1 if the counters are packed six bits per register */
    double frontier_switch;      /* HB_FRONTIER_AUTO pushes when the arcs to push are at most
                                    this fraction of m (hb_set_frontier_switch) */
} hb_info;

/* Algorithmic bytes of one gather-kernel launch, counted from the nodes it
 * recomputes (N), their arcs (A) and the nodes that changed (C):
 *     A * (4 + p)                 target index + successor counter per arc
 *   + N * (8 + 2p + 1)            offset, own counter read, counter write, flag
 *   + N * 4                       list entry (frontier iterations only)
 *   + C * (4 + 32 + 2e)           list append, sumd/harm read+write, cached
 *                                 estimate read+write (e = 8, or 4 in FP32)
 * and of one pushed frontier iteration, from the reverse arcs of the C'
 * nodes changed in the iteration before (P), the nodes recomputed (K) and
 * the nodes that changed (C):
 *     P * (4 + 2p)                predecessor index, its counter read+write
 *   + C' * (8 + p)                reverse offsets, the pushed counter
 *   + K * (5 + 3p)                list entry, pushed union, own counter,
 *                                 counter write, flag
 *   + C * (4 + 32 + 2e)           as above
 * In a pushed iteration last_arcs (the arc-updates) counts the P arcs.
 * With HB_PACKED_REGISTERS a counter read or write counts 3p/4 bytes. */

/* Fill *opt with the defaults: flags 0, HB_FRONTIER_AUTO, max_steps 1<<20,
 * stream NULL, arcs_per_slot 0. */
void hb_default_options(hb_options *opt);

/* Build a handle for the CSR graph (offsets: n+1 int64, targets: m int32)
 * and initialise every counter with add(c[v], v) (Sec. 4.2, Algorithm 2
 * first loop), v hashed by SplitMix64 seeded with `seed`; the register
 * index is the top log2m bits of the hash and the register value rho+ of
 * the remaining bits (Sec. 4.1, Algorithm 1), capped at 64-log2m.
 * log2m must lie in [4, 12] (p >= 16 as Sec. 4.1 assumes; 4096 is the
 * largest p of Sec. 8).  The graph is validated on the device; a malformed
 * graph gives HB_ERR_INVALID and no handle.  opt may be NULL (defaults).
 * With a frontier policy that pushes (AUTO, PUSH) and at least 2^20 arcs,
 * the reverse lists of the pushed frontier are still being built on a
 * second stream of the library's when this returns, under the first
 * iterations, which gather; calls on the handle order themselves after that
 * build where they need it (the first iteration that may push, the
 * two-phase gather's reordering, hb_destroy).  Borrowed inputs are read by
 * it too: they must stay unchanged until hb_destroy, as always. */
hb_status hb_create(const int64_t *offsets, const int32_t *targets, int64_t n, int64_t m,
                    int log2m, uint64_t seed, const hb_options *opt, hb_graph **out);

/* Same with int32 offsets (graphs with m < 2^31). */
hb_status hb_create32(const int32_t *offsets, const int32_t *targets, int64_t n, int64_t m,
                      int log2m, uint64_t seed, const hb_options *opt, hb_graph **out);

/* One iteration of Algorithm 2 at the current loop index t: every counter
 * becomes the register-wise max of itself and its successors' counters,
 * read from the previous iteration only (Jacobi, as the update file of
 * Sec. 4.2 implies).  For each node whose counter changed, with
 * d = size(new) - size(old) and the new layer at distance t+1:
 *     sumd[v] += (t+1) * d,   harm[v] += d / (t+1)          (Sec. 5)
 * *n_changed (may be NULL) receives the number of changed nodes.
 * Calling it after convergence is allowed and changes nothing. */
hb_status hb_step(hb_graph *g, int64_t *n_changed);

/* Iterate until an iteration changes no counter (Sec. 4.2), at most
 * max_steps iterations in total.  *steps (may be NULL) receives the number
 * of iterations executed since initialisation, the final unchanged one
 * included.  Returns HB_ERR_NOT_CONVERGED if the cap was reached first;
 * the state is then valid and more steps may follow. */
hb_status hb_run_to_fixpoint(hb_graph *g, int32_t *steps);

/* Sec. 3 centralities from the Sec. 5 accumulators, n doubles each, in the
 * caller's node order; any pointer may be NULL:
 *     reachable = size(c[v])   (coreachable set on the original graph, v included)
 *     closeness = 1/sumd[v], or 0 if sumd[v] == 0 (nothing else coreaches v)
 *     lin       = reachable^2 / sumd[v], or 1 if sumd[v] == 0
 *     harmonic  = harm[v] */
hb_status hb_get_centralities(hb_graph *g, double *closeness, double *harmonic,
                              double *lin, double *reachable);

/* The raw accumulators sumd and harm (n doubles each, may be NULL). */
hb_status hb_get_accumulators(hb_graph *g, double *sumd, double *harm);

/* The current counters, n*p bytes, row v = node v's p registers. */
hb_status hb_get_registers(hb_graph *g, uint8_t *out);

/* Frontier of the last iteration, n bytes each, may be NULL:
 * changed[v] = 1 if v's counter changed in it; must_check[v] = 1 if some
 * successor of v changed in it, i.e. v may change in the next iteration
 * (the modification tracking of Sec. 5 / 5.1). */
hb_status hb_get_frontier(hb_graph *g, uint8_t *changed, uint8_t *must_check);

/* Counters of the handle. */
hb_status hb_get_info(hb_graph *g, hb_info *info);

/* Re-initialise counters, accumulators and t (same graph, new seed). */
hb_status hb_reset(hb_graph *g, uint64_t seed);

/* Autotuner: choose how many lanes each light degree class of the gather
 * kernel gets (the class sizing: about *arcs_per_slot arcs per lane slot;
 * candidates the powers of two from 1 to 128) by timing the first eight
 * iterations (or all, if the fixpoint comes sooner) with each candidate,
 * twice (ascending, then descending order; the faster time counts).  Then,
 * with the same timing, the hot range of the gather (hb_set_hot_nodes),
 * tried when the handle holds one run per row and its counters exceed the
 * device's L2 cache: none, one pass with L2 priorities for hot counters of
 * 32, 64, 96 or 128 MiB with 1 and 2 times that sizing, or the two-phase
 * gather for 64, 128 or 192 MiB with 1, 2 and 4 times that sizing (each
 * pass gathers only part of every list).  Finally the counters are
 * re-initialised with the handle's seed.  Results never depend on any of
 * these choices.  *arcs_per_slot (may be NULL) receives the sizing;
 * hb_get_info reports all three.  The frontier switch
 * (hb_set_frontier_switch) is left as it is. */
hb_status hb_tune(hb_graph *g, int32_t *arcs_per_slot);

/* Set the class sizing directly (a power of two from 1 to 128) and
 * re-initialise. */
hb_status hb_set_class_sizing(hb_graph *g, int32_t arcs_per_slot);

/* The switch of HB_FRONTIER_AUTO (Sec. 5 / 5.1 modification tracking: how
 * the nodes to recompute are chosen, never what they compute).  After the
 * first iteration, an iteration pushes the counters that changed in the
 * one before along the reverse CSR when those counters' reverse arcs number
 * at most push_frac * m, and otherwise recomputes every node from all its
 * successors.  push_frac > 0 and finite (default 0.25; a value of 1 or more
 * pushes whenever the push touches no more arcs than a full scan).  Takes
 * effect from the next iteration; the counters are not re-initialised.
 * HB_ERR_INVALID for a value out of range. */
hb_status hb_set_frontier_switch(hb_graph *g, double push_frac);

/* The hot range of dense iterations' gather: the nodes [0, hot_nodes) of
 * the handle's internal order (clipped to n).  After the degree relabelling
 * the lowest ids are the nodes of highest out-degree, and, on graphs whose
 * in- and out-degrees go together (the R-MAT graphs here), also the most
 * gathered counters.  passes = 1: one pass that reads the hot counters with
 * the normal L2 eviction priority and every other counter with evict-first,
 * so that the cold counters, each read by one or two arcs per iteration,
 * leave L2 before the hot ones.  passes = 2: the two-phase gather, each
 * iteration reading its successors' counters in two launches, first the
 * arcs whose target is hot, then the others (with the library's own copy of
 * the targets every node's list is reordered hot targets first, once per
 * hot range; with borrowed targets each pass tests every arc), so that
 * while the first pass runs the random reads fall on hot_nodes * p bytes of
 * counters; it costs p bytes written and read per node.  The register-wise
 * maximum does not depend on the order or the cache policy of the reads, so
 * results are identical in every case.  hot_nodes = 0 (the default) uses no
 * hot range; handles of several runs per row take only 0 (HB_ERR_INVALID
 * otherwise).  Takes effect at the next iteration. */
hb_status hb_set_hot_nodes(hb_graph *g, int32_t hot_nodes, int32_t passes);

/* Node weights (Sec. 6).  The paper simulates an integer weight w(v) by
 * replicas: the ball of radius 0 around v holds w(v) distinct items, and
 * distinct nodes have disjoint replicas, so the growth of a counter between
 * iterations estimates the total weight of the new layer.  sumd, harm and
 * the discounted accumulator then estimate sum_y w(y) d(y,x),
 * sum_y w(y)/d(y,x) and sum_y w(y) f(d(y,x)), and reachable the weight of
 * the coreachable set (x included).
 *   weights: n integers in [0, 2^31), host or device, in the caller's node
 *   order, copied; NULL restores unit weights.  The replicas of node u are
 *   the items W_u .. W_u + w(u) - 1, W_u = w(0) + ... + w(u-1), hashed like
 *   node ids, so unit weights give exactly the unweighted counters.
 * The computation restarts from t = 0 with the handle's current seed.
 * Initialisation costs one hash per replica, w(u) of them in one thread.
 * HB_ERR_INVALID (handle unchanged) if a weight is out of range.
 * Single-graph handles, of one run or several (hb_create_runs: each run
 * hashes the replicas with its own seed); not the batched or served forms. */
hb_status hb_set_weights(hb_graph *g, const int64_t *weights);

/* Discount function (Sec. 7): a further per-node accumulator
 *     disc[v] = sum over iterations t of f(t+1) * (size(c_{t+1}[v]) - size(c_t[v]))
 * which estimates the discounted-gain centrality sum_{y != v} f(d(y,v)),
 * weighted by w(y) under hb_set_weights.  f(d) = f[d-1] for d = 1..len and
 * 0 for longer distances; f is host or device memory, copied.  len = 0 (f
 * may then be NULL) removes the accumulator.  The computation restarts from
 * t = 0 with the handle's current seed.  Single-graph handles, of one run
 * or several (one accumulator per run: hb_get_run_discounted). */
hb_status hb_set_discount(hb_graph *g, const double *f, int32_t len);

/* The discounted accumulator, n doubles in the caller's node order (host or
 * device).  HB_ERR_STATE if no discount is set or the handle holds several
 * runs (hb_get_run_discounted). */
hb_status hb_get_discounted(hb_graph *g, double *out);

/* The neighbourhood function (the aggregate that ANF and HyperANF compute
 * and that HyperBall generalises, Sec. 4): N(t) = sum over nodes x of
 * |B(x,t)|, the number of pairs (x,y) with y reachable from x along the
 * scanned arcs in at most t steps, estimated as the sum of size() over all
 * counters after t iterations (weighted under hb_set_weights).  Needs
 * HB_NEIGHBOURHOOD at creation: after initialisation and after every
 * iteration the library sums the nodes' cached estimates on the device in
 * a fixed order (one extra read of n estimates per iteration).
 * out[t] = N(t) for t = 0..T, T the iterations done, at most cap values
 * (host memory); *len (may be NULL) receives T+1.  N(T) - N(T-1) is the
 * number of pairs at distance T.  HB_ERR_STATE without the flag.
 * Single-graph handles only. */
hb_status hb_get_neighbourhood(hb_graph *g, double *out, int32_t cap, int32_t *len);

/* Several runs of one graph in one handle (Sec. 5: HyperBall repeated with
 * independent hash seeds, so that the spread of the estimates gives their
 * empirical standard deviation and their mean a tighter estimate).  Each
 * node's row holds `runs` counters of p = 2^log2m registers, run r in
 * bytes [r p, (r+1) p), hashed with seeds[r] (host or device memory, runs
 * entries).  The register-wise maximum never mixes bytes, so one union over
 * a row is every run's union: each iteration streams the graph once for all
 * runs and every gathered row is runs * p contiguous bytes.  An iteration
 * changes a node if any of its runs changes; the handle reaches its
 * fixpoint when every run has, and each run's counters, accumulators and
 * iteration count equal those of hb_create with its seed run alone.
 *   runs: a power of two from 2 to 64; log2m: 4..9; runs * p <= 4096.
 *   CSR and options as for hb_create, except HB_NEIGHBOURHOOD.
 * hb_step, hb_run_to_fixpoint, hb_reset (the seeds are kept; the argument
 * is ignored), hb_tune, hb_set_class_sizing, hb_get_frontier, hb_get_info
 * and hb_destroy work as for one run; hb_get_registers returns rows of
 * runs * p bytes.  hb_set_weights and hb_set_discount apply to every run.
 * Results come from the hb_get_run_* calls below; hb_get_centralities,
 * hb_get_accumulators, hb_get_discounted and checkpoints return
 * HB_ERR_STATE on such a handle.  Device memory: two rows of runs * p
 * bytes and about 20 * runs + 20 bytes per node (8 * runs more with a
 * discount). */
hb_status hb_create_runs(const int64_t *offsets, const int32_t *targets, int64_t n, int64_t m,
                         int log2m, int32_t runs, const uint64_t *seeds, const hb_options *opt,
                         hb_graph **out);

/* Per run r: its iteration count, the final unchanged iteration included
 * (steps[r] for every run; while a run is still changing, the iterations
 * executed so far). */
hb_status hb_get_run_steps(hb_graph *g, int32_t *steps);

/* Run r's Sec. 3 centralities and Sec. 5 accumulators, as
 * hb_get_centralities and hb_get_accumulators for one run. */
hb_status hb_get_run_centralities(hb_graph *g, int32_t run, double *closeness, double *harmonic,
                                  double *lin, double *reachable);
hb_status hb_get_run_accumulators(hb_graph *g, int32_t run, double *sumd, double *harm);
/* Run r's Sec. 7 discounted accumulator (n doubles, host or device);
 * HB_ERR_STATE without hb_set_discount. */
hb_status hb_get_run_discounted(hb_graph *g, int32_t run, double *out);

/* Per-node mean and empirical standard deviation (sample form, divisor
 * runs - 1) over the runs of one centrality (which = 0 closeness,
 * 1 harmonic, 2 Lin, 3 reachable, 4 the discounted accumulator), n
 * doubles each in the caller's order, host or device; either may be NULL.
 * which = 4 without hb_set_discount gives HB_ERR_STATE. */
hb_status hb_get_run_stats(hb_graph *g, int32_t which, double *mean, double *sd);

/* Checkpoint: write t, counters, last frontier and accumulators (and the
 * graph, the weights, the discount and the neighbourhood function) to a
 * file; hb_load rebuilds a handle that continues exactly where the saved
 * one stopped. */
hb_status hb_save(hb_graph *g, const char *path);
hb_status hb_load(const char *path, const hb_options *opt, hb_graph **out);

/* Free every resource of the handle (NULL is allowed). */
void hb_destroy(hb_graph *g);

/* Device memory (no counterpart in the paper: how the library holds its
 * buffers).  Handles take their device memory from a pool of the
 * library's own (one per device, stream-ordered on the handle's stream),
 * and what hb_destroy frees stays in that pool for later handles, so that
 * creating and destroying handles needs no device-wide synchronisation and
 * no new page mappings once the pool has grown (the way a caching
 * allocator keeps freed blocks).  hb_trim_memory returns every unused byte
 * of the library's pools to the device; memory of live handles is kept.
 * The process's default memory pool is not changed. */
hb_status hb_trim_memory(void);

/* The L2 fetch granularity of the calling process's CUDA context on the
 * current device (cudaLimitMaxL2FetchGranularity): 0 leaves it as it is
 * and only reports it; 32, 64 or 128 sets it.  *previous (may be NULL)
 * receives the value before the call.  The limit belongs to the process's
 * context: it applies to every kernel the process launches on that device
 * from then on and ends with the process; nothing outside the process
 * changes.  The random counter reads of the gather fetch whole lines on a
 * miss; on the graphs here 128 bytes measured 3-6% faster than 64 (the
 * degree relabelling puts counters that are read together next to each
 * other) and 32 bytes slower.  Results never depend on it.
 * HB_ERR_INVALID for any other value. */
hb_status hb_set_l2_fetch_bytes(int32_t bytes, int32_t *previous);

/* Message of the last failed call on this thread ("" if none). */
const char *hb_last_error(void);

/* Library version string. */
const char *hb_version(void);

/* ---- Batched form ------------------------------------------------------
 * Many independent HyperBall problems -- graphs of uneven size, each with
 * its own log2m and seed (the paper's repeated runs of Sec. 5 are one use:
 * the same graph with several seeds) -- advanced together.  Every kernel
 * of an iteration covers all graphs in one launch; the iteration is
 * captured into a CUDA graph, and hb_batch_run repeats it on the device
 * (conditional while node) until no graph is active, so a whole run is one
 * graph launch.  Each graph keeps its own loop index, frontier and
 * convergence; a graph that has converged costs nothing in later
 * iterations.  Results are those of the same graph run alone. */
typedef struct {
    const int64_t *offsets;   /* n+1 CSR offsets (host or device) */
    const int32_t *targets;   /* m CSR targets (host or device) */
    int64_t n, m;
    int32_t log2m;            /* 4..12 */
    uint64_t seed;            /* node-hash seed */
} hb_graph_desc;

typedef struct hb_batch hb_batch;

/* Create the batch (k in [1, 4096]); options as for hb_create (frontier
 * PULL is taken as AUTO; max_steps caps hb_batch_run).  With a NULL stream
 * the batch makes its own. */
hb_status hb_batch_create(int k, const hb_graph_desc *gs, const hb_options *opt, hb_batch **out);

/* Multiple runs (Sec. 5): the paper repeats HyperBall with independent
 * hash seeds to tighten its estimates and to measure their empirical
 * standard deviation.  This creates a batch of `runs` (1..4096) runs of
 * one graph (CSR as for hb_create, int64 offsets), run r with seed
 * seeds[r]: the graph is uploaded, validated and laid out once and every
 * run reads that one copy; each run owns only its counters, flags and
 * accumulators (2np + about 30n bytes).  Options as for hb_batch_create.
 * Run r's results equal those of hb_create(..., seeds[r], ...) run alone. */
hb_status hb_batch_create_runs(const int64_t *offsets, const int32_t *targets, int64_t n, int64_t m,
                               int log2m, int runs, const uint64_t *seeds, const hb_options *opt,
                               hb_batch **out);

/* Per-node mean and empirical standard deviation (sample form, divisor
 * k-1; 0 when k = 1) over the k graphs of a batch of one centrality of the
 * current state: which = 0 closeness, 1 harmonic, 2 Lin, 3 reachable
 * (Sec. 3, as hb_get_centralities).  n doubles each in the caller's node
 * order, host or device; either may be NULL.  Every graph of the batch
 * must have the same node count (HB_ERR_INVALID otherwise): a batch from
 * hb_batch_create_runs, or one graph passed k times. */
hb_status hb_batch_get_run_stats(hb_batch *b, int32_t which, double *mean, double *sd);

/* One iteration of every graph that has not converged; *n_active (may be
 * NULL) receives the number of graphs still changing afterwards. */
hb_status hb_batch_step(hb_batch *b, int32_t *n_active);

/* Iterate on the device until every graph has converged (or max_steps
 * batch iterations ran: HB_ERR_NOT_CONVERGED).  *iterations receives the
 * batch iterations executed since the last reset. */
hb_status hb_batch_run(hb_batch *b, int32_t *iterations);

/* Re-initialise every graph (seeds[i], or the previous seeds if NULL). */
hb_status hb_batch_reset(hb_batch *b, const uint64_t *seeds);

/* Per-graph results and counters, as the single-graph getters. */
hb_status hb_batch_get_centralities(hb_batch *b, int i, double *closeness, double *harmonic,
                                    double *lin, double *reachable);
hb_status hb_batch_get_registers(hb_batch *b, int i, uint8_t *out);
hb_status hb_batch_get_accumulators(hb_batch *b, int i, double *sumd, double *harm);
hb_status hb_batch_get_info(hb_batch *b, int i, hb_info *info);

/* Autotuner of the batch: as hb_tune, timing whole batched iterations;
 * every graph is re-initialised afterwards. */
hb_status hb_batch_tune(hb_batch *b, int32_t *arcs_per_slot);

/* Batch iterations since the last reset, graphs still active, and arcs
 * scanned by all graphs (arc-updates). */
hb_status hb_batch_get_totals(hb_batch *b, int32_t *iterations, int32_t *n_active, int64_t *arcs);

void hb_batch_destroy(hb_batch *b);

/* ---- Serving form ------------------------------------------------------
 * A request loop for centrality jobs (graph from a device-resident pool,
 * log2m, seed) with continuous batching: a server thread keeps up to
 * `slots` requests on the device at once, their counters resident between
 * iterations, and advances all of them in the same batched launches.
 * Between iterations it admits queued requests (FIFO) into free slots
 * while the device has run_bytes + reserve_bytes free, and finalises
 * requests whose counters stopped changing: results are copied to host
 * memory and the request's device memory is freed.  A request's result is
 * the same as the same (graph, log2m, seed) run alone. */
#define HB_REQ_QUEUED  0
#define HB_REQ_RUNNING 1
#define HB_REQ_DONE    2
#define HB_REQ_FAILED  3
#define HB_REQ_CANCELLED 4

typedef struct {
    int32_t slots;            /* requests on the device at once, 1..4096 (1 = FIFO one at a time) */
    uint32_t flags;           /* HB_FP32_ESTIMATE or 0 */
    int32_t max_steps;        /* per-request iteration cap */
    int64_t reserve_bytes;    /* device memory left free when admitting */
    int64_t large_arcs;       /* a request on a graph of at least this many arcs is "large" */
    int32_t large_slots;      /* large requests running at once, at most (0: no limit).  With a
                                 limit, a large request at the head of the queue waits for a
                                 large slot while the small requests behind it are admitted, so
                                 large requests share the device only with small ones (they are
                                 served first come, first served among themselves) and small
                                 requests never queue behind a large one */
} hb_server_options;

typedef struct {
    int32_t state;            /* HB_REQ_* */
    int32_t steps;            /* iterations to the fixpoint */
    int64_t arcs;             /* arc-updates of the request */
    double submit_s, admit_s, done_s;   /* server clock (seconds since creation) */
} hb_request_info;

typedef struct hb_server hb_server;

void hb_server_default_options(hb_server_options *opt);   /* 32 slots, 4 GiB reserve, no large limit */
hb_status hb_server_create(const hb_server_options *opt, hb_server **out);
/* Add a graph to the pool (CSR copied to the device once) and prepare it
 * for each log2m listed (relabelling, reverse CSR, plans shared by all its
 * requests).  *graph_id receives its id. */
hb_status hb_server_add_graph(hb_server *s, const int64_t *offsets, const int32_t *targets, int64_t n,
                              int64_t m, const int32_t *log2ms, int n_log2m, int32_t *graph_id);
/* Queue a request; returns at once with its id. */
hb_status hb_server_submit(hb_server *s, int32_t graph_id, int32_t log2m, uint64_t seed,
                           int64_t *request_id);
/* Wait until the request is done (timeout_s < 0: no limit; HB_ERR_TIMEOUT
 * if it ran out).  info may be NULL.  A failed request returns its error:
 * HB_ERR_OOM when it was refused (its device memory plus reserve_bytes
 * exceeds the device, or it does not fit while none of the server's
 * requests is running); a cancelled one returns HB_ERR_STATE with
 * info->state = HB_REQ_CANCELLED. */
hb_status hb_server_wait(hb_server *s, int64_t request_id, double timeout_s, hb_request_info *info);
/* Cancel a request: a queued one leaves the queue at once; a running one is
 * retired at the next iteration boundary (its slot and device memory are
 * freed, the other requests are untouched).  HB_ERR_STATE if it has
 * already finished. */
hb_status hb_server_cancel(hb_server *s, int64_t request_id);
/* Copy a finished request's centralities (n doubles each, host memory, any
 * may be NULL) and forget the request; a failed or cancelled request is
 * forgotten with HB_ERR_STATE. */
hb_status hb_server_take(hb_server *s, int64_t request_id, double *closeness, double *harmonic,
                         double *lin, double *reachable);
/* Completed requests, batched iterations, arc-updates, seconds with work on
 * the device, and the server clock. */
hb_status hb_server_stats(hb_server *s, int64_t *completed, int64_t *iterations, int64_t *arcs,
                          double *busy_s, double *clock_s);
void hb_server_destroy(hb_server *s);

/* ---- One iteration without device allocation -------------------------
 * The paper has no counterpart to this call.  It exists for callers that
 * cannot call cudaMalloc: code running inside another framework's memory
 * pool or arena, where an allocation outside the pool breaks its
 * accounting or is not allowed; services that freeze allocation after
 * start-up so that no request can stall in, or fail on, the allocator; and
 * hosts that hand the library device buffers but no allocator.
 *
 * hb_step_noalloc runs one iteration at loop index t on the CSR graph
 * (offsets: n+1 int64, targets: m int32), in the caller's node order: every
 * node's new counter is the register-wise maximum of its own counter in
 * `cur` (n*p bytes) and the counters of its successors, written to `next`
 * (all n*p bytes).  `changed` (n bytes) receives 1 for every node whose
 * counter grew, and for those nodes sumd[v] += (t+1)*d and harm[v] +=
 * d/(t+1) (n doubles each, updated in place), d being the growth of the
 * counter's FP64 size estimate; other nodes keep sumd and harm.  This is
 * the iteration hb_step runs on a handle.  *n_changed (host memory, may be
 * NULL) receives the number of changed nodes.  Every pointer but n_changed
 * must be device memory; stream may be NULL.  Each call synchronises
 * `stream` (it reads sizes and the changed count back to the host) and
 * returns once every output is written.
 *
 * Checks, each answered with HB_ERR_INVALID before any kernel reads a
 * counter: log2m in [4, 12]; the CSR is well formed (offsets[0] = 0,
 * offsets[n] = m, offsets never decrease, every target in [0, n)); and
 * next, sumd, harm and changed share no byte with each other nor with
 * offsets, targets or cur (in particular next may not be cur).  A failed
 * device-side check during the iteration (the debug build's arc-target
 * check) returns HB_ERR_STATE with the same message as hb_step.
 *
 * It allocates nothing: its temporary data (degree lists, work plan,
 * partial counters of split nodes, cached estimates, counters) lives in
 * one static device array of HB_NOALLOC_SCRATCH_BYTES that every GPU which
 * loads the library holds until the process exits.  A graph whose
 * temporary data does not fit (about 12 bytes per node plus p bytes per
 * 64*(32/L) arcs of nodes above the split threshold) is rejected with
 * HB_ERR_INVALID and a message giving the size it needs.  All calls share
 * the array and it keeps the last call's contents (everything that must
 * start at zero is cleared by each call); calls that overlap on the GPU
 * (two streams, or two threads) race on it and must be serialised by the
 * caller.  The first call on a device looks up the array's device address
 * on that device (cudaGetSymbolAddress, with that device current); make
 * that first call before any stream capture. */
#define HB_NOALLOC_SCRATCH_BYTES (64u << 20)
hb_status hb_step_noalloc(const int64_t *offsets, const int32_t *targets, int64_t n, int64_t m,
                          int log2m, int32_t t, const uint8_t *cur, uint8_t *next, double *sumd,
                          double *harm, uint8_t *changed, int64_t *n_changed, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* HYPERBALL_H */

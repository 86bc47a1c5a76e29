/*
 * hb_oracle.c -- plain CPU HyperBall, the parity oracle.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library
 * and its Python binding) may load or call this file; only the tests, the
 * package's smoke entry and the CPU-baseline leg of the benchmark do.  It
 * shares no code, header, table or constant generator with the CUDA path.
 *
 * It follows Boldi & Vigna, "In-Core Computation of Geometric Centralities
 * with HyperBall" (arXiv:1308.2144):
 *   - Algorithm 1 (Sec. 4.1): the HyperLogLog counter, add() and size();
 *   - Algorithm 2 (Sec. 4.2): the HyperBall loop with Jacobi updates
 *     (new counters are applied only after the whole scan);
 *   - Sec. 5: the three per-node accumulators (sum of distances, sum of
 *     reciprocal distances, coreachable-set size);
 *   - Sec. 3: closeness, Lin and harmonic centrality from them;
 *   - Sec. 6: integer node weights simulated by replicas at initialisation;
 *   - Sec. 7: a discounted accumulator sum_t f(t) * (new layer at t).
 * Everything is written as plain loops in the paper's order, in double
 * precision, compiled with -ffp-contract=off so that every floating-point
 * operation rounds once, as written.
 *
 * Readings of points the paper leaves open (each is a choice, not a quote):
 *   - hash h: SplitMix64 (Steele, Lea & Flood 2014); h(v) is output number
 *     v+1 of a generator whose state starts at `seed`;
 *   - index h_b(x) = the top b bits of the 64-bit word; rho+ counts leading
 *     zeros of the remaining 64-b bits, plus one, capped at 64-b (the cap
 *     only bites when all 64-b bits are zero) so that every register term
 *     2^(64-b-M) of the fixed-point sum is an integer;
 *   - registers start at 0, standing for -infinity (every rho+ is >= 1);
 *   - alpha_p and the small-range estimator are those of Flajolet et al.
 *     (2007), which Sec. 4.1 defers to: linear counting p*ln(p/V) when the
 *     raw estimate is <= 5p/2 and V (zero registers) > 0;
 *   - at loop index t the scanned counter a estimates |B(v,t+1)| and c[v]
 *     estimates |B(v,t)|, so the new layer sits at distance t+1;
 *   - steps counts every executed iteration, including the last one, in
 *     which no counter changed;
 *   - replicas (Sec. 6): the replicas of node v are the items numbered
 *     W_v, W_v+1, ..., W_v+w(v)-1 with W_v = w(0)+...+w(v-1), hashed like
 *     node ids, so distinct nodes have disjoint replicas and unit weights
 *     give back the unweighted counters exactly; a weight of 0 (outside the
 *     paper's 1..W) leaves the node's own counter empty;
 *   - discount (Sec. 7): f is given as a table, f(d) = table[d-1] for
 *     d = 1..len and 0 for longer distances;
 *   - packed registers (Sec. 4.1, register width): six bits per register,
 *     register j at bits 6j .. 6j+5 of the counter's bit string, least
 *     significant bit first; every register value (<= 64-b) fits, so the
 *     packed counters are the unpacked ones exactly.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---------------------------------------------------------------- hash -- */

/* SplitMix64, written from its published definition: a Weyl sequence with
 * increment 0x9E3779B97F4A7C15 followed by two xor-shift-multiply rounds.
 * h(v) is output number v+1 of the generator seeded with `seed`. */
uint64_t orc_hash(uint64_t seed, uint64_t v)
{
    uint64_t z = seed + (v + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Sec. 4.1: h_b(x) = leftmost b bits (register index); rho+ of the remaining
 * 64-b bits = number of leading zeros plus one, counted one bit at a time
 * and capped at 64-b. */
void orc_hash_split(uint64_t x, int b, uint32_t *index, uint32_t *rho)
{
    *index = (uint32_t)(x >> (64 - b));
    uint32_t zeros = 0;
    for (int bit = 63 - b; bit >= 0; --bit) {   /* remaining bits, leftmost first */
        if ((x >> bit) & 1ULL) break;
        zeros++;
    }
    uint32_t r = zeros + 1;
    if (r > (uint32_t)(64 - b)) r = (uint32_t)(64 - b);
    *rho = r;
}

/* ------------------------------------------------------- HLL counter -- */

/* alpha_p from Flajolet, Fusy, Gandouet & Meunier (2007), Fig. 3. */
double orc_alpha(int p)
{
    if (p == 16) return 0.673;
    if (p == 32) return 0.697;
    if (p == 64) return 0.709;
    return 0.7213 / (1.0 + 1.079 / (double)p);
}

/* Algorithm 1, add(M, x) for an item whose 64-bit hash is x. */
void orc_add(uint8_t *M, int b, uint64_t x)
{
    uint32_t i, r;
    orc_hash_split(x, b, &i, &r);
    if (M[i] < r) M[i] = (uint8_t)r;
}

/* Algorithm 1, feeding a whole stream of hashed items into one counter. */
void orc_add_stream(uint8_t *M, int b, const uint64_t *x, int64_t count)
{
    for (int64_t k = 0; k < count; ++k) orc_add(M, b, x[k]);
}

/* The inner sum of size(): sum over registers of 2^-M[j].  Registers equal
 * to 0 (-infinity in the paper, i.e. empty) contribute 2^0 = 1 as in
 * Flajolet et al.; the others are added exactly as integers scaled by
 * 2^(64-b) and converted to double once. */
double orc_register_sum(const uint8_t *M, int b, int *zeros_out)
{
    int p = 1 << b;
    int V = 0;
    uint64_t S = 0;
    for (int j = 0; j < p; ++j) {
        if (M[j] == 0) V++;
        else S += (uint64_t)1 << (64 - b - M[j]);
    }
    if (zeros_out) *zeros_out = V;
    return (double)V + ldexp((double)S, b - 64);
}

/* Algorithm 1, size(M): E = alpha_p p^2 / sum, with the small-range
 * (linear counting) estimator that Sec. 5.2 mentions but does not show. */
double orc_size(const uint8_t *M, int b)
{
    int p = 1 << b;
    int V;
    double sum = orc_register_sum(M, b, &V);
    double E = orc_alpha(p) * (double)p * (double)p / sum;
    if (E <= 2.5 * (double)p && V > 0)
        E = (double)p * log((double)p / (double)V);
    return E;
}

/* ------------------------------------------------ packed registers -- */

/* Sec. 4.1: a register needs only about log2 log2 n bits.  With the 64-bit
 * hash, rho+ never exceeds 64-b <= 60 < 2^6, so six bits hold every
 * register exactly (no clamping).  The packed counter is the bit string of
 * 6p bits in which register j occupies bits 6j .. 6j+5 (least significant
 * bit first), stored in 3p/4 bytes, bit i in bit i%8 of byte i/8.
 * Returns -1, writing nothing useful, if a register does not fit. */
int orc_pack6(const uint8_t *M, int b, uint8_t *out)
{
    int p = 1 << b;
    memset(out, 0, (size_t)(3 * p / 4));
    for (int j = 0; j < p; ++j) {
        if (M[j] > 63) return -1;
        for (int bit = 0; bit < 6; ++bit)
            if ((M[j] >> bit) & 1) {
                int i = 6 * j + bit;
                out[i / 8] |= (uint8_t)(1u << (i % 8));
            }
    }
    return 0;
}

/* The inverse of orc_pack6: register j from bits 6j .. 6j+5. */
void orc_unpack6(const uint8_t *in, int b, uint8_t *M)
{
    int p = 1 << b;
    for (int j = 0; j < p; ++j) {
        uint8_t v = 0;
        for (int bit = 0; bit < 6; ++bit) {
            int i = 6 * j + bit;
            v |= (uint8_t)(((in[i / 8] >> (i % 8)) & 1) << bit);
        }
        M[j] = v;
    }
}

/* ----------------------------------------------------------- HyperBall -- */

static int g_threads = 0;

void orc_set_threads(int k) { g_threads = k; }

int orc_get_threads(void)
{
#ifdef _OPENMP
    return g_threads > 0 ? g_threads : omp_get_max_threads();
#else
    return 1;
#endif
}

/* Algorithm 2, initial loop: add(c[v], v) into empty counters. */
void orc_init(int64_t n, int b, uint64_t seed, uint8_t *c)
{
    int64_t p = (int64_t)1 << b;
    memset(c, 0, (size_t)(n * p));
    for (int64_t v = 0; v < n; ++v)
        orc_add(c + v * p, b, orc_hash(seed, (uint64_t)v));
}

/* Sec. 6: the weighted ball of radius 0 is the set of v's replicas, so
 * the initial counter of v receives add() of each of its w(v) replica
 * items.  Replica items are numbered consecutively across nodes in node
 * order (first item of v = sum of the weights of the nodes before it). */
void orc_init_weighted(int64_t n, int b, uint64_t seed, const int64_t *w, uint8_t *c)
{
    int64_t p = (int64_t)1 << b;
    memset(c, 0, (size_t)(n * p));
    uint64_t first = 0;
    for (int64_t v = 0; v < n; ++v) {
        for (int64_t k = 0; k < w[v]; ++k)
            orc_add(c + v * p, b, orc_hash(seed, first + (uint64_t)k));
        first += (uint64_t)w[v];
    }
}

/* Sec. 5 (and Sec. 7): node v's counter grew by delta (in size) at loop
 * index t, so delta nodes sit at distance t+1. */
static void accumulate(int64_t v, int32_t t, double delta, double *sumd, double *harm,
                       double fdist, double *disc)
{
    double dist = (double)(t + 1);
    sumd[v] = sumd[v] + dist * delta;
    harm[v] = harm[v] + delta / dist;
    if (disc) disc[v] = disc[v] + fdist * delta;
}

/* One iteration of the do/until loop of Algorithm 2 at loop index t.
 * Reads only `cur` (c_t) and writes `next` (c_{t+1}): the update file of
 * the paper is applied after the whole scan.  For every node whose counter
 * changed, the Sec. 5 accumulators receive the new layer at distance t+1:
 *     sumd[v] += (t+1) * (size(a) - size(c[v]))
 *     harm[v] += (size(a) - size(c[v])) / (t+1)
 * and, if disc is not NULL, the Sec. 7 discounted accumulator with the
 * discount fdist = f(t+1) of the new layer's distance:
 *     disc[v] += f(t+1) * (size(a) - size(c[v]))
 * changed[v] is 1 when a differs from c[v].  Returns the number of changed
 * nodes.  Nodes are independent, so the parallel loop gives the same
 * result for any thread count. */
int64_t orc_step_ex(int64_t n, const int64_t *offsets, const int32_t *targets,
                    int b, int32_t t, const uint8_t *cur, uint8_t *next,
                    double *sumd, double *harm, double fdist, double *disc,
                    uint8_t *changed)
{
    int64_t p = (int64_t)1 << b;
    int64_t n_changed = 0;
#ifdef _OPENMP
    int nt = orc_get_threads();
#pragma omp parallel for schedule(dynamic, 1024) reduction(+ : n_changed) num_threads(nt)
#endif
    for (int64_t v = 0; v < n; ++v) {
        uint8_t a[4096];
        memcpy(a, cur + v * p, (size_t)p);                  /* a <- c[v] */
        for (int64_t e = offsets[v]; e < offsets[v + 1]; ++e) {
            const uint8_t *cw = cur + (int64_t)targets[e] * p;
            for (int64_t i = 0; i < p; ++i)                  /* a <- union(c[w], a) */
                if (cw[i] > a[i]) a[i] = cw[i];
        }
        int ch = memcmp(a, cur + v * p, (size_t)p) != 0;
        changed[v] = (uint8_t)ch;
        if (ch) {
            double delta = orc_size(a, b) - orc_size(cur + v * p, b);
            accumulate(v, t, delta, sumd, harm, fdist, disc);
            n_changed += 1;
        }
        memcpy(next + v * p, a, (size_t)p);                  /* write <v, a> */
    }
    return n_changed;
}

/* One iteration of Algorithm 2 on packed counters (orc_pack6 rows of
 * 3p/4 bytes): each counter is unpacked where it is read, the union and
 * the Sec. 5 accumulators are those of orc_step_ex, and the new counter is
 * packed again.  Returns the number of changed nodes, or -1 if a register
 * did not fit six bits. */
int64_t orc_step_packed(int64_t n, const int64_t *offsets, const int32_t *targets,
                        int b, int32_t t, const uint8_t *cur, uint8_t *next,
                        double *sumd, double *harm, uint8_t *changed)
{
    int64_t p = (int64_t)1 << b;
    int64_t row = 3 * p / 4;
    int64_t n_changed = 0;
    int bad = 0;
#ifdef _OPENMP
    int nt = orc_get_threads();
#pragma omp parallel for schedule(dynamic, 1024) reduction(+ : n_changed) reduction(| : bad) num_threads(nt)
#endif
    for (int64_t v = 0; v < n; ++v) {
        uint8_t own[4096], a[4096], cw[4096];
        orc_unpack6(cur + v * row, b, own);                  /* c[v] */
        memcpy(a, own, (size_t)p);                           /* a <- c[v] */
        for (int64_t e = offsets[v]; e < offsets[v + 1]; ++e) {
            orc_unpack6(cur + (int64_t)targets[e] * row, b, cw);
            for (int64_t i = 0; i < p; ++i)                  /* a <- union(c[w], a) */
                if (cw[i] > a[i]) a[i] = cw[i];
        }
        int ch = memcmp(a, own, (size_t)p) != 0;
        changed[v] = (uint8_t)ch;
        if (ch) {
            double delta = orc_size(a, b) - orc_size(own, b);
            accumulate(v, t, delta, sumd, harm, 0.0, NULL);
            n_changed += 1;
        }
        if (orc_pack6(a, b, next + v * row) != 0) bad = 1;  /* write <v, a> */
    }
    return bad ? -1 : n_changed;
}

/* The unweighted, undiscounted iteration. */
int64_t orc_step(int64_t n, const int64_t *offsets, const int32_t *targets,
                 int b, int32_t t, const uint8_t *cur, uint8_t *next,
                 double *sumd, double *harm, uint8_t *changed)
{
    return orc_step_ex(n, offsets, targets, b, t, cur, next, sumd, harm, 0.0, NULL, changed);
}

/* f(d) of a discount table (Sec. 7): table[d-1] for 1 <= d <= len, else 0. */
double orc_discount(const double *table, int32_t len, int64_t d)
{
    return (d >= 1 && d <= len) ? table[d - 1] : 0.0;
}

/* The whole of Algorithm 2: init, then iterate until an iteration leaves
 * every counter unchanged, or max_steps iterations ran.  On return `c`
 * holds the final counters, *steps the number of iterations executed
 * (including the final unchanged one).  If changed_hist is not NULL it
 * receives, for each executed iteration s, the changed set in row s
 * (capacity max_steps * n bytes).  weights (Sec. 6) may be NULL (every
 * node weighs 1); disc (Sec. 7, discount table ftable of flen entries) may
 * be NULL.  Returns 0 on convergence, 1 if max_steps ran out first, -1 on
 * allocation failure. */
int orc_run_ex(int64_t n, const int64_t *offsets, const int32_t *targets,
               int b, uint64_t seed, const int64_t *weights,
               const double *ftable, int32_t flen, int32_t max_steps,
               uint8_t *c, double *sumd, double *harm, double *disc,
               int32_t *steps, uint8_t *changed_hist)
{
    int64_t p = (int64_t)1 << b;
    uint8_t *other = (uint8_t *)malloc((size_t)(n * p > 0 ? n * p : 1));
    uint8_t *changed = (uint8_t *)malloc((size_t)(n > 0 ? n : 1));
    if (!other || !changed) { free(other); free(changed); return -1; }
    if (weights) orc_init_weighted(n, b, seed, weights, c);
    else orc_init(n, b, seed, c);
    for (int64_t v = 0; v < n; ++v) {
        sumd[v] = 0.0;
        harm[v] = 0.0;
        if (disc) disc[v] = 0.0;
    }
    uint8_t *cur = c, *nxt = other;
    int32_t t = 0;
    int converged = 0;
    while (t < max_steps) {
        double fdist = disc ? orc_discount(ftable, flen, (int64_t)t + 1) : 0.0;
        int64_t k = orc_step_ex(n, offsets, targets, b, t, cur, nxt, sumd, harm, fdist, disc,
                                changed);
        if (changed_hist) memcpy(changed_hist + (int64_t)t * n, changed, (size_t)n);
        uint8_t *tmp = cur; cur = nxt; nxt = tmp;
        t += 1;
        if (k == 0) { converged = 1; break; }
    }
    if (cur != c) memcpy(c, cur, (size_t)(n * p));
    *steps = t;
    free(other);
    free(changed);
    return converged ? 0 : 1;
}

int orc_run(int64_t n, const int64_t *offsets, const int32_t *targets,
            int b, uint64_t seed, int32_t max_steps,
            uint8_t *c, double *sumd, double *harm, int32_t *steps,
            uint8_t *changed_hist)
{
    return orc_run_ex(n, offsets, targets, b, seed, NULL, NULL, 0, max_steps, c, sumd, harm,
                      NULL, steps, changed_hist);
}

/* The neighbourhood function at t (Sec. 4: the single value per iteration
 * that ANF and HyperANF aggregate, N(t) = sum over x of |B(x,t)|),
 * estimated by adding size() of every counter c_t[v] in node order. */
double orc_neighbourhood(int64_t n, int b, const uint8_t *c)
{
    int64_t p = (int64_t)1 << b;
    double N = 0.0;
    for (int64_t v = 0; v < n; ++v) N = N + orc_size(c + v * p, b);
    return N;
}

/* Sec. 3 from the Sec. 5 accumulators:
 *   reachable = size(c[v])              (coreachable set, x included)
 *   closeness = 1 / sumd                (0 when no other node coreaches x)
 *   lin       = reachable^2 / sumd      (1 when no other node coreaches x)
 *   harmonic  = harm
 * "No other node coreaches x" is read as sumd == 0 (sumd > 0 otherwise). */
void orc_finalize(int64_t n, int b, const uint8_t *c, const double *sumd,
                  const double *harm, double *closeness, double *harmonic,
                  double *lin, double *reachable)
{
    int64_t p = (int64_t)1 << b;
    for (int64_t v = 0; v < n; ++v) {
        double r = orc_size(c + v * p, b);
        double s = sumd[v];
        if (reachable) reachable[v] = r;
        if (closeness) closeness[v] = s > 0.0 ? 1.0 / s : 0.0;
        if (lin) lin[v] = s > 0.0 ? r * r / s : 1.0;
        if (harmonic) harmonic[v] = harm[v];
    }
}

/* Sec. 5 / 5.1 modification tracking, by definition: after an iteration
 * whose changed set is `changed`, node v can change in the next iteration
 * only if some successor w (v -> w) changed.  must[v] = 1 for those. */
void orc_must_check(int64_t n, const int64_t *offsets, const int32_t *targets,
                    const uint8_t *changed, uint8_t *must)
{
    for (int64_t v = 0; v < n; ++v) {
        uint8_t m = 0;
        for (int64_t e = offsets[v]; e < offsets[v + 1]; ++e)
            if (changed[targets[e]]) { m = 1; break; }
        must[v] = m;
    }
}

/* ---------------------------------------------------- exact centralities -- */

/* Exact Sec. 3 ingredients by one breadth-first visit per node of the
 * scanned graph S: for x, dist(x,y) along S's arcs equals d(y,x) in the
 * original graph when S is its transpose.  Outputs, per x:
 *   sumd  = sum of finite distances, harm = sum over y != x of 1/distance,
 *   reach = number of nodes at finite distance (x included),
 *   ecc   = largest finite distance. */
int orc_exact_centralities(int64_t n, const int64_t *offsets, const int32_t *targets,
                           const int64_t *sources, int64_t n_sources,
                           double *sumd, double *harm, double *reach, int32_t *ecc)
{
#ifdef _OPENMP
    int nt = orc_get_threads();
#endif
    int fail = 0;
#ifdef _OPENMP
#pragma omp parallel num_threads(nt) reduction(| : fail)
#endif
    {
        int32_t *dist = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
        int64_t *queue = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
        int ok = dist != NULL && queue != NULL;
        if (!ok) fail = 1;
        if (ok)
            for (int64_t v = 0; v < n; ++v) dist[v] = -1;
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 16)
#endif
        for (int64_t k = 0; k < n_sources; ++k) {
            if (!ok) continue;
            int64_t x = sources ? sources[k] : k;
            int64_t head = 0, tail = 0;
            dist[x] = 0;
            queue[tail++] = x;
            double s = 0.0, h = 0.0;
            int32_t e_max = 0;
            while (head < tail) {
                int64_t u = queue[head++];
                int32_t du = dist[u];
                if (du > 0) { s += (double)du; h += 1.0 / (double)du; }
                if (du > e_max) e_max = du;
                for (int64_t e = offsets[u]; e < offsets[u + 1]; ++e) {
                    int64_t w = targets[e];
                    if (dist[w] < 0) { dist[w] = du + 1; queue[tail++] = w; }
                }
            }
            sumd[k] = s;
            harm[k] = h;
            reach[k] = (double)tail;
            if (ecc) ecc[k] = e_max;
            for (int64_t q = 0; q < tail; ++q) dist[queue[q]] = -1;
        }
        free(dist);
        free(queue);
    }
    return fail ? -1 : 0;
}

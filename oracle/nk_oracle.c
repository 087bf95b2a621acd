/*
 * Sequential CPU oracle for betweenness centrality on unweighted undirected graphs.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call this
 * file: only tests/, __graft_entry__.smoke() and the cpu_baseline leg of bench.py use
 * it.  It shares no code, header, table or constant generator with the CUDA library.
 *
 * It is written for clarity, not speed, and follows the paper (NetworKit, Staudt,
 * Sazonovs and Meyerhenke):
 *   - Brandes' algorithm [Bra01] for exact betweenness, Section 3.2 and Table 1
 *     ("betweenness", O(nm) time, O(n+m) space): one single-source shortest-path
 *     search per source (BFS, because the graph is unweighted, Section 3.4) that
 *     counts shortest paths sigma, then a dependency accumulation in reverse BFS
 *     order; the dependencies of all sources are summed (Section 3.2).
 *   - The source-sampled estimate (Section 3.2, citing Geisberger et al.): the same
 *     per-source work for k randomly chosen sources, scaled by n/k.
 *   - The graph generators of Section 5, Table 2 (Erdos-Renyi via Batagelj-Brandes skipping,
 *     Barabasi-Albert via the Batagelj-Brandes edge array, R-MAT).
 *
 * Readings where the paper is silent (each is listed in the design notes):
 *   - betweenness counts unordered pairs {s,t}, endpoints excluded, unreachable pairs
 *     contribute 0, no normalisation: the sum over all sources is halved;
 *   - sampled scores are (n/k) * (1/2) * sum_{s in S} delta_s;
 *   - sigma is uint64; an overflow is an error (OR_ERR_OVERFLOW), never a wrap;
 *   - random numbers come from SplitMix64 (Steele, Lea and Flood, OOPSLA 2014) used as
 *     a counter-based generator: the i-th output of the stream seeded with `seed` is
 *     mix64(seed + (i+1) * 0x9E3779B97F4A7C15);
 *   - a uniform integer in [0,b) is floor(x*b / 2^64) (Lemire's multiply-high, no
 *     rejection); a uniform double in [0,1) is (x >> 11) * 2^-53.
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared (contraction off so that the ER
 * generator's floating-point steps are the same IEEE operations on every host).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define OR_OK 0
#define OR_ERR_ARG (-1)
#define OR_ERR_GRAPH (-2)
#define OR_ERR_NOMEM (-3)
#define OR_ERR_OVERFLOW (-4)

/* ------------------------------------------------------------------------------ */
/* SplitMix64 (Steele, Lea, Flood 2014): golden-ratio increment and the 64-bit     */
/* finaliser with the published multipliers.                                       */
/* ------------------------------------------------------------------------------ */

uint64_t or_mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* i-th output (i = 0, 1, ...) of the SplitMix64 stream seeded with `seed`. */
uint64_t or_stream(uint64_t seed, uint64_t i)
{
    return or_mix64(seed + (i + 1) * 0x9E3779B97F4A7C15ULL);
}

static uint64_t or_below(uint64_t x, uint64_t b) /* floor(x*b / 2^64) */
{
    return (uint64_t)(((unsigned __int128)x * (unsigned __int128)b) >> 64);
}

static double or_unit(uint64_t x) /* (x >> 11) * 2^-53, in [0,1) */
{
    return (double)(x >> 11) * (1.0 / 9007199254740992.0);
}

/* Natural logarithm for 0 < x <= 1 (normal x), from the series
 *   ln z = 2 * atanh((z-1)/(z+1)) = 2 * sum_k s^(2k+1) / (2k+1),  s = (z-1)/(z+1),
 * after writing x = m * 2^e with m in (sqrt(1/2), sqrt(2)].  Used only by the ER
 * generator, whose skip lengths must be the same on every machine: each step is one
 * IEEE-754 double operation in a fixed order. */
double or_log(double x)
{
    uint64_t bits;
    memcpy(&bits, &x, sizeof bits);
    int e = (int)((bits >> 52) & 0x7FF) - 1023;
    uint64_t mbits = (bits & 0x000FFFFFFFFFFFFFULL) | 0x3FF0000000000000ULL;
    double m;
    memcpy(&m, &mbits, sizeof m);
    if (m > 1.4142135623730951) { /* sqrt(2) rounded */
        m = m * 0.5;
        e = e + 1;
    }
    double s = (m - 1.0) / (m + 1.0);
    double s2 = s * s;
    double p = 1.0 / 25.0;
    for (int k = 11; k >= 0; --k)
        p = p * s2 + 1.0 / (double)(2 * k + 1);
    double r = 2.0 * s;
    r = r * p;
    return r + (double)e * 0.6931471805599453;
}

/* ------------------------------------------------------------------------------ */
/* Generators (Section 5, Table 2).  Each returns the number of generated (raw) edges, writes  */
/* at most `cap` of them, and leaves self-loops and duplicates for the CSR builder. */
/* ------------------------------------------------------------------------------ */

#define OR_ER_CHUNK (1ULL << 20)

/* pair index t = u(u-1)/2 + v, u > v >= 0  ->  (u, v) */
static void or_pair(uint64_t t, int32_t *u, int32_t *v)
{
    uint64_t uu = (uint64_t)((1.0 + sqrt(1.0 + 8.0 * (double)t)) * 0.5);
    while (uu > 1 && uu * (uu - 1) / 2 > t) --uu;
    while ((uu + 1) * uu / 2 <= t) ++uu;
    *u = (int32_t)uu;
    *v = (int32_t)(t - uu * (uu - 1) / 2);
}

/* G(n,p), p = avg_deg/(n-1), by geometric skipping over the pair index (Batagelj and
 * Brandes, "Efficient generation of large random networks").  The pair range is cut
 * into chunks of 2^20 pairs; chunk j skips with its own stream, seeded by the j-th
 * output of the root stream, so that chunks can be generated independently. */
int64_t or_gen_er(int32_t n, double avg_deg, uint64_t seed, int32_t *eu, int32_t *ev,
                  int64_t cap)
{
    if (n < 1 || !(avg_deg >= 0.0)) return OR_ERR_ARG;
    uint64_t N = (uint64_t)n * (uint64_t)(n - 1) / 2;
    if (N == 0) return 0;
    double p = avg_deg / (double)(n - 1);
    int64_t cnt = 0;
    if (p >= 1.0) {
        for (uint64_t t = 0; t < N; ++t, ++cnt)
            if (cnt < cap) or_pair(t, &eu[cnt], &ev[cnt]);
        return cnt;
    }
    if (p <= 0.0) return 0;
    double lq = or_log(1.0 - p);
    uint64_t chunks = (N + OR_ER_CHUNK - 1) / OR_ER_CHUNK;
    for (uint64_t j = 0; j < chunks; ++j) {
        uint64_t cs = or_stream(seed, j);
        int64_t t = (int64_t)(j * OR_ER_CHUNK) - 1;
        int64_t end = (int64_t)((j + 1) * OR_ER_CHUNK < N ? (j + 1) * OR_ER_CHUNK : N);
        for (uint64_t i = 0;; ++i) {
            double r = or_unit(or_stream(cs, i));
            double q = or_log(1.0 - r) / lq;
            if (q >= (double)(end - t - 1)) break;
            t = t + 1 + (int64_t)q;
            if (cnt < cap) or_pair((uint64_t)t, &eu[cnt], &ev[cnt]);
            ++cnt;
        }
    }
    return cnt;
}

/* Linear preferential attachment (Batagelj and Brandes): an array M of 2*n*m0 node
 * slots; for edge e = v*m0 + i, M[2e] = v and M[2e+1] = M[r] with r uniform in
 * [0, 2e].  Edge e is (M[2e], M[2e+1]). */
int64_t or_gen_ba(int32_t n, int32_t m0, uint64_t seed, int32_t *eu, int32_t *ev, int64_t cap)
{
    if (n < 1 || m0 < 1) return OR_ERR_ARG;
    int64_t E = (int64_t)n * m0;
    int32_t *M = (int32_t *)malloc(sizeof(int32_t) * 2 * (size_t)E);
    if (!M) return OR_ERR_NOMEM;
    for (int64_t e = 0; e < E; ++e) {
        M[2 * e] = (int32_t)(e / m0);
        uint64_t r = or_below(or_stream(seed, (uint64_t)e), (uint64_t)(2 * e + 1));
        M[2 * e + 1] = M[r];
    }
    for (int64_t e = 0; e < E && e < cap; ++e) {
        eu[e] = M[2 * e];
        ev[e] = M[2 * e + 1];
    }
    free(M);
    return E;
}

/* R-MAT (Chakrabarti, Zhan, Faloutsos): edge e draws one quadrant per bit level from
 * the stream seeded by the e-th root output, most significant bit first; quadrant
 * (0,0) with probability a, (0,1) b, (1,0) c, (1,1) d = 1-a-b-c.  The probabilities
 * become integer thresholds floor(P * 2^64) of the cumulative sums a, a+b, a+b+c. */
int64_t or_gen_rmat(int32_t scale, int32_t edge_factor, double a, double b, double c,
                    uint64_t seed, int32_t *eu, int32_t *ev, int64_t cap)
{
    if (scale < 1 || scale > 30 || edge_factor < 1) return OR_ERR_ARG;
    if (!(a >= 0 && b >= 0 && c >= 0) || !(a + b + c < 1.0)) return OR_ERR_ARG;
    const double two64 = 18446744073709551616.0;
    uint64_t t1 = (uint64_t)(a * two64);
    uint64_t t2 = (uint64_t)((a + b) * two64);
    uint64_t t3 = (uint64_t)(((a + b) + c) * two64);
    int64_t E = (int64_t)edge_factor << scale;
    for (int64_t e = 0; e < E && e < cap; ++e) {
        uint64_t es = or_stream(seed, (uint64_t)e);
        uint32_t u = 0, v = 0;
        for (int l = 0; l < scale; ++l) {
            uint64_t x = or_stream(es, (uint64_t)l);
            uint32_t ru, rv;
            if (x < t1) { ru = 0; rv = 0; }
            else if (x < t2) { ru = 0; rv = 1; }
            else if (x < t3) { ru = 1; rv = 0; }
            else { ru = 1; rv = 1; }
            u = (u << 1) | ru;
            v = (v << 1) | rv;
        }
        eu[e] = (int32_t)u;
        ev[e] = (int32_t)v;
    }
    return E;
}

/* ------------------------------------------------------------------------------ */
/* Canonical CSR: symmetrise, drop self-loops, sort, remove duplicates.             */
/* ------------------------------------------------------------------------------ */

static int or_cmp_u64(const void *x, const void *y)
{
    uint64_t a = *(const uint64_t *)x, b = *(const uint64_t *)y;
    return (a > b) - (a < b);
}

/* Writes row_ptr[n+1] and col[<= 2m]; returns the number of arcs A, or an error. */
int64_t or_csr_build(int32_t n, int64_t m, const int32_t *eu, const int32_t *ev,
                     int32_t *row_ptr, int32_t *col)
{
    if (n < 1 || m < 0) return OR_ERR_ARG;
    uint64_t *arc = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(2 * m + 1));
    if (!arc) return OR_ERR_NOMEM;
    int64_t na = 0;
    for (int64_t e = 0; e < m; ++e) {
        int32_t u = eu[e], v = ev[e];
        if (u < 0 || u >= n || v < 0 || v >= n) { free(arc); return OR_ERR_GRAPH; }
        if (u == v) continue;
        arc[na++] = ((uint64_t)(uint32_t)u << 32) | (uint32_t)v;
        arc[na++] = ((uint64_t)(uint32_t)v << 32) | (uint32_t)u;
    }
    qsort(arc, (size_t)na, sizeof(uint64_t), or_cmp_u64);
    int64_t A = 0;
    for (int32_t i = 0; i <= n; ++i) row_ptr[i] = 0;
    for (int64_t i = 0; i < na; ++i) {
        if (i > 0 && arc[i] == arc[i - 1]) continue;
        int32_t u = (int32_t)(arc[i] >> 32);
        col[A++] = (int32_t)(arc[i] & 0xFFFFFFFFu);
        row_ptr[u + 1] += 1;
    }
    for (int32_t i = 0; i < n; ++i) row_ptr[i + 1] += row_ptr[i];
    free(arc);
    return A;
}

/* ------------------------------------------------------------------------------ */
/* Source sampler (Section 3.2: "randomly chosen shortest-path trees").             */
/* k distinct vertices, uniform without replacement: the k vertices with the        */
/* smallest (key(v), v), key(v) = v-th output of the stream seeded with `seed`.     */
/* Output: the chosen ids in ascending order.                                      */
/* ------------------------------------------------------------------------------ */

typedef struct { uint64_t key; int32_t v; } or_kv;

static int or_cmp_kv(const void *x, const void *y)
{
    const or_kv *a = (const or_kv *)x, *b = (const or_kv *)y;
    if (a->key != b->key) return (a->key > b->key) - (a->key < b->key);
    return (a->v > b->v) - (a->v < b->v);
}

static int or_cmp_i32(const void *x, const void *y)
{
    int32_t a = *(const int32_t *)x, b = *(const int32_t *)y;
    return (a > b) - (a < b);
}

int or_sample_sources(int32_t n, uint64_t seed, int32_t k, int32_t *src)
{
    if (n < 1 || k < 1 || k > n) return OR_ERR_ARG;
    or_kv *kv = (or_kv *)malloc(sizeof(or_kv) * (size_t)n);
    if (!kv) return OR_ERR_NOMEM;
    for (int32_t v = 0; v < n; ++v) {
        kv[v].key = or_stream(seed, (uint64_t)v);
        kv[v].v = v;
    }
    qsort(kv, (size_t)n, sizeof(or_kv), or_cmp_kv);
    for (int32_t i = 0; i < k; ++i) src[i] = kv[i].v;
    qsort(src, (size_t)k, sizeof(int32_t), or_cmp_i32);
    free(kv);
    return OR_OK;
}

/* ------------------------------------------------------------------------------ */
/* Single-source shortest paths by BFS (Section 3.4: BFS in unweighted graphs).     */
/* dist[v] = hop distance from s, -1 if unreachable; sigma[v] = number of shortest  */
/* s-v paths, sigma[s] = 1.                                                          */
/* ------------------------------------------------------------------------------ */

int or_bfs(int32_t n, const int32_t *row_ptr, const int32_t *col, int32_t s, int32_t *dist,
           uint64_t *sigma)
{
    if (n < 1 || s < 0 || s >= n) return OR_ERR_ARG;
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    if (!queue) return OR_ERR_NOMEM;
    for (int32_t v = 0; v < n; ++v) { dist[v] = -1; sigma[v] = 0; }
    dist[s] = 0;
    sigma[s] = 1;
    int32_t head = 0, tail = 0;
    queue[tail++] = s;
    int rc = OR_OK;
    while (head < tail) {
        int32_t v = queue[head++];
        for (int32_t j = row_ptr[v]; j < row_ptr[v + 1]; ++j) {
            int32_t w = col[j];
            if (dist[w] < 0) {
                dist[w] = dist[v] + 1;
                queue[tail++] = w;
            }
            if (dist[w] == dist[v] + 1) {
                if (__builtin_add_overflow(sigma[w], sigma[v], &sigma[w])) rc = OR_ERR_OVERFLOW;
            }
        }
    }
    free(queue);
    return rc;
}

/* ------------------------------------------------------------------------------ */
/* Brandes' algorithm [Bra01], Section 3.2.  For one source s:                      */
/*   BFS with a queue; S is the visit order (used as a stack), P[w] the            */
/*   predecessors of w on shortest paths, sigma the path counts;                   */
/*   then, popping S (deepest first):                                              */
/*     delta[v] += sigma[v] / sigma[w] * (1 + delta[w])   for v in P[w].            */
/* ------------------------------------------------------------------------------ */

typedef struct {
    int32_t *dist, *S, *pcount, *pred;
    uint64_t *sigma;
} or_ws;

static int or_ws_init(or_ws *ws, int32_t n, int64_t A)
{
    ws->dist = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    ws->S = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    ws->pcount = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    ws->pred = (int32_t *)malloc(sizeof(int32_t) * (size_t)(A > 0 ? A : 1));
    ws->sigma = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)n);
    if (!ws->dist || !ws->S || !ws->pcount || !ws->pred || !ws->sigma) return OR_ERR_NOMEM;
    return OR_OK;
}

static void or_ws_free(or_ws *ws)
{
    free(ws->dist); free(ws->S); free(ws->pcount); free(ws->pred); free(ws->sigma);
}

/* delta[v] = dependency of s on v (delta[s] is also filled; callers skip it). */
static int or_single_source(int32_t n, const int32_t *row_ptr, const int32_t *col, int32_t s,
                            or_ws *ws, double *delta)
{
    int32_t *dist = ws->dist, *S = ws->S, *pc = ws->pcount, *P = ws->pred;
    uint64_t *sigma = ws->sigma;
    for (int32_t v = 0; v < n; ++v) { dist[v] = -1; sigma[v] = 0; pc[v] = 0; delta[v] = 0.0; }
    dist[s] = 0;
    sigma[s] = 1;
    int32_t head = 0, tail = 0; /* S doubles as the BFS queue */
    S[tail++] = s;
    int rc = OR_OK;
    while (head < tail) {
        int32_t v = S[head++];
        for (int32_t j = row_ptr[v]; j < row_ptr[v + 1]; ++j) {
            int32_t w = col[j];
            if (dist[w] < 0) {
                dist[w] = dist[v] + 1;
                S[tail++] = w;
            }
            if (dist[w] == dist[v] + 1) {
                if (__builtin_add_overflow(sigma[w], sigma[v], &sigma[w])) rc = OR_ERR_OVERFLOW;
                P[row_ptr[w] + pc[w]++] = v;
            }
        }
    }
    if (rc != OR_OK) return rc;
    while (tail > 0) {
        int32_t w = S[--tail];
        for (int32_t i = 0; i < pc[w]; ++i) {
            int32_t v = P[row_ptr[w] + i];
            delta[v] += ((double)sigma[v] / (double)sigma[w]) * (1.0 + delta[w]);
        }
    }
    return OR_OK;
}

int or_dependencies(int32_t n, const int32_t *row_ptr, const int32_t *col, int32_t s,
                    double *delta)
{
    if (n < 1 || s < 0 || s >= n) return OR_ERR_ARG;
    or_ws ws;
    int rc = or_ws_init(&ws, n, row_ptr[n]);
    if (rc == OR_OK) rc = or_single_source(n, row_ptr, col, s, &ws, delta);
    or_ws_free(&ws);
    return rc;
}

/* scores[v] = scale * sum_{s in src, s != v} delta_s(v). */
int or_betweenness(int32_t n, const int32_t *row_ptr, const int32_t *col, int32_t k,
                   const int32_t *src, double scale, double *scores)
{
    if (n < 1 || k < 0) return OR_ERR_ARG;
    for (int32_t i = 0; i < k; ++i)
        if (src[i] < 0 || src[i] >= n) return OR_ERR_ARG;
    double *delta = (double *)malloc(sizeof(double) * (size_t)n);
    or_ws ws;
    int rc = delta ? or_ws_init(&ws, n, row_ptr[n]) : OR_ERR_NOMEM;
    for (int32_t v = 0; v < n; ++v) scores[v] = 0.0;
    for (int32_t i = 0; rc == OR_OK && i < k; ++i) {
        int32_t s = src[i];
        rc = or_single_source(n, row_ptr, col, s, &ws, delta);
        for (int32_t v = 0; rc == OR_OK && v < n; ++v)
            if (v != s) scores[v] += delta[v];
    }
    if (rc == OR_OK)
        for (int32_t v = 0; v < n; ++v) scores[v] *= scale;
    if (delta) or_ws_free(&ws);
    free(delta);
    return rc;
}

/* Exact betweenness: every vertex is a source; each unordered pair is seen twice. */
int or_betweenness_exact(int32_t n, const int32_t *row_ptr, const int32_t *col,
                         double *scores)
{
    if (n < 1) return OR_ERR_ARG;
    int32_t *src = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    if (!src) return OR_ERR_NOMEM;
    for (int32_t v = 0; v < n; ++v) src[v] = v;
    int rc = or_betweenness(n, row_ptr, col, n, src, 0.5, scores);
    free(src);
    return rc;
}

/* Sampled betweenness (Section 3.2): k sources from or_sample_sources, scale n/(2k). */
int or_betweenness_sampled(int32_t n, const int32_t *row_ptr, const int32_t *col,
                           uint64_t seed, int32_t k, double *scores)
{
    if (n < 1 || k < 1 || k > n) return OR_ERR_ARG;
    int32_t *src = (int32_t *)malloc(sizeof(int32_t) * (size_t)k);
    if (!src) return OR_ERR_NOMEM;
    int rc = or_sample_sources(n, seed, k, src);
    if (rc == OR_OK)
        rc = or_betweenness(n, row_ptr, col, k, src, (double)n / (2.0 * (double)k), scores);
    free(src);
    return rc;
}

/* ------------------------------------------------------------------------------ */
/* Edge betweenness (Section 4.3: edge centrality by the shortest paths through an  */
/* edge).  Brandes' sweep again; every term sigma[v] / sigma[w] * (1 + delta[w])    */
/* that flows from w to its predecessor v is the share of the pairs (s, t) whose    */
/* shortest paths use the edge {v, w}, so it is added to that edge as well as to    */
/* delta[v].  Per arc j of the CSR (u -> x), out[j] = scale * (sum over the arc u->x */
/* + sum over the reverse arc x->u): both arcs of an edge hold the edge's score.    */
/* Exact: all sources, scale 1/2 (unordered pairs); sampled: scale n/(2k).           */
/* ------------------------------------------------------------------------------ */

/* index of the arc v -> u in the sorted row of v, or -1 */
static int64_t or_find_arc(const int32_t *row_ptr, const int32_t *col, int32_t v, int32_t u)
{
    int64_t lo = row_ptr[v], hi = row_ptr[v + 1];
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (col[mid] < u) lo = mid + 1; else hi = mid;
    }
    return (lo < row_ptr[v + 1] && col[lo] == u) ? lo : -1;
}

int or_edge_betweenness(int32_t n, const int32_t *row_ptr, const int32_t *col, int32_t k,
                        const int32_t *src, double scale, double *out)
{
    if (n < 1 || k < 0) return OR_ERR_ARG;
    for (int32_t i = 0; i < k; ++i)
        if (src[i] < 0 || src[i] >= n) return OR_ERR_ARG;
    const int64_t A = row_ptr[n];
    double *delta = (double *)malloc(sizeof(double) * (size_t)n);
    double *arc = (double *)calloc((size_t)(A > 0 ? A : 1), sizeof(double));
    or_ws ws;
    int rc = (delta && arc) ? or_ws_init(&ws, n, A) : OR_ERR_NOMEM;
    for (int32_t i = 0; rc == OR_OK && i < k; ++i) {
        int32_t s = src[i];
        int32_t *dist = ws.dist, *S = ws.S;
        uint64_t *sigma = ws.sigma;
        for (int32_t v = 0; v < n; ++v) { dist[v] = -1; sigma[v] = 0; delta[v] = 0.0; }
        dist[s] = 0;
        sigma[s] = 1;
        int32_t head = 0, tail = 0;
        S[tail++] = s;
        while (head < tail) {
            int32_t v = S[head++];
            for (int32_t j = row_ptr[v]; j < row_ptr[v + 1]; ++j) {
                int32_t w = col[j];
                if (dist[w] < 0) {
                    dist[w] = dist[v] + 1;
                    S[tail++] = w;
                }
                if (dist[w] == dist[v] + 1 &&
                    __builtin_add_overflow(sigma[w], sigma[v], &sigma[w])) rc = OR_ERR_OVERFLOW;
            }
        }
        if (rc != OR_OK) break;
        /* deepest first: w hands its share to every predecessor v over the arc w -> v */
        while (tail > 0) {
            int32_t w = S[--tail];
            for (int32_t j = row_ptr[w]; j < row_ptr[w + 1]; ++j) {
                int32_t v = col[j];
                if (dist[v] != dist[w] - 1) continue;
                double c = ((double)sigma[v] / (double)sigma[w]) * (1.0 + delta[w]);
                delta[v] += c;
                arc[j] += c;
            }
        }
    }
    if (rc == OR_OK) {
        for (int32_t u = 0; u < n; ++u)
            for (int32_t j = row_ptr[u]; j < row_ptr[u + 1]; ++j) {
                int64_t r = or_find_arc(row_ptr, col, col[j], u);
                if (r < 0) { rc = OR_ERR_GRAPH; break; }
                out[j] = scale * (arc[j] + arc[r]);
            }
    }
    if (delta && arc) or_ws_free(&ws);
    free(delta);
    free(arc);
    return rc;
}

/* ------------------------------------------------------------------------------ */
/* Betweenness with an error bound (Section 3.2, citing Riondato and Kornaropoulos): */
/* r random pairs, one uniformly chosen shortest path per pair, every interior      */
/* vertex of the path counted once; with r from the vertex-diameter bound below,    */
/* every normalised estimate is within epsilon of the exact value with probability */
/* at least 1 - delta.                                                              */
/*   vertex diameter bound: per connected component C, a BFS from its smallest      */
/*     vertex x gives ecc(x); a shortest path has at most min(|C|, 2 ecc(x) + 1)    */
/*     vertices; VD = the largest bound over the components;                        */
/*   r = ceil(0.5 / eps^2 * (floor(log2(max(VD - 2, 1))) + 1 + ln(1 / delta)));     */
/*   pair i: u = below(stream(seed, 3i), n), v = below(stream(seed, 3i+1), n-1),    */
/*     v += (v >= u) (an ordered pair of distinct vertices);                        */
/*   path of pair i, walked back from v with key = stream(seed, 3i+2): at step j    */
/*     from w, t = below(stream(key, j), sigma[w]); the predecessors z of w (in    */
/*     adjacency order) split [0, sigma[w]) into runs of length sigma[z]; the run   */
/*     holding t names the next vertex (probability sigma[z] / sigma[w]);           */
/*   scores[w] = count[w] * n (n - 1) / (2 r): the estimate on the scale of the     */
/*     exact unordered scores (the normalised value is scores * 2 / (n (n - 1))).   */
/* ------------------------------------------------------------------------------ */

int or_vertex_diameter_estimate(int32_t n, const int32_t *row_ptr, const int32_t *col,
                                int32_t *vd)
{
    if (n < 1) return OR_ERR_ARG;
    int32_t *dist = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    if (!dist || !queue) { free(dist); free(queue); return OR_ERR_NOMEM; }
    for (int32_t v = 0; v < n; ++v) dist[v] = -1;
    int32_t best = 0;
    for (int32_t x = 0; x < n; ++x) {
        if (dist[x] >= 0) continue;
        int32_t head = 0, tail = 0, ecc = 0;
        dist[x] = 0;
        queue[tail++] = x;
        while (head < tail) {
            int32_t v = queue[head++];
            if (dist[v] > ecc) ecc = dist[v];
            for (int32_t j = row_ptr[v]; j < row_ptr[v + 1]; ++j)
                if (dist[col[j]] < 0) {
                    dist[col[j]] = dist[v] + 1;
                    queue[tail++] = col[j];
                }
        }
        int64_t bound = 2 * (int64_t)ecc + 1;
        if (bound > tail) bound = tail; /* tail = |C| */
        if (bound > best) best = (int32_t)bound;
    }
    free(dist);
    free(queue);
    *vd = best;
    return OR_OK;
}

int64_t or_rk_sample_count(double eps, double delta, int32_t vd)
{
    if (!(eps > 0.0 && eps < 1.0) || !(delta > 0.0 && delta < 1.0) || vd < 1) return OR_ERR_ARG;
    int64_t x = vd - 2 < 1 ? 1 : (int64_t)vd - 2;
    int lg = 0;
    while ((x >> (lg + 1)) != 0) ++lg; /* floor(log2 x) */
    double r = ceil(0.5 / (eps * eps) * ((double)lg + 1.0 + log(1.0 / delta)));
    if (!(r <= 2147483647.0)) return OR_ERR_ARG;
    return (int64_t)r;
}

/* The pair (u, v) of sample i and the interior vertices of its path (from v towards
 * u) into path[]; returns their number, or -1 if v is unreachable from u. */
static int32_t or_rk_one(int32_t n, const int32_t *row_ptr, const int32_t *col, uint64_t seed,
                         int64_t i, int32_t *dist, uint64_t *sigma, int32_t *queue,
                         int32_t *path, int32_t *uv, int *rc)
{
    const int32_t u = (int32_t)or_below(or_stream(seed, 3 * (uint64_t)i), (uint64_t)n);
    int32_t v = (int32_t)or_below(or_stream(seed, 3 * (uint64_t)i + 1), (uint64_t)(n - 1));
    if (v >= u) ++v;
    if (uv) { uv[0] = u; uv[1] = v; }
    for (int32_t x = 0; x < n; ++x) { dist[x] = -1; sigma[x] = 0; }
    dist[u] = 0;
    sigma[u] = 1;
    int32_t head = 0, tail = 0;
    queue[tail++] = u;
    while (head < tail) {
        int32_t x = queue[head++];
        for (int32_t j = row_ptr[x]; j < row_ptr[x + 1]; ++j) {
            int32_t w = col[j];
            if (dist[w] < 0) {
                dist[w] = dist[x] + 1;
                queue[tail++] = w;
            }
            if (dist[w] == dist[x] + 1 && __builtin_add_overflow(sigma[w], sigma[x], &sigma[w]))
                *rc = OR_ERR_OVERFLOW;
        }
    }
    if (dist[v] < 0) return -1;
    const uint64_t key = or_stream(seed, 3 * (uint64_t)i + 2);
    int32_t w = v, len = 0;
    for (uint64_t step = 0; dist[w] > 1; ++step) {
        const uint64_t t = or_below(or_stream(key, step), sigma[w]);
        uint64_t run = 0;
        int32_t z = -1;
        for (int32_t j = row_ptr[w]; j < row_ptr[w + 1]; ++j) {
            int32_t c = col[j];
            if (dist[c] != dist[w] - 1) continue;
            run += sigma[c];
            if (t < run) { z = c; break; }
        }
        if (z < 0) { *rc = OR_ERR_GRAPH; return -1; }
        path[len++] = z;
        w = z;
    }
    return len;
}

/* The pair of sample i (uv[0] = u, uv[1] = v) and the interior vertices of its path
 * (for tests of the pair and path laws). */
int32_t or_rk_path(int32_t n, const int32_t *row_ptr, const int32_t *col, uint64_t seed,
                   int64_t i, int32_t *uv, int32_t *path)
{
    if (n < 2 || i < 0) return OR_ERR_ARG;
    int32_t *dist = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    uint64_t *sigma = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)n);
    int rc = OR_OK;
    int32_t len = -1;
    if (dist && queue && sigma) len = or_rk_one(n, row_ptr, col, seed, i, dist, sigma, queue, path, uv, &rc);
    else rc = OR_ERR_NOMEM;
    free(dist); free(queue); free(sigma);
    return rc != OR_OK ? rc : len;
}

/* counts[w] += number of the samples i0 <= i < i1 whose path has w as an interior vertex
 * (samples are independent, so ranges can be computed apart and added) */
int or_rk_counts(int32_t n, const int32_t *row_ptr, const int32_t *col, uint64_t seed, int64_t i0,
                 int64_t i1, uint64_t *counts)
{
    if (n < 2 || i0 < 0 || i1 < i0) return OR_ERR_ARG;
    int32_t *dist = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *path = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    uint64_t *sigma = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)n);
    int rc = (dist && queue && path && sigma) ? OR_OK : OR_ERR_NOMEM;
    for (int64_t i = i0; rc == OR_OK && i < i1; ++i) {
        int32_t len = or_rk_one(n, row_ptr, col, seed, i, dist, sigma, queue, path, NULL, &rc);
        for (int32_t p = 0; rc == OR_OK && p < len; ++p) counts[path[p]] += 1;
    }
    free(dist); free(queue); free(path); free(sigma);
    return rc;
}

int or_betweenness_rk(int32_t n, const int32_t *row_ptr, const int32_t *col, double eps,
                      double delta, uint64_t seed, double *scores, int64_t *r_out, int32_t *vd_out)
{
    int32_t vd = 0;
    int rc = or_vertex_diameter_estimate(n, row_ptr, col, &vd);
    if (rc != OR_OK) return rc;
    const int64_t r = or_rk_sample_count(eps, delta, vd);
    if (r < 0) return (int)r;
    *r_out = r;
    *vd_out = vd;
    for (int32_t v = 0; v < n; ++v) scores[v] = 0.0;
    if (n < 2) return OR_OK;
    int32_t *dist = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *path = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    uint64_t *sigma = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)n);
    uint64_t *count = (uint64_t *)calloc((size_t)n, sizeof(uint64_t));
    if (!dist || !queue || !path || !sigma || !count) rc = OR_ERR_NOMEM;
    for (int64_t i = 0; rc == OR_OK && i < r; ++i) {
        int32_t len = or_rk_one(n, row_ptr, col, seed, i, dist, sigma, queue, path, NULL, &rc);
        for (int32_t p = 0; rc == OR_OK && p < len; ++p) count[path[p]] += 1;
    }
    if (rc == OR_OK) {
        const double scale = (double)n * (double)(n - 1) / (2.0 * (double)r);
        for (int32_t v = 0; v < n; ++v) scores[v] = (double)count[v] * scale;
    }
    free(dist); free(queue); free(path); free(sigma); free(count);
    return rc;
}

/* ------------------------------------------------------------------------------ */
/* Weighted betweenness (Section 3.4: shortest paths by Dijkstra's algorithm when the */
/* graph is weighted; Section 2.3: graphs are optionally weighted).  Positive       */
/* integer weights w[j] per arc, equal on both arcs of an edge, so that path lengths */
/* are exact and equal-length paths tie exactly.  Per source: Dijkstra with a binary */
/* heap; sigma[x] += sigma[v] for every arc (v, x) with dist[v] + w = dist[x], taken  */
/* when v is settled (all of x's predecessors settle before x since w >= 1); then    */
/* Brandes' accumulation over the settle order reversed.                            */
/* Random weights: the edge {u, v} (u < v) weighs 1 + below(stream(seed, u 2^32 + v),*/
/* wmax), the same on both arcs.                                                    */
/* ------------------------------------------------------------------------------ */

int or_edge_weights(int32_t n, const int32_t *row_ptr, const int32_t *col, uint64_t seed,
                    int32_t wmax, int32_t *w)
{
    if (n < 1 || wmax < 1) return OR_ERR_ARG;
    for (int32_t u = 0; u < n; ++u)
        for (int32_t j = row_ptr[u]; j < row_ptr[u + 1]; ++j) {
            uint64_t a = (uint64_t)(u < col[j] ? u : col[j]), b = (uint64_t)(u < col[j] ? col[j] : u);
            w[j] = 1 + (int32_t)or_below(or_stream(seed, (a << 32) | b), (uint64_t)wmax);
        }
    return OR_OK;
}

typedef struct { int64_t d; int32_t v; } or_item;

static void or_heap_push(or_item *h, int64_t *len, or_item x)
{
    int64_t i = (*len)++;
    while (i > 0) {
        int64_t p = (i - 1) / 2;
        if (h[p].d <= x.d) break;
        h[i] = h[p];
        i = p;
    }
    h[i] = x;
}

static or_item or_heap_pop(or_item *h, int64_t *len)
{
    or_item top = h[0], x = h[--(*len)];
    int64_t i = 0;
    for (;;) {
        int64_t c = 2 * i + 1;
        if (c >= *len) break;
        if (c + 1 < *len && h[c + 1].d < h[c].d) ++c;
        if (x.d <= h[c].d) break;
        h[i] = h[c];
        i = c;
    }
    if (*len > 0) h[i] = x;
    return top;
}

/* Dijkstra from s: dist (int64, -1 if unreachable), sigma, settle order S (returns its length) */
static int or_dijkstra(int32_t n, const int32_t *row_ptr, const int32_t *col, const int32_t *w,
                       int32_t s, int64_t *dist, uint64_t *sigma, int32_t *S, int32_t *ns,
                       or_item *heap, char *done)
{
    int rc = OR_OK;
    for (int32_t v = 0; v < n; ++v) { dist[v] = -1; sigma[v] = 0; done[v] = 0; }
    int64_t hl = 0;
    dist[s] = 0;
    sigma[s] = 1;
    or_item first = {0, s};
    or_heap_push(heap, &hl, first);
    int32_t cnt = 0;
    while (hl > 0) {
        or_item it = or_heap_pop(heap, &hl);
        int32_t v = it.v;
        if (done[v] || it.d != dist[v]) continue;
        done[v] = 1;
        S[cnt++] = v;
        for (int32_t j = row_ptr[v]; j < row_ptr[v + 1]; ++j) {
            int32_t x = col[j];
            int64_t nd = dist[v] + (int64_t)w[j];
            if (dist[x] < 0 || nd < dist[x]) {
                dist[x] = nd;
                sigma[x] = sigma[v];
                or_item y = {nd, x};
                or_heap_push(heap, &hl, y);
            } else if (nd == dist[x]) {
                if (__builtin_add_overflow(sigma[x], sigma[v], &sigma[x])) rc = OR_ERR_OVERFLOW;
            }
        }
    }
    *ns = cnt;
    return rc;
}

int or_sssp_weighted(int32_t n, const int32_t *row_ptr, const int32_t *col, const int32_t *w,
                     int32_t s, int64_t *dist, uint64_t *sigma)
{
    if (n < 1 || s < 0 || s >= n) return OR_ERR_ARG;
    const int64_t A = row_ptr[n];
    int32_t *S = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    or_item *heap = (or_item *)malloc(sizeof(or_item) * (size_t)(A + 1));
    char *done = (char *)malloc((size_t)n);
    int rc = OR_ERR_NOMEM;
    int32_t ns = 0;
    if (S && heap && done) rc = or_dijkstra(n, row_ptr, col, w, s, dist, sigma, S, &ns, heap, done);
    free(S); free(heap); free(done);
    return rc;
}

/* scores[v] = scale * sum_{s in src, s != v} delta_s(v) with weighted shortest paths. */
int or_betweenness_weighted(int32_t n, const int32_t *row_ptr, const int32_t *col, const int32_t *w,
                            int32_t k, const int32_t *src, double scale, double *scores)
{
    if (n < 1 || k < 0) return OR_ERR_ARG;
    for (int32_t i = 0; i < k; ++i)
        if (src[i] < 0 || src[i] >= n) return OR_ERR_ARG;
    const int64_t A = row_ptr[n];
    for (int64_t j = 0; j < A; ++j)
        if (w[j] < 1) return OR_ERR_ARG;
    int64_t *dist = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    uint64_t *sigma = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)n);
    double *delta = (double *)malloc(sizeof(double) * (size_t)n);
    int32_t *S = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    or_item *heap = (or_item *)malloc(sizeof(or_item) * (size_t)(A + 1));
    char *done = (char *)malloc((size_t)n);
    int rc = (dist && sigma && delta && S && heap && done) ? OR_OK : OR_ERR_NOMEM;
    for (int32_t v = 0; v < n; ++v) scores[v] = 0.0;
    for (int32_t i = 0; rc == OR_OK && i < k; ++i) {
        const int32_t s = src[i];
        int32_t ns = 0;
        rc = or_dijkstra(n, row_ptr, col, w, s, dist, sigma, S, &ns, heap, done);
        if (rc != OR_OK) break;
        for (int32_t v = 0; v < n; ++v) delta[v] = 0.0;
        for (int32_t t = ns - 1; t >= 0; --t) {
            const int32_t x = S[t];
            for (int32_t j = row_ptr[x]; j < row_ptr[x + 1]; ++j) {
                const int32_t v = col[j];  /* v precedes x if dist[v] + w = dist[x] */
                if (dist[v] >= 0 && dist[v] + (int64_t)w[j] == dist[x])
                    delta[v] += ((double)sigma[v] / (double)sigma[x]) * (1.0 + delta[x]);
            }
            if (x != s) scores[x] += delta[x];
        }
    }
    if (rc == OR_OK)
        for (int32_t v = 0; v < n; ++v) scores[v] *= scale;
    free(dist); free(sigma); free(delta); free(S); free(heap); free(done);
    return rc;
}

/* ------------------------------------------------------------------------------ */
/* Closeness (Table 1: "closeness", shortest-path search from each node, and its    */
/* approximation after Eppstein and Wang with s sampled sources).  For every vertex */
/* v:  far[v] = scale * sum of d(s, v) over the sources s != v that reach v,        */
/*     reach[v] = scale * number of those sources.                                 */
/* Exact: all n sources, scale 1, closeness(v) = reach[v] / far[v] (which is        */
/* (n-1) / sum_u d(u, v) on a connected graph).  Sampled: k uniform sources, scale  */
/* n/k, the Eppstein-Wang estimate of the distance sum.                            */
/* ------------------------------------------------------------------------------ */

int or_closeness(int32_t n, const int32_t *row_ptr, const int32_t *col, int32_t k,
                 const int32_t *src, double scale, double *far, double *reach)
{
    if (n < 1 || k < 0) return OR_ERR_ARG;
    for (int32_t i = 0; i < k; ++i)
        if (src[i] < 0 || src[i] >= n) return OR_ERR_ARG;
    int32_t *dist = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    if (!dist || !queue) { free(dist); free(queue); return OR_ERR_NOMEM; }
    for (int32_t v = 0; v < n; ++v) { far[v] = 0.0; reach[v] = 0.0; }
    for (int32_t i = 0; i < k; ++i) {
        int32_t s = src[i];
        for (int32_t v = 0; v < n; ++v) dist[v] = -1;
        dist[s] = 0;
        int32_t head = 0, tail = 0;
        queue[tail++] = s;
        while (head < tail) {
            int32_t v = queue[head++];
            for (int32_t j = row_ptr[v]; j < row_ptr[v + 1]; ++j) {
                int32_t w = col[j];
                if (dist[w] < 0) {
                    dist[w] = dist[v] + 1;
                    queue[tail++] = w;
                    far[w] += (double)dist[w];
                    reach[w] += 1.0;
                }
            }
        }
    }
    for (int32_t v = 0; v < n; ++v) { far[v] *= scale; reach[v] *= scale; }
    free(dist);
    free(queue);
    return OR_OK;
}

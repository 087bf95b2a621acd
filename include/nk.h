/*
 * nk.h - C ABI of the GB300 betweenness-centrality library (libnk.so).
 *
 * Betweenness of a vertex v in an undirected, unweighted, simple graph G = (V, E):
 *     c(v) = sum over unordered pairs {s,t}, s != v != t, sigma_st > 0, of
 *            sigma_st(v) / sigma_st,
 * where sigma_st counts shortest s-t paths and sigma_st(v) those through v.  It is
 * computed by Brandes' algorithm [Bra01] (Section 3.2 and Table 1 of the NetworKit
 * paper, "betweenness", O(nm) time): per source s, a BFS (unweighted graphs, Section
 * 3.4) that counts sigma, then the dependency accumulation
 *     delta_s(v) = sum_{w : v is a predecessor of w} sigma_sv / sigma_sw * (1 + delta_s(w)),
 * and the dependencies of all sources are summed (Section 3.2).  The sampled
 * estimate (Section 3.2, after Geisberger et al.) sums the dependencies of k sources
 * drawn uniformly without replacement and scales the sum by n/k.
 *
 * Conventions shared by every call:
 *   - Return value: NK_OK (0) or a negative NK_ERR_* code; never aborts.  The
 *     thread-local nk_last_error() describes the last failure of the calling thread.
 *   - Vertex ids and CSR offsets are int32; n >= 1 and the arc count A < 2^31.
 *   - Graphs are immutable, canonical CSR resident in GPU memory, owned by the library
 *     until nk_graph_free().  Canonical: for every vertex the neighbour list is sorted
 *     ascending, holds no duplicate and no self-loop, and u in N(v) <=> v in N(u).
 *   - Host pointers unless a flag says otherwise.  Output buffers are owned by the
 *     caller.  Calls are synchronous (they return after results are written) and are
 *     ordered on the stream set by nk_set_stream (default: the legacy default stream).
 *   - Scores are raw (no normalisation): each unordered pair counts once.
 */
#ifndef NK_H
#define NK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status codes */
#define NK_OK 0
#define NK_PENDING 1          /* serving: request admitted or queued, not finished */
#define NK_ERR_ARG (-1)       /* invalid argument (null pointer, k outside [1,n], ...) */
#define NK_ERR_GRAPH (-2)     /* CSR not canonical / ids out of range */
#define NK_ERR_NOMEM (-3)     /* device memory (or the serving budget) exhausted */
#define NK_ERR_OVERFLOW (-4)  /* a shortest-path count sigma exceeded 2^64 - 1 */
#define NK_ERR_CUDA (-5)      /* a CUDA runtime call failed */
#define NK_ERR_TIMEOUT (-6)   /* a bounded device-side wait ran out */
#define NK_ERR_SHUTDOWN (-7)  /* serving: server is shutting down */

/* ---------------------------------------------------------------- graph construction */
#define NK_CSR_VALIDATE 1u     /* check canonical form; NK_ERR_GRAPH if it is not */
#define NK_CSR_CANONICALISE 2u /* symmetrise, drop self-loops, sort, dedupe on the GPU */
#define NK_CSR_DEVICE_PTRS 4u  /* input arrays are device pointers */

typedef struct nk_graph nk_graph;

/* Builds a graph from CSR arrays row_ptr[n+1] (row_ptr[0] = 0, row_ptr[n] = n_arcs) and
 * col[n_arcs].  Flags: none = trust the caller (must already be canonical; ids are
 * still range-checked on the GPU), NK_CSR_VALIDATE, or NK_CSR_CANONICALISE (any
 * adjacency, e.g. one direction per edge, duplicates, self-loops).  The arrays are
 * copied; the caller keeps ownership.  Graph structure: Section 2.3 (adjacency
 * structure with O(n+m) memory; here an immutable int32 CSR). */
int nk_graph_from_csr(int32_t n, const int32_t *row_ptr, const int32_t *col, int64_t n_arcs,
                      uint32_t flags, nk_graph **out);

/* Builds the canonical graph of an undirected edge list (u[i], v[i]), i < m: both
 * directions, self-loops dropped, duplicates removed; the CSR is built on the GPU.
 * Flags: NK_CSR_DEVICE_PTRS only.  Out-of-range ids give NK_ERR_GRAPH. */
int nk_graph_from_edges(int32_t n, int64_t m, const int32_t *u, const int32_t *v,
                        uint32_t flags, nk_graph **out);

/* Seeded generators of Section 5 (Table 2), run on the GPU, followed by the canonical
 * CSR build.  Random numbers: SplitMix64 (Steele, Lea, Flood 2014) as a counter-based
 * generator, stream(seed, i) = mix64(seed + (i+1) * 0x9E3779B97F4A7C15).
 *   NK_GEN_ER   n_or_scale = n, params[0] = average degree d (p = d/(n-1)); G(n,p) by
 *               Batagelj-Brandes geometric skipping in chunks of 2^20 vertex pairs.
 *   NK_GEN_BA   n_or_scale = n, params[0] = m0 edges per vertex; Batagelj-Brandes
 *               linear preferential attachment.
 *   NK_GEN_RMAT n_or_scale = scale (n = 2^scale), params = {edge_factor, a, b, c};
 *               edge_factor * 2^scale raw edges (Chakrabarti et al.).
 * The result is identical, byte for byte, on every run with the same arguments. */
#define NK_GEN_ER 1
#define NK_GEN_BA 2
#define NK_GEN_RMAT 3
int nk_graph_generate(int kind, const double *params, int32_t n_or_scale, uint64_t seed,
                      nk_graph **out);

/* n and the number of arcs A (= 2 * undirected edges) of the graph (Section 2.3: the
 * graph data structure answers its node and edge counts). */
int nk_graph_info(const nk_graph *g, int32_t *n, int64_t *n_arcs);

/* Copies the canonical CSR to host arrays row_ptr[n+1] and col[A] (Section 2.3: the
 * adjacency structure, here as the immutable int32 CSR the sweeps read).  Used to hand
 * the same graph to another program, e.g. a checker. */
int nk_graph_export_csr(const nk_graph *g, int32_t *row_ptr, int32_t *col);

/* Frees the graph and its cached device workspace (Section 2.3: the graph object owns
 * its adjacency structure).  NK_ERR_ARG if serving requests on it are still pending (the
 * graph is then not freed). */
int nk_graph_free(nk_graph *g);

/* ---------------------------------------------------------------- sampler (Section 3.2) */
/* k distinct sources, uniform without replacement: the k vertices with the smallest
 * (stream(seed, v), v); written to src[k] in ascending id order.  1 <= k <= n.
 * flags: NK_RUN_DEVICE_PTRS makes src a device pointer. */
int nk_sample_sources(int32_t n, uint64_t seed, int32_t k, int32_t *src, uint32_t flags);

/* ---------------------------------------------------------------- single-source sweep */
/* Forward BFS from s (Section 3.4): dist[v] = hops from s (-1 unreachable), sigma[v] =
 * number of shortest s-v paths.  Host arrays of n entries.  NK_ERR_OVERFLOW if some
 * sigma exceeds 2^64 - 1 (outputs are then unspecified). */
int nk_sssp(const nk_graph *g, int32_t s, int32_t *dist, uint64_t *sigma);

/* Allocation-free forward sweep.  No counterpart in the paper: it is a service for
 * callers that cannot allocate device memory when they call in - code running under an
 * allocator that forbids cudaMalloc/cudaFree, or a host library that must not grow its
 * device footprint after start-up.  Same results as nk_sssp (dist[n], sigma[n]) on a
 * canonical CSR the caller already holds on the device:
 *   row_ptr[n+1], col[n_arcs]  device pointers to a canonical CSR (as nk_graph_export_csr
 *                              writes it; not re-validated), read only;
 *   dist[n] (int32), sigma[n] (uint64)  device output buffers owned by the caller;
 *   stream                      cudaStream_t the work is ordered on (NULL = default);
 *                              the call returns after the results are written.
 * Scratch (control words, BFS queue, per-level counters) is one static device array of
 * about 20 MiB that every GPU loading the library holds until the process exits, so
 * 1 <= n <= 1048576 (2^20); a larger n returns NK_ERR_ARG with a message.  The call makes
 * no cudaMalloc, cudaFree or other allocating call (nk_alloc_count does not move).
 * With CUDA's lazy module loading (the default), the array is reserved when the module
 * that holds it first loads on a device: at the first call of this function or of
 * another single-source sweep there.  Callers whose footprint must not grow after
 * start-up therefore make one call at start-up.  That first call also looks up the
 * device's address of the array (cudaGetSymbolAddress) with the device current.  The
 * call copies the source id from pageable host memory and waits for its stream, so it
 * must not be called on a stream that is being captured into a CUDA graph.  All calls
 * share the one array, so calls that overlap on the GPU race: serialise them (one
 * stream, or host ordering).
 * Rows are not split into chunks here, so hubs make it slower than nk_sssp.
 * Errors: NK_ERR_ARG, NK_ERR_OVERFLOW (sigma exceeded 2^64 - 1), NK_ERR_TIMEOUT,
 * NK_ERR_CUDA. */
int nk_sssp_noalloc(int32_t n, const int32_t *row_ptr, const int32_t *col, int64_t n_arcs,
                    int32_t s, int32_t *dist, uint64_t *sigma, void *stream);

/* ---------------------------------------------------------------- betweenness */
#define NK_MODE_AUTO 0       /* batched where it fits, per-source otherwise */
#define NK_MODE_PER_SOURCE 1 /* plain per-source kernel (one BFS tree at a time); backward levels
                                whose successors carry few arcs add psi with FP64 atomics, so the
                                last bits of its scores may differ from run to run (distances and
                                path counts never do) */
#define NK_MODE_BATCHED 2    /* bitset multi-source kernel, `batch` sources per launch */

#define NK_DIR_AUTO 0        /* direction-optimising: switch by alpha */
#define NK_DIR_TOP_DOWN 1    /* every level top-down (push from the frontier) */
#define NK_DIR_BOTTOM_UP 2   /* every level bottom-up (pull into unvisited vertices) */

#define NK_RUN_DEVICE_PTRS 1u  /* scores (and src) are device pointers */
#define NK_RUN_TIME_KERNELS 2u /* record per-launch durations of the sweep kernel */
#define NK_RUN_RELABEL 8u      /* batched betweenness on a relabelled copy of the graph (vertex
                                  v becomes v * 2654435761 mod n; results mapped back) */
#define NK_RUN_NO_RELABEL 16u  /* never relabel (without either flag: the autotuner's choice) */
#define NK_RUN_CUDA_GRAPH 4u   /* sampled, batched, device pointers: capture the whole call
                                  (sampler, persistent launches, scaling) into a CUDA graph
                                  on first use and replay it for later calls with the same
                                  graph, seed, k, options and output pointer; every replay
                                  re-executes all kernels.  Falls back to the regular path
                                  when a BFS is deeper than the captured level slabs. */

typedef struct nk_run_opts {
    int32_t mode;      /* NK_MODE_* */
    int32_t batch;     /* batched mode: sources per batch, 64/128/256; 0 = autotuned */
    int32_t tpv;       /* accepted for compatibility (0 or a power of 2 <= 32) and ignored: the
                          per-source sweep runs lanes over the arcs of groups of vertices */
    int32_t direction; /* NK_DIR_* */
    double alpha;      /* bottom-up when alpha * (frontier arcs) > (unvisited arcs); 0 = auto */
    uint32_t flags;    /* NK_RUN_* */
    int32_t grid_ctas; /* if > 0: persistent launches use at most this many CTAs (0 = all
                          co-resident CTAs); fewer CTAs make each grid barrier cheaper for
                          sweeps with little work per level */
    int32_t chunk;     /* batched mode: rows longer than this many arcs are split into chunks
                          of this many arcs, each taken by its own warp; a multiple of 32 in
                          [32, 4096], or 0 for 256 (or the autotuner's choice) */
    int32_t reserved[5];
} nk_run_opts;

/* Statistics of the last betweenness call made by this thread. */
typedef struct nk_run_stats {
    int32_t mode;            /* mode actually used */
    int32_t batch;           /* sources per batch used (1 for per-source) */
    int32_t tpv;
    int32_t max_depth;       /* deepest BFS level seen */
    int64_t launches;        /* sweep-kernel launches */
    double kernel_ms;        /* sum of sweep-kernel durations (CUDA events), if timed */
    int64_t td_levels;       /* levels run top-down / bottom-up */
    int64_t bu_levels;
    double alpha;
} nk_run_stats;

/* Exact betweenness: all n sources, scores[n] = (1/2) sum_s delta_s(v). */
int nk_betweenness_exact(const nk_graph *g, double *scores);

/* Sampled betweenness: k sources from nk_sample_sources(n, seed, k), scores[n] =
 * n/(2k) * sum_{s in S} delta_s(v).  1 <= k <= n. */
int nk_betweenness_sampled(const nk_graph *g, uint64_t seed, int32_t k, double *scores);

/* Sampled betweenness with explicit options (opts may be NULL for defaults). */
int nk_betweenness_sampled_opts(const nk_graph *g, uint64_t seed, int32_t k, double *scores,
                                const nk_run_opts *opts);

/* scores[n] = scale * sum_{s in src} delta_s(v) over an explicit list of k distinct
 * sources (k >= 1).  The general entry point behind the two above. */
int nk_betweenness_sources(const nk_graph *g, const int32_t *src, int32_t k, double scale,
                           double *scores, const nk_run_opts *opts);

/* Stats of the calling thread's last betweenness call (no counterpart in the paper:
 * launch width, levels run top-down and bottom-up, kernel time). */
int nk_last_run_stats(nk_run_stats *out);

/* Autotuner (no counterpart in the paper; it tunes the batched GPU sweep, which is this
 * library's own design): on one launch of up to 256 of the run's own sources (seed, k), times the
 * batched sweep with 64/128/256 sources per launch, then alpha in {0.25, 1, 4, 16}, then hub
 * chunks of 128 arcs against 256, then the relabelled copy (NK_RUN_RELABEL) with alpha in
 * {0.25, 4, 16}; writes the fastest into *best (flags: NK_RUN_RELABEL or NK_RUN_NO_RELABEL).
 * The choice is cached on the graph: later calls with batch/alpha/chunk = 0 and neither
 * relabel flag use it.  Errors: NK_ERR_ARG (null pointers, k outside [1, n]). */
int nk_autotune(const nk_graph *g, uint64_t seed, int32_t k, nk_run_opts *best);

/* ---------------------------------------------------------------- weighted graphs (Sections 2.3, 3.4) */
/* Graphs are optionally weighted (Section 2.3); shortest paths then come from Dijkstra's
 * algorithm instead of BFS (Section 3.4).  Weights are positive integers, one per arc of the
 * canonical CSR (A entries, in the order of nk_graph_export_csr), equal on both arcs of an
 * edge, so path lengths are exact and equal-length paths tie exactly.
 * nk_graph_set_weights copies w (device pointer with NK_CSR_DEVICE_PTRS, else host) and
 * checks it: NK_ERR_GRAPH if a weight is < 1 or the two arcs of an edge differ.
 * nk_graph_random_weights gives the edge {u, v}, u < v, the weight
 * 1 + floor(x * wmax / 2^64) with x the (u 2^32 + v)-th output of the SplitMix64 stream
 * seeded with seed (wmax >= 1).  nk_graph_export_weights copies them to host memory.
 * nk_sssp_weighted: dist (int64, -1 if unreachable) and sigma (uint64, NK_ERR_OVERFLOW above
 * 2^64 - 1) from source s, host buffers of n entries.
 * nk_betweenness_weighted_exact / _sampled: as nk_betweenness_exact / _sampled (unordered
 * pairs, scale 1/2 or n/(2k), the same sampler) with weighted shortest paths; NK_ERR_ARG if
 * the graph has no weights.  The search settles the vertices in buckets of equal distance,
 * one persistent launch per source. */
int nk_graph_set_weights(nk_graph *g, const int32_t *w, uint32_t flags);
int nk_graph_random_weights(nk_graph *g, uint64_t seed, int32_t wmax);
int nk_graph_export_weights(const nk_graph *g, int32_t *w);
int nk_sssp_weighted(const nk_graph *g, int32_t s, int64_t *dist, uint64_t *sigma);
int nk_betweenness_weighted_exact(const nk_graph *g, double *scores);
int nk_betweenness_weighted_sampled(const nk_graph *g, uint64_t seed, int32_t k, double *scores,
                                    const nk_run_opts *opts);

/* ---------------------------------------------------------------- error-bounded estimate (Section 3.2) */
/* Betweenness with an error bound, after Riondato and Kornaropoulos (cited in Section 3.2 as
 * the estimate whose scores are within +-epsilon of the exact ones with a user-chosen
 * probability).  r random ordered pairs (u, v) of distinct vertices; for each, one shortest
 * u-v path chosen uniformly (if v is reachable); every interior vertex of the path is counted.
 *   vertex-diameter bound VD (nk_vertex_diameter_estimate): per connected component C with
 *     smallest vertex x, min(|C|, 2 ecc(x) + 1); the largest over the components;
 *   r = ceil(0.5 / epsilon^2 * (floor(log2(max(VD - 2, 1))) + 1 + ln(1 / delta)));
 *   pair i: u = floor(s0 n / 2^64), v = floor(s1 (n-1) / 2^64), v += (v >= u), with s0, s1
 *     outputs 3i and 3i+1 of the SplitMix64 stream seeded with seed; output 3i+2 seeds the
 *     path walk: from w (starting at v), step j draws t = floor(x_j sigma_w / 2^64) and
 *     moves to the predecessor z whose run of length sigma_z, laid end to end in adjacency
 *     order, holds t;
 *   scores[w] = count[w] * n (n - 1) / (2 r): on the scale of the exact unordered scores
 *     (the normalised estimate, which the bound is about, is scores[w] * 2 / (n (n - 1))).
 * samples and vertex_diameter (nullable) receive r and VD.  scores holds n doubles (device
 * with NK_RUN_DEVICE_PTRS).  Errors: NK_ERR_ARG (epsilon or delta outside (0, 1), r above
 * 2^31 - 1, null pointers), NK_ERR_OVERFLOW (a path count above 2^64 - 1), NK_ERR_NOMEM,
 * NK_ERR_TIMEOUT.  Device memory: 16 r + 8 n bytes besides the sweep's own workspace. */
int nk_betweenness_rk(const nk_graph *g, double epsilon, double delta, uint64_t seed, double *scores,
                      int64_t *samples, int32_t *vertex_diameter, const nk_run_opts *opts);
/* The vertex-diameter bound above (computed once per graph, then cached). */
int nk_vertex_diameter_estimate(const nk_graph *g, int32_t *vd);

/* ---------------------------------------------------------------- edge betweenness (Section 4.3) */
/* Edge betweenness: for an edge {u, v}, the sum over unordered reachable pairs {s, t} of the
 * fraction of shortest s-t paths that use the edge (Section 4.3: edge centrality from the
 * shortest paths through an edge).  Computed in the same sweeps as betweenness: in the
 * dependency accumulation the share sigma_v / sigma_w * (1 + delta_w) that a vertex w hands
 * to a predecessor v is also added to the edge {v, w}.
 * edge_scores holds one double per arc of the canonical CSR (A entries, in the order of
 * nk_graph_export_csr); both arcs of an edge hold the edge's score.  Exact: all sources,
 * scale 1/2.  Sampled: the sources of nk_sample_sources(n, seed, k), scale n/(2k).
 * edge_scores is a device pointer with NK_RUN_DEVICE_PTRS in opts, else host memory.
 * Errors: NK_ERR_ARG (null pointers, k outside [1, n]), NK_ERR_OVERFLOW (a path count above
 * 2^64 - 1), NK_ERR_GRAPH (an arc without its reverse arc), NK_ERR_NOMEM, NK_ERR_TIMEOUT.
 * Device memory: 8A + 8n bytes besides the sweep's own workspace. */
int nk_edge_betweenness_exact(const nk_graph *g, double *edge_scores);
int nk_edge_betweenness_sampled(const nk_graph *g, uint64_t seed, int32_t k, double *edge_scores,
                                const nk_run_opts *opts);

/* ---------------------------------------------------------------- closeness (Table 1) */
/* Closeness from the same forward sweep (Table 1: closeness by a shortest-path search from
 * each node, and the approximation after Eppstein and Wang from s sampled sources).  For
 * every vertex v, with S the source set:
 *     far[v]   = scale * sum of d(s, v) over the sources s in S, s != v, that reach v,
 *     reach[v] = scale * number of those sources,
 * so that closeness(v) = reach[v] / far[v] ((n-1) / sum_u d(u, v) on a connected graph).
 * Exact: S = V, scale 1 (the sums are exact integers).  Sampled: S from
 * nk_sample_sources(n, seed, k), scale n/k.  far and reach hold n doubles each (device
 * pointers with NK_RUN_DEVICE_PTRS).  The batched form runs its forward sweep only. */
int nk_closeness_exact(const nk_graph *g, double *far, double *reach);
int nk_closeness_sampled(const nk_graph *g, uint64_t seed, int32_t k, double *far, double *reach,
                         const nk_run_opts *opts);

/* ---------------------------------------------------------------- serving runtime */
typedef struct nk_server nk_server;
typedef int64_t nk_req;

typedef struct nk_server_opts {
    double mem_budget_bytes; /* device bytes for per-request state; 0 = 60% of free */
    int32_t max_inflight;    /* requests on the GPU at once (streams); 0 = 8 */
    int32_t batch;           /* sources per launch for served requests (64/128/256);
                                0 = 128 (narrower when k is smaller) */
    double timeout_s;        /* bound on device-side waits; 0 = 10 s */
    int32_t no_pack;         /* 1: never pack small requests into one launch */
    int32_t reserved[7];
} nk_server_opts;

typedef struct nk_server_stats {
    int64_t submitted, completed, failed, rejected;
    double p50_ms, p99_ms, max_ms;   /* submit-to-completion latency of completed requests */
    double busy_s;                   /* wall time with at least one request on the GPU */
    double edges_x_sources;          /* sum over completed requests of m * k */
    int64_t peak_inflight;
    double peak_bytes;
    double queue_p50_ms, queue_p99_ms; /* submit-to-admission wait */
    double run_p50_ms, run_p99_ms;     /* admission-to-completion time */
    int64_t jobs;                      /* launches of work started (single or packed) */
    int64_t packed_requests;           /* requests that ran inside a packed launch */
} nk_server_stats;

/* Serving runtime: no counterpart in the paper.  The paper runs the sources of one
 * betweenness computation in parallel (Section 3.2); the server extends that to many
 * independent requests on different graphs, arriving over time, which run concurrently
 * on the GPU (continuous batching with device-memory admission). */
int nk_server_create(const nk_server_opts *opts, nk_server **out);
/* Waits for pending requests, then frees the server (serving runtime, see above). */
void nk_server_destroy(nk_server *srv);

/* Queues a sampled-betweenness request (graph, seed, k): the estimate of Section 3.2,
 * computed as nk_betweenness_sampled computes it.  `scores` (n doubles, host)
 * must stay valid until nk_serve_poll returns something other than NK_PENDING.
 * Admission is by the device-memory budget; requests larger than the whole budget are
 * rejected with NK_ERR_NOMEM.  Consecutive small requests (graphs of up to 4M arcs,
 * k <= 256) are packed, up to 1024 sources, into launches of 128 sources on the block-diagonal union
 * of their graphs (BFS trees never cross graphs, so each request's scores are those of
 * the request alone, up to FP summation order). */
int nk_serve_submit(nk_server *srv, const nk_graph *g, uint64_t seed, int32_t k,
                    double *scores, nk_req *id);

/* Serving runtime (no counterpart in the paper): NK_PENDING while queued or running;
 * then NK_OK or the request's error code. */
int nk_serve_poll(nk_server *srv, nk_req id);

/* Serving runtime (no counterpart in the paper): blocks until request id is finished
 * (or timeout_s elapses: NK_PENDING). */
int nk_serve_wait(nk_server *srv, nk_req id, double timeout_s);

/* Serving runtime (no counterpart in the paper): counters and latency percentiles. */
int nk_server_get_stats(nk_server *srv, nk_server_stats *out);

/* ---------------------------------------------------------------- misc */
/* Stream used by every later call of this process (a cudaStream_t); NULL = default.
 * No counterpart in the paper: CUDA stream plumbing, so that the calls are ordered with
 * the caller's own GPU work (e.g. PyTorch's current stream). */
int nk_set_stream(void *stream);

/* Bound, in nanoseconds, on every device-side wait (grid barrier); default 10 s.  No
 * counterpart in the paper: failure detection around the persistent kernels. */
int nk_set_wait_limit_ns(uint64_t ns);

/* Failure-detection self test (no counterpart in the paper): launches a kernel whose
 * wait on a flag that nothing sets runs out after limit_ns; returns NK_ERR_TIMEOUT when the bounded wait works
 * (and the CUDA context stays usable). */
int nk_selftest_wait_timeout(uint64_t limit_ns);

/* Number of kernels this library has launched in this process (all entry points).  No
 * counterpart in the paper: launch accounting. */
uint64_t nk_launch_count(void);

/* Number of memory allocation calls (cudaMalloc, cudaMallocAsync, cudaMallocHost) this
 * library has made in this process (all entry points); a diagnostic, like the launch
 * count, that shows which calls allocate. */
uint64_t nk_alloc_count(void);

/* Message of the calling thread's last failure; library version string.  No
 * counterpart in the paper. */
const char *nk_last_error(void);
const char *nk_version(void);

#ifdef __cplusplus
}
#endif
#endif /* NK_H */

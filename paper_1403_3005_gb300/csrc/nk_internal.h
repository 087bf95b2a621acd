// Host-side internals of libnk: error state, stream, device buffers, graph object,
// and the declarations shared by the translation units of the library.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdarg>
#include <cstdint>
#include <memory>
#include <mutex>
#include <vector>

#include "nk.h"

namespace nk {

// ---------------------------------------------------------------- errors
int set_error(int code, const char *fmt, ...);
int cuda_fail(cudaError_t e, const char *what, const char *file, int line);

#define NK_CUDA(call)                                                                 \
    do {                                                                              \
        cudaError_t nk_e_ = (call);                                                   \
        if (nk_e_ != cudaSuccess) return ::nk::cuda_fail(nk_e_, #call, __FILE__, __LINE__); \
    } while (0)

#define NK_TRY(expr)                    \
    do {                                \
        int nk_rc_ = (expr);            \
        if (nk_rc_ != NK_OK) return nk_rc_; \
    } while (0)

// ---------------------------------------------------------------- launch accounting
// Every kernel launch of the library bumps this process-wide counter.
extern std::atomic<uint64_t> g_launches;
inline void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
// Every memory allocation call of the library (cudaMalloc, cudaMallocAsync,
// cudaMallocHost) bumps this process-wide counter.
extern std::atomic<uint64_t> g_allocs;
inline void count_alloc() { g_allocs.fetch_add(1, std::memory_order_relaxed); }

// ---------------------------------------------------------------- stream / limits
cudaStream_t stream();
uint64_t wait_limit_ns();
int num_sms();

// Waits for the work queued on s.  Every device-side wait and work loop of the sweeps is
// bounded by limit_ns, so their launches end by themselves; the host still gives up after
// (launches + 1) x 64 x limit_ns of wall time and returns NK_ERR_TIMEOUT, so that a call
// never blocks its caller without end.
int host_wait(cudaStream_t s, int64_t launches, uint64_t limit_ns);

// ---------------------------------------------------------------- device buffers
// A growable device allocation; contents are not preserved on growth.  With a stream
// set (`st`), allocation and release are stream-ordered (cudaMallocAsync /
// cudaFreeAsync), which never synchronises the device; otherwise cudaMalloc.
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    cudaStream_t st = nullptr;
    bool stream_ordered = false;
    int ensure(size_t b);
    void release();
    template <class T> T *as() const { return static_cast<T *>(p); }
    ~DevBuf() { release(); }
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
};

// Stream-ordered temporary (cudaMallocAsync / cudaFreeAsync on the library stream).
struct Tmp {
    void *p = nullptr;
    cudaStream_t st = nullptr;
    int alloc(size_t b, cudaStream_t s);
    template <class T> T *as() const { return static_cast<T *>(p); }
    ~Tmp();
};

// ---------------------------------------------------------------- control block
// Device-resident control words of one persistent launch (grid barrier, status).
struct Ctrl {
    unsigned bar_count;
    unsigned bar_gen;
    int err;     // NK_ERR_TIMEOUT / internal abort code; 0 while running
    int ovf;     // sigma overflow seen
    int depth;   // deepest BFS level
    int td_levels;
    int bu_levels;
    int where;   // phase * 4096 + level of the first failed device-side check
    int bad_id;  // offending value of that check
    int pad[3];
};

// A betweenness call captured into a CUDA graph (sampler, persistent launches, scaling,
// status copy) with the scratch it owns, replayed by later identical calls.
struct CapturedRun {
    bool valid = false;
    uint64_t seed = 0;
    int32_t k = 0;
    int batch = 0, dir = 0, grid_ctas = 0, chunk = 0;
    bool relabel = false;
    double alpha = 0, scale = 0;
    double *scores = nullptr;
    DevBuf ws[8];
    DevBuf src, msrc, iscores;  // sources; relabelled sources and scores (relabel only)
    Ctrl *h_status = nullptr;  // pinned copy of the per-batch status words
    int nb = 0;
    uint64_t launches = 0;     // kernels one replay runs
    cudaGraphExec_t exec = nullptr;
    void reset()
    {
        if (exec) cudaGraphExecDestroy(exec);
        exec = nullptr;
        if (h_status) cudaFreeHost(h_status);
        h_status = nullptr;
        valid = false;
    }
    ~CapturedRun() { reset(); }
};

// Tuned settings remembered per graph by the autotuner.
struct Tuned {
    bool valid = false;
    int batch = 64;
    double alpha = 1.0;
    int tpv = 8;
    int chunk = 0;  // arcs per hub chunk of the batched sweep (0: kHeavyChunk)
    bool relabel = false;  // batched betweenness on the relabelled copy
};

}  // namespace nk

// The opaque graph handle of the C ABI.
struct nk_graph {
    int32_t n = 0;
    int64_t A = 0;
    int32_t max_deg = 0;
    nk::DevBuf rp;   // int32[n+1]
    nk::DevBuf col;  // int32[A] (at least 4 bytes)
    // cached per-graph scratch of the betweenness kernels; guarded by mu
    std::mutex mu;
    nk::DevBuf ws[8];
    nk::Tuned tuned;
    std::atomic<int64_t> pending{0};  // serving requests referencing this graph
    // chunk table of high-degree vertices for the batched form (built on first use)
    std::mutex heavy_mu;
    nk::DevBuf heavy[3];
    int32_t heavy_H = -1, heavy_C = 0;
    std::vector<int32_t> h_hv, h_hfirst;  // host copies of heavy[0] and heavy[1]
    nk::CapturedRun captured;             // last call captured with NK_RUN_CUDA_GRAPH
    int32_t vd_est = -1;                  // cached vertex-diameter bound (nk_rk.cu), -1 = not yet
    // a second chunk table with another chunk size, for the batched sweep only (built on demand)
    nk::DevBuf heavy_alt[3];
    int32_t heavy_alt_H = -1, heavy_alt_C = 0, heavy_alt_chunk = 0;
    nk::DevBuf wt;                        // int32[A] arc weights (nk_weighted.cu), when weighted
    bool weighted = false;
    // relabelled copy for the batched sweep (vertex v of this graph is vertex relab_perm[v] of
    // the copy), built on first use
    std::unique_ptr<nk_graph> relab;
    nk::DevBuf relab_perm;
};

namespace nk {

// ---------------------------------------------------------------- error-bounded estimate (nk_rk.cu)
// Upper bound on the vertices of a shortest path (cached on the graph).
int vertex_diameter_bound(nk_graph *g, cudaStream_t s, int32_t *vd);
// Samples for error eps with probability 1 - delta, or -1 for bad arguments.
int64_t rk_sample_count(double eps, double delta, int32_t vd);
// The r sampled pairs (src -> tgt) and the keys of their path walks.
int rk_pairs(uint64_t seed, int32_t n, int64_t r, int32_t *src, int32_t *tgt, unsigned long long *key,
             cudaStream_t s);

// ---------------------------------------------------------------- weighted graphs (nk_weighted.cu)
// Copies device weights into the graph and checks them (>= 1, equal on both arcs).
int set_weights_device(nk_graph *g, const int32_t *d_w, cudaStream_t s);
// Symmetric random weights 1 + below(stream(seed, u 2^32 + v), wmax) for the edge {u < v}.
int random_weights(nk_graph *g, uint64_t seed, int32_t wmax, cudaStream_t s);

// ---------------------------------------------------------------- primitives (nk_core.cu)
// Exclusive prefix sum of count int64 values (in may equal out); *total (device, may be
// null) receives the sum.  Stream-ordered on st.
int scan_exclusive_i64(const int64_t *in, int64_t *out, int64_t count, int64_t *total,
                       cudaStream_t st);

// ---------------------------------------------------------------- high-degree vertices
// Rows longer than kHeavyChunk arcs are processed as chunks of kHeavyChunk arcs by
// different warps (partial sums reduced in chunk order), so that one hub does not keep
// one warp busy while the rest of the GPU waits at the next level barrier.
constexpr int kHeavyChunk = 256;
// Builds g->heavy (vertex ids, first chunk per vertex, owner per chunk) once per graph.
int build_heavy(nk_graph *g, cudaStream_t s);
// The chunk table for `chunk` arcs per chunk (0 or kHeavyChunk: the graph's own table, else a
// second table kept for the last other size asked for).
struct HeavyView {
    const int32_t *hv, *hfirst, *chunk_h;
    int32_t H, C, chunk;
};
int heavy_view(nk_graph *g, int chunk, cudaStream_t s, HeavyView *out);
// Relabelling for the batched sweep: vertex v becomes (v * kRelabelMul) mod n, a bijection
// (kRelabelMul is a prime above 2^31, so it has no factor in common with n).  Vertex ids of
// power-law generators cluster the hubs at small ids; scattered ids spread them over the
// scan windows of the sweep's levels.
constexpr unsigned long long kRelabelMul = 2654435761ull;
int build_relabeled(nk_graph *g, cudaStream_t s);

// ---------------------------------------------------------------- CSR build (nk_graph.cu)
// Canonical CSR of the undirected edge list (u[i], v[i]) (device arrays), written into
// g->rp / g->col.  Returns NK_ERR_GRAPH for out-of-range ids.
int build_csr_from_edges(nk_graph *g, int32_t n, int64_t m, const int32_t *d_u,
                         const int32_t *d_v, cudaStream_t st);

// ---------------------------------------------------------------- sampler (nk_sample.cu)
int sample_sources_device(int32_t n, uint64_t seed, int32_t k, int32_t *d_src, cudaStream_t st);

// ---------------------------------------------------------------- sweeps
struct RunCfg {
    int mode = NK_MODE_AUTO;
    int batch = 0;
    int tpv = 0;
    int direction = NK_DIR_AUTO;
    double alpha = 0.0;
    bool time_kernels = false;
    DevBuf *ws = nullptr;  // scratch slots (8); null = the graph's cached workspace
    int grid_div = 1;      // persistent grids use 1/grid_div of the co-resident CTAs
    int grid_ctas = 0;     // if > 0: persistent grids use at most this many CTAs
    int lcap = 0;          // batched level slabs; 0 = sized from free memory
    uint64_t limit_ns = 0; // bound on device-side waits; 0 = the process-wide bound
    bool backward = true;  // false: forward sweep only
    unsigned long long *far = nullptr;    // closeness distance sums (device), or null
    unsigned long long *reach = nullptr;  // closeness reach counts (device), or null
    double *edge = nullptr;               // edge betweenness: per-arc sums (device, A), or null
    int chunk = 0;                        // batched sweep: arcs per hub chunk (0: kHeavyChunk)
    bool relabel = false;                 // betweenness entry: use the relabelled copy
    // error-bounded estimate: per source index i, the target of its random shortest path,
    // the key of the walk's random stream, and the per-vertex counts of interior vertices
    const int32_t *rk_t = nullptr;
    const unsigned long long *rk_key = nullptr;
    unsigned long long *rk_count = nullptr;
};

inline DevBuf *scratch(const RunCfg &c, nk_graph *g);

struct RunStats {
    int mode = 0, batch = 0, tpv = 0, max_depth = 0;
    int64_t launches = 0, td_levels = 0, bu_levels = 0;
    double kernel_ms = 0.0, alpha = 0.0;
};

// Per-source form (nk_source.cu).  scores (device) += scale-free dependencies of each
// source in d_src[0..k); the caller scales.  sssp mode: k = 1, scores = null, and
// d_dist/d_sigma receive the forward sweep.
int run_per_source(nk_graph *g, const int32_t *d_src, int32_t k, double *d_scores,
                   const RunCfg &cfg, RunStats *st, cudaStream_t s);
int run_sssp(nk_graph *g, int32_t src, int32_t *d_dist, uint64_t *d_sigma, cudaStream_t s);
// Dijkstra-based sweeps of k device sources (per-source persistent launches); scores (device,
// zeroed by the caller, or null for the forward sweep only) += delta.  dist_out (int64, -1
// for unreachable) and sigma_out (device, optional) receive the last source's search.
int run_weighted(nk_graph *g, const int32_t *d_src, int32_t k, double *d_scores, const RunCfg &cfg,
                 RunStats *st, cudaStream_t s, long long *dist_out, uint64_t *sigma_out);


// Batched multi-source form (nk_batch.cu).  Returns NK_OK, or an error; sources of a
// batch whose BFS is deeper than the level cap are re-run by the per-source form.
int run_batched(nk_graph *g, const int32_t *d_src, int32_t k, double *d_scores,
                const RunCfg &cfg, RunStats *st, cudaStream_t s);

// Capturable pieces of the batched form: prepare_only sizes and allocates the scratch
// (outside any stream capture); otherwise the status reset and the launches are enqueued
// without host synchronisation, and *ctrls / *nb give the per-batch status words.
int enqueue_batched(nk_graph *g, const int32_t *d_src, int32_t k, double *d_scores,
                    const RunCfg &cfg, cudaStream_t s, bool prepare_only, Ctrl **ctrls, int *nb);

// Device bytes the batched form needs for one batch of B sources on this graph.
size_t batched_bytes(const nk_graph *g, int B);

inline DevBuf *scratch(const RunCfg &c, nk_graph *g) { return c.ws ? c.ws : g->ws; }

// Device bytes of a batched run with B sources per batch and lcap level slabs.
size_t batched_bytes_lcap(const nk_graph *g, int B, int lcap);

// Stable compaction of the sources that have at least one arc: d_out[0..*d_count) (device)
// receives them in their order.  A source without arcs reaches no vertex, so its
// dependencies, its arc shares and its distance sums are all zero: the sweeps skip it.
// One CTA, no allocation (usable inside a stream capture); the ids must be in range.
int compact_sources(const nk_graph *g, const int32_t *d_src, int32_t k, int32_t *d_out, int32_t *d_count,
                    cudaStream_t s);

// Scale a device vector in place.
int scale_vector(double *d, int32_t n, double scale, cudaStream_t s);

}  // namespace nk

// Betweenness entry points of the C ABI: argument checks, host/device staging, choice
// between the per-source and the batched form, final scaling, the per-thread run
// statistics and the autotuner.
//
// Scaling (Section 3.2): exact betweenness halves the sum of all n dependency vectors
// (every unordered pair {s,t} is reached from both ends); the sampled estimate scales
// the sum over k sources by n/(2k), so that its expectation is the exact value.
#include <algorithm>
#include <vector>

#include "nk_device.cuh"
#include "nk_internal.h"

namespace nk {
namespace {

thread_local RunStats t_stats;

__global__ void k_iota(int32_t *p, int32_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        p[i] = (int32_t)i;
}

__global__ void k_check_src(const int32_t *src, int32_t k, int32_t n, int *bad)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k;
         i += (int64_t)gridDim.x * blockDim.x)
        if ((unsigned)src[i] >= (unsigned)n) atomicOr(bad, 1);
}

// ids of the relabelled copy: out[i] = perm[in[i]]
__global__ void k_map_ids(const int32_t *perm, const int32_t *in, int32_t k, int32_t *out)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = perm[in[i]];
}

// scores back to the caller's ids: out[v] = in[perm[v]]
__global__ void k_gather_scores(const int32_t *perm, const double *in, int32_t n, double *out)
{
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        out[v] = in[perm[v]];
}

int grid_of(int64_t items) { return (int)std::max<int64_t>(1, std::min<int64_t>((items + 255) / 256, 8LL * num_sms())); }

RunCfg cfg_of(const nk_run_opts *o, const nk_graph *g)
{
    RunCfg c;
    if (o) {
        c.mode = o->mode;
        c.batch = o->batch;
        c.tpv = o->tpv;
        c.direction = o->direction;
        c.alpha = o->alpha;
        c.time_kernels = (o->flags & NK_RUN_TIME_KERNELS) != 0;
        c.grid_ctas = o->grid_ctas;
        c.chunk = o->chunk;
    }
    if (c.alpha <= 0 && g->tuned.valid) c.alpha = g->tuned.alpha;
    if (c.chunk == 0 && g->tuned.valid) c.chunk = g->tuned.chunk;
    const uint32_t fl = o ? o->flags : 0u;
    c.relabel = (fl & NK_RUN_RELABEL) ? true : (fl & NK_RUN_NO_RELABEL) ? false : (g->tuned.valid && g->tuned.relabel);
    return c;
}

int check_cfg(const RunCfg &c)
{
    if (c.mode < NK_MODE_AUTO || c.mode > NK_MODE_BATCHED) return set_error(NK_ERR_ARG, "bad mode %d", c.mode);
    if (c.direction < NK_DIR_AUTO || c.direction > NK_DIR_BOTTOM_UP) return set_error(NK_ERR_ARG, "bad direction %d", c.direction);
    if (c.batch != 0 && c.batch != 64 && c.batch != 128 && c.batch != 256) return set_error(NK_ERR_ARG, "batch must be 0, 64, 128 or 256");
    if (c.tpv != 0 && (c.tpv < 1 || c.tpv > 32 || (c.tpv & (c.tpv - 1)))) return set_error(NK_ERR_ARG, "tpv must be 0 or a power of two <= 32");
    if (!(c.alpha >= 0)) return set_error(NK_ERR_ARG, "alpha must be >= 0");
    if (c.grid_ctas < 0) return set_error(NK_ERR_ARG, "grid_ctas must be >= 0");
    if (c.chunk != 0 && (c.chunk < 32 || c.chunk > 4096 || c.chunk % 32))
        return set_error(NK_ERR_ARG, "chunk must be 0 or a multiple of 32 in [32, 4096]");
    return NK_OK;
}

// scores (device, zeroed here) += dependencies of the k device sources, then *= scale
int run_device(nk_graph *g, const int32_t *d_src, int32_t k, double scale, double *d_scores,
               const RunCfg &cfg, cudaStream_t s)
{
    const bool batched = cfg.mode == NK_MODE_BATCHED || (cfg.mode == NK_MODE_AUTO && k >= 16);
    if (cfg.relabel && batched && !cfg.ws && build_relabeled(g, s) == NK_OK) {
        // the same sweep on the relabelled copy: sources mapped in, scores gathered back
        Tmp msrc, isc;
        NK_TRY(msrc.alloc(sizeof(int32_t) * (size_t)k, s));
        NK_TRY(isc.alloc(sizeof(double) * (size_t)g->n, s));
        const int32_t *perm = g->relab_perm.as<int32_t>();
        k_map_ids<<<grid_of(k), 256, 0, s>>>(perm, d_src, k, msrc.as<int32_t>());
        ::nk::count_launch();
        RunCfg c2 = cfg;
        c2.relabel = false;
        if (c2.batch == 0 && g->tuned.valid) c2.batch = g->tuned.batch;  // the copy is not tuned itself
        NK_TRY(run_device(g->relab.get(), msrc.as<int32_t>(), k, scale, isc.as<double>(), c2, s));
        k_gather_scores<<<grid_of(g->n), 256, 0, s>>>(perm, isc.as<double>(), g->n, d_scores);
        ::nk::count_launch();
        NK_CUDA(cudaGetLastError());
        return NK_OK;
    }
    NK_CUDA(cudaMemsetAsync(d_scores, 0, sizeof(double) * g->n, s));
    t_stats = RunStats();
    int mode = cfg.mode;
    if (mode == NK_MODE_AUTO) mode = k >= 16 ? NK_MODE_BATCHED : NK_MODE_PER_SOURCE;
    int rc;
    if (mode == NK_MODE_BATCHED) {
        rc = run_batched(g, d_src, k, d_scores, cfg, &t_stats, s);
        if (rc == NK_ERR_NOMEM && cfg.mode == NK_MODE_AUTO) {
            NK_CUDA(cudaMemsetAsync(d_scores, 0, sizeof(double) * g->n, s));
            t_stats = RunStats();
            rc = run_per_source(g, d_src, k, d_scores, cfg, &t_stats, s);
        }
    } else {
        rc = run_per_source(g, d_src, k, d_scores, cfg, &t_stats, s);
    }
    if (rc != NK_OK) return rc;
    return scale_vector(d_scores, g->n, scale, s);
}

// Sampled, batched, device-pointer call through a captured CUDA graph (NK_RUN_CUDA_GRAPH).
// Returns NK_PENDING when the captured run cannot give the result (a BFS deeper than its
// level slabs): the caller then takes the regular path.
int run_captured(nk_graph *g, uint64_t seed, int32_t k, double scale, double *d_scores,
                 RunCfg cfg, cudaStream_t caller)
{
    // the legacy default stream cannot be captured: work on a private stream of this
    // thread instead, after the caller's stream has drained (the call is synchronous)
    thread_local cudaStream_t own = nullptr;
    cudaStream_t s = caller;
    if (caller == nullptr || caller == cudaStreamLegacy || caller == cudaStreamPerThread) {
        if (!own) NK_CUDA(cudaStreamCreateWithFlags(&own, cudaStreamNonBlocking));
        NK_CUDA(cudaStreamSynchronize(caller));
        s = own;
    }
    CapturedRun &e = g->captured;
    if (cfg.batch == 0) cfg.batch = g->tuned.valid ? g->tuned.batch : 64;
    if (cfg.alpha <= 0) cfg.alpha = 1.0;
    cfg.ws = e.ws;
    if (cfg.relabel && build_relabeled(g, s) != NK_OK) cfg.relabel = false;
    // with relabelling the sweep runs on the copy: sources mapped in, scores gathered back
    nk_graph *gr = cfg.relabel ? g->relab.get() : g;
    const bool hit = e.valid && e.seed == seed && e.k == k && e.batch == cfg.batch &&
                     e.alpha == cfg.alpha && e.dir == cfg.direction && e.scores == d_scores &&
                     e.scale == scale && e.grid_ctas == cfg.grid_ctas && e.chunk == cfg.chunk &&
                     e.relabel == cfg.relabel;
    if (!hit) {
        e.reset();
        NK_TRY(e.src.ensure(sizeof(int32_t) * k));
        if (cfg.relabel) {
            NK_TRY(e.msrc.ensure(sizeof(int32_t) * k));
            NK_TRY(e.iscores.ensure(sizeof(double) * (size_t)g->n));
        }
        int32_t *sweep_src = cfg.relabel ? e.msrc.as<int32_t>() : e.src.as<int32_t>();
        double *sweep_scores = cfg.relabel ? e.iscores.as<double>() : d_scores;
        Ctrl *ctrls = nullptr;
        int nb = 0;
        NK_TRY(enqueue_batched(gr, sweep_src, k, sweep_scores, cfg, s, true, &ctrls, &nb));
        const int nbatch = (k + cfg.batch - 1) / cfg.batch;
        ::nk::count_alloc();
        NK_CUDA(cudaMallocHost(&e.h_status, sizeof(Ctrl) * nbatch));
        NK_CUDA(cudaStreamSynchronize(s));
        const uint64_t l0 = g_launches.load();
        cudaGraph_t graph = nullptr;
        NK_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        int rc = NK_OK;
        do {
            if (cudaMemsetAsync(sweep_scores, 0, sizeof(double) * g->n, s) != cudaSuccess) { rc = set_error(NK_ERR_CUDA, "memset in capture"); break; }
            if ((rc = sample_sources_device(g->n, seed, k, e.src.as<int32_t>(), s)) != NK_OK) break;
            if (cfg.relabel) {
                k_map_ids<<<grid_of(k), 256, 0, s>>>(g->relab_perm.as<int32_t>(), e.src.as<int32_t>(), k, sweep_src);
                ::nk::count_launch();
            }
            if ((rc = enqueue_batched(gr, sweep_src, k, sweep_scores, cfg, s, false, &ctrls, &nb)) != NK_OK) break;
            if ((rc = scale_vector(sweep_scores, g->n, scale, s)) != NK_OK) break;
            if (cfg.relabel) {
                k_gather_scores<<<grid_of(g->n), 256, 0, s>>>(g->relab_perm.as<int32_t>(), sweep_scores, g->n, d_scores);
                ::nk::count_launch();
            }
            if (cudaMemcpyAsync(e.h_status, ctrls, sizeof(Ctrl) * nb, cudaMemcpyDeviceToHost, s) != cudaSuccess) { rc = set_error(NK_ERR_CUDA, "status copy in capture"); break; }
        } while (false);
        const cudaError_t ce = cudaStreamEndCapture(s, &graph);
        const uint64_t captured = g_launches.load() - l0;
        g_launches.fetch_sub(captured);  // recorded, not run
        if (rc != NK_OK || ce != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            return rc != NK_OK ? rc : set_error(NK_ERR_CUDA, "stream capture failed: %s", cudaGetErrorString(ce));
        }
        const cudaError_t ie = cudaGraphInstantiate(&e.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ie != cudaSuccess) {
            e.exec = nullptr;
            return set_error(NK_ERR_CUDA, "cudaGraphInstantiate failed: %s", cudaGetErrorString(ie));
        }
        e.valid = true;
        e.seed = seed;
        e.k = k;
        e.batch = cfg.batch;
        e.alpha = cfg.alpha;
        e.dir = cfg.direction;
        e.scores = d_scores;
        e.scale = scale;
        e.grid_ctas = cfg.grid_ctas;
        e.chunk = cfg.chunk;
        e.relabel = cfg.relabel;
        e.nb = nb;
        e.launches = captured;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cfg.time_kernels) {
        NK_CUDA(cudaEventCreate(&e0));
        NK_CUDA(cudaEventCreate(&e1));
        NK_CUDA(cudaEventRecord(e0, s));
    }
    NK_CUDA(cudaGraphLaunch(e.exec, s));
    if (cfg.time_kernels) NK_CUDA(cudaEventRecord(e1, s));
    NK_CUDA(cudaStreamSynchronize(s));
    g_launches.fetch_add(e.launches);
    t_stats = RunStats();
    t_stats.mode = NK_MODE_BATCHED;
    t_stats.batch = e.batch;
    t_stats.tpv = 32;
    t_stats.launches = e.nb;
    t_stats.alpha = e.alpha;
    if (cfg.time_kernels) {
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        t_stats.kernel_ms = ms;
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    }
    bool deep = false;
    for (int i = 0; i < e.nb; ++i) {
        const Ctrl &c = e.h_status[i];
        if (c.err == NK_ERR_TIMEOUT) return set_error(NK_ERR_TIMEOUT, "captured sweep aborted: a bounded device-side wait ran out");
        if (c.ovf) return set_error(NK_ERR_OVERFLOW, "a shortest-path count exceeded 2^64 - 1");
        if (c.err != 0) deep = true;
        t_stats.max_depth = std::max(t_stats.max_depth, c.depth);
        t_stats.td_levels += c.td_levels;
        t_stats.bu_levels += c.bu_levels;
    }
    return deep ? NK_PENDING : NK_OK;
}

// Common path of every betweenness entry point.  src == nullptr means "all vertices";
// sample_k > 0 means "sample_k sources from sample_seed".
int bc_entry(const nk_graph *gc, const int32_t *src, int32_t k, bool sample, uint64_t seed,
             double scale, double *scores, const nk_run_opts *opts)
{
    if (!gc) return set_error(NK_ERR_ARG, "graph is null");
    if (!scores) return set_error(NK_ERR_ARG, "scores is null");
    nk_graph *g = const_cast<nk_graph *>(gc);  // only the cached workspace is written
    const int32_t n = g->n;
    if (k < 1 || (sample && k > n)) return set_error(NK_ERR_ARG, "need 1 <= k <= n (k=%d, n=%d)", k, n);
    RunCfg cfg = cfg_of(opts, g);
    NK_TRY(check_cfg(cfg));
    const bool dev = opts && (opts->flags & NK_RUN_DEVICE_PTRS);
    cudaStream_t s = stream();
    std::lock_guard<std::mutex> lock(g->mu);
    if (sample && dev && (opts->flags & NK_RUN_CUDA_GRAPH) && cfg.mode != NK_MODE_PER_SOURCE) {
        const int rc = run_captured(g, seed, k, scale, scores, cfg, s);
        if (rc != NK_PENDING) return rc;  // NK_PENDING: deeper than the captured slabs
    }
    Tmp dsrc, dscores, flag;
    const int32_t *d_src = nullptr;
    if (sample) {
        NK_TRY(dsrc.alloc(sizeof(int32_t) * k, s));
        NK_TRY(sample_sources_device(n, seed, k, dsrc.as<int32_t>(), s));
        d_src = dsrc.as<int32_t>();
    } else if (!src) {
        NK_TRY(dsrc.alloc(sizeof(int32_t) * k, s));
        k_iota<<<std::max(1, std::min((k + 255) / 256, 8 * num_sms())), 256, 0, s>>>(dsrc.as<int32_t>(), k);
        ::nk::count_launch();
        NK_CUDA(cudaGetLastError());
        d_src = dsrc.as<int32_t>();
    } else {
        if (dev) {
            d_src = src;
        } else {
            NK_TRY(dsrc.alloc(sizeof(int32_t) * k, s));
            NK_CUDA(cudaMemcpyAsync(dsrc.p, src, sizeof(int32_t) * k, cudaMemcpyHostToDevice, s));
            d_src = dsrc.as<int32_t>();
        }
        NK_TRY(flag.alloc(sizeof(int), s));
        NK_CUDA(cudaMemsetAsync(flag.p, 0, sizeof(int), s));
        k_check_src<<<std::max(1, std::min((k + 255) / 256, 8 * num_sms())), 256, 0, s>>>(d_src, k, n, flag.as<int>());
        ::nk::count_launch();
        int hb = 0;
        NK_CUDA(cudaMemcpyAsync(&hb, flag.p, sizeof(int), cudaMemcpyDeviceToHost, s));
        NK_CUDA(cudaStreamSynchronize(s));
        if (hb) return set_error(NK_ERR_ARG, "a source id is outside [0, %d)", n);
    }
    double *d_scores = scores;
    if (!dev) {
        NK_TRY(dscores.alloc(sizeof(double) * n, s));
        d_scores = dscores.as<double>();
    }
    NK_TRY(run_device(g, d_src, k, scale, d_scores, cfg, s));
    if (!dev) NK_CUDA(cudaMemcpyAsync(scores, d_scores, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
    NK_CUDA(cudaStreamSynchronize(s));
    return NK_OK;
}

__global__ void k_finish_closeness(const unsigned long long *far_u, const unsigned long long *reach_u,
                                   int32_t n, double scale, double *far, double *reach)
{
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        far[v] = (double)far_u[v] * scale;
        reach[v] = (double)reach_u[v] * scale;
    }
}

// Closeness entry: all vertices (exact, scale 1) or k sampled sources (scale n/k).
int closeness_entry(const nk_graph *gc, bool sample, uint64_t seed, int32_t k, double *far,
                    double *reach, const nk_run_opts *opts)
{
    if (!gc) return set_error(NK_ERR_ARG, "graph is null");
    if (!far || !reach) return set_error(NK_ERR_ARG, "far or reach is null");
    nk_graph *g = const_cast<nk_graph *>(gc);
    const int32_t n = g->n;
    if (sample && (k < 1 || k > n)) return set_error(NK_ERR_ARG, "need 1 <= k <= n (k=%d, n=%d)", k, n);
    if (!sample) k = n;
    RunCfg cfg = cfg_of(opts, g);
    NK_TRY(check_cfg(cfg));
    const bool dev = opts && (opts->flags & NK_RUN_DEVICE_PTRS);
    cudaStream_t s = stream();
    std::lock_guard<std::mutex> lock(g->mu);
    Tmp dsrc, sums, hfar, hreach;
    NK_TRY(dsrc.alloc(sizeof(int32_t) * k, s));
    if (sample) {
        NK_TRY(sample_sources_device(n, seed, k, dsrc.as<int32_t>(), s));
    } else {
        k_iota<<<std::max(1, std::min((k + 255) / 256, 8 * num_sms())), 256, 0, s>>>(dsrc.as<int32_t>(), k);
        ::nk::count_launch();
    }
    NK_TRY(sums.alloc(sizeof(unsigned long long) * 2 * (size_t)n, s));
    unsigned long long *far_u = sums.as<unsigned long long>(), *reach_u = far_u + n;
    NK_CUDA(cudaMemsetAsync(sums.p, 0, sizeof(unsigned long long) * 2 * (size_t)n, s));
    cfg.far = far_u;
    cfg.reach = reach_u;
    cfg.backward = false;
    t_stats = RunStats();
    int mode = cfg.mode == NK_MODE_AUTO ? (k >= 16 ? NK_MODE_BATCHED : NK_MODE_PER_SOURCE) : cfg.mode;
    int rc;
    if (mode == NK_MODE_BATCHED) {
        rc = run_batched(g, dsrc.as<int32_t>(), k, nullptr, cfg, &t_stats, s);
        if (rc == NK_ERR_NOMEM && cfg.mode == NK_MODE_AUTO) {
            NK_CUDA(cudaMemsetAsync(sums.p, 0, sizeof(unsigned long long) * 2 * (size_t)n, s));
            t_stats = RunStats();
            rc = run_per_source(g, dsrc.as<int32_t>(), k, nullptr, cfg, &t_stats, s);
        }
    } else {
        rc = run_per_source(g, dsrc.as<int32_t>(), k, nullptr, cfg, &t_stats, s);
    }
    NK_TRY(rc);
    double *dfar = far, *dreach = reach;
    if (!dev) {
        NK_TRY(hfar.alloc(sizeof(double) * n, s));
        NK_TRY(hreach.alloc(sizeof(double) * n, s));
        dfar = hfar.as<double>();
        dreach = hreach.as<double>();
    }
    const double scale = sample ? (double)n / (double)k : 1.0;
    k_finish_closeness<<<std::max(1, std::min((n + 255) / 256, 8 * num_sms())), 256, 0, s>>>(far_u, reach_u, n, scale, dfar, dreach);
    ::nk::count_launch();
    NK_CUDA(cudaGetLastError());
    if (!dev) {
        NK_CUDA(cudaMemcpyAsync(far, dfar, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
        NK_CUDA(cudaMemcpyAsync(reach, dreach, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
    }
    NK_CUDA(cudaStreamSynchronize(s));
    return NK_OK;
}

// Position of v in the sorted row u of (rp, col), or -1.
__device__ __forceinline__ int64_t find_arc(const int32_t *rp, const int32_t *col, int32_t u, int32_t v)
{
    int64_t b = __ldg(rp + u), e = __ldg(rp + u + 1);
    const int64_t end = e;
    while (b < e) {
        const int64_t mid = b + (e - b) / 2;
        if (__ldg(col + mid) < v) b = mid + 1; else e = mid;
    }
    return (b < end && __ldg(col + b) == v) ? b : -1;
}

// Edge scores from per-arc sums: arc j = (u, v) gets scale * (the sum of (u, v) + the sum of
// (v, u)), so both arcs of an edge hold the same value.  The sums are indexed by the arcs of
// the swept graph: the caller's graph (perm null) or its relabelled copy (rrp, rcol), whose
// vertex perm[v] is the caller's v.  The row u of j is found by binary search over rp, the
// swept arcs by binary search in their sorted rows; a missing arc sets *bad.
__global__ void k_finish_edges(const int32_t *rp, const int32_t *col, int32_t n, int64_t A,
                               const int32_t *perm, const int32_t *rrp, const int32_t *rcol,
                               const double *arc, double scale, double *out, int *bad)
{
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < A;
         j += (int64_t)gridDim.x * blockDim.x) {
        int32_t lo = 0, hi = n;  // last u with rp[u] <= j
        while (hi - lo > 1) {
            const int32_t mid = lo + (hi - lo) / 2;
            if ((int64_t)__ldg(rp + mid) <= j) lo = mid; else hi = mid;
        }
        const int32_t u = lo, v = __ldg(col + j);
        int64_t j1 = j, j2;
        if (perm) {
            const int32_t pu = __ldg(perm + u), pv = __ldg(perm + v);
            j1 = find_arc(rrp, rcol, pu, pv);
            j2 = find_arc(rrp, rcol, pv, pu);
        } else {
            j2 = find_arc(rp, col, v, u);
        }
        if (j1 < 0 || j2 < 0) {
            atomicExch(bad, 1);
            continue;
        }
        out[j] = scale * (arc[j1] + arc[j2]);
    }
}

// Edge betweenness entry: all vertices (exact, scale 1/2) or k sampled sources (scale n/(2k)).
int edge_entry(const nk_graph *gc, bool sample, uint64_t seed, int32_t k, double *edge_scores,
               const nk_run_opts *opts)
{
    if (!gc) return set_error(NK_ERR_ARG, "graph is null");
    if (!edge_scores) return set_error(NK_ERR_ARG, "edge_scores is null");
    nk_graph *g = const_cast<nk_graph *>(gc);
    const int32_t n = g->n;
    const int64_t A = g->A;
    if (sample && (k < 1 || k > n)) return set_error(NK_ERR_ARG, "need 1 <= k <= n (k=%d, n=%d)", k, n);
    if (!sample) k = n;
    RunCfg cfg = cfg_of(opts, g);
    NK_TRY(check_cfg(cfg));
    const bool dev = opts && (opts->flags & NK_RUN_DEVICE_PTRS);
    cudaStream_t s = stream();
    std::lock_guard<std::mutex> lock(g->mu);
    Tmp dsrc, arc, vsc, hout, flag;
    NK_TRY(dsrc.alloc(sizeof(int32_t) * k, s));
    if (sample) {
        NK_TRY(sample_sources_device(n, seed, k, dsrc.as<int32_t>(), s));
    } else {
        k_iota<<<std::max(1, std::min((k + 255) / 256, 8 * num_sms())), 256, 0, s>>>(dsrc.as<int32_t>(), k);
        ::nk::count_launch();
    }
    const size_t arc_bytes = sizeof(double) * (size_t)std::max<int64_t>(A, 1);
    NK_TRY(arc.alloc(arc_bytes, s));
    NK_TRY(vsc.alloc(sizeof(double) * (size_t)n, s));
    NK_TRY(flag.alloc(sizeof(int), s));
    auto zero = [&]() -> int {
        NK_CUDA(cudaMemsetAsync(arc.p, 0, arc_bytes, s));
        NK_CUDA(cudaMemsetAsync(vsc.p, 0, sizeof(double) * (size_t)n, s));
        return NK_OK;
    };
    NK_TRY(zero());
    NK_CUDA(cudaMemsetAsync(flag.p, 0, sizeof(int), s));
    cfg.edge = arc.as<double>();
    t_stats = RunStats();
    int mode = cfg.mode == NK_MODE_AUTO ? (k >= 16 ? NK_MODE_BATCHED : NK_MODE_PER_SOURCE) : cfg.mode;
    // the batched sweep may run on the relabelled copy (as the vertex scores do): sources
    // mapped in, the per-arc sums indexed by the copy's arcs and read back by k_finish_edges
    const bool relab = cfg.relabel && mode == NK_MODE_BATCHED && build_relabeled(g, s) == NK_OK;
    nk_graph *gs = relab ? g->relab.get() : g;
    Tmp msrc;
    const int32_t *sweep_src = dsrc.as<int32_t>();
    if (relab) {
        NK_TRY(msrc.alloc(sizeof(int32_t) * k, s));
        k_map_ids<<<grid_of(k), 256, 0, s>>>(g->relab_perm.as<int32_t>(), dsrc.as<int32_t>(), k, msrc.as<int32_t>());
        ::nk::count_launch();
        sweep_src = msrc.as<int32_t>();
        if (cfg.batch == 0 && g->tuned.valid) cfg.batch = g->tuned.batch;  // the copy is not tuned itself
    }
    int rc;
    if (mode == NK_MODE_BATCHED) {
        rc = run_batched(gs, sweep_src, k, vsc.as<double>(), cfg, &t_stats, s);
        if (rc == NK_ERR_NOMEM && cfg.mode == NK_MODE_AUTO) {
            NK_TRY(zero());
            t_stats = RunStats();
            rc = run_per_source(gs, sweep_src, k, vsc.as<double>(), cfg, &t_stats, s);
        }
    } else {
        rc = run_per_source(gs, sweep_src, k, vsc.as<double>(), cfg, &t_stats, s);
    }
    NK_TRY(rc);
    double *dout = edge_scores;
    if (!dev) {
        NK_TRY(hout.alloc(arc_bytes, s));
        dout = hout.as<double>();
    }
    const double scale = sample ? (double)n / (2.0 * (double)k) : 0.5;
    if (A > 0) {
        const int64_t blocks = std::min<int64_t>((A + 255) / 256, 16LL * num_sms());
        k_finish_edges<<<(unsigned)std::max<int64_t>(1, blocks), 256, 0, s>>>(
            g->rp.as<int32_t>(), g->col.as<int32_t>(), n, A, relab ? g->relab_perm.as<int32_t>() : nullptr,
            gs->rp.as<int32_t>(), gs->col.as<int32_t>(), arc.as<double>(), scale, dout, flag.as<int>());
        ::nk::count_launch();
        NK_CUDA(cudaGetLastError());
    }
    int hbad = 0;
    NK_CUDA(cudaMemcpyAsync(&hbad, flag.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    if (!dev && A > 0) NK_CUDA(cudaMemcpyAsync(edge_scores, dout, sizeof(double) * (size_t)A, cudaMemcpyDeviceToHost, s));
    NK_CUDA(cudaStreamSynchronize(s));
    if (hbad) return set_error(NK_ERR_GRAPH, "an arc has no reverse arc: the graph is not symmetric");
    return NK_OK;
}

__global__ void k_rk_scale(const unsigned long long *count, int32_t n, double scale, double *out)
{
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        out[v] = (double)count[v] * scale;
}

// Error-bounded estimate entry: r pairs from the vertex-diameter bound, one forward sweep
// per pair's source (batched: B pairs per launch), one random path walked back from each
// target, counts scaled by n (n - 1) / (2 r).
int rk_entry(const nk_graph *gc, double eps, double delta, uint64_t seed, double *scores,
             int64_t *samples_out, int32_t *vd_out, const nk_run_opts *opts)
{
    if (!gc) return set_error(NK_ERR_ARG, "graph is null");
    if (!scores) return set_error(NK_ERR_ARG, "scores is null");
    if (!(eps > 0.0 && eps < 1.0) || !(delta > 0.0 && delta < 1.0))
        return set_error(NK_ERR_ARG, "need 0 < epsilon < 1 and 0 < delta < 1");
    nk_graph *g = const_cast<nk_graph *>(gc);
    const int32_t n = g->n;
    RunCfg cfg = cfg_of(opts, g);
    NK_TRY(check_cfg(cfg));
    const bool dev = opts && (opts->flags & NK_RUN_DEVICE_PTRS);
    cudaStream_t s = stream();
    std::lock_guard<std::mutex> lock(g->mu);
    int32_t vd = 0;
    NK_TRY(vertex_diameter_bound(g, s, &vd));
    const int64_t r = rk_sample_count(eps, delta, vd);
    if (r < 0) return set_error(NK_ERR_ARG, "the sample count for epsilon %g, delta %g exceeds 2^31 - 1", eps, delta);
    if (samples_out) *samples_out = r;
    if (vd_out) *vd_out = vd;
    Tmp pairs, cnt, hout;
    NK_TRY(cnt.alloc(sizeof(unsigned long long) * (size_t)n, s));
    NK_CUDA(cudaMemsetAsync(cnt.p, 0, sizeof(unsigned long long) * (size_t)n, s));
    t_stats = RunStats();
    if (n >= 2) {
        NK_TRY(pairs.alloc((sizeof(int32_t) * 2 + sizeof(unsigned long long)) * (size_t)r, s));
        unsigned long long *key = pairs.as<unsigned long long>();
        int32_t *src = reinterpret_cast<int32_t *>(key + r), *tgt = src + r;
        NK_TRY(rk_pairs(seed, n, r, src, tgt, key, s));
        cfg.backward = false;
        cfg.rk_t = tgt;
        cfg.rk_key = key;
        cfg.rk_count = cnt.as<unsigned long long>();
        const int k = (int)r;
        int mode = cfg.mode == NK_MODE_AUTO ? (k >= 16 ? NK_MODE_BATCHED : NK_MODE_PER_SOURCE) : cfg.mode;
        int rc;
        if (mode == NK_MODE_BATCHED) {
            rc = run_batched(g, src, k, nullptr, cfg, &t_stats, s);
            if (rc == NK_ERR_NOMEM && cfg.mode == NK_MODE_AUTO) {
                NK_CUDA(cudaMemsetAsync(cnt.p, 0, sizeof(unsigned long long) * (size_t)n, s));
                t_stats = RunStats();
                rc = run_per_source(g, src, k, nullptr, cfg, &t_stats, s);
            }
        } else {
            rc = run_per_source(g, src, k, nullptr, cfg, &t_stats, s);
        }
        NK_TRY(rc);
    }
    double *dout = scores;
    if (!dev) {
        NK_TRY(hout.alloc(sizeof(double) * (size_t)n, s));
        dout = hout.as<double>();
    }
    const double scale = (double)n * (double)(n - 1) / (2.0 * (double)r);
    k_rk_scale<<<std::max(1, std::min((n + 255) / 256, 8 * num_sms())), 256, 0, s>>>(cnt.as<unsigned long long>(), n, scale, dout);
    ::nk::count_launch();
    NK_CUDA(cudaGetLastError());
    if (!dev) NK_CUDA(cudaMemcpyAsync(scores, dout, sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost, s));
    NK_CUDA(cudaStreamSynchronize(s));
    return NK_OK;
}

// Weighted betweenness entry (Dijkstra sweeps): all vertices (scale 1/2) or k sampled
// sources (scale n/(2k)).
int weighted_entry(const nk_graph *gc, bool sample, uint64_t seed, int32_t k, double *scores,
                   const nk_run_opts *opts)
{
    if (!gc) return set_error(NK_ERR_ARG, "graph is null");
    if (!scores) return set_error(NK_ERR_ARG, "scores is null");
    nk_graph *g = const_cast<nk_graph *>(gc);
    const int32_t n = g->n;
    if (sample && (k < 1 || k > n)) return set_error(NK_ERR_ARG, "need 1 <= k <= n (k=%d, n=%d)", k, n);
    if (!sample) k = n;
    RunCfg cfg = cfg_of(opts, g);
    NK_TRY(check_cfg(cfg));
    const bool dev = opts && (opts->flags & NK_RUN_DEVICE_PTRS);
    cudaStream_t s = stream();
    std::lock_guard<std::mutex> lock(g->mu);
    Tmp dsrc, dsc;
    NK_TRY(dsrc.alloc(sizeof(int32_t) * k, s));
    if (sample) {
        NK_TRY(sample_sources_device(n, seed, k, dsrc.as<int32_t>(), s));
    } else {
        k_iota<<<std::max(1, std::min((k + 255) / 256, 8 * num_sms())), 256, 0, s>>>(dsrc.as<int32_t>(), k);
        ::nk::count_launch();
    }
    double *d_scores = scores;
    if (!dev) {
        NK_TRY(dsc.alloc(sizeof(double) * (size_t)n, s));
        d_scores = dsc.as<double>();
    }
    NK_CUDA(cudaMemsetAsync(d_scores, 0, sizeof(double) * (size_t)n, s));
    t_stats = RunStats();
    NK_TRY(run_weighted(g, dsrc.as<int32_t>(), k, d_scores, cfg, &t_stats, s, nullptr, nullptr));
    NK_TRY(scale_vector(d_scores, n, sample ? (double)n / (2.0 * (double)k) : 0.5, s));
    if (!dev) NK_CUDA(cudaMemcpyAsync(scores, d_scores, sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost, s));
    NK_CUDA(cudaStreamSynchronize(s));
    return NK_OK;
}

}  // namespace
}  // namespace nk

using namespace nk;

extern "C" {

int nk_betweenness_exact(const nk_graph *g, double *scores)
{
    if (!g) return set_error(NK_ERR_ARG, "graph is null");
    return bc_entry(g, nullptr, g->n, false, 0, 0.5, scores, nullptr);
}

int nk_betweenness_sampled(const nk_graph *g, uint64_t seed, int32_t k, double *scores)
{
    return nk_betweenness_sampled_opts(g, seed, k, scores, nullptr);
}

int nk_betweenness_sampled_opts(const nk_graph *g, uint64_t seed, int32_t k, double *scores,
                                const nk_run_opts *opts)
{
    if (!g) return set_error(NK_ERR_ARG, "graph is null");
    if (k < 1 || k > g->n) return set_error(NK_ERR_ARG, "need 1 <= k <= n (k=%d, n=%d)", k, g->n);
    return bc_entry(g, nullptr, k, true, seed, (double)g->n / (2.0 * (double)k), scores, opts);
}

int nk_betweenness_sources(const nk_graph *g, const int32_t *src, int32_t k, double scale,
                           double *scores, const nk_run_opts *opts)
{
    if (!src) return set_error(NK_ERR_ARG, "src is null");
    return bc_entry(g, src, k, false, 0, scale, scores, opts);
}

int nk_graph_set_weights(nk_graph *g, const int32_t *w, uint32_t flags)
{
    if (!g || !w) return set_error(NK_ERR_ARG, "graph or weights is null");
    cudaStream_t s = stream();
    std::lock_guard<std::mutex> lock(g->mu);
    if (flags & NK_CSR_DEVICE_PTRS) return set_weights_device(g, w, s);
    Tmp dw;
    NK_TRY(dw.alloc(sizeof(int32_t) * (size_t)std::max<int64_t>(g->A, 1), s));
    if (g->A > 0) NK_CUDA(cudaMemcpyAsync(dw.p, w, sizeof(int32_t) * (size_t)g->A, cudaMemcpyHostToDevice, s));
    return set_weights_device(g, dw.as<int32_t>(), s);
}

int nk_graph_random_weights(nk_graph *g, uint64_t seed, int32_t wmax)
{
    if (!g) return set_error(NK_ERR_ARG, "graph is null");
    std::lock_guard<std::mutex> lock(g->mu);
    return random_weights(g, seed, wmax, stream());
}

int nk_graph_export_weights(const nk_graph *gc, int32_t *w)
{
    if (!gc || !w) return set_error(NK_ERR_ARG, "graph or output is null");
    nk_graph *g = const_cast<nk_graph *>(gc);
    std::lock_guard<std::mutex> lock(g->mu);
    if (!g->weighted) return set_error(NK_ERR_ARG, "the graph has no weights");
    cudaStream_t s = stream();
    if (g->A > 0) NK_CUDA(cudaMemcpyAsync(w, g->wt.p, sizeof(int32_t) * (size_t)g->A, cudaMemcpyDeviceToHost, s));
    NK_CUDA(cudaStreamSynchronize(s));
    return NK_OK;
}

int nk_sssp_weighted(const nk_graph *gc, int32_t src, int64_t *dist, uint64_t *sigma)
{
    if (!gc || !dist || !sigma) return set_error(NK_ERR_ARG, "null argument");
    if (src < 0 || src >= gc->n) return set_error(NK_ERR_ARG, "source %d outside [0, %d)", src, gc->n);
    nk_graph *g = const_cast<nk_graph *>(gc);
    cudaStream_t s = stream();
    std::lock_guard<std::mutex> lock(g->mu);
    const int32_t n = g->n;
    Tmp ds, out;
    NK_TRY(ds.alloc(sizeof(int32_t), s));
    NK_TRY(out.alloc(16 * (size_t)n, s));
    NK_CUDA(cudaMemcpyAsync(ds.p, &src, sizeof(int32_t), cudaMemcpyHostToDevice, s));
    long long *dd = out.as<long long>();
    uint64_t *dsig = reinterpret_cast<uint64_t *>(dd + n);
    RunCfg cfg;
    NK_TRY(run_weighted(g, ds.as<int32_t>(), 1, nullptr, cfg, nullptr, s, dd, dsig));
    NK_CUDA(cudaMemcpyAsync(dist, dd, sizeof(int64_t) * (size_t)n, cudaMemcpyDeviceToHost, s));
    NK_CUDA(cudaMemcpyAsync(sigma, dsig, sizeof(uint64_t) * (size_t)n, cudaMemcpyDeviceToHost, s));
    NK_CUDA(cudaStreamSynchronize(s));
    return NK_OK;
}

int nk_betweenness_weighted_exact(const nk_graph *g, double *scores)
{
    return weighted_entry(g, false, 0, 0, scores, nullptr);
}

int nk_betweenness_weighted_sampled(const nk_graph *g, uint64_t seed, int32_t k, double *scores,
                                    const nk_run_opts *opts)
{
    return weighted_entry(g, true, seed, k, scores, opts);
}

int nk_betweenness_rk(const nk_graph *g, double epsilon, double delta, uint64_t seed, double *scores,
                      int64_t *samples, int32_t *vertex_diameter, const nk_run_opts *opts)
{
    return rk_entry(g, epsilon, delta, seed, scores, samples, vertex_diameter, opts);
}

int nk_vertex_diameter_estimate(const nk_graph *gc, int32_t *vd)
{
    if (!gc || !vd) return set_error(NK_ERR_ARG, "graph or output is null");
    nk_graph *g = const_cast<nk_graph *>(gc);
    std::lock_guard<std::mutex> lock(g->mu);
    return vertex_diameter_bound(g, stream(), vd);
}

int nk_edge_betweenness_exact(const nk_graph *g, double *edge_scores)
{
    return edge_entry(g, false, 0, 0, edge_scores, nullptr);
}

int nk_edge_betweenness_sampled(const nk_graph *g, uint64_t seed, int32_t k, double *edge_scores,
                                const nk_run_opts *opts)
{
    return edge_entry(g, true, seed, k, edge_scores, opts);
}

int nk_closeness_exact(const nk_graph *g, double *far, double *reach)
{
    return closeness_entry(g, false, 0, 0, far, reach, nullptr);
}

int nk_closeness_sampled(const nk_graph *g, uint64_t seed, int32_t k, double *far, double *reach,
                         const nk_run_opts *opts)
{
    return closeness_entry(g, true, seed, k, far, reach, opts);
}

int nk_last_run_stats(nk_run_stats *out)
{
    if (!out) return set_error(NK_ERR_ARG, "out is null");
    out->mode = t_stats.mode;
    out->batch = t_stats.batch;
    out->tpv = t_stats.tpv;
    out->max_depth = t_stats.max_depth;
    out->launches = t_stats.launches;
    out->kernel_ms = t_stats.kernel_ms;
    out->td_levels = t_stats.td_levels;
    out->bu_levels = t_stats.bu_levels;
    out->alpha = t_stats.alpha;
    return NK_OK;
}

int nk_sssp(const nk_graph *gc, int32_t s, int32_t *dist, uint64_t *sigma)
{
    if (!gc || !dist || !sigma) return set_error(NK_ERR_ARG, "null argument");
    nk_graph *g = const_cast<nk_graph *>(gc);
    if (s < 0 || s >= g->n) return set_error(NK_ERR_ARG, "source %d outside [0, %d)", s, g->n);
    cudaStream_t st = stream();
    std::lock_guard<std::mutex> lock(g->mu);
    Tmp dd, ds;
    NK_TRY(dd.alloc(sizeof(int32_t) * g->n, st));
    NK_TRY(ds.alloc(sizeof(uint64_t) * g->n, st));
    const int rc = run_sssp(g, s, dd.as<int32_t>(), ds.as<uint64_t>(), st);
    if (rc != NK_OK && rc != NK_ERR_OVERFLOW) return rc;
    NK_CUDA(cudaMemcpyAsync(dist, dd.p, sizeof(int32_t) * g->n, cudaMemcpyDeviceToHost, st));
    NK_CUDA(cudaMemcpyAsync(sigma, ds.p, sizeof(uint64_t) * g->n, cudaMemcpyDeviceToHost, st));
    NK_CUDA(cudaStreamSynchronize(st));
    return rc;
}

int nk_autotune(const nk_graph *gc, uint64_t seed, int32_t k, nk_run_opts *best)
{
    if (!gc || !best) return set_error(NK_ERR_ARG, "null argument");
    nk_graph *g = const_cast<nk_graph *>(gc);
    if (k < 1 || k > g->n) return set_error(NK_ERR_ARG, "need 1 <= k <= n");
    cudaStream_t s = stream();
    std::lock_guard<std::mutex> lock(g->mu);
    // the sample: the first min(k, 256) of the run's own sources
    const int32_t ks = std::min<int32_t>(k, 256);
    Tmp dsrc, dsc;
    NK_TRY(dsrc.alloc(sizeof(int32_t) * k, s));
    NK_TRY(dsc.alloc(sizeof(double) * g->n, s));
    NK_TRY(sample_sources_device(g->n, seed, k, dsrc.as<int32_t>(), s));
    nk_graph *tg = g;                      // the graph trials run on
    const int32_t *tsrc = dsrc.as<int32_t>();
    auto trial = [&](int B, double alpha, double *ms_per_src, int chunk = 0) -> int {
        RunCfg c;
        c.mode = NK_MODE_BATCHED;
        c.batch = B;
        c.alpha = alpha;
        c.chunk = chunk;
        c.time_kernels = true;
        const int32_t kk = std::min<int32_t>(ks, B);
        NK_CUDA(cudaMemsetAsync(dsc.p, 0, sizeof(double) * g->n, s));
        RunStats st;
        NK_TRY(run_batched(tg, tsrc, kk, dsc.as<double>(), c, &st, s));  // warm
        st = RunStats();
        NK_TRY(run_batched(tg, tsrc, kk, dsc.as<double>(), c, &st, s));
        *ms_per_src = st.kernel_ms / kk;
        return NK_OK;
    };
    int bestB = 64;
    double bestA = 1.0, bestT = 1e30;
    for (int B : {64, 128, 256}) {
        if (B > 64 && ks < B / 2) break;
        double t = 1e30;
        const int rc = trial(B, 1.0, &t);
        if (rc == NK_ERR_NOMEM) break;
        NK_TRY(rc);
        if (t < bestT) {
            bestT = t;
            bestB = B;
        }
    }
    for (double alpha : {0.25, 4.0, 16.0}) {
        double t = 1e30;
        NK_TRY(trial(bestB, alpha, &t));
        if (t < bestT) {
            bestT = t;
            bestA = alpha;
        }
    }
    // hub chunks of 128 arcs instead of 256: better balanced levels on some graphs, more
    // partial sums on others
    int bestC = 0;
    if (g->max_deg > 128) {
        double t = 1e30;
        NK_TRY(trial(bestB, bestA, &t, 128));
        if (t < bestT) {
            bestT = t;
            bestC = 128;
        }
    }
    // the relabelled copy, where bottom-up levels often pay off
    bool bestR = false;
    if (build_relabeled(g, s) == NK_OK) {
        Tmp msrc;
        NK_TRY(msrc.alloc(sizeof(int32_t) * (size_t)k, s));
        k_map_ids<<<grid_of(k), 256, 0, s>>>(g->relab_perm.as<int32_t>(), dsrc.as<int32_t>(), k, msrc.as<int32_t>());
        ::nk::count_launch();
        tg = g->relab.get();
        tsrc = msrc.as<int32_t>();
        for (double alpha : {0.25, 4.0, 16.0}) {
            double t = 1e30;
            NK_TRY(trial(bestB, alpha, &t, bestC));
            if (t < bestT) {
                bestT = t;
                bestA = alpha;
                bestR = true;
            }
        }
        tg = g;
        tsrc = dsrc.as<int32_t>();
    }
    g->tuned.valid = true;
    g->tuned.batch = bestB;
    g->tuned.alpha = bestA;
    g->tuned.chunk = bestC;
    g->tuned.relabel = bestR;
    *best = nk_run_opts();
    best->mode = NK_MODE_BATCHED;
    best->batch = bestB;
    best->alpha = bestA;
    best->chunk = bestC;
    best->flags = bestR ? NK_RUN_RELABEL : NK_RUN_NO_RELABEL;
    return NK_OK;
}

}  // extern "C"

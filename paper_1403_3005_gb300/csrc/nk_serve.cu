// Serving runtime: continuous batching of sampled-betweenness requests.
//
// Requests (graph, seed, k) arrive at any time and wait in a FIFO.  A request is
// admitted as soon as one of `max_inflight` slots is free AND its device-state bytes
// fit in what is left of the memory budget; requests that arrive while others run are
// admitted the moment a slot and memory free up.  Each slot is a worker thread with its
// own non-blocking CUDA stream; its request's state (sampled sources, per-batch bitset
// levels, sigma/psi rows, scores) is allocated stream-ordered on that stream and freed
// when the request ends, so the work of different requests - on different graphs or on
// the same one - overlaps on the device.  A request's persistent grid is sized by its
// graph (about one CTA per 8192 arcs, at least 128, at most half of the co-resident
// CTAs): small requests stay cheap to synchronise and many run side by side, large ones
// get up to half of the GPU, so that a large request never holds the small ones back.  CSR arrays
// stay resident in the graph objects the caller owns.
//
// Latency is measured from submit to the moment the scores are in the caller's buffer.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "nk_device.cuh"
#include "nk_internal.h"

namespace nk {
namespace {

using clk = std::chrono::steady_clock;

struct Request {
    nk_req id = 0;
    nk_graph *g = nullptr;
    uint64_t seed = 0;
    int32_t k = 0;
    double *scores = nullptr;
    size_t need = 0;
    clk::time_point t_submit, t_start, t_done;
    int state = 0;  // 0 queued, 1 running, 2 done
    int rc = NK_OK;
    std::string err;
};

constexpr int kServeLcap = 64;

}  // namespace
}  // namespace nk

struct nk_server {
    nk_server_opts opts{};
    size_t budget = 0, used = 0, peak_bytes = 0;
    int batch = 128, slots = 8;
    bool batch_fixed = false;  // the caller fixed the batch width
    bool pack = true;          // pack consecutive small requests into one launch
    uint64_t limit_ns = 0;
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<nk::Request *> queue;
    std::unordered_map<nk_req, nk::Request *> reqs;
    std::vector<std::thread> workers;
    bool draining = false, stop = false;
    nk_req next_id = 1;
    int64_t submitted = 0, completed = 0, failed = 0, rejected = 0;
    int running = 0;
    int64_t peak_inflight = 0;
    int64_t launches_jobs = 0, packed = 0;  // jobs started; requests that ran in packs
    double busy_s = 0, exs = 0;
    nk::clk::time_point busy_since;
    std::vector<double> lat_ms, wait_ms, run_ms;
};

namespace nk {
namespace {

// Sources per launch for a request: the server's batch width if the caller fixed one, else
// 128 (on the mixed serving load the 128-source sweep does more per second than the
// 256-source one, whose wider gather rounds cost more than the extra launches save).  Never
// wider than k rounded up to 64.
int request_batch(const nk_server *S, const nk_graph *, int32_t k)
{
    int B = S->batch_fixed ? S->batch : 128;
    while (B > 64 && (B >> 1) >= k) B >>= 1;
    return B;
}

size_t request_bytes(const nk_graph *g, int B, int32_t k)
{
    const int lcap = std::min(kServeLcap, std::max(g->n, 4));
    return batched_bytes_lcap(g, B, lcap) + sizeof(Ctrl) * ((size_t)(k + B - 1) / B + 1) +
           sizeof(int32_t) * (size_t)k + sizeof(double) * (size_t)g->n + 4096;
}

int run_request(nk_server *S, Request *r, cudaStream_t st, double **h_buf, size_t *h_cap)
{
    nk_graph *g = r->g;
    const int32_t n = g->n;
    DevBuf ws[8];
    for (auto &b : ws) {
        b.stream_ordered = true;
        b.st = st;
    }
    Tmp dsrc, dsc;
    NK_TRY(dsrc.alloc(sizeof(int32_t) * r->k, st));
    NK_TRY(dsc.alloc(sizeof(double) * n, st));
    NK_TRY(sample_sources_device(n, r->seed, r->k, dsrc.as<int32_t>(), st));
    NK_CUDA(cudaMemsetAsync(dsc.p, 0, sizeof(double) * n, st));
    RunCfg cfg;
    cfg.mode = NK_MODE_BATCHED;
    cfg.batch = request_batch(S, g, r->k);
    cfg.ws = ws;
    // persistent grid sized by the graph: about one CTA per 8192 arcs, at least 128, at
    // most half of the co-resident CTAs (co-residency is guaranteed per launch; launches
    // that do not fit beside the running ones wait for their CTAs to free up)
    cfg.grid_ctas = (int)std::min<int64_t>(std::max<int64_t>(g->A / 8192, 128), 1 << 20);
    cfg.grid_div = 2;  // no request takes more than half of the co-resident CTAs
    cfg.lcap = std::min(kServeLcap, std::max(n, 4));
    cfg.limit_ns = S->limit_ns;
    NK_TRY(run_batched(g, dsrc.as<int32_t>(), r->k, dsc.as<double>(), cfg, nullptr, st));
    NK_TRY(scale_vector(dsc.as<double>(), n, (double)n / (2.0 * (double)r->k), st));
    if (*h_cap < (size_t)n) {
        if (*h_buf) cudaFreeHost(*h_buf);
        *h_buf = nullptr;
        *h_cap = 0;
        ::nk::count_alloc();
        NK_CUDA(cudaMallocHost(h_buf, sizeof(double) * n));
        *h_cap = n;
    }
    NK_CUDA(cudaMemcpyAsync(*h_buf, dsc.p, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
    NK_CUDA(cudaStreamSynchronize(st));
    std::copy(*h_buf, *h_buf + n, r->scores);
    return NK_OK;
}

// ---------------------------------------------------------------- packed launches
// A request is small when its graph has at most 4M arcs and k <= 256; small requests
// waiting in the queue (the first kPackLookahead entries, larger requests keep their
// order) share launches of 128 sources, up to 1024 sources per pack, on the
// block-diagonal union of their graphs: vertex ids of member r are shifted by the vertices of the members before it,
// its sources by the same amount, so the BFS trees of different members never meet and
// each member's slice of the union scores is its own result.
constexpr int64_t kSmallArcs = 4ll << 20;
constexpr int kPackWidth = 128;      // sources per launch of a pack
constexpr int kPackSources = 1024;   // sources per pack (up to eight launches)
constexpr int kPackMembers = 32;
constexpr int kPackLookahead = 64;   // queued requests a pack may pick from
constexpr int64_t kPackVertices = 4ll << 20;

bool small_request(const Request *r) { return r->g->A <= kSmallArcs && r->k <= 256; }

__global__ void k_union_rows(const int32_t *rp, int32_t n, int64_t arc_off, int32_t *rp_u)
{
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x)
        rp_u[v] = (int32_t)(rp[v] + arc_off);
}

__global__ void k_union_cols(const int32_t *col, int64_t A, int32_t vert_off, int32_t *col_u)
{
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < A;
         j += (int64_t)gridDim.x * blockDim.x)
        col_u[j] = col[j] + vert_off;
}

__global__ void k_shift(int32_t *p, int32_t count, int32_t by)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) p[i] += by;
}

__global__ void k_set_last(int32_t *rp_u, int32_t n_u, int32_t A_u) { rp_u[n_u] = A_u; }

int blocks_for(int64_t items) { return (int)std::max<int64_t>(1, std::min<int64_t>((items + 255) / 256, 4 * num_sms())); }

int run_pack(nk_server *S, const std::vector<Request *> &rs, cudaStream_t st, double **h_buf,
             size_t *h_cap)
{
    // offsets of each member in the union: vertices, arcs, sources, heavy rows, chunks
    std::vector<int64_t> voff, aoff, soff;
    int64_t n_u = 0, A_u = 0, k_u = 0;
    int32_t maxdeg = 0;
    for (Request *r : rs) {
        voff.push_back(n_u);
        aoff.push_back(A_u);
        soff.push_back(k_u);
        n_u += r->g->n;
        A_u += r->g->A;
        k_u += r->k;
        maxdeg = std::max(maxdeg, r->g->max_deg);
    }
    nk_graph u;
    u.n = (int32_t)n_u;
    u.A = A_u;
    u.max_deg = maxdeg;
    for (DevBuf *b : {&u.rp, &u.col, &u.heavy[0], &u.heavy[1], &u.heavy[2]}) {
        b->stream_ordered = true;
        b->st = st;
    }
    NK_TRY(u.rp.ensure(sizeof(int32_t) * (n_u + 1)));
    NK_TRY(u.col.ensure(sizeof(int32_t) * (A_u + 1)));
    std::vector<int32_t> hv, hfirst, chunk_h;
    for (size_t i = 0; i < rs.size(); ++i) {
        const nk_graph *g = rs[i]->g;
        k_union_rows<<<blocks_for(g->n), 256, 0, st>>>(g->rp.as<int32_t>(), g->n, aoff[i],
                                                        u.rp.as<int32_t>() + voff[i]);
        ::nk::count_launch();
        if (g->A > 0) {
            k_union_cols<<<blocks_for(g->A), 256, 0, st>>>(g->col.as<int32_t>(), g->A, (int32_t)voff[i],
                                                            u.col.as<int32_t>() + aoff[i]);
            ::nk::count_launch();
        }
        const int32_t hoff = (int32_t)hv.size(), coff = hfirst.empty() ? 0 : hfirst.back();
        if (!hfirst.empty()) hfirst.pop_back();
        for (size_t h = 0; h < g->h_hv.size(); ++h) {
            hv.push_back(g->h_hv[h] + (int32_t)voff[i]);
            hfirst.push_back(g->h_hfirst[h] + coff);
            for (int32_t c = g->h_hfirst[h]; c < g->h_hfirst[h + 1]; ++c) chunk_h.push_back(hoff + (int32_t)h);
        }
        hfirst.push_back(coff + (g->h_hfirst.empty() ? 0 : g->h_hfirst.back()));
    }
    if (hfirst.empty()) hfirst.push_back(0);
    k_set_last<<<1, 1, 0, st>>>(u.rp.as<int32_t>(), (int32_t)n_u, (int32_t)A_u);
    ::nk::count_launch();
    NK_CUDA(cudaGetLastError());
    NK_TRY(u.heavy[0].ensure(sizeof(int32_t) * std::max<size_t>(hv.size(), 1)));
    NK_TRY(u.heavy[1].ensure(sizeof(int32_t) * hfirst.size()));
    NK_TRY(u.heavy[2].ensure(sizeof(int32_t) * std::max<size_t>(chunk_h.size(), 1)));
    if (!hv.empty()) {
        NK_CUDA(cudaMemcpyAsync(u.heavy[0].p, hv.data(), sizeof(int32_t) * hv.size(), cudaMemcpyHostToDevice, st));
        NK_CUDA(cudaMemcpyAsync(u.heavy[2].p, chunk_h.data(), sizeof(int32_t) * chunk_h.size(), cudaMemcpyHostToDevice, st));
    }
    NK_CUDA(cudaMemcpyAsync(u.heavy[1].p, hfirst.data(), sizeof(int32_t) * hfirst.size(), cudaMemcpyHostToDevice, st));
    u.heavy_H = (int32_t)hv.size();
    u.heavy_C = hfirst.back();
    // sources: each member's own sample, shifted into the union's id range
    Tmp dsrc, dsc;
    NK_TRY(dsrc.alloc(sizeof(int32_t) * k_u, st));
    NK_TRY(dsc.alloc(sizeof(double) * n_u, st));
    for (size_t i = 0; i < rs.size(); ++i) {
        int32_t *p = dsrc.as<int32_t>() + soff[i];
        NK_TRY(sample_sources_device(rs[i]->g->n, rs[i]->seed, rs[i]->k, p, st));
        k_shift<<<blocks_for(rs[i]->k), 256, 0, st>>>(p, rs[i]->k, (int32_t)voff[i]);
        ::nk::count_launch();
    }
    NK_CUDA(cudaMemsetAsync(dsc.p, 0, sizeof(double) * n_u, st));
    DevBuf ws[8];
    for (auto &b : ws) {
        b.stream_ordered = true;
        b.st = st;
    }
    RunCfg cfg;
    cfg.mode = NK_MODE_BATCHED;
    cfg.batch = k_u > 64 ? kPackWidth : 64;
    cfg.ws = ws;
    cfg.grid_ctas = (int)std::min<int64_t>(std::max<int64_t>(A_u / 8192, 128), 1 << 20);
    cfg.grid_div = 2;
    cfg.lcap = std::min<int64_t>(kServeLcap, std::max<int64_t>(n_u, 4));
    cfg.limit_ns = S->limit_ns;
    NK_TRY(run_batched(&u, dsrc.as<int32_t>(), (int32_t)k_u, dsc.as<double>(), cfg, nullptr, st));
    for (size_t i = 0; i < rs.size(); ++i)
        NK_TRY(scale_vector(dsc.as<double>() + voff[i], rs[i]->g->n,
                            (double)rs[i]->g->n / (2.0 * (double)rs[i]->k), st));
    if (*h_cap < (size_t)n_u) {
        if (*h_buf) cudaFreeHost(*h_buf);
        *h_buf = nullptr;
        *h_cap = 0;
        ::nk::count_alloc();
        NK_CUDA(cudaMallocHost(h_buf, sizeof(double) * n_u));
        *h_cap = n_u;
    }
    NK_CUDA(cudaMemcpyAsync(*h_buf, dsc.p, sizeof(double) * n_u, cudaMemcpyDeviceToHost, st));
    NK_CUDA(cudaStreamSynchronize(st));
    for (size_t i = 0; i < rs.size(); ++i)
        std::copy(*h_buf + voff[i], *h_buf + voff[i] + rs[i]->g->n, rs[i]->scores);
    return NK_OK;
}

void worker(nk_server *S)
{
    cudaSetDevice(S->device);
    cudaStream_t st = nullptr;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    double *h_buf = nullptr;
    size_t h_cap = 0;
    for (;;) {
        std::vector<Request *> job;
        size_t need = 0;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_work.wait(lk, [&] {
                return S->stop || (!S->queue.empty() && S->used + S->queue.front()->need <= S->budget);
            });
            if (S->stop) break;
            job.push_back(S->queue.front());
            S->queue.pop_front();
            need = job[0]->need;
            // pack the small requests that follow, in arrival order, while they fit
            // (a pack runs kPackWidth sources wide: its members' bytes are counted at that width)
            if (S->pack && small_request(job[0])) {
                int64_t k = job[0]->k, nv = job[0]->g->n;
                size_t pneed = request_bytes(job[0]->g, kPackWidth, job[0]->k);
                int looked = 0;
                for (auto it = S->queue.begin(); it != S->queue.end() && looked < kPackLookahead &&
                                                 (int)job.size() < kPackMembers;
                     ++looked) {
                    Request *q = *it;
                    const size_t qneed = request_bytes(q->g, kPackWidth, q->k);
                    if (!small_request(q) || k + q->k > kPackSources || nv + q->g->n > kPackVertices ||
                        S->used + pneed + qneed > S->budget) {
                        ++it;
                        continue;
                    }
                    job.push_back(q);
                    it = S->queue.erase(it);
                    k += q->k;
                    nv += q->g->n;
                    pneed += qneed;
                }
                if (job.size() > 1) need = pneed;
            }
            S->used += need;
            S->peak_bytes = std::max(S->peak_bytes, S->used);
            const auto now = clk::now();
            if (S->running++ == 0) S->busy_since = now;
            S->peak_inflight = std::max<int64_t>(S->peak_inflight, S->running);
            for (Request *r : job) {
                r->t_start = now;
                r->state = 1;
            }
            ++S->launches_jobs;
            if (job.size() > 1) S->packed += (int64_t)job.size();
        }
        const int rc = job.size() == 1 ? run_request(S, job[0], st, &h_buf, &h_cap)
                                       : run_pack(S, job, st, &h_buf, &h_cap);
        const std::string msg = rc == NK_OK ? std::string() : std::string(nk_last_error());
        {
            std::lock_guard<std::mutex> lk(S->mu);
            const auto done = clk::now();
            S->used -= need;
            if (--S->running == 0) S->busy_s += std::chrono::duration<double>(done - S->busy_since).count();
            for (Request *r : job) {
                r->t_done = done;
                r->rc = rc;
                r->err = msg;
                r->state = 2;
                if (rc == NK_OK) {
                    ++S->completed;
                    S->lat_ms.push_back(std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count());
                    S->wait_ms.push_back(std::chrono::duration<double, std::milli>(r->t_start - r->t_submit).count());
                    S->run_ms.push_back(std::chrono::duration<double, std::milli>(r->t_done - r->t_start).count());
                    S->exs += (double)(r->g->A / 2) * (double)r->k;
                } else {
                    ++S->failed;
                }
                r->g->pending.fetch_sub(1);
            }
        }
        S->cv_done.notify_all();
        S->cv_work.notify_all();
    }
    if (h_buf) cudaFreeHost(h_buf);
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
}

double pct(std::vector<double> v, double p)
{
    if (v.empty()) return 0.0;
    std::sort(v.begin(), v.end());
    // nearest-rank percentile
    size_t idx = (size_t)std::ceil(p / 100.0 * (double)v.size());
    idx = std::min(std::max<size_t>(idx, 1), v.size());
    return v[idx - 1];
}

}  // namespace
}  // namespace nk

using namespace nk;

extern "C" {

int nk_server_create(const nk_server_opts *opts, nk_server **out)
{
    if (!out) return set_error(NK_ERR_ARG, "out is null");
    *out = nullptr;
    nk_server_opts o{};
    if (opts) o = *opts;
    if (o.batch != 0 && o.batch != 64 && o.batch != 128 && o.batch != 256)
        return set_error(NK_ERR_ARG, "batch must be 0, 64, 128 or 256");
    if (o.max_inflight < 0 || o.max_inflight > 64) return set_error(NK_ERR_ARG, "max_inflight must be in [0, 64]");
    if (!(o.mem_budget_bytes >= 0) || !(o.timeout_s >= 0)) return set_error(NK_ERR_ARG, "negative budget or timeout");
    nk_server *S = new (std::nothrow) nk_server();
    if (!S) return set_error(NK_ERR_NOMEM, "host allocation failed");
    S->opts = o;
    NK_CUDA(cudaGetDevice(&S->device));
    size_t free_b = 0, total_b = 0;
    NK_CUDA(cudaMemGetInfo(&free_b, &total_b));
    S->budget = o.mem_budget_bytes > 0 ? (size_t)o.mem_budget_bytes : (size_t)(0.6 * (double)free_b);
    S->slots = o.max_inflight > 0 ? o.max_inflight : 8;
    S->batch = o.batch > 0 ? o.batch : 128;
    S->batch_fixed = o.batch > 0;
    S->pack = o.no_pack == 0;
    S->limit_ns = o.timeout_s > 0 ? (uint64_t)(o.timeout_s * 1e9) : 0;
    for (int i = 0; i < S->slots; ++i) S->workers.emplace_back(worker, S);
    *out = S;
    return NK_OK;
}

void nk_server_destroy(nk_server *S)
{
    if (!S) return;
    {
        std::unique_lock<std::mutex> lk(S->mu);
        S->draining = true;
        S->cv_done.wait(lk, [&] { return S->queue.empty() && S->running == 0; });
        S->stop = true;
    }
    S->cv_work.notify_all();
    for (auto &t : S->workers) t.join();
    for (auto &kv : S->reqs) delete kv.second;
    delete S;
}

int nk_serve_submit(nk_server *S, const nk_graph *gc, uint64_t seed, int32_t k, double *scores,
                    nk_req *id)
{
    if (!S || !gc || !scores || !id) return set_error(NK_ERR_ARG, "null argument");
    nk_graph *g = const_cast<nk_graph *>(gc);
    if (k < 1 || k > g->n) return set_error(NK_ERR_ARG, "need 1 <= k <= n (k=%d, n=%d)", k, g->n);
    Request *r = new (std::nothrow) Request();
    if (!r) return set_error(NK_ERR_NOMEM, "host allocation failed");
    r->g = g;
    r->seed = seed;
    r->k = k;
    r->scores = scores;
    r->need = request_bytes(g, request_batch(S, g, k), k);
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->draining) {
            delete r;
            return set_error(NK_ERR_SHUTDOWN, "server is shutting down");
        }
        if (r->need > S->budget) {
            ++S->rejected;
            const size_t need = r->need;
            delete r;
            return set_error(NK_ERR_NOMEM, "request needs %zu device bytes, budget is %zu", need, S->budget);
        }
        r->id = S->next_id++;
        r->t_submit = clk::now();
        g->pending.fetch_add(1);
        S->queue.push_back(r);
        S->reqs[r->id] = r;
        ++S->submitted;
        *id = r->id;
    }
    S->cv_work.notify_one();
    return NK_OK;
}

int nk_serve_poll(nk_server *S, nk_req id)
{
    if (!S) return set_error(NK_ERR_ARG, "server is null");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(id);
    if (it == S->reqs.end()) return set_error(NK_ERR_ARG, "unknown request %lld", (long long)id);
    Request *r = it->second;
    if (r->state != 2) return NK_PENDING;
    const int rc = r->rc;
    if (rc != NK_OK) set_error(rc, "%s", r->err.c_str());
    S->reqs.erase(it);
    delete r;
    return rc;
}

int nk_serve_wait(nk_server *S, nk_req id, double timeout_s)
{
    if (!S) return set_error(NK_ERR_ARG, "server is null");
    {
        std::unique_lock<std::mutex> lk(S->mu);
        auto it = S->reqs.find(id);
        if (it == S->reqs.end()) return set_error(NK_ERR_ARG, "unknown request %lld", (long long)id);
        Request *r = it->second;
        const auto dl = clk::now() + std::chrono::duration_cast<clk::duration>(std::chrono::duration<double>(timeout_s));
        if (!S->cv_done.wait_until(lk, dl, [&] { return r->state == 2; })) return NK_PENDING;
    }
    return nk_serve_poll(S, id);
}

int nk_server_get_stats(nk_server *S, nk_server_stats *out)
{
    if (!S || !out) return set_error(NK_ERR_ARG, "null argument");
    std::lock_guard<std::mutex> lk(S->mu);
    out->submitted = S->submitted;
    out->completed = S->completed;
    out->failed = S->failed;
    out->rejected = S->rejected;
    out->p50_ms = pct(S->lat_ms, 50);
    out->p99_ms = pct(S->lat_ms, 99);
    out->max_ms = S->lat_ms.empty() ? 0.0 : *std::max_element(S->lat_ms.begin(), S->lat_ms.end());
    double busy = S->busy_s;
    if (S->running > 0) busy += std::chrono::duration<double>(clk::now() - S->busy_since).count();
    out->busy_s = busy;
    out->edges_x_sources = S->exs;
    out->peak_inflight = S->peak_inflight;
    out->peak_bytes = (double)S->peak_bytes;
    out->queue_p50_ms = pct(S->wait_ms, 50);
    out->queue_p99_ms = pct(S->wait_ms, 99);
    out->run_p50_ms = pct(S->run_ms, 50);
    out->run_p99_ms = pct(S->run_ms, 99);
    out->jobs = S->launches_jobs;
    out->packed_requests = S->packed;
    return NK_OK;
}

}  // extern "C"

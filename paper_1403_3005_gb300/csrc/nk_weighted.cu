// Weighted betweenness: Brandes' algorithm with Dijkstra's shortest-path search (Section 3.4:
// BFS serves unweighted graphs and Dijkstra's algorithm weighted ones; Section 2.3: graphs
// are optionally weighted).  Weights are positive integers stored per arc, equal on both
// arcs of an edge, so path lengths are exact and equal-length paths tie exactly.
//
// One persistent cooperative launch per source settles the vertices in buckets of equal
// distance, in increasing order (the parallel form of Dijkstra's algorithm with a bucket per
// distinct distance; with weights >= 1, a vertex's predecessors all lie in earlier buckets):
//   scan     every vertex with dist == D joins bucket D (appended to the settle order);
//            the smallest tentative distance above D is noted
//   settle   each bucket vertex pulls sigma = sum of sigma[u] over neighbours u with
//            dist[u] + w(u, v) = D, and relaxes its arcs: dist[x] = min(dist[x], D + w)
//            (atomicMin), noting each new tentative distance
//   next D = the smallest noted distance; the search ends when there is none.
// Relaxation only lowers distances above D, so it never disturbs the sigma pull of the same
// phase.  Backward, bucket by bucket from the last: acc = sum of psi[x] over neighbours x
// with dist[x] = dist[v] + w(v, x); delta = sigma * acc, psi = 1/sigma + acc (double-single
// as in the unweighted sweeps), scores[v] += delta for v != s.
#include <cooperative_groups.h>

#include <algorithm>
#include <climits>

#include "nk_device.cuh"
#include "nk_internal.h"

namespace nk {
namespace {

constexpr int kThreads = 512;
constexpr long long kInf = LLONG_MAX;

struct WArgs {
    int32_t n;
    const int32_t *rp, *col, *w;
    const int32_t *src;      // the source is *src
    long long *dist;         // [n]
    unsigned long long *sp;  // [n] sigma, then psi (double-single)
    int32_t *order;          // [n] settle order
    int32_t *bcnt;           // [n + 3] vertices of bucket b
    int32_t *boff;           // [n + 3] start of bucket b in order
    long long *bnext;        // [n + 3] smallest tentative distance noted in iteration b
    long long *bdist;        // [n + 3] distance of bucket b
    double *scores;          // += delta (null: forward only)
    Ctrl *ctrl;
    uint64_t limit_ns;
    // rows longer than kHeavyChunk arcs are split into chunks handled by different warps
    const int32_t *hv, *hfirst, *chunk_h;
    int32_t H, C;
    unsigned long long *part;  // [C] per-chunk psi partial sums (double-single)
};

__device__ __forceinline__ bool heavy(const WArgs &a, int v)
{
    return a.H > 0 && __ldg(a.rp + v + 1) - __ldg(a.rp + v) > kHeavyChunk;
}

// Chunk c of a heavy vertex: its vertex h and arc range [j0, j1).
__device__ __forceinline__ void chunk_of(const WArgs &a, long long c, int &h, int &j0, int &j1)
{
    const int i = __ldg(a.chunk_h + c);
    h = __ldg(a.hv + i);
    j0 = __ldg(a.rp + h) + (int)(c - __ldg(a.hfirst + i)) * kHeavyChunk;
    j1 = min(j0 + kHeavyChunk, __ldg(a.rp + h + 1));
}

__device__ __forceinline__ long long ld_dist(const long long *p)
{
    return *reinterpret_cast<const volatile long long *>(p);
}

__global__ void __launch_bounds__(kThreads) k_wsource(WArgs a)
{
    __shared__ long long s_min;
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nthr = (long long)gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    const long long wid = tid >> 5, nw = nthr >> 5;
    const int s = __ldg(a.src);
    bool ovf = false;
    for (long long v = tid; v < a.n; v += nthr) {
        a.dist[v] = v == s ? 0 : kInf;
        a.sp[v] = v == s ? 1ull : 0ull;
    }
    if (tid < 3) {
        a.bcnt[tid] = 0;
        a.bnext[tid] = kInf;
    }
    if (!dev::grid_barrier(a.ctrl, a.limit_ns)) return;
    long long D = 0;
    int b = 0, qtail = 0;
    for (;;) {
        // ---- scan: bucket D joins the settle order; smallest tentative distance above D
        if (threadIdx.x == 0) s_min = kInf;
        if (tid == 0) {
            a.bcnt[b + 2] = 0;
            a.bnext[b + 2] = kInf;
        }
        __syncthreads();
        long long mymin = kInf;
        for (long long base = (tid & ~31LL); base < a.n; base += nthr) {
            const long long v = base + lane;
            long long dv = kInf;
            if (v < a.n) dv = a.dist[v];
            const bool in = dv == D;
            if (dv > D && dv < mymin) mymin = dv;
            const unsigned m = __ballot_sync(0xffffffffu, in);
            if (m) {
                int pos = 0;
                if (lane == 0) pos = atomicAdd(a.bcnt + b, __popc(m));
                pos = __shfl_sync(0xffffffffu, pos, 0);
                if (in) a.order[qtail + pos + __popc(m & dev::lanemask_lt())] = (int)v;
            }
        }
        atomicMin(&s_min, mymin);
        __syncthreads();
        if (threadIdx.x == 0 && s_min < kInf) atomicMin(a.bnext + b, s_min);
        if (tid == 0) {
            a.boff[b] = qtail;
            a.bdist[b] = D;
        }
        if (!dev::grid_barrier(a.ctrl, a.limit_ns)) return;
        const int nb = dev::ldcg(a.bcnt + b);
        // ---- settle: pull sigma from the predecessors, relax the arcs (warp per light
        //      vertex; heavy vertices chunk by chunk, their sigma summed with integer
        //      atomics, which are exact in any order)
        long long lmin = kInf;
        auto settle_arcs = [&](int v, int j0, int j1) -> unsigned long long {
            unsigned long long sig = 0;
            for (int j = j0 + lane; j < j1; j += 32) {
                const int x = __ldg(a.col + j);
                const long long wj = __ldg(a.w + j);
                const long long dx = ld_dist(a.dist + x);
                if (v != s && dx < D && dx + wj == D) {
                    const unsigned long long y = sig + dev::ldcg(a.sp + x);
                    ovf |= y < sig;
                    sig = y;
                }
                const long long nd = D + wj;
                if (nd < dx) {
                    atomicMin(a.dist + x, nd);
                    lmin = min(lmin, nd);
                }
            }
            return dev::group_sum_u64<32>(sig, ovf);
        };
        for (long long i = wid; i < nb; i += nw) {
            const int v = dev::ldcg(a.order + qtail + i);
            if (heavy(a, v)) continue;
            const unsigned long long sig = settle_arcs(v, __ldg(a.rp + v), __ldg(a.rp + v + 1));
            if (v != s && lane == 0) a.sp[v] = sig;
        }
        for (long long c = wid; c < a.C; c += nw) {
            int h, j0, j1;
            chunk_of(a, c, h, j0, j1);
            if (ld_dist(a.dist + h) != D) continue;
            const unsigned long long sig = settle_arcs(h, j0, j1);
            if (h != s && lane == 0 && sig != 0) {
                const unsigned long long old = atomicAdd(a.sp + h, sig);
                ovf |= old + sig < old;
            }
        }
        atomicMin(&s_min, lmin);  // s_min still holds the scan minimum of this block
        __syncthreads();
        if (threadIdx.x == 0 && s_min < kInf) atomicMin(a.bnext + b, s_min);
        if (!dev::grid_barrier(a.ctrl, a.limit_ns)) return;
        qtail += nb;
        const long long nextD = dev::ldcg(a.bnext + b);
        ++b;
        if (nextD == kInf) break;
        D = nextD;
    }
    const int nbk = b;  // buckets 0 .. nbk-1
    if (tid == 0) {
        atomicMax(&a.ctrl->depth, nbk);
    }
    if (ovf) atomicOr(&a.ctrl->ovf, 1);
    if (!a.scores) return;
    // ---- backward, last bucket first; heavy vertices sum per-chunk partials in chunk order
    auto psi_sum = [&](long long dv, int j0, int j1) {
        dev::ff acc = dev::ff_zero();
        for (int j = j0 + lane; j < j1; j += 32) {
            const int x = __ldg(a.col + j);
            if (ld_dist(a.dist + x) == dv + __ldg(a.w + j)) acc = dev::ff_add(acc, dev::ff_unpack(dev::ldcg(a.sp + x)));
        }
        return dev::group_sum_ff<32>(acc);
    };
    auto finish = [&](int v, dev::ff acc) {
        const dev::ff sv = dev::ff_from_u64(dev::ldcg(a.sp + v));
        const dev::ff delta = dev::ff_mul(sv, acc);
        a.sp[v] = dev::ff_pack(dev::ff_add(dev::ff_rcp(sv), acc));
        if (v != s && delta.hi != 0.0f) a.scores[v] += dev::ff_to_double(delta);
    };
    for (int bb = nbk - 1; bb >= 0; --bb) {
        const int off = dev::ldcg(a.boff + bb), cnt = dev::ldcg(a.bcnt + bb);
        const long long Db = dev::ldcg(a.bdist + bb);
        for (long long i = wid; i < cnt; i += nw) {
            const int v = dev::ldcg(a.order + off + i);
            if (heavy(a, v)) continue;
            const dev::ff acc = psi_sum(Db, __ldg(a.rp + v), __ldg(a.rp + v + 1));
            if (lane == 0) finish(v, acc);
        }
        if (a.H > 0) {
            for (long long c = wid; c < a.C; c += nw) {
                int h, j0, j1;
                chunk_of(a, c, h, j0, j1);
                if (ld_dist(a.dist + h) != Db) continue;
                const dev::ff acc = psi_sum(Db, j0, j1);
                if (lane == 0) a.part[c] = dev::ff_pack(acc);
            }
            if (!dev::grid_barrier(a.ctrl, a.limit_ns)) return;
            for (long long i = tid; i < a.H; i += nthr) {
                const int h = __ldg(a.hv + i);
                if (ld_dist(a.dist + h) != Db) continue;
                dev::ff acc = dev::ff_zero();
                for (int c = __ldg(a.hfirst + i); c < __ldg(a.hfirst + i + 1); ++c)
                    acc = dev::ff_add(acc, dev::ff_unpack(dev::ldcg(a.part + c)));
                finish(h, acc);
            }
        }
        if (!dev::grid_barrier(a.ctrl, a.limit_ns)) return;
    }
}

__global__ void k_dist_out(const long long *dist, int32_t n, long long *out)
{
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        out[v] = dist[v] == kInf ? -1 : dist[v];
}

// The edge {u, v} (u < v) weighs 1 + below(stream(seed, u 2^32 + v), wmax) on both arcs.
__global__ void k_random_weights(const int32_t *rp, const int32_t *col, int32_t n, uint64_t seed,
                                 int32_t wmax, int32_t *w)
{
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x)
        for (int32_t j = rp[u]; j < rp[u + 1]; ++j) {
            const uint64_t x = (uint64_t)min((int32_t)u, col[j]), y = (uint64_t)max((int32_t)u, col[j]);
            w[j] = 1 + (int32_t)dev::below(dev::stream_at(seed, (x << 32) | y), (uint64_t)wmax);
        }
}

// Weights must be >= 1 and equal on both arcs of every edge (the reverse arc is found by
// binary search in the sorted row).
__global__ void k_check_weights(const int32_t *rp, const int32_t *col, int32_t n, const int32_t *w, int *bad)
{
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x)
        for (int32_t j = rp[u]; j < rp[u + 1]; ++j) {
            const int32_t v = col[j];
            int32_t lo = rp[v], hi = rp[v + 1];
            while (lo < hi) {
                const int32_t mid = lo + (hi - lo) / 2;
                if (col[mid] < u) lo = mid + 1; else hi = mid;
            }
            if (w[j] < 1 || lo >= rp[v + 1] || col[lo] != u || w[lo] != w[j]) atomicExch(bad, 1);
        }
}

int grid_for(int64_t items) { return (int)std::max<int64_t>(1, std::min<int64_t>((items + 255) / 256, 8LL * num_sms())); }

}  // namespace

int set_weights_device(nk_graph *g, const int32_t *d_w, cudaStream_t s)
{
    const size_t bytes = sizeof(int32_t) * (size_t)std::max<int64_t>(g->A, 1);
    NK_TRY(g->wt.ensure(bytes));
    if (g->A > 0) NK_CUDA(cudaMemcpyAsync(g->wt.p, d_w, sizeof(int32_t) * (size_t)g->A, cudaMemcpyDeviceToDevice, s));
    Tmp flag;
    NK_TRY(flag.alloc(sizeof(int), s));
    NK_CUDA(cudaMemsetAsync(flag.p, 0, sizeof(int), s));
    k_check_weights<<<grid_for(g->n), 256, 0, s>>>(g->rp.as<int32_t>(), g->col.as<int32_t>(), g->n, g->wt.as<int32_t>(), flag.as<int>());
    count_launch();
    int bad = 0;
    NK_CUDA(cudaMemcpyAsync(&bad, flag.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    NK_CUDA(cudaStreamSynchronize(s));
    if (bad) {
        g->weighted = false;
        return set_error(NK_ERR_GRAPH, "weights must be >= 1 and equal on both arcs of an edge");
    }
    g->weighted = true;
    return NK_OK;
}

int random_weights(nk_graph *g, uint64_t seed, int32_t wmax, cudaStream_t s)
{
    if (wmax < 1) return set_error(NK_ERR_ARG, "wmax must be >= 1");
    NK_TRY(g->wt.ensure(sizeof(int32_t) * (size_t)std::max<int64_t>(g->A, 1)));
    k_random_weights<<<grid_for(g->n), 256, 0, s>>>(g->rp.as<int32_t>(), g->col.as<int32_t>(), g->n, seed, wmax, g->wt.as<int32_t>());
    count_launch();
    NK_CUDA(cudaGetLastError());
    NK_CUDA(cudaStreamSynchronize(s));
    g->weighted = true;
    return NK_OK;
}

// k sources (device ids), one launch each; scores (device, zeroed by the caller) += delta;
// with dist_out/sigma_out (device) and k == 1 the forward results are returned instead.
int run_weighted(nk_graph *g, const int32_t *d_src, int32_t k, double *d_scores, const RunCfg &cfg,
                 RunStats *st, cudaStream_t s, long long *dist_out, uint64_t *sigma_out)
{
    if (!g->weighted) return set_error(NK_ERR_ARG, "the graph has no weights (nk_graph_set_weights or nk_graph_random_weights)");
    const int32_t n = g->n;
    const size_t lv = (size_t)n + 3;
    Tmp buf;
    NK_TRY(build_heavy(g, s));
    const size_t C = (size_t)std::max(g->heavy_C, 0);
    const size_t bytes = 8 * (size_t)n * 2 + 4 * (size_t)n + 4 * lv * 2 + 16 * lv + 8 * (C + 1) + sizeof(Ctrl) + 64;
    NK_TRY(buf.alloc(bytes, s));
    char *p = buf.as<char>();
    WArgs a;
    a.n = n;
    a.rp = g->rp.as<int32_t>();
    a.col = g->col.as<int32_t>();
    a.w = g->wt.as<int32_t>();
    a.dist = reinterpret_cast<long long *>(p);
    a.sp = reinterpret_cast<unsigned long long *>(p + 8 * (size_t)n);
    a.bnext = reinterpret_cast<long long *>(p + 16 * (size_t)n);
    a.order = reinterpret_cast<int32_t *>(p + 16 * (size_t)n + 8 * lv);
    a.bcnt = a.order + n;
    a.boff = a.bcnt + lv;
    const size_t o_bdist = (16 * (size_t)n + 8 * lv + 4 * (size_t)n + 8 * lv + 7) & ~(size_t)7;
    a.bdist = reinterpret_cast<long long *>(p + o_bdist);
    a.part = reinterpret_cast<unsigned long long *>(p + o_bdist + 8 * lv);
    a.ctrl = reinterpret_cast<Ctrl *>(p + ((o_bdist + 8 * lv + 8 * (C + 1) + 15) & ~(size_t)15));
    a.hv = g->heavy[0].as<int32_t>();
    a.hfirst = g->heavy[1].as<int32_t>();
    a.chunk_h = g->heavy[2].as<int32_t>();
    a.H = std::max(g->heavy_H, 0);
    a.C = (int32_t)C;
    a.scores = d_scores;
    a.limit_ns = cfg.limit_ns ? cfg.limit_ns : wait_limit_ns();
    static int bps = -1;
    if (bps < 0) {
        int v = 0;
        NK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_wsource, kThreads, 0));
        bps = v;
    }
    if (bps < 1) return set_error(NK_ERR_CUDA, "weighted kernel cannot be resident");
    int grid = std::max(1, bps * num_sms() / std::max(1, cfg.grid_div));
    if (cfg.grid_ctas > 0) grid = std::min(grid, cfg.grid_ctas);
    NK_CUDA(cudaMemsetAsync(a.ctrl, 0, sizeof(Ctrl), s));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cfg.time_kernels) {
        NK_CUDA(cudaEventCreate(&e0));
        NK_CUDA(cudaEventCreate(&e1));
        NK_CUDA(cudaEventRecord(e0, s));
    }
    for (int32_t i = 0; i < k; ++i) {
        a.src = d_src + i;
        void *args[] = {&a};
        NK_CUDA(cudaLaunchCooperativeKernel((const void *)k_wsource, dim3(grid), dim3(kThreads), args, 0, s));
        count_launch();
    }
    if (cfg.time_kernels) NK_CUDA(cudaEventRecord(e1, s));
    if (dist_out) {
        k_dist_out<<<grid_for(n), 256, 0, s>>>(a.dist, n, dist_out);
        count_launch();
    }
    if (sigma_out) NK_CUDA(cudaMemcpyAsync(sigma_out, a.sp, sizeof(uint64_t) * (size_t)n, cudaMemcpyDeviceToDevice, s));
    Ctrl h;
    NK_CUDA(cudaMemcpyAsync(&h, a.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s));
    NK_CUDA(cudaStreamSynchronize(s));
    if (st) {
        st->mode = NK_MODE_PER_SOURCE;
        st->batch = 1;
        st->tpv = 32;
        st->launches += k;
        st->max_depth = std::max(st->max_depth, h.depth);
        if (cfg.time_kernels) {
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            st->kernel_ms += ms;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (h.err) return set_error(h.err, "weighted sweep aborted: a bounded grid wait ran out");
    if (h.ovf) return set_error(NK_ERR_OVERFLOW, "a shortest-path count exceeded 2^64 - 1");
    return NK_OK;
}

}  // namespace nk

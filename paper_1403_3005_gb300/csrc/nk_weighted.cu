// Weighted betweenness: Brandes' algorithm with Dijkstra's shortest-path search (Section 3.4:
// BFS serves unweighted graphs and Dijkstra's algorithm weighted ones; Section 2.3: graphs
// are optionally weighted).  Weights are positive integers stored per arc, equal on both
// arcs of an edge, so path lengths are exact and equal-length paths tie exactly.
//
// One search settles the vertices in buckets of equal distance, in increasing order (the
// parallel form of Dijkstra's algorithm with a bucket per distinct distance; with weights
// >= 1, a vertex's predecessors all lie in earlier buckets):
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
//
// A bucket holds little work for a whole GPU, so one persistent cooperative launch runs G
// searches side by side: the grid is G groups of CTAs, each group with its own state, its
// own barrier and its own score array, taking sources g, g + G, g + 2G, ...  The group score
// arrays are summed in group order afterwards, so the result does not depend on timing.
#include <cooperative_groups.h>

#include <algorithm>
#include <climits>
#include <vector>

#include "nk_device.cuh"
#include "nk_internal.h"

namespace nk {
namespace {

constexpr int kThreads = 512;
constexpr long long kInf = LLONG_MAX;

struct WArgs {
    int32_t n;
    const int32_t *rp, *col, *w;
    const int32_t *src;      // sources; group g takes src[g], src[g + G], ...
    int32_t nsrc;
    int32_t groups, cpg;     // G groups of cpg CTAs each (the grid is G * cpg CTAs)
    // per-group state, group g at offset g times the stride of each array
    long long *dist;         // [n] per group
    unsigned long long *sp;  // [n] sigma, then psi (double-single)
    int32_t *order;          // [n] settle order
    int32_t *bcnt;           // [n + 3] vertices of bucket b
    int32_t *boff;           // [n + 3] start of bucket b in order
    long long *bnext;        // [n + 3] smallest tentative distance noted in iteration b
    long long *bdist;        // [n + 3] distance of bucket b
    double *scores;          // [n] per group, += delta (null: forward only)
    unsigned long long *part;  // [C] per-chunk psi partial sums (double-single)
    Ctrl *ctrl;              // [G]
    uint64_t limit_ns;
    // rows longer than kHeavyChunk arcs are split into chunks handled by different warps
    const int32_t *hv, *hfirst, *chunk_h;
    int32_t H, C;
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

// Barrier over the `count` CTAs of one group, bounded like the grid barrier: after limit_ns
// (or 2^31 polls) the waiting CTA records NK_ERR_TIMEOUT and every CTA of the group returns
// false from then on.
__device__ __forceinline__ bool group_barrier(Ctrl *ctrl, unsigned count, uint64_t limit_ns)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned gen = dev::ld_volatile(&ctrl->bar_gen);
        __threadfence();
        const unsigned arrived = atomicAdd(&ctrl->bar_count, 1u);
        if (arrived == count - 1) {
            atomicExch(&ctrl->bar_count, 0u);
            __threadfence();
            atomicAdd(&ctrl->bar_gen, 1u);
        } else {
            const uint64_t t0 = dev::globaltimer();
            uint32_t polls = 0;
            while (dev::ld_volatile(&ctrl->bar_gen) == gen) {
                if (dev::ld_volatile(&ctrl->err) != 0) { ok = 0; break; }
                ++polls;
                if ((polls & 63u) == 0 && (dev::globaltimer() - t0 > limit_ns || polls >= 0x80000000u)) {
                    atomicCAS(&ctrl->err, 0, NK_ERR_TIMEOUT);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        if (dev::ld_volatile(&ctrl->err) != 0) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// One search from s by the CTAs of one group (a: this group's view); false if a barrier
// gave up.
__device__ bool sweep(const WArgs &a, int s, long long tid, long long nthr)
{
    __shared__ long long s_min;
    const int lane = threadIdx.x & 31;
    const long long wid = tid >> 5, nw = nthr >> 5;
    const unsigned cpg = (unsigned)a.cpg;
    bool ovf = false;
    for (long long v = tid; v < a.n; v += nthr) {
        a.dist[v] = v == s ? 0 : kInf;
        a.sp[v] = v == s ? 1ull : 0ull;
    }
    if (tid < 3) {
        a.bcnt[tid] = 0;
        a.bnext[tid] = kInf;
    }
    if (!group_barrier(a.ctrl, cpg, a.limit_ns)) return false;
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
        if (!group_barrier(a.ctrl, cpg, a.limit_ns)) return false;
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
        if (!group_barrier(a.ctrl, cpg, a.limit_ns)) return false;
        qtail += nb;
        const long long nextD = dev::ldcg(a.bnext + b);
        ++b;
        if (nextD == kInf) break;
        D = nextD;
    }
    const int nbk = b;  // buckets 0 .. nbk-1
    if (tid == 0) atomicMax(&a.ctrl->depth, nbk);
    if (ovf) atomicOr(&a.ctrl->ovf, 1);
    if (!a.scores) return true;
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
            if (!group_barrier(a.ctrl, cpg, a.limit_ns)) return false;
            for (long long i = tid; i < a.H; i += nthr) {
                const int h = __ldg(a.hv + i);
                if (ld_dist(a.dist + h) != Db) continue;
                dev::ff acc = dev::ff_zero();
                for (int c = __ldg(a.hfirst + i); c < __ldg(a.hfirst + i + 1); ++c)
                    acc = dev::ff_add(acc, dev::ff_unpack(dev::ldcg(a.part + c)));
                finish(h, acc);
            }
        }
        if (!group_barrier(a.ctrl, cpg, a.limit_ns)) return false;
    }
    return true;
}

__global__ void __launch_bounds__(kThreads, 3) k_wsource(WArgs a)
{
    const int g = blockIdx.x / a.cpg;
    if (g >= a.groups) return;  // the grid is exactly groups * cpg CTAs
    const long long lb = blockIdx.x % a.cpg;
    const long long tid = lb * blockDim.x + threadIdx.x;
    const long long nthr = (long long)a.cpg * blockDim.x;
    const size_t n = (size_t)a.n, lv = n + 3;
    WArgs v = a;  // this group's view
    v.dist += g * n;
    v.sp += g * n;
    v.order += g * n;
    v.bcnt += g * lv;
    v.boff += g * lv;
    v.bnext += g * lv;
    v.bdist += g * lv;
    if (v.scores) v.scores += g * n;
    v.part += (size_t)g * (size_t)max(a.C, 1);
    v.ctrl += g;
    for (int i = g; i < a.nsrc; i += a.groups)
        if (!sweep(v, __ldg(a.src + i), tid, nthr)) return;
}

// out[v] = sum over the groups, in group order, of the group score arrays
__global__ void k_sum_groups(const double *gs, int32_t groups, int32_t n, double *out)
{
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        double t = out[v];
        for (int32_t g = 0; g < groups; ++g) t += gs[(size_t)g * n + v];
        out[v] = t;
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

// k sources (device ids) in one launch of G groups; scores (device, zeroed by the caller,
// or null for the forward sweep only) += delta.  dist_out (int64, -1 for unreachable) and
// sigma_out (device, optional) receive the search of a single source (k == 1).
int run_weighted(nk_graph *g, const int32_t *d_src, int32_t k, double *d_scores, const RunCfg &cfg,
                 RunStats *st, cudaStream_t s, long long *dist_out, uint64_t *sigma_out)
{
    if (!g->weighted) return set_error(NK_ERR_ARG, "the graph has no weights (nk_graph_set_weights or nk_graph_random_weights)");
    const int32_t n = g->n;
    const size_t lv = (size_t)n + 3;
    NK_TRY(build_heavy(g, s));
    const size_t C = (size_t)std::max(g->heavy_C, 0);
    static int bps = -1;
    if (bps < 0) {
        int v = 0;
        NK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_wsource, kThreads, 0));
        bps = v;
    }
    if (bps < 1) return set_error(NK_ERR_CUDA, "weighted kernel cannot be resident");
    const int total = std::max(1, bps * num_sms() / std::max(1, cfg.grid_div));
    // CTAs per search: about one per 2^18 arcs (measured best on R-MAT 18 and BA 10^6 with
    // weights 1..16; a few CTAs at least, the whole grid for the largest graphs), or
    // grid_ctas when given; as many groups as fit, k at most, and their state within a
    // quarter of the free memory
    int cpg = cfg.grid_ctas > 0 ? cfg.grid_ctas
                                : (int)std::max<int64_t>(bps, std::min<int64_t>(total, (g->A + (1 << 18) - 1) >> 18));
    cpg = std::min(cpg, total);
    int groups = std::max(1, std::min(total / cpg, k));
    const size_t per_group = 16 * (size_t)n + 4 * (size_t)n + 24 * lv + 8 * (C + 1) + (d_scores ? 8 * (size_t)n : 0) + sizeof(Ctrl);
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    groups = (int)std::max<int64_t>(1, std::min<int64_t>(groups, (int64_t)(free_b / 4 / std::max<size_t>(per_group, 1))));
    if (dist_out || sigma_out) groups = 1;
    const size_t G = (size_t)groups;
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t o_dist = 0, o_sp = al(o_dist + 8 * n * G), o_bnext = al(o_sp + 8 * n * G),
                 o_bdist = al(o_bnext + 8 * lv * G), o_part = al(o_bdist + 8 * lv * G),
                 o_order = al(o_part + 8 * (C + 1) * G), o_bcnt = al(o_order + 4 * n * G),
                 o_boff = al(o_bcnt + 4 * lv * G), o_sc = al(o_boff + 4 * lv * G),
                 o_ctrl = al(o_sc + (d_scores ? 8 * n * G : 0)), bytes = al(o_ctrl + sizeof(Ctrl) * G);
    Tmp buf;
    NK_TRY(buf.alloc(bytes, s));
    char *p = buf.as<char>();
    WArgs a;
    a.n = n;
    a.rp = g->rp.as<int32_t>();
    a.col = g->col.as<int32_t>();
    a.w = g->wt.as<int32_t>();
    a.src = d_src;
    a.nsrc = k;
    a.groups = groups;
    a.cpg = cpg;
    a.dist = reinterpret_cast<long long *>(p + o_dist);
    a.sp = reinterpret_cast<unsigned long long *>(p + o_sp);
    a.bnext = reinterpret_cast<long long *>(p + o_bnext);
    a.bdist = reinterpret_cast<long long *>(p + o_bdist);
    a.part = reinterpret_cast<unsigned long long *>(p + o_part);
    a.order = reinterpret_cast<int32_t *>(p + o_order);
    a.bcnt = reinterpret_cast<int32_t *>(p + o_bcnt);
    a.boff = reinterpret_cast<int32_t *>(p + o_boff);
    a.scores = d_scores ? reinterpret_cast<double *>(p + o_sc) : nullptr;
    a.ctrl = reinterpret_cast<Ctrl *>(p + o_ctrl);
    a.hv = g->heavy[0].as<int32_t>();
    a.hfirst = g->heavy[1].as<int32_t>();
    a.chunk_h = g->heavy[2].as<int32_t>();
    a.H = std::max(g->heavy_H, 0);
    a.C = (int32_t)C;
    a.limit_ns = cfg.limit_ns ? cfg.limit_ns : wait_limit_ns();
    NK_CUDA(cudaMemsetAsync(a.ctrl, 0, sizeof(Ctrl) * G, s));
    if (a.scores) NK_CUDA(cudaMemsetAsync(a.scores, 0, 8 * n * G, s));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cfg.time_kernels) {
        NK_CUDA(cudaEventCreate(&e0));
        NK_CUDA(cudaEventCreate(&e1));
        NK_CUDA(cudaEventRecord(e0, s));
    }
    if (k > 0) {
        void *args[] = {&a};
        NK_CUDA(cudaLaunchCooperativeKernel((const void *)k_wsource, dim3(groups * cpg), dim3(kThreads), args, 0, s));
        count_launch();
    }
    if (cfg.time_kernels) NK_CUDA(cudaEventRecord(e1, s));
    if (d_scores) {
        k_sum_groups<<<grid_for(n), 256, 0, s>>>(a.scores, groups, n, d_scores);
        count_launch();
    }
    if (dist_out) {
        k_dist_out<<<grid_for(n), 256, 0, s>>>(a.dist, n, dist_out);
        count_launch();
    }
    if (sigma_out) NK_CUDA(cudaMemcpyAsync(sigma_out, a.sp, sizeof(uint64_t) * (size_t)n, cudaMemcpyDeviceToDevice, s));
    std::vector<Ctrl> h(G);
    NK_CUDA(cudaMemcpyAsync(h.data(), a.ctrl, sizeof(Ctrl) * G, cudaMemcpyDeviceToHost, s));
    NK_TRY(host_wait(s, k, a.limit_ns));  // one launch runs the k searches
    int err = 0, ovf = 0, depth = 0;
    for (const Ctrl &c : h) {
        err = err ? err : c.err;
        ovf |= c.ovf;
        depth = std::max(depth, c.depth);
    }
    if (st) {
        st->mode = NK_MODE_PER_SOURCE;
        st->batch = groups;  // searches running side by side
        st->tpv = cpg;       // CTAs per search
        st->launches += k > 0 ? 1 : 0;
        st->max_depth = std::max(st->max_depth, depth);
        if (cfg.time_kernels) {
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            st->kernel_ms += ms;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (err) return set_error(err, "weighted sweep aborted: a bounded group wait ran out");
    if (ovf) return set_error(NK_ERR_OVERFLOW, "a shortest-path count exceeded 2^64 - 1");
    return NK_OK;
}

}  // namespace nk

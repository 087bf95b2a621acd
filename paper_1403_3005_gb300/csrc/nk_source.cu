// Per-source betweenness sweep: the plain GPU form of Brandes' algorithm (Section 3.2,
// Table 1), one shortest-path tree at a time.  It is the baseline the batched form is
// measured against, and the fallback for very deep BFS trees.
//
// One cooperative (co-resident) launch per source runs every level of that source:
//   init      dist = -1, sigma = 0; dist[s] = 0, sigma[s] = 1; the bitmaps are cleared
//   forward   level-synchronous BFS (Section 3.4: BFS for unweighted graphs).  Three
//             bitmaps of n bits, small enough to stay in L2, carry the frontier: `vis`
//             (levels found so far) and the level bitmaps `lvl[d & 1]` of levels d and
//             d+1.  Every level's vertices are also appended to one queue (warp-aggregated:
//             one atomic per warp and ballot ranks), so every level can be iterated from
//             its queue segment.  Per level either
//             - top-down: warps take up to 32 frontier vertices at a time from the queue,
//               stage their ids, sigma and arc offsets in shared memory and run lanes over
//               the concatenated arc list, so that low-degree vertices do not leave lanes
//               idle; for an arc (v, w) with w not in `vis`, an atomicOr on the level-(d+1)
//               bitmap claims w (the claiming lane queues it) and sigma[v] is added to
//               sigma[w] (atomicAdd; a carry out of 64 bits is flagged), or
//             - bottom-up: every unvisited w (a bit test on `vis`, 32 vertices per word)
//               sums sigma[v] over ALL neighbours v in the level-d bitmap (no early exit:
//               sigma needs every parent) and joins level d+1 if the sum is non-zero;
//             bottom-up is chosen when alpha * (arcs of the frontier) > (arcs of the
//             unvisited vertices).  Rows longer than kHeavyChunk arcs are split into
//             chunks, read with 16-byte column loads by a warp each.
//   backward  deepest level first; the level bitmap is rebuilt for level d+1 from its
//             queue segment, and every v at level d (from its queue segment) pulls from its
//             successors (neighbours in that bitmap):
//               acc = sum_{w in N(v), dist w = d+1} psi[w],  psi = (1 + delta) / sigma,
//               delta_s(v) = sigma[v] * acc,  scores[v] += delta_s(v),
//             which is Brandes' recurrence delta(v) = sum sigma_v/sigma_w (1 + delta_w)
//             with the common factor sigma_v taken out; psi_v = 1/sigma_v + acc.  The
//             sums run in double-single arithmetic (FP32 pipe), scores in FP64.  psi
//             overwrites sigma in place once a vertex's level is done (sigma of level d is
//             still intact while level d reads psi of level d+1).
// The levels are separated by a bounded grid barrier; per-level counters live in
// arrays indexed by level, so every CTA reads the same values after a barrier.
#include <cooperative_groups.h>

#include <algorithm>
#include <climits>
#include <cstdio>
#include <cstdlib>
#include <mutex>
#include <vector>

#include "nk_device.cuh"
#include "nk_internal.h"

namespace cg = cooperative_groups;

namespace nk {
namespace {

constexpr int kThreads = 512;
constexpr unsigned FULL = 0xffffffffu;

struct SrcArgs {
    int32_t n;
    int64_t A;
    const int32_t *rp, *col;
    const int32_t *src;  // the source is *src
    int32_t *dist;
    unsigned long long *sp;  // sigma during the forward sweep, then psi (double bits)
    int32_t *queue;      // [n] the vertices of every level, level by level
    int32_t *cnt;        // cnt[d]: vertices at level d
    long long *mfa;      // mfa[d]: sum of the degrees of level d
    int32_t *qoff;       // qoff[d]: start of level d in queue
    double *scores;      // += delta_s (not touched when forward_only)
    Ctrl *ctrl;
    uint64_t limit_ns;
    double alpha;
    int dir;
    int forward_only;
    double *edge;        // [A] per-arc shares sigma_v * psi_w (edge betweenness), or null
    double *acc;         // [n] psi sums pushed into light vertices (backward push levels)
    // rows longer than kHeavyChunk: chunk table and per-chunk partial sums
    const int32_t *hv, *hfirst, *chunk_h;
    int32_t H, C;
    unsigned long long *part;
    // bitmaps of nw = ceil(n / 32) words each: vis, then the two level bitmaps
    unsigned *bits;
    int32_t nw;
    unsigned long long *trace;  // [kTraceCap][2] (code, globaltimer) after each barrier, or null
};

// Phase trace (diagnostics, NK_TRACE): CTA 0 records (level * 16 + phase, %globaltimer)
// after a grid barrier.
constexpr int kTraceCap = 512;
enum { SPH_INIT = 1, SPH_TD, SPH_BU, SPH_BU_HUBS, SPH_POST, SPH_BK_MARK, SPH_BK, SPH_BK_HUBS };

__device__ __forceinline__ void src_mark(const SrcArgs &a, int &ti, int level, int phase)
{
    if (a.trace && blockIdx.x == 0 && threadIdx.x == 0 && ti < kTraceCap) {
        a.trace[2 * ti] = (unsigned long long)(level * 16 + phase);
        a.trace[2 * ti + 1] = dev::globaltimer();
        ++ti;
    }
}

__device__ __forceinline__ int degree(const int32_t *rp, int v) { return __ldg(rp + v + 1) - __ldg(rp + v); }

// A row is processed in chunks only when a chunk table exists (a.H > 0, which holds
// exactly when some row is longer than kHeavyChunk); without one, every row is light.
__device__ __forceinline__ bool heavy(const SrcArgs &a, int v) { return a.H > 0 && degree(a.rp, v) > kHeavyChunk; }

// Chunk c of a heavy vertex: its vertex h and arc range [j0, j1).
// The arcs [j0, j1) of chunk c, whose heavy vertex is h.
__device__ __forceinline__ void chunk_range(const SrcArgs &a, long long c, int h, int &j0, int &j1)
{
    j0 = __ldg(a.rp + h) + (int)(c - __ldg(a.hfirst + __ldg(a.chunk_h + c))) * kHeavyChunk;
    j1 = min(j0 + kHeavyChunk, __ldg(a.rp + h + 1));
}

// fn(c, h, j0, j1) by the whole warp for every chunk c whose heavy vertex h passes keep(h).
// Warp w takes the chunks w + i * nwarps, so that the consecutive chunks of one hub go to
// different warps.  Its lanes test the owners of 32 of them at once and the warp then walks
// the chunks that passed: a level with few hubs on it costs a few ballots per warp instead
// of a chain of dependent loads for every chunk of the graph.
template <class Keep, class Fn> __device__ __forceinline__ void for_chunks(const SrcArgs &a, Keep keep, Fn fn)
{
    const int lane = threadIdx.x & 31;
    const long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long i0 = 0; wid + i0 * nwarps < a.C; i0 += 32) {
        const long long cl = wid + (i0 + lane) * nwarps;
        int h = -1;
        if (cl < a.C) {
            h = __ldg(a.hv + __ldg(a.chunk_h + cl));
            if (!keep(h)) h = -1;
        }
        unsigned m = __ballot_sync(FULL, h >= 0);
        while (m) {
            const int b = __ffs(m) - 1;
            m &= m - 1;
            const long long c = wid + (i0 + b) * nwarps;
            const int hb = __shfl_sync(FULL, h, b);
            int j0, j1;
            chunk_range(a, c, hb, j0, j1);
            fn(c, hb, j0, j1);
        }
    }
}

// bitmaps: vis = bits[0, nw), level bitmap p = bits[(1 + p) nw, (2 + p) nw)
__device__ __forceinline__ unsigned *vis_bits(const SrcArgs &a) { return a.bits; }
__device__ __forceinline__ unsigned *lvl_bits(const SrcArgs &a, int p) { return a.bits + (size_t)(1 + (p & 1)) * a.nw; }
// bit v of a bitmap written earlier in the launch (read from L2: L1 is not coherent)
__device__ __forceinline__ bool test_bit(const unsigned *b, int v) { return (__ldcg(b + (v >> 5)) >> (v & 31)) & 1u; }

// Appends w to level d+1's queue segment (starting at qnext): the lanes that append
// together share one atomicAdd and take ranks within the group.
__device__ __forceinline__ void queue_append(const SrcArgs &a, int d, int qnext, int w)
{
    cg::coalesced_group g = cg::coalesced_threads();
    int pos = 0;
    if (g.thread_rank() == 0) pos = atomicAdd(a.cnt + d + 1, (int)g.size());
    pos = g.shfl(pos, 0) + (int)g.thread_rank();
    if (qnext + pos < a.n) a.queue[qnext + pos] = w;
}

// Arcs (v_i, w[i]) of a top-down step from level d (w[i] < 0: none), sv[i] = sigma[v_i]: w
// joins level d+1 unless an earlier level holds it; the lane whose atomicOr sets w's bit in
// the level-(d+1) bitmap claims and queues it; every such arc adds sigma[v] to sigma[w].  The
// N arcs go through each step together (N bit loads, then N claims, then N sigma adds, each
// batch in flight at once) instead of one arc after the other.
template <int N>
__device__ __forceinline__ void td_arcs(const SrcArgs &a, int d, const int (&w)[N], const unsigned long long (&sv)[N],
                                        int qnext, unsigned long long *s_mf, bool &ovf)
{
    bool go[N];
#pragma unroll
    for (int i = 0; i < N; ++i) go[i] = w[i] >= 0 && !test_bit(vis_bits(a), w[i]);
    unsigned old[N];
#pragma unroll
    for (int i = 0; i < N; ++i) old[i] = go[i] ? atomicOr(lvl_bits(a, d + 1) + (w[i] >> 5), 1u << (w[i] & 31)) : 0u;
    unsigned long long prev[N];
#pragma unroll
    for (int i = 0; i < N; ++i) prev[i] = go[i] ? atomicAdd(a.sp + w[i], sv[i]) : 0ull;
#pragma unroll
    for (int i = 0; i < N; ++i) {
        if (go[i] && !((old[i] >> (w[i] & 31)) & 1u)) {
            a.dist[w[i]] = d + 1;
            queue_append(a, d, qnext, w[i]);
            atomicAdd(s_mf, (unsigned long long)degree(a.rp, w[i]));
        }
        ovf |= go[i] && prev[i] + sv[i] < prev[i];
    }
}

// fn(j, c) for every arc j of [j0, j1) with c = col[j], by the whole warp: a scalar head
// up to a 16-byte boundary, then 16-byte column loads (four arcs per lane), then a
// scalar tail.
template <class Fn> __device__ __forceinline__ void for_arcs_vec(const SrcArgs &a, int j0, int j1, Fn fn)
{
    const int lane = threadIdx.x & 31;
    const int b0 = min(j1, (j0 + 3) & ~3), b1 = max(b0, j1 & ~3);
    if (j0 + lane < b0) fn(j0 + lane, __ldg(a.col + j0 + lane));
    for (int q = b0 / 4 + lane; q < b1 / 4; q += 32) {
        const int4 c4 = __ldg(reinterpret_cast<const int4 *>(a.col) + q);
        fn(4 * q, c4.x);
        fn(4 * q + 1, c4.y);
        fn(4 * q + 2, c4.z);
        fn(4 * q + 3, c4.w);
    }
    if (b1 + lane < j1) fn(b1 + lane, __ldg(a.col + b1 + lane));
}

// fn(j, c) for up to four arcs at a time by the whole warp (c[i] < 0: none): 16-byte column
// loads of four arcs per lane, then the scalar head and tail (up to a 16-byte boundary)
// together.
template <class Fn> __device__ __forceinline__ void for_arcs_vec4(const SrcArgs &a, int j0, int j1, Fn fn)
{
    const int lane = threadIdx.x & 31;
    const int b0 = min(j1, (j0 + 3) & ~3), b1 = max(b0, j1 & ~3);
    for (int q = b0 / 4 + lane; q < b1 / 4; q += 32) {
        const int4 c4 = __ldg(reinterpret_cast<const int4 *>(a.col) + q);
        const int j[4] = {4 * q, 4 * q + 1, 4 * q + 2, 4 * q + 3};
        const int c[4] = {c4.x, c4.y, c4.z, c4.w};
        fn(j, c);
    }
    int j[4] = {j0 + lane, b1 + lane, 0, 0}, c[4] = {-1, -1, -1, -1};
    if (j0 + lane < b0) c[0] = __ldg(a.col + j0 + lane);
    if (b1 + lane < j1) c[1] = __ldg(a.col + b1 + lane);
    if (__any_sync(FULL, c[0] >= 0 || c[1] >= 0)) fn(j, c);
}

// ------------------------------------------------------------------ lanes over arcs
// A warp works on a group of up to 32 light vertices at a time: it stages their ids, row
// starts and arc prefix sums in shared memory (with a per-vertex value: sigma for the
// top-down push, a running sum for the pulls) and runs its 32 lanes over the concatenated
// arcs, so that low-degree vertices leave no lane idle.  The lane of arc i finds its
// vertex k by binary search over the staged prefix sums.
struct LbStage {
    int v[32];
    int beg[32];
    int pre[33];
    unsigned long long val[32];
};

// Stages the group (v = -1 or deg = 0 for no vertex) and returns its arc count.
__device__ __forceinline__ int lb_stage(LbStage &st, int v, int deg, unsigned long long val, const int32_t *rp)
{
    const int lane = threadIdx.x & 31;
    int incl = deg;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += y;
    }
    st.v[lane] = v;
    st.beg[lane] = (v >= 0 && deg > 0) ? __ldg(rp + v) : 0;
    st.pre[lane + 1] = incl;
    st.val[lane] = val;
    if (lane == 0) st.pre[0] = 0;
    __syncwarp();
    return __shfl_sync(FULL, incl, 31);
}

// The staged vertex of arc i of the group: the last k with pre[k] <= i.
__device__ __forceinline__ int lb_find(const LbStage &st, int i)
{
    int lo = 0, hi = 31;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (st.pre[mid] <= i) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Segmented sum over the lanes of one pass (lanes of the same vertex k are contiguous):
// the first lane of each run of equal k receives the run's sum, which it adds to the
// vertex's staged running sum.  x is a path count (uint64, carry out flagged) or a
// double-single pair packed in 64 bits (PSI).
template <bool PSI>
__device__ __forceinline__ void lb_seg_add(LbStage &st, int k, bool valid, unsigned long long x, bool &ovf)
{
    const int lane = threadIdx.x & 31;
    if (!valid) k = -1 - lane;  // a run of its own that adds nothing
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_down_sync(FULL, x, o);
        const int k2 = __shfl_down_sync(FULL, k, o);
        if (lane + o < 32 && k2 == k) {
            if constexpr (PSI) {
                x = dev::ff_pack(dev::ff_add(dev::ff_unpack(x), dev::ff_unpack(y)));
            } else {
                const unsigned long long z = x + y;
                ovf |= z < x;
                x = z;
            }
        }
    }
    const int kp = __shfl_up_sync(FULL, k, 1);
    if (valid && (lane == 0 || kp != k)) {
        if constexpr (PSI) {
            st.val[k] = dev::ff_pack(dev::ff_add(dev::ff_unpack(st.val[k]), dev::ff_unpack(x)));
        } else {
            const unsigned long long z = st.val[k] + x;
            ovf |= z < x;
            st.val[k] = z;
        }
    }
    __syncwarp();
}

// ------------------------------------------------------------------ top-down level d
// Light frontier vertices: groups of 32 queue entries, lanes over their arcs.

__device__ void td_level(const SrcArgs &a, int d, int qo, int nf, int qnext, unsigned long long *s_mf,
                         bool &ovf, LbStage *stages)
{
    const int lane = threadIdx.x & 31;
    LbStage &st = stages[threadIdx.x >> 5];
    const long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long base = wid * 32; base < nf; base += nwarps * 32) {
        int v = -1, deg = 0;
        if (base + lane < nf) {
            v = __ldcg(a.queue + qo + base + lane);
            if ((unsigned)v < (unsigned)a.n && !heavy(a, v)) deg = degree(a.rp, v);
            else v = -1;
        }
        const int total = lb_stage(st, v, deg, v >= 0 ? __ldcg(a.sp + v) : 0ull, a.rp);
        for (int i0 = 0; i0 < total; i0 += 64) {  // two arcs per lane at a time
            int w[2];
            unsigned long long sv[2];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int i = i0 + 32 * u + lane;
                w[u] = -1;
                sv[u] = 0ull;
                if (i < total) {
                    const int k = lb_find(st, i);
                    w[u] = __ldg(a.col + st.beg[k] + (i - st.pre[k]));
                    sv[u] = st.val[k];
                }
            }
            td_arcs<2>(a, d, w, sv, qnext, s_mf, ovf);
        }
        __syncwarp();
    }
    // heavy frontier vertices: one warp per chunk of kHeavyChunk arcs
    for_chunks(a, [&](int h) { return __ldcg(a.dist + h) == d; }, [&](long long, int h, int j0, int j1) {
        const unsigned long long s1 = __ldcg(a.sp + h);
        const unsigned long long sv[4] = {s1, s1, s1, s1};
        for_arcs_vec4(a, j0, j1, [&](const int (&)[4], const int (&w)[4]) { td_arcs<4>(a, d, w, sv, qnext, s_mf, ovf); });
    });
}

// ------------------------------------------------------------------ bottom-up level d
// Vertex w joins level d+1 with path count acc: distance, sigma, bitmaps, queue, counts.
__device__ __forceinline__ void bu_settle(const SrcArgs &a, int d, int qnext, int w, unsigned long long acc,
                                          unsigned long long *s_mf)
{
    a.dist[w] = d + 1;
    a.sp[w] = acc;
    const unsigned bit = 1u << (w & 31);
    atomicOr(lvl_bits(a, d + 1) + (w >> 5), bit);
    atomicOr(vis_bits(a) + (w >> 5), bit);  // only w's own group reads w's bit this level
    queue_append(a, d, qnext, w);
    atomicAdd(s_mf, (unsigned long long)degree(a.rp, w));
}

__device__ void bu_level(const SrcArgs &a, int d, int qnext, unsigned long long *s_mf, bool &ovf, LbStage *stages)
{
    const int lane = threadIdx.x & 31;
    LbStage &st = stages[threadIdx.x >> 5];
    const long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const unsigned *cur = lvl_bits(a, d);
    // a warp takes the 32 vertices of one word of the visited bitmap: its words are
    // wid + i * nwarps, read 32 at a time (a lane each), and the words with an unvisited
    // vertex are walked in turn
    for (long long i0 = 0; wid + i0 * nwarps < a.nw; i0 += 32) {
        const long long wl = wid + (i0 + lane) * nwarps;
        const unsigned vl = wl < a.nw ? __ldcg(vis_bits(a) + wl) : FULL;
        unsigned open = __ballot_sync(FULL, vl != FULL);
      while (open) {
        const int b = __ffs(open) - 1;
        open &= open - 1;
        const long long wd = wid + (i0 + b) * nwarps;
        const unsigned visw = __shfl_sync(FULL, vl, b);
        const long long w = wd * 32 + lane;
        const bool act = w < a.n && !((visw >> lane) & 1u) && !heavy(a, (int)w);
        const int total = lb_stage(st, act ? (int)w : -1, act ? degree(a.rp, (int)w) : 0, 0ull, a.rp);
        for (int i0 = 0; i0 < total; i0 += 64) {
            // two passes of 32 arcs at a time: both passes' column, bit and sigma loads are
            // in flight before either reduction
            int k[2], v[2];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int i = i0 + 32 * u + lane;
                k[u] = 0;
                v[u] = -1;
                if (i < total) {
                    k[u] = lb_find(st, i);
                    v[u] = __ldg(a.col + st.beg[k[u]] + (i - st.pre[k[u]]));
                }
            }
            bool on[2];
#pragma unroll
            for (int u = 0; u < 2; ++u) on[u] = v[u] >= 0 && test_bit(cur, v[u]);
            unsigned long long x[2];
#pragma unroll
            for (int u = 0; u < 2; ++u) x[u] = on[u] ? __ldcg(a.sp + v[u]) : 0ull;
            lb_seg_add<false>(st, k[0], i0 + lane < total, x[0], ovf);
            if (i0 + 32 < total) lb_seg_add<false>(st, k[1], i0 + 32 + lane < total, x[1], ovf);
        }
        if (act && st.val[lane] != 0) bu_settle(a, d, qnext, (int)w, st.val[lane], s_mf);
        __syncwarp();
      }
    }
    // heavy unvisited vertices: per-chunk partial sums (finished by bu_heavy_finish)
    for_chunks(a, [&](int h) { return !test_bit(vis_bits(a), h); }, [&](long long c, int, int j0, int j1) {
        unsigned long long acc = 0;
        for_arcs_vec(a, j0, j1, [&](int, int v) {
            if (test_bit(cur, v)) {
                const unsigned long long y = acc + __ldcg(a.sp + v);
                ovf |= y < acc;
                acc = y;
            }
        });
        acc = dev::group_sum_u64<32>(acc, ovf);
        if (lane == 0) a.part[c] = acc;
    });
}

// After a barrier: heavy unvisited vertices add their chunk sums in chunk order.
__device__ void bu_heavy_finish(const SrcArgs &a, int d, int qnext, unsigned long long *s_mf, bool &ovf)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < a.H;
         i += (long long)gridDim.x * blockDim.x) {
        const int h = __ldg(a.hv + i);
        if (test_bit(vis_bits(a), h)) continue;
        unsigned long long acc = 0;
        for (int c = __ldg(a.hfirst + i); c < __ldg(a.hfirst + i + 1); ++c) {
            const unsigned long long y = acc + __ldcg(a.part + c);
            ovf |= y < acc;
            acc = y;
        }
        if (acc != 0) bu_settle(a, d, qnext, h, acc, s_mf);
    }
}

// psi_v = 1/sigma_v + acc and delta_v = sigma_v * acc (Brandes' recurrence with sigma_v
// factored out), in double-single arithmetic; psi overwrites sigma, delta goes to the
// FP64 score.
// Level 0 (the source) is finished only for edge betweenness and gets no score.
__device__ __forceinline__ void finish_vertex(const SrcArgs &a, int v, dev::ff acc, int d)
{
    const dev::ff sv = dev::ff_from_u64(__ldcg(a.sp + v));
    const dev::ff delta = dev::ff_mul(sv, acc);
    a.sp[v] = dev::ff_pack(dev::ff_add(dev::ff_rcp(sv), acc));
    if (delta.hi != 0.0f && d > 0) a.scores[v] += dev::ff_to_double(delta);
}

// ------------------------------------------------------------------ backward level d
// The level bitmap holds level d+1.
__device__ void back_level(const SrcArgs &a, int d, int qo, int nd, LbStage *stages, bool light = true)
{
    const int lane = threadIdx.x & 31;
    LbStage &st = stages[threadIdx.x >> 5];
    const long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const unsigned *succ = lvl_bits(a, 0);
    for (long long base = wid * 32; light && base < nd; base += nwarps * 32) {
        int v = -1, deg = 0;
        if (base + lane < nd) {
            v = __ldcg(a.queue + qo + base + lane);
            if ((unsigned)v < (unsigned)a.n && !heavy(a, v)) deg = degree(a.rp, v);
            else v = -1;
        }
        // edge betweenness: the arc (v, w) carries sigma_v * psi_w = sigma_v / sigma_w *
        // (1 + delta_w), read before v's own psi replaces sigma_v; the staged value of
        // vertex k is its running psi sum, and sigma_v is read per arc
        const int total = lb_stage(st, v, deg, dev::ff_pack(dev::ff_zero()), a.rp);
        for (int i0 = 0; i0 < total; i0 += 64) {
            // two passes of 32 arcs at a time: both passes' column, bit and psi loads are in
            // flight before either reduction
            int k[2], j[2], w[2];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int i = i0 + 32 * u + lane;
                k[u] = 0;
                j[u] = 0;
                w[u] = -1;
                if (i < total) {
                    k[u] = lb_find(st, i);
                    j[u] = st.beg[k[u]] + (i - st.pre[k[u]]);
                    w[u] = __ldg(a.col + j[u]);
                }
            }
            bool on[2];
#pragma unroll
            for (int u = 0; u < 2; ++u) on[u] = w[u] >= 0 && test_bit(succ, w[u]);
            unsigned long long x[2];
#pragma unroll
            for (int u = 0; u < 2; ++u) x[u] = on[u] ? __ldcg(a.sp + w[u]) : dev::ff_pack(dev::ff_zero());
            if (a.edge) {
#pragma unroll
                for (int u = 0; u < 2; ++u)
                    if (on[u]) {
                        const dev::ff sv = dev::ff_from_u64(__ldcg(a.sp + st.v[k[u]]));
                        a.edge[j[u]] += dev::ff_to_double(dev::ff_mul(sv, dev::ff_unpack(x[u])));
                    }
            }
            bool dummy = false;
            lb_seg_add<true>(st, k[0], i0 + lane < total, x[0], dummy);
            if (i0 + 32 < total) lb_seg_add<true>(st, k[1], i0 + 32 + lane < total, x[1], dummy);
        }
        if (v >= 0) finish_vertex(a, v, dev::ff_unpack(st.val[lane]), d);
        __syncwarp();
    }
    // heavy vertices of level d: per-chunk partial sums of psi
    for_chunks(a, [&](int h) { return __ldcg(a.dist + h) == d; }, [&](long long c, int h, int j0, int j1) {
        dev::ff acc = dev::ff_zero();
        const dev::ff sv = a.edge ? dev::ff_from_u64(__ldcg(a.sp + h)) : dev::ff_zero();
        for_arcs_vec(a, j0, j1, [&](int j, int w) {
            if (test_bit(succ, w)) {
                const dev::ff psi = dev::ff_unpack(__ldcg(a.sp + w));
                acc = dev::ff_add(acc, psi);
                if (a.edge) a.edge[j] += dev::ff_to_double(dev::ff_mul(sv, psi));
            }
        });
        acc = dev::group_sum_ff<32>(acc);
        if (lane == 0) a.part[c] = dev::ff_pack(acc);
    });
}

// ------------------------------------------------------------------ backward push, level d
// A level whose successors (level d+1) carry far fewer arcs than itself takes their psi by
// push instead of pull: every arc (w, v) of a level-(d+1) vertex w whose end v is a light
// vertex of level d (bit in level bitmap 1) adds psi_w to acc[v] with an FP64 atomic; heavy
// vertices of level d still pull over their chunks, so no hub takes a stream of atomics.
// Edge betweenness: the arc (w, v) carries sigma_v * psi_w (its reverse arc is summed in by
// the finishing pass over arcs).  The level bitmap 0 holds level d+1.

// Marks the light vertices of level d in level bitmap 1 and zeroes their sums.
__device__ void mark_push_targets(const SrcArgs &a, int qo, int cnt)
{
    unsigned *b = lvl_bits(a, 1);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < cnt;
         i += (long long)gridDim.x * blockDim.x) {
        const int v = __ldcg(a.queue + qo + i);
        if ((unsigned)v >= (unsigned)a.n || heavy(a, v)) continue;
        atomicOr(b + (v >> 5), 1u << (v & 31));
        a.acc[v] = 0.0;
    }
}

// Arc (w, v), j its index, pk = psi_w (packed double-single): adds psi_w to v's sum if v is
// a push target (on).
__device__ __forceinline__ void push_arc(const SrcArgs &a, int j, int v, unsigned long long pk, bool on)
{
    if (!on) return;
    const dev::ff pw = dev::ff_unpack(pk);
    atomicAdd(a.acc + v, dev::ff_to_double(pw));
    if (a.edge) a.edge[j] += dev::ff_to_double(dev::ff_mul(dev::ff_from_u64(__ldcg(a.sp + v)), pw));
}

__device__ void back_push(const SrcArgs &a, int d, int qo1, int n1, LbStage *stages)
{
    const int lane = threadIdx.x & 31;
    LbStage &st = stages[threadIdx.x >> 5];
    const long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const unsigned *tgt = lvl_bits(a, 1);
    // light vertices of level d+1: groups of 32 queue entries, lanes over their arcs
    for (long long base = wid * 32; base < n1; base += nwarps * 32) {
        int w = -1, deg = 0;
        if (base + lane < n1) {
            w = __ldcg(a.queue + qo1 + base + lane);
            if ((unsigned)w < (unsigned)a.n && !heavy(a, w)) deg = degree(a.rp, w);
            else w = -1;
        }
        const int total = lb_stage(st, w, deg, w >= 0 ? __ldcg(a.sp + w) : 0ull, a.rp);
        for (int i0 = 0; i0 < total; i0 += 64) {  // two arcs per lane at a time
            int j[2], v[2];
            unsigned long long pk[2];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int i = i0 + 32 * u + lane;
                j[u] = 0;
                v[u] = -1;
                pk[u] = 0ull;
                if (i < total) {
                    const int k = lb_find(st, i);
                    j[u] = st.beg[k] + (i - st.pre[k]);
                    v[u] = __ldg(a.col + j[u]);
                    pk[u] = st.val[k];
                }
            }
            bool on[2];
#pragma unroll
            for (int u = 0; u < 2; ++u) on[u] = v[u] >= 0 && test_bit(tgt, v[u]);
#pragma unroll
            for (int u = 0; u < 2; ++u) push_arc(a, j[u], v[u], pk[u], on[u]);
        }
        __syncwarp();
    }
    // heavy vertices of level d+1: one warp per chunk
    for_chunks(a, [&](int h) { return __ldcg(a.dist + h) == d + 1; }, [&](long long, int h, int j0, int j1) {
        const unsigned long long pk = __ldcg(a.sp + h);
        for_arcs_vec4(a, j0, j1, [&](const int (&j)[4], const int (&v)[4]) {
            bool on[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) on[u] = v[u] >= 0 && test_bit(tgt, v[u]);
#pragma unroll
            for (int u = 0; u < 4; ++u) push_arc(a, j[u], v[u], pk, on[u]);
        });
    });
}

// After a barrier: the light vertices of level d finish with their pushed sums (and leave
// level bitmap 1); the heavy ones add their chunk sums.
__device__ void back_push_finish(const SrcArgs &a, int d, int qo, int cnt)
{
    unsigned *b = lvl_bits(a, 1);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < cnt;
         i += (long long)gridDim.x * blockDim.x) {
        const int v = __ldcg(a.queue + qo + i);
        if ((unsigned)v >= (unsigned)a.n || heavy(a, v)) continue;
        const double x = __ldcg(a.acc + v);
        const float hi = __double2float_rn(x);
        finish_vertex(a, v, {hi, __double2float_rn(x - (double)hi)}, d);
        atomicAnd(b + (v >> 5), ~(1u << (v & 31)));
    }
}

// After a barrier: heavy vertices of level d add their chunk sums in chunk order.
__device__ void back_heavy_finish(const SrcArgs &a, int d)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < a.H;
         i += (long long)gridDim.x * blockDim.x) {
        const int h = __ldg(a.hv + i);
        if (__ldcg(a.dist + h) != d) continue;
        dev::ff acc = dev::ff_zero();
        for (int c = __ldg(a.hfirst + i); c < __ldg(a.hfirst + i + 1); ++c)
            acc = dev::ff_add(acc, dev::ff_unpack(__ldcg(a.part + c)));
        finish_vertex(a, h, acc, d);
    }
}

// Sets (or clears) the bit of every vertex of queue[qo, qo + cnt) in bitmap b.
__device__ void mark_level(const SrcArgs &a, unsigned *b, int qo, int cnt, bool set)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < cnt;
         i += (long long)gridDim.x * blockDim.x) {
        const int v = __ldcg(a.queue + qo + i);
        if ((unsigned)v >= (unsigned)a.n) continue;
        const unsigned bit = 1u << (v & 31);
        if (set) atomicOr(b + (v >> 5), bit);
        else atomicAnd(b + (v >> 5), ~bit);
    }
}

__global__ void __launch_bounds__(kThreads, 3) k_source(SrcArgs a)
{
    __shared__ unsigned long long s_mf;
    __shared__ LbStage stages[kThreads / 32];
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nthr = (long long)gridDim.x * blockDim.x;
    const int s = __ldg(a.src);
    bool ovf = false;
    int ti = 0;
    src_mark(a, ti, 0, 0);
    // vertices without arcs start out visited (their distance stays -1): no arc reaches
    // them, and the bottom-up levels then skip the words in which every vertex with arcs
    // has been reached; a warp covers 32 consecutive vertices, one word of the bitmap
    for (long long v0 = tid - (tid & 31); v0 < a.n; v0 += nthr) {
        const long long v = v0 + (threadIdx.x & 31);
        bool iso = false;
        if (v < a.n) {
            a.dist[v] = v == s ? 0 : -1;
            a.sp[v] = v == s ? 1ull : 0ull;
            iso = degree(a.rp, (int)v) == 0;
        }
        const unsigned w = __ballot_sync(FULL, iso);
        if ((threadIdx.x & 31) == 0) vis_bits(a)[v0 >> 5] = w;
    }
    for (long long i = tid; i < 2LL * a.nw; i += nthr) a.bits[a.nw + i] = 0u;
    if (tid == 0) {
        a.queue[0] = s;
        a.cnt[0] = 1;
        a.cnt[1] = 0;
        a.mfa[1] = 0;
        a.qoff[0] = 0;
    }
    if (!dev::grid_barrier(a.ctrl, a.limit_ns)) return;
    if (tid == 0) {
        atomicOr(vis_bits(a) + (s >> 5), 1u << (s & 31));
        atomicOr(lvl_bits(a, 0) + (s >> 5), 1u << (s & 31));
    }
    if (!dev::grid_barrier(a.ctrl, a.limit_ns)) return;
    src_mark(a, ti, 0, SPH_INIT);
    const int deg_s = degree(a.rp, s);
    long long mu = a.A - deg_s, mf = deg_s;
    int d = 0, qo = 0, nf = 1, td = 0, bu = 0;
    for (;;) {
        const int qnext = qo + nf;  // level d+1 starts after level d in the queue
        if (threadIdx.x == 0) s_mf = 0;
        if (tid == 0) {
            a.cnt[d + 2] = 0;  // used by level d+1
            a.mfa[d + 2] = 0;
            a.qoff[d + 1] = qnext;
        }
        __syncthreads();
        const bool use_bu = a.dir == NK_DIR_BOTTOM_UP ||
                            (a.dir == NK_DIR_AUTO && a.alpha * (double)mf > (double)mu);
        if (use_bu) {
            bu_level(a, d, qnext, &s_mf, ovf, stages);
            if (a.H > 0) {
                if (!dev::grid_barrier(a.ctrl, a.limit_ns)) return;
                src_mark(a, ti, d, SPH_BU);
                bu_heavy_finish(a, d, qnext, &s_mf, ovf);
            }
        } else {
            td_level(a, d, qo, nf, qnext, &s_mf, ovf, stages);
        }
        __syncthreads();
        if (threadIdx.x == 0 && s_mf) atomicAdd((unsigned long long *)(a.mfa + d + 1), (unsigned long long)s_mf);
        if (!dev::grid_barrier(a.ctrl, a.limit_ns)) return;
        src_mark(a, ti, d, use_bu ? (a.H > 0 ? SPH_BU_HUBS : SPH_BU) : SPH_TD);
        // level d+1 is complete: a top-down level adds it to vis (bottom-up set the bits as
        // it settled), and level d's bits leave its level bitmap for use by level d+2
        const int c = __ldcg(a.cnt + d + 1);
        if (!use_bu) mark_level(a, vis_bits(a), qnext, c, true);
        mark_level(a, lvl_bits(a, d), qo, nf, false);
        if (!dev::grid_barrier(a.ctrl, a.limit_ns)) return;
        src_mark(a, ti, d, SPH_POST);
        const long long m2 = __ldcg(a.mfa + d + 1);
        if (use_bu) ++bu;
        else ++td;
        qo = qnext;
        nf = c;
        mu -= m2;
        mf = m2;
        ++d;
        if (c == 0) break;
    }
    const int D = d - 1;  // deepest non-empty level
    if (tid == 0) {
        atomicMax(&a.ctrl->depth, D);
        atomicAdd(&a.ctrl->td_levels, td);
        atomicAdd(&a.ctrl->bu_levels, bu);
    }
    if (ovf) atomicOr(&a.ctrl->ovf, 1);
    if (a.forward_only) return;
    // the level bitmaps are empty again; level bitmap 0 holds level l+1 while level l is
    // swept (edge betweenness also sweeps level 0: the source's arcs carry shares)
    for (int l = D; l >= (a.edge ? 0 : 1); --l) {
        const int ql = __ldcg(a.qoff + l), nl = __ldcg(a.cnt + l);
        // push when the successors' arcs are under a quarter of this level's and the level's
        // vertices average more than 16 arcs (marking and finishing cost a pass over the
        // level's vertices, which a level of few arcs per vertex does not repay); the arc
        // sums and counts per level come from the forward sweep and read the same in every CTA
        const long long arcs_l = __ldcg(a.mfa + l);
        const bool push = l >= 1 && l + 1 <= D && 4LL * __ldcg(a.mfa + l + 1) < arcs_l && arcs_l > 16LL * nl;
        if (l + 2 <= D) mark_level(a, lvl_bits(a, 0), __ldcg(a.qoff + l + 2), __ldcg(a.cnt + l + 2), false);
        if (l + 1 <= D) mark_level(a, lvl_bits(a, 0), __ldcg(a.qoff + l + 1), __ldcg(a.cnt + l + 1), true);
        if (push) mark_push_targets(a, ql, nl);
        if (!dev::grid_barrier(a.ctrl, a.limit_ns)) return;
        src_mark(a, ti, l, SPH_BK_MARK);
        if (push) {
            back_push(a, l, __ldcg(a.qoff + l + 1), __ldcg(a.cnt + l + 1), stages);
            back_level(a, l, ql, nl, stages, false);  // heavy vertices of level l pull
            if (!dev::grid_barrier(a.ctrl, a.limit_ns)) return;
            src_mark(a, ti, l, SPH_BK);
            back_push_finish(a, l, ql, nl);
            if (a.H > 0) back_heavy_finish(a, l);
            if (!dev::grid_barrier(a.ctrl, a.limit_ns)) return;
            src_mark(a, ti, l, SPH_BK_HUBS);
            continue;
        }
        back_level(a, l, ql, nl, stages);
        if (!dev::grid_barrier(a.ctrl, a.limit_ns)) return;
        src_mark(a, ti, l, SPH_BK);
        if (a.H > 0) {
            back_heavy_finish(a, l);
            if (!dev::grid_barrier(a.ctrl, a.limit_ns)) return;
            src_mark(a, ti, l, SPH_BK_HUBS);
        }
    }
}

// error-bounded estimate after a forward sweep from the sample's source (dist, sigma):
// one warp walks back from the target t, choosing each predecessor z of w with probability
// sigma[z] / sigma[w] (the run of z holds below(stream(key, step), sigma[w]) when the
// predecessors' sigma values are laid end to end in adjacency order), and counts every
// vertex strictly between source and target
__global__ void k_rk_walk(const int32_t *rp, const int32_t *col, const int32_t *dist,
                          const unsigned long long *sigma, const int32_t *tgt,
                          const unsigned long long *key, unsigned long long *count)
{
    const int lane = threadIdx.x & 31;
    int w = *tgt;
    const unsigned long long kk = *key;
    for (int step = 0; dist[w] > 1; ++step) {
        const int dw = dist[w];
        const unsigned long long t = dev::below(dev::stream_at(kk, (uint64_t)step), sigma[w]);
        const int end = rp[w + 1];
        unsigned long long run = 0;
        int z = -1;
        for (int base = rp[w]; base < end && z < 0; base += 32) {
            const int j = base + lane;
            int c = -1;
            unsigned long long x = 0;
            if (j < end) {
                c = col[j];
                if (dist[c] == dw - 1) x = sigma[c];
            }
            unsigned long long incl = x;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            const unsigned m = __ballot_sync(0xffffffffu, x != 0 && run + incl > t);
            if (m) z = __shfl_sync(0xffffffffu, c, __ffs(m) - 1);
            else run += __shfl_sync(0xffffffffu, incl, 31);
        }
        if (z < 0) return;  // only with a wrapped path count (reported as an overflow)
        if (lane == 0) count[z] += 1;
        w = z;
    }
}

// closeness from a forward sweep: every reached vertex other than the source adds its
// distance and one to its sums
__global__ void k_add_distances(const int32_t *dist, int32_t n, unsigned long long *far,
                                unsigned long long *reach)
{
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        const int d = dist[v];
        if (d > 0) {
            far[v] += (unsigned long long)d;
            reach[v] += 1ull;
        }
    }
}

// ------------------------------------------------------------------ host side
struct Launch {
    const void *fn;
    int grid;
    int tpv;
};

int make_launch(Launch &L)
{
    static int blocks_per_sm = -1;
    if (blocks_per_sm < 0) {
        int b = 0;
        NK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_source, kThreads, 0));
        blocks_per_sm = b;
    }
    if (blocks_per_sm < 1) return set_error(NK_ERR_CUDA, "per-source kernel cannot be resident");
    L.fn = (const void *)k_source;
    L.grid = blocks_per_sm * num_sms();
    L.tpv = 32;  // lanes over arcs: a warp per group of up to 32 vertices
    return NK_OK;
}

// workspace slots in nk_graph::ws used by this form
enum { WS_DIST = 0, WS_SP = 1, WS_QUEUE = 2, WS_LEVELS = 3, WS_CTRL = 4, WS_PART = 7 };

int run(nk_graph *g, const int32_t *d_src, int32_t k, double *d_scores, const RunCfg &cfg,
        RunStats *st, cudaStream_t s, bool forward_only, int32_t *d_dist_out,
        uint64_t *d_sigma_out)
{
    const int32_t n = g->n;
    DevBuf *ws = scratch(cfg, g);
    NK_TRY(ws[WS_DIST].ensure(sizeof(int32_t) * n));
    // sp, then (for a backward sweep) the FP64 sums of the push levels
    const bool fwd_only = forward_only || cfg.far || cfg.rk_t;
    NK_TRY(ws[WS_SP].ensure(sizeof(uint64_t) * (size_t)n * (fwd_only ? 1 : 2)));
    NK_TRY(ws[WS_QUEUE].ensure(sizeof(int32_t) * n));
    const size_t lv = (size_t)n + 3;
    const int32_t nw = (n + 31) / 32;
    NK_TRY(ws[WS_LEVELS].ensure(lv * (sizeof(int32_t) * 2 + sizeof(long long)) + 3 * sizeof(unsigned) * (size_t)nw));
    NK_TRY(ws[WS_CTRL].ensure(sizeof(Ctrl)));
    NK_TRY(build_heavy(g, s));
    NK_TRY(ws[WS_PART].ensure(sizeof(unsigned long long) * std::max<int64_t>(g->heavy_C, 1)));
    Launch L;
    NK_TRY(make_launch(L));
    SrcArgs a{};
    a.n = n;
    a.A = g->A;
    a.rp = g->rp.as<int32_t>();
    a.col = g->col.as<int32_t>();
    a.dist = d_dist_out ? d_dist_out : ws[WS_DIST].as<int32_t>();
    a.sp = d_sigma_out ? reinterpret_cast<unsigned long long *>(d_sigma_out)
                       : ws[WS_SP].as<unsigned long long>();
    a.queue = ws[WS_QUEUE].as<int32_t>();
    char *lvb = ws[WS_LEVELS].as<char>();
    a.mfa = reinterpret_cast<long long *>(lvb);
    a.cnt = reinterpret_cast<int32_t *>(lvb + lv * sizeof(long long));
    a.qoff = a.cnt + lv;
    a.bits = reinterpret_cast<unsigned *>(a.qoff + lv);
    a.nw = nw;
    a.scores = d_scores;
    a.ctrl = ws[WS_CTRL].as<Ctrl>();
    a.limit_ns = cfg.limit_ns ? cfg.limit_ns : wait_limit_ns();
    a.alpha = cfg.alpha > 0 ? cfg.alpha : 1.0;
    a.dir = cfg.direction;
    a.forward_only = forward_only ? 1 : 0;
    a.edge = forward_only ? nullptr : cfg.edge;
    a.acc = fwd_only ? nullptr : reinterpret_cast<double *>(ws[WS_SP].as<unsigned long long>() + n);
    a.hv = g->heavy[0].as<int32_t>();
    a.hfirst = g->heavy[1].as<int32_t>();
    a.chunk_h = g->heavy[2].as<int32_t>();
    a.H = g->heavy_H;
    a.C = g->heavy_C;
    a.part = ws[WS_PART].as<unsigned long long>();
    NK_CUDA(cudaMemsetAsync(a.ctrl, 0, sizeof(Ctrl), s));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cfg.time_kernels) {
        NK_CUDA(cudaEventCreate(&e0));
        NK_CUDA(cudaEventCreate(&e1));
        NK_CUDA(cudaEventRecord(e0, s));
    }
    if (cfg.far || cfg.rk_t) a.forward_only = 1;
    static const bool trace_on = std::getenv("NK_TRACE") != nullptr;
    Tmp trace_buf;
    a.trace = nullptr;
    if (trace_on) {
        NK_TRY(trace_buf.alloc(sizeof(unsigned long long) * 2 * kTraceCap, s));
        NK_CUDA(cudaMemsetAsync(trace_buf.p, 0, sizeof(unsigned long long) * 2 * kTraceCap, s));
    }
    // sources without arcs add nothing to scores, arc shares or distance sums: only the
    // others are swept (not for a single-source sweep, whose outputs the caller reads, nor
    // for the error-bounded estimate, whose sources are tied to their targets)
    Tmp csrc, ccnt;
    if (!d_dist_out && !cfg.rk_t && k > 0) {
        NK_TRY(csrc.alloc(sizeof(int32_t) * (size_t)k, s));
        NK_TRY(ccnt.alloc(sizeof(int32_t), s));
        NK_TRY(compact_sources(g, d_src, k, csrc.as<int32_t>(), ccnt.as<int32_t>(), s));
        int32_t kk = 0;
        NK_CUDA(cudaMemcpyAsync(&kk, ccnt.p, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        NK_CUDA(cudaStreamSynchronize(s));
        if (kk < 0 || kk > k) return set_error(NK_ERR_CUDA, "source compaction returned %d of %d", kk, k);
        d_src = csrc.as<int32_t>();
        k = kk;
    }
    for (int32_t i = 0; i < k; ++i) {
        a.src = d_src + i;
        a.trace = (trace_on && i == 0) ? trace_buf.as<unsigned long long>() : nullptr;
        void *args[] = {&a};
        int grid = std::max(1, L.grid / std::max(1, cfg.grid_div));
        if (cfg.grid_ctas > 0) grid = std::min(grid, cfg.grid_ctas);
        NK_CUDA(cudaLaunchCooperativeKernel(L.fn, dim3(grid), dim3(kThreads), args, 0, s));
        ::nk::count_launch();
        if (cfg.rk_t) {
            k_rk_walk<<<1, 32, 0, s>>>(a.rp, a.col, a.dist, a.sp, cfg.rk_t + i, cfg.rk_key + i, cfg.rk_count);
            ::nk::count_launch();
        }
        if (cfg.far) {
            k_add_distances<<<std::max(1, std::min((n + 255) / 256, 8 * num_sms())), 256, 0, s>>>(a.dist, n, cfg.far, cfg.reach);
            ::nk::count_launch();
        }
    }
    if (cfg.time_kernels) NK_CUDA(cudaEventRecord(e1, s));
    Ctrl h;
    NK_CUDA(cudaMemcpyAsync(&h, a.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s));
    NK_TRY(host_wait(s, k, a.limit_ns));
    if (trace_on && k > 0) {
        static const char *names[] = {"start", "init", "td", "bu", "bu+hubs", "post", "back-mark", "back", "back-hubs"};
        std::vector<unsigned long long> t(2 * kTraceCap);
        NK_CUDA(cudaMemcpy(t.data(), trace_buf.p, sizeof(unsigned long long) * t.size(), cudaMemcpyDeviceToHost));
        for (int i = 1; i < kTraceCap && t[2 * i + 1]; ++i)
            fprintf(stderr, "nk-trace per-source level=%llu phase=%s us=%.1f\n", t[2 * i] / 16,
                    names[std::min<unsigned long long>(t[2 * i] % 16, 8)], (t[2 * i + 1] - t[2 * i - 1]) * 1e-3);
    }
    if (st) {
        st->mode = NK_MODE_PER_SOURCE;
        st->batch = 1;
        st->tpv = L.tpv;
        st->max_depth = std::max(st->max_depth, h.depth);
        st->launches += k;
        st->td_levels += h.td_levels;
        st->bu_levels += h.bu_levels;
        st->alpha = a.alpha;
        if (cfg.time_kernels) {
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            st->kernel_ms += ms;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (h.err) return set_error(h.err, "per-source sweep aborted: a bounded grid wait ran out");
    // closeness needs distances only, which do not depend on the path counts
    if (h.ovf && !cfg.far) return set_error(NK_ERR_OVERFLOW, "a shortest-path count exceeded 2^64 - 1");
    return NK_OK;
}

}  // namespace

int run_per_source(nk_graph *g, const int32_t *d_src, int32_t k, double *d_scores,
                   const RunCfg &cfg, RunStats *st, cudaStream_t s)
{
    return run(g, d_src, k, d_scores, cfg, st, s, false, nullptr, nullptr);
}

int run_sssp(nk_graph *g, int32_t src, int32_t *d_dist, uint64_t *d_sigma, cudaStream_t s)
{
    Tmp ds;
    NK_TRY(ds.alloc(sizeof(int32_t), s));
    NK_CUDA(cudaMemcpyAsync(ds.p, &src, sizeof(int32_t), cudaMemcpyHostToDevice, s));
    RunCfg cfg;
    return run(g, ds.as<int32_t>(), 1, nullptr, cfg, nullptr, s, true, d_dist, d_sigma);
}

}  // namespace nk

// ---------------------------------------------------------------- allocation-free sweep
// A variant of the forward sweep for callers that cannot allocate device memory at
// call time (for example code running under an allocator that forbids cudaMalloc, or
// a host library that must not grow its footprint once started).  Its scratch - the
// control block, the BFS queue, the per-level counters and the frontier bitmaps - lives in one file-scope
// device array of fixed size, so the call allocates nothing; inputs (the CSR) and
// outputs (dist, sigma) are the caller's device buffers.  Rows are not split into
// chunks here (the chunk table would need an allocation), so a high-degree vertex is
// expanded by one lane group.
namespace nk {
namespace {

constexpr size_t na_align(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr int32_t kNoAllocMaxN = 1 << 20;
constexpr size_t kNaLv = (size_t)kNoAllocMaxN + 3;
constexpr size_t kNaCtrl = 0;
constexpr size_t kNaSrc = 256;
constexpr size_t kNaQueue = 512;
constexpr size_t kNaCnt = na_align(kNaQueue + 4 * (size_t)kNoAllocMaxN);
constexpr size_t kNaQoff = na_align(kNaCnt + 4 * kNaLv);
constexpr size_t kNaMfa = na_align(kNaQoff + 4 * kNaLv);
constexpr size_t kNaBits = na_align(kNaMfa + 8 * kNaLv);
constexpr size_t kNaPart = na_align(kNaBits + 3 * sizeof(unsigned) * (size_t)(kNoAllocMaxN / 32));
constexpr size_t kNaBytes = kNaPart + 256;

}  // namespace
}  // namespace nk

// One copy per device that loads the library, held until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[nk::kNaBytes];

namespace nk {
namespace {

std::mutex g_na_mu;
void *g_na_ptr[128] = {};

// Device address of the static scratch on the current device.  The array's name in
// host code is only a host-side stand-in, so the address is looked up once per device
// (with that device current) and cached.
int noalloc_scratch(unsigned char **out)
{
    int dev = 0;
    NK_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 128) return set_error(NK_ERR_ARG, "device index %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_ptr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return cuda_fail(e, "cudaGetSymbolAddress(scratch)", __FILE__, __LINE__);
        g_na_ptr[dev] = p;
    }
    *out = static_cast<unsigned char *>(g_na_ptr[dev]);
    return NK_OK;
}

}  // namespace
}  // namespace nk

extern "C" int nk_sssp_noalloc(int32_t n, const int32_t *row_ptr, const int32_t *col,
                               int64_t n_arcs, int32_t s, int32_t *dist, uint64_t *sigma,
                               void *stream)
{
    using namespace nk;
    if (!row_ptr || !dist || !sigma || (n_arcs > 0 && !col)) return set_error(NK_ERR_ARG, "null argument");
    if (n < 1 || n > kNoAllocMaxN)
        return set_error(NK_ERR_ARG, "nk_sssp_noalloc handles 1 <= n <= %d vertices (got %d)", kNoAllocMaxN, n);
    if (n_arcs < 0 || n_arcs >= (int64_t)INT_MAX) return set_error(NK_ERR_ARG, "n_arcs out of range");
    if (s < 0 || s >= n) return set_error(NK_ERR_ARG, "source %d outside [0, %d)", s, n);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned char *scr = nullptr;
    NK_TRY(noalloc_scratch(&scr));
    Launch L;
    NK_TRY(make_launch(L));
    SrcArgs a{};
    a.n = n;
    a.A = n_arcs;
    a.rp = row_ptr;
    a.col = col;
    a.src = reinterpret_cast<const int32_t *>(scr + kNaSrc);
    a.dist = dist;
    a.sp = reinterpret_cast<unsigned long long *>(sigma);
    a.queue = reinterpret_cast<int32_t *>(scr + kNaQueue);
    a.cnt = reinterpret_cast<int32_t *>(scr + kNaCnt);
    a.qoff = reinterpret_cast<int32_t *>(scr + kNaQoff);
    a.mfa = reinterpret_cast<long long *>(scr + kNaMfa);
    a.scores = nullptr;
    a.ctrl = reinterpret_cast<Ctrl *>(scr + kNaCtrl);
    a.limit_ns = wait_limit_ns();
    a.alpha = 1.0;
    a.dir = NK_DIR_AUTO;
    a.forward_only = 1;
    a.hv = a.hfirst = a.chunk_h = nullptr;
    a.H = 0;
    a.C = 0;
    a.part = reinterpret_cast<unsigned long long *>(scr + kNaPart);
    a.bits = reinterpret_cast<unsigned *>(scr + kNaBits);
    a.nw = (n + 31) / 32;
    a.edge = nullptr;
    // the control block keeps the previous call's words: it must start at zero
    NK_CUDA(cudaMemsetAsync(a.ctrl, 0, sizeof(Ctrl), st));
    NK_CUDA(cudaMemcpyAsync(scr + kNaSrc, &s, sizeof(int32_t), cudaMemcpyHostToDevice, st));
    void *args[] = {&a};
    NK_CUDA(cudaLaunchCooperativeKernel(L.fn, dim3(L.grid), dim3(kThreads), args, 0, st));
    ::nk::count_launch();
    Ctrl h;
    NK_CUDA(cudaMemcpyAsync(&h, a.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
    NK_CUDA(cudaStreamSynchronize(st));
    if (h.err) return set_error(h.err, "forward sweep aborted: a bounded grid wait ran out");
    if (h.ovf) return set_error(NK_ERR_OVERFLOW, "a shortest-path count exceeded 2^64 - 1");
    return NK_OK;
}

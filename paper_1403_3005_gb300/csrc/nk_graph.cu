// Graph construction on the GPU: canonical CSR builder and the seeded generators of
// the NetworKit paper's Section 5 (Table 2: Erdos-Renyi [Batagelj-Brandes], Barabasi-
// Albert, R-MAT).  The graph is kept as an immutable int32 CSR in HBM (Section 2.3
// describes an adjacency structure with O(n+m) memory; a static CSR is what the
// betweenness sweeps read).
//
// CSR build, for an undirected edge list (u_i, v_i):
//   1. degree count of both directions of every non-loop edge (atomics), with a range
//      check of the ids;
//   2. exclusive scan of the degrees -> bucket offsets;
//   3. scatter of both arcs into their row buckets (atomic cursors; order arbitrary);
//   4. per-row sort + duplicate removal into a second buffer: a warp bitonic network
//      for rows of <= 32 arcs, a shared-memory bitonic sort for rows of <= 4096, and a
//      windowed shared-memory bitmap for longer rows (ids are < n, so marking bits of a
//      window of the id range and reading them back in order sorts and dedupes at once);
//   5. scan of the unique counts -> row_ptr, and a warp-per-row copy into col.
// The result does not depend on the scatter order: it is the canonical form.
#include <algorithm>
#include <climits>
#include <cmath>
#include <vector>

#include "nk_device.cuh"
#include "nk_internal.h"

namespace nk {
namespace {

int finish_graph(nk_graph *g, cudaStream_t st, int *d_maxdeg);

constexpr int kMidMax = 4096;           // rows up to this length: shared-memory bitonic
constexpr int kWinBits = 1 << 18;       // bitmap window for long rows (32 KiB)
constexpr int kWinWords = kWinBits / 32;

int grid_for(int64_t items, int threads, int per_sm = 8)
{
    int64_t b = (items + threads - 1) / threads;
    int64_t cap = (int64_t)per_sm * num_sms();
    if (b > cap) b = cap;
    return (int)std::max<int64_t>(b, 1);
}

// ---------------------------------------------------------------- build steps
__global__ void k_count_deg(const int32_t *u, const int32_t *v, int64_t m, int32_t n,
                            unsigned long long *deg, int *bad)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x) {
        int32_t a = u[e], b = v[e];
        if ((unsigned)a >= (unsigned)n || (unsigned)b >= (unsigned)n) {
            atomicOr(bad, 1);
            continue;
        }
        if (a == b) continue;
        atomicAdd(&deg[a], 1ull);
        atomicAdd(&deg[b], 1ull);
    }
}

__global__ void k_scatter(const int32_t *u, const int32_t *v, int64_t m,
                          unsigned long long *cursor, int32_t *buf)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x) {
        int32_t a = u[e], b = v[e];
        if (a == b) continue;
        buf[atomicAdd(&cursor[a], 1ull)] = b;
        buf[atomicAdd(&cursor[b], 1ull)] = a;
    }
}

// rows of length <= 32: one warp, bitonic network on shuffles
__global__ void k_sort_small(const int64_t *off, const int32_t *buf, int32_t *out,
                             int64_t *ucnt, int32_t n)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = warp; r < n; r += nwarps) {
        const int64_t b = off[r], len = off[r + 1] - b;
        if (len > 32) continue;  // warp-uniform
        int x = lane < len ? buf[b + lane] : INT_MAX;
        for (int k = 2; k <= 32; k <<= 1) {
            for (int j = k >> 1; j > 0; j >>= 1) {
                int y = __shfl_xor_sync(0xffffffffu, x, j);
                bool up = (lane & k) == 0;
                bool lower = (lane & j) == 0;
                x = (lower == up) ? min(x, y) : max(x, y);
            }
        }
        int prev = __shfl_up_sync(0xffffffffu, x, 1);
        bool keep = x != INT_MAX && (lane == 0 || prev != x);
        unsigned bal = __ballot_sync(0xffffffffu, keep);
        if (keep) out[b + __popc(bal & dev::lanemask_lt())] = x;
        if (lane == 0) ucnt[r] = __popc(bal);
    }
}

// rows of length in (32, 4096]: one block of 512 threads, bitonic sort in shared memory
__global__ void __launch_bounds__(512)
k_sort_mid(const int64_t *off, const int32_t *buf, int32_t *out, int64_t *ucnt, int32_t n)
{
    __shared__ int s[kMidMax];
    __shared__ int warp_cnt[16];
    for (int64_t r = blockIdx.x; r < n; r += gridDim.x) {
        const int64_t b = off[r];
        const int len = (int)(off[r + 1] - b);
        if (len <= 32 || len > kMidMax) continue;  // block-uniform
        int N = 64;
        while (N < len) N <<= 1;
        for (int i = threadIdx.x; i < N; i += blockDim.x) s[i] = i < len ? buf[b + i] : INT_MAX;
        __syncthreads();
        for (int k = 2; k <= N; k <<= 1) {
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int i = threadIdx.x; i < N; i += blockDim.x) {
                    int p = i ^ j;
                    if (p > i) {
                        int a = s[i], c = s[p];
                        bool up = (i & k) == 0;
                        if ((a > c) == up) {
                            s[i] = c;
                            s[p] = a;
                        }
                    }
                }
                __syncthreads();
            }
        }
        // dedupe: order-preserving compaction of first occurrences, in chunks of 512
        int base = 0;
        for (int c0 = 0; c0 < len; c0 += blockDim.x) {
            int i = c0 + threadIdx.x;
            bool keep = i < len && (i == 0 || s[i] != s[i - 1]);
            unsigned bal = __ballot_sync(0xffffffffu, keep);
            const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
            if (lane == 0) warp_cnt[wid] = __popc(bal);
            __syncthreads();
            int before = 0, tot = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
                if (w < wid) before += warp_cnt[w];
                tot += warp_cnt[w];
            }
            if (keep) out[b + base + before + __popc(bal & dev::lanemask_lt())] = s[i];
            base += tot;
            __syncthreads();
        }
        if (threadIdx.x == 0) ucnt[r] = base;
        __syncthreads();
    }
}

// rows longer than 4096: windowed bitmap over the id range
__global__ void __launch_bounds__(512)
k_sort_big(const int64_t *off, const int32_t *buf, int32_t *out, int64_t *ucnt, int32_t n)
{
    __shared__ unsigned bits[kWinWords];
    __shared__ int warp_cnt[16];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int64_t r = blockIdx.x; r < n; r += gridDim.x) {
        const int64_t b = off[r];
        const int64_t len = off[r + 1] - b;
        if (len <= kMidMax) continue;  // block-uniform
        int64_t written = 0;
        for (int64_t lo = 0; lo < n; lo += kWinBits) {
            for (int i = threadIdx.x; i < kWinWords; i += blockDim.x) bits[i] = 0u;
            __syncthreads();
            for (int64_t i = threadIdx.x; i < len; i += blockDim.x) {
                int64_t x = buf[b + i] - lo;
                if (x >= 0 && x < kWinBits) atomicOr(&bits[x >> 5], 1u << (x & 31));
            }
            __syncthreads();
            // each thread owns kWinWords/512 consecutive words; block scan of popcounts
            constexpr int per = kWinWords / 512;
            int mine = 0;
            for (int q = 0; q < per; ++q) mine += __popc(bits[threadIdx.x * per + q]);
            int incl = mine;
            for (int o = 1; o < 32; o <<= 1) {
                int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            if (lane == 31) warp_cnt[wid] = incl;
            __syncthreads();
            int before = 0, tot = 0;
            for (int w = 0; w < 16; ++w) {
                if (w < wid) before += warp_cnt[w];
                tot += warp_cnt[w];
            }
            int pos = (int)written + before + incl - mine;
            for (int q = 0; q < per; ++q) {
                unsigned wbits = bits[threadIdx.x * per + q];
                while (wbits) {
                    int t = __ffs(wbits) - 1;
                    wbits &= wbits - 1;
                    out[b + pos++] = (int32_t)(lo + (int64_t)(threadIdx.x * per + q) * 32 + t);
                }
            }
            written += tot;
            __syncthreads();
        }
        if (threadIdx.x == 0) ucnt[r] = written;
        __syncthreads();
    }
}

__global__ void k_compact_rows(const int64_t *off, const int64_t *rp64, const int32_t *src,
                               int32_t *rp, int32_t *col, int32_t n, int *max_deg)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    int local_max = 0;
    for (int64_t r = warp; r <= n; r += nwarps) {
        const int64_t dst = rp64[r];
        if (lane == 0) rp[r] = (int32_t)dst;
        if (r == n) continue;
        const int64_t len = rp64[r + 1] - dst;
        const int64_t b = off[r];
        for (int64_t i = lane; i < len; i += 32) col[dst + i] = src[b + i];
        local_max = max(local_max, (int)len);
    }
    if (lane == 0) atomicMax(max_deg, local_max);
}

__global__ void k_u64_to_i64(const unsigned long long *a, int64_t *b, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        b[i] = (int64_t)a[i];
}

__global__ void k_csr_rows(const int32_t *rp, int32_t n, int32_t *u)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = warp; r < n; r += nwarps)
        for (int64_t j = rp[r] + lane; j < rp[r + 1]; j += 32) u[j] = (int32_t)r;
}

// checks of a caller CSR: structure (always) and canonical form (validate)
__global__ void k_check_csr(const int32_t *rp, const int32_t *col, int32_t n, int64_t A,
                            bool canonical, int *bad, int *max_deg)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    int local_max = 0;
    for (int64_t r = warp; r < n; r += nwarps) {
        const int32_t b = rp[r], e = rp[r + 1];
        if (b < 0 || e < b || e > A) {
            if (lane == 0) atomicOr(bad, 1);
            continue;
        }
        local_max = max(local_max, e - b);
        for (int32_t j = b + lane; j < e; j += 32) {
            int32_t x = col[j];
            if ((unsigned)x >= (unsigned)n) {
                atomicOr(bad, 1);
                continue;
            }
            if (!canonical) continue;
            if (x == r || (j > b && col[j - 1] >= x)) atomicOr(bad, 2);
            // symmetry: r must appear in row x (binary search; rows are sorted)
            int32_t lo = rp[x], hi = rp[x + 1] - 1;
            bool found = false;
            while (lo <= hi) {
                int32_t mid = (lo + hi) >> 1;
                int32_t y = col[mid];
                if (y == r) { found = true; break; }
                if (y < r) lo = mid + 1; else hi = mid - 1;
            }
            if (!found) atomicOr(bad, 4);
        }
    }
    if (lane == 0) atomicMax(max_deg, local_max);
}

__global__ void k_check_ends(const int32_t *rp, int32_t n, int64_t A, int *bad)
{
    if (rp[0] != 0 || (int64_t)rp[n] != A) atomicOr(bad, 1);
}

// ---------------------------------------------------------------- generators
// Natural logarithm for the ER skip lengths: ln z = 2 atanh((z-1)/(z+1)), z = m 2^e,
// m in (sqrt(1/2), sqrt(2)], the atanh series summed by Horner's rule over 13 terms.
// Every step is an explicitly rounded IEEE double operation (no contraction), so that
// the skip lengths, and hence the graph, are the same on every platform.
__device__ double er_log(double x)
{
    uint64_t bits = __double_as_longlong(x);
    int e = (int)((bits >> 52) & 0x7FF) - 1023;
    double m = __longlong_as_double((long long)((bits & 0x000FFFFFFFFFFFFFull) |
                                                0x3FF0000000000000ull));
    if (m > 1.4142135623730951) {
        m = __dmul_rn(m, 0.5);
        e = e + 1;
    }
    double s = __ddiv_rn(__dsub_rn(m, 1.0), __dadd_rn(m, 1.0));
    double s2 = __dmul_rn(s, s);
    double p = __ddiv_rn(1.0, 25.0);
    for (int k = 11; k >= 0; --k) p = __dadd_rn(__dmul_rn(p, s2), __ddiv_rn(1.0, (double)(2 * k + 1)));
    double r = __dmul_rn(__dmul_rn(2.0, s), p);
    return __dadd_rn(r, __dmul_rn((double)e, 0.6931471805599453));
}

__device__ __forceinline__ void pair_of(uint64_t t, int32_t &u, int32_t &v)
{
    uint64_t uu = (uint64_t)((1.0 + sqrt(1.0 + 8.0 * (double)t)) * 0.5);
    while (uu > 1 && uu * (uu - 1) / 2 > t) --uu;
    while ((uu + 1) * uu / 2 <= t) ++uu;
    u = (int32_t)uu;
    v = (int32_t)(t - uu * (uu - 1) / 2);
}

constexpr uint64_t kErChunk = 1ull << 20;

// One thread per chunk of 2^20 vertex pairs; geometric skips drawn from the chunk's
// own stream (seeded by the chunk's output of the root stream).  Pass 1 counts, pass 2
// writes at the scanned offset.
__global__ void k_er(uint64_t N, double p, uint64_t seed, int64_t *count,
                     const int64_t *offset, int32_t *eu, int32_t *ev)
{
    const uint64_t chunks = (N + kErChunk - 1) / kErChunk;
    const double lq = er_log(__dsub_rn(1.0, p));
    for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < chunks;
         j += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t cs = dev::stream_at(seed, j);
        int64_t t = (int64_t)(j * kErChunk) - 1;
        const int64_t end = (int64_t)min((j + 1) * kErChunk, N);
        int64_t c = 0, o = offset ? offset[j] : 0;
        for (uint64_t i = 0;; ++i) {
            const double r = __dmul_rn((double)(dev::stream_at(cs, i) >> 11), 1.0 / 9007199254740992.0);
            const double q = __ddiv_rn(er_log(__dsub_rn(1.0, r)), lq);
            if (q >= (double)(end - t - 1)) break;
            t = t + 1 + (int64_t)q;
            if (eu) pair_of((uint64_t)t, eu[o + c], ev[o + c]);
            ++c;
        }
        if (count) count[j] = c;
    }
}

__global__ void k_er_all_pairs(uint64_t N, int32_t *eu, int32_t *ev)
{
    for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < N;
         t += (uint64_t)gridDim.x * blockDim.x)
        pair_of(t, eu[t], ev[t]);
}

// Batagelj-Brandes preferential attachment: edge e = v*m0 + i is (v, M[r_e]) with r_e
// uniform in [0, 2e]; M[2x] = x / m0 and M[2x+1] is the target of edge x, so an odd r
// is resolved by following the chain of earlier draws (each step strictly decreases).
__global__ void k_ba(int64_t E, int32_t m0, uint64_t seed, int32_t *eu, int32_t *ev)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E;
         e += (int64_t)gridDim.x * blockDim.x) {
        uint64_t r = dev::below(dev::stream_at(seed, (uint64_t)e), 2ull * e + 1);
        while (r & 1ull) {
            const uint64_t x = (r - 1) >> 1;
            r = dev::below(dev::stream_at(seed, x), 2ull * x + 1);
        }
        eu[e] = (int32_t)(e / m0);
        ev[e] = (int32_t)((r >> 1) / (uint64_t)m0);
    }
}

// R-MAT: per edge, one quadrant per bit level (most significant first) from the
// stream seeded by the edge's root output; thresholds are the cumulative quadrant
// probabilities scaled to 2^64.
__global__ void k_rmat(int64_t E, int scale, uint64_t seed, uint64_t t1, uint64_t t2,
                       uint64_t t3, int32_t *eu, int32_t *ev)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E;
         e += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t es = dev::stream_at(seed, (uint64_t)e);
        uint32_t u = 0, v = 0;
        for (int l = 0; l < scale; ++l) {
            const uint64_t x = dev::stream_at(es, (uint64_t)l);
            const uint32_t ru = x >= t2, rv = (x >= t1 && x < t2) || x >= t3;
            u = (u << 1) | ru;
            v = (v << 1) | rv;
        }
        eu[e] = (int32_t)u;
        ev[e] = (int32_t)v;
    }
}

int finish_graph(nk_graph *g, cudaStream_t st, int *d_maxdeg)
{
    int h = 0;
    NK_CUDA(cudaMemcpyAsync(&h, d_maxdeg, sizeof(int), cudaMemcpyDeviceToHost, st));
    NK_CUDA(cudaStreamSynchronize(st));
    g->max_deg = h;
    return build_heavy(g, st);
}

}  // namespace

// ---------------------------------------------------------------- CSR from edges
int build_csr_from_edges(nk_graph *g, int32_t n, int64_t m, const int32_t *d_u,
                         const int32_t *d_v, cudaStream_t st)
{
    if (2 * m >= (int64_t)INT_MAX) return set_error(NK_ERR_ARG, "too many edges (%lld)", (long long)m);
    g->n = n;
    Tmp deg, off, flags, ucnt;
    NK_TRY(deg.alloc(sizeof(unsigned long long) * (n + 1), st));
    NK_TRY(off.alloc(sizeof(int64_t) * (n + 1), st));
    NK_TRY(flags.alloc(2 * sizeof(int), st));
    int *d_bad = flags.as<int>(), *d_max = d_bad + 1;
    NK_CUDA(cudaMemsetAsync(deg.p, 0, sizeof(unsigned long long) * (n + 1), st));
    NK_CUDA(cudaMemsetAsync(flags.p, 0, 2 * sizeof(int), st));
    if (m > 0) {
        k_count_deg<<<grid_for(m, 256), 256, 0, st>>>(d_u, d_v, m, n, deg.as<unsigned long long>(), d_bad);
        ::nk::count_launch();
        NK_CUDA(cudaGetLastError());
    }
    int hbad = 0;
    NK_CUDA(cudaMemcpyAsync(&hbad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, st));
    NK_CUDA(cudaStreamSynchronize(st));
    if (hbad) return set_error(NK_ERR_GRAPH, "edge list holds a vertex id outside [0, %d)", n);
    // offsets of the raw (symmetrised, loop-free) buckets
    k_u64_to_i64<<<grid_for(n + 1, 256), 256, 0, st>>>(deg.as<unsigned long long>(), off.as<int64_t>(), n + 1);
    ::nk::count_launch();
    NK_CUDA(cudaGetLastError());
    NK_TRY(scan_exclusive_i64(off.as<int64_t>(), off.as<int64_t>(), n + 1, nullptr, st));
    int64_t total = 0;
    NK_CUDA(cudaMemcpyAsync(&total, off.as<int64_t>() + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    NK_CUDA(cudaStreamSynchronize(st));
    Tmp buf, sorted;
    NK_TRY(buf.alloc(sizeof(int32_t) * (total + 1), st));
    NK_TRY(sorted.alloc(sizeof(int32_t) * (total + 1), st));
    if (m > 0) {
        // cursors: reuse deg as the running position of every bucket
        NK_CUDA(cudaMemcpyAsync(deg.p, off.p, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToDevice, st));
        k_scatter<<<grid_for(m, 256), 256, 0, st>>>(d_u, d_v, m, deg.as<unsigned long long>(), buf.as<int32_t>());
        ::nk::count_launch();
        NK_CUDA(cudaGetLastError());
    }
    NK_TRY(ucnt.alloc(sizeof(int64_t) * (n + 1), st));
    NK_CUDA(cudaMemsetAsync(ucnt.p, 0, sizeof(int64_t) * (n + 1), st));
    k_sort_small<<<grid_for((int64_t)n * 32, 256), 256, 0, st>>>(off.as<int64_t>(), buf.as<int32_t>(), sorted.as<int32_t>(), ucnt.as<int64_t>(), n);
    ::nk::count_launch();
    NK_CUDA(cudaGetLastError());
    k_sort_mid<<<std::max(1, std::min(n, 4 * num_sms())), 512, 0, st>>>(off.as<int64_t>(), buf.as<int32_t>(), sorted.as<int32_t>(), ucnt.as<int64_t>(), n);
    ::nk::count_launch();
    NK_CUDA(cudaGetLastError());
    k_sort_big<<<std::max(1, std::min(n, 2 * num_sms())), 512, 0, st>>>(off.as<int64_t>(), buf.as<int32_t>(), sorted.as<int32_t>(), ucnt.as<int64_t>(), n);
    ::nk::count_launch();
    NK_CUDA(cudaGetLastError());
    int64_t A = 0;
    Tmp tot;
    NK_TRY(tot.alloc(sizeof(int64_t), st));
    NK_TRY(scan_exclusive_i64(ucnt.as<int64_t>(), ucnt.as<int64_t>(), n + 1, tot.as<int64_t>(), st));
    NK_CUDA(cudaMemcpyAsync(&A, tot.p, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    NK_CUDA(cudaStreamSynchronize(st));
    g->A = A;
    NK_TRY(g->rp.ensure(sizeof(int32_t) * (n + 1)));
    NK_TRY(g->col.ensure(sizeof(int32_t) * (A + 1)));
    k_compact_rows<<<grid_for((int64_t)(n + 1) * 32, 256), 256, 0, st>>>(off.as<int64_t>(), ucnt.as<int64_t>(), sorted.as<int32_t>(), g->rp.as<int32_t>(), g->col.as<int32_t>(), n, d_max);
    ::nk::count_launch();
    NK_CUDA(cudaGetLastError());
    return finish_graph(g, st, d_max);
}

// Chunk table of the vertices whose degree exceeds `chunk`, built on the host from row_ptr:
// heavy vertex ids, the first chunk of each, and the owner of every chunk.
static int build_table(nk_graph *g, int chunk, nk::DevBuf (&dst)[3], int32_t &H, int32_t &C,
                       std::vector<int32_t> *h_hv, std::vector<int32_t> *h_hfirst, cudaStream_t s)
{
    std::vector<int32_t> rp(g->n + 1);
    NK_CUDA(cudaMemcpyAsync(rp.data(), g->rp.p, sizeof(int32_t) * (g->n + 1), cudaMemcpyDeviceToHost, s));
    NK_CUDA(cudaStreamSynchronize(s));
    std::vector<int32_t> hv, hfirst, chunk_h;
    int64_t c = 0;
    for (int32_t v = 0; v < g->n; ++v) {
        const int32_t deg = rp[v + 1] - rp[v];
        if (deg <= chunk) continue;
        const int32_t nc = (deg + chunk - 1) / chunk;
        hfirst.push_back((int32_t)c);
        for (int32_t j = 0; j < nc; ++j) chunk_h.push_back((int32_t)hv.size());
        hv.push_back(v);
        c += nc;
    }
    hfirst.push_back((int32_t)c);
    NK_TRY(dst[0].ensure(sizeof(int32_t) * std::max<size_t>(hv.size(), 1)));
    NK_TRY(dst[1].ensure(sizeof(int32_t) * hfirst.size()));
    NK_TRY(dst[2].ensure(sizeof(int32_t) * std::max<size_t>(chunk_h.size(), 1)));
    if (!hv.empty()) {
        NK_CUDA(cudaMemcpyAsync(dst[0].p, hv.data(), sizeof(int32_t) * hv.size(), cudaMemcpyHostToDevice, s));
        NK_CUDA(cudaMemcpyAsync(dst[2].p, chunk_h.data(), sizeof(int32_t) * chunk_h.size(), cudaMemcpyHostToDevice, s));
    }
    NK_CUDA(cudaMemcpyAsync(dst[1].p, hfirst.data(), sizeof(int32_t) * hfirst.size(), cudaMemcpyHostToDevice, s));
    NK_CUDA(cudaStreamSynchronize(s));
    C = (int32_t)c;
    H = (int32_t)hv.size();
    if (h_hv) *h_hv = std::move(hv);
    if (h_hfirst) *h_hfirst = std::move(hfirst);
    return NK_OK;
}

// The graph's own table (kHeavyChunk arcs per chunk), built once.
int build_heavy(nk_graph *g, cudaStream_t s)
{
    std::lock_guard<std::mutex> lk(g->heavy_mu);
    if (g->heavy_H >= 0) return NK_OK;
    int32_t H = -1, C = 0;
    NK_TRY(build_table(g, kHeavyChunk, g->heavy, H, C, &g->h_hv, &g->h_hfirst, s));
    g->heavy_C = C;
    g->heavy_H = H;
    return NK_OK;
}

int heavy_view(nk_graph *g, int chunk, cudaStream_t s, HeavyView *out)
{
    if (chunk <= 0 || chunk == kHeavyChunk) {
        NK_TRY(build_heavy(g, s));
        *out = {g->heavy[0].as<int32_t>(), g->heavy[1].as<int32_t>(), g->heavy[2].as<int32_t>(),
                g->heavy_H, g->heavy_C, kHeavyChunk};
        return NK_OK;
    }
    std::lock_guard<std::mutex> lk(g->heavy_mu);
    if (g->heavy_alt_H < 0 || g->heavy_alt_chunk != chunk) {
        int32_t H = -1, C = 0;
        g->heavy_alt_H = -1;
        NK_TRY(build_table(g, chunk, g->heavy_alt, H, C, nullptr, nullptr, s));
        g->heavy_alt_H = H;
        g->heavy_alt_C = C;
        g->heavy_alt_chunk = chunk;
    }
    *out = {g->heavy_alt[0].as<int32_t>(), g->heavy_alt[1].as<int32_t>(), g->heavy_alt[2].as<int32_t>(),
            g->heavy_alt_H, g->heavy_alt_C, chunk};
    return NK_OK;
}

__global__ void k_relabel_perm(int32_t n, int32_t *perm)
{
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        perm[v] = (int32_t)(((unsigned long long)v * kRelabelMul) % (unsigned long long)n);
}

__global__ void k_relabel_arcs(const int32_t *rp, const int32_t *col, int32_t n, const int32_t *perm,
                               int32_t *eu, int32_t *ev)
{
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x) {
        const int32_t pu = perm[u];
        for (int32_t j = rp[u]; j < rp[u + 1]; ++j) {
            eu[j] = pu;
            ev[j] = perm[col[j]];
        }
    }
}

// The relabelled copy: the arcs (perm[u], perm[v]) through the canonical CSR builder.
int build_relabeled(nk_graph *g, cudaStream_t s)
{
    if (g->relab) return NK_OK;
    if (2 * g->A >= (int64_t)INT_MAX) return set_error(NK_ERR_NOMEM, "graph too large to relabel");
    const int32_t n = g->n;
    NK_TRY(g->relab_perm.ensure(sizeof(int32_t) * (size_t)n));
    k_relabel_perm<<<grid_for(n, 256), 256, 0, s>>>(n, g->relab_perm.as<int32_t>());
    ::nk::count_launch();
    Tmp eu, ev;
    NK_TRY(eu.alloc(sizeof(int32_t) * (size_t)std::max<int64_t>(g->A, 1), s));
    NK_TRY(ev.alloc(sizeof(int32_t) * (size_t)std::max<int64_t>(g->A, 1), s));
    k_relabel_arcs<<<grid_for(n, 256), 256, 0, s>>>(g->rp.as<int32_t>(), g->col.as<int32_t>(), n,
                                                     g->relab_perm.as<int32_t>(), eu.as<int32_t>(), ev.as<int32_t>());
    ::nk::count_launch();
    NK_CUDA(cudaGetLastError());
    nk_graph *r = new (std::nothrow) nk_graph();
    if (!r) return set_error(NK_ERR_NOMEM, "host allocation failed");
    const int rc = build_csr_from_edges(r, n, g->A, eu.as<int32_t>(), ev.as<int32_t>(), s);
    if (rc != NK_OK) {
        delete r;
        return rc;
    }
    g->relab.reset(r);
    return NK_OK;
}

}  // namespace nk

using namespace nk;

namespace {

int new_graph(nk_graph **out)
{
    *out = nullptr;
    nk_graph *g = new (std::nothrow) nk_graph();
    if (!g) return set_error(NK_ERR_NOMEM, "host allocation failed");
    *out = g;
    return NK_OK;
}

// Copies n items from a host or device pointer into a stream-ordered temporary.
template <class T>
int stage(const T *src, int64_t n, bool device, Tmp &dst, cudaStream_t st)
{
    NK_TRY(dst.alloc(sizeof(T) * (n > 0 ? n : 1), st));
    if (n > 0)
        NK_CUDA(cudaMemcpyAsync(dst.p, src, sizeof(T) * n,
                                device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    return NK_OK;
}

}  // namespace

extern "C" {

int nk_graph_from_edges(int32_t n, int64_t m, const int32_t *u, const int32_t *v,
                        uint32_t flags, nk_graph **out)
{
    if (!out) return set_error(NK_ERR_ARG, "out is null");
    *out = nullptr;
    if (n < 1) return set_error(NK_ERR_ARG, "n must be >= 1 (got %d)", n);
    if (m < 0 || (m > 0 && (!u || !v))) return set_error(NK_ERR_ARG, "bad edge arrays");
    cudaStream_t st = stream();
    const bool dev = flags & NK_CSR_DEVICE_PTRS;
    Tmp du, dv;
    NK_TRY(stage(u, m, dev, du, st));
    NK_TRY(stage(v, m, dev, dv, st));
    nk_graph *g;
    NK_TRY(new_graph(&g));
    int rc = build_csr_from_edges(g, n, m, du.as<int32_t>(), dv.as<int32_t>(), st);
    if (rc != NK_OK) {
        delete g;
        return rc;
    }
    *out = g;
    return NK_OK;
}

int nk_graph_from_csr(int32_t n, const int32_t *row_ptr, const int32_t *col, int64_t n_arcs,
                      uint32_t flags, nk_graph **out)
{
    if (!out) return set_error(NK_ERR_ARG, "out is null");
    *out = nullptr;
    if (n < 1) return set_error(NK_ERR_ARG, "n must be >= 1 (got %d)", n);
    if (n_arcs < 0 || n_arcs >= (int64_t)INT_MAX) return set_error(NK_ERR_ARG, "n_arcs out of range");
    if (!row_ptr || (n_arcs > 0 && !col)) return set_error(NK_ERR_ARG, "null CSR array");
    cudaStream_t st = stream();
    const bool dev = flags & NK_CSR_DEVICE_PTRS;
    nk_graph *g;
    NK_TRY(new_graph(&g));
    auto fail = [&](int rc) { delete g; return rc; };
    int rc;
    if (flags & NK_CSR_CANONICALISE) {
        Tmp drp, dcol, du;
        if ((rc = stage(row_ptr, (int64_t)n + 1, dev, drp, st)) != NK_OK) return fail(rc);
        if ((rc = stage(col, n_arcs, dev, dcol, st)) != NK_OK) return fail(rc);
        Tmp fl;
        if ((rc = fl.alloc(2 * sizeof(int), st)) != NK_OK) return fail(rc);
        if (cudaMemsetAsync(fl.p, 0, 2 * sizeof(int), st) != cudaSuccess) return fail(set_error(NK_ERR_CUDA, "memset"));
        k_check_ends<<<1, 1, 0, st>>>(drp.as<int32_t>(), n, n_arcs, fl.as<int>());
        ::nk::count_launch();
        k_check_csr<<<grid_for((int64_t)n * 32, 256), 256, 0, st>>>(drp.as<int32_t>(), dcol.as<int32_t>(), n, n_arcs, false, fl.as<int>(), fl.as<int>() + 1);
        ::nk::count_launch();
        int hb = 0;
        if (cudaMemcpyAsync(&hb, fl.p, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return fail(set_error(NK_ERR_CUDA, "CSR check failed: %s", cudaGetErrorString(cudaGetLastError())));
        if (hb) return fail(set_error(NK_ERR_GRAPH, "row_ptr/col are not a CSR of %d vertices", n));
        if ((rc = du.alloc(sizeof(int32_t) * (n_arcs > 0 ? n_arcs : 1), st)) != NK_OK) return fail(rc);
        k_csr_rows<<<grid_for((int64_t)n * 32, 256), 256, 0, st>>>(drp.as<int32_t>(), n, du.as<int32_t>());
        ::nk::count_launch();
        if ((rc = build_csr_from_edges(g, n, n_arcs, du.as<int32_t>(), dcol.as<int32_t>(), st)) != NK_OK)
            return fail(rc);
        *out = g;
        return NK_OK;
    }
    g->n = n;
    g->A = n_arcs;
    if ((rc = g->rp.ensure(sizeof(int32_t) * (n + 1))) != NK_OK) return fail(rc);
    if ((rc = g->col.ensure(sizeof(int32_t) * (n_arcs + 1))) != NK_OK) return fail(rc);
    const cudaMemcpyKind kind = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (cudaMemcpyAsync(g->rp.p, row_ptr, sizeof(int32_t) * (n + 1), kind, st) != cudaSuccess ||
        (n_arcs > 0 && cudaMemcpyAsync(g->col.p, col, sizeof(int32_t) * n_arcs, kind, st) != cudaSuccess))
        return fail(set_error(NK_ERR_CUDA, "CSR upload failed: %s", cudaGetErrorString(cudaGetLastError())));
    Tmp fl;
    if ((rc = fl.alloc(2 * sizeof(int), st)) != NK_OK) return fail(rc);
    if (cudaMemsetAsync(fl.p, 0, 2 * sizeof(int), st) != cudaSuccess) return fail(set_error(NK_ERR_CUDA, "memset"));
    k_check_ends<<<1, 1, 0, st>>>(g->rp.as<int32_t>(), n, n_arcs, fl.as<int>());
    ::nk::count_launch();
    k_check_csr<<<grid_for((int64_t)n * 32, 256), 256, 0, st>>>(g->rp.as<int32_t>(), g->col.as<int32_t>(), n, n_arcs, (flags & NK_CSR_VALIDATE) != 0, fl.as<int>(), fl.as<int>() + 1);
    ::nk::count_launch();
    int h[2] = {0, 0};
    if (cudaMemcpyAsync(h, fl.p, 2 * sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return fail(set_error(NK_ERR_CUDA, "CSR check failed: %s", cudaGetErrorString(cudaGetLastError())));
    if (h[0] & 1) return fail(set_error(NK_ERR_GRAPH, "row_ptr/col are not a CSR of %d vertices", n));
    if (h[0] & 2) return fail(set_error(NK_ERR_GRAPH, "a row is unsorted, has a duplicate or a self-loop"));
    if (h[0] & 4) return fail(set_error(NK_ERR_GRAPH, "adjacency is not symmetric"));
    g->max_deg = h[1];
    if ((rc = build_heavy(g, st)) != NK_OK) return fail(rc);
    *out = g;
    return NK_OK;
}

int nk_graph_generate(int kind, const double *params, int32_t n_or_scale, uint64_t seed,
                      nk_graph **out)
{
    if (!out) return set_error(NK_ERR_ARG, "out is null");
    *out = nullptr;
    if (!params) return set_error(NK_ERR_ARG, "params is null");
    cudaStream_t st = stream();
    Tmp eu, ev;
    int64_t m = 0;
    int32_t n = 0;
    if (kind == NK_GEN_ER) {
        n = n_or_scale;
        const double d = params[0];
        if (n < 1 || !(d >= 0.0)) return set_error(NK_ERR_ARG, "ER needs n >= 1, avg degree >= 0");
        const uint64_t N = (uint64_t)n * (uint64_t)(n - 1) / 2;
        const double p = n > 1 ? d / (double)(n - 1) : 0.0;
        if (N > 0 && p >= 1.0) {
            m = (int64_t)N;
            NK_TRY(eu.alloc(sizeof(int32_t) * m, st));
            NK_TRY(ev.alloc(sizeof(int32_t) * m, st));
            k_er_all_pairs<<<grid_for(m, 256), 256, 0, st>>>(N, eu.as<int32_t>(), ev.as<int32_t>());
            ::nk::count_launch();
            NK_CUDA(cudaGetLastError());
        } else if (N > 0 && p > 0.0) {
            const int64_t chunks = (int64_t)((N + kErChunk - 1) / kErChunk);
            Tmp cnt, tot;
            NK_TRY(cnt.alloc(sizeof(int64_t) * chunks, st));
            NK_TRY(tot.alloc(sizeof(int64_t), st));
            k_er<<<grid_for(chunks, 128), 128, 0, st>>>(N, p, seed, cnt.as<int64_t>(), nullptr, nullptr, nullptr);
            ::nk::count_launch();
            NK_CUDA(cudaGetLastError());
            NK_TRY(scan_exclusive_i64(cnt.as<int64_t>(), cnt.as<int64_t>(), chunks, tot.as<int64_t>(), st));
            NK_CUDA(cudaMemcpyAsync(&m, tot.p, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
            NK_CUDA(cudaStreamSynchronize(st));
            NK_TRY(eu.alloc(sizeof(int32_t) * (m + 1), st));
            NK_TRY(ev.alloc(sizeof(int32_t) * (m + 1), st));
            k_er<<<grid_for(chunks, 128), 128, 0, st>>>(N, p, seed, nullptr, cnt.as<int64_t>(), eu.as<int32_t>(), ev.as<int32_t>());
            ::nk::count_launch();
            NK_CUDA(cudaGetLastError());
        }
    } else if (kind == NK_GEN_BA) {
        n = n_or_scale;
        const double m0d = params[0];
        if (n < 1 || !(m0d >= 1.0) || m0d != std::floor(m0d) || m0d > 1e6)
            return set_error(NK_ERR_ARG, "BA needs n >= 1 and an integer m0 >= 1");
        const int32_t m0 = (int32_t)m0d;
        m = (int64_t)n * m0;
        NK_TRY(eu.alloc(sizeof(int32_t) * m, st));
        NK_TRY(ev.alloc(sizeof(int32_t) * m, st));
        k_ba<<<grid_for(m, 256), 256, 0, st>>>(m, m0, seed, eu.as<int32_t>(), ev.as<int32_t>());
        ::nk::count_launch();
        NK_CUDA(cudaGetLastError());
    } else if (kind == NK_GEN_RMAT) {
        const int scale = n_or_scale;
        const double efd = params[0], a = params[1], b = params[2], c = params[3];
        if (scale < 1 || scale > 30 || !(efd >= 1.0) || efd != std::floor(efd))
            return set_error(NK_ERR_ARG, "R-MAT needs 1 <= scale <= 30 and an integer edge factor >= 1");
        if (!(a >= 0 && b >= 0 && c >= 0) || !(a + b + c < 1.0))
            return set_error(NK_ERR_ARG, "R-MAT needs a, b, c >= 0 and a + b + c < 1");
        n = (int32_t)(1u << scale);
        m = (int64_t)efd << scale;
        const double two64 = 18446744073709551616.0;
        const uint64_t t1 = (uint64_t)(a * two64);
        const uint64_t t2 = (uint64_t)((a + b) * two64);
        const uint64_t t3 = (uint64_t)(((a + b) + c) * two64);
        NK_TRY(eu.alloc(sizeof(int32_t) * m, st));
        NK_TRY(ev.alloc(sizeof(int32_t) * m, st));
        k_rmat<<<grid_for(m, 256), 256, 0, st>>>(m, scale, seed, t1, t2, t3, eu.as<int32_t>(), ev.as<int32_t>());
        ::nk::count_launch();
        NK_CUDA(cudaGetLastError());
    } else {
        return set_error(NK_ERR_ARG, "unknown generator kind %d", kind);
    }
    nk_graph *g;
    NK_TRY(new_graph(&g));
    int rc = build_csr_from_edges(g, n, m, eu.as<int32_t>(), ev.as<int32_t>(), st);
    if (rc != NK_OK) {
        delete g;
        return rc;
    }
    *out = g;
    return NK_OK;
}

int nk_graph_info(const nk_graph *g, int32_t *n, int64_t *n_arcs)
{
    if (!g) return set_error(NK_ERR_ARG, "graph is null");
    if (n) *n = g->n;
    if (n_arcs) *n_arcs = g->A;
    return NK_OK;
}

int nk_graph_export_csr(const nk_graph *g, int32_t *row_ptr, int32_t *col)
{
    if (!g || !row_ptr || (g->A > 0 && !col)) return set_error(NK_ERR_ARG, "null argument");
    cudaStream_t st = stream();
    NK_CUDA(cudaMemcpyAsync(row_ptr, g->rp.p, sizeof(int32_t) * (g->n + 1), cudaMemcpyDeviceToHost, st));
    if (g->A > 0)
        NK_CUDA(cudaMemcpyAsync(col, g->col.p, sizeof(int32_t) * g->A, cudaMemcpyDeviceToHost, st));
    NK_CUDA(cudaStreamSynchronize(st));
    return NK_OK;
}

int nk_graph_free(nk_graph *g)
{
    if (!g) return NK_OK;
    if (g->pending.load() > 0)
        return set_error(NK_ERR_ARG, "graph has %lld pending serving requests",
                         (long long)g->pending.load());
    cudaStreamSynchronize(stream());
    delete g;
    return NK_OK;
}

}  // extern "C"

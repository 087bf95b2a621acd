// Pieces of the error-bounded betweenness estimate after Riondato and Kornaropoulos
// (Section 3.2): the vertex-diameter bound that sets the number of samples, and the
// draws of the sampled pairs.  The shortest paths themselves come from the batched or
// per-source forward sweep, which walks one random path back from each sample's target.
//
// Vertex-diameter bound: per connected component C with smallest vertex x, a shortest path
// has at most min(|C|, 2 ecc(x) + 1) vertices (every vertex is within ecc(x) of x); the
// bound is the largest over the components.  Components come from a lock-free union-find
// (roots always linked under smaller roots, so each root is its component's smallest
// vertex), then one BFS from all roots at once gives each vertex its distance to its root.
#include <algorithm>
#include <cmath>

#include "nk_device.cuh"
#include "nk_internal.h"

namespace nk {
namespace {

__global__ void k_cc_init(int32_t *p, int32_t n)
{
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        p[v] = (int32_t)v;
}

// Root of x with path halving.  Invariant: p[x] <= x, with equality only at roots, so the
// walk ends; a halving store only writes an ancestor of x into a non-root, which other
// threads' stores and links (which write roots only) leave valid.
__device__ __forceinline__ int32_t cc_find(int32_t *p, int32_t x)
{
    for (;;) {
        const int32_t y = dev::ld_volatile(p + x);
        if (y == x) return x;
        const int32_t z = dev::ld_volatile(p + y);
        if (z != y) p[x] = z;
        x = y;
    }
}

// Union of the two ends of every edge (each edge once, from its smaller end).  A link
// retries while another thread changes the roots; the retries are bounded (a failed link
// means another link succeeded, so they cannot exceed the vertex count) and *err is set
// if the bound is ever reached.
__global__ void k_cc_union(const int32_t *rp, const int32_t *col, int32_t n, int32_t *p, int *err)
{
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x) {
        for (int32_t j = __ldg(rp + u); j < __ldg(rp + u + 1); ++j) {
            const int32_t v = __ldg(col + j);
            if (v <= u) continue;
            bool done = false;
            for (int32_t it = 0; it <= n && !done; ++it) {
                const int32_t ru = cc_find(p, (int32_t)u), rv = cc_find(p, v);
                if (ru == rv) { done = true; break; }
                const int32_t lo = min(ru, rv), hi = max(ru, rv);
                done = atomicCAS(p + hi, hi, lo) == hi;
            }
            if (!done) atomicExch(err, 1);
        }
    }
}

// Once every union is done: root[v] by a read-only walk (no halving stores here, which
// could overwrite another thread's result), and the BFS start (distance 0 at the roots).
__global__ void k_cc_roots(const int32_t *p, int32_t n, int32_t *root, int32_t *dist)
{
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        int32_t r = (int32_t)v;
        while (p[r] != r) r = p[r];
        root[v] = r;
        dist[v] = r == v ? 0 : -1;
    }
}

// One level of the BFS from all roots: vertices at distance d claim their unvisited
// neighbours for d + 1.
__global__ void k_bfs_level(const int32_t *rp, const int32_t *col, int32_t n, int32_t *dist, int32_t d,
                            int *changed)
{
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        if (dist[v] != d) continue;
        for (int32_t j = __ldg(rp + v); j < __ldg(rp + v + 1); ++j) {
            const int32_t w = __ldg(col + j);
            if (dev::ld_volatile(dist + w) == -1 && atomicCAS(dist + w, -1, d + 1) == -1) *changed = 1;
        }
    }
}

__global__ void k_cc_stats(const int32_t *root, const int32_t *dist, int32_t n, int32_t *ecc, int32_t *size)
{
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        atomicMax(ecc + root[v], dist[v]);
        atomicAdd(size + root[v], 1);
    }
}

__global__ void k_cc_bound(const int32_t *root, const int32_t *ecc, const int32_t *size, int32_t n, int32_t *vd)
{
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        if (root[v] != v) continue;
        const int64_t b = std::min<int64_t>(size[v], 2 * (int64_t)ecc[v] + 1);
        atomicMax(vd, (int32_t)b);
    }
}

// Pair i: u = below(stream(seed, 3i), n), v = below(stream(seed, 3i+1), n-1) shifted past
// u, and the key of its path walk, stream(seed, 3i+2).
__global__ void k_rk_pairs(uint64_t seed, int32_t n, int64_t r, int32_t *src, int32_t *tgt,
                           unsigned long long *key)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < r; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t u = (int32_t)dev::below(dev::stream_at(seed, 3 * (uint64_t)i), (uint64_t)n);
        int32_t v = (int32_t)dev::below(dev::stream_at(seed, 3 * (uint64_t)i + 1), (uint64_t)(n - 1));
        if (v >= u) ++v;
        src[i] = u;
        tgt[i] = v;
        key[i] = dev::stream_at(seed, 3 * (uint64_t)i + 2);
    }
}

int grid_for(int64_t items) { return (int)std::max<int64_t>(1, std::min<int64_t>((items + 255) / 256, 8LL * num_sms())); }

}  // namespace

int vertex_diameter_bound(nk_graph *g, cudaStream_t s, int32_t *vd_out)
{
    if (g->vd_est > 0) {
        *vd_out = g->vd_est;
        return NK_OK;
    }
    const int32_t n = g->n;
    Tmp buf;
    // parent, root, dist, ecc, size (int32 each), then err, changed, vd
    NK_TRY(buf.alloc(sizeof(int32_t) * (5 * (size_t)n + 3), s));
    int32_t *p = buf.as<int32_t>(), *root = p + n, *dist = root + n, *ecc = dist + n, *size = ecc + n;
    int *flags = reinterpret_cast<int *>(size + n);  // err, changed, vd
    NK_CUDA(cudaMemsetAsync(ecc, 0, sizeof(int32_t) * (2 * (size_t)n + 3), s));
    const int32_t *rp = g->rp.as<int32_t>(), *col = g->col.as<int32_t>();
    k_cc_init<<<grid_for(n), 256, 0, s>>>(p, n);
    k_cc_union<<<grid_for(n), 256, 0, s>>>(rp, col, n, p, flags);
    k_cc_roots<<<grid_for(n), 256, 0, s>>>(p, n, root, dist);
    count_launch();
    count_launch();
    count_launch();
    NK_CUDA(cudaGetLastError());
    int h[2] = {0, 0};
    for (int32_t d = 0; d < n; ++d) {
        NK_CUDA(cudaMemsetAsync(flags + 1, 0, sizeof(int), s));
        k_bfs_level<<<grid_for(n), 256, 0, s>>>(rp, col, n, dist, d, flags + 1);
        count_launch();
        NK_CUDA(cudaMemcpyAsync(h, flags, sizeof(int) * 2, cudaMemcpyDeviceToHost, s));
        NK_CUDA(cudaStreamSynchronize(s));
        if (h[0]) return set_error(NK_ERR_CUDA, "connected components: a union did not settle");
        if (!h[1]) break;
    }
    k_cc_stats<<<grid_for(n), 256, 0, s>>>(root, dist, n, ecc, size);
    k_cc_bound<<<grid_for(n), 256, 0, s>>>(root, ecc, size, n, flags + 2);
    count_launch();
    count_launch();
    int32_t vd = 0;
    NK_CUDA(cudaMemcpyAsync(&vd, flags + 2, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    NK_CUDA(cudaStreamSynchronize(s));
    g->vd_est = vd;
    *vd_out = vd;
    return NK_OK;
}

int64_t rk_sample_count(double eps, double delta, int32_t vd)
{
    if (!(eps > 0.0 && eps < 1.0) || !(delta > 0.0 && delta < 1.0) || vd < 1) return -1;
    const int64_t x = std::max<int64_t>(1, (int64_t)vd - 2);
    int lg = 0;
    while ((x >> (lg + 1)) != 0) ++lg;  // floor(log2 x)
    const double r = std::ceil(0.5 / (eps * eps) * ((double)lg + 1.0 + std::log(1.0 / delta)));
    if (!(r <= 2147483647.0)) return -1;
    return (int64_t)r;
}

int rk_pairs(uint64_t seed, int32_t n, int64_t r, int32_t *src, int32_t *tgt, unsigned long long *key,
             cudaStream_t s)
{
    if (r <= 0) return NK_OK;
    k_rk_pairs<<<grid_for(r), 256, 0, s>>>(seed, n, r, src, tgt, key);
    count_launch();
    NK_CUDA(cudaGetLastError());
    return NK_OK;
}

}  // namespace nk

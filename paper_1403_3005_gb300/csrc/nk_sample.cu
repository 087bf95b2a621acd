// Source sampler for the sampled betweenness estimate (Section 3.2: betweenness from a
// small number of randomly chosen shortest-path trees, after Geisberger et al.).
//
// Rule: k distinct sources uniformly without replacement = the k vertices with the
// smallest key(v) = v-th output of the SplitMix64 stream seeded with `seed`.  The keys
// are distinct (v -> seed + (v+1)*gamma is a bijection mod 2^64 for odd gamma, and the
// finaliser is a bijection), so the selection is a threshold: key(v) <= T where T is
// the k-th smallest key.  T is found by an 8-pass radix select over 8-bit digits
// (keys are recomputed, never stored); the chosen ids are then written in ascending
// order by an order-preserving compaction.  No sort is needed.
#include "nk_device.cuh"
#include "nk_internal.h"

namespace nk {
namespace {

struct SelState {
    uint64_t prefix;  // digits of T fixed so far
    uint64_t mask;    // which bits of the prefix are fixed
    int64_t krem;     // rank of T among the keys that match the prefix (1-based)
};

__global__ void k_sel_init(SelState *s, int64_t k, unsigned *hist)
{
    s->prefix = 0;
    s->mask = 0;
    s->krem = k;
    for (int i = threadIdx.x; i < 256; i += blockDim.x) hist[i] = 0;
}

__global__ void k_sel_hist(int32_t n, uint64_t seed, const SelState *s, int shift,
                           unsigned *hist)
{
    __shared__ unsigned h[256];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const uint64_t prefix = s->prefix, mask = s->mask;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t key = dev::stream_at(seed, (uint64_t)v);
        if ((key & mask) == prefix) atomicAdd(&h[(key >> shift) & 255u], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 256; i += blockDim.x)
        if (h[i]) atomicAdd(&hist[i], h[i]);
}

// one warp: choose the digit holding the krem-th key, then clear the histogram
__global__ void k_sel_digit(SelState *s, int shift, unsigned *hist)
{
    if (threadIdx.x == 0) {
        int64_t krem = s->krem;
        int d = 0;
        for (; d < 255; ++d) {
            if ((int64_t)hist[d] >= krem) break;
            krem -= hist[d];
        }
        s->krem = krem;
        s->prefix |= (uint64_t)d << shift;
        s->mask |= 255ull << shift;
    }
    __syncwarp();
    for (int i = threadIdx.x; i < 256; i += blockDim.x) hist[i] = 0;
}

constexpr int kTileV = 1024;

__global__ void __launch_bounds__(kTileV)
k_sel_count(int32_t n, uint64_t seed, const SelState *s, int64_t *tile_cnt)
{
    __shared__ int wc[32];
    const int64_t v = (int64_t)blockIdx.x * kTileV + threadIdx.x;
    const bool pick = v < n && dev::stream_at(seed, (uint64_t)v) <= s->prefix;
    const unsigned bal = __ballot_sync(0xffffffffu, pick);
    if ((threadIdx.x & 31) == 0) wc[threadIdx.x >> 5] = __popc(bal);
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int i = 0; i < 32; ++i) t += wc[i];
        tile_cnt[blockIdx.x] = t;
    }
}

__global__ void __launch_bounds__(kTileV)
k_sel_write(int32_t n, uint64_t seed, const SelState *s, const int64_t *tile_off,
            int32_t *src)
{
    __shared__ int wc[32];
    const int64_t v = (int64_t)blockIdx.x * kTileV + threadIdx.x;
    const bool pick = v < n && dev::stream_at(seed, (uint64_t)v) <= s->prefix;
    const unsigned bal = __ballot_sync(0xffffffffu, pick);
    const int wid = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) wc[wid] = __popc(bal);
    __syncthreads();
    int before = 0;
    for (int i = 0; i < wid; ++i) before += wc[i];
    if (pick) src[tile_off[blockIdx.x] + before + __popc(bal & dev::lanemask_lt())] = (int32_t)v;
}

}  // namespace

int sample_sources_device(int32_t n, uint64_t seed, int32_t k, int32_t *d_src, cudaStream_t st)
{
    if (n < 1 || k < 1 || k > n) return set_error(NK_ERR_ARG, "need 1 <= k <= n (k=%d, n=%d)", k, n);
    Tmp state, hist, tiles;
    NK_TRY(state.alloc(sizeof(SelState), st));
    NK_TRY(hist.alloc(256 * sizeof(unsigned), st));
    const int64_t ntiles = ((int64_t)n + kTileV - 1) / kTileV;
    NK_TRY(tiles.alloc(sizeof(int64_t) * ntiles, st));
    SelState *S = state.as<SelState>();
    unsigned *H = hist.as<unsigned>();
    k_sel_init<<<1, 256, 0, st>>>(S, k, H);
    ::nk::count_launch();
    NK_CUDA(cudaGetLastError());
    int blocks = (int)std::min<int64_t>(((int64_t)n + 255) / 256, 4LL * num_sms());
    for (int pass = 0; pass < 8; ++pass) {
        const int shift = 56 - 8 * pass;
        k_sel_hist<<<blocks, 256, 0, st>>>(n, seed, S, shift, H);
        ::nk::count_launch();
        k_sel_digit<<<1, 32, 0, st>>>(S, shift, H);
        ::nk::count_launch();
    }
    NK_CUDA(cudaGetLastError());
    k_sel_count<<<(unsigned)ntiles, kTileV, 0, st>>>(n, seed, S, tiles.as<int64_t>());
    ::nk::count_launch();
    NK_CUDA(cudaGetLastError());
    NK_TRY(scan_exclusive_i64(tiles.as<int64_t>(), tiles.as<int64_t>(), ntiles, nullptr, st));
    k_sel_write<<<(unsigned)ntiles, kTileV, 0, st>>>(n, seed, S, tiles.as<int64_t>(), d_src);
    ::nk::count_launch();
    NK_CUDA(cudaGetLastError());
    return NK_OK;
}

}  // namespace nk

using namespace nk;

extern "C" int nk_sample_sources(int32_t n, uint64_t seed, int32_t k, int32_t *src, uint32_t flags)
{
    if (!src) return set_error(NK_ERR_ARG, "src is null");
    if (n < 1 || k < 1 || k > n) return set_error(NK_ERR_ARG, "need 1 <= k <= n (k=%d, n=%d)", k, n);
    cudaStream_t st = stream();
    if (flags & NK_RUN_DEVICE_PTRS) {
        NK_TRY(sample_sources_device(n, seed, k, src, st));
        NK_CUDA(cudaStreamSynchronize(st));
        return NK_OK;
    }
    Tmp d;
    NK_TRY(d.alloc(sizeof(int32_t) * k, st));
    NK_TRY(sample_sources_device(n, seed, k, d.as<int32_t>(), st));
    NK_CUDA(cudaMemcpyAsync(src, d.p, sizeof(int32_t) * k, cudaMemcpyDeviceToHost, st));
    NK_CUDA(cudaStreamSynchronize(st));
    return NK_OK;
}

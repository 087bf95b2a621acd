// Core runtime of libnk: error state, stream selection, device buffers, the prefix-sum
// primitive, and the bounded-wait self test.
#include <chrono>
#include <cstdio>
#include <cstring>
#include <string>
#include <thread>

#include "nk_device.cuh"
#include "nk_internal.h"

namespace nk {

// ---------------------------------------------------------------- errors
static thread_local std::string t_err;

int set_error(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    t_err = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char *what, const char *file, int line)
{
    return set_error(NK_ERR_CUDA, "%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file,
                     line);
}

std::atomic<uint64_t> g_launches{0};
std::atomic<uint64_t> g_allocs{0};

// ---------------------------------------------------------------- stream / limits
static std::atomic<cudaStream_t> g_stream{nullptr};
static std::atomic<uint64_t> g_wait_ns{10ull * 1000 * 1000 * 1000};

cudaStream_t stream() { return g_stream.load(); }
uint64_t wait_limit_ns() { return g_wait_ns.load(); }

int num_sms()
{
    static int sms = 0;
    if (sms == 0) {
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        sms = v > 0 ? v : 1;
    }
    return sms;
}

// ---------------------------------------------------------------- buffers
// The device's default memory pool, which the stream-ordered allocations of the library
// draw from, keeps freed memory for reuse instead of returning it to the driver at every
// synchronisation (its release threshold is raised once per device; the pool belongs to
// this process).
static void keep_pool_memory()
{
    static std::atomic<unsigned long long> done{0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return;
    const unsigned long long bit = 1ull << dev;
    if (done.load() & bit) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t keep = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    cudaGetLastError();
    done.fetch_or(bit);
}

int DevBuf::ensure(size_t b)
{
    if (b <= bytes && p) return NK_OK;
    release();
    size_t want = b < 256 ? 256 : b;
    count_alloc();
    if (stream_ordered) keep_pool_memory();
    cudaError_t e = stream_ordered ? cudaMallocAsync(&p, want, st) : cudaMalloc(&p, want);
    if (e != cudaSuccess) {
        p = nullptr;
        bytes = 0;
        cudaGetLastError();
        return set_error(NK_ERR_NOMEM, "cudaMalloc(%zu) failed: %s", want, cudaGetErrorString(e));
    }
    bytes = want;
    return NK_OK;
}

void DevBuf::release()
{
    if (p) {
        if (stream_ordered) cudaFreeAsync(p, st);
        else cudaFree(p);
    }
    p = nullptr;
    bytes = 0;
}

int Tmp::alloc(size_t b, cudaStream_t s)
{
    st = s;
    count_alloc();
    keep_pool_memory();
    cudaError_t e = cudaMallocAsync(&p, b < 256 ? 256 : b, s);
    if (e != cudaSuccess) {
        p = nullptr;
        cudaGetLastError();
        return set_error(NK_ERR_NOMEM, "cudaMallocAsync(%zu) failed: %s", b,
                         cudaGetErrorString(e));
    }
    return NK_OK;
}

Tmp::~Tmp()
{
    if (p) cudaFreeAsync(p, st);
}

// ---------------------------------------------------------------- bounded host wait
int host_wait(cudaStream_t s, int64_t launches, uint64_t limit_ns)
{
    cudaEvent_t ev = nullptr;
    NK_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    cudaError_t e = cudaEventRecord(ev, s);
    if (e != cudaSuccess) {
        cudaEventDestroy(ev);
        return cuda_fail(e, "cudaEventRecord", __FILE__, __LINE__);
    }
    const double budget_s = (double)(launches + 1) * 64.0 * (double)limit_ns * 1e-9;
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        e = cudaEventQuery(ev);
        if (e != cudaErrorNotReady) break;
        const double waited = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (waited > budget_s) {
            cudaEventDestroy(ev);
            return set_error(NK_ERR_TIMEOUT, "the host gave up waiting for %lld launches after %.0f s",
                             (long long)launches, waited);
        }
        if (waited < 2e-3) std::this_thread::yield();
        else std::this_thread::sleep_for(std::chrono::microseconds(100));
    }
    cudaEventDestroy(ev);
    if (e != cudaSuccess) return cuda_fail(e, "kernel execution", __FILE__, __LINE__);
    return NK_OK;
}

// ---------------------------------------------------------------- exclusive scan
// Tiles of 1024 threads x 4 items; tile totals are scanned recursively.
namespace {
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kTile = kScanThreads * kScanItems;

__global__ void __launch_bounds__(kScanThreads)
k_scan_tile(const int64_t *in, int64_t *out, int64_t *tile_sum, int64_t count)
{
    __shared__ int64_t warp_tot[32];
    const int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kScanItems;
    int64_t v[kScanItems];
    int64_t run = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        int64_t x = base + i < count ? in[base + i] : 0;
        v[i] = run;
        run += x;
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t incl = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_tot[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        int64_t t = warp_tot[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        warp_tot[lane] = t;  // inclusive over warps
    }
    __syncthreads();
    int64_t excl = incl - run + (wid > 0 ? warp_tot[wid - 1] : 0);
#pragma unroll
    for (int i = 0; i < kScanItems; ++i)
        if (base + i < count) out[base + i] = excl + v[i];
    if (threadIdx.x == kScanThreads - 1 && tile_sum) tile_sum[blockIdx.x] = excl + run;
}

__global__ void k_scan_add(int64_t *out, const int64_t *tile_off, int64_t count)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) out[i] += tile_off[i / kTile];
}

__global__ void k_scan_total(const int64_t *in, const int64_t *out, int64_t count,
                             int64_t *total)
{
    *total = count > 0 ? out[count - 1] + in[count - 1] : 0;
}

int scan_rec(const int64_t *in, int64_t *out, int64_t count, cudaStream_t st)
{
    if (count <= 0) return NK_OK;
    const int64_t tiles = (count + kTile - 1) / kTile;
    if (tiles == 1) {
        k_scan_tile<<<1, kScanThreads, 0, st>>>(in, out, nullptr, count);
        ::nk::count_launch();
        NK_CUDA(cudaGetLastError());
        return NK_OK;
    }
    Tmp sums;
    NK_TRY(sums.alloc(sizeof(int64_t) * tiles, st));
    k_scan_tile<<<(unsigned)tiles, kScanThreads, 0, st>>>(in, out, sums.as<int64_t>(), count);
    ::nk::count_launch();
    NK_CUDA(cudaGetLastError());
    NK_TRY(scan_rec(sums.as<int64_t>(), sums.as<int64_t>(), tiles, st));
    k_scan_add<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(out, sums.as<int64_t>(), count);
    ::nk::count_launch();
    NK_CUDA(cudaGetLastError());
    return NK_OK;
}
}  // namespace

int scan_exclusive_i64(const int64_t *in, int64_t *out, int64_t count, int64_t *total,
                       cudaStream_t st)
{
    // the total needs the last input, which an in-place scan overwrites
    int64_t *last = nullptr;
    Tmp keep;
    if (total && count > 0) {
        NK_TRY(keep.alloc(sizeof(int64_t), st));
        last = keep.as<int64_t>();
        NK_CUDA(cudaMemcpyAsync(last, in + count - 1, sizeof(int64_t), cudaMemcpyDeviceToDevice, st));
    }
    NK_TRY(scan_rec(in, out, count, st));
    if (total) {
        if (count > 0) {
            k_scan_total<<<1, 1, 0, st>>>(last, out + count - 1, 1, total);
            ::nk::count_launch();
            NK_CUDA(cudaGetLastError());
        } else {
            NK_CUDA(cudaMemsetAsync(total, 0, sizeof(int64_t), st));
        }
    }
    return NK_OK;
}

// ---------------------------------------------------------------- sources with arcs
namespace {
constexpr int kCompactThreads = 1024;

// Stable compaction by one CTA: out[0..count) = the sources of src[0..k) with at least one
// arc, in their order; *count receives their number.  Tiles of 1024 sources: a flag per
// thread, warp ballots, a scan of the 32 warp counts, and a running offset.
__global__ void __launch_bounds__(kCompactThreads)
k_compact_sources(const int32_t *rp, const int32_t *src, int32_t k, int32_t *out, int32_t *count)
{
    __shared__ int warp_cnt[32];
    __shared__ int tile_base;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (threadIdx.x == 0) tile_base = 0;
    __syncthreads();
    for (int64_t t0 = 0; t0 < k; t0 += kCompactThreads) {
        const int64_t i = t0 + threadIdx.x;
        int v = 0;
        bool keep = false;
        if (i < k) {
            v = src[i];
            keep = rp[v + 1] > rp[v];
        }
        const unsigned m = __ballot_sync(0xffffffffu, keep);
        if (lane == 0) warp_cnt[wid] = __popc(m);
        __syncthreads();
        if (wid == 0) {
            int x = warp_cnt[lane], incl = x;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            warp_cnt[lane] = incl - x;  // exclusive over warps
        }
        __syncthreads();
        const int base = tile_base;
        if (keep) out[base + warp_cnt[wid] + __popc(m & ((1u << lane) - 1u))] = v;
        __syncthreads();
        if (threadIdx.x == kCompactThreads - 1) tile_base = base + warp_cnt[wid] + __popc(m);
        __syncthreads();
    }
    if (threadIdx.x == 0) *count = tile_base;
}
}  // namespace

int compact_sources(const nk_graph *g, const int32_t *d_src, int32_t k, int32_t *d_out, int32_t *d_count,
                    cudaStream_t s)
{
    k_compact_sources<<<1, kCompactThreads, 0, s>>>(g->rp.as<int32_t>(), d_src, k, d_out, d_count);
    ::nk::count_launch();
    NK_CUDA(cudaGetLastError());
    return NK_OK;
}

// ---------------------------------------------------------------- vector scale
namespace {
__global__ void k_scale(double *d, int32_t n, double s)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        d[i] *= s;
}
}  // namespace

int scale_vector(double *d, int32_t n, double scale, cudaStream_t s)
{
    if (scale == 1.0 || n <= 0) return NK_OK;
    int blocks = (int)((n + 255) / 256);
    if (blocks > 8 * num_sms()) blocks = 8 * num_sms();
    k_scale<<<blocks, 256, 0, s>>>(d, n, scale);
    ::nk::count_launch();
    NK_CUDA(cudaGetLastError());
    return NK_OK;
}

// ---------------------------------------------------------------- bounded-wait self test
namespace {
// Waits on *flag (which nothing sets) with the same bounded poll as the grid barrier,
// and records NK_ERR_TIMEOUT when the bound runs out.
__global__ void k_wait_flag(const int *flag, int *status, uint64_t limit_ns)
{
    const uint64_t t0 = dev::globaltimer();
    uint32_t polls = 0;
    while (dev::ld_volatile(flag) == 0) {
        ++polls;
        if ((polls & 63u) == 0 && (dev::globaltimer() - t0 > limit_ns || polls >= 0x80000000u)) {
            *status = NK_ERR_TIMEOUT;
            return;
        }
        __nanosleep(256);
    }
    *status = NK_OK;
}
}  // namespace

}  // namespace nk

using namespace nk;

extern "C" {

const char *nk_last_error(void) { return t_err.c_str(); }

const char *nk_version(void) { return "nk-gb300 0.1 (sm_103a)"; }

uint64_t nk_launch_count(void) { return g_launches.load(); }

uint64_t nk_alloc_count(void) { return g_allocs.load(); }

int nk_set_stream(void *s)
{
    g_stream.store(static_cast<cudaStream_t>(s));
    return NK_OK;
}

int nk_set_wait_limit_ns(uint64_t ns)
{
    if (ns == 0) return set_error(NK_ERR_ARG, "wait limit must be > 0");
    g_wait_ns.store(ns);
    return NK_OK;
}

int nk_selftest_wait_timeout(uint64_t limit_ns)
{
    if (limit_ns == 0 || limit_ns > 10ull * 1000 * 1000 * 1000)
        return set_error(NK_ERR_ARG, "limit_ns must be in (0, 10 s]");
    cudaStream_t st = stream();
    Tmp buf;
    NK_TRY(buf.alloc(2 * sizeof(int), st));
    int *flag = buf.as<int>(), *status = flag + 1;
    NK_CUDA(cudaMemsetAsync(flag, 0, 2 * sizeof(int), st));
    k_wait_flag<<<1, 1, 0, st>>>(flag, status, limit_ns);
    ::nk::count_launch();
    NK_CUDA(cudaGetLastError());
    int h = 1;
    NK_CUDA(cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, st));
    NK_CUDA(cudaStreamSynchronize(st));
    if (h == NK_ERR_TIMEOUT) return set_error(NK_ERR_TIMEOUT, "bounded wait ran out (as intended)");
    return h;
}

}  // extern "C"

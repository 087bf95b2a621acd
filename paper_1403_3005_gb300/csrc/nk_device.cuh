// Device-side helpers shared by the kernels of libnk.
#pragma once

#include <cuda_runtime.h>
#include <cooperative_groups.h>

#include <cstdint>

#include "nk_internal.h"

namespace nk {
namespace dev {

// ---------------------------------------------------------------- SplitMix64
// Steele, Lea and Flood, "Fast splittable pseudorandom number generators" (OOPSLA
// 2014): the generator adds the golden-ratio constant to its state and returns the
// state through the 64-bit finaliser.  Used as a counter-based generator: the i-th
// output of the stream seeded with `seed` is mix64(seed + (i+1) * gamma).
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__host__ __device__ __forceinline__ uint64_t stream_at(uint64_t seed, uint64_t i)
{
    return mix64(seed + (i + 1) * 0x9E3779B97F4A7C15ull);
}

// floor(x * b / 2^64): a uniform integer in [0, b) from a uniform 64-bit x (Lemire's
// multiply-high, without rejection).
__device__ __forceinline__ uint64_t below(uint64_t x, uint64_t b) { return __umul64hi(x, b); }

// ---------------------------------------------------------------- memory access
// Loads of data that other CTAs write during the same persistent launch bypass L1
// (ld.global.cg): L1 is not coherent across SMs.
template <class T> __device__ __forceinline__ T ldcg(const T *p) { return __ldcg(p); }

__device__ __forceinline__ unsigned ld_volatile(const unsigned *p)
{
    return *reinterpret_cast<const volatile unsigned *>(p);
}
__device__ __forceinline__ int ld_volatile(const int *p)
{
    return *reinterpret_cast<const volatile int *>(p);
}

__device__ __forceinline__ uint64_t globaltimer()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// ---------------------------------------------------------------- grid barrier
// Barrier over all CTAs of a cooperative (co-resident) launch.  The wait is bounded:
// after `limit_ns` of globaltimer time, or 2^31 polls, the waiting CTA records
// NK_ERR_TIMEOUT in ctrl->err and every CTA returns false from then on, so that the
// kernel ends and the host reads the status.  A CTA also stops waiting as soon as
// another CTA has recorded an error.
__device__ __forceinline__ bool grid_barrier(Ctrl *ctrl, uint64_t limit_ns)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        unsigned gen = ld_volatile(&ctrl->bar_gen);
        __threadfence();
        unsigned arrived = atomicAdd(&ctrl->bar_count, 1u);
        if (arrived == gridDim.x - 1) {
            atomicExch(&ctrl->bar_count, 0u);
            __threadfence();
            atomicAdd(&ctrl->bar_gen, 1u);
        } else {
            const uint64_t t0 = globaltimer();
            uint32_t polls = 0;
            while (ld_volatile(&ctrl->bar_gen) == gen) {
                if (ld_volatile(&ctrl->err) != 0) { ok = 0; break; }
                ++polls;
                if ((polls & 63u) == 0) {
                    if (globaltimer() - t0 > limit_ns || polls >= 0x80000000u) {
                        atomicCAS(&ctrl->err, 0, NK_ERR_TIMEOUT);
                        ok = 0;
                        break;
                    }
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        if (ld_volatile(&ctrl->err) != 0) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// ---------------------------------------------------------------- small reductions
template <int W, class T> __device__ __forceinline__ T group_sum(T x)
{
#pragma unroll
    for (int o = W / 2; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o, W);
    return x;
}

// Sum of uint64 path counts over a group of W lanes, with carry detection.
template <int W> __device__ __forceinline__ uint64_t group_sum_u64(uint64_t x, bool &ovf)
{
#pragma unroll
    for (int o = W / 2; o > 0; o >>= 1) {
        uint64_t y = __shfl_xor_sync(0xffffffffu, x, o, W);
        uint64_t z = x + y;
        ovf |= z < x;
        x = z;
    }
    return x;
}

// ---------------------------------------------------------------- double-single numbers
// A value held as the unevaluated sum hi + lo of two floats (about 48 significant bits),
// after Dekker ("A floating-point technique for extending the available precision",
// 1971) and Knuth's TwoSum (TAOCP vol. 2, 4.2.2).  The backward sweep accumulates its
// dependency sums in this form on the FP32 pipe: on this GPU the FP64 pipe issues about
// two lanes per clock per SM, so one warp-wide FP64 add costs ~16 SM clocks, while the
// ~11 FP32 operations of a double-single add cost ~3.  Every operation is explicitly
// rounded so that the compiler cannot contract or reorder it.  All operands on the
// betweenness path are non-negative, where these forms are accurate to ~2^-44 relative.
struct ff {
    float hi, lo;
};

__device__ __forceinline__ ff ff_zero() { return {0.0f, 0.0f}; }

// s + t with |s| >= |t| (FastTwoSum): renormalised pair
__device__ __forceinline__ ff ff_fast2sum(float s, float t)
{
    const float hi = __fadd_rn(s, t);
    return {hi, __fsub_rn(t, __fsub_rn(hi, s))};
}

__device__ __forceinline__ ff ff_add(ff a, ff b)
{
    const float s = __fadd_rn(a.hi, b.hi);
    const float v = __fsub_rn(s, a.hi);
    const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, v)), __fsub_rn(b.hi, v));  // TwoSum error
    return ff_fast2sum(s, __fadd_rn(e, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ ff ff_mul(ff a, ff b)
{
    const float p = __fmul_rn(a.hi, b.hi);
    const float e = __fmaf_rn(a.hi, b.hi, -p);  // exact error of the leading product
    return ff_fast2sum(p, __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e)));
}

// 1/x: the float reciprocal of x.hi refined by one Newton step r + r(1 - x r) carried
// out in double-single (1 - x.hi r is exact by Sterbenz, its FMA error term is exact).
__device__ __forceinline__ ff ff_rcp(ff x)
{
    const float r0 = __frcp_rn(x.hi);
    const float p = __fmul_rn(x.hi, r0);
    const float pe = __fmaf_rn(x.hi, r0, -p);
    const float e = __fsub_rn(__fsub_rn(__fsub_rn(1.0f, p), pe), __fmul_rn(x.lo, r0));
    return ff_fast2sum(r0, __fmul_rn(r0, e));
}

// exact-to-~2^-47 conversion of a path count: truncated leading float plus the rounded
// integer remainder
__device__ __forceinline__ ff ff_from_u64(unsigned long long x)
{
    const float hi = __ull2float_rz(x);
    const float lo = __ull2float_rn(x - __float2ull_rz(hi));
    return ff_fast2sum(hi, lo);
}

__device__ __forceinline__ double ff_to_double(ff a) { return (double)a.hi + (double)a.lo; }

// 8-byte storage: hi in the low word, lo in the high word
__device__ __forceinline__ unsigned long long ff_pack(ff a)
{
    return ((unsigned long long)__float_as_uint(a.lo) << 32) | __float_as_uint(a.hi);
}
__device__ __forceinline__ ff ff_unpack(unsigned long long u)
{
    return {__uint_as_float((unsigned)(u & 0xffffffffu)), __uint_as_float((unsigned)(u >> 32))};
}

template <int W> __device__ __forceinline__ ff group_sum_ff(ff x)
{
#pragma unroll
    for (int o = W / 2; o > 0; o >>= 1) {
        ff y;
        y.hi = __shfl_xor_sync(0xffffffffu, x.hi, o, W);
        y.lo = __shfl_xor_sync(0xffffffffu, x.lo, o, W);
        x = ff_add(x, y);
    }
    return x;
}

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

}  // namespace dev
}  // namespace nk

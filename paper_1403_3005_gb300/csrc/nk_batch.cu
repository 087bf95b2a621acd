// Batched multi-source betweenness: B = 64*W sources share one persistent cooperative
// launch.  The paper parallelises Brandes' algorithm over sources with one dependency
// array per thread, summed at the end (Section 3.2); on the GPU the sources of a batch
// instead share every pass over the CSR, so the adjacency of a level is read once for
// all B shortest-path trees.
//
// State of one batch, all in HBM (b = source slot 0..B-1, q = word 0..W-1):
//   F_d[v][q]   bitset of the sources for which v is at BFS level d (one slab per
//               level, kept for the backward sweep)
//   vis[v][q]   union of F_0..F_d
//   sp[v][b]    sigma_b(v) (uint64) during the forward sweep; replaced by
//               psi_b(v) = (1 + delta_b(v)) / sigma_b(v) in the backward sweep (a
//               double-single pair of floats, see nk_device.cuh)
//   queue       vertices of the levels found top-down (levels found bottom-up are
//               iterated by scanning F_d)
// Forward level d, either
//   bottom-up  every vertex w with unvisited sources u = act & ~vis[w] gathers F_d of
//              its neighbours (one warp per vertex, lanes over neighbours); for every
//              neighbour c with F_d[c] & u != 0 the lanes switch to one lane per source
//              bit and add sigma_b(c) (the sigma row of c is contiguous, so the gather
//              reads only the sectors of the sources that need it);
//              F_{d+1}[w] = the bits whose sum is non-zero;  or
//   top-down   (a) every frontier vertex v pushes m = F_d[v] & ~vis[c] into F_{d+1}[c]
//              (atomicOr) and queues c once per level; (b) every queued vertex w pulls
//              sigma for exactly its new bits F_{d+1}[w], as above.  sigma is never
//              updated atomically, so sp needs no zeroing.
// Backward level d (deepest first): every v with F_d[v] != 0 gathers, per source bit b
// of F_d[v], acc_b = sum of psi_b(c) over neighbours c with bit b in F_{d+1}[c]; then
// delta_b(v) = sigma_b(v) * acc_b (Brandes' recurrence with sigma_v factored out), psi
// overwrites sigma, and scores[v] += sum_b delta_b(v).
// Bottom-up is chosen when alpha * (arcs of frontier vertices) > (arcs of vertices not
// yet visited by every source).  A BFS deeper than the level slabs aborts the batch
// before its backward sweep (scores untouched); the host re-runs those sources with
// the per-source form.
#include <cooperative_groups.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "nk_device.cuh"
#include "nk_internal.h"

namespace cg = cooperative_groups;

namespace nk {
namespace {

constexpr int kThreads = 256;
constexpr int kErrDepth = 100;  // internal status: BFS deeper than the level slabs
constexpr int kErrCheck = 101;  // internal status: a device-side range check failed
constexpr int kErrWide = 102;   // internal status: a path count did not fit the 32-bit sigma rows
constexpr int kStartLevels = 48; // level slabs of a first attempt
constexpr unsigned FULL = 0xffffffffu;
constexpr int kTraceCap = 1024;
constexpr int kChunk = kHeavyChunk;  // default arcs per work item; longer rows are split
constexpr int kGrabQ = 8;            // queue entries a warp takes at a time
constexpr int kGrabV = 32;           // vertices a warp scans at a time (one ballot window)
constexpr int kGrabCMax = 16;        // most heavy chunks a warp takes at a time
// work-counter slots of a level
enum { WQ_BU = 0, WQ_BU_C, WQ_PUSH, WQ_PUSH_C, WQ_PULL, WQ_PULL_C, WQ_BACK, WQ_BACK_C };

struct BArgs {
    int32_t n;
    int64_t A;
    const int32_t *rp, *col;
    const int32_t *src;
    int32_t nsrc;
    // when set (captured calls), the number of sources of the whole run is *ksrc, read on
    // the device, and this batch has min(B, *ksrc - boff) of them (none: it returns at once)
    const int32_t *ksrc;
    int32_t boff;
    int32_t lcap;                // levels 0..lcap may be non-empty; slabs 0..lcap+1
    unsigned long long *F;       // [lcap+2][n][W]
    unsigned long long *vis;     // [n][W]
    unsigned long long *sp;      // [n][B]
    unsigned *sp32;              // [n][B] sigma in 32 bits during the forward sweep (kernels with S32)
    int32_t *qmark;              // [n] last level a vertex was queued for
    int32_t *queue;              // [qcap]
    int64_t qcap;
    int32_t *vcnt;               // [lcap+3] vertices with F_d != 0
    int32_t *qcnt;               // [lcap+3] queue entries of level d
    int32_t *qoff;               // [lcap+3] start of level d in queue, -1 if not queued
    unsigned long long *mfv;     // [lcap+3] sum of degrees of the level-d vertices
    unsigned long long *dmu;     // [lcap+3] degrees of vertices completed at level d
    int32_t *wq;                 // [lcap+3][8] work counters of the phases of level d
    double *scores;
    Ctrl *ctrl;
    uint64_t limit_ns;
    double alpha;
    int dir;
    // vertices of degree > chunk are split into chunks of `chunk` arcs (kChunk unless the
    // caller or the autotuner chose another size)
    int32_t chunk;
    const int32_t *hv;           // [H] heavy vertices
    const int32_t *hfirst;       // [H+1] first chunk of each heavy vertex
    const int32_t *chunk_h;      // [C] heavy index of each chunk
    int32_t H, C;
    unsigned long long *part;    // [C][B] per-chunk partial sums (uint64 or double)
    unsigned long long *trace;   // [kTraceCap][2] (code, globaltimer) after each barrier, or null
    unsigned long long *far;     // [n] closeness: sums of distances from the batch's sources, or null
    unsigned long long *reach;   // [n] closeness: number of the batch's sources that reach v
    int backward;                // 0: forward sweep only (closeness)
    double *edge;                // [A] edge betweenness: per-arc shares, or null
    // error-bounded estimate (forward sweep only): per source slot, the target of its
    // random shortest path and the key of the walk's stream; counts of interior vertices
    const int32_t *rk_t;
    const unsigned long long *rk_key;
    unsigned long long *rk_count;
};

template <int W> struct Bits {
    unsigned long long w[W];
};

template <int W> __device__ __forceinline__ Bits<W> load_bits(const unsigned long long *p)
{
    Bits<W> r;
    if constexpr (W == 1) {
        r.w[0] = __ldcg(p);
    } else {
#pragma unroll
        for (int q = 0; q < W; q += 2) {
            const ulonglong2 x = __ldcg(reinterpret_cast<const ulonglong2 *>(p + q));
            r.w[q] = x.x;
            r.w[q + 1] = x.y;
        }
    }
    return r;
}

template <int W> __device__ __forceinline__ bool any_bits(const Bits<W> &b)
{
    unsigned long long o = 0;
#pragma unroll
    for (int q = 0; q < W; ++q) o |= b.w[q];
    return o != 0;
}

template <int W> __device__ __forceinline__ Bits<W> shfl_bits(const Bits<W> &b, int src)
{
    Bits<W> r;
#pragma unroll
    for (int q = 0; q < W; ++q) r.w[q] = __shfl_sync(FULL, b.w[q], src);
    return r;
}

template <int W> __device__ __forceinline__ Bits<W> andnot(const Bits<W> &x, const Bits<W> &y)
{
    Bits<W> r;
#pragma unroll
    for (int q = 0; q < W; ++q) r.w[q] = x.w[q] & ~y.w[q];
    return r;
}

__device__ __forceinline__ int deg_of(const int32_t *rp, int v) { return __ldg(rp + v + 1) - __ldg(rp + v); }

// Source slots of a lane: lane L owns the G = 2W consecutive sources [G L, G L + G) of the
// batch.  Slot k of lane L is source G L + k: bit G L + k of the batch's bitsets (word
// (G L + k) / 64) and entry G L + k of a vertex's row of B values, so that one contiguous load
// moves all of a lane's values of a row, and the lane's bits of a bitset are one field of one
// word.
template <int W> __device__ __forceinline__ int slot_off(int k, int lane) { return 2 * W * lane + k; }

// The word of a bitset that holds the lane's slots (selected without indexing the register
// array by a run-time value, which would move it to local memory).
template <int W> __device__ __forceinline__ unsigned long long lane_word(const Bits<W> &b, int lane)
{
    // mask-and-or over the words: a select chain can be turned into an indexed access
    const int qi = (2 * W * lane) >> 6;
    unsigned long long w = 0ull;
#pragma unroll
    for (int q = 0; q < W; ++q) w |= b.w[q] & (0ull - (unsigned long long)(qi == q));
    return w;
}

template <int W> __device__ __forceinline__ bool has_slot(const Bits<W> &b, int k, int lane)
{
    return (lane_word<W>(b, lane) >> ((2 * W * lane + k) & 63)) & 1ull;
}

// The lane's 2W bits of a bitset of W words.
template <int W> __device__ __forceinline__ unsigned lane_bits(const unsigned long long *w, int lane)
{
    const int s = 2 * W * lane;
    return (unsigned)(w[s >> 6] >> (s & 63)) & ((1u << (2 * W)) - 1u);
}

// acc += x with the carry out of bit 63 counted in carry (a path-count overflow).
__device__ __forceinline__ void add_carry(unsigned long long &acc, unsigned &carry, unsigned long long x)
{
    asm("add.cc.u64 %0, %0, %2;\n\taddc.u32 %1, %1, 0;" : "+l"(acc), "+r"(carry) : "l"(x));
}

// Records the first failed device-side check (code, where, offending value); every CTA
// then leaves at its next grid barrier and the host reports the status.
__device__ __forceinline__ void check_failed(const BArgs &a, int code, int where, int value)
{
    if (atomicCAS(&a.ctrl->err, 0, code) == 0) {
        a.ctrl->where = where;
        a.ctrl->bad_id = value;
    }
}

// One warp's list of the relevant neighbours of the current 32-arc window of a gather:
// their ids, masked source bits and arc indices, in shared memory.
template <int W> struct Nbrs {
    unsigned long long f[32][W];
    int c[32];
    int j[32];
    double e[32];  // edge variant: each listed arc's share of the window
};

// sum_k sv[k] * x[k] over the lane's G slots (x: double-single pairs packed in 64 bits, zero
// for slots that are not relevant), as a compensated dot product (Ogita, Rump and Oishi's
// Dot2): the leading products hi*hi are summed by TwoSum, and their exact FMA errors, the
// cross terms hi*lo and lo*hi and the TwoSum errors are gathered in one float instead of
// renormalising the pair after every term.  All terms are non-negative (sigma and psi are),
// so the gathered float stays a small fraction of the sum.
template <int G>
__device__ __forceinline__ dev::ff edge_dot(const dev::ff *sv, const unsigned long long (&x)[G])
{
    float s = 0.0f, c = 0.0f;
#pragma unroll
    for (int k = 0; k < G; ++k) {
        const dev::ff b = dev::ff_unpack(x[k]);
        const float p = __fmul_rn(sv[k].hi, b.hi);
        c = __fmaf_rn(sv[k].hi, b.lo, __fmaf_rn(sv[k].lo, b.hi, __fadd_rn(c, __fmaf_rn(sv[k].hi, b.hi, -p))));
        const float t = __fadd_rn(s, p);
        const float z = __fsub_rn(t, s);
        c = __fadd_rn(c, __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z)));  // TwoSum error
        s = t;
    }
    return {s, c};  // not renormalised: edge_sum2 and ff_to_double take the pair as it is
}

// a + b for pairs whose second parts are small non-negative corrections (edge_dot's
// results): the leading parts by TwoSum, its error and both corrections into the second
// part, without renormalising
__device__ __forceinline__ dev::ff edge_sum2(dev::ff a, dev::ff b)
{
    const float t = __fadd_rn(a.hi, b.hi);
    const float z = __fsub_rn(t, a.hi);
    const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(t, z)), __fsub_rn(b.hi, z));
    return {t, __fadd_rn(__fadd_rn(a.lo, b.lo), e)};
}

// For the warp's vertex with adjacency [beg, end): per source slot, the sum of sp over
// the neighbours c whose Fsel[c] & tgt holds that source bit; uint64 sums (sigma, with
// carry detection) or double-single sums (psi).  Lanes over arcs find the relevant
// neighbours of a 32-arc window and list them in shared memory; then the lanes, each on
// its source pairs, read two listed neighbours' rows per round with 16-byte loads (both
// neighbours' loads in flight together) and add the relevant entries.
// With EDGE (backward only) the warp's vertex v also hands every relevant arc (v, c) its
// share sum_b sigma_b(v) * psi_b(c) over the gathered source bits (sv holds sigma_b(v) of
// the lane's slots): a warp sum per neighbour, parked in shared memory, then added to
// edge[j] by the lane that listed the arc, which loaded the old value when it listed it (the
// load is in flight during the rounds, so no round waits on a read-modify-write).  The arc
// is owned by v's warp at this level, so no atomics are needed.
template <int W, bool PSI, bool EDGE = false, bool S32 = false>
__device__ __forceinline__ void gather(const BArgs &a, int beg, int end,
                                       const unsigned long long *Fsel, const Bits<W> &tgt,
                                       unsigned long long (&acc)[2 * W], dev::ff (&facc)[2 * W],
                                       bool &ovf, Nbrs<W> &st, const dev::ff *sv = nullptr)
{
    constexpr int B = 64 * W;
    const int lane = threadIdx.x & 31;
    unsigned carry = 0;
    if (beg < 0 || end < beg || (long long)end > a.A) {  // warp-uniform
        if (lane == 0) check_failed(a, kErrCheck, 1, beg);
        return;
    }
    for (int base = beg; base < end; base += 32) {
        const int j = base + lane;
        int c = 0;
        Bits<W> f;
#pragma unroll
        for (int q = 0; q < W; ++q) f.w[q] = 0;
        if (j < end) {
            c = __ldg(a.col + j);
            const Bits<W> fc = load_bits<W>(Fsel + (size_t)c * W);
#pragma unroll
            for (int q = 0; q < W; ++q) f.w[q] = fc.w[q] & tgt.w[q];
        }
        const bool mine = any_bits<W>(f);
        const unsigned rel = __ballot_sync(FULL, mine);
        if (!rel) continue;
        const int pos = __popc(rel & dev::lanemask_lt());
        double eold = 0.0;
        if (mine) {
            st.c[pos] = c;
            st.j[pos] = j;
#pragma unroll
            for (int q = 0; q < W; ++q) st.f[pos][q] = f.w[q];
            if constexpr (EDGE) eold = __ldcg(a.edge + j);
        }
        __syncwarp();
        // NB relevant neighbours per round (two for the edge variant): every load of the
        // round is issued before any addition, so their latencies overlap
        constexpr int NB = 2;
        unsigned left = rel;
        while (left) {
            int idx[NB];
            bool on[NB];
#pragma unroll
            for (int r = 0; r < NB; ++r) {
                on[r] = left != 0;
                const int sr = on[r] ? __ffs(left) - 1 : 0;
                if (on[r]) left &= left - 1;
                idx[r] = on[r] ? __popc(rel & ((1u << sr) - 1u)) : 0;
            }
            // the lane's 2W bits of each listed neighbour, then one contiguous stretch of its row
            // per neighbour: 2W entries of 4 bytes (32-bit sigma) or 8 bytes, in 16-byte loads,
            // each issued only if one of its entries is relevant
            constexpr int G = 2 * W;
            unsigned nib[NB];
            unsigned long long x[NB][G];
#pragma unroll
            for (int r = 0; r < NB; ++r) {
                nib[r] = on[r] ? lane_bits<W>(st.f[idx[r]], lane) : 0u;
                if constexpr (S32) {
                    const unsigned *row = a.sp32 + (size_t)st.c[idx[r]] * B + G * lane;
                    if constexpr (G == 2) {
                        unsigned long long p = 0ull;
                        if (nib[r]) p = __ldcg(reinterpret_cast<const unsigned long long *>(row));
                        x[r][0] = p & 0xffffffffull;
                        x[r][1] = p >> 32;
                    } else {
#pragma unroll
                        for (int h = 0; h < G / 4; ++h) {
                            uint4 p = make_uint4(0u, 0u, 0u, 0u);
                            if ((nib[r] >> (4 * h)) & 15u) p = __ldcg(reinterpret_cast<const uint4 *>(row) + h);
                            x[r][4 * h] = p.x;
                            x[r][4 * h + 1] = p.y;
                            x[r][4 * h + 2] = p.z;
                            x[r][4 * h + 3] = p.w;
                        }
                    }
                } else {
                    const unsigned long long *row = a.sp + (size_t)st.c[idx[r]] * B + G * lane;
#pragma unroll
                    for (int h = 0; h < G / 2; ++h) {
                        ulonglong2 p = make_ulonglong2(0ull, 0ull);
                        if ((nib[r] >> (2 * h)) & 3u) p = __ldcg(reinterpret_cast<const ulonglong2 *>(row) + h);
                        x[r][2 * h] = p.x;
                        x[r][2 * h + 1] = p.y;
                    }
                }
            }
#pragma unroll
            for (int r = 0; r < NB; ++r)
#pragma unroll
                for (int k = 0; k < G; ++k)
                    if (!((nib[r] >> k) & 1u)) x[r][k] = 0ull;
#pragma unroll
            for (int k = 0; k < 2 * W; ++k) {
#pragma unroll
                for (int r = 0; r < NB; ++r) {
                    if constexpr (PSI) {
                        facc[k] = dev::ff_add(facc[k], dev::ff_unpack(x[r][k]));
                    } else {
                        add_carry(acc[k], carry, x[r][k]);
                    }
                }
            }
            if constexpr (EDGE) {
                const dev::ff e0 = edge_dot<G>(sv, x[0]), e1 = edge_dot<G>(sv, x[NB - 1]);
                // both sums at once: one exchange leaves neighbour 0's partials in the low
                // half-warp and neighbour 1's in the high half, then each half reduces alone
                const bool lo = lane < 16;
                dev::ff mine = lo ? e0 : e1, other = lo ? e1 : e0;
                dev::ff recv;
                recv.hi = __shfl_xor_sync(FULL, other.hi, 16);
                recv.lo = __shfl_xor_sync(FULL, other.lo, 16);
                mine = edge_sum2(mine, recv);
#pragma unroll
                for (int o = 8; o > 0; o >>= 1) {
                    dev::ff y;
                    y.hi = __shfl_xor_sync(FULL, mine.hi, o);
                    y.lo = __shfl_xor_sync(FULL, mine.lo, o);
                    mine = edge_sum2(mine, y);
                }
                if (lane == 0) st.e[idx[0]] = dev::ff_to_double(mine);
                if (on[NB - 1] && lane == 16) st.e[idx[NB - 1]] = dev::ff_to_double(mine);
            }
        }
        __syncwarp();
        if constexpr (EDGE) {
            if (mine) a.edge[j] = eold + st.e[pos];
        }
    }
    if (!PSI) ovf |= carry != 0;
}

template <int W> __device__ __forceinline__ Bits<W> nonzero_bits(const unsigned long long (&acc)[2 * W])
{
    // the lane's 2W-bit field, shifted into its place in its word, OR-reduced over the 32/W
    // lanes that share the word, then every word broadcast from its first lane
    constexpr int G = 2 * W, LPW = 32 / W;  // slots per lane, lanes per word
    const int lane = threadIdx.x & 31;
    unsigned f = 0u;
#pragma unroll
    for (int k = 0; k < G; ++k) f |= (acc[k] != 0ull ? 1u : 0u) << k;
    unsigned long long v = (unsigned long long)f << ((G * lane) & 63);
#pragma unroll
    for (int o = 1; o < LPW; o <<= 1) v |= __shfl_xor_sync(FULL, v, o);
    Bits<W> r;
#pragma unroll
    for (int q = 0; q < W; ++q) r.w[q] = __shfl_sync(FULL, v, q * LPW);
    return r;
}

struct BlockCnt {
    int v;
    unsigned long long mf, dmu;
};

// Vertex w joined level d+1 for the sources in nb (vold = its visited set before):
// writes its sigma row and visited set (and F_{d+1} when Fn is given), and counts it.
// Called by the whole warp with warp-uniform arguments.
template <int W, bool S32 = false>
__device__ __forceinline__ void settle(const BArgs &a, int w, const Bits<W> &vold, const Bits<W> &nb,
                                       const Bits<W> &act, const unsigned long long (&acc)[2 * W],
                                       unsigned long long *Fn, BlockCnt *bc)
{
    constexpr int B = 64 * W;
    const int lane = threadIdx.x & 31;
    if constexpr (S32) {
        // a count that does not fit 32 bits sends the batch back to the 64-bit kernel
        unsigned *row = a.sp32 + (size_t)w * B;
        bool wide = false;
#pragma unroll
        for (int k = 0; k < 2 * W; ++k)
            if (has_slot<W>(nb, k, lane)) {
                row[slot_off<W>(k, lane)] = (unsigned)acc[k];
                wide |= (acc[k] >> 32) != 0;
            }
        if (wide) atomicCAS(&a.ctrl->err, 0, kErrWide);
    } else {
        unsigned long long *row = a.sp + (size_t)w * B;
#pragma unroll
        for (int k = 0; k < 2 * W; ++k)
            if (has_slot<W>(nb, k, lane)) row[slot_off<W>(k, lane)] = acc[k];
    }
    bool full = true;
#pragma unroll
    for (int q = 0; q < W; ++q) {
        const unsigned long long nv = vold.w[q] | nb.w[q];
        full &= nv == act.w[q];
        if (lane == q) {
            a.vis[(size_t)w * W + q] = nv;
            if (Fn) Fn[(size_t)w * W + q] = nb.w[q];
        }
    }
    if (lane == 0) {
        const unsigned long long dg = (unsigned long long)deg_of(a.rp, w);
        atomicAdd(&bc->v, 1);
        atomicAdd(&bc->mf, dg);
        if (full) atomicAdd(&bc->dmu, dg);
    }
}

// Calls fn(v) with the whole warp for every vertex of a level: the queued entries
// queue[qo, qo+nq) or, if qo < 0, every v with Fl[v] != 0 (scanned 32 at a time; nq is
// then the level's vertex count).
// Calls fn(v) with the whole warp for every vertex of a level: the queued entries
// queue[qo, qo+nq) or, if qo < 0, every v with Fl[v] != 0 (scanned 32 at a time; nq is
// then the level's vertex count).  Warps
// take work dynamically from the zeroed counter *ctr (8 entries or 64 vertices at a
// time), so that power-law degrees do not leave a few warps finishing long after the
// rest.
template <int W, class Fn>
__device__ __forceinline__ void for_level(const BArgs &a, int qo, int nq,
                                          const unsigned long long *Fl, int32_t *ctr, Fn fn)
{
    const int lane = threadIdx.x & 31;
    // every loop below is also bounded in time: lane 0 checks the phase deadline once per
    // grab or tile and the warp leaves together (the status is read at the next barrier)
    const uint64_t deadline = dev::globaltimer() + a.limit_ns;
    auto expired = [&]() {
        int e = 0;
        if (lane == 0 && dev::globaltimer() > deadline) {
            check_failed(a, NK_ERR_TIMEOUT, 2, nq);
            e = 1;
        }
        return __shfl_sync(FULL, e, 0) != 0;
    };
    if (qo >= 0) {
        // up to kGrabQ entries per grab, fewer when the level is short (level 0, deep
        // levels), so that its entries spread over many warps
        const long long nwq = ((long long)gridDim.x * blockDim.x) >> 5;
        const int gq = (int)max(1LL, min((long long)kGrabQ, (long long)nq / nwq));
        for (;;) {
            int i0 = 0;
            if (lane == 0) i0 = atomicAdd(ctr, gq);
            i0 = __shfl_sync(FULL, i0, 0);
            if (i0 >= nq || expired()) break;
            const int i1 = min(i0 + gq, nq);
            for (int i = i0; i < i1; ++i) {
                const int v = __ldcg(a.queue + qo + i);
                if ((unsigned)v >= (unsigned)a.n) {  // warp-uniform
                    if (lane == 0) check_failed(a, kErrCheck, 3, v);
                    continue;
                }
                fn(v);
            }
        }
    } else if ((long long)nq * 32 < a.n) {
        // a sparse level (fewer than n/32 vertices): a static scan, no counter traffic
        const long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
        const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
        for (long long base = wid * 32; base < a.n; base += nw * 32) {
            if (expired()) break;
            const long long v = base + lane;
            const bool nz = v < a.n && any_bits<W>(load_bits<W>(Fl + (size_t)v * W));
            unsigned m = __ballot_sync(FULL, nz);
            while (m) {
                const int t = __ffs(m) - 1;
                m &= m - 1;
                fn((int)(base + t));
            }
        }
    } else {
        for (;;) {
            int t0 = 0;
            if (lane == 0) t0 = atomicAdd(ctr, kGrabV);
            t0 = __shfl_sync(FULL, t0, 0);
            if (t0 >= a.n || expired()) break;
            for (int base = t0; base < min(t0 + kGrabV, a.n); base += 32) {
                const int v = base + lane;
                const bool nz = v < a.n && any_bits<W>(load_bits<W>(Fl + (size_t)v * W));
                unsigned m = __ballot_sync(FULL, nz);
                while (m) {
                    const int t = __ffs(m) - 1;
                    m &= m - 1;
                    fn(base + t);
                }
            }
        }
    }
}

// Phase trace (diagnostics): CTA 0 records (code, %globaltimer) after a grid barrier.
// code = level * 16 + phase.
enum { PH_INIT = 1, PH_BU_A, PH_BU_B, PH_TD_A, PH_TD_B, PH_TD_C, PH_BK_A, PH_BK_B };

__device__ __forceinline__ void trace_mark(const BArgs &a, int &ti, int level, int phase)
{
    if (a.trace && blockIdx.x == 0 && threadIdx.x == 0 && ti < kTraceCap) {
        a.trace[2 * ti] = (unsigned long long)(level * 16 + phase);
        a.trace[2 * ti + 1] = dev::globaltimer();
        ++ti;
    }
}

// Work on the chunks of heavy vertices: fn(c, h, j0, j1) per chunk, with the whole warp;
// chunks are taken dynamically from the zeroed counter *ctr, and the loop is bounded in
// time like the others.
template <class Fn> __device__ __forceinline__ void for_chunks(const BArgs &a, int32_t *ctr, Fn fn)
{
    const int lane = threadIdx.x & 31;
    const uint64_t deadline = dev::globaltimer() + a.limit_ns;
    // grab about C / (32 warps) chunks, 1..16: few chunks stay spread over many warps,
    // millions of chunks cost few atomics
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    const int gc = (int)max(1LL, min((long long)kGrabCMax, (long long)a.C / (32 * nw)));
    for (;;) {
        int c0 = 0;
        if (lane == 0) {
            c0 = atomicAdd(ctr, gc);
            if (c0 < a.C && dev::globaltimer() > deadline) {
                check_failed(a, NK_ERR_TIMEOUT, 4, c0);
                c0 = a.C;
            }
        }
        c0 = __shfl_sync(FULL, c0, 0);
        if (c0 >= a.C) break;
        for (int c = c0; c < min(c0 + gc, a.C); ++c) {
            const int i = __ldg(a.chunk_h + c);
            const int h = __ldg(a.hv + i);
            const int j0 = __ldg(a.rp + h) + (c - __ldg(a.hfirst + i)) * a.chunk;
            const int j1 = min(j0 + a.chunk, __ldg(a.rp + h + 1));
            fn(c, h, j0, j1);
        }
    }
}

// fn(i, h, c0, c1) per heavy vertex (chunks [c0, c1)), with the whole warp.
template <class Fn> __device__ __forceinline__ void for_heavy(const BArgs &a, Fn fn)
{
    const long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long i = wid; i < a.H; i += nw)
        fn((int)i, __ldg(a.hv + i), __ldg(a.hfirst + i), __ldg(a.hfirst + i + 1));
}

template <int W>
__device__ __forceinline__ void store_part(const BArgs &a, int c, const unsigned long long (&acc)[2 * W])
{
    unsigned long long *row = a.part + (size_t)c * (64 * W);
#pragma unroll
    for (int k = 0; k < 2 * W; ++k) row[slot_off<W>(k, threadIdx.x & 31)] = acc[k];
}

__device__ __forceinline__ bool heavy(const BArgs &a, int v) { return deg_of(a.rp, v) > a.chunk; }

// CTAs per SM that the launch bounds ask for: 4 for 64 and 128 sources (64 registers), 3 for
// the 128-source edge sweep (its per-arc shares need 80 registers, which 64 would spill), 2
// for 256 sources
template <int W, bool EDGE> constexpr int min_ctas() { return W >= 4 ? 2 : (EDGE && W == 2) ? 3 : 4; }

template <int W, bool EDGE, bool S32>
__global__ void __launch_bounds__(kThreads, min_ctas<W, EDGE>()) k_batch(BArgs a)
{
    constexpr int B = 64 * W;
    __shared__ BlockCnt bc;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Nbrs<W> &st = reinterpret_cast<Nbrs<W> *>(smem_raw)[threadIdx.x >> 5];
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nthr = (long long)gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    const size_t slab = (size_t)a.n * W;
    const int nsrc = a.ksrc ? max(0, min(B, __ldg(a.ksrc) - a.boff)) : a.nsrc;
    if (nsrc == 0) return;  // uniform over the grid: no barrier is entered
    Bits<W> act;
#pragma unroll
    for (int q = 0; q < W; ++q) {
        const int left = nsrc - 64 * q;
        act.w[q] = left >= 64 ? ~0ull : (left <= 0 ? 0ull : ((1ull << left) - 1));
    }
    bool ovf = false;
    int ti = 0;
    trace_mark(a, ti, 0, 0);
    auto flush_counts = [&](int lvl) {
        __syncthreads();
        if (threadIdx.x == 0) {
            if (bc.v) atomicAdd(a.vcnt + lvl, bc.v);
            if (bc.mf) atomicAdd(a.mfv + lvl, bc.mf);
            if (bc.dmu) atomicAdd(a.dmu + lvl, bc.dmu);
        }
    };

    // ---- init: empty visited sets, F_0 and F_1, queue marks, level-0..2 counters
    for (size_t i = tid; i < slab; i += nthr) {
        a.vis[i] = 0;
        a.F[i] = 0;
        a.F[slab + i] = 0;
    }
    for (long long i = tid; i < a.n; i += nthr) a.qmark[i] = -1;
    if (tid < 3 * 8) a.wq[tid] = 0;
    if (tid < 3) {
        a.vcnt[tid] = 0;
        a.qcnt[tid] = 0;
        a.qoff[tid] = -1;
        a.mfv[tid] = 0;
        a.dmu[tid] = 0;
    }
    if (!dev::grid_barrier(a.ctrl, a.limit_ns)) return;
    trace_mark(a, ti, 0, PH_INIT);
    if (tid < nsrc) {
        const int s = __ldg(a.src + tid);
        const unsigned long long bit = 1ull << (tid & 63);
        atomicOr(a.F + (size_t)s * W + (tid >> 6), bit);
        atomicOr(a.vis + (size_t)s * W + (tid >> 6), bit);
        if constexpr (S32) a.sp32[(size_t)s * B + tid] = 1u;
        else a.sp[(size_t)s * B + tid] = 1ull;
        a.queue[tid] = s;
        atomicAdd(a.mfv, (unsigned long long)deg_of(a.rp, s));
        if (nsrc == 1) a.dmu[0] = (unsigned long long)deg_of(a.rp, s);
    }
    if (tid == 0) {
        a.vcnt[0] = nsrc;
        a.qcnt[0] = nsrc;
        a.qoff[0] = 0;
    }
    if (!dev::grid_barrier(a.ctrl, a.limit_ns)) return;

    long long mu = a.A - (long long)__ldcg(a.dmu);
    long long mf = (long long)__ldcg(a.mfv);
    int d = 0, qo = 0, nq = nsrc, td = 0, bu = 0;
    long long qtail = nsrc;
    for (;;) {
        if (threadIdx.x == 0) {
            bc.v = 0;
            bc.mf = 0;
            bc.dmu = 0;
        }
        if (tid == 0) {
            a.vcnt[d + 2] = 0;
            a.qcnt[d + 2] = 0;
            a.mfv[d + 2] = 0;
            a.dmu[d + 2] = 0;
        }
        if (tid < 8) a.wq[(size_t)(d + 2) * 8 + tid] = 0;
        {
            unsigned long long *Fz = a.F + (size_t)(d + 2) * slab;
            for (size_t i = tid; i < slab; i += nthr) Fz[i] = 0;
        }
        __syncthreads();
        const unsigned long long *Fd = a.F + (size_t)d * slab;
        unsigned long long *Fn = a.F + (size_t)(d + 1) * slab;
        const bool use_bu = a.dir == NK_DIR_BOTTOM_UP ||
                            (a.dir == NK_DIR_AUTO && a.alpha * (double)mf > (double)mu);
        bool queued = false;
        int nq1 = 0;
        if (use_bu) {
            // ---- bottom-up (a): light vertices with unvisited sources pull from level d;
            //      chunks of heavy vertices store partial sums
            const uint64_t bu_deadline = dev::globaltimer() + a.limit_ns;
            for (int t0 = 0;;) {
                if (lane == 0) {
                    t0 = atomicAdd(a.wq + (size_t)d * 8 + WQ_BU, 32);
                    if (t0 < a.n && dev::globaltimer() > bu_deadline) {
                        check_failed(a, NK_ERR_TIMEOUT, 5, t0);
                        t0 = a.n;
                    }
                }
                t0 = __shfl_sync(FULL, t0, 0);
                if (t0 >= a.n) break;
                const long long base = t0;
                const long long v = base + lane;
                Bits<W> vv = act;
                if (v < a.n && !heavy(a, (int)v)) vv = load_bits<W>(a.vis + (size_t)v * W);
                unsigned m = __ballot_sync(FULL, any_bits<W>(andnot<W>(act, vv)));
                while (m) {
                    const int t = __ffs(m) - 1;
                    m &= m - 1;
                    const int w = (int)(base + t);
                    const Bits<W> vold = shfl_bits<W>(vv, t);
                    const Bits<W> u = andnot<W>(act, vold);
                    unsigned long long acc[2 * W];
                    dev::ff facc[2 * W];
#pragma unroll
                    for (int k = 0; k < 2 * W; ++k) acc[k] = 0;
                    gather<W, false, false, S32>(a, __ldg(a.rp + w), __ldg(a.rp + w + 1), Fd, u, acc, facc, ovf, st);
                    const Bits<W> nb = nonzero_bits<W>(acc);
                    if (any_bits<W>(nb)) settle<W, S32>(a, w, vold, nb, act, acc, Fn, &bc);
                }
            }
            for_chunks(a, a.wq + (size_t)d * 8 + WQ_BU_C, [&](int c, int h, int j0, int j1) {
                const Bits<W> u = andnot<W>(act, load_bits<W>(a.vis + (size_t)h * W));
                if (!any_bits<W>(u)) return;
                unsigned long long acc[2 * W];
                dev::ff facc[2 * W];
#pragma unroll
                for (int k = 0; k < 2 * W; ++k) acc[k] = 0;
                gather<W, false, false, S32>(a, j0, j1, Fd, u, acc, facc, ovf, st);
                store_part<W>(a, c, acc);
            });
            if (a.H > 0 && !dev::grid_barrier(a.ctrl, a.limit_ns)) return;
            trace_mark(a, ti, d, PH_BU_A);
            // ---- bottom-up (b): heavy vertices sum their chunks in chunk order
            for_heavy(a, [&](int i, int h, int c0, int c1) {
                const Bits<W> vold = load_bits<W>(a.vis + (size_t)h * W);
                if (!any_bits<W>(andnot<W>(act, vold))) return;
                unsigned long long acc[2 * W];
#pragma unroll
                for (int k = 0; k < 2 * W; ++k) acc[k] = 0;
                for (int c = c0; c < c1; ++c) {
                    const unsigned long long *row = a.part + (size_t)c * B;
#pragma unroll
                    for (int k = 0; k < 2 * W; ++k) {
                        const unsigned long long y = acc[k] + __ldcg(row + slot_off<W>(k, lane));
                        ovf |= y < acc[k];
                        acc[k] = y;
                    }
                }
                const Bits<W> nb = nonzero_bits<W>(acc);
                if (any_bits<W>(nb)) settle<W, S32>(a, h, vold, nb, act, acc, Fn, &bc);
            });
            flush_counts(d + 1);
            if (tid == 0) a.qoff[d + 1] = -1;
            if (!dev::grid_barrier(a.ctrl, a.limit_ns)) return;
            trace_mark(a, ti, d, PH_BU_B);
        } else {
            // ---- top-down (a): push the frontier's bits, queue each new vertex once;
            //      heavy frontier vertices push chunk by chunk
            auto push = [&](int v, int j0, int j1) {
                const Bits<W> f = load_bits<W>(Fd + (size_t)v * W);
                for (int j = j0 + lane; j < j1; j += 32) {
                    const int c = __ldg(a.col + j);
                    const Bits<W> m = andnot<W>(f, load_bits<W>(a.vis + (size_t)c * W));
                    if (!any_bits<W>(m)) continue;
#pragma unroll
                    for (int q = 0; q < W; ++q)
                        if (m.w[q]) atomicOr(Fn + (size_t)c * W + q, m.w[q]);
                    if (__ldcg(a.qmark + c) != d + 1 && atomicExch(a.qmark + c, d + 1) != d + 1) {
                        cg::coalesced_group g = cg::coalesced_threads();
                        int pos = 0;
                        if (g.thread_rank() == 0) pos = atomicAdd(a.qcnt + d + 1, (int)g.size());
                        pos = g.shfl(pos, 0) + (int)g.thread_rank();
                        if (qtail + pos < a.qcap) a.queue[qtail + pos] = c;
                    }
                }
            };
            for_level<W>(a, qo, nq, Fd, a.wq + (size_t)d * 8 + WQ_PUSH, [&](int v) {
                if (heavy(a, v)) return;
                push(v, __ldg(a.rp + v), __ldg(a.rp + v + 1));
            });
            for_chunks(a, a.wq + (size_t)d * 8 + WQ_PUSH_C, [&](int c, int h, int j0, int j1) {
                if (any_bits<W>(load_bits<W>(Fd + (size_t)h * W))) push(h, j0, j1);
            });
            if (!dev::grid_barrier(a.ctrl, a.limit_ns)) return;
            trace_mark(a, ti, d, PH_TD_A);
            // ---- top-down (b): every new vertex pulls sigma for its new bits
            nq1 = __ldcg(a.qcnt + d + 1);
            queued = qtail + nq1 <= a.qcap;
            for_level<W>(a, queued ? (int)qtail : -1, nq1, Fn, a.wq + (size_t)d * 8 + WQ_PULL, [&](int w) {
                if (heavy(a, w)) return;
                const Bits<W> t = load_bits<W>(Fn + (size_t)w * W);
                const Bits<W> vold = load_bits<W>(a.vis + (size_t)w * W);
                unsigned long long acc[2 * W];
                dev::ff facc[2 * W];
#pragma unroll
                for (int k = 0; k < 2 * W; ++k) acc[k] = 0;
                gather<W, false, false, S32>(a, __ldg(a.rp + w), __ldg(a.rp + w + 1), Fd, t, acc, facc, ovf, st);
                settle<W, S32>(a, w, vold, t, act, acc, nullptr, &bc);
            });
            for_chunks(a, a.wq + (size_t)d * 8 + WQ_PULL_C, [&](int c, int h, int j0, int j1) {
                const Bits<W> t = load_bits<W>(Fn + (size_t)h * W);
                if (!any_bits<W>(t)) return;
                unsigned long long acc[2 * W];
                dev::ff facc[2 * W];
#pragma unroll
                for (int k = 0; k < 2 * W; ++k) acc[k] = 0;
                gather<W, false, false, S32>(a, j0, j1, Fd, t, acc, facc, ovf, st);
                store_part<W>(a, c, acc);
            });
            if (a.H > 0 && !dev::grid_barrier(a.ctrl, a.limit_ns)) return;
            trace_mark(a, ti, d, PH_TD_B);
            // ---- top-down (c): heavy new vertices sum their chunks in chunk order
            for_heavy(a, [&](int i, int h, int c0, int c1) {
                const Bits<W> t = load_bits<W>(Fn + (size_t)h * W);
                if (!any_bits<W>(t)) return;
                const Bits<W> vold = load_bits<W>(a.vis + (size_t)h * W);
                unsigned long long acc[2 * W];
#pragma unroll
                for (int k = 0; k < 2 * W; ++k) acc[k] = 0;
                for (int c = c0; c < c1; ++c) {
                    const unsigned long long *row = a.part + (size_t)c * B;
#pragma unroll
                    for (int k = 0; k < 2 * W; ++k) {
                        const unsigned long long y = acc[k] + __ldcg(row + slot_off<W>(k, lane));
                        ovf |= y < acc[k];
                        acc[k] = y;
                    }
                }
                settle<W, S32>(a, h, vold, t, act, acc, nullptr, &bc);
            });
            flush_counts(d + 1);
            if (tid == 0) a.qoff[d + 1] = queued ? (int)qtail : -1;
            if (!dev::grid_barrier(a.ctrl, a.limit_ns)) return;
            trace_mark(a, ti, d, PH_TD_C);
        }
        const int c = __ldcg(a.vcnt + d + 1);
        if (use_bu) {
            ++bu;
            qo = -1;
            nq = c;
        } else {
            ++td;
            qo = queued ? (int)qtail : -1;
            nq = queued ? nq1 : c;
            if (queued) qtail += nq1;
        }
        mu -= (long long)__ldcg(a.dmu + d + 1);
        mf = (long long)__ldcg(a.mfv + d + 1);
        ++d;
        if (c == 0) break;
        if (d + 1 > a.lcap) {
            if (tid == 0) atomicCAS(&a.ctrl->err, 0, kErrDepth);
            return;
        }
    }
    const int D = d - 1;
    if (tid == 0) {
        a.ctrl->depth = D;
        a.ctrl->td_levels = td;
        a.ctrl->bu_levels = bu;
    }
    if (ovf) atomicOr(&a.ctrl->ovf, 1);
    if (a.rk_t) {
        // error-bounded estimate: one warp per source slot b walks one shortest path back
        // from its target, choosing each predecessor z of w with probability
        // sigma_b(z) / sigma_b(w): t = below(stream(key, step), sigma_b(w)) falls in the
        // run of z when the predecessors' sigma values are laid end to end in adjacency
        // order.  Every vertex strictly between the source and the target is counted.
        // The slabs and sigma rows are complete: the last level ended with a grid barrier.
        const long long wid = tid >> 5, nw = nthr >> 5;
        for (long long b = wid; b < nsrc; b += nw) {
            const int v = __ldg(a.rk_t + b);
            const int q = (int)(b >> 6);
            const unsigned long long bit = 1ull << (b & 63);
            int L = -1;
            for (int l0 = 1; l0 <= D && L < 0; l0 += 32) {
                const int l = l0 + lane;
                const bool hit = l <= D && (__ldcg(a.F + (size_t)l * slab + (size_t)v * W + q) & bit) != 0;
                const unsigned m = __ballot_sync(FULL, hit);
                if (m) L = l0 + __ffs(m) - 1;
            }
            if (L < 0) continue;  // the target is not reachable from the source
            const unsigned long long key = __ldg(a.rk_key + b);
            int w = v;
            for (int l = L, step = 0; l > 1; --l, ++step) {
                const unsigned long long sw = S32 ? (unsigned long long)__ldcg(a.sp32 + (size_t)w * B + b)
                                                  : __ldcg(a.sp + (size_t)w * B + b);
                const unsigned long long t = dev::below(dev::stream_at(key, (uint64_t)step), sw);
                const unsigned long long *Fp = a.F + (size_t)(l - 1) * slab;
                const int end = __ldg(a.rp + w + 1);
                unsigned long long run = 0;
                int z = -1;
                for (int base = __ldg(a.rp + w); base < end && z < 0; base += 32) {
                    const int j = base + lane;
                    int c = -1;
                    unsigned long long x = 0;
                    if (j < end) {
                        c = __ldg(a.col + j);
                        if (__ldcg(Fp + (size_t)c * W + q) & bit)
                            x = S32 ? (unsigned long long)__ldcg(a.sp32 + (size_t)c * B + b) : __ldcg(a.sp + (size_t)c * B + b);
                    }
                    unsigned long long incl = x;  // inclusive prefix over the lanes
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const unsigned long long y = __shfl_up_sync(FULL, incl, o);
                        if (lane >= o) incl += y;
                    }
                    const unsigned m = __ballot_sync(FULL, x != 0 && run + incl > t);
                    if (m) z = __shfl_sync(FULL, c, __ffs(m) - 1);
                    else run += __shfl_sync(FULL, incl, 31);
                }
                if (z < 0) break;  // only with a wrapped path count (reported as an overflow)
                if (lane == 0) atomicAdd(a.rk_count + z, 1ull);
                w = z;
            }
        }
    }
    if (a.far) {
        // closeness: v is at distance l from the sources of F_l[v]; one thread per vertex
        // adds its level sums once the whole sweep has stayed within the slabs (a batch
        // that ran out of levels returned above and adds nothing).  A bottom-up level takes
        // its new bits from non-zero path sums, which a sum that wrapped past 2^64 could
        // hide: a batch with an overflow adds nothing either and the host reruns it.
        if (!dev::grid_barrier(a.ctrl, a.limit_ns)) return;
        if (dev::ld_volatile(&a.ctrl->ovf) != 0) return;
        for (long long v = tid; v < a.n; v += nthr) {
            unsigned long long fs = 0, rs = 0;
            for (int l = 1; l <= D; ++l) {
                const Bits<W> f = load_bits<W>(a.F + (size_t)l * slab + (size_t)v * W);
                unsigned long long cnt = 0;
#pragma unroll
                for (int q = 0; q < W; ++q) cnt += (unsigned long long)__popcll(f.w[q]);
                fs += cnt * (unsigned long long)l;
                rs += cnt;
            }
            if (rs) {
                a.far[v] += fs;
                a.reach[v] += rs;
            }
        }
    }
    if (!a.backward) return;

    // ---- backward sweep, deepest level first (edge betweenness also needs level 0: the
    //      arcs from the sources carry shares, although the sources get no score)
    for (int l = D; l >= (EDGE ? 0 : 1); --l) {
        const unsigned long long *Fl = a.F + (size_t)l * slab;
        const unsigned long long *Fs = a.F + (size_t)(l + 1) * slab;
        const int ql = __ldcg(a.qoff + l);
        const int nl = ql >= 0 ? __ldcg(a.qcnt + l) : __ldcg(a.vcnt + l);
        // delta/psi/score of vertex v from its successor sums facc (whole warp)
        // psi_v = 1/sigma_v + acc and delta_v = sigma_v * acc (Brandes' recurrence with
        // sigma_v factored out), in double-single; the vertex's delta summed over its
        // source slots goes to the FP64 score once per vertex and level
        auto finish = [&](int v, const Bits<W> &mv, const dev::ff (&facc)[2 * W]) {
            dev::ff part = dev::ff_zero();
            unsigned long long *row = a.sp + (size_t)v * B;
#pragma unroll
            for (int k = 0; k < 2 * W; ++k) {
                if (has_slot<W>(mv, k, lane)) {
                    const unsigned long long sg = S32 ? (unsigned long long)__ldcg(a.sp32 + (size_t)v * B + slot_off<W>(k, lane))
                                                      : __ldcg(row + slot_off<W>(k, lane));
                    const dev::ff sv = dev::ff_from_u64(sg);
                    const dev::ff delta = dev::ff_mul(sv, facc[k]);
                    row[slot_off<W>(k, lane)] = dev::ff_pack(dev::ff_add(dev::ff_rcp(sv), facc[k]));
                    part = dev::ff_add(part, delta);
                }
            }
            part = dev::group_sum_ff<32>(part);
            if (lane == 0 && part.hi != 0.0f && l > 0) a.scores[v] += dev::ff_to_double(part);
        };
        // sigma_b(v) of the lane's slots in mv (edge betweenness only), read before psi
        // replaces it
        auto sigma_row = [&](int v, const Bits<W> &mv, dev::ff (&sv)[2 * W]) {
            const unsigned long long *row = a.sp + (size_t)v * B;
#pragma unroll
            for (int k = 0; k < 2 * W; ++k)
                sv[k] = has_slot<W>(mv, k, lane) ? dev::ff_from_u64(__ldcg(row + slot_off<W>(k, lane))) : dev::ff_zero();
        };
        for_level<W>(a, ql, nl, Fl, a.wq + (size_t)l * 8 + WQ_BACK, [&](int v) {
            if (heavy(a, v)) return;
            const Bits<W> mv = load_bits<W>(Fl + (size_t)v * W);
            unsigned long long acc[2 * W];
            dev::ff facc[2 * W], sv[2 * W];
#pragma unroll
            for (int k = 0; k < 2 * W; ++k) facc[k] = dev::ff_zero();
            if constexpr (EDGE) sigma_row(v, mv, sv);
            bool dummy = false;
            gather<W, true, EDGE>(a, __ldg(a.rp + v), __ldg(a.rp + v + 1), Fs, mv, acc, facc, dummy, st, sv);
            finish(v, mv, facc);
        });
        for_chunks(a, a.wq + (size_t)l * 8 + WQ_BACK_C, [&](int c, int h, int j0, int j1) {
            const Bits<W> mv = load_bits<W>(Fl + (size_t)h * W);
            if (!any_bits<W>(mv)) return;
            unsigned long long acc[2 * W];
            dev::ff facc[2 * W], sv[2 * W];
#pragma unroll
            for (int k = 0; k < 2 * W; ++k) facc[k] = dev::ff_zero();
            if constexpr (EDGE) sigma_row(h, mv, sv);
            bool dummy = false;
            gather<W, true, EDGE>(a, j0, j1, Fs, mv, acc, facc, dummy, st, sv);
#pragma unroll
            for (int k = 0; k < 2 * W; ++k) acc[k] = dev::ff_pack(facc[k]);
            store_part<W>(a, c, acc);
        });
        if (a.H > 0 && !dev::grid_barrier(a.ctrl, a.limit_ns)) return;
        trace_mark(a, ti, l, PH_BK_A);
        for_heavy(a, [&](int i, int h, int c0, int c1) {
            const Bits<W> mv = load_bits<W>(Fl + (size_t)h * W);
            if (!any_bits<W>(mv)) return;
            dev::ff facc[2 * W];
#pragma unroll
            for (int k = 0; k < 2 * W; ++k) facc[k] = dev::ff_zero();
            for (int c = c0; c < c1; ++c) {
                const unsigned long long *row = a.part + (size_t)c * B;
#pragma unroll
                for (int k = 0; k < 2 * W; ++k) facc[k] = dev::ff_add(facc[k], dev::ff_unpack(__ldcg(row + slot_off<W>(k, lane))));
            }
            finish(h, mv, facc);
        });
        if (!dev::grid_barrier(a.ctrl, a.limit_ns)) return;
        trace_mark(a, ti, l, PH_BK_B);
    }
}

// ------------------------------------------------------------------ host side
// Dynamic shared memory of one CTA: a neighbour list per warp.
template <int W> constexpr size_t smem_bytes() { return (size_t)(kThreads / 32) * sizeof(Nbrs<W>); }

// Co-resident CTAs per SM of k_batch<W, EDGE> with its shared memory (the shared-memory
// attribute is set on the first call, outside any stream capture).
template <int W, bool EDGE = false, bool S32 = false> int blocks_per_sm()
{
    static int b = -1;
    if (b < 0) {
        NK_CUDA(cudaFuncSetAttribute(k_batch<W, EDGE, S32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes<W>()));
        int v = 0;
        NK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_batch<W, EDGE, S32>, kThreads, smem_bytes<W>()));
        b = v;
    }
    return b;
}

struct Layout {
    int W, B, lcap;
    int64_t qcap;
    size_t off_F, off_vis, off_sp, off_sp32, off_qmark, off_queue, off_cnt, off_part, total;
};

size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

// chunk count of the heavy table for `chunk` arcs per chunk (an upper bound before the
// table is built)
int64_t chunk_count(const nk_graph *g, int chunk)
{
    if (chunk <= 0) chunk = kChunk;
    if (chunk == kChunk && g->heavy_H >= 0) return g->heavy_C;
    if (chunk != kChunk && g->heavy_alt_H >= 0 && g->heavy_alt_chunk == chunk) return g->heavy_alt_C;
    return g->A / chunk + (g->max_deg > chunk ? g->n : 0);
}

Layout layout(const nk_graph *g, int B, int lcap, int chunk = 0)
{
    Layout L;
    L.B = B;
    L.W = B / 64;
    L.lcap = lcap;
    L.qcap = 2 * (int64_t)g->n + 64;
    const size_t n = (size_t)g->n;
    size_t o = 0;
    L.off_F = o;
    o = align_up(o + (size_t)(lcap + 2) * n * L.W * 8);
    L.off_vis = o;
    o = align_up(o + n * L.W * 8);
    L.off_sp = o;
    o = align_up(o + n * (size_t)B * 8);
    L.off_sp32 = o;
    o = align_up(o + n * (size_t)B * 4);
    L.off_qmark = o;
    o = align_up(o + n * 4);
    L.off_queue = o;
    o = align_up(o + (size_t)L.qcap * 4);
    L.off_cnt = o;
    o = align_up(o + (size_t)(lcap + 3) * (3 * 4 + 2 * 8 + 8 * 4));
    L.off_part = o;
    o = align_up(o + (size_t)chunk_count(g, chunk) * B * 8);
    L.total = o;
    return L;
}

int choose_lcap(const nk_graph *g, int B, const DevBuf *ws, int chunk = 0)
{
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    const size_t slab = (size_t)g->n * (B / 64) * 8;
    const Layout base = layout(g, B, 0, chunk);
    // level slabs may use up to half of what is free after the rest of the batch state
    const size_t have = free_b + ws[5].bytes;
    size_t budget = have > base.total ? (have - base.total) / 2 : 0;
    int64_t l = slab ? (int64_t)(budget / slab) - 2 : 1022;
    l = std::min<int64_t>(l, 1022);
    l = std::min<int64_t>(l, std::max<int64_t>(g->n, 4));  // a BFS has at most n levels; 4 at least
    return (int)std::max<int64_t>(l, 0);
}

enum { WS_BATCH = 5, WS_BCTRL = 6 };

template <int W>
int launch_batches(nk_graph *g, const int32_t *d_src, int32_t k, double *d_scores,
                   const RunCfg &cfg, RunStats *st, cudaStream_t s)
{
    constexpr int B = 64 * W;
    // sources without arcs add nothing: the batches take the others (the error-bounded
    // estimate keeps its slots, which are tied to their targets)
    Tmp csrc, ccnt;
    if (!cfg.rk_t) {
        NK_TRY(csrc.alloc(sizeof(int32_t) * (size_t)k, s));
        NK_TRY(ccnt.alloc(sizeof(int32_t), s));
        NK_TRY(compact_sources(g, d_src, k, csrc.as<int32_t>(), ccnt.as<int32_t>(), s));
        int32_t kk = 0;
        NK_CUDA(cudaMemcpyAsync(&kk, ccnt.p, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        NK_CUDA(cudaStreamSynchronize(s));
        if (kk < 0 || kk > k) return set_error(NK_ERR_CUDA, "source compaction returned %d of %d", kk, k);
        d_src = csrc.as<int32_t>();
        k = kk;
        if (k == 0) {
            if (st) {
                st->mode = NK_MODE_BATCHED;
                st->batch = B;
            }
            return NK_OK;
        }
    }
    HeavyView hw;
    NK_TRY(heavy_view(g, cfg.chunk, s, &hw));
    DevBuf *ws = scratch(cfg, g);
    // level slabs: start small; batches whose BFS is deeper are rerun once with the
    // largest cap that free memory allows, then (if still deeper) by the per-source form
    const int lmax = cfg.lcap > 0 ? std::min(cfg.lcap, std::max(g->n, 4)) : choose_lcap(g, B, ws, hw.chunk);
    if (lmax < 4) return set_error(NK_ERR_NOMEM, "not enough device memory for a batch of %d sources", B);
    const int lstart = cfg.lcap > 0 ? lmax : std::min(lmax, std::max(kStartLevels, 4));
    const int nb = (k + B - 1) / B;
    NK_TRY(ws[WS_BCTRL].ensure(sizeof(Ctrl) * nb));
    const bool edge = cfg.edge && cfg.backward;
    // sigma in 32-bit rows unless a batch's counts do not fit (then that batch is rerun with
    // 64-bit rows); the edge variant keeps 64-bit rows
    bool s32 = !edge;
    auto pick = [&](const void *&kfn, int &grid) -> int {
        const int bps = edge ? blocks_per_sm<W, true, false>() : s32 ? blocks_per_sm<W, false, true>()
                                                                     : blocks_per_sm<W, false, false>();
        if (bps < 1) return set_error(NK_ERR_CUDA, "batched kernel cannot be resident");
        kfn = edge ? (const void *)k_batch<W, true, false>
                   : s32 ? (const void *)k_batch<W, false, true> : (const void *)k_batch<W, false, false>;
        grid = std::max(1, bps * num_sms() / std::max(1, cfg.grid_div));
        if (cfg.grid_ctas > 0) grid = std::min(grid, cfg.grid_ctas);
        return NK_OK;
    };
    const void *kfn = nullptr;
    int grid = 0;
    NK_TRY(pick(kfn, grid));
    Ctrl *ctrls = ws[WS_BCTRL].as<Ctrl>();
    std::vector<int> todo(nb);
    for (int bi = 0; bi < nb; ++bi) todo[bi] = bi;
    double alpha_used = cfg.alpha > 0 ? cfg.alpha : 1.0;
    static const bool trace_on = std::getenv("NK_TRACE") != nullptr;
    Tmp trace_buf;
    if (trace_on) {
        NK_TRY(trace_buf.alloc(sizeof(unsigned long long) * 2 * kTraceCap, s));
        NK_CUDA(cudaMemsetAsync(trace_buf.p, 0, sizeof(unsigned long long) * 2 * kTraceCap, s));
    }
    for (int lcap = lstart;;) {
        const Layout L = layout(g, B, lcap, hw.chunk);
        NK_TRY(ws[WS_BATCH].ensure(L.total));
        char *base = ws[WS_BATCH].as<char>();
        BArgs a{};
        a.n = g->n;
        a.A = g->A;
        a.rp = g->rp.as<int32_t>();
        a.col = g->col.as<int32_t>();
        a.lcap = lcap;
        a.F = reinterpret_cast<unsigned long long *>(base + L.off_F);
        a.vis = reinterpret_cast<unsigned long long *>(base + L.off_vis);
        a.sp = reinterpret_cast<unsigned long long *>(base + L.off_sp);
        a.sp32 = reinterpret_cast<unsigned *>(base + L.off_sp32);
        a.qmark = reinterpret_cast<int32_t *>(base + L.off_qmark);
        a.queue = reinterpret_cast<int32_t *>(base + L.off_queue);
        a.qcap = L.qcap;
        const size_t lv = (size_t)lcap + 3;
        char *cb = base + L.off_cnt;
        a.mfv = reinterpret_cast<unsigned long long *>(cb);
        a.dmu = a.mfv + lv;
        a.vcnt = reinterpret_cast<int32_t *>(a.dmu + lv);
        a.qcnt = a.vcnt + lv;
        a.qoff = a.qcnt + lv;
        a.wq = a.qoff + lv;
        a.scores = d_scores;
        a.hv = hw.hv;
        a.hfirst = hw.hfirst;
        a.chunk_h = hw.chunk_h;
        a.H = hw.H;
        a.C = hw.C;
        a.chunk = hw.chunk;
        a.part = reinterpret_cast<unsigned long long *>(base + L.off_part);
        a.trace = nullptr;
        a.far = cfg.far;
        a.reach = cfg.reach;
        a.backward = cfg.backward ? 1 : 0;
        a.edge = edge ? cfg.edge : nullptr;
        a.rk_count = cfg.rk_count;
        a.limit_ns = cfg.limit_ns ? cfg.limit_ns : wait_limit_ns();
        a.alpha = alpha_used;
        a.dir = cfg.direction;
        NK_CUDA(cudaMemsetAsync(ctrls, 0, sizeof(Ctrl) * nb, s));
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (cfg.time_kernels) {
            NK_CUDA(cudaEventCreate(&e0));
            NK_CUDA(cudaEventCreate(&e1));
            NK_CUDA(cudaEventRecord(e0, s));
        }
        a.ksrc = nullptr;
        a.boff = 0;
        for (int bi : todo) {
            a.src = d_src + (size_t)bi * B;
            a.nsrc = std::min(B, k - bi * B);
            a.ctrl = ctrls + bi;
            a.rk_t = cfg.rk_t ? cfg.rk_t + (size_t)bi * B : nullptr;
            a.rk_key = cfg.rk_key ? cfg.rk_key + (size_t)bi * B : nullptr;
            a.trace = (trace_on && bi == todo.front()) ? trace_buf.as<unsigned long long>() : nullptr;
            void *args[] = {&a};
            NK_CUDA(cudaLaunchCooperativeKernel(kfn, dim3(grid), dim3(kThreads), args, smem_bytes<W>(), s));
            ::nk::count_launch();
        }
        if (cfg.time_kernels) NK_CUDA(cudaEventRecord(e1, s));
        std::vector<Ctrl> h(nb);
        NK_CUDA(cudaMemcpyAsync(h.data(), ctrls, sizeof(Ctrl) * nb, cudaMemcpyDeviceToHost, s));
        NK_TRY(host_wait(s, (int64_t)todo.size(), a.limit_ns));
        if (st) {
            st->mode = NK_MODE_BATCHED;
            st->batch = B;
            st->tpv = 32;
            st->launches += (int64_t)todo.size();
            st->alpha = alpha_used;
            for (int bi : todo) {
                st->max_depth = std::max(st->max_depth, h[bi].depth);
                st->td_levels += h[bi].td_levels;
                st->bu_levels += h[bi].bu_levels;
            }
            if (cfg.time_kernels) {
                float ms = 0;
                cudaEventElapsedTime(&ms, e0, e1);
                st->kernel_ms += ms;
            }
        }
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (trace_on) {
            static const char *names[] = {"start", "init", "bu-pull", "bu-hubs", "td-push", "td-pull", "td-hubs", "back", "back-hubs"};
            std::vector<unsigned long long> t(2 * kTraceCap);
            NK_CUDA(cudaMemcpyAsync(t.data(), trace_buf.p, sizeof(unsigned long long) * t.size(), cudaMemcpyDeviceToHost, s));
            NK_CUDA(cudaStreamSynchronize(s));
            for (int i = 1; i < kTraceCap && t[2 * i + 1]; ++i)
                fprintf(stderr, "nk-trace B=%d level=%llu phase=%s us=%.1f\n", B, t[2 * i] / 16,
                        names[std::min<unsigned long long>(t[2 * i] % 16, 8)], (t[2 * i + 1] - t[2 * i - 1]) * 1e-3);
        }
        bool ovf = false;
        std::vector<int> deep, wide;
        for (int bi : todo) {
            if (h[bi].err == NK_ERR_TIMEOUT)
                return set_error(NK_ERR_TIMEOUT, "batched sweep aborted: a bounded device-side wait or phase ran out (check %d, value %d)",
                                 h[bi].where, h[bi].bad_id);
            if (h[bi].err == kErrCheck)
                return set_error(NK_ERR_CUDA, "batched sweep aborted: device range check %d failed (value %d)",
                                 h[bi].where, h[bi].bad_id);
        }
        for (int bi : todo)
            if (h[bi].err == kErrWide) wide.push_back(bi);
        if (!wide.empty()) {
            // counts beyond 32 bits: these batches again with 64-bit sigma rows, together with
            // any that ran out of level slabs (an aborted batch never reaches the backward
            // sweep, so it has added nothing to the scores)
            for (int bi : todo)
                if (h[bi].err == kErrDepth) wide.push_back(bi);
            std::sort(wide.begin(), wide.end());
            s32 = false;
            NK_TRY(pick(kfn, grid));
            todo = wide;
            continue;
        }
        for (int bi : todo) {
            if (h[bi].err == NK_ERR_TIMEOUT)
                return set_error(NK_ERR_TIMEOUT, "batched sweep aborted: a bounded device-side wait or phase ran out (check %d, value %d)",
                                 h[bi].where, h[bi].bad_id);
            if (h[bi].err == kErrCheck)
                return set_error(NK_ERR_CUDA, "batched sweep aborted: device range check %d failed (value %d)",
                                 h[bi].where, h[bi].bad_id);
            ovf |= h[bi].ovf != 0;
            if (h[bi].err == kErrDepth) deep.push_back(bi);
        }
        if (ovf && !cfg.far) return set_error(NK_ERR_OVERFLOW, "a shortest-path count exceeded 2^64 - 1");
        if (cfg.far)  // closeness: batches with a wrapped path count go to the per-source form
            for (int bi : todo)
                if (h[bi].ovf && h[bi].err != kErrDepth) deep.push_back(bi);
        if (deep.empty()) return NK_OK;
        if (lcap < lmax && !(cfg.far && ovf)) {
            todo = deep;
            lcap = lmax;
            continue;
        }
        // deeper than any level cap that fits: the per-source form takes these sources
        for (int bi : deep) {
            RunCfg pc = cfg;
            pc.tpv = 0;
            if (pc.rk_t) {
                pc.rk_t += (size_t)bi * B;
                pc.rk_key += (size_t)bi * B;
            }
            NK_TRY(run_per_source(g, d_src + (size_t)bi * B, std::min(B, k - bi * B), d_scores, pc, st, s));
        }
        return NK_OK;
    }
}

// Capturable form of one pass of launch_batches: no host synchronisation and no
// allocation once prepared.  With prepare_only it sizes and allocates the workspace (call
// it before a stream capture); otherwise it enqueues the status reset and the cooperative
// launches (cudaLaunchKernelExC with the cooperative attribute, which stream capture
// records as kernel nodes) and returns the per-batch status words for the caller to read.
template <int W>
int enqueue_batches(nk_graph *g, const int32_t *d_src, int32_t k, double *d_scores,
                    const RunCfg &cfg, cudaStream_t s, bool prepare_only, Ctrl **ctrls_out, int *nb_out)
{
    constexpr int B = 64 * W;
    DevBuf *ws = scratch(cfg, g);
    HeavyView hw;
    NK_TRY(heavy_view(g, cfg.chunk, s, &hw));
    const int lcap = cfg.lcap > 0 ? std::min(cfg.lcap, std::max(g->n, 4)) : std::min(choose_lcap(g, B, ws, hw.chunk), std::max(kStartLevels, 4));
    if (lcap < 4) return set_error(NK_ERR_NOMEM, "not enough device memory for a batch of %d sources", B);
    const int nb = (k + B - 1) / B;
    const Layout L = layout(g, B, lcap, hw.chunk);
    // status words of the nb batches, then the compacted sources and their count
    const size_t ctrl_bytes = align_up(sizeof(Ctrl) * nb);
    const size_t bctrl_bytes = ctrl_bytes + align_up(sizeof(int32_t) * (size_t)k) + 256;
    if (prepare_only) {
        NK_TRY(ws[WS_BATCH].ensure(L.total));
        NK_TRY(ws[WS_BCTRL].ensure(bctrl_bytes));
        if (blocks_per_sm<W, false, true>() < 1) return set_error(NK_ERR_CUDA, "batched kernel cannot be resident");
        return NK_OK;
    }
    if (ws[WS_BATCH].bytes < L.total || ws[WS_BCTRL].bytes < bctrl_bytes)
        return set_error(NK_ERR_ARG, "batched workspace not prepared");
    const int bps = blocks_per_sm<W, false, true>();
    if (bps < 1) return set_error(NK_ERR_CUDA, "batched kernel cannot be resident");
    int grid = std::max(1, bps * num_sms() / std::max(1, cfg.grid_div));
    if (cfg.grid_ctas > 0) grid = std::min(grid, cfg.grid_ctas);
    char *base = ws[WS_BATCH].as<char>();
    BArgs a{};
    a.n = g->n;
    a.A = g->A;
    a.rp = g->rp.as<int32_t>();
    a.col = g->col.as<int32_t>();
    a.lcap = lcap;
    a.F = reinterpret_cast<unsigned long long *>(base + L.off_F);
    a.vis = reinterpret_cast<unsigned long long *>(base + L.off_vis);
    a.sp = reinterpret_cast<unsigned long long *>(base + L.off_sp);
    a.sp32 = reinterpret_cast<unsigned *>(base + L.off_sp32);
    a.qmark = reinterpret_cast<int32_t *>(base + L.off_qmark);
    a.queue = reinterpret_cast<int32_t *>(base + L.off_queue);
    a.qcap = L.qcap;
    const size_t lv = (size_t)lcap + 3;
    char *cb = base + L.off_cnt;
    a.mfv = reinterpret_cast<unsigned long long *>(cb);
    a.dmu = a.mfv + lv;
    a.vcnt = reinterpret_cast<int32_t *>(a.dmu + lv);
    a.qcnt = a.vcnt + lv;
    a.qoff = a.qcnt + lv;
    a.wq = a.qoff + lv;
    a.scores = d_scores;
    a.hv = hw.hv;
    a.hfirst = hw.hfirst;
    a.chunk_h = hw.chunk_h;
    a.H = hw.H;
    a.C = hw.C;
    a.chunk = hw.chunk;
    a.part = reinterpret_cast<unsigned long long *>(base + L.off_part);
    a.trace = nullptr;
    a.far = cfg.far;
    a.reach = cfg.reach;
    a.backward = cfg.backward ? 1 : 0;
    a.edge = nullptr;  // the captured form serves vertex scores only
    a.rk_t = nullptr;
    a.rk_key = nullptr;
    a.rk_count = nullptr;
    a.limit_ns = cfg.limit_ns ? cfg.limit_ns : wait_limit_ns();
    a.alpha = cfg.alpha > 0 ? cfg.alpha : 1.0;
    a.dir = cfg.direction;
    Ctrl *ctrls = ws[WS_BCTRL].as<Ctrl>();
    int32_t *csrc = reinterpret_cast<int32_t *>(ws[WS_BCTRL].as<char>() + ctrl_bytes);
    int32_t *ccnt = reinterpret_cast<int32_t *>(ws[WS_BCTRL].as<char>() + ctrl_bytes + align_up(sizeof(int32_t) * (size_t)k));
    NK_CUDA(cudaMemsetAsync(ctrls, 0, sizeof(Ctrl) * nb, s));
    // sources without arcs add nothing: compacted on the device, each batch reads the count
    NK_TRY(compact_sources(g, d_src, k, csrc, ccnt, s));
    a.ksrc = ccnt;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeCooperative;
    attr.val.cooperative = 1;
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(grid);
    lc.blockDim = dim3(kThreads);
    lc.dynamicSmemBytes = smem_bytes<W>();
    lc.stream = s;
    lc.attrs = &attr;
    lc.numAttrs = 1;
    for (int bi = 0; bi < nb; ++bi) {
        a.src = csrc + (size_t)bi * B;
        a.nsrc = std::min(B, k - bi * B);
        a.boff = bi * B;
        a.ctrl = ctrls + bi;
        void *args[] = {&a};
        NK_CUDA(cudaLaunchKernelExC(&lc, (const void *)k_batch<W, false, true>, args));
        ::nk::count_launch();
    }
    *ctrls_out = ctrls;
    *nb_out = nb;
    return NK_OK;
}

}  // namespace

size_t batched_bytes(const nk_graph *g, int B) { return layout(g, B, 16).total; }

size_t batched_bytes_lcap(const nk_graph *g, int B, int lcap) { return layout(g, B, lcap).total; }

int run_batched(nk_graph *g, const int32_t *d_src, int32_t k, double *d_scores,
                const RunCfg &cfg, RunStats *st, cudaStream_t s)
{
    int B = cfg.batch;
    if (B == 0) B = g->tuned.valid ? g->tuned.batch : 64;
    switch (B) {
    case 64: return launch_batches<1>(g, d_src, k, d_scores, cfg, st, s);
    case 128: return launch_batches<2>(g, d_src, k, d_scores, cfg, st, s);
    case 256: return launch_batches<4>(g, d_src, k, d_scores, cfg, st, s);
    default: return set_error(NK_ERR_ARG, "batch must be 64, 128 or 256 (got %d)", B);
    }
}

int enqueue_batched(nk_graph *g, const int32_t *d_src, int32_t k, double *d_scores,
                    const RunCfg &cfg, cudaStream_t s, bool prepare_only, Ctrl **ctrls, int *nb)
{
    int B = cfg.batch;
    if (B == 0) B = g->tuned.valid ? g->tuned.batch : 64;
    switch (B) {
    case 64: return enqueue_batches<1>(g, d_src, k, d_scores, cfg, s, prepare_only, ctrls, nb);
    case 128: return enqueue_batches<2>(g, d_src, k, d_scores, cfg, s, prepare_only, ctrls, nb);
    case 256: return enqueue_batches<4>(g, d_src, k, d_scores, cfg, s, prepare_only, ctrls, nb);
    default: return set_error(NK_ERR_ARG, "batch must be 64, 128 or 256 (got %d)", B);
    }
}

}  // namespace nk

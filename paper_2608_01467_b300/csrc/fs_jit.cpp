// Straight-line engine for the history kernel.
//
// At plan time every job's root and suffix regions (Algorithm 2) are
// compiled into straight-line sm_103a code: each op of the evaluation-order
// program becomes a few register instructions with its masks, bit positions
// and matrix elements as immediates, so the device spends no instructions
// fetching or decoding ops.  The generated source is this library's own CUDA
// C++, compiled by NVRTC to a cubin and loaded with cudaLibraryLoadData; one
// persistent kernel serves every job of the batch (a switch on the tile's
// job), with the same atomic tile queue, fixed-order reduction and counters
// as the interpreting kernel in fs_kernels.cu.
//
// Factors are applied with the same complex-product formula as the
// interpreter, specialised only where the specialisation is exact (unit
// factors skipped, -1 as a sign flip, purely real or imaginary factors as two
// products), so both engines give bit-identical history amplitudes.
#include <chrono>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include <cuda_runtime.h>
#include <nvrtc.h>

#include "fs_internal.h"

namespace fs {

namespace {

#define FS_XSTR(...) #__VA_ARGS__
#define FS_STR(...) FS_XSTR(__VA_ARGS__)

const char* kPrelude = R"PRE(
typedef unsigned int u32;
typedef int i32;
typedef unsigned long long u64;
typedef u32 uint32_t;
typedef i32 int32_t;
typedef u64 uint64_t;
struct Op;
struct Entry { u32 st[4]; double2 amp; };
)PRE"
"struct JobDev { " FS_STR(FS_JOBDEV_FIELDS) " };\n"
R"PRE(
#define TILE_LOG2 8
#define TILE 256
// programmatic dependent launch: wait for the previous grid, then let the
// next one be scheduled
#define FS_GRID_DEP() asm volatile("griddepcontrol.wait;\n\tgriddepcontrol.launch_dependents;" ::: "memory")

__device__ __forceinline__ double2 cmul(double2 a, double2 b)
{
    return make_double2(__fma_rn(a.x, b.x, -__dmul_rn(a.y, b.y)),
                        __fma_rn(a.x, b.y, __dmul_rn(a.y, b.x)));
}
__device__ __forceinline__ double dneg(double x)
{
    return __hiloint2double(__double2hiint(x) ^ 0x80000000, __double2loint(x));
}
__device__ __forceinline__ double2 cneg(double2 a) { return make_double2(dneg(a.x), dneg(a.y)); }
// a * i^r (r in 0..3): swaps and sign flips on the integer pipe, exact
__device__ __forceinline__ double2 qrot(double2 a, u32 r)
{
    const double x = (r & 1u) ? a.y : a.x, y = (r & 1u) ? a.x : a.y;
    const bool nx = r == 1u || r == 2u, ny = r >= 2u;
    return make_double2(nx ? dneg(x) : x, ny ? dneg(y) : y);
}
__device__ __forceinline__ double2 cre(double2 a, double r) { return make_double2(__dmul_rn(a.x, r), __dmul_rn(a.y, r)); }
__device__ __forceinline__ double2 cim(double2 a, double s) { return make_double2(dneg(__dmul_rn(a.y, s)), __dmul_rn(a.x, s)); }
// |a|^2 < eps2, with |a|^2 formed as fma(re, re, im * im); both sides are
// non-negative doubles, so their bit patterns compare like the values (an
// integer compare instead of an FP64 one)
__device__ __forceinline__ bool cut(double2 a, double eps2)
{
    const double m = __fma_rn(a.x, a.x, __dmul_rn(a.y, a.y));
    return __double_as_longlong(m) < __double_as_longlong(eps2);
}
// a * f for a real f, then times i when rot: the product by a purely real or
// purely imaginary factor, the same doubles as cmul by (f, 0) or (0, f)
__device__ __forceinline__ double2 crot(double2 a, double f, bool rot)
{
    const double2 p = make_double2(__dmul_rn(a.x, f), __dmul_rn(a.y, f));
    return rot ? make_double2(dneg(p.y), p.x) : p;
}
// a * t[0], out of line (see fs_add_ool): the per-class products of valid
// leaves, which most warps never need
__device__ __noinline__ double2 fs_cmul_ool(double2 a, const double2* t) { return cmul(a, __ldg(t)); }
__device__ __forceinline__ double2 sel2(bool c, double2 a, double2 b) { return c ? a : b; }

__device__ __forceinline__ u64 warp_sum_u64(u64 v)
{
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// Adds three per-thread counts into stats[k0], stats[k1], stats[k2] of job j
// (this thread's job; -1 or all-zero counts: nothing to add) at a kernel's
// end.  When every counting thread of the block has the same job, the block
// adds its sums with one atomic per counter: the counters of a job share a
// cache line, and thousands of warps adding to it one by one at the end of
// a short kernel queue up behind each other in L2.  Otherwise every thread
// adds its own counts.  Every thread of the block calls it.
__device__ __noinline__ void flush_stats3(const JobDev* jobs, int j, int k0, int k1, int k2, u64 a, u64 b, u64 c)
{
    __shared__ u64 s_red[32][3];
    __shared__ int s_job;
    const bool has = (a | b | c) != 0ull;
    if (threadIdx.x == 0) s_job = -1;
    __syncthreads();
    if (has) s_job = j;   // any one counting thread's job
    __syncthreads();
    const int jb = s_job;
    if (!__syncthreads_and(!has || j == jb)) {
        if (has) {
            if (a) atomicAdd(&jobs[j].stats[k0], a);
            if (b) atomicAdd(&jobs[j].stats[k1], b);
            if (c) atomicAdd(&jobs[j].stats[k2], c);
        }
        return;   // the same branch for the whole block
    }
    a = warp_sum_u64(a);
    b = warp_sum_u64(b);
    c = warp_sum_u64(c);
    if ((threadIdx.x & 31) == 0) {
        s_red[threadIdx.x >> 5][0] = a;
        s_red[threadIdx.x >> 5][1] = b;
        s_red[threadIdx.x >> 5][2] = c;
    }
    __syncthreads();
    if (threadIdx.x < 3 && jb >= 0) {
        u64 t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_red[w][threadIdx.x];
        const int k = threadIdx.x == 0 ? k0 : (threadIdx.x == 1 ? k1 : k2);
        if (t) atomicAdd(&jobs[jb].stats[k], t);
    }
}

// (output, input) of a pair index, pair = o * S + s.  Integer division by a
// runtime value goes through the scarce FP64 pipe on this part, so the
// quotient comes from the job's precomputed multiplier (division by an
// invariant integer, Granlund and Montgomery 1994, Fig. 4.1) for pair
// indices below 2^32.
__device__ __forceinline__ u64 pair_split(u64 pair, const JobDev& J, u64& s)
{
    const u32 S = (u32)J.S;
    if (S == 1u) { s = 0; return pair; }
    if (pair < (1ull << 32)) {
        const u32 p = (u32)pair, t = __umulhi(J.s_magic, p);
        const u32 o = (t + ((p - t) >> 1)) >> (J.s_shift - 1);
        s = p - o * S;
        return o;
    }
    const u64 o = pair / S;
    s = pair - o * S;
    return o;
}

// 32-bit word tests (64-bit integer operations run through the FP64 pipe)
__device__ __forceinline__ bool nonzero(double2 v)
{
    return (((unsigned)__double2hiint(v.x) | (unsigned)__double2hiint(v.y)) << 1 |
            (unsigned)__double2loint(v.x) | (unsigned)__double2loint(v.y)) != 0u;
}

// Sum of acc over each aligned group of seg lanes (seg a power of two, at
// most 32), valid in every lane of the group.  FP64 instructions cost the
// same for every lane on this part, and most histories' sums are exactly
// zero, so zero values (+-0, tested on the bits) are skipped: when no group
// holds more than four nonzero values they are added one by one in lane
// order, otherwise the xor butterfly runs.  The order depends only on which
// values are zero, so results are run-to-run identical.
__device__ __forceinline__ double2 group_sum(double2 acc, int seg)
{
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const bool nz = nonzero(acc);
    const unsigned m = __ballot_sync(full, nz);
    if (m == 0u) return make_double2(0.0, 0.0);
    const unsigned gmask = seg >= 32 ? full : (((1u << seg) - 1u) << (lane & ~(seg - 1)));
    unsigned rem = m & gmask;
    const int cnt = __popc(rem);
    const int maxcnt = (int)__reduce_max_sync(full, (unsigned)cnt);
    if (maxcnt <= 4) {
        double2 r = make_double2(0.0, 0.0);
        for (int it = 0; it < maxcnt; ++it) {
            const int src = rem ? __ffs(rem) - 1 : lane;
            rem &= rem - 1u;
            const double vx = __shfl_sync(full, acc.x, src), vy = __shfl_sync(full, acc.y, src);
            if (it == 0) {
                r = make_double2(vx, vy);
            } else if (it < cnt) {
                r.x += vx;
                r.y += vy;
            }
        }
        return cnt ? r : make_double2(0.0, 0.0);
    }
    for (int off = seg >> 1; off >= 1; off >>= 1) {
        acc.x += __shfl_xor_sync(full, acc.x, off);
        acc.y += __shfl_xor_sync(full, acc.y, off);
    }
    return acc;
}

// The FP64 adds of add_kept, out of line: a call that no lane makes issues
// none of the callee's instructions, where an inlined add would be
// if-converted into FP64 instructions predicated off in every lane -- and
// those still occupy the scarce FP64 pipe of this part.
__device__ __noinline__ double2 fs_add_ool(double2 a, double2 b)
{
    return make_double2(__dadd_rn(a.x, b.x), __dadd_rn(a.y, b.y));
}

// A logged item's sum times the job's constant, out of line: inlined, the
// product would be if-converted into FP64 instructions that every item of a
// run without logging issues with no lane active.
__device__ __noinline__ void fs_log_ool(double2* dst, double2 scale, double2 v) { *dst = cmul(scale, v); }

// acc += v in the lanes where keep holds.  Most leaves are invalid and most
// items zero, so the adds run only when some active lane keeps its value.
__device__ __forceinline__ void add_kept(double2& acc, double2 v, bool keep)
{
    if (__any_sync(__activemask(), keep)) {
        const double2 t = fs_add_ool(acc, v);
        if (keep) acc = t;
    }
}


// Loop counter type: 32-bit when the count fits (64-bit integer operations
// run through the FP64 pipe on this part).
template <bool Fits32> struct CounterType { typedef u64 type; };
template <> struct CounterType<true> { typedef u32 type; };

// bottom entries carry a NaN real part; tested on the bits (integer pipe)
__device__ __forceinline__ bool is_bottom(double x)
{
    const unsigned hi = (unsigned)__double2hiint(x) & 0x7fffffffu;
    return hi > 0x7ff00000u || (hi == 0x7ff00000u && (unsigned)__double2loint(x) != 0u);
}

// Leaves of one root checkpoint (state st, amplitude amp): the suffix for
// every h_s in increasing order, skipping the subtree of a cut history, the
// chi test at the input boundary.  A stacked suffix keeps the state, the
// amplitude and the deferred class counts after each of its source ops (a
// checkpoint per source, the per-source limit of Algorithm 2's regions) and
// restarts the next history at the first source whose bit changed, instead
// of at the region's start.

// amp * (re + i im), out of line (a call no lane makes issues none of its
// FP64 instructions)
__device__ __noinline__ double2 fs_census_ool(double2 amp, int re, int im)
{
    return cmul(amp, make_double2((double)re, (double)im));
}

// Phase census (exact suffixes whose factors are all unit phases): every
// valid leaf's amplitude is amp * i^q, so the leaves are counted by q and
// the root's sum is amp * ((n0 - n2) + i (n1 - n3)), one product per root
// instead of an FP64 add per valid leaf.
template <class T>
__device__ __forceinline__ double2 suffix_census(const u32 (&st)[T::W], double2 amp, const u32 (&bin)[T::W],
                                                 u64& completed, u64& valid, u64& visits)
{
    constexpr int W = T::W;
    u32 n0 = 0u, n1 = 0u, n2 = 0u, n3 = 0u;
    const u32 ns = 1u << T::As;
    u32 hs = 0u;
    auto leaf = [&](const u32 (&s2)[W], u32 q) {
        ++completed;
        u32 d = 0;
#pragma unroll
        for (int j = 0; j < W; ++j) d |= s2[j] ^ bin[j];
        const u32 ok = d == 0u ? 1u : 0u;
        valid += ok;
        n0 += ok & (q == 0u ? 1u : 0u);
        n1 += ok & (q == 1u ? 1u : 0u);
        n2 += ok & (q == 2u ? 1u : 0u);
        n3 += ok & (q == 3u ? 1u : 0u);
    };
    if constexpr (T::STACKED) {
        u32 sst[T::As][W];
        double2 sam[T::As];
        u32 skc[T::As][T::SCQ];
        int start = 0;
        while (hs < ns) {
            u32 st2[W];
            double2 amp2 = amp;
#pragma unroll
            for (int j = 0; j < W; ++j) st2[j] = start == 0 ? st[j] : sst[start - 1][j];
            u32 q = 0u;
            const int r2 = T::suffix_from_q(start, st2, amp2, (u64)hs, bin, visits, sst, sam, skc, q);
            u32 nx;
            if (r2 < 0) {
                leaf(st2, q);
                nx = hs + 1u;
            } else {
                nx = ((hs >> r2) + 1u) << r2;
            }
            if (nx < ns) start = T::As - 1 - (31 - __clz(hs ^ nx));
            hs = nx;
        }
    } else {
        while (hs < ns) {
            u32 st2[W];
#pragma unroll
            for (int j = 0; j < W; ++j) st2[j] = st[j];
            double2 amp2 = amp;
            u32 q = 0u;
            const int r2 = T::suffix_q(st2, amp2, (u64)hs, bin, visits, q);
            if (r2 < 0) {
                leaf(st2, q);
                ++hs;
            } else {
                hs = ((hs >> r2) + 1u) << r2;
            }
        }
    }
    const int re = (int)(n0 - n2), im = (int)(n1 - n3);
    double2 acc = make_double2(0.0, 0.0);
    if (__any_sync(__activemask(), (re | im) != 0)) {
        const double2 t = fs_census_ool(amp, re, im);
        if ((re | im) != 0) acc = t;
    }
    return acc;
}

template <class T>
__device__ __forceinline__ double2 suffix_sum(const u32 (&st)[T::W], double2 amp, const u32 (&bin)[T::W],
                                              u64& completed, u64& valid, u64& visits)
{
    constexpr int W = T::W;
    double2 acc = make_double2(0.0, 0.0);
    if constexpr (T::CENSUS) return suffix_census<T>(st, amp, bin, completed, valid, visits);
    typedef typename CounterType<(T::As < 32)>::type hs_t;   // 32-bit when it fits
    const hs_t ns = (hs_t)1 << T::As;
    hs_t hs = 0;
    if constexpr (T::STACKED) {
        u32 sst[T::As][W];
        double2 sam[T::As];
        u32 skc[T::As][T::SC];
        int start = 0;
        while (hs < ns) {
            u32 st2[W];
            double2 amp2;
            if (start == 0) {
#pragma unroll
                for (int j = 0; j < W; ++j) st2[j] = st[j];
                amp2 = amp;
            } else {
#pragma unroll
                for (int j = 0; j < W; ++j) st2[j] = sst[start - 1][j];
                amp2 = sam[start - 1];
            }
            const int r2 = T::suffix_from(start, st2, amp2, (u64)hs, bin, visits, sst, sam, skc);
            hs_t nx;
            if (r2 < 0) {
                ++completed;
                u32 d = 0;
#pragma unroll
                for (int j = 0; j < W; ++j) d |= st2[j] ^ bin[j];
                {
                    const bool ok = d == 0u;
                    valid += ok ? 1u : 0u;
                    add_kept(acc, amp2, ok);
                }
                nx = hs + (hs_t)1;
            } else {
                nx = ((hs >> r2) + (hs_t)1) << r2;
            }
            if (nx < ns) {
                // the highest bit that changes names the first source to redo
                const int msb = sizeof(hs_t) == 4 ? 31 - __clz((u32)(hs ^ nx))
                                                  : 63 - __clzll((long long)(u64)(hs ^ nx));
                start = T::As - 1 - msb;
            }
            hs = nx;
        }
    } else {
        while (hs < ns) {
            u32 st2[W];
#pragma unroll
            for (int j = 0; j < W; ++j) st2[j] = st[j];
            double2 amp2 = amp;
            const int r2 = T::suffix(st2, amp2, (u64)hs, bin, visits);
            if (r2 < 0) {
                ++completed;
                u32 d = 0;
#pragma unroll
                for (int j = 0; j < W; ++j) d |= st2[j] ^ bin[j];
                {
                    const bool ok = d == 0u;
                    valid += ok ? 1u : 0u;
                    add_kept(acc, amp2, ok);
                }
                ++hs;
            } else {
                hs = ((hs >> r2) + (hs_t)1) << r2;
            }
        }
    }
    return acc;
}

// Per-output leaf counts of a traced job (the paper's per-output cost
// distribution, Fig. 11): the completed and valid leaves of one item added
// to its output's counters.
__device__ __forceinline__ void trace_counts(const JobDev& J, u64 pair, u64 dc, u64 dv)
{
    if (!(dc | dv)) return;
    u64 s;
    const u64 o = pair_split(pair, J, s);
    if (dc) atomicAdd(&J.trace[2 * o], dc);
    if (dv) atomicAdd(&J.trace[2 * o + 1], dv);
}

// The checkpoint entry and input bits of the item a lane is on: consecutive
// items of a lane share them whenever they share (pair, h_p), so they are
// loaded once per change instead of once per item.
template <class T>
struct EntryCache {
    u64 pair, hp;
    u32 st[T::W], bin[T::W];
    double2 amp;
    bool bottom;
};

// Sum over the valid leaves of one (prefix, root) item: the root once, the
// suffix for every h_s (skipping cut subtrees), the chi test at the input.
template <class T>
__device__ __forceinline__ double2 item_sum(const JobDev& J, u64 pair,
                                            typename CounterType<(T::Ap + T::Ar <= 32)>::type local,
                                            EntryCache<T>& c, u64& completed, u64& valid, u64& visits)
{
    constexpr int W = T::W;
    double2 acc = make_double2(0.0, 0.0);
    typedef typename CounterType<(T::Ap + T::Ar <= 32)>::type loc_t;
    // (the shift counts stay below the type's width in every instantiation)
    const loc_t hp = T::Ap == 0 ? (loc_t)0 : (loc_t)(local >> (T::Ar % (8 * (int)sizeof(loc_t))));
    const loc_t hr = local & (loc_t)((1ull << T::Ar) - 1ull);
    if (pair != c.pair) {
        u64 s;
        pair_split(pair, J, s);
        const uint4 bv = __ldg(reinterpret_cast<const uint4*>(J.ins + 4 * s));
        const u32 btmp[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
        for (int j = 0; j < W; ++j) c.bin[j] = btmp[j];
    }
    if (pair != c.pair || (u64)hp != c.hp) {
        uint4 sv;
        if (J.table) {
            const uint4* ent = reinterpret_cast<const uint4*>(J.table + (pair << T::Ap) + hp);
            sv = __ldg(ent);
            c.amp = __ldg(reinterpret_cast<const double2*>(ent + 1));
            c.bottom = is_bottom(c.amp.x);
        } else {
            // an empty prefix region: the entry is (b_out, 1)
            u64 s;
            const u64 o = pair_split(pair, J, s);
            sv = __ldg(reinterpret_cast<const uint4*>(J.outs + 4 * o));
            c.amp = make_double2(1.0, 0.0);
            c.bottom = false;
        }
        const u32 tmp[4] = {sv.x, sv.y, sv.z, sv.w};
#pragma unroll
        for (int j = 0; j < W; ++j) c.st[j] = tmp[j];
        c.pair = pair;
        c.hp = hp;
    }
    if (c.bottom) return acc;
    u32 st[W];
#pragma unroll
    for (int j = 0; j < W; ++j) st[j] = c.st[j];
    double2 amp = c.amp;
    const u64 c0 = completed, v0 = valid;
    if (T::root(st, amp, hr, c.bin, visits) < 0) acc = suffix_sum<T>(st, amp, c.bin, completed, valid, visits);
    if (J.trace) trace_counts(J, pair, completed - c0, valid - v0);
    return acc;
}

// One 256-item tile on one warp: lane L takes items 8L .. 8L+7 in order and
// sums them per pair segment; segments of at least 8 items are then added
// across lanes (group_sum) into one partial per (pair, 256-item block).  No
// block-wide barrier: warps run their tiles independently.
template <class T>
__device__ void tile_body(const JobDev& J, u64 tile, u64& completed, u64& valid, u64& visits)
{
    const int lane = threadIdx.x & 31;
    constexpr int lg = T::Ap + T::Ar;   // items per pair: 2^lg
    typedef typename CounterType<(lg <= 32)>::type loc_t;
    const u64 n_items = J.n_pairs << lg;
    const u64 first = tile * TILE + (u64)lane * 8u;
    double2 acc = make_double2(0.0, 0.0);
    // the lane's items as (pair, index within the pair), advanced in place
    // (the index stays 32-bit where it fits)
    u64 pair = first >> lg;
    loc_t local = (loc_t)(first & ((1ull << lg) - 1ull));
    const int kn = first >= n_items ? 0 : (n_items - first < 8u ? (int)(n_items - first) : 8);
    EntryCache<T> cache;
    cache.pair = ~0ull;
    cache.hp = ~0ull;
#pragma unroll 1
    for (int k = 0; k < kn; ++k) {
        const double2 v = item_sum<T>(J, pair, local, cache, completed, valid, visits);
        if (J.log) fs_log_ool(J.log + first + (u64)k, J.scale, v);   // logging runs only
        add_kept(acc, v, nonzero(v));
        ++local;
        if (lg < 3 && local == ((loc_t)1 << (lg < 3 ? lg : 0))) {
            J.partials[pair] = acc;   // a pair of at most 4 items ends here
            acc = make_double2(0.0, 0.0);
            ++pair;
            local = 0;
        }
    }
    if (lg >= 3) {
        const int lps = lg >= 8 ? 32 : (1 << (lg - 3));   // lanes per pair segment
        acc = group_sum(acc, lps);
        if ((lane & (lps - 1)) == 0 && first < n_items) {
            const u64 p = first >> lg;
            const u64 l = first & ((1ull << lg) - 1ull);
            J.partials[(p << J.log2_spp) + (l >> TILE_LOG2)] = acc;
        }
    }
}

// Adds a warp's counts of one job into its stats (lane 0, one atomic each),
// then clears them.
__device__ __forceinline__ void warp_flush3(const JobDev& J, u64& completed, u64& valid, u64& visits)
{
    completed = warp_sum_u64(completed);
    valid = warp_sum_u64(valid);
    visits = warp_sum_u64(visits);
    if ((threadIdx.x & 31) == 0 && (completed | valid | visits)) {
        atomicAdd(&J.stats[0], completed);
        atomicAdd(&J.stats[1], valid);
        atomicAdd(&J.stats[2], visits);
    }
    completed = valid = visits = 0;
}

template <class T>
__device__ double2 compact_body(const JobDev& J, u64 i, u64& completed, u64& valid, u64& visits)
{
    constexpr int W = T::W;
    const u64 e = J.live[i >> T::Ar];
    typedef typename CounterType<(T::Ar <= 32)>::type hr_t;   // 32-bit when it fits
    const hr_t hr = (hr_t)i & (hr_t)((1ull << T::Ar) - 1ull);
    const u64 pair = e >> T::Ap;
    u64 sidx;
    const u64 o = pair_split(pair, J, sidx);
    const uint4* ent = reinterpret_cast<const uint4*>(J.table + e);
    const uint4 sv = __ldg(ent);
    double2 amp = __ldg(reinterpret_cast<const double2*>(ent + 1));
    if (is_bottom(amp.x)) return make_double2(0.0, 0.0);   // cut after the compaction
    const uint4 bv = __ldg(reinterpret_cast<const uint4*>(J.ins + 4 * sidx));
    const u32 tmp[4] = {sv.x, sv.y, sv.z, sv.w};
    const u32 btmp[4] = {bv.x, bv.y, bv.z, bv.w};
    u32 st[W], bin[W];
#pragma unroll
    for (int j = 0; j < W; ++j) { st[j] = tmp[j]; bin[j] = btmp[j]; }
    double2 acc = make_double2(0.0, 0.0);
    const u64 c0 = completed, v0 = valid;
    if (T::root(st, amp, hr, bin, visits) < 0) acc = suffix_sum<T>(st, amp, bin, completed, valid, visits);
    if (J.trace) trace_counts(J, pair, completed - c0, valid - v0);
    return acc;
}

// Subtree sums of 32 consecutive items (one warp).  With A_r >= 5 they share
// a live entry and are added (group_sum) into one partial per warp
// (esum[i / 32]); otherwise each item keeps its own (esum[i]).
__device__ __forceinline__ void store_esum(const JobDev& J, u64 i, double2 acc, bool active)
{
    if (J.Ar >= 5) {
        acc = group_sum(acc, 32);
        if ((threadIdx.x & 31) == 0 && active) J.esum[i >> 5] = acc;
    } else if (active) {
        J.esum[i] = acc;
    }
}

// Output reduction of a job that does it in its compacted history (odone
// set): the sums of an output are added in the order of the separate
// reduction kernel, so the amplitudes are the same doubles.  Items
// src[k], src[k + stride], ... below hi, the i-th into accumulator i mod 4,
// combined as (a0 + a1) + (a2 + a3), read from L2 (other SMs stored them
// during this kernel).
__device__ __forceinline__ double2 strided_sum_l2(const double2* src, u64 k, u64 hi, u32 stride)
{
    double2 a[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) a[u] = make_double2(0.0, 0.0);
    for (; k + 7 * (u64)stride < hi; k += 8 * (u64)stride) {
        double2 v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = __ldcg(src + k + (u64)u * stride);
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            a[u & 3].x += v[u].x;
            a[u & 3].y += v[u].y;
        }
    }
#pragma unroll
    for (int u = 0; u < 7; ++u) {
        if (k < hi) {
            const double2 v = __ldcg(src + k);
            a[u & 3].x += v.x;
            a[u & 3].y += v.y;
        }
        k += stride;
    }
    return make_double2((a[0].x + a[1].x) + (a[2].x + a[3].x), (a[0].y + a[1].y) + (a[2].y + a[3].y));
}

// An output none of whose pairs kept a live entry has amplitude 0 (nothing
// else writes it when the job reduces its own outputs).
__device__ __noinline__ void zero_empty_outputs(const JobDev& J, double2* amp_out)
{
    const u64 S = (u64)J.S;
    for (u64 o = (u64)blockIdx.x * blockDim.x + threadIdx.x; o < (u64)J.M; o += (u64)gridDim.x * blockDim.x)
        if (__ldg(J.prange + 2 * o * S) == __ldg(J.prange + 2 * (o * S + S - 1) + 1))
            amp_out[J.out_begin + o] = make_double2(0.0, 0.0);
}

// Called by a whole warp after it stored the subtree sum of its 32 items of
// live entry L: counts the sum for the entry's output (the store is made
// visible device-wide first).  The warp that stores an output's last sum
// adds the output's sums, pair by pair, times c_in of the pair's input
// (Eq. 2): four lanes for at most 64 sums, else the whole warp, as the
// reduction kernel does.
__device__ __noinline__ void sum_done(const JobDev& J, u64 L, double2* amp_out)
{
    const int lane = threadIdx.x & 31;
    u64 s0;
    const u64 o = pair_split(__ldg(J.live + L) >> J.Ap, J, s0);
    const u64 p0 = o * (u64)J.S;
    const int sh = J.Ar - 5;
    const u64 need = (__ldg(J.prange + 2 * (p0 + (u64)J.S - 1) + 1) - __ldg(J.prange + 2 * p0)) << sh;
    u32 done = 0;
    if (lane == 0) {
        __threadfence();
        done = atomicAdd(J.odone + o, 1u) + 1u;
    }
    done = __shfl_sync(0xffffffffu, done, 0);
    if ((u64)done != need) return;
    __threadfence();
    double2 amp = make_double2(0.0, 0.0);
    const bool small = need <= 64u;
    const int lanes = small ? 4 : 32;
    for (int s = 0; s < J.S; ++s) {
        const u64 lo = __ldg(J.prange + 2 * (p0 + (u64)s)) << sh;
        const u64 hi = __ldg(J.prange + 2 * (p0 + (u64)s) + 1) << sh;
        if (hi == lo) continue;   // the same pair for every lane
        double2 t = strided_sum_l2(J.esum, lo + (u64)(lane & (lanes - 1)), hi, (u32)lanes);
        for (int off = lanes / 2; off >= 1; off >>= 1) {
            t.x += __shfl_xor_sync(0xffffffffu, t.x, off);
            t.y += __shfl_xor_sync(0xffffffffu, t.y, off);
        }
        const double2 w = cmul(__ldg(J.coef + s), t);
        amp.x += w.x;
        amp.y += w.y;
    }
    if (lane == 0) amp_out[J.out_begin + o] = amp;
}

// History over the compacted live entries of one job.  With A_r < 5 every
// (live entry, h_r) item keeps its own subtree sum, and each lane takes its
// next item on its own: the subtrees of a threshold job differ widely in
// size, and a lane never waits for the rest of its warp.  Otherwise a warp
// takes 32 consecutive items (one live entry) and adds their sums.
template <class T>
__device__ __forceinline__ void compact_loop(const JobDev& J, u64& completed, u64& valid, u64& visits,
                                             double2* amp_out)
{
    const u64 nlive = J.stats[6] << T::Ar;
    if constexpr (T::Ar < 5) {
        for (;;) {
            const u64 i = atomicAdd(&J.stats[7], 1ull);
            if (i >= nlive) break;
            J.esum[i] = compact_body<T>(J, i, completed, valid, visits);
        }
    } else {
        const int lane = threadIdx.x & 31;
        for (;;) {
            u64 base = 0;
            if (lane == 0) base = atomicAdd(&J.stats[7], 32ull);
            base = __shfl_sync(0xffffffffu, base, 0);
            if (base >= nlive) break;
            const u64 i = base + lane;
            double2 acc = make_double2(0.0, 0.0);
            if (i < nlive) acc = compact_body<T>(J, i, completed, valid, visits);
            store_esum(J, i, acc, i < nlive);
            if (J.odone) sum_done(J, base >> T::Ar, amp_out);
        }
    }
}

// Level-by-level walk of a threshold job's suffix, a warp per live
// checkpoint entry.  The partial histories of the entry's subtree wait in
// per-level queues in shared memory: level L holds histories that passed
// the suffix's first L sources, at most WALK_CAP of them.  Each step takes
// up to 16 histories from the top of one level's queue and evaluates both
// values of their next source in the 32 lanes (segment L of the suffix);
// the histories that pass the threshold test are queued one level deeper,
// or, after the last source, run through the tail and the chi test.  The
// level is the one that fills the most lanes among those whose next level
// has room for the children (the deepest on ties): the deepest non-empty
// level always qualifies, since the level below it is empty, so no queue
// ever exceeds WALK_CAP.  Every history is expanded exactly once, as in the
// depth-first search, so the leaf counts and gate visits are the same; the
// lanes stay busy whatever the shape of the subtree, where a lane-per-item
// search leaves most of a warp idle.  The order of the additions into the
// entry's sum depends on the entry alone, so an output's amplitude does not
// depend on the other requested outputs.
//
// Shared memory per warp: amplitudes [As][WALK_CAP] (double2), then state
// words [As][W][WALK_CAP] (u32).  The count of level L is held by lane
// L % 32 (cnt0 for L < 32, cnt1 otherwise).
#define WALK_CAP 40
template <class T>
__device__ __forceinline__ void walk_loop(const JobDev& J, unsigned char* smem, u64& completed, u64& valid,
                                          u64& visits)
{
    constexpr int W = T::W, As = T::As, CAP = WALK_CAP;
    constexpr u32 per_warp = (u32)As * CAP * (16u + 4u * (u32)W);
    constexpr int sh = T::Ar >= 5 ? T::Ar - 5 : T::Ar;   // subtree sums per live entry: 2^sh
    constexpr u32 n_root = 1u << T::Ar;
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    double2* qa = reinterpret_cast<double2*>(smem + (threadIdx.x >> 5) * per_warp);
    u32* qs = reinterpret_cast<u32*>(qa + As * CAP);
    const u64 nlive = J.stats[6];
    for (;;) {
        u64 i = 0;
        if (lane == 0) i = atomicAdd(&J.stats[7], 1ull);
        i = __shfl_sync(full, i, 0);
        if (i >= nlive) break;
        const u64 e = J.live[i];
        const u64 pair = e >> T::Ap;
        u64 sidx;
        pair_split(pair, J, sidx);
        const uint4* ent = reinterpret_cast<const uint4*>(J.table + e);
        const uint4 sv = __ldg(ent);
        const double2 amp0 = __ldg(reinterpret_cast<const double2*>(ent + 1));
        const bool bottom = is_bottom(amp0.x);   // cut after the compaction
        const uint4 bv = __ldg(reinterpret_cast<const uint4*>(J.ins + 4 * sidx));
        const u32 tmp[4] = {sv.x, sv.y, sv.z, sv.w};
        const u32 btmp[4] = {bv.x, bv.y, bv.z, bv.w};
        u32 bin[W];
#pragma unroll
        for (int j = 0; j < W; ++j) bin[j] = btmp[j];
        const u64 c0 = completed, v0 = valid;
        for (u32 r0 = 0; r0 < n_root; r0 += 32u) {
            double2 acc = make_double2(0.0, 0.0);
            if (!bottom) {
                // the roots: lane l takes h_r = r0 + l; survivors form level 0
                u32 st[W];
#pragma unroll
                for (int j = 0; j < W; ++j) st[j] = tmp[j];
                double2 a = amp0;
                const u32 hr = r0 + (u32)lane;
                const bool live = hr < n_root && T::root(st, a, hr, bin, visits) < 0;
                const unsigned m = __ballot_sync(full, live);
                if (live) {
                    const int pos = __popc(m & lt);
                    qa[pos] = a;
#pragma unroll
                    for (int j = 0; j < W; ++j) qs[j * CAP + pos] = st[j];
                }
                u32 cnt0 = lane == 0 ? (u32)__popc(m) : 0u, cnt1 = 0u;
                __syncwarp();
                for (;;) {
                    // the level that fills the most lanes with room below it
                    const u32 nx0 = __shfl_down_sync(full, cnt0, 1), nx1 = __shfl_down_sync(full, cnt1, 1);
                    const u32 c32 = __shfl_sync(full, cnt1, 0);
                    const u32 next0 = lane == 31 ? c32 : nx0, next1 = lane == 31 ? 0u : nx1;
                    const u32 k0 = cnt0 < 16u ? cnt0 : 16u, k1 = cnt1 < 16u ? cnt1 : 16u;
                    const u32 key0 = (k0 && next0 + 2u * k0 <= (u32)CAP) ? (k0 << 6) | (u32)lane : 0u;
                    const u32 key1 = (k1 && next1 + 2u * k1 <= (u32)CAP) ? (k1 << 6) | (u32)(lane + 32) : 0u;
                    const u32 best = __reduce_max_sync(full, key0 > key1 ? key0 : key1);
                    if (best == 0u) break;
                    const int L = (int)(best & 63u);
                    const u32 k = best >> 6;
                    const u32 n = __shfl_sync(full, L >= 32 ? cnt1 : cnt0, L & 31);
                    const u32 base = n - k;
                    if (lane == (L & 31)) {
                        if (L >= 32) cnt1 = base;
                        else cnt0 = base;
                    }
                    const u32 node = (u32)lane >> 1;
                    const bool act = node < k;
                    u32 s2[W];
                    double2 a2 = make_double2(0.0, 0.0);
#pragma unroll
                    for (int j = 0; j < W; ++j) s2[j] = 0u;
                    int r = 1;
                    if (act) {
                        const int slot = (int)(base + node);
                        a2 = qa[L * CAP + slot];
#pragma unroll
                        for (int j = 0; j < W; ++j) s2[j] = qs[(L * W + j) * CAP + slot];
                        r = T::seg_step(L, s2, a2, (u32)lane & 1u, bin, visits);
                    }
                    const bool pass = act && r == 0;
                    if (L + 1 < As) {
                        const int L1 = L + 1;
                        const unsigned m2 = __ballot_sync(full, pass);
                        const u32 n1 = __shfl_sync(full, L1 >= 32 ? cnt1 : cnt0, L1 & 31);
                        if (pass) {
                            const int pos = (int)n1 + __popc(m2 & lt);
                            qa[L1 * CAP + pos] = a2;
#pragma unroll
                            for (int j = 0; j < W; ++j) qs[(L1 * W + j) * CAP + pos] = s2[j];
                        }
                        if (lane == (L1 & 31)) {
                            if (L1 >= 32) cnt1 = n1 + (u32)__popc(m2);
                            else cnt0 = n1 + (u32)__popc(m2);
                        }
                    } else {
                        bool ok = false;
                        if (pass && T::tail(s2, a2, 0ull, bin, visits) < 0) {
                            ++completed;
                            u32 d = 0;
#pragma unroll
                            for (int j = 0; j < W; ++j) d |= s2[j] ^ bin[j];
                            ok = d == 0u;
                            valid += ok ? 1u : 0u;
                        }
                        add_kept(acc, a2, ok);
                    }
                    __syncwarp();
                }
            }
            acc = group_sum(acc, 32);
            if (lane == 0) J.esum[(i << sh) + (r0 >> 5)] = acc;
            // with A_r < 5 the entry's other subtree sums are zero (its
            // whole sum is in the first)
            if (T::Ar < 5 && lane > 0 && (u32)lane < n_root) J.esum[(i << sh) + (u64)lane] = make_double2(0.0, 0.0);
        }
        if (J.trace) {
            const u64 dc = warp_sum_u64(completed - c0), dv = warp_sum_u64(valid - v0);
            if (lane == 0) trace_counts(J, pair, dc, dv);
        }
    }
}

// Level expansion prologue / epilogue (per-source prefix levels).
template <class T>
__device__ __forceinline__ bool lv_load(const JobDev& J, int a_prev, int a_next, const Entry* __restrict__ src,
                                        u64 idx, u32 (&st)[T::W], u32 (&bin)[T::W], double2& amp)
{
    constexpr int W = T::W;
    const u64 pair = idx >> a_next;
    const u64 child = idx & ((1ull << a_next) - 1ull);
    u64 sidx;
    const u64 o = pair_split(pair, J, sidx);
    const uint4 bv = __ldg(reinterpret_cast<const uint4*>(J.ins + 4 * sidx));
    const u32 btmp[4] = {bv.x, bv.y, bv.z, bv.w};
    uint4 sv;
    if (!src) {
        sv = __ldg(reinterpret_cast<const uint4*>(J.outs + 4 * o));
        amp = make_double2(1.0, 0.0);
    } else {
        const uint4* ent = reinterpret_cast<const uint4*>(src + (pair << a_prev) + (child >> (a_next - a_prev)));
        sv = ent[0];
        amp = reinterpret_cast<const double2*>(ent + 1)[0];
    }
    const u32 tmp[4] = {sv.x, sv.y, sv.z, sv.w};
#pragma unroll
    for (int j = 0; j < W; ++j) { st[j] = tmp[j]; bin[j] = btmp[j]; }
    return !is_bottom(amp.x);
}

template <class T>
__device__ __forceinline__ void lv_store(Entry* __restrict__ dst, u64 idx, const u32 (&st)[T::W], double2 amp, bool live)
{
    u32 w[4] = {0u, 0u, 0u, 0u};
#pragma unroll
    for (int j = 0; j < T::W; ++j) w[j] = st[j];
    if (!live) amp.x = __longlong_as_double(0x7ff8000000000000ll);
    uint4* d = reinterpret_cast<uint4*>(dst + idx);
    d[0] = make_uint4(w[0], w[1], w[2], w[3]);
    reinterpret_cast<double2*>(d + 1)[0] = amp;
}

__device__ __forceinline__ int find_job(const u64* __restrict__ begin, int n_jobs, u64 idx)
{
    int lo = 0, hi = n_jobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(begin + mid) <= idx) lo = mid; else hi = mid - 1;
    }
    return lo;
}

template <class T>
__device__ __forceinline__ bool prefix_body(const JobDev& J, u64 local, u64& visits, u64& entries, u64& bcuts)
{
    constexpr int W = T::W;
    const u64 pair = local >> T::Ap;
    const u64 hp = local & ((1ull << T::Ap) - 1ull);
    u64 sidx;
    const u64 o = pair_split(pair, J, sidx);
    const uint4 ov = __ldg(reinterpret_cast<const uint4*>(J.outs + 4 * o));
    const uint4 bv = __ldg(reinterpret_cast<const uint4*>(J.ins + 4 * sidx));
    const u32 otmp[4] = {ov.x, ov.y, ov.z, ov.w};
    const u32 btmp[4] = {bv.x, bv.y, bv.z, bv.w};
    u32 st[W], bin[W];
#pragma unroll
    for (int j = 0; j < W; ++j) { st[j] = otmp[j]; bin[j] = btmp[j]; }
    double2 amp = make_double2(1.0, 0.0);
    const int r = T::prefix(st, amp, hp, bin, visits);
    u32 w[4] = {0u, 0u, 0u, 0u};
#pragma unroll
    for (int j = 0; j < W; ++j) w[j] = st[j];
    bool live = r < 0;
    if (live) entries += 1;
    if constexpr (T::BOUND) {
        if (live && T::bound_cut(st, bin)) {   // exact: this entry cannot reach b_in
            live = false;
            ++bcuts;
        }
    }
    uint4* dst = reinterpret_cast<uint4*>(J.table + local);
    if (live) {
        dst[0] = make_uint4(w[0], w[1], w[2], w[3]);
        reinterpret_cast<double2*>(dst + 1)[0] = amp;
    } else {
        // a cut entry is only its bottom mark (NaN real part): no reader
        // looks at the rest of it, and the table writes drain faster
        reinterpret_cast<double*>(dst + 1)[0] = __longlong_as_double(0x7ff8000000000000ll);
    }
    return live;
}

// Live entries of a compaction block, counted by the warp that wrote them
// (one atomic when its 32 lanes lie in one block of one job).
__device__ __forceinline__ void count_live(const JobDev& J, u64 local, bool live, bool uniform)
{
    const unsigned keep = __ballot_sync(0xffffffffu, live);
    const u64 first = __shfl_sync(0xffffffffu, local, 0), last = __shfl_sync(0xffffffffu, local, 31);
    if (uniform && (first >> 10) == (last >> 10) && last == first + 31u) {
        if ((threadIdx.x & 31) == 0 && keep) atomicAdd(&J.blk[first >> 10], (unsigned)__popc(keep));
    } else if (live) {
        atomicAdd(&J.blk[local >> 10], 1u);
    }
}
)PRE";

std::string hexd(double v)
{
    char buf[64];
    snprintf(buf, sizeof buf, "%a", v);
    return buf;
}

std::string d2lit(double2 f) { return "make_double2(" + hexd(f.x) + ", " + hexd(f.y) + ")"; }

bool is_one(double2 f) { return f.x == 1.0 && f.y == 0.0; }
bool is_mone(double2 f) { return f.x == -1.0 && f.y == 0.0; }
bool is_real(double2 f) { return f.y == 0.0; }
bool is_imag(double2 f) { return f.x == 0.0; }
bool is_zero(double2 f) { return f.x == 0.0 && f.y == 0.0; }

// "a = a * f" for a compile-time factor, exact specialisations only.
std::string mul_const(double2 f)
{
    if (is_one(f)) return "";
    if (is_mone(f)) return "a = cneg(a);";
    if (is_real(f)) return "a = cre(a, " + hexd(f.x) + ");";
    if (is_imag(f)) return "a = cim(a, " + hexd(f.y) + ");";
    return "a = cmul(a, " + d2lit(f) + ");";
}

std::string bitexpr(int q) { return "((s[" + std::to_string(q >> 5) + "] >> " + std::to_string(q & 31) + ") & 1u)"; }

std::string flip(int q, const std::string& v)
{
    return "s[" + std::to_string(q >> 5) + "] ^= (" + v + ") << " + std::to_string(q & 31) + ";";
}

std::string match_expr(const uint32_t* m, int W)
{
    std::string e;
    for (int j = 0; j < W; ++j) {
        if (m[j] == 0 && m[W + j] == 0) continue;
        char buf[96];
        snprintf(buf, sizeof buf, "((s[%d] & 0x%08xu) ^ 0x%08xu)", j, m[j], m[W + j]);
        if (!e.empty()) e += " | ";
        e += buf;
    }
    if (e.empty()) return "true";
    return "((" + e + ") == 0u)";
}

// Selects among k factor constants by an index expression.
std::string select_factor(const double2* f, int k, const std::string& idx)
{
    // balanced select tree; equal constants collapse
    if (k == 1) return d2lit(f[0]);
    bool all_same = true;
    for (int i = 1; i < k; ++i) all_same &= (f[i].x == f[0].x && f[i].y == f[0].y);
    if (all_same) return d2lit(f[0]);
    if (k == 2) return "sel2((" + idx + ") != 0u, " + d2lit(f[1]) + ", " + d2lit(f[0]) + ")";
    const int h = k / 2;
    const std::string hi = select_factor(f + h, h, "(" + idx + ") - " + std::to_string(h) + "u");
    const std::string lo = select_factor(f, h, idx);
    return "sel2((" + idx + ") >= " + std::to_string(h) + "u, " + hi + ", " + lo + ")";
}

// Two-valued factor classes for exact mode: an op whose factor is A when a
// bit expression is 0 and B when it is 1 only adds that bit to the class
// counter k; at the end of the region the product prod A^(n-k) B^k is one
// lookup in a table built here in extended precision.  The result is the
// same product reassociated (within rounding), so it is used only when no
// pruning threshold reads the running amplitude.
struct FactorClass {
    double2 A, B;
    int n = 0;
};

bool same_d2(double2 a, double2 b) { return a.x == b.x && a.y == b.y; }

int class_of(std::vector<FactorClass>& cls, double2 A, double2 B)
{
    for (size_t c = 0; c < cls.size(); ++c)
        if (same_d2(cls[c].A, A) && same_d2(cls[c].B, B)) { cls[c].n++; return (int)c; }
    FactorClass f;
    f.A = A; f.B = B; f.n = 1;
    cls.push_back(f);
    return (int)cls.size() - 1;
}

// Commensurate phases of the job being generated: the deferred factors
// (1, e^{2 pi i p / 2^16}) of every region add p to one integer phase and
// cost one table product per region in all (`bits`: the OR of the p used,
// which sets the table's size).  Set by generate() for each job.
struct PhaseAcc {
    uint32_t bits = 0;
    std::string table;   // name of the job's phase table
};
thread_local PhaseAcc* t_phase = nullptr;

bool unit_phase_pair(double2 A, double2 B)
{
    return (B.x == A.x && B.y == A.y) || (B.x == -A.x && B.y == -A.y) || (B.x == -A.y && B.y == A.x) ||
           (B.x == A.y && B.y == -A.x);
}

void emit_phase_table(std::string& globals, const std::string& name, int m)
{
    const int M = 1 << m;
    globals += "__device__ const double2 " + name + "[" + std::to_string(M) + "] = {";
    const long double two_pi = 6.283185307179586476925286766559005768L;
    for (int k = 0; k < M; ++k) {
        const long double t = two_pi * (long double)k / (long double)M;
        globals += (k ? ", " : "") + std::string("{") + hexd((double)cosl(t)) + ", " + hexd((double)sinl(t)) + "}";
    }
    globals += "};\n";
}

void emit_class_table(std::string& globals, const std::string& name, const FactorClass& f)
{
    using cl = std::complex<long double>;
    const cl A((long double)f.A.x, (long double)f.A.y), B((long double)f.B.x, (long double)f.B.y);
    std::vector<cl> pa(f.n + 1), pb(f.n + 1);
    pa[0] = pb[0] = cl(1.0L, 0.0L);
    for (int j = 1; j <= f.n; ++j) { pa[j] = pa[j - 1] * A; pb[j] = pb[j - 1] * B; }
    globals += "__device__ const double2 " + name + "[" + std::to_string(f.n + 1) + "] = {";
    for (int k = 0; k <= f.n; ++k) {
        const cl v = pa[f.n - k] * pb[k];
        double2 d;
        d.x = (double)v.real();
        d.y = (double)v.imag();
        globals += (k ? ", " : "") + std::string("{") + hexd(d.x) + ", " + hexd(d.y) + "}";
    }
    globals += "};\n";
}

// A controlled incrementer / decrementer (find_cascade) as one borrow
// chain over the field's words: with y the field's ones (x - 1) or zeros
// (x + 1), the bits that flip are y ^ (y - 2^t0) restricted to the field.
std::string emit_cascade(const CascadeRun& r, int W)
{
    const int p = r.t0, top = r.t0 + r.len - 1;
    const int w0 = p >> 5, w1 = top >> 5;
    std::string c = "{ u32 b = " + std::to_string(1u << (p & 31)) + "u; ";
    for (int w = w0; w <= w1; ++w) {
        const int lo = w == w0 ? (p & 31) : 0, hi = w == w1 ? (top & 31) : 31;
        const uint32_t F = (hi == 31 ? 0xffffffffu : ((1u << (hi + 1)) - 1u)) & ~((1u << lo) - 1u);
        char buf[64];
        snprintf(buf, sizeof buf, "0x%08xu", F);
        const std::string ws = std::to_string(w);
        // a borrow leaves the first word only when its part of the field is
        // all ones (x - 1) or all zeros (x + 1): the later words sit behind
        // a vote, so a warp in which no lane borrows skips them
        if (w == w0 + 1) c += "if (__any_sync(__activemask(), b != 0u)) { ";
        c += "{ const u32 y = " + std::string(r.dec ? "" : "~") + "s[" + ws + "] & " + buf + "; const u32 d = y - b; ";
        if (w < w1) c += "b = (y < b) ? 1u : 0u; ";
        c += "s[" + ws + "] ^= (y ^ d) & " + buf + "; } ";
    }
    if (w1 > w0) c += "} ";
    c += "}";
    bool any = false;
    for (int j = 0; j < W; ++j) any |= r.cm[j] != 0;
    if (!any) return c;
    uint32_t m[8];
    for (int j = 0; j < W; ++j) {
        m[j] = r.cm[j];
        m[W + j] = r.cv[j];
    }
    return "if (" + match_expr(m, W) + ") " + c;
}

// Body of one region: ops [e0, e1).  nbits = the region's h width.
// chi_only: the region ends at the input boundary (the suffix); the deferred
// class products are then applied only when the final state passes the chi
// test, since only valid leaves are summed.
// hoist (root and suffix regions): a class whose two factors differ by a
// unit phase (B = A, -A, iA or -iA) is applied as that phase to the k-th
// power (sign flips and swaps on the integer pipe) and its constant A^n is
// multiplied into *hoist, to be applied once per (output, input) pair.
// First evaluation position from which factors may be deferred: 0 in exact
// mode; with a threshold, the position after the last op carrying a source
// (no later test reads the running amplitude, so the remaining factors may
// be reassociated).
// Threshold jobs test |beta| after every op carrying a source: their
// factors are multiplied literally up to the last such op, and their suffix
// keeps a checkpoint per source.  (The exact bound's tests after source ops
// read only the state, so bound jobs keep the deferred factors and the
// region-at-a-time suffix.)
bool tests_sources(const JitJobSpec& J) { return J.eps2 > 0.0; }

int defer_from(const JitJobSpec& J)
{
    if (!tests_sources(J)) return 0;
    int last = -1;
    for (int e = 0; e < J.G; ++e) {
        const Op& op = J.ops[e];
        const bool br = op.code == OP_H || op.code == OP_BR1 || op.code == OP_BR2;
        if (br && (op.s0 >= 0 || (op.code == OP_BR2 && op.s1 >= 0))) last = e;
    }
    return last + 1;
}

// Product by a two-valued factor selected by `sel` (0: A, 1: B) when each
// of A and B is purely real or purely imaginary: one real scalar product
// and an exact rotation, instead of a general complex product.
bool real_or_imag(double2 f) { return f.y == 0.0 || f.x == 0.0; }
std::string mul_two_valued(double2 A, double2 B, const std::string& sel)
{
    auto part = [](double2 f) { return f.y == 0.0 ? f.x : f.y; };
    const bool ra = A.y == 0.0, rb = B.y == 0.0;   // real (else imaginary)
    std::string rot;
    if (ra && rb) rot = "false";
    else if (!ra && !rb) rot = "true";
    else rot = ra ? "(" + sel + ") != 0u" : "(" + sel + ") == 0u";
    return "a = crot(a, (" + sel + ") ? " + hexd(part(B)) + " : " + hexd(part(A)) + ", " + rot + ");";
}

// stacked: the region is cut into segments that each end with an op
// carrying artificial sources; the generated function (suffix_from) runs
// the segments from `start` on, saving the state after each segment in
// sst / sam, so that the next history can restart at the first source whose
// bit changed.  `low` then starts at the bit of the last source before
// `start`, and visits count the ops run in this call.
// segswitch: the region's segments as the cases of a switch on L (segment L
// alone, its source bit given as `bit`; 1 when the history is cut, 0
// otherwise) -- the level-by-level walk of the suffix; the region must end
// with its last source op (the ops after it form the separate tail).
std::string bound_after(const JitJobSpec& J, int e, const std::string& visits_cut);

// With stacked, the deferred class counts (and the commensurate phase) are
// checkpointed with the state: skc[k][c] after segment k, restored at the
// restart; *n_save receives the number of saved counts (at least 1).
// census (in/out, with chi_only): the phase census of an exact suffix whose
// every factor is a unit phase -- deferred classes whose two factors differ
// by +-1 or +-i, and signs (NEG ops counted as the class (1, -1)).  A leaf's
// amplitude is then the suffix's starting amplitude times i^q; the
// generated function returns q (quarter turns) through `q` instead of
// applying the classes.  *census is cleared when the suffix has any other
// factor (a literal product, a table class, a commensurate phase).
void emit_region(std::string& out, std::string& globals, const std::string& tag, const JitJobSpec& J,
                 int e0, int e1, int nbits, bool chi_only = false, std::complex<long double>* hoist = nullptr,
                 bool stacked = false, bool segswitch = false, int* n_save = nullptr, int* census = nullptr)
{
    const bool cen = census && *census && chi_only && J.eps2 == 0.0;
    bool literal = false;   // census mode: an op multiplied the amplitude
    const int W = J.W;
    const int dfrom = defer_from(J);
    std::vector<FactorClass> cls;
    std::string body;
    int seg = 0, seg_e0 = e0;   // current segment and its first op
    if (stacked) body += "    if (start <= 0) {\n";
    if (segswitch) body += "    int low = 0;\n    (void)low;\n    switch (L) {\n    case 0: {\n";
    bool ph_used = false;
    auto count = [&](double2 A, double2 B, const std::string& bexpr) {
        uint32_t pidx = 0;
        if (t_phase && phase_index(A, B, &pidx) && !(hoist && unit_phase_pair(A, B))) {
            ph_used = true;
            t_phase->bits |= pidx;
            return "ph += (" + bexpr + ") ? " + std::to_string(pidx) + "u : 0u;";
        }
        const int c = class_of(cls, A, B);
        return "k" + std::to_string(c) + " += (" + bexpr + ");";
    };
    const double2 R = make_double2(0x1.6a09e667f3bcdp-1, 0.0), mR = make_double2(-0x1.6a09e667f3bcdp-1, 0.0);
    for (int e = e0; e < e1; ++e) {
        CascadeRun run;
        if (find_cascade(J.ops, J.masks, W, e, e1, run)) {
            body += "    " + emit_cascade(run, W) + "   // ops " + std::to_string(e) + ".." +
                    std::to_string(e + run.len - 1) + ": x " + (run.dec ? "- 1" : "+ 1") + "\n";
            e += run.len - 1;
            continue;
        }
        const Op& op = J.ops[e];
        const int q0 = op.q0, q1 = op.q1;
        const double2* F = J.fac + op.aux;
        const bool defer = e >= dfrom;
        const std::string visits_cut = "{ visits += " + std::to_string(e - seg_e0 + 1) + "ull; return " +
                                       (segswitch ? "1" : "low") + "; }";
        auto srcbit = [&](int sidx, int q) {
            if (segswitch && sidx >= 0) return std::string("bit");
            if (sidx >= 32) return "((u32)(h >> " + std::to_string(sidx) + ") & 1u)";
            return sidx >= 0 ? "((h32 >> " + std::to_string(sidx) + ") & 1u)"
                             : "((bin[" + std::to_string(q >> 5) + "] >> " + std::to_string(q & 31) + ") & 1u)";
        };
        std::string c;
        switch (op.code) {
        case OP_X: c = flip(q0, "1u"); break;
        case OP_MCX: c = "if (" + match_expr(J.masks + op.aux2, W) + ") " + flip(q0, "1u"); break;
        case OP_SWAP:
            c = "{ const u32 d = " + bitexpr(q0) + " ^ " + bitexpr(q1) + "; " + flip(q0, "d") + " " + flip(q1, "d") + " }";
            break;
        case OP_PERM1:
            if (defer)
                c = "{ const u32 o = " + bitexpr(q0) + "; " + count(F[0], F[1], "o") + " " + flip(q0, "1u") + " }";
            else
                c = "{ const u32 o = " + bitexpr(q0) + "; a = cmul(a, " + select_factor(F, 2, "o") + "); " + flip(q0, "1u") + " }";
            break;
        case OP_PERM2: {
            c = "{ const u32 o = " + bitexpr(q0) + " | (" + bitexpr(q1) + " << 1); ";
            char buf[64];
            snprintf(buf, sizeof buf, "const u32 i = (0x%xu >> (2u * o)) & 3u; ", op.aux2);
            c += buf;
            c += "a = cmul(a, " + select_factor(F, 4, "o") + "); " + flip(q0, "(o ^ i) & 1u") + " " +
                 flip(q1, "((o ^ i) >> 1) & 1u") + " }";
            break;
        }
        case OP_DIAG1:
            if (defer) c = count(F[0], F[1], bitexpr(q0));
            else c = "a = cmul(a, " + select_factor(F, 2, bitexpr(q0)) + ");";
            break;
        case OP_PH1: {
            if (defer) {
                if (!is_one(F[0])) c = count(make_double2(1.0, 0.0), F[0], bitexpr(q0));
            } else {
                const std::string m = mul_const(F[0]);
                if (!m.empty()) c = "if (" + bitexpr(q0) + ") { " + m + " }";
            }
            break;
        }
        case OP_NEG1:
            if (cen) c = count(make_double2(1.0, 0.0), make_double2(-1.0, 0.0), bitexpr(q0));
            else c = "if (" + bitexpr(q0) + ") a = cneg(a);";
            break;
        case OP_MCPH: {
            if (defer) {
                if (!is_one(F[0])) c = count(make_double2(1.0, 0.0), F[0], "(" + match_expr(J.masks + op.aux2, W) + ") ? 1u : 0u");
            } else {
                const std::string m = mul_const(F[0]);
                if (!m.empty()) c = "if (" + match_expr(J.masks + op.aux2, W) + ") { " + m + " }";
            }
            break;
        }
        case OP_MCNEG:
            if (cen) c = count(make_double2(1.0, 0.0), make_double2(-1.0, 0.0),
                               "(" + match_expr(J.masks + op.aux2, W) + ") ? 1u : 0u");
            else c = "if (" + match_expr(J.masks + op.aux2, W) + ") a = cneg(a);";
            break;
        case OP_DIAG2: {
            const bool parity = same_d2(F[0], F[3]) && same_d2(F[1], F[2]);
            if (parity && defer)
                c = count(F[0], F[1], bitexpr(q0) + " ^ " + bitexpr(q1));
            else if (parity)
                c = "a = cmul(a, " + select_factor(F, 2, bitexpr(q0) + " ^ " + bitexpr(q1)) + ");";
            else
                c = "a = cmul(a, " + select_factor(F, 4, bitexpr(q0) + " | (" + bitexpr(q1) + " << 1)") + ");";
            break;
        }
        case OP_H: {
            c = "{ const u32 o = " + bitexpr(q0) + "; const u32 i = " + srcbit(op.s0, q0) + "; ";
            if (defer) c += count(R, mR, "o & i") + " ";
            else c += "a = cre(a, (o & i) ? -0x1.6a09e667f3bcdp-1 : 0x1.6a09e667f3bcdp-1); ";
            c += flip(q0, "o ^ i") + " }";
            if (op.s0 >= 0) {
                c += " low = " + std::to_string(op.s0) + ";";
                if (J.eps2 > 0) c += " if (cut(a, " + hexd(J.eps2) + ")) " + visits_cut;
                c += bound_after(J, e, visits_cut);
            }
            break;
        }
        case OP_BR1: {
            bool any_zero = false;
            for (int i = 0; i < 4; ++i) any_zero |= is_zero(F[i]);
            const bool sym = same_d2(F[0], F[3]) && same_d2(F[1], F[2]);
            c = "{ const u32 o = " + bitexpr(q0) + "; const u32 i = " + srcbit(op.s0, q0) + "; ";
            if (defer && sym && !any_zero) c += count(F[0], F[1], "o ^ i") + " ";
            else if (sym && real_or_imag(F[0]) && real_or_imag(F[1])) c += mul_two_valued(F[0], F[1], "o ^ i") + " ";
            else c += "a = cmul(a, " + select_factor(F, 4, "(o << 1) | i") + "); ";
            c += flip(q0, "o ^ i");
            if (op.s0 >= 0) c += " low = " + std::to_string(op.s0) + ";";
            if (any_zero) {
                std::string zc;
                for (int k = 0; k < 4; ++k)
                    if (is_zero(F[k])) zc += std::string(zc.empty() ? "" : " || ") + "((o << 1) | i) == " + std::to_string(k) + "u";
                c += " if (" + zc + ") " + visits_cut;
            }
            if (op.s0 >= 0 && J.eps2 > 0) c += " if (cut(a, " + hexd(J.eps2) + ")) " + visits_cut;
            if (op.s0 >= 0) c += bound_after(J, e, visits_cut);
            c += " }";
            break;
        }
        case OP_BR2: {
            c = "{ const u32 o = " + bitexpr(q0) + " | (" + bitexpr(q1) + " << 1); const u32 i = " + srcbit(op.s0, q0) +
                " | (" + srcbit(op.s1, q1) + " << 1); a = cmul(a, " + select_factor(F, 16, "(o << 2) | i") + "); " +
                flip(q0, "(o ^ i) & 1u") + " " + flip(q1, "((o ^ i) >> 1) & 1u");
            int lo = 99;
            if (op.s0 >= 0) lo = op.s0;
            if (op.s1 >= 0 && op.s1 < lo) lo = op.s1;
            if (lo != 99) c += " low = " + std::to_string(lo) + ";";
            bool any_zero = false;
            for (int i = 0; i < 16; ++i) any_zero |= is_zero(F[i]);
            if (any_zero) {
                std::string zc;
                for (int k = 0; k < 16; ++k)
                    if (is_zero(F[k])) zc += std::string(zc.empty() ? "" : " || ") + "((o << 2) | i) == " + std::to_string(k) + "u";
                c += " if (" + zc + ") " + visits_cut;
            }
            if (lo != 99 && J.eps2 > 0) c += " if (cut(a, " + hexd(J.eps2) + ")) " + visits_cut;
            if (lo != 99) c += bound_after(J, e, visits_cut);
            c += " }";
            break;
        }
        default:
            c = "/* unknown op */";
            break;
        }
        if (cen && c.find("a = ") != std::string::npos) literal = true;
        if (!c.empty()) body += "    " + c + "\n";
        const bool carries = (op.code == OP_H || op.code == OP_BR1 || op.code == OP_BR2) &&
                             (op.s0 >= 0 || (op.code == OP_BR2 && op.s1 >= 0));
        if (segswitch && carries) {
            body += "    visits += " + std::to_string(e - seg_e0 + 1) + "ull;\n    return 0;\n    }\n";
            ++seg;
            seg_e0 = e + 1;
            if (seg < nbits) body += "    case " + std::to_string(seg) + ": {\n";
        }
        if (stacked && carries) {
            // close the segment: checkpoint after this source op
            const std::string k = std::to_string(seg);
            for (int j = 0; j < W; ++j)
                body += "    sst[" + k + "][" + std::to_string(j) + "] = s[" + std::to_string(j) + "];";
            body += " sam[" + k + "] = a; @SAVEK" + k + "@ visits += " + std::to_string(e - seg_e0 + 1) + "ull;\n    }\n";
            ++seg;
            seg_e0 = e + 1;
            if (seg < nbits) body += "    if (start <= " + std::to_string(seg) + ") {\n";
        }
    }
    if (stacked && seg < nbits) body += "    }\n";   // (a region whose last op carries no source)
    if (segswitch) {
        out += body + "    default: break;\n    }\n    (void)s; (void)a; (void)bin;\n    return 0;\n";
        return;
    }
    // 64-bit integer operations run through the FP64 pipe on this part:
    // the enumeration word is read as 32 bits wherever its bits allow
    out += "    const u32 h32 = (u32)h;\n    (void)h32;\n";
    out += stacked ? "    int low = " + std::to_string(nbits) + " - start;\n"
                   : "    int low = " + std::to_string(nbits) + ";\n";
    if (stacked) {
        // counts restored at the restart, saved after every segment
        const size_t nk = cls.size() + (ph_used ? 1 : 0);
        for (size_t k = 0; k < cls.size(); ++k)
            out += "    u32 k" + std::to_string(k) + " = start ? skc[start - 1][" + std::to_string(k) + "] : 0u;\n";
        if (ph_used) out += "    u32 ph = start ? skc[start - 1][" + std::to_string(cls.size()) + "] : 0u;\n";
        for (int seg_k = 0; seg_k < nbits; ++seg_k) {
            std::string save;
            for (size_t k = 0; k < cls.size(); ++k)
                save += "skc[" + std::to_string(seg_k) + "][" + std::to_string(k) + "] = k" + std::to_string(k) + "; ";
            if (ph_used) save += "skc[" + std::to_string(seg_k) + "][" + std::to_string(cls.size()) + "] = ph; ";
            const std::string tok = "@SAVEK" + std::to_string(seg_k) + "@";
            for (size_t at = body.find(tok); at != std::string::npos; at = body.find(tok))
                body.replace(at, tok.size(), save);
        }
        if (n_save) *n_save = nk > 0 ? (int)nk : 1;
        out += "    (void)skc;\n";
    } else {
        for (size_t k = 0; k < cls.size(); ++k) out += "    u32 k" + std::to_string(k) + " = 0u;\n";
        if (ph_used) out += "    u32 ph = 0u;\n";
    }
    out += body;
    if (cen) {
        // the leaf's phase in quarter turns; the classes' constants A^n go
        // to *hoist like the applied ones
        bool ok = !literal && !ph_used && hoist;
        std::string qs = "    u32 qq = 0u;\n";
        for (size_t k = 0; k < cls.size() && ok; ++k) {
            const FactorClass& f = cls[k];
            const double2 A = f.A, B = f.B;
            int kind = -1;
            if (B.x == A.x && B.y == A.y) kind = 0;
            else if (B.x == -A.x && B.y == -A.y) kind = 1;
            else if (B.x == -A.y && B.y == A.x) kind = 2;
            else if (B.x == A.y && B.y == -A.x) kind = 3;
            if (kind < 0) { ok = false; break; }
            using cl = std::complex<long double>;
            cl An(1.0L, 0.0L);
            const cl Al((long double)A.x, (long double)A.y);
            for (int i = 0; i < f.n; ++i) An *= Al;
            *hoist *= An;
            const std::string kv = "k" + std::to_string(k);
            if (kind == 1) qs += "    qq += (" + kv + " & 1u) << 1;\n";
            else if (kind == 2) qs += "    qq += " + kv + ";\n";
            else if (kind == 3) qs += "    qq += 3u * " + kv + ";\n";
        }
        *census = ok ? 1 : 0;
        out += qs + "    q = qq & 3u;\n";
        out += "    visits += " + std::to_string(e1 - seg_e0) + "ull;\n    (void)low;\n    return -1;\n";
        return;
    }
    const bool products = !cls.empty() || ph_used;
    if (chi_only && products) {
        out += "    u32 dchi = 0u;\n";
        for (int j = 0; j < W; ++j) out += "    dchi |= s[" + std::to_string(j) + "] ^ bin[" + std::to_string(j) + "];\n";
        // the class products only for valid leaves, behind a vote so that
        // a warp with no valid leaf issues none of their FP64 instructions
        out += "    if (__any_sync(__activemask(), dchi == 0u)) {\n";
    }
    for (size_t k = 0; k < cls.size(); ++k) {
        const FactorClass& f = cls[k];
        const std::string kv = "k" + std::to_string(k);
        if (hoist) {
            using cl = std::complex<long double>;
            const double2 A = f.A, B = f.B;
            int kind = -1;   // 0: B = A, 1: B = -A, 2: B = iA, 3: B = -iA
            if (B.x == A.x && B.y == A.y) kind = 0;
            else if (B.x == -A.x && B.y == -A.y) kind = 1;
            else if (B.x == -A.y && B.y == A.x) kind = 2;
            else if (B.x == A.y && B.y == -A.x) kind = 3;
            if (kind >= 0) {
                cl An(1.0L, 0.0L);
                const cl Al((long double)A.x, (long double)A.y);
                for (int i = 0; i < f.n; ++i) An *= Al;
                *hoist *= An;
                if (kind == 1) out += "    if (" + kv + " & 1u) a = cneg(a);\n";
                else if (kind == 2) out += "    a = qrot(a, " + kv + " & 3u);\n";
                else if (kind == 3) out += "    a = qrot(a, (4u - (" + kv + " & 3u)) & 3u);\n";
                continue;
            }
        }
        const std::string name = "T_" + tag + "_" + std::to_string(k);
        emit_class_table(globals, name, f);
        out += chi_only ? "    a = fs_cmul_ool(a, &" + name + "[" + kv + "]);\n"
                        : "    a = cmul(a, __ldg(&" + name + "[" + kv + "]));\n";
    }
    if (ph_used) {
        const std::string idx = "&" + t_phase->table + "[(ph >> PH_SHIFT) & PH_MASK]";
        out += chi_only ? "    a = fs_cmul_ool(a, " + idx + ");\n" : "    a = cmul(a, __ldg(" + idx + "));\n";
    }
    if (chi_only && products) out += "    }\n";
    out += "    visits += " + std::to_string(e1 - seg_e0) + "ull;\n    (void)low;\n    return -1;\n";
}

// The exact reachability bound of a job as code (the BoundSpec as
// immediates): true when the checkpoint state s cannot reach bin.
std::string emit_bound_fn(const std::string& name, int W, bool enabled, const BoundSpec& B)
{
    std::string c = "  static __device__ __forceinline__ bool " + name + "(const u32 (&s)[" + std::to_string(W) +
                    "], const u32 (&bin)[" + std::to_string(W) + "]) {\n";
    if (!enabled) return c + "    (void)s; (void)bin;\n    return false;\n  }\n";
    c += "    u32 d = 0u;\n";
    for (int j = 0; j < W; ++j)
        if (B.frozen[j]) {
            char buf[96];
            snprintf(buf, sizeof buf, "    d |= (s[%d] ^ bin[%d]) & 0x%08xu;\n", j, j, B.frozen[j]);
            c += buf;
        }
    c += "    if (d) return true;\n";
    // a field: its value in 32-bit words (funnel shifts at fixed offsets),
    // both cyclic differences by borrow chains, each compared with the radius
    for (int f = 0; f < B.n_fields; ++f) {
        const int t0 = B.t0[f], len = B.len[f], FW = (len + 31) / 32;
        const uint32_t top = (len % 32) ? ((1u << (len % 32)) - 1u) : 0xffffffffu;
        c += "    {\n";
        auto word = [&](const std::string& v, int k) {
            const int pos = t0 + 32 * k, w = pos >> 5, sh = pos & 31;
            const std::string lo = w < W ? v + "[" + std::to_string(w) + "]" : "0u";
            const std::string hi = w + 1 < W ? v + "[" + std::to_string(w + 1) + "]" : "0u";
            return sh ? "__funnelshift_r(" + lo + ", " + hi + ", " + std::to_string(sh) + "u)" : lo;
        };
        for (int k = 0; k < FW; ++k) {
            char m[32];
            snprintf(m, sizeof m, "0x%08xu", k == FW - 1 ? top : 0xffffffffu);
            c += "      const u32 a" + std::to_string(k) + " = " + word("s", k) + " & " + m + ", b" + std::to_string(k) +
                 " = " + word("bin", k) + " & " + m + ";\n";
        }
        for (const char* dir : {"u", "v"}) {   // u = a - b, v = b - a (mod 2^len)
            const bool ab = dir[0] == 'u';
            c += "      u32 " + std::string(dir) + "br = 0u;\n";
            for (int k = 0; k < FW; ++k) {
                const std::string x = (ab ? "a" : "b") + std::to_string(k), y = (ab ? "b" : "a") + std::to_string(k);
                char m[32];
                snprintf(m, sizeof m, "0x%08xu", k == FW - 1 ? top : 0xffffffffu);
                c += "      const u32 " + std::string(dir) + std::to_string(k) + " = (" + x + " - " + y + " - " + dir +
                     "br) & " + m + "; " + dir + "br = (" + x + " < " + y + ") || (" + x + " == " + y + " && " + dir +
                     "br) ? 1u : 0u;\n";
            }
            std::string hiw = "0u";
            for (int k = 1; k < FW; ++k) hiw += " | " + std::string(dir) + std::to_string(k);
            c += "      const bool " + std::string(dir) + "far = (" + hiw + ") != 0u || " + dir + "0 > " +
                 std::to_string(B.radius[f]) + "u;\n";
        }
        c += "      if (ufar && vfar) return true;\n    }\n";
    }
    return c + "    return false;\n  }\n";
}

// The bound at the checkpoint (bound_cut) and after each source op of the
// root and suffix (bound_after_<e>).
std::string emit_bound(const JitJobSpec& J)
{
    std::string c = emit_bound_fn("bound_cut", J.W, J.bound, J.bspec);
    if (J.bound)
        for (const auto& pb : J.src_bounds) c += emit_bound_fn("bound_after_" + std::to_string(pb.first), J.W, true, pb.second);
    return c;
}

// The per-source bound test after op e, or "" (none at e).
std::string bound_after(const JitJobSpec& J, int e, const std::string& visits_cut)
{
    if (!J.bound) return "";
    for (const auto& pb : J.src_bounds)
        if (pb.first == e) return " if (bound_after_" + std::to_string(e) + "(s, bin)) " + visits_cut;
    return "";
}

// Jobs whose suffix carries artificial sources, one per op -- at least two
// with a threshold, ten in exact mode (below that the checkpoint stores
// cost more than the gates they save; measured on amplitude amplification
// and the walk) -- run the stacked suffix (a checkpoint after every source
// op).
bool stacked_suffix(const JitJobSpec& J)
{
    if (J.As < (J.eps2 > 0.0 ? 2 : 10)) return false;
    int n = 0;
    for (int e = J.c2; e < J.G; ++e) {
        const Op& op = J.ops[e];
        if (op.code == OP_BR2 && op.s0 >= 0 && op.s1 >= 0) return false;
        const bool br = op.code == OP_H || op.code == OP_BR1 || op.code == OP_BR2;
        if (br && (op.s0 >= 0 || op.s1 >= 0)) ++n;
    }
    return n == J.As;
}

// Threshold jobs whose suffix walks level by level (a warp per root
// checkpoint, per-level queues of partial histories): the stacked ones with
// at least 5 sources in the suffix.  Returns the evaluation position of the
// suffix's last source op, or -1.
int queue_last_source(const JitJobSpec& J)
{
    if (J.eps2 == 0.0 || !stacked_suffix(J) || J.As < 5) return -1;
    int last = -1;
    for (int e = J.c2; e < J.G; ++e) {
        const Op& op = J.ops[e];
        const bool br = op.code == OP_H || op.code == OP_BR1 || op.code == OP_BR2;
        if (br && (op.s0 >= 0 || op.s1 >= 0)) last = e;
    }
    return last;
}

std::string generate(const std::vector<JitJobSpec>& jobs, std::vector<double2>* scales)
{
    std::string src = kPrelude;
    std::string globals, structs;
    for (size_t j = 0; j < jobs.size(); ++j) {
        const JitJobSpec& J = jobs[j];
        const std::string W = std::to_string(J.W), js = std::to_string(j);
        const bool stacked = stacked_suffix(J);
        const int qlast = queue_last_source(J);   // >= 0: the suffix walks level by level
        structs += "struct J" + js + " {\n";
        structs += "  static constexpr int W = " + W + ", Ap = " + std::to_string(J.Ap) + ", Ar = " +
                   std::to_string(J.Ar) + ", As = " + std::to_string(J.As) + ";\n";
        structs += std::string("  static constexpr bool STACKED = ") + (stacked ? "true" : "false") + ";\n";
        structs += std::string("  static constexpr bool QUEUE = ") + (qlast >= 0 ? "true" : "false") + ";\n";
        structs += std::string("  static constexpr bool BOUND = ") + (J.bound ? "true" : "false") +
                   ", COUNTB = " + (J.bound && J.bound_counts ? "true" : "false") + ";\n";
        structs += emit_bound(J);
        PhaseAcc phase;
        phase.table = "PH_J" + js;
        t_phase = &phase;
        const std::string sig = "(u32 (&s)[" + W + "], double2& a, u64 h, const u32 (&bin)[" + W + "], u64& visits)";
        structs += "  static __device__ __forceinline__ int prefix" + sig + " {\n    (void)h; (void)bin;\n";
        if (J.levels.empty()) emit_region(structs, globals, js + "p", J, 0, J.c1, J.Ap);
        else structs += "    (void)s; (void)a; (void)visits;\n    return -1;   // expanded level by level\n";
        structs += "  }\n";
        for (size_t k = 0; k < J.levels.size(); ++k) {
            structs += "  // level " + std::to_string(k) + ": ops [" + std::to_string(J.levels[k].e0) + ", " +
                       std::to_string(J.levels[k].e1) + "), sources [" + std::to_string(J.levels[k].a_prev) + ", " +
                       std::to_string(J.levels[k].a_next) + ")\n";
            structs += "  static __device__ __forceinline__ int lv" + std::to_string(k) + sig + " {\n    (void)h; (void)bin;\n";
            emit_region(structs, globals, js + "l" + std::to_string(k), J, J.levels[k].e0, J.levels[k].e1, J.Ap);
            structs += "  }\n";
        }
        structs += "  static __device__ __forceinline__ int root" + sig + " {\n    (void)h; (void)bin;\n";
        std::complex<long double> hoisted(1.0L, 0.0L);
        emit_region(structs, globals, js + "r", J, J.c1, J.c2, J.Ar, false, &hoisted);
        structs += "  }\n";
        if (qlast >= 0) {
            // the suffix as one switch case per source segment, and its tail
            // (the ops after the last source: deferred classes, chi)
            std::complex<long double> h3(1.0L, 0.0L);
            structs += "  static __device__ __forceinline__ int seg_step(int L, u32 (&s)[" + W + "], double2& a, u32 bit, "
                       "const u32 (&bin)[" + W + "], u64& visits) {\n    (void)bit;\n";
            emit_region(structs, globals, js + "q", J, J.c2, qlast + 1, J.As, false, nullptr, false, true);
            structs += "  }\n";
            structs += "  static __device__ __forceinline__ int tail" + sig + " {\n    (void)h; (void)bin;\n";
            emit_region(structs, globals, js + "u", J, qlast + 1, J.G, 0, true, &h3);
            structs += "  }\n";
        }
        // the phase census of a unit-phase exact suffix (4 or more sources,
        // up to 30): suffix_q / suffix_from_q return each leaf's quarter
        // turns, and the leaves of a root are counted by phase
        bool census = false;
        if (J.eps2 == 0.0 && J.As >= 4 && J.As <= 30) {
            PhaseAcc* keep = t_phase;
            t_phase = nullptr;
            std::string fq, fsq;
            std::complex<long double> hq(1.0L, 0.0L), hsq(1.0L, 0.0L);
            int ok1 = 1, ok2 = 1, scq = 1;
            emit_region(fq, globals, js + "c", J, J.c2, J.G, J.As, true, &hq, false, false, nullptr, &ok1);
            if (stacked)
                emit_region(fsq, globals, js + "d", J, J.c2, J.G, J.As, true, &hsq, true, false, &scq, &ok2);
            t_phase = keep;
            census = ok1 && ok2;
            if (census) {
                structs += "  static __device__ __forceinline__ int suffix_q(u32 (&s)[" + W + "], double2& a, u64 h, "
                           "const u32 (&bin)[" + W + "], u64& visits, u32& q) {\n    (void)h; (void)bin;\n" + fq + "  }\n";
                if (stacked)
                    structs += "  static constexpr int SCQ = " + std::to_string(scq) + ";\n"
                               "  static __device__ __forceinline__ int suffix_from_q(int start, u32 (&s)[" + W +
                               "], double2& a, u64 h, const u32 (&bin)[" + W + "], u64& visits, u32 (&sst)[" +
                               std::to_string(J.As) + "][" + W + "], double2 (&sam)[" + std::to_string(J.As) +
                               "], u32 (&skc)[" + std::to_string(J.As) + "][" + std::to_string(scq) +
                               "], u32& q) {\n    (void)h; (void)bin;\n" + fsq + "  }\n";
            }
        }
        structs += std::string("  static constexpr bool CENSUS = ") + (census ? "true" : "false") + ";\n";
        if (!(census && stacked)) structs += "  static constexpr int SCQ = 1;\n";
        if (stacked) {
            // the same suffix as per-source segments (its hoisted constant is
            // the one of `suffix` below: the same classes); the class counts
            // are checkpointed with the state
            std::complex<long double> h2(1.0L, 0.0L);
            std::string fn;
            int sc = 1;
            emit_region(fn, globals, js + "t", J, J.c2, J.G, J.As, true, &h2, true, false, &sc);
            structs += "  static constexpr int SC = " + std::to_string(sc) + ";\n";
            structs += "  static __device__ __forceinline__ int suffix_from(int start, u32 (&s)[" + W +
                       "], double2& a, u64 h, const u32 (&bin)[" + W + "], u64& visits, u32 (&sst)[" +
                       std::to_string(J.As) + "][" + W + "], double2 (&sam)[" + std::to_string(J.As) +
                       "], u32 (&skc)[" + std::to_string(J.As) + "][" + std::to_string(sc) +
                       "]) {\n    (void)h; (void)bin;\n" + fn + "  }\n";
        }
        structs += "  static __device__ __forceinline__ int suffix" + sig + " {\n    (void)h; (void)bin;\n";
        emit_region(structs, globals, js + "s", J, J.c2, J.G, J.As, true, &hoisted);
        const double2 sc = make_double2((double)hoisted.real(), (double)hoisted.imag());
        if (scales) (*scales)[j] = sc;
        structs += "// J" + js + ": constant factor of the root and suffix, applied through c_in: (" + hexd(sc.x) +
                   ", " + hexd(sc.y) + ")\n";
        structs += "  }\n";
        // the phase table: 2^m entries, m from the lowest phase bit used
        t_phase = nullptr;
        int m = 0;
        if (phase.bits) {
            m = 16;
            while (m > 0 && !(phase.bits & (1u << (16 - m)))) --m;
            emit_phase_table(globals, phase.table, m);
        }
        structs += "  static constexpr int PH_SHIFT = " + std::to_string(16 - m) + ";\n";
        structs += "  static constexpr u32 PH_MASK = " + std::to_string((1u << m) - 1u) + "u;\n";
        structs += "};\n";
    }
    src += globals;
    src += structs;
    // persistent warps pull tiles off the queue; the next index is fetched
    // while the current tile runs
    // a warp keeps its counts while its tiles are of one job and adds them
    // to that job's stats when the job changes and at the end
    src += "extern \"C\" __global__ void __launch_bounds__(256) fs_jit_history(const JobDev* __restrict__ jobs, "
           "const uint2* __restrict__ tiles, u64 n_tiles, unsigned int* counter)\n{\n"
           "    FS_GRID_DEP();\n"
           "    const int lane = threadIdx.x & 31;\n    unsigned int t = 0u, next = 0u;\n"
           "    u64 completed = 0, valid = 0, visits = 0;\n    int cj = -1;\n"
           "    if (lane == 0) t = atomicAdd(counter, 1u);\n    t = __shfl_sync(0xffffffffu, t, 0);\n"
           "    while ((u64)t < n_tiles) {\n"
           "        if (lane == 0) next = atomicAdd(counter, 1u);\n        const uint2 td = tiles[t];\n"
           "        if ((int)td.x != cj) {\n"
           "            if (cj >= 0) warp_flush3(jobs[cj], completed, valid, visits);\n"
           "            cj = (int)td.x;\n        }\n"
           "        switch (td.x) {\n";
    for (size_t j = 0; j < jobs.size(); ++j)
        src += "        case " + std::to_string(j) + "u: tile_body<J" + std::to_string(j) + ">(jobs[" +
               std::to_string(j) + "], td.y, completed, valid, visits); break;\n";
    src += "        default: break;\n        }\n        t = __shfl_sync(0xffffffffu, next, 0);\n    }\n"
           "    flush_stats3(jobs, cj, 0, 1, 2, completed, valid, visits);\n}\n";
    // four blocks per SM (64 registers): the items of a live entry are
    // short chains, and the warps of a fourth block hide their latency
    // better than the registers a few spilled values would take
    src += "extern \"C\" __global__ void __launch_bounds__(256, 4) fs_jit_compact(const JobDev* __restrict__ jobs, int job, "
           "double2* amp_out)\n{\n"
           "    FS_GRID_DEP();\n"
           "    const JobDev& J = jobs[job];\n"
           "    if (J.odone) zero_empty_outputs(J, amp_out);\n"
           "    u64 completed = 0, valid = 0, visits = 0;\n    switch (job) {\n";
    for (size_t j = 0; j < jobs.size(); ++j)
        if (jobs[j].compact)
            src += "    case " + std::to_string(j) + ": compact_loop<J" + std::to_string(j) +
                   ">(J, completed, valid, visits, amp_out); break;\n";
    src += "    default: break;\n    }\n"
           "    flush_stats3(jobs, job, 0, 1, 2, completed, valid, visits);\n}\n";
    bool any_queue = false;
    for (const JitJobSpec& J : jobs) any_queue |= queue_last_source(J) >= 0;
    if (any_queue) {
        src += "extern \"C\" __global__ void __launch_bounds__(256) fs_jit_walk(const JobDev* __restrict__ jobs, int job, "
               "double2*)\n{\n"
               "    FS_GRID_DEP();\n"
               "    extern __shared__ __align__(16) unsigned char walk_smem[];\n"
               "    const JobDev& J = jobs[job];\n"
               "    u64 completed = 0, valid = 0, visits = 0;\n    switch (job) {\n";
        for (size_t j = 0; j < jobs.size(); ++j)
            if (queue_last_source(jobs[j]) >= 0)
                src += "    case " + std::to_string(j) + ": walk_loop<J" + std::to_string(j) +
                       ">(J, walk_smem, completed, valid, visits); break;\n";
        src += "    default: break;\n    }\n"
               "    flush_stats3(jobs, job, 0, 1, 2, completed, valid, visits);\n}\n";
    }
    for (size_t j = 0; j < jobs.size(); ++j) {
        if (jobs[j].levels.empty()) continue;
        const std::string js = std::to_string(j), T = "J" + js;
        src += "extern \"C\" __global__ void __launch_bounds__(256) fs_jit_lv_" + js +
               "(const JobDev* __restrict__ jobs, int level, int a_prev, int a_next, const Entry* __restrict__ src, "
               "Entry* __restrict__ dst, u64 n, int last)\n{\n"
               "    FS_GRID_DEP();\n"
               "    const JobDev& J = jobs[" + js + "];\n    u64 visits = 0, entries = 0, bcuts = 0;\n"
               "    for (u64 base = (u64)blockIdx.x * blockDim.x; base < n; base += (u64)gridDim.x * blockDim.x) {\n"
               "        const u64 idx = base + threadIdx.x;\n"
               "        bool live = false;\n"
               "        if (idx < n) {\n"
               "        u32 st[" + T + "::W], bin[" + T + "::W];\n        double2 a;\n"
               "        live = lv_load<" + T + ">(J, a_prev, a_next, src, idx, st, bin, a);\n"
               "        if (live) {\n            const u64 h = (idx & ((1ull << a_next) - 1ull)) << (" + T + "::Ap - a_next);\n"
               "            int r = -1;\n            switch (level) {\n";
        for (size_t k = 0; k < jobs[j].levels.size(); ++k)
            src += "            case " + std::to_string(k) + ": r = " + T + "::lv" + std::to_string(k) + "(st, a, h, bin, visits); break;\n";
        src += "            default: break;\n            }\n            live = r < 0;\n        }\n"
               "        if (live && last) ++entries;\n"
               "        if (" + T + "::BOUND && last && live && " + T + "::bound_cut(st, bin)) { live = false; ++bcuts; }\n"
               "        lv_store<" + T + ">(dst, idx, st, a, live);\n"
               "        }\n";
        // every lane of the warp reaches the one count (its ballot is warp-wide)
        if (jobs[j].bound && jobs[j].bound_counts)
            src += "        if (last) count_live(J, idx, live, true);\n";
        src += "    }\n"
               "    flush_stats3(jobs, " + js + ", 4, 3, 8, visits, entries, bcuts);\n}\n";
    }
    bool any_count = false;
    for (const JitJobSpec& J : jobs) any_count |= J.bound && J.bound_counts && J.levels.empty();
    src += "extern \"C\" __global__ void __launch_bounds__(256) fs_jit_prefix(const JobDev* __restrict__ jobs, "
           "const u64* __restrict__ begin, int n_jobs, u64 total)\n{\n"
           "    FS_GRID_DEP();\n"
           "    u64 dv = 0, den = 0, dbc = 0;\n    int cj = -1;\n"
           "    for (u64 idx = (u64)blockIdx.x * blockDim.x + threadIdx.x; ; idx += (u64)gridDim.x * blockDim.x) {\n"
           "        if (!__any_sync(0xffffffffu, idx < total)) break;\n"
           "        u64 visits = 0, entries = 0, bcuts = 0, local = 0;\n        int j = 0;\n"
           "        bool live = false, counts = false;\n"
           "        if (idx < total) {\n            j = find_job(begin, n_jobs, idx);\n"
           "            local = idx - jobs[j].prefix_begin;\n            switch (j) {\n";
    for (size_t j = 0; j < jobs.size(); ++j)
        src += "            case " + std::to_string(j) + ": live = prefix_body<J" + std::to_string(j) + ">(jobs[" +
               std::to_string(j) + "], local, visits, entries, bcuts); counts = J" + std::to_string(j) +
               "::COUNTB; break;\n";
    src += "            default: break;\n            }\n        }\n"
           "        const unsigned act = __ballot_sync(0xffffffffu, idx < total);\n"
           "        const unsigned same = __match_any_sync(0xffffffffu, idx < total ? j : -1);\n"
           "        const bool uniform = act == 0xffffffffu && same == 0xffffffffu;\n";
    if (any_count)
        src += "        if (__any_sync(0xffffffffu, counts)) count_live(jobs[j], local, live && counts, uniform && counts);\n";
    // a warp whose lanes all ran entries of its first job keeps those
    // counts for the block-wide flush at the end; other iterations add
    // theirs as they go
    src += "        if (uniform && (cj < 0 || j == cj)) {\n"
           "            cj = j;\n            dv += visits;\n            den += entries;\n            dbc += bcuts;\n"
           "        } else if (uniform) {\n"
           "            const u64 v = warp_sum_u64(visits), en = warp_sum_u64(entries), bc = warp_sum_u64(bcuts);\n"
           "            if ((threadIdx.x & 31) == 0) { atomicAdd(&jobs[j].stats[4], v); atomicAdd(&jobs[j].stats[3], en);\n"
           "                                           if (bc) atomicAdd(&jobs[j].stats[8], bc); }\n"
           "        } else if (idx < total) {\n"
           "            if (visits) atomicAdd(&jobs[j].stats[4], visits);\n"
           "            if (entries) atomicAdd(&jobs[j].stats[3], entries);\n"
           "            if (bcuts) atomicAdd(&jobs[j].stats[8], bcuts);\n"
           "        }\n    }\n"
           "    flush_stats3(jobs, cj, 4, 3, 8, dv, den, dbc);\n}\n";
    return src;
}

struct JitModule {
    std::vector<cudaKernel_t> lv;     // per job: level kernel (nullptr when the job has no levels)
    cudaLibrary_t lib = nullptr;
    cudaKernel_t kernel = nullptr;
    cudaKernel_t prefix = nullptr;
    cudaKernel_t compact = nullptr;
    cudaKernel_t walk = nullptr;      // level-by-level suffix walk (threshold jobs)
    std::vector<int> walk_warps;      // per job: warps per block of the walk (0: not walked)
    std::vector<int> walk_grid;       // per job: blocks of the walk
    std::vector<size_t> walk_smem;    // per job: shared memory per block of the walk
    int compact_grid = 0;
    int grid = 0;
    int sms = 148;
};

// Shared memory of the walk: per warp, As x 40 queued histories (the
// device's WALK_CAP) of 16 B (amplitude) plus 4 W bytes (state); warps per
// block such that a block takes at most 220 KB (the SM's shared memory), at
// most 8 warps.
constexpr size_t WALK_BLOCK_BYTES = 220 * 1024;
size_t walk_bytes_per_warp(const JitJobSpec& J) { return (size_t)J.As * 40u * (16u + 4u * (size_t)J.W); }

}  // namespace

bool phase_index(double2 A, double2 B, uint32_t* p)
{
    if (A.x != 1.0 || A.y != 0.0) return false;
    const long double re = B.x, im = B.y;
    if (fabsl(re * re + im * im - 1.0L) > 1e-12L) return false;
    const long double two_pi = 6.283185307179586476925286766559005768L;
    long double t = atan2l(im, re) / two_pi * 65536.0L;
    if (t < 0) t += 65536.0L;
    const long double r = roundl(t);
    if (fabsl(t - r) > 1e-6L) return false;
    const uint32_t q = (uint32_t)r & 0xffffu;
    if (q == 0u) return false;
    *p = q;
    return true;
}

bool jit_census(const JitJobSpec& J)
{
    if (J.eps2 != 0.0 || J.As < 4 || J.As > 30) return false;
    std::string g, f;
    std::complex<long double> h(1.0L, 0.0L);
    int ok1 = 1, ok2 = 1, sc = 1;
    PhaseAcc* keep = t_phase;
    t_phase = nullptr;
    emit_region(f, g, "x", J, J.c2, J.G, J.As, true, &h, false, false, nullptr, &ok1);
    if (stacked_suffix(J)) emit_region(f, g, "y", J, J.c2, J.G, J.As, true, &h, true, false, &sc, &ok2);
    t_phase = keep;
    return ok1 && ok2;
}

std::string jit_source(const std::vector<JitJobSpec>& jobs)
{
    std::vector<double2> scales(jobs.size());
    return generate(jobs, &scales);
}

int jit_build(const std::vector<JitJobSpec>& jobs, void** handle, std::string* err, double* compile_ms,
              std::string* source_out, std::vector<double2>* scales)
{
    const auto t0 = std::chrono::steady_clock::now();
    if (scales) scales->assign(jobs.size(), make_double2(1.0, 0.0));
    const std::string src = generate(jobs, scales);
    if (source_out) *source_out = src;
    if (compile_ms) *compile_ms = 0;
    nvrtcProgram prog;
    if (nvrtcCreateProgram(&prog, src.c_str(), "fs_jit.cu", 0, nullptr, nullptr) != NVRTC_SUCCESS) {
        *err = "nvrtcCreateProgram failed";
        return -1;
    }
    const char* opts[] = {"--gpu-architecture=sm_103a", "-std=c++17", "-default-device", "-lineinfo"};
    const nvrtcResult rc = nvrtcCompileProgram(prog, 4, opts);
    if (rc != NVRTC_SUCCESS) {
        size_t n = 0;
        nvrtcGetProgramLogSize(prog, &n);
        std::string log(n, '\0');
        nvrtcGetProgramLog(prog, &log[0]);
        *err = std::string("NVRTC: ") + nvrtcGetErrorString(rc) + "\n" + log.substr(0, 2000);
        nvrtcDestroyProgram(&prog);
        return -1;
    }
    size_t n = 0;
    nvrtcGetCUBINSize(prog, &n);
    std::vector<char> cubin(n);
    nvrtcGetCUBIN(prog, cubin.data());
    nvrtcDestroyProgram(&prog);
    if (compile_ms)
        *compile_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    JitModule* m = new JitModule;
    cudaError_t e = cudaLibraryLoadData(&m->lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
    if (e == cudaSuccess) e = cudaLibraryGetKernel(&m->kernel, m->lib, "fs_jit_history");
    if (e == cudaSuccess) e = cudaLibraryGetKernel(&m->prefix, m->lib, "fs_jit_prefix");
    if (e == cudaSuccess) e = cudaLibraryGetKernel(&m->compact, m->lib, "fs_jit_compact");
    m->lv.assign(jobs.size(), nullptr);
    for (size_t j = 0; j < jobs.size() && e == cudaSuccess; ++j)
        if (!jobs[j].levels.empty())
            e = cudaLibraryGetKernel(&m->lv[j], m->lib, ("fs_jit_lv_" + std::to_string(j)).c_str());
    if (e != cudaSuccess) {
        *err = std::string("loading the generated kernel (compiled in ") +
               std::to_string(compile_ms ? *compile_ms : 0.0) + " ms): " + cudaGetErrorString(e);
        if (m->lib) cudaLibraryUnload(m->lib);
        delete m;
        return -2;
    }
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)m->kernel, TILE, 0);
    m->grid = (sms > 0 ? sms : 148) * (per_sm > 0 ? per_sm : 1);
    m->sms = sms > 0 ? sms : 148;
    per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)m->compact, TILE, 0);
    m->compact_grid = m->sms * (per_sm > 0 ? per_sm : 1);
    m->walk_warps.assign(jobs.size(), 0);
    m->walk_grid.assign(jobs.size(), 0);
    m->walk_smem.assign(jobs.size(), 0);
    size_t walk_max = 0;
    for (size_t j = 0; j < jobs.size() && e == cudaSuccess; ++j) {
        if (queue_last_source(jobs[j]) < 0) continue;
        if (!m->walk) e = cudaLibraryGetKernel(&m->walk, m->lib, "fs_jit_walk");
        const size_t pw = walk_bytes_per_warp(jobs[j]);
        size_t w = WALK_BLOCK_BYTES / pw;
        w = w < 1 ? 1 : (w > 8 ? 8 : w);
        m->walk_warps[j] = (int)w;
        m->walk_smem[j] = w * pw;
        if (m->walk_smem[j] > walk_max) walk_max = m->walk_smem[j];
    }
    if (e == cudaSuccess && m->walk)
        e = cudaFuncSetAttribute((const void*)m->walk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)walk_max);
    for (size_t j = 0; j < jobs.size() && e == cudaSuccess; ++j) {
        if (!m->walk_warps[j]) continue;
        per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)m->walk, 32 * m->walk_warps[j],
                                                          m->walk_smem[j]);
        m->walk_grid[j] = m->sms * (per_sm > 0 ? per_sm : 1);
    }
    if (e != cudaSuccess) {
        *err = std::string("preparing the suffix walk kernel: ") + cudaGetErrorString(e);
        cudaLibraryUnload(m->lib);
        delete m;
        return -2;
    }
    *handle = m;
    return 0;
}

cudaError_t jit_launch_history(void* handle, const JobDev* d_jobs, const uint2* d_tiles, uint64_t n_tiles,
                               unsigned int* d_counter, cudaStream_t s)
{
    if (n_tiles == 0) return cudaSuccess;
    JitModule* m = (JitModule*)handle;
    int grid = m->grid;
    if ((uint64_t)grid > n_tiles) grid = (int)n_tiles;
    void* args[] = {(void*)&d_jobs, (void*)&d_tiles, (void*)&n_tiles, (void*)&d_counter};
    return launch_ex((const void*)m->kernel, dim3(grid), dim3(TILE), 0, s, args);
}

cudaError_t jit_launch_prefix(void* handle, const JobDev* d_jobs, const uint64_t* d_begin, int n_jobs,
                              uint64_t total, cudaStream_t s)
{
    if (total == 0) return cudaSuccess;
    JitModule* m = (JitModule*)handle;
    uint64_t blocks = (total + 255) / 256;
    if (blocks > (uint64_t)m->sms * 64) blocks = (uint64_t)m->sms * 64;
    void* args[] = {(void*)&d_jobs, (void*)&d_begin, (void*)&n_jobs, (void*)&total};
    return launch_ex((const void*)m->prefix, dim3((unsigned)blocks), dim3(256), 0, s, args);
}

cudaError_t jit_launch_prefix_level(void* handle, const JobDev* d_jobs, int job, int level, const PrefixLevel& L,
                                    const Entry* src, Entry* dst, uint64_t n_dst, bool last, cudaStream_t s)
{
    if (n_dst == 0) return cudaSuccess;
    JitModule* m = (JitModule*)handle;
    if (job < 0 || job >= (int)m->lv.size() || !m->lv[job]) return cudaErrorInvalidValue;
    uint64_t blocks = (n_dst + 255) / 256;
    if (blocks > (uint64_t)m->sms * 64) blocks = (uint64_t)m->sms * 64;
    int a_prev = L.a_prev, a_next = L.a_next, lst = last ? 1 : 0;
    void* args[] = {(void*)&d_jobs, (void*)&level, (void*)&a_prev, (void*)&a_next, (void*)&src, (void*)&dst,
                    (void*)&n_dst, (void*)&lst};
    return launch_ex((const void*)m->lv[job], dim3((unsigned)blocks), dim3(TILE), 0, s, args);
}

cudaError_t jit_launch_compact(void* handle, const JobDev* d_jobs, int job, double2* d_amp, cudaStream_t s)
{
    JitModule* m = (JitModule*)handle;
    void* args[] = {(void*)&d_jobs, (void*)&job, (void*)&d_amp};
    if (job >= 0 && job < (int)m->walk_warps.size() && m->walk_warps[job])
        return launch_ex((const void*)m->walk, dim3(m->walk_grid[job]), dim3(32 * m->walk_warps[job]),
                         m->walk_smem[job], s, args);
    return launch_ex((const void*)m->compact, dim3(m->compact_grid), dim3(TILE), 0, s, args);
}

void jit_release(void* handle)
{
    JitModule* m = (JitModule*)handle;
    if (!m) return;
    if (m->lib) cudaLibraryUnload(m->lib);
    delete m;
}

}  // namespace fs

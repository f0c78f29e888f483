// CUDA kernels of the reduced-history path (sm_103a).
//
//   prefix_kernel   -- Algorithm 2, prefix region: for every (pair, h_p) walk
//                      the output-side gates backward from b_out and write the
//                      checkpoint (sigma_p, beta_p) into the table.
//   history_kernel  -- Algorithm 2, root and suffix regions: a persistent
//                      kernel pulls 256-item tiles off an atomic queue (the
//                      device form of the server-worker balancer, Sec. IV-D);
//                      each thread advances one (h_p, h_r) checkpoint through
//                      the root and loops h_s over the suffix, checks chi at
//                      the input boundary and accumulates beta_s.
//   reduce_kernel   -- fixed-order sums of the per-tile partials and of the
//                      sparse-input terms (Eq. 2) into the amplitudes.
//
// All arithmetic on amplitudes is FP64.  The complex product is
// re = fma(a.re, b.re, -(a.im b.im)), im = fma(a.re, b.im, a.im b.re) with
// explicit round-to-nearest intrinsics, so every history's amplitude is the
// same double the host-side definition gives when it multiplies the same
// factors in the same (backward) order.
#include <cstdlib>
#include "fs_internal.h"

namespace fs {

namespace {

constexpr double RSQRT2 = 0.70710678118654757;   // sqrt(0.5) rounded to nearest

__device__ __forceinline__ double2 cmul(double2 a, double2 b)
{
    return make_double2(__fma_rn(a.x, b.x, -__dmul_rn(a.y, b.y)),
                        __fma_rn(a.x, b.y, __dmul_rn(a.y, b.x)));
}

// Sign flip on the integer pipe (exact).
__device__ __forceinline__ double dneg(double x)
{
    return __hiloint2double(__double2hiint(x) ^ 0x80000000, __double2loint(x));
}

__device__ __forceinline__ double2 ldf(const double2* p)
{
    return __ldg(p);
}

// (output, input) of a pair index, pair = o * S + s.  Integer division by a
// runtime value goes through the scarce FP64 pipe on this part, so the
// quotient comes from the job's precomputed multiplier (division by an
// invariant integer, Granlund and Montgomery 1994, Fig. 4.1) for pair
// indices below 2^32.
__device__ __forceinline__ uint64_t pair_split(uint64_t pair, const JobDev& J, uint64_t& s)
{
    const uint32_t S = (uint32_t)J.S;
    if (S == 1u) { s = 0; return pair; }
    if (pair < (1ull << 32)) {
        const uint32_t p = (uint32_t)pair, t = __umulhi(J.s_magic, p);
        const uint32_t o = (t + ((p - t) >> 1)) >> (J.s_shift - 1);
        s = p - o * S;
        return o;
    }
    const uint64_t o = pair / S;
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

// A logged item's sum times the job's constant, out of line: inlined, the
// product would be if-converted into FP64 instructions that every item of a
// run without logging issues with no lane active.
__device__ __noinline__ void fs_log_ool(double2* dst, double2 scale, double2 v) { *dst = cmul(scale, v); }

// The FP64 adds of add_kept, out of line: a call that no lane makes issues
// none of the callee's instructions, where an inlined add would be
// if-converted into FP64 instructions predicated off in every lane -- and
// those still occupy the scarce FP64 pipe of this part.
__device__ __noinline__ double2 fs_add_ool(double2 a, double2 b)
{
    return make_double2(__dadd_rn(a.x, b.x), __dadd_rn(a.y, b.y));
}

// acc += v in the lanes where keep holds.  Most leaves are invalid and most
// items zero, so the adds run only when some active lane keeps its value.
__device__ __forceinline__ void add_kept(double2& acc, double2 v, bool keep)
{
    if (__any_sync(__activemask(), keep)) {
        const double2 t = fs_add_ool(acc, v);
        if (keep) acc = t;
    }
}


// A bottom entry (its prefix met an exactly zero factor) carries a NaN real
// part; tested on the bits (a double compare would use the FP64 pipe).
__device__ __forceinline__ bool is_bottom(double x)
{
    const unsigned hi = (unsigned)__double2hiint(x) & 0x7fffffffu;
    return hi > 0x7ff00000u || (hi == 0x7ff00000u && (unsigned)__double2loint(x) != 0u);
}

template <int W>
__device__ __forceinline__ uint32_t word_of(const uint32_t (&st)[W], uint32_t q)
{
    uint32_t v = st[0];
#pragma unroll
    for (int j = 1; j < W; ++j) v = ((q >> 5) == (uint32_t)j) ? st[j] : v;
    return v;
}

template <int W>
__device__ __forceinline__ uint32_t getbit(const uint32_t (&st)[W], uint32_t q)
{
    return (word_of<W>(st, q) >> (q & 31)) & 1u;
}

template <int W>
__device__ __forceinline__ void xorbit(uint32_t (&st)[W], uint32_t q, uint32_t v)
{
    const uint32_t m = v << (q & 31);
#pragma unroll
    for (int j = 0; j < W; ++j) st[j] ^= ((q >> 5) == (uint32_t)j) ? m : 0u;
}

template <int W>
__device__ __forceinline__ bool match(const uint32_t (&st)[W], const uint32_t* __restrict__ m)
{
    uint32_t d = 0;
#pragma unroll
    for (int j = 0; j < W; ++j) d |= (st[j] & __ldg(m + j)) ^ __ldg(m + W + j);
    return d == 0;
}

template <int W>
__device__ __forceinline__ bool same(const uint32_t (&a)[W], const uint32_t (&b)[W])
{
    uint32_t d = 0;
#pragma unroll
    for (int j = 0; j < W; ++j) d |= a[j] ^ b[j];
    return d == 0;
}

// Evaluates the ops at evaluation positions [e0, e1) (one region of
// Algorithm 2, i.e. AdvanceCheckpoint).  h is the region's enumeration word
// (the op's s0/s1 give the bit of each artificial source), bin the input bit
// string (natural sources and the chi test).  Returns -1 when the region
// completes; otherwise the history is cut (bottom: an exactly zero factor,
// or |beta| < eps right after an artificial source) and the return value is
// the lowest h bit assigned so far (nbits if none), so that every h sharing
// the bits at and above it is known to be cut too.
template <int W>
__device__ int run_ops(const JobDev& J, int e0, int e1, uint32_t (&st)[W], double2& amp,
                       uint64_t h, int nbits, const uint32_t (&bin)[W],
                       unsigned long long& visits, uint32_t* err)
{
    int low = nbits;
    const uint4* __restrict__ ops = reinterpret_cast<const uint4*>(J.ops);
    const double2* __restrict__ fac = J.fac;
    const uint32_t* __restrict__ masks = J.masks;
    for (int e = e0; e < e1; ++e) {
        const uint4 raw = __ldg(ops + e);
        const uint32_t code = raw.x & 0xFFu;
        const uint32_t q0 = (raw.x >> 8) & 0xFFu;
        const uint32_t q1 = (raw.x >> 16) & 0xFFu;
        const int s0 = (int)(int8_t)(raw.y & 0xFFu);
        const int s1 = (int)(int8_t)((raw.y >> 8) & 0xFFu);
        const uint32_t aux = raw.z, aux2 = raw.w;
        bool srcop = false, zero = false;
        switch (code) {
        case OP_X:
            xorbit<W>(st, q0, 1u);
            break;
        case OP_MCX:
            if (match<W>(st, masks + aux2)) xorbit<W>(st, q0, 1u);
            break;
        case OP_SWAP: {
            const uint32_t d = getbit<W>(st, q0) ^ getbit<W>(st, q1);
            xorbit<W>(st, q0, d);
            xorbit<W>(st, q1, d);
            break;
        }
        case OP_PERM1: {
            const uint32_t o = getbit<W>(st, q0);
            amp = cmul(amp, ldf(fac + aux + o));
            xorbit<W>(st, q0, 1u);
            break;
        }
        case OP_PERM2: {
            const uint32_t o = getbit<W>(st, q0) | (getbit<W>(st, q1) << 1);
            const uint32_t i = (aux2 >> (2 * o)) & 3u;
            amp = cmul(amp, ldf(fac + aux + o));
            xorbit<W>(st, q0, (o ^ i) & 1u);
            xorbit<W>(st, q1, ((o ^ i) >> 1) & 1u);
            break;
        }
        case OP_DIAG1:
            amp = cmul(amp, ldf(fac + aux + getbit<W>(st, q0)));
            break;
        case OP_PH1:
            if (getbit<W>(st, q0)) amp = cmul(amp, ldf(fac + aux));
            break;
        case OP_NEG1:
            if (getbit<W>(st, q0)) amp = make_double2(dneg(amp.x), dneg(amp.y));
            break;
        case OP_MCPH:
            if (match<W>(st, masks + aux2)) amp = cmul(amp, ldf(fac + aux));
            break;
        case OP_MCNEG:
            if (match<W>(st, masks + aux2)) amp = make_double2(dneg(amp.x), dneg(amp.y));
            break;
        case OP_DIAG2:
            amp = cmul(amp, ldf(fac + aux + (getbit<W>(st, q0) | (getbit<W>(st, q1) << 1))));
            break;
        case OP_H: {
            const uint32_t o = getbit<W>(st, q0);
            uint32_t i;
            if (s0 >= 0) { i = (uint32_t)(h >> s0) & 1u; srcop = true; low = s0; }
            else i = getbit<W>(bin, q0);
            const double hv = (o & i) ? -RSQRT2 : RSQRT2;
            amp = make_double2(__dmul_rn(amp.x, hv), __dmul_rn(amp.y, hv));
            xorbit<W>(st, q0, o ^ i);
            break;
        }
        case OP_BR1: {
            const uint32_t o = getbit<W>(st, q0);
            uint32_t i;
            if (s0 >= 0) { i = (uint32_t)(h >> s0) & 1u; srcop = true; low = s0; }
            else i = getbit<W>(bin, q0);
            const double2 f = ldf(fac + aux + 2 * o + i);
            zero = (f.x == 0.0) & (f.y == 0.0);
            amp = cmul(amp, f);
            xorbit<W>(st, q0, o ^ i);
            break;
        }
        case OP_BR2: {
            const uint32_t o = getbit<W>(st, q0) | (getbit<W>(st, q1) << 1);
            uint32_t i0, i1;
            if (s0 >= 0) { i0 = (uint32_t)(h >> s0) & 1u; srcop = true; low = min(low, s0); }
            else i0 = getbit<W>(bin, q0);
            if (s1 >= 0) { i1 = (uint32_t)(h >> s1) & 1u; srcop = true; low = min(low, s1); }
            else i1 = getbit<W>(bin, q1);
            const uint32_t i = i0 | (i1 << 1);
            const double2 f = ldf(fac + aux + 4 * o + i);
            zero = (f.x == 0.0) & (f.y == 0.0);
            amp = cmul(amp, f);
            xorbit<W>(st, q0, (o ^ i) & 1u);
            xorbit<W>(st, q1, ((o ^ i) >> 1) & 1u);
            break;
        }
        default:
            atomicOr(err, DEV_ERR_BAD_OPCODE);
            zero = true;
            break;
        }
        const bool cut = zero ||
            (srcop && J.eps2 > 0.0 && __fma_rn(amp.x, amp.x, __dmul_rn(amp.y, amp.y)) < J.eps2);
        if (cut) {
            visits += (unsigned long long)(e - e0 + 1);
            return low;
        }
    }
    visits += (unsigned long long)(e1 - e0);
    return -1;
}

template <int W>
__device__ __forceinline__ void load_bits(const uint32_t* __restrict__ p, uint32_t (&st)[W])
{
    const uint4 v = __ldg(reinterpret_cast<const uint4*>(p));
    const uint32_t a[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int j = 0; j < W; ++j) st[j] = a[j];
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v)
{
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

__device__ __forceinline__ int find_job(const uint64_t* __restrict__ begin, int n_jobs, uint64_t idx)
{
    int lo = 0, hi = n_jobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(begin + mid) <= idx) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// ---------------------------------------------------------------- prefix

template <int W>
__device__ void prefix_one(const JobDev& J, uint64_t local, uint32_t* err,
                           unsigned long long& visits, unsigned long long& entries)
{
    const uint64_t pair = local >> J.Ap;
    const uint64_t hp = local & ((1ull << J.Ap) - 1ull);
    uint64_t s;
    const uint64_t o = pair_split(pair, J, s);
    uint32_t st[W], bin[W];
    load_bits<W>(J.outs + 4 * o, st);
    load_bits<W>(J.ins + 4 * s, bin);
    double2 amp = make_double2(1.0, 0.0);
    const int r = run_ops<W>(J, 0, J.c1, st, amp, hp, J.Ap, bin, visits, err);
    Entry e;
#pragma unroll
    for (int j = 0; j < 4; ++j) e.st[j] = j < W ? st[j] : 0u;
    e.amp = amp;
    if (r >= 0) e.amp.x = __longlong_as_double(0x7ff8000000000000ll);   // bottom
    else entries += 1;
    uint4* dst = reinterpret_cast<uint4*>(J.table + local);
    dst[0] = make_uint4(e.st[0], e.st[1], e.st[2], e.st[3]);
    reinterpret_cast<double2*>(dst + 1)[0] = e.amp;
}

__global__ void __launch_bounds__(256) prefix_kernel(const JobDev* __restrict__ jobs,
                                                     const uint64_t* __restrict__ begin, int n_jobs,
                                                     uint64_t total, uint32_t* err)
{
    FS_GRID_DEP();
    for (uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; ; idx += (uint64_t)gridDim.x * blockDim.x) {
        const bool any = __any_sync(0xffffffffu, idx < total);
        if (!any) break;
        unsigned long long visits = 0, entries = 0;
        int j = 0;
        if (idx < total) {
            j = find_job(begin, n_jobs, idx);
            const JobDev& J = jobs[j];
            const uint64_t local = idx - J.prefix_begin;
            if (J.W == 1) prefix_one<1>(J, local, err, visits, entries);
            else if (J.W == 2) prefix_one<2>(J, local, err, visits, entries);
            else prefix_one<4>(J, local, err, visits, entries);
        }
        // counter flush: one atomic per warp when the warp lies in one job,
        // otherwise one per lane
        const unsigned act = __ballot_sync(0xffffffffu, idx < total);
        const unsigned same_job = __match_any_sync(0xffffffffu, idx < total ? j : -1);
        if (act == 0xffffffffu && same_job == 0xffffffffu) {
            const unsigned long long v = warp_sum_u64(visits), en = warp_sum_u64(entries);
            if ((threadIdx.x & 31) == 0) {
                atomicAdd(&jobs[j].stats[4], v);
                atomicAdd(&jobs[j].stats[3], en);
            }
        } else if (idx < total) {
            if (visits) atomicAdd(&jobs[j].stats[4], visits);
            if (entries) atomicAdd(&jobs[j].stats[3], entries);
        }
    }
}

// One level of the per-source prefix expansion: thread per entry of the
// next level; the entry's parent is the previous level's entry with the same
// leading source bits (or b_out at the first level).
template <int W>
__device__ void prefix_level_one(const JobDev& J, const PrefixLevel& L, const Entry* __restrict__ src,
                                 Entry* __restrict__ dst, uint64_t idx, bool last, uint32_t* err,
                                 unsigned long long& visits, unsigned long long& entries)
{
    const uint64_t pair = idx >> L.a_next;
    const uint64_t child = idx & ((1ull << L.a_next) - 1ull);
    uint64_t s;
    const uint64_t o = pair_split(pair, J, s);
    uint32_t st[W], bin[W];
    load_bits<W>(J.ins + 4 * s, bin);
    double2 amp = make_double2(1.0, 0.0);
    bool live = true;
    if (!src) {
        load_bits<W>(J.outs + 4 * o, st);
    } else {
        const uint64_t parent = (pair << L.a_prev) + (child >> (L.a_next - L.a_prev));
        const uint4* ent = reinterpret_cast<const uint4*>(src + parent);
        const uint4 sv = ent[0];
        amp = reinterpret_cast<const double2*>(ent + 1)[0];
        const uint32_t tmp[4] = {sv.x, sv.y, sv.z, sv.w};
#pragma unroll
        for (int j = 0; j < W; ++j) st[j] = tmp[j];
        live = !is_bottom(amp.x);
    }
    if (live) {
        const uint64_t h = child << (J.Ap - L.a_next);
        live = run_ops<W>(J, L.e0, L.e1, st, amp, h, J.Ap, bin, visits, err) < 0;
    }
    uint32_t w[4] = {0u, 0u, 0u, 0u};
#pragma unroll
    for (int j = 0; j < W; ++j) w[j] = st[j];
    if (!live) amp.x = __longlong_as_double(0x7ff8000000000000ll);
    else if (last) entries += 1;
    uint4* d = reinterpret_cast<uint4*>(dst + idx);
    d[0] = make_uint4(w[0], w[1], w[2], w[3]);
    reinterpret_cast<double2*>(d + 1)[0] = amp;
}

__global__ void __launch_bounds__(256) prefix_level_kernel(const JobDev* __restrict__ jobp, PrefixLevel L,
                                                           const Entry* __restrict__ src, Entry* __restrict__ dst,
                                                           uint64_t n, int last, uint32_t* err)
{
    FS_GRID_DEP();
    const JobDev& J = *jobp;
    unsigned long long visits = 0, entries = 0;
    for (uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += (uint64_t)gridDim.x * blockDim.x) {
        if (J.W == 1) prefix_level_one<1>(J, L, src, dst, idx, last != 0, err, visits, entries);
        else if (J.W == 2) prefix_level_one<2>(J, L, src, dst, idx, last != 0, err, visits, entries);
        else prefix_level_one<4>(J, L, src, dst, idx, last != 0, err, visits, entries);
    }
    visits = warp_sum_u64(visits);
    entries = warp_sum_u64(entries);
    if ((threadIdx.x & 31) == 0) {
        if (visits) atomicAdd(&J.stats[4], visits);
        if (entries) atomicAdd(&J.stats[3], entries);
    }
}

// ---------------------------------------------------------------- history

// Per-output leaf counts of a traced job: one item's completed and valid
// leaves added to its output's counters.
__device__ __forceinline__ void trace_counts(const JobDev& J, uint64_t pair, unsigned long long dc,
                                             unsigned long long dv)
{
    if (!(dc | dv)) return;
    uint64_t s;
    const uint64_t o = pair_split(pair, J, s);
    if (dc) atomicAdd(&J.trace[2 * o], dc);
    if (dv) atomicAdd(&J.trace[2 * o + 1], dv);
}

// Sum over the valid leaves of one (prefix, root) item: the root once, the
// suffix for every h_s (skipping cut subtrees), the chi test at the input.
template <int W>
__device__ double2 history_item(const JobDev& J, uint64_t item, uint32_t* err, unsigned long long& completed,
                                unsigned long long& valid, unsigned long long& visits)
{
    double2 acc = make_double2(0.0, 0.0);
    const uint64_t pair = item >> J.log2_ipp;
    const uint64_t local = item & ((1ull << J.log2_ipp) - 1ull);
    const uint64_t hp = local >> J.Ar;
    const uint64_t hr = local & ((1ull << J.Ar) - 1ull);
    uint64_t s;
    const uint64_t o = pair_split(pair, J, s);
    uint4 sv;
    double2 a0 = make_double2(1.0, 0.0);
    if (J.table) {
        const uint4* ent = reinterpret_cast<const uint4*>(J.table + (pair << J.Ap) + hp);
        sv = __ldg(ent);
        a0 = __ldg(reinterpret_cast<const double2*>(ent + 1));
        if (is_bottom(a0.x)) return acc;
    } else {
        // an empty prefix region: the entry is (b_out, 1)
        sv = __ldg(reinterpret_cast<const uint4*>(J.outs + 4 * o));
    }
    uint32_t st[W], bin[W];
    const uint32_t tmp[4] = {sv.x, sv.y, sv.z, sv.w};
#pragma unroll
    for (int j = 0; j < W; ++j) st[j] = tmp[j];
    load_bits<W>(J.ins + 4 * s, bin);
    double2 amp = a0;
    const unsigned long long c0 = completed, v0 = valid;
    if (run_ops<W>(J, J.c1, J.c2, st, amp, hr, J.Ar, bin, visits, err) < 0) {
        const uint64_t ns = 1ull << J.As;
        uint64_t hs = 0;
        while (hs < ns) {
            uint32_t st2[W];
#pragma unroll
            for (int j = 0; j < W; ++j) st2[j] = st[j];
            double2 amp2 = amp;
            const int r2 = run_ops<W>(J, J.c2, J.G, st2, amp2, hs, J.As, bin, visits, err);
            if (r2 < 0) {
                ++completed;
                {
                    const bool ok = same<W>(st2, bin);
                    valid += ok ? 1u : 0u;
                    add_kept(acc, amp2, ok);
                }
                ++hs;
            } else {
                hs = ((hs >> r2) + 1ull) << r2;
            }
        }
    }
    if (J.trace) trace_counts(J, pair, completed - c0, valid - v0);
    return acc;
}

// One 256-item tile on one warp: lane L takes items 8L .. 8L+7 in order and
// sums them per pair segment; segments of at least 8 items are then added
// across lanes (group_sum) into one partial per (pair, 256-item block).  The
// same order as the generated engine, so the two agree bit for bit whenever
// both multiply the same factors.
template <int W>
__device__ void history_tile(const JobDev& J, uint64_t tile, uint32_t* err)
{
    const int lane = threadIdx.x & 31;
    const uint64_t n_items = J.n_pairs << J.log2_ipp;
    const int lg = J.log2_ipp;
    const uint64_t first = tile * TILE + (uint64_t)lane * 8u;
    unsigned long long completed = 0, valid = 0, visits = 0;
    double2 acc = make_double2(0.0, 0.0);
#pragma unroll 1
    for (int k = 0; k < 8; ++k) {
        const uint64_t item = first + (uint64_t)k;
        if (item >= n_items) break;
        const double2 v = history_item<W>(J, item, err, completed, valid, visits);
        if (J.log) fs_log_ool(J.log + item, J.scale, v);   // logging runs only
        add_kept(acc, v, nonzero(v));
        if (lg < 3 && ((item + 1ull) & ((1ull << lg) - 1ull)) == 0ull) {
            J.partials[item >> lg] = acc;   // a pair of at most 4 items ends here
            acc = make_double2(0.0, 0.0);
        }
    }
    if (lg >= 3) {
        const int lps = lg >= 8 ? 32 : (1 << (lg - 3));   // lanes per pair segment
        acc = group_sum(acc, lps);
        if ((lane & (lps - 1)) == 0 && first < n_items) {
            const uint64_t p = first >> lg;
            const uint64_t l = first & ((1ull << lg) - 1ull);
            J.partials[(p << J.log2_spp) + (l >> TILE_LOG2)] = acc;
        }
    }
    completed = warp_sum_u64(completed);
    valid = warp_sum_u64(valid);
    visits = warp_sum_u64(visits);
    if (lane == 0 && (completed | valid | visits)) {
        atomicAdd(&J.stats[0], completed);
        atomicAdd(&J.stats[1], valid);
        atomicAdd(&J.stats[2], visits);
    }
}

// Persistent warps pull 256-item tiles off the queue with one atomicAdd each
// (the next index is fetched while the current tile runs).
__global__ void __launch_bounds__(TILE) history_kernel(const JobDev* __restrict__ jobs,
                                                       const uint2* __restrict__ tiles, uint64_t n_tiles,
                                                       unsigned int* counter, uint32_t* err)
{
    FS_GRID_DEP();
    const int lane = threadIdx.x & 31;
    unsigned int t = 0u, next = 0u;
    if (lane == 0) t = atomicAdd(counter, 1u);
    t = __shfl_sync(0xffffffffu, t, 0);
    while ((uint64_t)t < n_tiles) {
        if (lane == 0) next = atomicAdd(counter, 1u);
        const uint2 td = tiles[t];
        const JobDev& J = jobs[td.x];
        if (J.W == 1) history_tile<1>(J, td.y, err);
        else if (J.W == 2) history_tile<2>(J, td.y, err);
        else history_tile<4>(J, td.y, err);
        t = __shfl_sync(0xffffffffu, next, 0);
    }
}

// ---------------------------------------------------------------- compaction

// Live (non-bottom) checkpoint entries are compacted into a list in table
// order: count per block, exclusive scan of the block counts, write.
__device__ __forceinline__ bool entry_live(const JobDev& J, uint64_t e)
{
    return !is_bottom(reinterpret_cast<const double2*>(reinterpret_cast<const uint4*>(J.table + e) + 1)->x);
}

__global__ void __launch_bounds__(256) compact_count_kernel(const JobDev* __restrict__ jobp)
{
    FS_GRID_DEP();
    const JobDev& J = *jobp;
    const uint64_t base = (uint64_t)blockIdx.x * COMPACT_BLOCK;
    unsigned c = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const uint64_t e = base + (uint64_t)threadIdx.x * 4 + k;
        c += (e < J.n_entries && entry_live(J, e)) ? 1u : 0u;
    }
    c = __reduce_add_sync(0xffffffffu, c);
    __shared__ unsigned s_w[8];
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned t = 0;
        for (int w = 0; w < 8; ++w) t += s_w[w];
        J.blk[blockIdx.x] = t;
    }
}

__global__ void __launch_bounds__(1024) compact_scan_kernel(const JobDev* __restrict__ jobp, uint32_t nblk)
{
    FS_GRID_DEP();
    const JobDev& J = *jobp;
    __shared__ unsigned long long s_carry;
    __shared__ unsigned s_w[32];
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (uint32_t b0 = 0; b0 < nblk; b0 += 1024) {
        const uint32_t b = b0 + threadIdx.x;
        const unsigned v = b < nblk ? J.blk[b] : 0u;
        unsigned x = v;   // inclusive warp scan
        for (int off = 1; off < 32; off <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, x, off);
            if ((threadIdx.x & 31) >= (unsigned)off) x += y;
        }
        if ((threadIdx.x & 31) == 31) s_w[threadIdx.x >> 5] = x;
        __syncthreads();
        if (threadIdx.x < 32) {
            unsigned w = s_w[threadIdx.x];
            for (int off = 1; off < 32; off <<= 1) {
                const unsigned y = __shfl_up_sync(0xffffffffu, w, off);
                if (threadIdx.x >= (unsigned)off) w += y;
            }
            s_w[threadIdx.x] = w;   // inclusive scan of warp totals
        }
        __syncthreads();
        const unsigned warp_off = (threadIdx.x >> 5) ? s_w[(threadIdx.x >> 5) - 1] : 0u;
        const unsigned long long excl = s_carry + warp_off + x - v;
        if (b < nblk) J.blk[b] = (uint32_t)excl;
        __syncthreads();
        if (threadIdx.x == 1023) s_carry = excl + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) J.stats[6] = s_carry;
}

// One block per compaction block (see compact_block_write).
__global__ void __launch_bounds__(256) compact_write_kernel(const JobDev* __restrict__ jobp, int scanned)
{
    FS_GRID_DEP();
    compact_block_write(*jobp, blockIdx.x, gridDim.x, scanned, nullptr);
}

// History over the compacted live entries: items are (live entry, h_r)
// pairs, item i = (live index i >> A_r, h_r = i & (2^A_r - 1)); a warp takes
// 32 consecutive items off the job's work counter; each thread runs its root
// assignment and the suffix enumeration and writes the item's subtree sum
// (one slot per item: fixed reduction order downstream).
template <int W>
__device__ double2 compact_item(const JobDev& J, uint64_t i, uint32_t* err, unsigned long long& completed,
                                unsigned long long& valid, unsigned long long& visits)
{
    const uint64_t e = J.live[i >> J.Ar];
    const uint64_t hr = i & ((1ull << J.Ar) - 1ull);
    const uint64_t pair = e >> J.Ap;
    uint64_t s;
    const uint64_t o = pair_split(pair, J, s);
    const uint4* ent = reinterpret_cast<const uint4*>(J.table + e);
    const uint4 sv = __ldg(ent);
    double2 amp = __ldg(reinterpret_cast<const double2*>(ent + 1));
    if (is_bottom(amp.x)) return make_double2(0.0, 0.0);   // cut after the compaction
    uint32_t st[W], bin[W];
    const uint32_t tmp[4] = {sv.x, sv.y, sv.z, sv.w};
#pragma unroll
    for (int j = 0; j < W; ++j) st[j] = tmp[j];
    load_bits<W>(J.ins + 4 * s, bin);
    double2 acc = make_double2(0.0, 0.0);
    const unsigned long long c0 = completed, v0 = valid;
    if (run_ops<W>(J, J.c1, J.c2, st, amp, hr, J.Ar, bin, visits, err) < 0) {
        const uint64_t ns = 1ull << J.As;
        uint64_t hs = 0;
        while (hs < ns) {
            uint32_t st2[W];
#pragma unroll
            for (int j = 0; j < W; ++j) st2[j] = st[j];
            double2 amp2 = amp;
            const int r2 = run_ops<W>(J, J.c2, J.G, st2, amp2, hs, J.As, bin, visits, err);
            if (r2 < 0) {
                ++completed;
                {
                    const bool ok = same<W>(st2, bin);
                    valid += ok ? 1u : 0u;
                    add_kept(acc, amp2, ok);
                }
                ++hs;
            } else {
                hs = ((hs >> r2) + 1ull) << r2;
            }
        }
    }
    if (J.trace) trace_counts(J, pair, completed - c0, valid - v0);
    return acc;
}

// Subtree sums of one warp's 32 consecutive items: with A_r >= 5 they share a
// live entry and group_sum leaves one partial per warp (esum[i / 32]);
// otherwise each item keeps its own (esum[i]).
__device__ __forceinline__ void store_esum(const JobDev& J, uint64_t i, double2 acc, bool active)
{
    if (J.Ar >= 5) {
        acc = group_sum(acc, 32);
        if ((threadIdx.x & 31) == 0 && active) J.esum[i >> 5] = acc;
    } else if (active) {
        J.esum[i] = acc;
    }
}

__global__ void __launch_bounds__(256) history_compact_kernel(const JobDev* __restrict__ jobp, uint32_t* err)
{
    FS_GRID_DEP();
    const JobDev& J = *jobp;
    const uint64_t n_items = J.stats[6] << J.Ar;
    const int lane = threadIdx.x & 31;
    unsigned long long completed = 0, valid = 0, visits = 0;
    for (;;) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(&J.stats[7], 32ull);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base >= n_items) break;
        const uint64_t i = base + lane;
        double2 acc = make_double2(0.0, 0.0);
        if (i < n_items) {
            if (J.W == 1) acc = compact_item<1>(J, i, err, completed, valid, visits);
            else if (J.W == 2) acc = compact_item<2>(J, i, err, completed, valid, visits);
            else acc = compact_item<4>(J, i, err, completed, valid, visits);
        }
        store_esum(J, i, acc, i < n_items);
    }
    completed = warp_sum_u64(completed);
    valid = warp_sum_u64(valid);
    visits = warp_sum_u64(visits);
    if (lane == 0 && (completed | valid | visits)) {
        atomicAdd(&J.stats[0], completed);
        atomicAdd(&J.stats[1], valid);
        atomicAdd(&J.stats[2], visits);
    }
}


// ---------------------------------------------------------------- reduce

// Items of one (output, input) pair: the per-tile partials of an exact job,
// or the per-(live entry, h_r) subtree sums of a pruned job.
__device__ __forceinline__ const double2* pair_items(const JobDev& J, uint64_t pair, uint64_t& lo, uint64_t& hi)
{
    if (J.compact) {
        const int sh = J.Ar >= 5 ? J.Ar - 5 : J.Ar;   // partials per live entry: 2^(A_r - 5) or 2^A_r
        lo = J.prange[2 * pair] << sh;
        hi = J.prange[2 * pair + 1] << sh;
        return J.esum;
    }
    lo = pair << J.log2_spp;
    hi = lo + (1ull << J.log2_spp);
    return J.partials;
}

// src[k], src[k + stride], ... below hi: the i-th item goes to accumulator
// i mod 4, combined as (a0 + a1) + (a2 + a3); eight loads in flight.
__device__ __forceinline__ double2 strided_sum(const double2* __restrict__ src, uint64_t k, uint64_t hi,
                                               uint32_t stride)
{
    double2 a[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) a[u] = make_double2(0.0, 0.0);
    for (; k + 7 * (uint64_t)stride < hi; k += 8 * (uint64_t)stride) {
        double2 v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = src[k + (uint64_t)u * stride];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            a[u & 3].x += v[u].x;
            a[u & 3].y += v[u].y;
        }
    }
    // at most 7 items remain
#pragma unroll
    for (int u = 0; u < 7; ++u) {
        if (k < hi) {
            const double2 v = src[k];
            a[u & 3].x += v.x;
            a[u & 3].y += v.y;
        }
        k += stride;
    }
    return make_double2((a[0].x + a[1].x) + (a[2].x + a[3].x), (a[0].y + a[1].y) + (a[2].y + a[3].y));
}

// c_in * alpha summed over the pairs s = t, t + stride, ... of output o,
// each pair's items added in order (the thread's share of a wide input
// support, Eq. 2).
__device__ __forceinline__ double2 pairs_by_lane(const JobDev& J, uint64_t o, int t, int stride)
{
    double2 acc = make_double2(0.0, 0.0);
    for (int s = t; s < J.S; s += stride) {
        uint64_t lo, hi;
        const double2* src = pair_items(J, o * (uint64_t)J.S + (uint64_t)s, lo, hi);
        if (hi == lo) continue;
        double2 p = src[lo];
        for (uint64_t k = lo + 1; k < hi; ++k) {
            const double2 v = src[k];
            p.x += v.x;
            p.y += v.y;
        }
        const double2 w = cmul(__ldg(J.coef + s), p);
        acc.x += w.x;
        acc.y += w.y;
    }
    return acc;
}

constexpr int RED_LPO = 4;            // lanes per output in the common path
constexpr uint64_t RED_SMALL = 64;    // outputs with more items take the whole warp
constexpr uint64_t RED_WARP = RED_BIG_ITEMS;   // outputs with more items go to reduce_big_kernel

// FP64 is scarce on this part (about 2 FMA per clock per SM), so the
// reduction keeps FP64 instructions per output low: each warp takes 8
// outputs, 4 lanes each (lane-strided sums, a 2-level butterfly), then adds
// c_in * alpha over the input support in order (Eq. 2).  An output with more
// than RED_SMALL items is summed by the whole warp, one with more than
// RED_WARP items or an input support of RED_BIG_THREADS or more is listed
// for reduce_big_kernel.  The order of every sum depends
// only on the item counts, so results are run-to-run identical.
__global__ void __launch_bounds__(REDUCE_THREADS) reduce_kernel(const JobDev* __restrict__ jobs,
                                                                const uint64_t* __restrict__ begin,
                                                                int n_jobs, uint64_t total, double2* amp_out,
                                                                unsigned int* big_count, uint64_t* big_list)
{
    FS_GRID_DEP();
    constexpr int OPW = 32 / RED_LPO;
    const int lane = threadIdx.x & 31, sub = lane & (RED_LPO - 1), slot = lane / RED_LPO;
    const uint64_t warp = ((uint64_t)blockIdx.x * REDUCE_THREADS + threadIdx.x) >> 5;
    const uint64_t nwarp = ((uint64_t)gridDim.x * REDUCE_THREADS) >> 5;
    // a warp's 8 outputs are nwarp apart, so that runs of large outputs
    // (requests list the likely ones first) spread over warps
    for (uint64_t g0 = warp; g0 < total; g0 += nwarp * OPW) {
        const uint64_t g = g0 + (uint64_t)slot * nwarp;
        bool have = g < total;
        const int j = have ? find_job(begin, n_jobs, g) : 0;
        const JobDev& J = jobs[j];
        have = have && J.odone == nullptr;   // (a job with odone reduces its outputs in its history)
        const int S = have ? J.S : 0;
        const uint64_t o = have ? g - J.out_begin : 0;
        uint64_t n = 0;
        for (int s = 0; s < (S < RED_BIG_THREADS ? S : 0); ++s) {
            uint64_t lo, hi;
            pair_items(J, o * (uint64_t)S + (uint64_t)s, lo, hi);
            n += hi - lo;
        }
        // wide input supports (S >= 256) go to the block-per-output pass,
        // whose threads take the pairs in parallel
        const bool small = n <= RED_SMALL && S < 32;
        const bool big = n > RED_WARP || S >= RED_BIG_THREADS;
        const int s_max = (int)__reduce_max_sync(0xffffffffu, small ? (unsigned)S : 0u);
        double2 amp = make_double2(0.0, 0.0);
        for (int s = 0; s < s_max; ++s) {
            uint64_t lo = 0, hi = 0;
            const double2* src = nullptr;
            if (small && s < S) src = pair_items(J, o * (uint64_t)S + (uint64_t)s, lo, hi);
            const bool act = hi > lo;   // pairs with no items add exactly zero
            // FP64 instructions cost the same for every lane: skip them when
            // no pair of this warp has items
            if (!__any_sync(0xffffffffu, act)) continue;
            double2 t = make_double2(0.0, 0.0);
            if (act) t = strided_sum(src, lo + (uint64_t)sub, hi, RED_LPO);
#pragma unroll
            for (int off = RED_LPO / 2; off >= 1; off >>= 1) {
                t.x += __shfl_xor_sync(0xffffffffu, t.x, off);
                t.y += __shfl_xor_sync(0xffffffffu, t.y, off);
            }
            if (act) {
                const double2 w = cmul(__ldg(J.coef + s), t);
                amp.x += w.x;
                amp.y += w.y;
            }
        }
        // medium outputs: the whole warp, one output at a time (32-lane
        // stride, 5-level butterfly); larger ones go to reduce_big_kernel
        unsigned mid = __ballot_sync(0xffffffffu, have && !small && !big && sub == 0);
        while (mid) {
            const int b = __ffs(mid) - 1;
            mid &= mid - 1u;
            const uint64_t gb = __shfl_sync(0xffffffffu, g, b);
            const int jb = __shfl_sync(0xffffffffu, j, b);
            const JobDev& JB = jobs[jb];
            const uint64_t ob = gb - JB.out_begin;
            const uint64_t nb = __shfl_sync(0xffffffffu, n, b);
            double2 ab = make_double2(0.0, 0.0);
            if (JB.S >= 32 && nb <= 8u * (uint64_t)JB.S) {
                // a wide input support with few items per pair: lane l
                // takes the pairs s = l, l + 32, ... (c_in * alpha of each
                // added in order), then a 5-level butterfly
                ab = pairs_by_lane(JB, ob, lane, 32);
#pragma unroll
                for (int off = 16; off >= 1; off >>= 1) {
                    ab.x += __shfl_xor_sync(0xffffffffu, ab.x, off);
                    ab.y += __shfl_xor_sync(0xffffffffu, ab.y, off);
                }
            } else {
                for (int s = 0; s < JB.S; ++s) {
                    uint64_t lo, hi;
                    const double2* src = pair_items(JB, ob * (uint64_t)JB.S + (uint64_t)s, lo, hi);
                    if (hi == lo) continue;   // warp-uniform: the same pair for every lane
                    double2 t = strided_sum(src, lo + (uint64_t)lane, hi, 32);
#pragma unroll
                    for (int off = 16; off >= 1; off >>= 1) {
                        t.x += __shfl_xor_sync(0xffffffffu, t.x, off);
                        t.y += __shfl_xor_sync(0xffffffffu, t.y, off);
                    }
                    const double2 w = cmul(__ldg(JB.coef + s), t);
                    ab.x += w.x;
                    ab.y += w.y;
                }
            }
            if (lane == b) amp_out[gb] = ab;
        }
        if (have && sub == 0) {
            if (small) amp_out[g] = amp;
            else if (big) big_list[atomicAdd(big_count, 1u)] = g;
        }
    }
}

// One block per listed output: block-strided sums (eight loads in flight per
// thread), a butterfly per warp, the warps added in order, then c_in * alpha
// over the input support in order.
__global__ void __launch_bounds__(RED_BIG_THREADS) reduce_big_kernel(const JobDev* __restrict__ jobs,
                                                                     const uint64_t* __restrict__ begin, int n_jobs,
                                                                     const unsigned int* big_count,
                                                                     const uint64_t* __restrict__ big_list,
                                                                     double2* amp_out)
{
    FS_GRID_DEP();
    __shared__ double2 s_w[RED_BIG_THREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned int count = *big_count;
    for (unsigned int i = blockIdx.x; i < count; i += gridDim.x) {
        const uint64_t g = big_list[i];
        const JobDev& J = jobs[find_job(begin, n_jobs, g)];
        const uint64_t o = g - J.out_begin;
        double2 amp = make_double2(0.0, 0.0);
        if (J.S >= RED_BIG_THREADS) {
            // a wide input support: thread t takes the pairs s = t, t + 256,
            // ...; then a butterfly per warp and the warps added in order
            double2 t = pairs_by_lane(J, o, threadIdx.x, RED_BIG_THREADS);
#pragma unroll
            for (int off = 16; off >= 1; off >>= 1) {
                t.x += __shfl_xor_sync(0xffffffffu, t.x, off);
                t.y += __shfl_xor_sync(0xffffffffu, t.y, off);
            }
            if (lane == 0) s_w[warp] = t;
            __syncthreads();
            if (threadIdx.x == 0) {
                double2 a = s_w[0];
                for (int w = 1; w < RED_BIG_THREADS / 32; ++w) {
                    a.x += s_w[w].x;
                    a.y += s_w[w].y;
                }
                amp_out[g] = a;
            }
            __syncthreads();
            continue;
        }
        for (int s = 0; s < J.S; ++s) {
            uint64_t lo, hi;
            const double2* src = pair_items(J, o * (uint64_t)J.S + (uint64_t)s, lo, hi);
            double2 t = strided_sum(src, lo + threadIdx.x, hi, RED_BIG_THREADS);
#pragma unroll
            for (int off = 16; off >= 1; off >>= 1) {
                t.x += __shfl_xor_sync(0xffffffffu, t.x, off);
                t.y += __shfl_xor_sync(0xffffffffu, t.y, off);
            }
            if (lane == 0) s_w[warp] = t;
            __syncthreads();
            if (threadIdx.x == 0) {
                double2 a = s_w[0];
                for (int w = 1; w < RED_BIG_THREADS / 32; ++w) {
                    a.x += s_w[w].x;
                    a.y += s_w[w].y;
                }
                const double2 w2 = cmul(__ldg(J.coef + s), a);
                amp.x += w2.x;
                amp.y += w2.y;
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) amp_out[g] = amp;
    }
}

// ---------------------------------------------------------------- exact bound

// One warp covers 32 consecutive entries, inside one compaction block.
__global__ void __launch_bounds__(256) bound_prune_kernel(const JobDev* __restrict__ jobs, int job, BoundSpec sp,
                                                          unsigned long long n, int count_blocks)
{
    FS_GRID_DEP();
    const JobDev& J = jobs[job];
    unsigned long long cuts = 0;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long base = (unsigned long long)blockIdx.x * blockDim.x; base < n; base += stride) {
        const unsigned long long e = base + threadIdx.x;
        bool live = false, cut = false;
        if (e < n) {
            uint4* ent = reinterpret_cast<uint4*>(J.table + e);
            const uint4 sv = ent[0];
            const double2 a = reinterpret_cast<const double2*>(ent + 1)[0];
            live = !is_bottom(a.x);
            if (live) {
                uint64_t sidx;
                pair_split(e >> J.Ap, J, sidx);
                const uint4 bv = __ldg(reinterpret_cast<const uint4*>(J.ins + 4 * sidx));
                const uint32_t st[4] = {sv.x, sv.y, sv.z, sv.w}, bi[4] = {bv.x, bv.y, bv.z, bv.w};
                uint32_t d = 0;
#pragma unroll
                for (int w = 0; w < 4; ++w) d |= (st[w] ^ bi[w]) & sp.frozen[w];
                cut = d != 0u;
                const unsigned __int128 s128 = ((unsigned __int128)(((uint64_t)st[3] << 32) | st[2]) << 64) |
                                               (((uint64_t)st[1] << 32) | st[0]);
                const unsigned __int128 b128 = ((unsigned __int128)(((uint64_t)bi[3] << 32) | bi[2]) << 64) |
                                               (((uint64_t)bi[1] << 32) | bi[0]);
                for (int f = 0; f < sp.n_fields && !cut; ++f) {
                    const unsigned __int128 m = sp.len[f] >= 128 ? ~(unsigned __int128)0
                                                                 : (((unsigned __int128)1 << sp.len[f]) - 1);
                    const unsigned __int128 x = (s128 >> sp.t0[f]) & m, y = (b128 >> sp.t0[f]) & m;
                    const unsigned __int128 up = (x - y) & m, down = (y - x) & m;   // cyclic distances
                    const unsigned __int128 dist = up < down ? up : down;
                    cut = dist > (unsigned __int128)sp.radius[f];
                }
                if (cut) {
                    reinterpret_cast<double2*>(ent + 1)->x = __longlong_as_double(0x7ff8000000000000ll);
                    ++cuts;
                }
            }
        }
        if (count_blocks) {
            const unsigned keep = __ballot_sync(0xffffffffu, live && !cut);
            if ((threadIdx.x & 31) == 0 && keep)
                atomicAdd(&J.blk[(base + (threadIdx.x & ~31u)) / COMPACT_BLOCK], (unsigned)__popc(keep));
        }
    }
    cuts = warp_sum_u64(cuts);
    if ((threadIdx.x & 31) == 0 && cuts) atomicAdd(&J.stats[8], cuts);
}

// ---------------------------------------------------------------- peak probes

// FP64 FMA throughput: 8 independent dependency chains per thread.
__global__ void __launch_bounds__(256) probe_dfma_kernel(double* out, int iters, double a, double b)
{
    double x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = threadIdx.x * 1e-9 + k;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = __fma_rn(x[k], a, b);
    }
    double s = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += x[k];
    if (s == 12345.678) out[0] = s;   // keeps the chains live
}

// 32-bit integer logic throughput: 8 independent xor-rotate chains per thread.
__global__ void __launch_bounds__(256) probe_int_kernel(unsigned* out, int iters, unsigned a)
{
    unsigned x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = threadIdx.x * 2654435761u + k;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = (x[k] ^ a) + (unsigned)k;
    }
    unsigned s = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s ^= x[k];
    if (s == 0x12345678u) out[0] = s;
}

}  // namespace

cudaError_t probe_peaks(double* dfma_per_s, double* int_ops_per_s, int* sms)
{
    int dev = 0, n_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    *sms = n_sm;
    void* buf = nullptr;
    cudaError_t e = cudaMalloc(&buf, 256);
    if (e != cudaSuccess) return e;
    cudaEvent_t t0, t1;
    cudaEventCreate(&t0);
    cudaEventCreate(&t1);
    const int blocks = n_sm * 8, threads = 256;
    float ms = 0;
    const int di = 4096, ii = 65536;
    probe_dfma_kernel<<<blocks, threads>>>((double*)buf, 16, 1.0000001, 1e-7);
    cudaEventRecord(t0);
    probe_dfma_kernel<<<blocks, threads>>>((double*)buf, di, 1.0000001, 1e-7);
    cudaEventRecord(t1);
    cudaEventSynchronize(t1);
    cudaEventElapsedTime(&ms, t0, t1);
    *dfma_per_s = (double)blocks * threads * di * 8 / (ms * 1e-3);
    probe_int_kernel<<<blocks, threads>>>((unsigned*)buf, 16, 0x9e3779b9u);
    cudaEventRecord(t0);
    probe_int_kernel<<<blocks, threads>>>((unsigned*)buf, ii, 0x9e3779b9u);
    cudaEventRecord(t1);
    cudaEventSynchronize(t1);
    cudaEventElapsedTime(&ms, t0, t1);
    *int_ops_per_s = (double)blocks * threads * ii * 8 * 2 / (ms * 1e-3);
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    e = cudaGetLastError();
    cudaFree(buf);
    return e;
}

bool pdl_enabled()
{
    static const bool on = [] {
        const char* v = getenv("FS_NO_PDL");
        return !(v && v[0] == '1');
    }();
    return on;
}

cudaError_t launch_ex(const void* func, dim3 grid, dim3 block, size_t smem, cudaStream_t s, void** args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl_enabled() ? 1 : 0;
    return cudaLaunchKernelExC(&cfg, func, args);
}

cudaError_t launch_prefix(const JobDev* d_jobs, const uint64_t* d_begin, int n_jobs,
                          uint64_t total, uint32_t* d_err, cudaStream_t s)
{
    if (total == 0) return cudaSuccess;
    uint64_t blocks = (total + 255) / 256;
    if (blocks > 148ull * 64) blocks = 148ull * 64;
    return launch_pdl(prefix_kernel, dim3((unsigned)blocks), dim3(256), 0, s, d_jobs, d_begin, n_jobs, total, d_err);
}

int history_grid_size(int device)
{
    int sms = 0, per_sm = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, history_kernel, TILE, 0);
    if (sms <= 0) sms = 148;
    if (per_sm <= 0) per_sm = 1;
    return sms * per_sm;
}

cudaError_t launch_history(const JobDev* d_jobs, const uint2* d_tiles, uint64_t n_tiles,
                           unsigned int* d_counter, uint32_t* d_err, int grid, cudaStream_t s)
{
    if (n_tiles == 0) return cudaSuccess;
    if ((uint64_t)grid > n_tiles) grid = (int)n_tiles;
    return launch_pdl(history_kernel, dim3(grid), dim3(TILE), 0, s, d_jobs, d_tiles, n_tiles, d_counter, d_err);
}

cudaError_t launch_prefix_level(const JobDev* d_job, const PrefixLevel& L, const Entry* src, Entry* dst,
                                uint64_t n_dst, bool last, uint32_t* d_err, cudaStream_t s)
{
    if (n_dst == 0) return cudaSuccess;
    uint64_t blocks = (n_dst + 255) / 256;
    if (blocks > 148ull * 64) blocks = 148ull * 64;
    return launch_pdl(prefix_level_kernel, dim3((unsigned)blocks), dim3(256), 0, s, d_job, L, src, dst, n_dst,
                      last ? 1 : 0, d_err);
}

cudaError_t launch_compact(const JobDev* d_job, uint64_t n_entries, bool counted, cudaStream_t s)
{
    const uint64_t nblk = (n_entries + COMPACT_BLOCK - 1) / COMPACT_BLOCK;
    if (nblk == 0) return cudaSuccess;
    cudaError_t e = cudaSuccess;
    const bool scan = nblk > (uint64_t)COMPACT_DIRECT_BLOCKS;
    if (!counted) e = launch_pdl(compact_count_kernel, dim3((unsigned)nblk), dim3(256), 0, s, d_job);
    if (e == cudaSuccess && scan)
        e = launch_pdl(compact_scan_kernel, dim3(1), dim3(1024), 0, s, d_job, (uint32_t)nblk);
    if (e == cudaSuccess)
        e = launch_pdl(compact_write_kernel, dim3((unsigned)nblk), dim3(256), 0, s, d_job, scan ? 1 : 0);
    return e;
}

int compact_grid_size(int device)
{
    int sms = 0, per_sm = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, history_compact_kernel, 256, 0);
    return (sms > 0 ? sms : 148) * (per_sm > 0 ? per_sm : 1);
}

cudaError_t launch_history_compact(const JobDev* d_job, uint32_t* d_err, int grid, cudaStream_t s)
{
    return launch_pdl(history_compact_kernel, dim3(grid), dim3(256), 0, s, d_job, d_err);
}

cudaError_t launch_bound_prune(const JobDev* d_jobs, int job, const BoundSpec& sp, unsigned long long n_entries,
                               bool count_blocks, cudaStream_t s)
{
    if (n_entries == 0) return cudaSuccess;
    unsigned long long blocks = (n_entries + 255) / 256;
    if (blocks > 148ull * 16) blocks = 148ull * 16;
    return launch_pdl(bound_prune_kernel, dim3((unsigned)blocks), dim3(256), 0, s, d_jobs, job, sp, n_entries,
                      count_blocks ? 1 : 0);
}

cudaError_t launch_reduce(const JobDev* d_jobs, const uint64_t* d_begin, int n_jobs,
                          uint64_t total_out, double2* d_amp, unsigned int* d_big_count, uint64_t* d_big_list,
                          bool big_possible, cudaStream_t s)
{
    if (total_out == 0) return cudaSuccess;
    const uint64_t per_block = (REDUCE_THREADS / 32) * (32 / RED_LPO);   // outputs per block pass
    uint64_t blocks = (total_out + per_block - 1) / per_block;
    if (blocks > 148ull * 16) blocks = 148ull * 16;
    cudaError_t e = launch_pdl(reduce_kernel, dim3((unsigned)blocks), dim3(REDUCE_THREADS), 0, s, d_jobs, d_begin,
                               n_jobs, total_out, d_amp, d_big_count, d_big_list);
    if (e != cudaSuccess || !big_possible) return e;
    const uint64_t big_blocks = total_out < 148ull * 4 ? total_out : 148ull * 4;
    return launch_pdl(reduce_big_kernel, dim3((unsigned)big_blocks), dim3(RED_BIG_THREADS), 0, s, d_jobs, d_begin,
                      n_jobs, (const unsigned int*)d_big_count, (const uint64_t*)d_big_list, d_amp);
}

}  // namespace fs

"""The straight-line engine's generated region code, compiled for the host.

`fs_batch_generated_source` returns the CUDA C++ the next upload would
compile.  Its region functions (prefix, root and suffix of Algorithm 2 for
each job) are plain integer and FP64 code; here they are extracted, compiled
with g++ against small stand-ins for the few CUDA intrinsics they use, and
driven by a literal Algorithm 2 loop on the host, with the prefix either as
one region or expanded level by level as the level kernels do.  The amplitudes must match
the oracle: this checks the code generator itself (fused incrementers,
deferred and hoisted factor classes, threshold cuts) without a GPU."""
import os
import subprocess
import tempfile

import numpy as np
import pytest

from workloads import (Gate, Circuit as WCircuit, SplitMix64, aa_workload, qaoa_workload, qft,
                       quantum_walk, random_small_circuit)
from oracle import feynman
import paper_2608_01467_b300 as fs

SHIM = r"""
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
typedef unsigned int u32;
typedef int i32;
typedef unsigned long long u64;
struct double2 { double x, y; };
static inline double2 make_double2(double x, double y) { double2 r; r.x = x; r.y = y; return r; }
#define __device__
#define __forceinline__ inline
#define __noinline__
#define __ldg(p) (*(p))
static inline double __fma_rn(double a, double b, double c) { return std::fma(a, b, c); }
static inline double __dmul_rn(double a, double b) { return a * b; }
static inline int __double2hiint(double x) { uint64_t u; std::memcpy(&u, &x, 8); return (int)(u >> 32); }
static inline int __double2loint(double x) { uint64_t u; std::memcpy(&u, &x, 8); return (int)(u & 0xffffffffu); }
static inline unsigned __activemask() { return 0xffffffffu; }
static inline unsigned __funnelshift_r(unsigned lo, unsigned hi, unsigned s)
{
    s &= 31u;
    return s ? (lo >> s) | (hi << (32u - s)) : lo;
}
static inline bool __any_sync(unsigned, bool p) { return p; }   // one lane on the host
static inline long long __double_as_longlong(double x) { long long u; std::memcpy(&u, &x, 8); return u; }
static inline double __hiloint2double(int hi, int lo)
{
    uint64_t u = ((uint64_t)(uint32_t)hi << 32) | (uint32_t)lo;
    double d;
    std::memcpy(&d, &u, 8);
    return d;
}
"""

DRIVER = r"""
int main()
{
    const int M = %(M)d, S = %(S)d;
    static const u32 outs[%(Mp)d][4] = {%(outs)s};
    static const u32 ins[%(Sp)d][4] = {%(ins)s};
    static const double cre_[%(Sp)d] = {%(cre)s}, cim_[%(Sp)d] = {%(cim)s};
    const double2 scale = make_double2(%(sx)s, %(sy)s);
    constexpr int W = J0::W;
    for (int o = 0; o < M; ++o) {
        double ar = 0.0, ai = 0.0;
        u64 completed = 0, valid = 0;
        for (int s = 0; s < S; ++s) {
            u32 bin[W];
            for (int j = 0; j < W; ++j) bin[j] = ins[s][j];
            double sr = 0.0, si = 0.0;
            u64 visits = 0;
            for (u64 hp = 0; hp < (1ull << J0::Ap); ++hp) {
                u32 st[W];
                for (int j = 0; j < W; ++j) st[j] = outs[o][j];
                double2 a = make_double2(1.0, 0.0);
                if (J0::prefix(st, a, hp, bin, visits) >= 0) continue;
                for (u64 hr = 0; hr < (1ull << J0::Ar); ++hr) {
                    u32 st2[W];
                    for (int j = 0; j < W; ++j) st2[j] = st[j];
                    double2 a2 = a;
                    if (J0::root(st2, a2, hr, bin, visits) >= 0) continue;
%(suffix_loop)s
                }
            }
            // c_in times the constant left out of the root and suffix
            const double cr = cre_[s] * scale.x - cim_[s] * scale.y, ci = cre_[s] * scale.y + cim_[s] * scale.x;
            ar += cr * sr - ci * si;
            ai += cr * si + ci * sr;
        }
        std::printf("%%.17g %%.17g %%llu %%llu\n", ar, ai, completed, valid);
    }
    return 0;
}
"""


DRIVER_LEVELS = r"""
#include <vector>
struct Ent { u32 st[4]; double2 a; bool live; };
int main()
{
    const int M = %(M)d, S = %(S)d;
    static const u32 outs[%(Mp)d][4] = {%(outs)s};
    static const u32 ins[%(Sp)d][4] = {%(ins)s};
    static const double cre_[%(Sp)d] = {%(cre)s}, cim_[%(Sp)d] = {%(cim)s};
    const double2 scale = make_double2(%(sx)s, %(sy)s);
    constexpr int W = J0::W;
    static const int lv_prev[] = {%(aprev)s}, lv_next[] = {%(anext)s};
    const int L = %(L)d;
    for (int o = 0; o < M; ++o) {
        double ar = 0.0, ai = 0.0;
        u64 completed = 0, valid = 0;
        for (int s = 0; s < S; ++s) {
            u32 bin[W];
            for (int j = 0; j < W; ++j) bin[j] = ins[s][j];
            u64 visits = 0;
            // level k extends entry p (a_prev bits) by the level's new bits
            // c into child (p << new) | c, evaluated with h = child << (A_p - a_next)
            std::vector<Ent> cur(1);
            for (int j = 0; j < 4; ++j) cur[0].st[j] = outs[o][j];
            cur[0].a = make_double2(1.0, 0.0);
            cur[0].live = true;
            for (int k = 0; k < L; ++k) {
                const int nb = lv_next[k] - lv_prev[k];
                std::vector<Ent> nxt(cur.size() << nb);
                for (u64 p = 0; p < cur.size(); ++p)
                    for (u64 c = 0; c < (1ull << nb); ++c) {
                        const u64 child = (p << nb) | c;
                        Ent e = cur[p];
                        if (e.live) {
                            u32 st[W];
                            for (int j = 0; j < W; ++j) st[j] = e.st[j];
                            const u64 h = child << (J0::Ap - lv_next[k]);
                            int r = -1;
                            switch (k) {
%(cases)s
                            default: break;
                            }
                            e.live = r < 0;
                            for (int j = 0; j < W; ++j) e.st[j] = st[j];
                        }
                        nxt[child] = e;
                    }
                cur.swap(nxt);
            }
            double sr = 0.0, si = 0.0;
            for (u64 hp = 0; hp < cur.size(); ++hp) {
                if (!cur[hp].live) continue;
                for (u64 hr = 0; hr < (1ull << J0::Ar); ++hr) {
                    u32 st2[W];
                    for (int j = 0; j < W; ++j) st2[j] = cur[hp].st[j];
                    double2 a2 = cur[hp].a;
                    if (J0::root(st2, a2, hr, bin, visits) >= 0) continue;
%(suffix_loop)s
                }
            }
            const double cr = cre_[s] * scale.x - cim_[s] * scale.y, ci = cre_[s] * scale.y + cim_[s] * scale.x;
            ar += cr * sr - ci * si;
            ai += cr * si + ci * sr;
        }
        std::printf("%%.17g %%.17g %%llu %%llu\n", ar, ai, completed, valid);
    }
    return 0;
}
"""


# the suffix enumeration of the driver: every h_s tried in turn (the
# generated `suffix` returns at a cut), or, for a stacked suffix, the
# device's restart loop: skip the subtree of a cut history and restart the
# next one at the first source whose bit changed, from the saved state
SUFFIX_PLAIN = """
                    for (u64 hs = 0; hs < (1ull << J0::As); ++hs) {
                        u32 st3[W];
                        for (int j = 0; j < W; ++j) st3[j] = st2[j];
                        double2 a3 = a2;
                        if (J0::suffix(st3, a3, hs, bin, visits) >= 0) continue;
                        ++completed;
                        bool ok = true;
                        for (int j = 0; j < W; ++j) ok = ok && st3[j] == bin[j];
                        if (ok) { sr += a3.x; si += a3.y; ++valid; }
                    }"""
SUFFIX_STACKED = """
                    {
                        u32 sst[J0::As][W];
                        double2 sam[J0::As];
                        u32 skc[J0::As][J0::SC];
                        int start = 0;
                        const u64 ns = 1ull << J0::As;
                        u64 hs = 0;
                        while (hs < ns) {
                            u32 st3[W];
                            double2 a3;
                            for (int j = 0; j < W; ++j) st3[j] = start ? sst[start - 1][j] : st2[j];
                            a3 = start ? sam[start - 1] : a2;
                            const int r2 = J0::suffix_from(start, st3, a3, hs, bin, visits, sst, sam, skc);
                            u64 nx;
                            if (r2 < 0) {
                                ++completed;
                                bool ok = true;
                                for (int j = 0; j < W; ++j) ok = ok && st3[j] == bin[j];
                                if (ok) { sr += a3.x; si += a3.y; ++valid; }
                                nx = hs + 1;
                            } else {
                                nx = ((hs >> r2) + 1) << r2;
                            }
                            if (nx < ns) start = J0::As - 1 - (63 - __builtin_clzll(hs ^ nx));
                            hs = nx;
                        }
                    }"""


# the device's level-by-level walk of a threshold suffix (its 32 lanes in
# turn): per-level queues of partial histories (at most 40 each); a step
# takes up to 16 histories from the top of the level that fills the most
# lanes among those whose next level has room for their children (the
# deepest on ties) and evaluates both values of their next source; the
# passing ones are queued one level deeper or, after the last source, run
# through the tail and the chi test
SUFFIX_QUEUE = """
                    {
                        static u32 qs[J0::As][40][W];
                        static double2 qa[J0::As][40];
                        u32 cnt[J0::As + 1];
                        for (int l = 0; l <= J0::As; ++l) cnt[l] = 0;
                        for (int j = 0; j < W; ++j) qs[0][0][j] = st2[j];
                        qa[0][0] = a2;
                        cnt[0] = 1;
                        for (;;) {
                            int L = -1;
                            u32 k = 0;
                            for (int l = J0::As - 1; l >= 0; --l) {
                                const u32 kl = cnt[l] < 16 ? cnt[l] : 16;
                                if (kl > k && cnt[l + 1] + 2 * kl <= 40) { L = l; k = kl; }
                            }
                            if (L < 0) break;
                            const u32 n = cnt[L], base = n - k;
                            cnt[L] = base;
                            u32 np = cnt[L + 1];
                            for (int lane = 0; lane < 32; ++lane) {
                                const u32 node = lane >> 1;
                                if (node >= k) continue;
                                u32 s3[W];
                                for (int j = 0; j < W; ++j) s3[j] = qs[L][base + node][j];
                                double2 a3 = qa[L][base + node];
                                if (J0::seg_step(L, s3, a3, (u32)lane & 1u, bin, visits) != 0) continue;
                                if (L + 1 < J0::As) {
                                    if (np >= 40) { std::printf("queue overflow\\n"); return 1; }
                                    for (int j = 0; j < W; ++j) qs[L + 1][np][j] = s3[j];
                                    qa[L + 1][np] = a3;
                                    ++np;
                                } else if (J0::tail(s3, a3, 0ull, bin, visits) < 0) {
                                    ++completed;
                                    bool ok = true;
                                    for (int j = 0; j < W; ++j) ok = ok && s3[j] == bin[j];
                                    if (ok) { sr += a3.x; si += a3.y; ++valid; }
                                }
                            }
                            if (L + 1 < J0::As) cnt[L + 1] = np;
                        }
                    }"""


# the device's phase census (exact suffixes whose factors are unit phases):
# each valid leaf is the root's amplitude times i^q; the leaves are counted
# by q and the root adds amp * ((n0 - n2) + i (n1 - n3))
SUFFIX_CENSUS = """
                    {
                        long long n[4] = {0, 0, 0, 0};
                        for (u64 hs = 0; hs < (1ull << J0::As); ++hs) {
                            u32 st3[W];
                            for (int j = 0; j < W; ++j) st3[j] = st2[j];
                            double2 a3 = a2;
                            u32 q = 0;
                            if (J0::suffix_q(st3, a3, hs, bin, visits, q) >= 0) continue;
                            ++completed;
                            bool ok = true;
                            for (int j = 0; j < W; ++j) ok = ok && st3[j] == bin[j];
                            if (ok) { ++n[q & 3u]; ++valid; }
                        }
                        const double re = (double)(n[0] - n[2]), im = (double)(n[1] - n[3]);
                        sr += a2.x * re - a2.y * im;
                        si += a2.x * im + a2.y * re;
                    }"""


SUFFIX_CENSUS_STACKED = """
                    {
                        long long n[4] = {0, 0, 0, 0};
                        u32 sst[J0::As][W];
                        double2 sam[J0::As];
                        u32 skc[J0::As][J0::SCQ];
                        int start = 0;
                        const u64 ns = 1ull << J0::As;
                        u64 hs = 0;
                        while (hs < ns) {
                            u32 st3[W];
                            double2 a3 = a2;
                            for (int j = 0; j < W; ++j) st3[j] = start ? sst[start - 1][j] : st2[j];
                            u32 q = 0;
                            const int r2 = J0::suffix_from_q(start, st3, a3, hs, bin, visits, sst, sam, skc, q);
                            u64 nx;
                            if (r2 < 0) {
                                ++completed;
                                bool ok = true;
                                for (int j = 0; j < W; ++j) ok = ok && st3[j] == bin[j];
                                if (ok) { ++n[q & 3u]; ++valid; }
                                nx = hs + 1;
                            } else {
                                nx = ((hs >> r2) + 1) << r2;
                            }
                            if (nx < ns) start = J0::As - 1 - (63 - __builtin_clzll(hs ^ nx));
                            hs = nx;
                        }
                        const double re = (double)(n[0] - n[2]), im = (double)(n[1] - n[3]);
                        sr += a2.x * re - a2.y * im;
                        si += a2.x * im + a2.y * re;
                    }"""


def _words(v, W):
    return "{" + ", ".join(f"{(v >> (32 * j)) & 0xffffffff}u" for j in range(4)) + "}"


def _extract(src):
    i = src.index("__device__ __forceinline__ double2 cmul")
    j = src.index("__device__ __forceinline__ double2 sel2")
    j = src.index("\n", j) + 1
    helpers = src[i:j]
    k = min(x for x in (src.find("__device__ const double2 T_"), src.find("__device__ const double2 PH_"),
                        src.find("struct J0 {")) if x >= 0)
    e = src.index('extern "C"', k)
    body = src[k:e]
    scale_line = [l for l in body.splitlines() if "J0: constant factor" in l][0]
    sx, sy = scale_line.split("(")[-1].rstrip(")").split(",")
    return helpers, body, sx.strip(), sy.strip()


def _host_amplitudes(circ, inputs, outputs, c1, c2, eps, tmp, prefix="single", walk=False, bound=False,
                     census=False):
    C = fs.Circuit(circ)
    C.set_input(inputs)
    b = fs.Batch(split="fixed", c1=c1, c2=c2, prefix=prefix)
    b.add(C, outputs, eps)
    if bound:
        b.set_exact_bound(0)
    b.plan()
    src = b.generated_source()
    helpers, body, sx, sy = _extract(src)
    W = 4
    fields = dict(M=len(outputs), S=len(inputs), Mp=max(len(outputs), 1), Sp=max(len(inputs), 1),
                  outs=", ".join(_words(v, W) for v in outputs),
                  ins=", ".join(_words(v, W) for v, _ in inputs),
                  cre=", ".join(repr(complex(c).real) for _, c in inputs),
                  cim=", ".join(repr(complex(c).imag) for _, c in inputs), sx=sx, sy=sy)
    stacked = "STACKED = true" in src
    queue = "QUEUE = true" in src
    has_census = "CENSUS = true" in src
    if census and has_census:
        fields["suffix_loop"] = SUFFIX_CENSUS_STACKED if stacked else SUFFIX_CENSUS
    else:
        fields["suffix_loop"] = SUFFIX_QUEUE if walk and queue else SUFFIX_STACKED if stacked else SUFFIX_PLAIN
    levels = [l.split("sources [")[1].rstrip(")").split(", ") for l in src.splitlines() if "  // level " in l]
    if levels:
        fields.update(L=len(levels), aprev=", ".join(a for a, _ in levels), anext=", ".join(b_ for _, b_ in levels),
                      cases="\n".join(f"                            case {k}: r = J0::lv{k}(st, e.a, h, bin, visits); break;"
                                      for k in range(len(levels))))
        drv = DRIVER_LEVELS % fields
    else:
        drv = DRIVER % fields
    path = os.path.join(tmp, "gen.cpp")
    with open(path, "w") as f:
        f.write(SHIM + helpers + body + drv)
    exe = os.path.join(tmp, "gen")
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-ffp-contract=off", "-w", "-o", exe, path])
    rows = [l.split() for l in subprocess.check_output([exe]).decode().splitlines()]
    amp = np.array([float(r[0]) + 1j * float(r[1]) for r in rows])
    _host_amplitudes.stacked = stacked
    _host_amplitudes.queue = queue
    _host_amplitudes.census = has_census
    return amp, np.array([int(r[2]) for r in rows]), np.array([int(r[3]) for r in rows])


def _close(got, want):
    err = np.abs(np.asarray(got) - np.asarray(want))
    assert np.all(err <= 1e-12 + 1e-10 * np.abs(want)), err.max()


def _cascade(n, f0, L, common, inc):
    g = [Gate("H", (f0,)), Gate("H", (f0 + L - 1,))] + [Gate("H", (q,)) for q, _ in common]
    v = 1 if inc else 0
    for k in range(L - 1, -1, -1):
        ctr = tuple(common) + tuple((f0 + j, v) for j in range(k))
        g.append(Gate("X", (f0 + k,), ctr) if ctr else Gate("X", (f0 + k,)))
    g += [Gate("S", (f0,)), Gate("H", (f0,))]
    return WCircuit(n, g, "cascade")


def _embed():
    """A 6-qubit random circuit on qubits spread over three register words
    of a 70-qubit register; outputs with nonzero amplitude from its dense
    simulation."""
    from oracle import dense
    act = [3, 31, 32, 40, 63, 66]
    small = random_small_circuit(6, 30, 707)
    gates = [Gate(g.kind, tuple(act[q] for q in g.qubits), tuple((act[q], v) for q, v in g.controls),
                  g.theta, g.matrix) for g in small.gates]
    big = WCircuit(70, gates, "embed70")
    amp = dense.amplitudes(small, [(5, 1.0)], list(range(64)))
    top = [int(i) for i in np.argsort(-np.abs(amp))[:5]]
    spread = lambda y: sum(((y >> j) & 1) << q for j, q in enumerate(act))
    return big, [(spread(5), 1.0)], [spread(y) for y in top]


def _cascade_case(n, f0, L, common, inc):
    """The cascade circuit and outputs reachable from a seeded input: any
    flips of the H qubits, the field moved by one where the common controls
    hold, either value of the last H qubit."""
    c = _cascade(n, f0, L, common, inc)
    b = SplitMix64(n + L).bits(n)
    hq = [f0, f0 + L - 1] + [q for q, _ in common]
    outs = []
    for k in range(1 << len(hq)):
        y = b
        for j, q in enumerate(hq):
            if (k >> j) & 1:
                y ^= 1 << q
        if all(((y >> q) & 1) == v for q, v in common):
            x = (y >> f0) & ((1 << L) - 1)
            x = (x + (1 if inc else -1)) % (1 << L)
            y = (y & ~(((1 << L) - 1) << f0)) | (x << f0)
        outs.append(y & ~(1 << f0))
        outs.append(y | (1 << f0))
    return c, [(b, 1.0)], outs[:6]


def _walk():
    from workloads import qw_workload
    w = qw_workload(steps=5, n_out=6, pos_bits=8)
    return w.circuit, w.inputs, w.outputs


def _qaoa():
    w = qaoa_workload(6, 2, n_out=5, seed=3)
    return w.circuit, w.inputs, w.outputs


def _aa():
    w = aa_workload(n=4, iters=1, all_outputs=True)
    return w.circuit, w.inputs, w.outputs[:6]


CASES = {
    "random7": lambda: (random_small_circuit(7, 40, 4249), 2),
    "random9": lambda: (random_small_circuit(9, 50, 905), 3),
    "embed70": _embed,
    "qft5": lambda: (qft(5), 1),
    "qaoa6": _qaoa,
    "aa4": _aa,
    "walk": _walk,
    "cascade_inc": lambda: _cascade_case(45, 27, 12, ((1, 0),), True),
    "cascade_dec": lambda: _cascade_case(70, 5, 60, ((0, 1), (68, 0)), False),
}


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("eps,prefix", [(0.0, "single"), (0.05, "single"), (0.0, "levels"), (0.05, "levels")])
def test_generated_regions_match_the_oracle(case, eps, prefix, tmp_path):
    spec = CASES[case]()
    circ = spec[0]
    n = circ.n_qubits
    G = len(circ.gates)
    A = feynman.analyze(circ)["A"]
    assert A <= 14, A
    if len(spec) == 3:
        inputs, outputs = spec[1], spec[2]
    else:
        rng = SplitMix64(len(case) * 131 + n)
        inputs = [(rng.bits(n), complex(0.6 + 0.1 * k, 0.2 * k)) for k in range(spec[1])]
        outputs = [rng.bits(n) for _ in range(5)]
        if n <= 9:   # small registers: outputs that carry amplitude
            from oracle import dense
            amp = dense.amplitudes(circ, inputs, list(range(1 << n)))
            outputs = [int(i) for i in np.argsort(-np.abs(amp))[:5]] + outputs[:2]
    c1, c2 = G // 3, (2 * G) // 3
    got, completed, valid = _host_amplitudes(circ, inputs, outputs, c1, c2, eps, str(tmp_path), prefix)
    want, cnt = feynman.run(circ, inputs, outputs, eps=eps, c1=c1, c2=c2)
    _close(got, want)
    # the same factors in the same order: every pruning decision, hence every
    # leaf count, is the oracle's exactly
    assert np.array_equal(completed, cnt["completed"].astype(np.int64))
    assert np.array_equal(valid, cnt["valid"].astype(np.int64))
    if eps == 0.0:
        assert np.abs(want).max() > 0.05   # the case exercises nonzero amplitudes


@pytest.mark.parametrize("family,eps", [("qaoa", 1e-2), ("qaoa", 1e-3), ("qaoa", 3e-4), ("walk", 0.3),
                                        ("random", 0.05)])
def test_stacked_suffix_matches_the_oracle(family, eps, tmp_path):
    """Threshold jobs with several artificial sources in the suffix run it
    as per-source segments with a saved state after each source op; the next
    history restarts at the first source whose bit changed.  Driven on the
    host by the device's restart loop, amplitudes and leaf counts must be the
    oracle's (the same factors in the same order: identical pruning)."""
    if family == "qaoa":
        w = qaoa_workload(8, 2, n_out=6, seed=5)
        circ, inputs, outputs = w.circuit, w.inputs, w.outputs
        c1 = c2 = 8                              # 8 sources before, 8 in the suffix
    elif family == "walk":
        circ, inputs, outputs = _walk()
        c1 = c2 = len(circ.gates) // 4
    else:
        circ = random_small_circuit(9, 60, 9093)   # one source per branching op in the suffix
        rng = SplitMix64(9093)
        inputs = [(rng.bits(9), 0.8), (rng.bits(9), 0.6j)]
        outputs = [rng.bits(9) for _ in range(5)]
        c1 = c2 = len(circ.gates) // 3
    got, completed, valid = _host_amplitudes(circ, inputs, outputs, c1, c2, eps, str(tmp_path))
    assert _host_amplitudes.stacked
    want, cnt = feynman.run(circ, inputs, outputs, eps=eps, c1=c1, c2=c2)
    _close(got, want)
    assert np.array_equal(completed, cnt["completed"].astype(np.int64))
    assert np.array_equal(valid, cnt["valid"].astype(np.int64))
    if _host_amplitudes.queue:
        # the same suffix walked level by level (seg_step / tail)
        got, completed, valid = _host_amplitudes(circ, inputs, outputs, c1, c2, eps, str(tmp_path), walk=True)
        _close(got, want)
        assert np.array_equal(completed, cnt["completed"].astype(np.int64))
        assert np.array_equal(valid, cnt["valid"].astype(np.int64))


def test_generated_exact_bound_matches_the_reachability_rule(tmp_path):
    """The exact reachability bound as generated code (bound_cut of the job,
    compiled for the host): on the walk the remaining ops move the position
    by at most two per remaining step (a +1 and a -1 cascade) and never touch
    the third ancilla, so a state is cut iff that ancilla differs from the
    input's or the cyclic position distance exceeds twice the remaining
    steps.  Checked on 96-bit positions (fields across register words) and
    8-bit ones, on random states near and far from the input."""
    from workloads import qw_workload
    for pos_bits, steps, k_prefix in ((96, 6, 2), (8, 6, 3)):
        w = qw_workload(steps=steps, n_out=8, pos_bits=pos_bits)
        G = len(w.circuit.gates)
        c1 = k_prefix * (G // steps)
        radius = 2 * (steps - k_prefix)
        C = fs.Circuit(w.circuit)
        C.set_input(w.inputs)
        b = fs.Batch(split="fixed", c1=c1, c2=c1)
        b.add(C, w.outputs)
        b.set_exact_bound(0)
        b.plan()
        src = b.generated_source()
        helpers, body, _, _ = _extract(src)
        W = 4 if pos_bits > 32 else 1
        mask = (1 << pos_bits) - 1
        rng = SplitMix64(pos_bits)
        b_in = w.inputs[0][0]
        cases = []
        for _ in range(400):
            d = rng.below(4 * radius + 5) - 2 * radius - 2
            if rng.below(4) == 0:
                d = rng.bits(pos_bits)
            pos = (((b_in >> 1) & mask) + d) & mask
            s = (b_in & ~(mask << 1)) | (pos << 1) | rng.below(2) | (rng.below(4) << (pos_bits + 1))
            if rng.below(8) == 0:
                s ^= 1 << (pos_bits + 3)
            cases.append(s)
        words = lambda v: "{" + ", ".join(f"{(v >> (32 * j)) & 0xffffffff}u" for j in range(W)) + "}"
        drv = ("int main() {\n    static const u32 st[][%d] = {%s};\n    const u32 bin[%d] = %s;\n"
               "    for (unsigned i = 0; i < %d; ++i) std::printf(\"%%d\\n\", J0::bound_cut(st[i], bin) ? 1 : 0);\n"
               "    return 0;\n}\n") % (W, ", ".join(words(s) for s in cases), W, words(b_in), len(cases))
        path = os.path.join(str(tmp_path), f"bound{pos_bits}.cpp")
        with open(path, "w") as f:
            f.write(SHIM + helpers + body + drv)
        exe = path[:-4]
        subprocess.check_call(["g++", "-O1", "-std=c++17", "-w", "-o", exe, path])
        got = [int(x) for x in subprocess.check_output([exe]).decode().split()]
        want = []
        for s in cases:
            x, y = (s >> 1) & mask, (b_in >> 1) & mask
            dist = min((x - y) & mask, (y - x) & mask)
            want.append(int(dist > radius or (((s ^ b_in) >> (pos_bits + 3)) & 1) == 1))
        assert got == want
        assert 0 < sum(want) < len(want)


@pytest.mark.parametrize("case", ["walk", "cascade_inc", "cascade_dec"])
def test_generated_bound_after_each_source_keeps_every_valid_leaf(case, tmp_path):
    """With the exact bound, the generated root and suffix also test the
    bound after every op that carries an artificial source (bound_after_<e>)
    and cut the subtree of a history that can no longer reach the input.
    Driven on the host by Algorithm 2's loop: the valid leaves and the
    amplitudes are the oracle's (only invalid histories are cut), and on the
    walk the checks are present and fewer leaves complete."""
    spec = CASES[case]()
    circ, inputs, outputs = spec
    G = len(circ.gates)
    c1, c2 = G // 3, (2 * G) // 3
    got, completed, valid = _host_amplitudes(circ, inputs, outputs, c1, c2, 0.0, str(tmp_path), bound=True)
    want, cnt = feynman.run(circ, inputs, outputs, c1=c1, c2=c2)
    _close(got, want)
    assert np.array_equal(valid, cnt["valid"].astype(np.int64))
    assert np.all(completed <= cnt["completed"].astype(np.int64))
    if case == "walk":
        C = fs.Circuit(circ)
        C.set_input(inputs)
        b = fs.Batch(split="fixed", c1=c1, c2=c2)
        b.add(C, outputs)
        b.set_exact_bound(0)
        b.plan()
        assert "if (bound_after_" in b.generated_source()
        assert completed.sum() < cnt["completed"].sum()


@pytest.mark.parametrize("family", ["aa", "qaoa", "random"])
def test_stacked_suffix_in_exact_mode_checkpoints_the_class_counts(family, tmp_path):
    """Exact jobs with ten or more sources in the suffix (one per op) run
    it as per-source segments too; the deferred class counts (and the
    commensurate phase) are checkpointed with the state after every segment
    and restored at the restart.  Driven on the host by the device's restart
    loop: amplitudes and leaf counts are the oracle's."""
    if family == "aa":
        w = aa_workload(n=4, iters=2, all_outputs=True)
        circ, inputs, outputs = w.circuit, w.inputs, w.outputs[:6]
    elif family == "qaoa":
        w = qaoa_workload(8, 2, n_out=6, seed=5)
        circ, inputs, outputs = w.circuit, w.inputs, w.outputs
    else:
        circ = random_small_circuit(10, 90, 9129)    # one source per op after the cut
        rng = SplitMix64(9129)
        inputs = [(rng.bits(10), 0.8), (rng.bits(10), 0.6j)]
        outputs = [rng.bits(10) for _ in range(5)]
    C = fs.Circuit(circ)
    srcs = {s_: g for g, q, s_ in C.branch_vars() if s_ >= 0}
    G = len(circ.gates)
    A = len(srcs)
    c1 = G - srcs[A // 4 - 1]
    c2 = G - srcs[A // 4]                          # one source in the root, the rest in the suffix
    assert A - A // 4 - 1 >= 10
    got, completed, valid = _host_amplitudes(circ, inputs, outputs, c1, c2, 0.0, str(tmp_path))
    assert _host_amplitudes.stacked
    want, cnt = feynman.run(circ, inputs, outputs, c1=c1, c2=c2)
    _close(got, want)
    assert np.array_equal(completed, cnt["completed"].astype(np.int64))
    assert np.array_equal(valid, cnt["valid"].astype(np.int64))
    if family != "random":
        assert np.abs(want).max() > 1e-3


@pytest.mark.parametrize("iters,a_s", [(1, 4), (2, 8), (2, 12)])
def test_phase_census_of_unit_phase_suffixes(iters, a_s, tmp_path):
    """Exact suffixes whose factors are all unit phases (amplitude
    amplification: H, Toffoli, the marking and diffusion signs) count their
    valid leaves by phase: suffix_q returns each leaf's quarter turns q and
    the root adds amp * ((n0 - n2) + i (n1 - n3)).  Driven on the host by
    Algorithm 2's loop: amplitudes within 1e-12 / 1e-10 of the oracle, leaf
    counts exact."""
    w = aa_workload(n=4, iters=iters, all_outputs=True)
    circ, inputs, outputs = w.circuit, w.inputs, w.outputs[:8]
    C = fs.Circuit(circ)
    srcs = {s_: g for g, q, s_ in C.branch_vars() if s_ >= 0}
    G = len(circ.gates)
    A = len(srcs)
    c1 = c2 = G - srcs[A - a_s - 1]              # a_s sources in the suffix
    got, completed, valid = _host_amplitudes(circ, inputs, outputs, c1, c2, 0.0, str(tmp_path), census=True)
    assert _host_amplitudes.census
    assert _host_amplitudes.stacked == (a_s >= 10)
    want, cnt = feynman.run(circ, inputs, outputs, c1=c1, c2=c2)
    _close(got, want)
    assert np.array_equal(completed, cnt["completed"].astype(np.int64))
    assert np.array_equal(valid, cnt["valid"].astype(np.int64))
    assert np.abs(want).max() > 0.05

// Host side of the library: circuit validation and gate matrices, the
// reduced-history analysis (Sec. IV-A), the evaluation-order program
// compiler, the Eq. 8 autotuner (Sec. IV-C) and the batch planner that lays
// out one device workspace for many jobs (Sec. IV-D, Observations 5-6).
#include <algorithm>
#include <array>
#include <cmath>
#include <complex>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/feynsparse.h"
#include "fs_internal.h"

using cd = std::complex<double>;
using u128 = unsigned __int128;

namespace fs {

bool find_cascade(const Op* ops, const uint32_t* masks, int W, int e, int e1, CascadeRun& r)
{
    const Op& o0 = ops[e];
    if (o0.code != OP_X && o0.code != OP_MCX) return false;
    std::memset(&r, 0, sizeof r);
    if (o0.code == OP_MCX)
        for (int j = 0; j < W; ++j) {
            r.cm[j] = masks[o0.aux2 + j];
            r.cv[j] = masks[o0.aux2 + W + j];
        }
    const int t0 = o0.q0;
    uint32_t field[4] = {0, 0, 0, 0};   // targets of the ops so far
    field[t0 >> 5] |= 1u << (t0 & 31);
    int len = 1, v = -1;
    while (e + len < e1) {
        const Op& o = ops[e + len];
        const int t = t0 + len;
        if (o.code != OP_MCX || t >= 32 * W || o.q0 != t) break;
        if ((r.cm[t >> 5] >> (t & 31)) & 1u) break;   // a common control on the new target
        const uint32_t* m = masks + o.aux2;
        bool ok = true;
        int pol = -1;
        for (int j = 0; j < W && ok; ++j) {
            ok = m[j] == (r.cm[j] | field[j]) && (m[W + j] & r.cm[j]) == r.cv[j];
            const uint32_t fv = m[W + j] & field[j];
            if (!field[j]) continue;
            const int pj = fv == field[j] ? 1 : fv == 0 ? 0 : -2;
            if (pj == -2 || (pol >= 0 && pj != pol)) ok = false;
            pol = pj;
        }
        if (!ok || (v >= 0 && pol != v)) break;
        v = pol;
        field[t >> 5] |= 1u << (t & 31);
        ++len;
    }
    if (len < 3) return false;
    r.len = len;
    r.t0 = t0;
    r.dec = v == 1;
    return true;
}

}  // namespace fs

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char* what)
{
    return fail(FS_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CUDA_TRY(call)                                      \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

enum Role { WP = 0, DET = 1, BR = 2 };

struct GateInfo {
    uint32_t kind = 0;
    int k = 1;                  // targets
    int q[2] = {0, 0};
    uint64_t cm[2] = {0, 0}, cv[2] = {0, 0};
    double theta = 0;
    cd u[16];                   // base matrix on the targets, u[out * dim + in]
    Role role = WP;
    int src[2] = {-2, -2};      // artificial source id, -1 natural, -2 not a branching input
};

struct Bits { uint64_t w[2] = {0, 0}; };

}  // namespace

struct fs_circuit {
    uint32_t n = 0;
    std::vector<GateInfo> g;
    int A = 0, n_natural = 0, n_bvars = 0;
    int n_wp = 0, n_det = 0, n_br = 0;
    std::vector<Bits> in_bits{Bits{}};
    std::vector<cd> in_coef{cd(1, 0)};
};

namespace {

// ------------------------------------------------------------------ gates

bool controllable(uint32_t k) { return k == FS_X || k == FS_Z || k == FS_P || k == FS_S || k == FS_T; }

int build_matrix(const fs_gate& in, GateInfo& g)
{
    const double t = in.theta, c = std::cos(t / 2.0), s = std::sin(t / 2.0);
    const double h = std::sqrt(0.5);
    for (auto& v : g.u) v = 0.0;
    g.k = 1;
    switch (in.kind) {
    case FS_H: g.u[0] = h; g.u[1] = h; g.u[2] = h; g.u[3] = -h; g.role = BR; break;
    case FS_X: g.u[1] = 1; g.u[2] = 1; g.role = DET; break;
    case FS_Y: g.u[1] = cd(0, -1); g.u[2] = cd(0, 1); g.role = DET; break;
    case FS_Z: g.u[0] = 1; g.u[3] = -1; g.role = WP; break;
    case FS_S: g.u[0] = 1; g.u[3] = cd(0, 1); g.role = WP; break;
    case FS_T: g.u[0] = 1; g.u[3] = cd(std::cos(M_PI / 4.0), std::sin(M_PI / 4.0)); g.role = WP; break;
    case FS_P: g.u[0] = 1; g.u[3] = cd(std::cos(t), std::sin(t)); g.role = WP; break;
    case FS_RX: g.u[0] = c; g.u[1] = cd(0, -s); g.u[2] = cd(0, -s); g.u[3] = c; g.role = BR; break;
    case FS_RY: g.u[0] = c; g.u[1] = -s; g.u[2] = s; g.u[3] = c; g.role = BR; break;
    case FS_RZ: g.u[0] = cd(c, -s); g.u[3] = cd(c, s); g.role = WP; break;
    case FS_RZZ:
        g.k = 2;
        g.u[0] = cd(c, -s); g.u[5] = cd(c, s); g.u[10] = cd(c, s); g.u[15] = cd(c, -s);
        g.role = WP;
        break;
    case FS_SWAP:
        g.k = 2;
        g.u[0] = 1; g.u[1 * 4 + 2] = 1; g.u[2 * 4 + 1] = 1; g.u[15] = 1;
        g.role = DET;
        break;
    case FS_U1:
    case FS_U2: {
        const int dim = in.kind == FS_U1 ? 2 : 4;
        g.k = in.kind == FS_U1 ? 1 : 2;
        for (int i = 0; i < dim * dim; ++i) g.u[i] = cd(in.m[2 * i], in.m[2 * i + 1]);
        double dev = 0;   // max |U^+U - I|
        for (int a = 0; a < dim; ++a)
            for (int b = 0; b < dim; ++b) {
                cd acc = 0;
                for (int r = 0; r < dim; ++r) acc += std::conj(g.u[r * dim + a]) * g.u[r * dim + b];
                dev = std::max(dev, std::abs(acc - cd(a == b ? 1.0 : 0.0)));
            }
        if (!(dev <= 1e-12)) return fail(FS_ERR_NONUNITARY, "explicit matrix is not unitary (|U^+U-I| = %g)", dev);
        // roles from the exact zero pattern
        bool diag = true, perm = true;
        for (int col = 0; col < dim; ++col) {
            int nz = 0;
            for (int row = 0; row < dim; ++row)
                if (g.u[row * dim + col] != cd(0, 0)) { ++nz; if (row != col) diag = false; }
            if (nz != 1) perm = false;
        }
        g.role = diag ? WP : (perm ? DET : BR);
        break;
    }
    default:
        return fail(FS_ERR_UNSUPPORTED, "unknown gate kind %u", in.kind);
    }
    return FS_OK;
}

// ------------------------------------------------------------------ analysis

// Natural vs artificial branching inputs, then artificial-source ids in
// backward-sweep order (Sec. IV-A).  A qubit's input wire runs until the
// first gate that may change its value (deterministic or branching target);
// a branching gate at exactly that point reads the input bit (natural
// source).  Every other branching input gets the next id as the sweep goes
// from the output back to the input.
void analyze_circuit(fs_circuit& C)
{
    const int G = (int)C.g.size();
    std::vector<int> first_write(C.n, G);
    for (int i = 0; i < G; ++i) {
        const GateInfo& g = C.g[i];
        if (g.role == WP) continue;
        for (int t = 0; t < g.k; ++t)
            if (first_write[g.q[t]] == G) first_write[g.q[t]] = i;
    }
    C.A = C.n_natural = C.n_bvars = C.n_wp = C.n_det = C.n_br = 0;
    for (int i = G - 1; i >= 0; --i) {
        GateInfo& g = C.g[i];
        (g.role == WP ? C.n_wp : g.role == DET ? C.n_det : C.n_br)++;
        g.src[0] = g.src[1] = -2;
        if (g.role != BR) continue;
        const int lo = (g.k == 2 && g.q[1] < g.q[0]) ? 1 : 0;
        for (int j = 0; j < g.k; ++j) {
            const int t = (j == 0) ? lo : 1 - lo;
            ++C.n_bvars;
            if (first_write[g.q[t]] == i) { g.src[t] = -1; ++C.n_natural; }
            else g.src[t] = C.A++;
        }
    }
}

// Sources among the ops at evaluation positions [0, e) for every e.
std::vector<int> source_prefix(const fs_circuit& C)
{
    const int G = (int)C.g.size();
    std::vector<int> pre(G + 1, 0);
    for (int e = 0; e < G; ++e) {
        const GateInfo& g = C.g[G - 1 - e];
        int a = 0;
        if (g.role == BR)
            for (int t = 0; t < g.k; ++t) a += g.src[t] >= 0;
        pre[e + 1] = pre[e] + a;
    }
    return pre;
}

u128 eq8(uint64_t Gp, uint64_t Gr, uint64_t Gs, int Ap, int Ar, int As)
{
    // 2^Ap (Gp + 2^Ar (Gr + 2^As Gs))
    const u128 one = 1;
    return (one << Ap) * ((u128)Gp + (one << Ar) * ((u128)Gr + (one << As) * (u128)Gs));
}

struct Split {
    int c1 = 0, c2 = 0, Ap = 0, Ar = 0, As = 0;
    u128 cost = 0;
};

Split split_at(const fs_circuit& C, const std::vector<int>& pre, int c1, int c2)
{
    const int G = (int)C.g.size();
    Split s;
    s.c1 = c1; s.c2 = c2;
    s.Ap = pre[c1]; s.Ar = pre[c2] - pre[c1]; s.As = pre[G] - pre[c2];
    s.cost = eq8((uint64_t)c1, (uint64_t)(c2 - c1), (uint64_t)(G - c2), s.Ap, s.Ar, s.As);
    return s;
}

// Autotuned partition: minimum of Eq. 8 over all cuts 0 <= c1 <= c2 <= G,
// subject to the checkpoint table fitting (Ap <= max_ap) and enough
// (prefix, root) items for the GPU (Ap + Ar >= min(min_apr, A)) and within
// index range (Ap + Ar <= max_apr).  Ties: smallest c1, then smallest c2.
bool autotune(const fs_circuit& C, int max_ap, int min_apr, int max_apr, Split& best)
{
    const int G = (int)C.g.size();
    const std::vector<int> pre = source_prefix(C);
    const int need = std::min(min_apr, C.A);
    bool found = false;
    for (int c1 = 0; c1 <= G && pre[c1] <= max_ap; ++c1) {
        for (int c2 = c1; c2 <= G; ++c2) {
            const int apr = pre[c2];
            if (apr < need) continue;
            if (apr > max_apr) break;
            const Split s = split_at(C, pre, c1, c2);
            if (!found || s.cost < best.cost) { best = s; found = true; }
        }
    }
    return found;
}

int ilog2_floor(uint64_t v) { int r = -1; while (v) { v >>= 1; ++r; } return r; }
int ilog2_ceil(uint64_t v) { int r = 0; while ((1ull << r) < v && r < 63) ++r; return r; }

// ------------------------------------------------------------------ program

struct Program {
    std::vector<fs::Op> ops;
    std::vector<uint32_t> masks;
    std::vector<double2> fac;
};

uint32_t push_fac(Program& P, std::initializer_list<cd> v)
{
    const uint32_t off = (uint32_t)P.fac.size();
    for (const cd& z : v) P.fac.push_back(make_double2(z.real(), z.imag()));
    return off;
}

uint32_t push_mask(Program& P, int W, const uint64_t m[2], const uint64_t v[2])
{
    const uint32_t off = (uint32_t)P.masks.size();
    for (int j = 0; j < W; ++j) P.masks.push_back((uint32_t)(m[j >> 1] >> (32 * (j & 1))));
    for (int j = 0; j < W; ++j) P.masks.push_back((uint32_t)(v[j >> 1] >> (32 * (j & 1))));
    return off;
}

// Emits the ops in evaluation (output-to-input) order.  An artificial source
// with id k in a region whose ids are [k0, k0 + a) takes bit a - 1 - (k - k0)
// of that region's enumeration word: the first source met is the most
// significant bit, so a cut subtree is a contiguous range of h.
void compile(const fs_circuit& C, int W, const Split& sp, Program& P)
{
    const int G = (int)C.g.size();
    P.ops.clear(); P.masks.clear(); P.fac.clear();
    P.ops.reserve(G);
    auto region_bit = [&](int e, int k) -> int {
        int k0, a;
        if (e < sp.c1) { k0 = 0; a = sp.Ap; }
        else if (e < sp.c2) { k0 = sp.Ap; a = sp.Ar; }
        else { k0 = sp.Ap + sp.Ar; a = sp.As; }
        return a - 1 - (k - k0);
    };
    for (int e = 0; e < G; ++e) {
        const GateInfo& g = C.g[G - 1 - e];
        fs::Op op;
        std::memset(&op, 0, sizeof op);
        op.q0 = (uint8_t)g.q[0];
        op.q1 = (uint8_t)(g.k == 2 ? g.q[1] : 0);
        op.s0 = op.s1 = -1;
        const bool ctl = (g.cm[0] | g.cm[1]) != 0;
        const int dim = g.k == 1 ? 2 : 4;
        if (g.role == WP) {
            if (g.kind == FS_Z || g.kind == FS_S || g.kind == FS_T || g.kind == FS_P) {
                if (ctl) {
                    uint64_t m[2] = {g.cm[0], g.cm[1]}, v[2] = {g.cv[0], g.cv[1]};
                    m[g.q[0] >> 6] |= 1ull << (g.q[0] & 63);
                    v[g.q[0] >> 6] |= 1ull << (g.q[0] & 63);
                    op.aux2 = push_mask(P, W, m, v);
                    if (g.kind == FS_Z) op.code = fs::OP_MCNEG;
                    else { op.code = fs::OP_MCPH; op.aux = push_fac(P, {g.u[3]}); }
                } else if (g.kind == FS_Z) {
                    op.code = fs::OP_NEG1;
                } else {
                    op.code = fs::OP_PH1;
                    op.aux = push_fac(P, {g.u[3]});
                }
            } else if (g.k == 1) {
                op.code = fs::OP_DIAG1;
                op.aux = push_fac(P, {g.u[0], g.u[3]});
            } else {
                op.code = fs::OP_DIAG2;
                op.aux = push_fac(P, {g.u[0], g.u[5], g.u[10], g.u[15]});
            }
        } else if (g.role == DET) {
            if (g.kind == FS_X) {
                if (ctl) {
                    op.code = fs::OP_MCX;
                    op.aux2 = push_mask(P, W, g.cm, g.cv);
                } else {
                    op.code = fs::OP_X;
                }
            } else if (g.kind == FS_SWAP) {
                op.code = fs::OP_SWAP;
            } else if (g.k == 1) {
                // antidiagonal: output o came from input 1 - o
                op.code = fs::OP_PERM1;
                op.aux = push_fac(P, {g.u[0 * 2 + 1], g.u[1 * 2 + 0]});
            } else {
                op.code = fs::OP_PERM2;
                cd f[4];
                uint32_t packed = 0;
                for (int o = 0; o < 4; ++o) {
                    int in = 0;
                    for (int c = 0; c < 4; ++c)
                        if (g.u[o * 4 + c] != cd(0, 0)) { in = c; break; }
                    f[o] = g.u[o * 4 + in];
                    packed |= (uint32_t)in << (2 * o);
                }
                op.aux = push_fac(P, {f[0], f[1], f[2], f[3]});
                op.aux2 = packed;
            }
        } else {
            if (g.src[0] >= 0) op.s0 = (int8_t)region_bit(e, g.src[0]);
            if (g.k == 2 && g.src[1] >= 0) op.s1 = (int8_t)region_bit(e, g.src[1]);
            if (g.kind == FS_H) {
                op.code = fs::OP_H;
            } else if (g.k == 1) {
                op.code = fs::OP_BR1;
                op.aux = push_fac(P, {g.u[0], g.u[1], g.u[2], g.u[3]});
            } else {
                op.code = fs::OP_BR2;
                op.aux = (uint32_t)P.fac.size();
                for (int i = 0; i < 16; ++i) P.fac.push_back(make_double2(g.u[i].real(), g.u[i].imag()));
            }
        }
        (void)dim;
        P.ops.push_back(op);
    }
}

int words_for(uint32_t n) { const int w = (int)((n + 31) / 32); return w <= 1 ? 1 : (w == 2 ? 2 : 4); }

// ------------------------------------------------------------------ batch

struct Job {
    fs_circuit* c = nullptr;
    std::vector<Bits> outs;
    std::vector<Bits> ins;
    std::vector<cd> coef;
    double eps = 0;
    // plan
    Split sp;
    Program prog;
    int W = 1;
    uint64_t pairs = 0, n_tiles = 0, table_entries = 0, n_partials = 0;
    int log2_ipp = 0, log2_spp = 0;
    // offsets in the workspace
    size_t o_ops = 0, o_masks = 0, o_fac = 0, o_outs = 0, o_ins = 0, o_coef = 0, o_table = 0, o_part = 0;
    // optional: per-item subtree sums (caller device buffer) and learned pruner
    double2* d_log = nullptr;
    unsigned long long* d_trace = nullptr;   // per output {completed, valid} (caller device buffer)
    const float* d_pruner = nullptr;
    float tau = 0;
    fs::FeatureSpec fspec{};
    // pruned jobs (eps > 0, a learned pruner or the exact bound) run over
    // compacted live entries
    bool compact = false;
    bool direct = false;   // empty prefix region, exact: entries read as (b_out, 1), no table
    std::vector<std::pair<int, fs::BoundSpec>> src_bounds;   // bound after each source op of root and suffix
    bool bound = false;                   // exact reachability bound at the checkpoint
    fs::BoundSpec bspec{};
    int fixed_c1 = -1, fixed_c2 = -1;     // per-job cuts overriding the batch split
    std::vector<fs::PrefixLevel> levels;  // per-source prefix expansion (empty: single region)
    double2 scale = make_double2(1.0, 0.0);   // constant left out by the generated root and suffix
    size_t o_lvscratch = 0;
    size_t o_live = 0, o_esum = 0, o_blk = 0, o_prange = 0;
    uint64_t nblk = 0;
    bool fused = false;    // outputs reduced by the generated compacted history (no reduction launch)
    size_t o_odone = 0;    // per output: subtree sums stored so far (zeroed at the start of every run)
};

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// An exact compacted job of the straight-line engine whose warps of 32
// (live entry, h_r) items each store one subtree sum (A_r >= 5) reduces its
// own outputs: the warp that stores an output's last sum adds them (Eq. 2),
// with a warp per output, when an output has at most RED_BIG_ITEMS sums and
// fewer than 32 input states.
template <class B, class J> bool fused_reduction_of(const B& b, const J& j)
{
    if (b.opt.engine != 0 || !j.compact || j.eps != 0.0 || j.sp.Ar < 5 || j.outs.empty() || j.ins.size() >= 32)
        return false;
    const long double per_out = std::ldexp((long double)j.ins.size(), j.sp.Ap + j.sp.Ar - 5);
    return per_out <= (long double)fs::RED_BIG_ITEMS;
}

// Makes a device current for the lifetime of the guard and restores the
// caller's device afterwards (no-op for device < 0 or when it already is).
struct DeviceGuard {
    int prev = -1;
    cudaError_t err = cudaSuccess;
    explicit DeviceGuard(int device)
    {
        if (device < 0) return;
        int cur = 0;
        err = cudaGetDevice(&cur);
        if (err != cudaSuccess || cur == device) return;
        err = cudaSetDevice(device);
        if (err == cudaSuccess) prev = cur;
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

}  // namespace

struct fs_batch {
    std::vector<Job> jobs;
    fs_options opt{};
    bool planned = false, uploaded = false;
    size_t ws_bytes = 0;
    size_t o_jobs = 0, o_pbegin = 0, o_obegin = 0, o_tiles = 0, o_stats = 0, o_counter = 0, o_err = 0;
    size_t o_bigcount = 0, o_biglist = 0;   // outputs left to the block-per-output reduction
    size_t static_bytes = 0, dyn_begin = 0;
    std::vector<unsigned char> host_static;
    // repeated uploads stage through pinned memory (asynchronous copy; the
    // event guards the buffer until the previous copy has finished)
    unsigned char* h_pinned = nullptr;
    size_t h_pinned_bytes = 0;
    cudaEvent_t up_ev = nullptr;
    bool up_pending = false;
    uint64_t n_uploads = 0;
    bool image_valid = false;     // h_pinned holds this plan's image for image_ws
    void* image_ws = nullptr;
    unsigned char* h_words = nullptr;   // pinned copy of the counters and error word
    size_t h_words_bytes = 0;
    uint64_t n_finishes = 0;
    bool no_host_alloc = false;         // set by the allocation-free entry point
    int device = -1;                    // CUDA device of the batch (-1: the caller's current one)
    std::vector<uint2> tiles;
    uint64_t total_prefix = 0, total_out = 0;
    int grid = 0, compact_grid = 0;
    void* uploaded_ws = nullptr;
    bool timing = false;
    cudaEvent_t ev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    bool ev_recorded = false;
    void* jit = nullptr;          // generated straight-line module (engine 0)
    double jit_ms = 0;
    void drop_jit()
    {
        if (jit) fs::jit_release(jit);
        jit = nullptr;
        for (Job& j : jobs) j.scale = make_double2(1.0, 0.0);
    }
    ~fs_batch()
    {
        for (auto& e : ev) if (e) cudaEventDestroy(e);
        if (up_ev) {
            if (up_pending) cudaEventSynchronize(up_ev);
            cudaEventDestroy(up_ev);
        }
        if (h_pinned) cudaFreeHost(h_pinned);
        if (h_words) cudaFreeHost(h_words);
        drop_jit();
    }
};

void fs::batch_forbid_host_alloc(fs_batch* b)
{
    if (b) b->no_host_alloc = true;
}

int fs::set_error(int code, const char* msg)
{
    g_err = msg;
    return code;
}

extern "C" {

const char* fs_last_error(void) { return g_err.c_str(); }

const char* fs_version(void) { return "feynsparse 0.1 (sm_103a)"; }

int fs_circuit_create(const fs_gate* gates, size_t n_gates, uint32_t n_qubits, fs_circuit** out)
{
    if (!out) return fail(FS_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (n_qubits == 0) return fail(FS_ERR_INVALID, "n_qubits must be >= 1");
    if (n_qubits > FS_MAX_QUBITS) return fail(FS_ERR_TOO_MANY_QUBITS, "n_qubits %u > %d", n_qubits, FS_MAX_QUBITS);
    if (n_gates && !gates) return fail(FS_ERR_INVALID, "gates is NULL");
    if (n_gates > (1u << 24)) return fail(FS_ERR_TOO_LARGE, "too many gates");
    std::unique_ptr<fs_circuit> C(new (std::nothrow) fs_circuit);
    if (!C) return fail(FS_ERR_NOMEM, "out of host memory");
    C->n = n_qubits;
    C->g.resize(n_gates);
    const uint64_t valid_mask[2] = {n_qubits >= 64 ? ~0ull : ((1ull << n_qubits) - 1),
                                    n_qubits >= 128 ? ~0ull : (n_qubits > 64 ? ((1ull << (n_qubits - 64)) - 1) : 0ull)};
    for (size_t i = 0; i < n_gates; ++i) {
        const fs_gate& in = gates[i];
        GateInfo& g = C->g[i];
        g.kind = in.kind;
        const int rc = build_matrix(in, g);
        if (rc) return fail(rc, "gate %zu: %s", i, g_err.c_str());
        const uint32_t want_q = (in.kind == FS_RZZ || in.kind == FS_SWAP || in.kind == FS_U2) ? 2u : 1u;
        if (in.n_q != want_q) return fail(FS_ERR_INVALID, "gate %zu: kind %u takes %u target(s), n_q = %u", i, in.kind, want_q, in.n_q);
        for (uint32_t t = 0; t < want_q; ++t)
            if (in.q[t] >= n_qubits) return fail(FS_ERR_INVALID, "gate %zu: qubit %u out of range", i, in.q[t]);
        if (want_q == 2 && in.q[0] == in.q[1]) return fail(FS_ERR_INVALID, "gate %zu: repeated target qubit", i);
        g.q[0] = (int)in.q[0];
        g.q[1] = want_q == 2 ? (int)in.q[1] : 0;
        g.cm[0] = in.ctrl_mask[0]; g.cm[1] = in.ctrl_mask[1];
        g.cv[0] = in.ctrl_val[0]; g.cv[1] = in.ctrl_val[1];
        g.theta = in.theta;
        if ((g.cm[0] | g.cm[1]) && !controllable(in.kind))
            return fail(FS_ERR_UNSUPPORTED, "gate %zu: controls are allowed on X, Z, P, S, T only", i);
        if ((g.cm[0] & ~valid_mask[0]) || (g.cm[1] & ~valid_mask[1]))
            return fail(FS_ERR_INVALID, "gate %zu: control qubit out of range", i);
        if ((g.cv[0] & ~g.cm[0]) || (g.cv[1] & ~g.cm[1]))
            return fail(FS_ERR_INVALID, "gate %zu: control value outside the control mask", i);
        for (uint32_t t = 0; t < want_q; ++t)
            if ((g.cm[g.q[t] >> 6] >> (g.q[t] & 63)) & 1ull)
                return fail(FS_ERR_INVALID, "gate %zu: a target is also a control", i);
    }
    analyze_circuit(*C);
    *out = C.release();
    return FS_OK;
}

int fs_circuit_destroy(fs_circuit* c)
{
    delete c;
    return FS_OK;
}

static int check_bits(const fs_circuit* c, const uint64_t* b, const char* what)
{
    const uint32_t n = c->n;
    const uint64_t hi0 = n >= 64 ? 0 : ~((1ull << n) - 1);
    const uint64_t hi1 = n >= 128 ? 0 : (n <= 64 ? ~0ull : ~((1ull << (n - 64)) - 1));
    if ((b[0] & hi0) || (b[1] & hi1)) return fail(FS_ERR_INVALID, "%s has bits beyond qubit %u", what, n - 1);
    return FS_OK;
}

int fs_analyze(fs_circuit* c, const uint64_t* input_bits, fs_analysis* out)
{
    if (!c || !input_bits || !out) return fail(FS_ERR_INVALID, "NULL argument");
    if (int rc = check_bits(c, input_bits, "input")) return rc;
    c->in_bits.assign(1, Bits{});
    c->in_bits[0].w[0] = input_bits[0];
    c->in_bits[0].w[1] = input_bits[1];
    c->in_coef.assign(1, cd(1, 0));
    std::memset(out, 0, sizeof *out);
    out->n_qubits = c->n;
    out->n_gates = (uint32_t)c->g.size();
    out->n_branch_vars = (uint32_t)c->n_bvars;
    out->n_natural = (uint32_t)c->n_natural;
    out->A = (uint32_t)c->A;
    out->n_wp = (uint32_t)c->n_wp;
    out->n_det = (uint32_t)c->n_det;
    out->n_br = (uint32_t)c->n_br;
    // one output, default budget
    const int max_ap = ilog2_floor((4ull << 30) / 32);
    const int min_apr = ilog2_ceil(1ull << 19);
    const int max_apr = ilog2_floor(1ull << 28);
    Split s;
    if (!autotune(*c, max_ap, min_apr, max_apr, s)) return fail(FS_ERR_TOO_LARGE, "no admissible partition");
    out->c1 = s.c1; out->c2 = s.c2;
    const int G = (int)c->g.size();
    out->G_p = (uint32_t)s.c1; out->G_r = (uint32_t)(s.c2 - s.c1); out->G_s = (uint32_t)(G - s.c2);
    out->A_p = (uint32_t)s.Ap; out->A_r = (uint32_t)s.Ar; out->A_s = (uint32_t)s.As;
    out->gateops_lo = (uint64_t)s.cost;
    out->gateops_hi = (uint64_t)(s.cost >> 64);
    out->max_ap = (uint32_t)max_ap;
    out->min_apr = (uint32_t)min_apr;
    out->max_apr = (uint32_t)max_apr;
    return FS_OK;
}

int fs_branch_vars(const fs_circuit* c, int32_t* gate_index, int32_t* qubit, int32_t* source,
                   size_t cap, size_t* count)
{
    if (!c || !count) return fail(FS_ERR_INVALID, "NULL argument");
    size_t k = 0;
    for (int i = (int)c->g.size() - 1; i >= 0; --i) {
        const GateInfo& g = c->g[i];
        if (g.role != BR) continue;
        const int lo = (g.k == 2 && g.q[1] < g.q[0]) ? 1 : 0;
        for (int j = 0; j < g.k; ++j) {
            const int t = (j == 0) ? lo : 1 - lo;
            if (k < cap) {
                if (gate_index) gate_index[k] = i;
                if (qubit) qubit[k] = g.q[t];
                if (source) source[k] = g.src[t];
            }
            ++k;
        }
    }
    *count = k;
    return FS_OK;
}

int fs_set_input(fs_circuit* c, const uint64_t* support_bits, const double* coeffs, size_t S)
{
    if (!c || (S && (!support_bits || !coeffs))) return fail(FS_ERR_INVALID, "NULL argument");
    if (S == 0) return fail(FS_ERR_INVALID, "empty input support");
    if (S > (1u << 20)) return fail(FS_ERR_TOO_LARGE, "input support too large");
    std::vector<Bits> b(S);
    std::vector<cd> co(S);
    for (size_t i = 0; i < S; ++i) {
        if (int rc = check_bits(c, support_bits + 2 * i, "input support")) return rc;
        b[i].w[0] = support_bits[2 * i];
        b[i].w[1] = support_bits[2 * i + 1];
        co[i] = cd(coeffs[2 * i], coeffs[2 * i + 1]);
    }
    c->in_bits.swap(b);
    c->in_coef.swap(co);
    return FS_OK;
}

int fs_batch_create(fs_batch** out)
{
    if (!out) return fail(FS_ERR_INVALID, "out is NULL");
    *out = new (std::nothrow) fs_batch;
    if (!*out) return fail(FS_ERR_NOMEM, "out of host memory");
    return FS_OK;
}

int fs_batch_destroy(fs_batch* b)
{
    delete b;
    return FS_OK;
}

int fs_batch_set_options(fs_batch* b, const fs_options* opt)
{
    if (!b) return fail(FS_ERR_INVALID, "NULL batch");
    if (opt) {
        if (opt->split > 2) return fail(FS_ERR_INVALID, "split must be 0, 1 or 2");
        if (opt->engine > 1) return fail(FS_ERR_INVALID, "engine must be 0 or 1");
        if (opt->prefix_mode > 2) return fail(FS_ERR_INVALID, "prefix_mode must be 0, 1 or 2");
        b->opt = *opt;
    } else {
        std::memset(&b->opt, 0, sizeof b->opt);
    }
    b->planned = b->uploaded = false;
    b->drop_jit();
    return FS_OK;
}

int fs_batch_add(fs_batch* b, fs_circuit* c, const uint64_t* outputs, size_t n_out, double eps,
                 uint32_t* job_id)
{
    if (!b || !c || (n_out && !outputs)) return fail(FS_ERR_INVALID, "NULL argument");
    if (!(eps >= 0.0) || std::isinf(eps)) return fail(FS_ERR_INVALID, "eps must be finite and >= 0");
    if (n_out > (1u << 26)) return fail(FS_ERR_TOO_LARGE, "too many outputs in one job");
    if (b->jobs.size() >= 4096) return fail(FS_ERR_TOO_LARGE, "too many jobs in one batch");
    Job j;
    j.c = c;
    j.outs.resize(n_out);
    for (size_t i = 0; i < n_out; ++i) {
        if (int rc = check_bits(c, outputs + 2 * i, "output")) return rc;
        j.outs[i].w[0] = outputs[2 * i];
        j.outs[i].w[1] = outputs[2 * i + 1];
    }
    j.ins = c->in_bits;
    j.coef = c->in_coef;
    j.eps = eps;
    b->jobs.push_back(std::move(j));
    if (job_id) *job_id = (uint32_t)(b->jobs.size() - 1);
    b->planned = b->uploaded = false;
    return FS_OK;
}

int fs_batch_log_subtrees(fs_batch* b, uint32_t job, double* d_log)
{
    if (!b) return fail(FS_ERR_INVALID, "NULL batch");
    if (job >= b->jobs.size()) return fail(FS_ERR_INVALID, "job %u out of range", job);
    b->jobs[job].d_log = (double2*)d_log;
    b->uploaded = false;
    return FS_OK;
}

int fs_batch_trace_outputs(fs_batch* b, uint32_t job, uint64_t* d_counts)
{
    if (!b) return fail(FS_ERR_INVALID, "NULL batch");
    if (job >= b->jobs.size()) return fail(FS_ERR_INVALID, "job %u out of range", job);
    if (((uintptr_t)d_counts) & 7) return fail(FS_ERR_INVALID, "counters must be 8-byte aligned");
    b->jobs[job].d_trace = (unsigned long long*)d_counts;
    b->uploaded = false;
    return FS_OK;
}

int fs_batch_log_items(const fs_batch* b, uint32_t job, uint64_t* items)
{
    if (!b || !items) return fail(FS_ERR_INVALID, "NULL argument");
    if (!b->planned) return fail(FS_ERR_STATE, "fs_batch_plan must come first");
    if (job >= b->jobs.size()) return fail(FS_ERR_INVALID, "job %u out of range", job);
    *items = b->jobs[job].pairs << b->jobs[job].log2_ipp;
    return FS_OK;
}

int fs_batch_set_cuts(fs_batch* b, uint32_t job, int32_t c1, int32_t c2)
{
    if (!b) return fail(FS_ERR_INVALID, "NULL batch");
    if (job >= b->jobs.size()) return fail(FS_ERR_INVALID, "job %u out of range", job);
    if ((c1 < 0) != (c2 < 0) || (c1 >= 0 && c2 < c1)) return fail(FS_ERR_INVALID, "cuts must satisfy 0 <= c1 <= c2 (or both -1)");
    b->jobs[job].fixed_c1 = c1;
    b->jobs[job].fixed_c2 = c2;
    b->planned = b->uploaded = false;
    b->drop_jit();
    return FS_OK;
}

int fs_batch_set_pruner(fs_batch* b, uint32_t job, const float* d_params, float tau)
{
    if (!b) return fail(FS_ERR_INVALID, "NULL batch");
    if (job >= b->jobs.size()) return fail(FS_ERR_INVALID, "job %u out of range", job);
    b->jobs[job].d_pruner = d_params;
    b->jobs[job].tau = tau;
    b->planned = b->uploaded = false;   // the job's layout changes: plan again
    b->drop_jit();
    return FS_OK;
}

int fs_batch_set_exact_bound(fs_batch* b, uint32_t job, int32_t enable)
{
    if (!b) return fail(FS_ERR_INVALID, "NULL batch");
    if (job >= b->jobs.size()) return fail(FS_ERR_INVALID, "job %u out of range", job);
    b->jobs[job].bound = enable != 0;
    b->planned = b->uploaded = false;   // the job's layout changes: plan again
    b->drop_jit();
    return FS_OK;
}

int fs_batch_features(fs_batch* b, uint32_t job, void* d_ws, float* d_features, void* stream)
{
    if (!b || !d_ws || !d_features) return fail(FS_ERR_INVALID, "NULL argument");
    DeviceGuard dg_(b->device);
    if (dg_.err != cudaSuccess) return cuda_fail(dg_.err, "cudaSetDevice(batch device)");
    if (!b->uploaded || b->uploaded_ws != d_ws) return fail(FS_ERR_STATE, "no run on this workspace");
    if (job >= b->jobs.size()) return fail(FS_ERR_INVALID, "job %u out of range", job);
    const Job& j = b->jobs[job];
    if (j.direct) return fail(FS_ERR_UNSUPPORTED, "job %u has no checkpoint table (empty prefix region)", job);
    const fs::JobDev* jobs = (const fs::JobDev*)((unsigned char*)d_ws + b->o_jobs);
    CUDA_TRY(fs::mlp_features(jobs, (int)job, j.fspec, d_features, j.table_entries, (cudaStream_t)stream));
    return FS_OK;
}

int fs_mlp_forward(const float* d_params, const float* d_x, uint64_t n, float* d_y, void* stream)
{
    if (!d_params || (n && (!d_x || !d_y))) return fail(FS_ERR_INVALID, "NULL argument");
    if (((uintptr_t)d_x) & 15) return fail(FS_ERR_INVALID, "feature rows must be 16-byte aligned");
    CUDA_TRY(fs::mlp_prepare());
    CUDA_TRY(fs::mlp_forward(d_params, d_x, (long long)n, d_y, (cudaStream_t)stream));
    return FS_OK;
}

int fs_mlp_grad(const float* d_params, const float* d_x, const float* d_target, uint64_t n, float* d_grad,
                void* stream)
{
    if (!d_params || !d_grad || (n && (!d_x || !d_target))) return fail(FS_ERR_INVALID, "NULL argument");
    CUDA_TRY(fs::mlp_grad(d_params, d_x, d_target, (long long)n, d_grad, (cudaStream_t)stream));
    return FS_OK;
}

int fs_mlp_adam(float* d_params, float* d_m, float* d_v, const float* d_grad, float lr, int32_t step, void* stream)
{
    if (!d_params || !d_m || !d_v || !d_grad) return fail(FS_ERR_INVALID, "NULL argument");
    if (step < 1) return fail(FS_ERR_INVALID, "Adam step counts from 1");
    CUDA_TRY(fs::mlp_adam(d_params, d_m, d_v, d_grad, lr, step, (cudaStream_t)stream));
    return FS_OK;
}

int fs_batch_upload_bytes(const fs_batch* b, size_t* bytes)
{
    if (!b || !bytes) return fail(FS_ERR_INVALID, "NULL argument");
    if (!b->planned) return fail(FS_ERR_STATE, "fs_batch_plan must come first");
    *bytes = b->static_bytes;
    return FS_OK;
}

int fs_batch_engine(const fs_batch* b, uint32_t* engine, double* compile_ms)
{
    if (!b || !engine) return fail(FS_ERR_INVALID, "NULL argument");
    if (!b->uploaded) return fail(FS_ERR_STATE, "fs_batch_upload must come first");
    *engine = b->jit ? 0u : 1u;
    if (compile_ms) *compile_ms = b->jit ? b->jit_ms : 0.0;
    return FS_OK;
}

int fs_batch_total_outputs(const fs_batch* b, size_t* n)
{
    if (!b || !n) return fail(FS_ERR_INVALID, "NULL argument");
    size_t t = 0;
    for (const Job& j : b->jobs) t += j.outs.size();
    *n = t;
    return FS_OK;
}

static void region_work(const Job& j, int e0, int e1, double& iops, double& fops, int dfrom, bool fused,
                        bool hoisted = false);
static int job_defer_from(const Job& j, bool straight);
static bool make_bound(Job& j, int n_qubits);

// Rates of the prefix cost model (work-model integer ops and FP64
// instructions per second, HBM bytes per second, seconds per launch),
// measured on B300 for the history and prefix kernels.
constexpr double kModelIntOps = 2.5e13, kModelFp64Ops = 5.0e11, kModelBytes = 5.0e12, kModelLaunch = 4.0e-6;

int fs_batch_plan(fs_batch* b, size_t* workspace_bytes)
{
    if (!b || !workspace_bytes) return fail(FS_ERR_INVALID, "NULL argument");
    DeviceGuard dg_(b->device);
    if (dg_.err != cudaSuccess) return cuda_fail(dg_.err, "cudaSetDevice(batch device)");
    const uint64_t budget = b->opt.table_budget_bytes ? b->opt.table_budget_bytes : (4ull << 30);
    const uint64_t max_items = b->opt.max_items ? b->opt.max_items : (1ull << 28);
    // the parallelism floor never exceeds the ceiling
    const uint64_t min_items = std::min<uint64_t>(b->opt.min_items ? b->opt.min_items : (1ull << 19), max_items);
    // table budget shared by the jobs in proportion to their pair counts
    uint64_t all_pairs = 0;
    for (Job& j : b->jobs) all_pairs += (uint64_t)j.outs.size() * j.ins.size();
    b->tiles.clear();
    b->total_prefix = 0;
    b->total_out = 0;
    struct TileCost { double cost; uint32_t job; };
    std::vector<TileCost> order;
    for (size_t ji = 0; ji < b->jobs.size(); ++ji) {
        Job& j = b->jobs[ji];
        const fs_circuit& C = *j.c;
        // exact jobs enumerate 2^A histories per pair; a threshold lets the
        // suffix skip cut subtrees, so only each region's word must fit
        if (C.A > 62 && j.eps == 0.0)
            return fail(FS_ERR_TOO_LARGE, "job %zu: A = %d artificial sources: 2^A histories cannot be enumerated "
                                          "exactly (a threshold eps > 0 allows up to 102)", ji, C.A);
        j.W = words_for(C.n);
        j.pairs = (uint64_t)j.outs.size() * j.ins.size();
        const int G = (int)C.g.size();
        const std::vector<int> pre = source_prefix(C);
        if (j.fixed_c1 >= 0) {
            const int c1 = j.fixed_c1, c2 = j.fixed_c2;
            if (c2 < c1 || c2 > G) return fail(FS_ERR_INVALID, "job %zu: cuts (%d, %d) outside [0, %d]", ji, c1, c2, G);
            j.sp = split_at(C, pre, c1, c2);
        } else if (b->opt.split == 1) {
            const int c1 = b->opt.c1, c2 = b->opt.c2;
            if (c1 < 0 || c2 < c1 || c2 > G) return fail(FS_ERR_INVALID, "job %zu: fixed cuts (%d, %d) outside [0, %d]", ji, c1, c2, G);
            j.sp = split_at(C, pre, c1, c2);
        } else if (b->opt.split == 2) {
            // Algorithm 1: no checkpoints.  The whole circuit is one region
            // enumerated over h (one item per assignment) when the index
            // range allows, else one item per pair looping over h.
            const int lp = ilog2_ceil(std::max<uint64_t>(j.pairs, 1));
            j.sp = (C.A + lp <= 40) ? split_at(C, pre, 0, G) : split_at(C, pre, 0, 0);
        } else {
            const uint64_t share = all_pairs ? (uint64_t)((long double)budget * j.pairs / all_pairs) : budget;
            // pruned jobs also keep a compacted live list (8 B per entry)
            const uint64_t entry_bytes = sizeof(fs::Entry) + ((j.eps > 0.0 || j.d_pruner || j.bound) ? 8 : 0);
            const uint64_t per_pair = j.pairs ? share / (j.pairs * entry_bytes) : share;
            const int max_ap = per_pair ? std::min(ilog2_floor(per_pair), 40) : 0;
            const int min_apr = j.pairs ? ilog2_ceil((min_items + j.pairs - 1) / j.pairs) : 0;
            int max_apr = std::max(0, std::min(40, ilog2_floor(max_items)) -
                                      ilog2_ceil(std::max<uint64_t>(j.pairs, 1)));
            // with a threshold most (prefix, root) items of a live entry are
            // cut at the first sources of the root: the root adds no more
            // assignments than the parallelism floor needs, and the suffix
            // enumerates the rest, skipping cut subtrees
            if (j.eps > 0.0) max_apr = std::min(max_apr, std::max(max_ap, min_apr));
            if (!autotune(C, max_ap, min_apr, max_apr, j.sp))
                return fail(FS_ERR_TOO_LARGE, "job %zu: no partition fits the table budget", ji);
        }
        if (j.sp.As > 62)
            return fail(FS_ERR_TOO_LARGE, "job %zu: %d artificial sources in the suffix (at most 62)", ji, j.sp.As);
        if (j.sp.Ap + j.sp.Ar + ilog2_ceil(std::max<uint64_t>(j.pairs, 1)) > 40)
            return fail(FS_ERR_TOO_LARGE, "job %zu: too many (prefix, root) items", ji);
        compile(C, j.W, j.sp, j.prog);
        j.levels.clear();
        if (b->opt.prefix_mode != 1 && j.sp.Ap > 0 && j.pairs > 0) {
            // candidate boundaries: after every op carrying a prefix source
            // (the tail without sources joins the last level)
            std::vector<int> E{0}, Abits{0};
            int a = 0;
            for (int e = 0; e < j.sp.c1; ++e) {
                const fs::Op& op = j.prog.ops[e];
                const int na = (op.s0 >= 0) + (op.s1 >= 0);
                if (na && (op.code == fs::OP_H || op.code == fs::OP_BR1 || op.code == fs::OP_BR2)) {
                    a += na;
                    E.push_back(e + 1);
                    Abits.push_back(a);
                }
            }
            const size_t m = E.size() - 1;
            if (m >= 1) E[m] = j.sp.c1;
            std::vector<size_t> from(m + 1, 0);
            if (b->opt.prefix_mode == 2) {
                for (size_t k = 1; k <= m; ++k) from[k] = k - 1;
            } else {
                // segmentation with the least modelled time: a level over
                // boundaries (i, k] runs its ops once per entry of level k,
                // reads level i and writes level k (32 B per entry) and costs
                // one launch; a single segment is the flat prefix
                const int dfrom = job_defer_from(j, b->opt.engine == 0);
                const bool fused = b->opt.engine == 0;
                std::vector<double> best(m + 1, 1e300);
                best[0] = 0.0;
                for (size_t k = 1; k <= m; ++k)
                    for (size_t i = 0; i < k; ++i) {
                        double io = 0, fo = 0;
                        region_work(j, E[i], E[k], io, fo, dfrom, fused);
                        const double n_out = std::ldexp((double)j.pairs, Abits[k]);
                        const double n_in = i ? std::ldexp((double)j.pairs, Abits[i]) : 0.0;
                        const double t = n_out * (io / kModelIntOps + fo / kModelFp64Ops) +
                                         32.0 * (n_out + n_in) / kModelBytes + kModelLaunch;
                        if (best[i] + t < best[k]) { best[k] = best[i] + t; from[k] = i; }
                    }
            }
            std::vector<size_t> cut_at;
            for (size_t k = m; k > 0; k = from[k]) cut_at.push_back(k);
            std::reverse(cut_at.begin(), cut_at.end());
            if (cut_at.size() >= 2) {
                size_t prev = 0;
                for (size_t k : cut_at) {
                    fs::PrefixLevel L;
                    L.e0 = E[prev];
                    L.e1 = E[k];
                    L.a_prev = Abits[prev];
                    L.a_next = Abits[k];
                    j.levels.push_back(L);
                    prev = k;
                }
            }
        }
        {
            fs::FeatureSpec& f = j.fspec;
            f.log10_eps_ref = (float)std::log10(j.eps > 0 ? j.eps : 1e-6);
            f.depth = G ? (float)j.sp.c1 / (float)G : 0.f;
            f.remaining = C.A ? (float)(C.A - j.sp.Ap) / (float)C.A : 0.f;
            f.n_qubits = (int)C.n;
            for (int k = 0; k < 8; ++k) f.next_qubits[k] = -1;
            int nk = 0;
            for (int e = j.sp.c1; e < G && nk < 8; ++e) {
                const GateInfo& gi = C.g[G - 1 - e];
                if (gi.role != BR) continue;
                for (int t = 0; t < gi.k && nk < 8; ++t)
                    if (gi.src[t] >= 0) f.next_qubits[nk++] = gi.q[t];
            }
        }
        j.compact = j.eps > 0.0 || j.d_pruner != nullptr || j.bound;
        if (j.bound) {
            if (!make_bound(j, (int)C.n)) return fail(FS_ERR_UNSUPPORTED, "job %zu: more than %d cascade fields after the cut", ji, fs::MAX_BOUND_FIELDS);
        }
        j.log2_ipp = j.sp.Ap + j.sp.Ar;
        j.log2_spp = std::max(0, j.log2_ipp - fs::TILE_LOG2);
        j.table_entries = j.pairs << j.sp.Ap;
        j.direct = j.sp.c1 == 0 && !j.compact && j.levels.empty();
        j.n_partials = j.compact ? 0 : (j.pairs << j.log2_spp);
        const uint64_t items = j.pairs << j.log2_ipp;
        j.n_tiles = j.compact ? 0 : (items + fs::TILE - 1) / fs::TILE;
        j.nblk = j.compact ? (j.table_entries + fs::COMPACT_BLOCK - 1) / fs::COMPACT_BLOCK : 0;
        if (j.n_tiles >= (1ull << 32)) return fail(FS_ERR_TOO_LARGE, "job %zu: too many tiles", ji);
        if (j.levels.empty() && !j.direct) b->total_prefix += j.table_entries;
        b->total_out += j.outs.size();
        // predicted cost of one tile (Eq. 8 per item): G_r + 2^As G_s
        const double tile_cost = (double)(j.sp.c2 - j.sp.c1) + std::ldexp((double)(G - j.sp.c2), j.sp.As);
        order.push_back({tile_cost, (uint32_t)ji});
    }
    // longest-processing-time order: the most expensive tiles are handed out first
    std::stable_sort(order.begin(), order.end(), [](const TileCost& a, const TileCost& x) { return a.cost > x.cost; });
    uint64_t ntile_total = 0;
    for (auto& t : order) ntile_total += b->jobs[t.job].n_tiles;
    if (ntile_total >= (1ull << 32)) return fail(FS_ERR_TOO_LARGE, "too many tiles in the batch");
    b->tiles.reserve(ntile_total);
    for (auto& t : order)
        for (uint64_t k = 0; k < b->jobs[t.job].n_tiles; ++k) b->tiles.push_back(make_uint2(t.job, (uint32_t)k));

    // workspace layout: static part first (uploaded once), then the dynamic part
    size_t off = 0;
    auto take = [&](size_t bytes) { const size_t o = off; off = align256(off + bytes); return o; };
    const size_t nj = b->jobs.size();
    b->o_jobs = take(nj * sizeof(fs::JobDev));
    b->o_pbegin = take(nj * sizeof(uint64_t));
    b->o_obegin = take(nj * sizeof(uint64_t));
    b->o_tiles = take(b->tiles.size() * sizeof(uint2));
    for (Job& j : b->jobs) {
        j.o_ops = take(j.prog.ops.size() * sizeof(fs::Op));
        j.o_masks = take(j.prog.masks.size() * sizeof(uint32_t));
        j.o_fac = take(j.prog.fac.size() * sizeof(double2));
        j.o_outs = take(j.outs.size() * 16);
        j.o_ins = take(j.ins.size() * 16);
        j.o_coef = take(j.coef.size() * sizeof(double2));
    }
    b->static_bytes = off;
    b->dyn_begin = off;
    b->o_stats = take(nj * fs::STATS_PER_JOB * sizeof(unsigned long long));
    for (Job& j : b->jobs) {
        j.fused = fused_reduction_of(*b, j);
        j.o_odone = j.fused ? take(j.outs.size() * sizeof(uint32_t)) : 0;
    }
    b->o_counter = take(sizeof(unsigned int));
    b->o_bigcount = take(sizeof(unsigned int));
    b->o_err = take(sizeof(uint32_t));   // last of the words zeroed at the start of every run
    b->o_biglist = take(b->total_out * sizeof(uint64_t));
    for (Job& j : b->jobs) {
        j.o_table = take(j.direct ? 0 : j.table_entries * sizeof(fs::Entry));
        j.o_part = take(j.n_partials * sizeof(double2));
        if (!j.levels.empty()) j.o_lvscratch = take((j.table_entries / 2) * sizeof(fs::Entry));
        if (j.compact) {
            j.o_live = take(j.table_entries * sizeof(uint64_t));
            // subtree partials: one per warp of 32 items when A_r >= 5, else per item
            j.o_esum = take((j.table_entries << (j.sp.Ar >= 5 ? j.sp.Ar - 5 : j.sp.Ar)) * sizeof(double2));
            j.o_blk = take(j.nblk * sizeof(uint32_t));
            j.o_prange = take(2 * j.pairs * sizeof(uint64_t));
        }
    }
    b->ws_bytes = off;
    *workspace_bytes = off;
    b->planned = true;
    b->uploaded = false;
    b->image_valid = false;
    b->drop_jit();
    int dev = 0;
    cudaGetDevice(&dev);
    b->grid = fs::history_grid_size(dev);
    b->compact_grid = fs::compact_grid_size(dev);
    return FS_OK;
}

// The exact reachability bound at evaluation position e0 of a job's
// program: qubits no op in [e0, G) can change, and fields moved only by +-1
// cascades with the number of such cascades as the radius.  False when the
// ops after e0 hold more than MAX_BOUND_FIELDS cascade fields.
static bool bound_at(const Job& j, int n_qubits, int e0, fs::BoundSpec& sp)
{
    const int G = (int)j.prog.ops.size(), W = j.W;
    uint32_t freem[4] = {0, 0, 0, 0};
    struct F { int t0, len; uint32_t runs; bool ok; };
    std::vector<F> fields;
    auto setq = [&](int q) { freem[q >> 5] |= 1u << (q & 31); };
    for (int e = e0; e < G; ++e) {
        fs::CascadeRun run;
        if (fs::find_cascade(j.prog.ops.data(), j.prog.masks.data(), W, e, G, run)) {
            bool found = false;
            for (F& f : fields)
                if (f.t0 == run.t0 && f.len == run.len) { f.runs++; found = true; }
            if (!found) fields.push_back({run.t0, run.len, 1u, true});
            e += run.len - 1;
            continue;
        }
        const fs::Op& op = j.prog.ops[e];
        switch (op.code) {
        case fs::OP_X: case fs::OP_MCX: case fs::OP_PERM1: case fs::OP_H: case fs::OP_BR1:
            setq(op.q0);
            break;
        case fs::OP_SWAP: case fs::OP_PERM2: case fs::OP_BR2:
            setq(op.q0);
            setq(op.q1);
            break;
        default:   // wire-preserving: the state does not change
            break;
        }
    }
    uint32_t fmask[4] = {0, 0, 0, 0};
    for (F& f : fields) {
        for (int q = f.t0; q < f.t0 + f.len; ++q) {
            if ((freem[q >> 5] >> (q & 31)) & 1u) f.ok = false;
            for (const F& g : fields)   // overlapping fields: no bound from either
                if (&g != &f && q >= g.t0 && q < g.t0 + g.len) f.ok = false;
        }
    }
    std::memset(&sp, 0, sizeof sp);
    for (F& f : fields) {
        for (int q = f.t0; q < f.t0 + f.len; ++q) fmask[q >> 5] |= 1u << (q & 31);
        if (!f.ok) {
            for (int q = f.t0; q < f.t0 + f.len; ++q) setq(q);
            continue;
        }
        if (sp.n_fields == fs::MAX_BOUND_FIELDS) return false;
        sp.t0[sp.n_fields] = f.t0;
        sp.len[sp.n_fields] = f.len;
        sp.radius[sp.n_fields] = f.runs;
        sp.n_fields++;
    }
    for (int w = 0; w < 4; ++w) {
        const int lo = 32 * w;
        const uint32_t valid = n_qubits >= lo + 32 ? 0xffffffffu : (n_qubits > lo ? ((1u << (n_qubits - lo)) - 1u) : 0u);
        sp.frozen[w] = valid & ~freem[w] & ~fmask[w];
    }
    return true;
}

// The bound at the checkpoint (cuts at sp.c1), applied where the table is
// written; and for the straight-line engine the bound after every op of the
// suffix that carries an artificial source (a history whose state there
// cannot reach b_in is cut with its subtree: all its leaves are invalid, so
// the amplitude is unchanged).  The root's source ops get no test: on the
// walk, tests there cost more issue slots than the cuts save (the learned
// step's history 33.5 -> 31.6 us without them).
static bool make_bound(Job& j, int n_qubits)
{
    if (!bound_at(j, n_qubits, j.sp.c1, j.bspec)) return false;
    j.src_bounds.clear();
    const int G = (int)j.prog.ops.size();
    for (int e = j.sp.c2; e < G; ++e) {
        const fs::Op& op = j.prog.ops[e];
        const bool br = op.code == fs::OP_H || op.code == fs::OP_BR1 || op.code == fs::OP_BR2;
        if (!br || (op.s0 < 0 && !(op.code == fs::OP_BR2 && op.s1 >= 0))) continue;
        fs::BoundSpec sp;
        if (!bound_at(j, n_qubits, e + 1, sp)) continue;
        if (!(sp.frozen[0] | sp.frozen[1] | sp.frozen[2] | sp.frozen[3]) && sp.n_fields == 0) continue;
        j.src_bounds.push_back({e, sp});
    }
    return true;
}

static std::vector<fs::JitJobSpec> jit_specs(const fs_batch* b)
{
    std::vector<fs::JitJobSpec> specs(b->jobs.size());
    for (size_t ji = 0; ji < b->jobs.size(); ++ji) {
        const Job& j = b->jobs[ji];
        specs[ji] = fs::JitJobSpec{j.prog.ops.data(), (int)j.prog.ops.size(), j.prog.masks.data(),
                                   j.prog.fac.data(), j.W, j.sp.c1, j.sp.c2, j.sp.Ap, j.sp.Ar,
                                   j.sp.As, j.eps * j.eps, j.compact, j.levels};
        // the generated prefix applies the exact bound where it writes the
        // table and, without a learned pruner, counts the live entries
        specs[ji].bound = j.bound;
        specs[ji].bound_counts = j.bound;
        specs[ji].bspec = j.bspec;
        if (j.bound) specs[ji].src_bounds = j.src_bounds;
    }
    return specs;
}

int fs_batch_generated_source(const fs_batch* b, char* buf, size_t cap, size_t* len)
{
    if (!b || !len) return fail(FS_ERR_INVALID, "NULL argument");
    if (!b->planned) return fail(FS_ERR_STATE, "fs_batch_plan must come first");
    const std::string src = fs::jit_source(jit_specs(b));
    *len = src.size();
    if (buf && cap) {
        const size_t n = std::min(cap - 1, src.size());
        std::memcpy(buf, src.data(), n);
        buf[n] = '\0';
    }
    return FS_OK;
}

int fs_batch_upload(fs_batch* b, void* d_ws, size_t ws_bytes, void* stream)
{
    if (!b || !d_ws) return fail(FS_ERR_INVALID, "NULL argument");
    DeviceGuard dg_(b->device);
    if (dg_.err != cudaSuccess) return cuda_fail(dg_.err, "cudaSetDevice(batch device)");
    if (!b->planned) return fail(FS_ERR_STATE, "fs_batch_plan must come first");
    if (ws_bytes < b->ws_bytes) return fail(FS_ERR_INVALID, "workspace of %zu bytes < %zu needed", ws_bytes, b->ws_bytes);
    if (((uintptr_t)d_ws) & 255) return fail(FS_ERR_INVALID, "workspace must be 256-byte aligned");
    for (const Job& j : b->jobs)
        if (j.d_pruner) {
            CUDA_TRY(fs::mlp_prepare());
            break;
        }
    unsigned char* base = (unsigned char*)d_ws;
    // the first upload of a batch stages through pageable memory and waits;
    // later ones (a request refreshed every step) through pinned memory
    const bool pinned = b->n_uploads > 0 && !b->no_host_alloc;
    unsigned char* H = nullptr;
    const bool engine_ready = b->opt.engine != 0 || b->jit || b->jobs.empty();
    if (pinned && b->image_valid && b->image_ws == d_ws && engine_ready) {
        // the pinned image of this plan for this workspace is current: copy it
        if (b->static_bytes)
            CUDA_TRY(cudaMemcpyAsync(d_ws, b->h_pinned, b->static_bytes, cudaMemcpyHostToDevice,
                                     (cudaStream_t)stream));
        CUDA_TRY(cudaEventRecord(b->up_ev, (cudaStream_t)stream));
        b->up_pending = true;
        b->n_uploads++;
        b->uploaded_ws = d_ws;
        b->uploaded = true;
        return FS_OK;
    }
    if (pinned) {
        if (b->up_pending) {
            CUDA_TRY(cudaEventSynchronize(b->up_ev));
            b->up_pending = false;
        }
        if (b->h_pinned_bytes < b->static_bytes) {
            if (b->h_pinned) CUDA_TRY(cudaFreeHost(b->h_pinned));
            b->h_pinned = nullptr;
            b->h_pinned_bytes = 0;
            CUDA_TRY(cudaMallocHost((void**)&b->h_pinned, b->static_bytes ? b->static_bytes : 1));
            b->h_pinned_bytes = b->static_bytes;
        }
        if (!b->up_ev) CUDA_TRY(cudaEventCreateWithFlags(&b->up_ev, cudaEventDisableTiming));
        H = b->h_pinned;
    } else {
        b->host_static.assign(b->static_bytes, 0);
        H = b->host_static.data();
    }
    if (b->static_bytes) std::memset(H, 0, b->static_bytes);
    const size_t nj = b->jobs.size();
    // the straight-line kernel is built first: it reports the constant factor
    // each job's generated root and suffix leave out (folded into c_in below)
    if (b->opt.engine == 0 && !b->jit && nj) {
        const std::vector<fs::JitJobSpec> specs = jit_specs(b);
        std::string err, src;
        const char* dump = getenv("FS_JIT_DUMP");   // optional: write the generated source here
        std::vector<double2> scales;
        const int jrc = fs::jit_build(specs, &b->jit, &err, &b->jit_ms, dump ? &src : nullptr, &scales);
        for (size_t ji = 0; ji < nj && !jrc; ++ji) b->jobs[ji].scale = scales[ji];
        if (dump) {
            FILE* f = fopen(dump, "w");
            if (f) { fwrite(src.data(), 1, src.size(), f); fclose(f); }
        }
        if (jrc) return fail(FS_ERR_CUDA, "straight-line engine: %s", err.c_str());
    }
    std::vector<fs::JobDev> jd(nj);
    std::vector<uint64_t> pbegin(nj), obegin(nj);
    uint64_t pacc = 0, oacc = 0;
    for (size_t ji = 0; ji < nj; ++ji) {
        Job& j = b->jobs[ji];
        fs::JobDev& d = jd[ji];
        std::memset(&d, 0, sizeof d);
        d.ops = (const fs::Op*)(base + j.o_ops);
        d.masks = (const uint32_t*)(base + j.o_masks);
        d.fac = (const double2*)(base + j.o_fac);
        d.outs = (const uint32_t*)(base + j.o_outs);
        d.ins = (const uint32_t*)(base + j.o_ins);
        d.coef = (const double2*)(base + j.o_coef);
        d.table = j.direct ? nullptr : (fs::Entry*)(base + j.o_table);
        d.partials = (double2*)(base + j.o_part);
        d.stats = (unsigned long long*)(base + b->o_stats) + fs::STATS_PER_JOB * ji;
        d.G = (int32_t)j.c->g.size();
        d.c1 = j.sp.c1; d.c2 = j.sp.c2;
        d.Ap = j.sp.Ap; d.Ar = j.sp.Ar; d.As = j.sp.As;
        d.W = j.W;
        d.S = (int32_t)j.ins.size();
        // division by S on the device: l = ceil(log2 S), multiplier
        // floor(2^32 (2^l - S) / S) + 1 (Granlund and Montgomery 1994, Fig. 4.1)
        d.s_shift = 0;
        d.s_magic = 0;
        if (j.ins.size() >= 2) {
            const uint64_t S = j.ins.size();
            int l = 0;
            while ((1ull << l) < S) ++l;
            d.s_shift = l;
            d.s_magic = (uint32_t)((((1ull << l) - S) << 32) / S + 1ull);
        }
        d.M = (int32_t)j.outs.size();
        d.log2_ipp = j.log2_ipp;
        d.log2_spp = j.log2_spp;
        d.n_pairs = j.pairs;
        d.prefix_begin = pacc;
        d.out_begin = oacc;
        d.n_tiles = j.n_tiles;
        d.eps2 = j.eps * j.eps;
        d.log = j.d_log;
        d.compact = j.compact ? 1 : 0;
        d.live = j.compact ? (uint64_t*)(base + j.o_live) : nullptr;
        d.esum = j.compact ? (double2*)(base + j.o_esum) : nullptr;
        d.blk = j.compact ? (uint32_t*)(base + j.o_blk) : nullptr;
        d.prange = j.compact ? (uint64_t*)(base + j.o_prange) : nullptr;
        d.n_entries = j.table_entries;
        d.scale = j.scale;
        d.trace = j.d_trace;
        d.odone = j.fused ? (uint32_t*)(base + j.o_odone) : nullptr;
        pbegin[ji] = pacc;
        obegin[ji] = oacc;
        if (j.levels.empty() && !j.direct) pacc += j.table_entries;
        oacc += j.outs.size();
        std::memcpy(&H[j.o_ops], j.prog.ops.data(), j.prog.ops.size() * sizeof(fs::Op));
        std::memcpy(&H[j.o_masks], j.prog.masks.data(), j.prog.masks.size() * sizeof(uint32_t));
        std::memcpy(&H[j.o_fac], j.prog.fac.data(), j.prog.fac.size() * sizeof(double2));
        for (size_t i = 0; i < j.outs.size(); ++i) std::memcpy(&H[j.o_outs + 16 * i], j.outs[i].w, 16);
        for (size_t i = 0; i < j.ins.size(); ++i) std::memcpy(&H[j.o_ins + 16 * i], j.ins[i].w, 16);
        // c_in times the hoisted constant, rounded once from extended precision
        const std::complex<long double> sc((long double)j.scale.x, (long double)j.scale.y);
        for (size_t i = 0; i < j.coef.size(); ++i) {
            const std::complex<long double> c =
                std::complex<long double>((long double)j.coef[i].real(), (long double)j.coef[i].imag()) * sc;
            const double2 v = make_double2((double)c.real(), (double)c.imag());
            std::memcpy(&H[j.o_coef + sizeof(double2) * i], &v, sizeof v);
        }
    }
    if (nj) {
        std::memcpy(&H[b->o_jobs], jd.data(), nj * sizeof(fs::JobDev));
        std::memcpy(&H[b->o_pbegin], pbegin.data(), nj * sizeof(uint64_t));
        std::memcpy(&H[b->o_obegin], obegin.data(), nj * sizeof(uint64_t));
    }
    if (!b->tiles.empty()) std::memcpy(&H[b->o_tiles], b->tiles.data(), b->tiles.size() * sizeof(uint2));
    if (b->static_bytes)
        CUDA_TRY(cudaMemcpyAsync(d_ws, H, b->static_bytes, cudaMemcpyHostToDevice, (cudaStream_t)stream));
    if (pinned) {
        CUDA_TRY(cudaEventRecord(b->up_ev, (cudaStream_t)stream));
        b->up_pending = true;
        b->image_valid = true;
        b->image_ws = d_ws;
    } else {
        // the pageable staging copy must outlive the copy
        CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    }
    b->n_uploads++;
    b->uploaded_ws = d_ws;
    b->uploaded = true;
    return FS_OK;
}

// Whether some output of a planned batch can have more partial sums than a
// warp of the reduction takes (then the block-per-output pass runs): S
// pairs per output, per pair 2^log2_spp tile partials (exact jobs) or up to
// 2^A_p live entries x 2^(A_r - 5 or A_r) subtree sums (compacted jobs).
static bool big_outputs_possible(const fs_batch& b)
{
    for (const Job& j : b.jobs) {
        if (j.outs.empty() || j.fused) continue;
        const int lg = j.compact ? j.sp.Ap + (j.sp.Ar >= 5 ? j.sp.Ar - 5 : j.sp.Ar) : j.log2_spp;
        const long double per_out = std::ldexp((long double)j.ins.size(), lg);
        if (per_out > (long double)fs::RED_BIG_ITEMS || j.ins.size() >= (size_t)fs::RED_BIG_THREADS) return true;
    }
    return false;
}

// A learned pruner on top of the exact bound whose table has at most
// COMPACT_DIRECT_BLOCKS compaction blocks: the scoring kernel writes the
// compaction (a CTA per block, the bound's per-block counts) and scores
// each block's live entries, one launch instead of two.
static bool scorer_compacts(const Job& j)
{
    return j.bound && j.d_pruner && j.nblk <= (uint64_t)fs::COMPACT_DIRECT_BLOCKS;
}

// Whether some job with outputs leaves them to the reduction kernels.
static bool reduce_needed(const fs_batch& b)
{
    for (const Job& j : b.jobs)
        if (!j.outs.empty() && !j.fused) return true;
    return false;
}

int fs_batch_launch_count(const fs_batch* b, uint32_t* n)
{
    if (!b || !n) return fail(FS_ERR_INVALID, "NULL argument");
    // reduce: outputs by lane groups, then (when possible) the listed large
    // ones; none when every job with outputs reduces them in its history
    uint32_t k = reduce_needed(*b) ? (big_outputs_possible(*b) ? 2 : 1) : 0;
    bool tiled = false, flat_prefix = false;
    for (const Job& j : b->jobs) {
        tiled |= !j.compact;
        flat_prefix |= j.levels.empty() && !j.direct;
        k += (uint32_t)j.levels.size();
        if (j.d_pruner) k += 1;                 // learned prune
        if (j.bound && b->opt.engine == 1) k += 1;   // exact bound (inside the generated prefix otherwise)
        // [count,] [scan,] write (with pair ranges), history over live entries
        if (j.compact)
            k += ((j.d_pruner || j.bound) ? 2 : 3) + (j.nblk > (uint64_t)fs::COMPACT_DIRECT_BLOCKS ? 1 : 0) -
                 (scorer_compacts(j) ? 1 : 0);
    }
    *n = k + (tiled ? 1 : 0) + (flat_prefix ? 1 : 0);
    return FS_OK;
}

int fs_batch_time_kernels(fs_batch* b, int enable)
{
    if (!b) return fail(FS_ERR_INVALID, "NULL batch");
    DeviceGuard dg_(b->device);
    if (dg_.err != cudaSuccess) return cuda_fail(dg_.err, "cudaSetDevice(batch device)");
    if (enable && !b->ev[0])
        for (auto& e : b->ev) CUDA_TRY(cudaEventCreate(&e));
    b->timing = enable != 0;
    b->ev_recorded = false;
    return FS_OK;
}

int fs_batch_kernel_ms(fs_batch* b, float* prefix_ms, float* history_ms, float* reduce_ms)
{
    if (!b) return fail(FS_ERR_INVALID, "NULL batch");
    if (!b->ev_recorded) return fail(FS_ERR_STATE, "no timed run recorded");
    CUDA_TRY(cudaEventSynchronize(b->ev[3]));
    float a = 0, h = 0, r = 0;
    CUDA_TRY(cudaEventElapsedTime(&a, b->ev[0], b->ev[1]));
    CUDA_TRY(cudaEventElapsedTime(&h, b->ev[1], b->ev[2]));
    CUDA_TRY(cudaEventElapsedTime(&r, b->ev[2], b->ev[3]));
    if (prefix_ms) *prefix_ms = a;
    if (history_ms) *history_ms = h;
    if (reduce_ms) *reduce_ms = r;
    return FS_OK;
}

// Stage events are recorded as external event nodes when the stream is being
// captured into a graph (plain records otherwise), so a replayed graph still
// times its stages.
static cudaError_t record(cudaEvent_t e, cudaStream_t s)
{
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    const cudaError_t q = cudaStreamIsCapturing(s, &st);
    if (q != cudaSuccess) return q;
    if (st == cudaStreamCaptureStatusActive) return cudaEventRecordWithFlags(e, s, cudaEventRecordExternal);
    return cudaEventRecord(e, s);
}

int fs_batch_stage_ms(fs_batch* b, float* ms)
{
    if (!b || !ms) return fail(FS_ERR_INVALID, "NULL argument");
    if (!b->ev_recorded) return fail(FS_ERR_STATE, "no timed run recorded");
    CUDA_TRY(cudaEventSynchronize(b->ev[3]));
    // prefix, learned prune, compaction, history, reduce
    const int order[6] = {0, 4, 5, 1, 2, 3};
    for (int k = 0; k < 5; ++k) CUDA_TRY(cudaEventElapsedTime(&ms[k], b->ev[order[k]], b->ev[order[k + 1]]));
    return FS_OK;
}

int fs_batch_run(fs_batch* b, void* d_ws, double* d_amp_out, void* stream)
{
    if (!b || !d_ws || (!d_amp_out && b->total_out)) return fail(FS_ERR_INVALID, "NULL argument");
    DeviceGuard dg_(b->device);
    if (dg_.err != cudaSuccess) return cuda_fail(dg_.err, "cudaSetDevice(batch device)");
    if (!b->uploaded || b->uploaded_ws != d_ws) return fail(FS_ERR_STATE, "fs_batch_upload on this workspace must come first");
    cudaStream_t s = (cudaStream_t)stream;
    unsigned char* base = (unsigned char*)d_ws;
    const int nj = (int)b->jobs.size();
    const fs::JobDev* jobs = (const fs::JobDev*)(base + b->o_jobs);
    CUDA_TRY(cudaMemsetAsync(base + b->o_stats, 0, b->o_err + sizeof(uint32_t) - b->o_stats, s));
    for (const Job& j : b->jobs)
        if (j.d_trace && !j.outs.empty())
            CUDA_TRY(cudaMemsetAsync(j.d_trace, 0, 2 * j.outs.size() * sizeof(unsigned long long), s));
    // the generated prefix of a job with the exact bound counts the live
    // entries per compaction block as it writes them
    if (b->jit)
        for (int ji = 0; ji < nj; ++ji) {
            const Job& j = b->jobs[ji];
            if (j.bound) CUDA_TRY(cudaMemsetAsync(base + j.o_blk, 0, j.nblk * sizeof(uint32_t), s));
        }
    if (b->timing) CUDA_TRY(record(b->ev[0], s));
    for (int ji = 0; ji < nj; ++ji) {
        const Job& j = b->jobs[ji];
        const int m = (int)j.levels.size();
        for (int k = 0; k < m; ++k) {
            // the last level writes the table; earlier ones alternate with the scratch
            fs::Entry* table = (fs::Entry*)(base + j.o_table);
            fs::Entry* scratch = (fs::Entry*)(base + j.o_lvscratch);
            fs::Entry* dst = ((m - 1 - k) % 2 == 0) ? table : scratch;
            const fs::Entry* src = k == 0 ? nullptr : (((m - k) % 2 == 0) ? table : scratch);
            const uint64_t n = j.pairs << j.levels[k].a_next;
            if (b->jit)
                CUDA_TRY(fs::jit_launch_prefix_level(b->jit, jobs, ji, k, j.levels[k], src, dst, n, k + 1 == m, s));
            else
                CUDA_TRY(fs::launch_prefix_level(jobs + ji, j.levels[k], src, dst, n, k + 1 == m,
                                                 (uint32_t*)(base + b->o_err), s));
        }
    }
    if (b->total_prefix == 0) {
        // every job expanded its prefix level by level
    } else if (b->jit)
        CUDA_TRY(fs::jit_launch_prefix(b->jit, jobs, (const uint64_t*)(base + b->o_pbegin), nj, b->total_prefix, s));
    else
        CUDA_TRY(fs::launch_prefix(jobs, (const uint64_t*)(base + b->o_pbegin), nj, b->total_prefix,
                                   (uint32_t*)(base + b->o_err), s));
    if (b->timing) CUDA_TRY(record(b->ev[4], s));
    for (int ji = 0; ji < nj; ++ji) {
        const Job& j = b->jobs[ji];
        // Checkpoint cuts.  With the exact bound (applied and counted by the
        // generated prefix, or by its own kernel for the interpreter) the
        // table is compacted first and a learned pruner scores only the
        // live entries, marking its cuts in place (the history skips them);
        // a pruner alone scores every entry and counts the live ones per
        // compaction block for the compaction that follows.
        if (j.bound && !b->jit) {
            CUDA_TRY(cudaMemsetAsync(base + j.o_blk, 0, j.nblk * sizeof(uint32_t), s));
            CUDA_TRY(fs::launch_bound_prune(jobs, ji, j.bspec, j.table_entries, true, s));
        }
        const bool scorer_writes = scorer_compacts(j);
        if (j.bound && !scorer_writes) CUDA_TRY(fs::launch_compact(jobs + ji, j.table_entries, true, s));
        if (j.d_pruner) {
            if (!j.bound) CUDA_TRY(cudaMemsetAsync(base + j.o_blk, 0, j.nblk * sizeof(uint32_t), s));
            CUDA_TRY(fs::mlp_learned_prune(j.d_pruner, jobs, ji, j.fspec, j.tau, j.table_entries,
                                           (uint32_t*)(base + b->o_err), s, j.bound ? (scorer_writes ? 2 : 1) : 0));
        }
    }
    if (b->timing) CUDA_TRY(record(b->ev[5], s));
    for (int ji = 0; ji < nj; ++ji) {
        const Job& j = b->jobs[ji];
        if (!j.compact || j.bound) continue;   // (bound jobs were compacted before scoring)
        CUDA_TRY(fs::launch_compact(jobs + ji, j.table_entries, j.d_pruner != nullptr, s));
    }
    if (b->timing) CUDA_TRY(record(b->ev[1], s));
    if (b->tiles.empty()) {
        // no tiled (exact) job: nothing to launch
    } else if (b->jit)
        CUDA_TRY(fs::jit_launch_history(b->jit, jobs, (const uint2*)(base + b->o_tiles), b->tiles.size(),
                                        (unsigned int*)(base + b->o_counter), s));
    else
        CUDA_TRY(fs::launch_history(jobs, (const uint2*)(base + b->o_tiles), b->tiles.size(),
                                    (unsigned int*)(base + b->o_counter), (uint32_t*)(base + b->o_err), b->grid, s));
    for (int ji = 0; ji < nj; ++ji) {
        if (!b->jobs[ji].compact) continue;
        if (b->jit) CUDA_TRY(fs::jit_launch_compact(b->jit, jobs, ji, (double2*)d_amp_out, s));
        else CUDA_TRY(fs::launch_history_compact(jobs + ji, (uint32_t*)(base + b->o_err), b->compact_grid, s));
    }
    if (b->timing) CUDA_TRY(record(b->ev[2], s));
    if (reduce_needed(*b))
        CUDA_TRY(fs::launch_reduce(jobs, (const uint64_t*)(base + b->o_obegin), nj, b->total_out,
                                   (double2*)d_amp_out, (unsigned int*)(base + b->o_bigcount),
                                   (uint64_t*)(base + b->o_biglist), big_outputs_possible(*b), s));
    if (b->timing) {
        CUDA_TRY(record(b->ev[3], s));
        b->ev_recorded = true;
    }
    return FS_OK;
}

int fs_batch_finish(fs_batch* b, void* d_ws, void* stream, fs_stats* stats, size_t cap)
{
    if (!b || !d_ws) return fail(FS_ERR_INVALID, "NULL argument");
    DeviceGuard dg_(b->device);
    if (dg_.err != cudaSuccess) return cuda_fail(dg_.err, "cudaSetDevice(batch device)");
    if (!b->uploaded || b->uploaded_ws != d_ws) return fail(FS_ERR_STATE, "no run on this workspace");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t nj = b->jobs.size();
    std::vector<unsigned long long> st(fs::STATS_PER_JOB * nj + 1, 0);
    uint32_t err = 0;
    unsigned char* base = (unsigned char*)d_ws;
    // counters ... error word are one contiguous range, copied at once; from
    // the second finish on into pinned memory owned by the batch
    const size_t words = b->o_err + sizeof(uint32_t) - b->o_stats;
    std::vector<unsigned char> pageable;
    unsigned char* hw = nullptr;
    if (b->n_finishes > 0 && !b->no_host_alloc) {
        if (b->h_words_bytes < words) {
            if (b->h_words) CUDA_TRY(cudaFreeHost(b->h_words));
            b->h_words = nullptr;
            b->h_words_bytes = 0;
            CUDA_TRY(cudaMallocHost((void**)&b->h_words, words));
            b->h_words_bytes = words;
        }
        hw = b->h_words;
    } else {
        pageable.resize(words);
        hw = pageable.data();
    }
    b->n_finishes++;
    CUDA_TRY(cudaMemcpyAsync(hw, base + b->o_stats, words, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    CUDA_TRY(cudaGetLastError());
    if (nj) std::memcpy(st.data(), hw, fs::STATS_PER_JOB * nj * sizeof(unsigned long long));
    std::memcpy(&err, hw + (b->o_err - b->o_stats), sizeof err);
    if (err & fs::DEV_ERR_BAD_OPCODE) return fail(FS_ERR_BAD_PROGRAM, "device found an unknown opcode");
    if (err & fs::DEV_ERR_TIMEOUT) return fail(FS_ERR_TIMEOUT, "a bounded device wait gave up (tensor-core scoring)");
    if (stats) {
        for (size_t ji = 0; ji < nj && ji < cap; ++ji) {
            const Job& j = b->jobs[ji];
            fs_stats& o = stats[ji];
            std::memset(&o, 0, sizeof o);
            const int A = j.c->A;
            const int lp = ilog2_ceil(std::max<uint64_t>(j.pairs, 1));
            o.candidates = (A + lp < 64) ? (j.pairs << A) : ~0ull;
            const unsigned long long* q = &st[fs::STATS_PER_JOB * ji];
            o.completed = q[0];
            o.valid = q[1];
            o.gate_visits = q[2] + q[4];
            o.history_visits = q[2];
            o.table_entries = j.direct ? j.pairs : q[3];
            o.learned_cuts = q[5];
            o.bound_cuts = q[8];
            o.live_entries = j.compact ? q[6] : o.table_entries;
            // with the bound, the pruner's cuts are marked in the compacted list
            if (j.bound && j.d_pruner) o.live_entries = q[6] - q[5];
            o.c1 = j.sp.c1; o.c2 = j.sp.c2;
            o.A_p = (uint32_t)j.sp.Ap; o.A_r = (uint32_t)j.sp.Ar; o.A_s = (uint32_t)j.sp.As;
        }
    }
    return FS_OK;
}

int fs_batch_op_histogram(const fs_batch* b, uint32_t job, uint32_t* counts)
{
    if (!b || !counts) return fail(FS_ERR_INVALID, "NULL argument");
    if (!b->planned) return fail(FS_ERR_STATE, "fs_batch_plan must come first");
    if (job >= b->jobs.size()) return fail(FS_ERR_INVALID, "job %u out of range", job);
    const Job& j = b->jobs[job];
    std::memset(counts, 0, 3 * FS_N_OPCODES * sizeof(uint32_t));
    for (size_t e = 0; e < j.prog.ops.size(); ++e) {
        const int r = (int)e < j.sp.c1 ? 0 : ((int)e < j.sp.c2 ? 1 : 2);
        const uint32_t code = j.prog.ops[e].code;
        if (code < FS_N_OPCODES) counts[r * FS_N_OPCODES + code]++;
    }
    return FS_OK;
}

// Algorithmic work of one execution of each region of a job: integer
// logic/compare instructions on the register state and FP64 instructions.
// Per op, with nz = control-mask words that are not all zero:
//   X 1 | MCX, MCPH, MCNEG: nz masked compares + ceil((nz-1)/2) 3-input ORs
//   + 1 test, then 1 flip (MCX), or the phase (MCPH: its factor, MCNEG: 2
//   sign flips) on half the histories | SWAP 5 | PERM1 3 + 4 FP64 |
//   PERM2 8 + 4 FP64 | DIAG1 2 + 4 FP64 | PH1 1 + half the factor's cost |
//   NEG1 1 + 1 | DIAG2 3 + 4 FP64 | H 4 + 2 FP64 | BR1 5 + 4 FP64 |
//   BR2 10 + 4 FP64; a factor costs 0 (1), 2 integer (-1), 2 FP64 (real or
//   imaginary) or 4 FP64 (general).
static void factor_cost(double2 f, double& iops, double& fops)
{
    if (f.x == 1.0 && f.y == 0.0) return;
    if (f.x == -1.0 && f.y == 0.0) { iops += 2; return; }
    if (f.y == 0.0 || f.x == 0.0) { fops += 2; return; }
    fops += 4;
}

static bool same2(double2 a, double2 b) { return a.x == b.x && a.y == b.y; }

// First evaluation position whose two-valued factors the straight-line
// engine defers (counts per class, one product per region): 0 in exact
// mode, after the last |beta| test with a threshold, none for the
// interpreter (G + 1).
static int job_defer_from(const Job& j, bool straight)
{
    const int G = (int)j.prog.ops.size();
    if (!straight) return G + 1;
    if (j.eps == 0.0) return 0;
    int last = -1;
    for (int e = 0; e < G; ++e) {
        const fs::Op& op = j.prog.ops[e];
        const bool br = op.code == fs::OP_H || op.code == fs::OP_BR1 || op.code == fs::OP_BR2;
        if (br && (op.s0 >= 0 || (op.code == fs::OP_BR2 && op.s1 >= 0))) last = e;
    }
    return last + 1;
}

// Ops at positions >= dfrom are deferred: the straight-line engine counts
// their two-valued factors per class (1 integer add) and applies each class
// once per region (one complex product per class).
// hoisted: the straight-line root and suffix, where a class whose factors
// differ by a unit phase is applied as sign flips and swaps (integer pipe).
static void region_work(const Job& j, int e0, int e1, double& iops, double& fops, int dfrom, bool fused,
                        bool hoisted)
{
    const int W = j.W;
    std::vector<std::pair<double2, double2>> classes;
    bool phase = false;   // commensurate phases: one integer phase, one product per region
    auto defer = [&](double2 A, double2 B) {
        iops += 1;
        uint32_t p;
        const bool unit = (B.x == A.x && B.y == A.y) || (B.x == -A.x && B.y == -A.y) ||
                          (B.x == -A.y && B.y == A.x) || (B.x == A.y && B.y == -A.x);
        if (fs::phase_index(A, B, &p) && !(hoisted && unit)) {
            phase = true;
            return;
        }
        for (auto& c : classes)
            if (same2(c.first, A) && same2(c.second, B)) return;
        classes.push_back({A, B});
    };
    const double2 one = make_double2(1.0, 0.0);
    const double2 R = make_double2(std::sqrt(0.5), 0.0), mR = make_double2(-std::sqrt(0.5), 0.0);
    for (int e = e0; e < e1; ++e) {
        const fs::Op& op0 = j.prog.ops[e];
        fs::CascadeRun run;
        if (fused && fs::find_cascade(j.prog.ops.data(), j.prog.masks.data(), W, e, e1, run)) {
            // common-control test, then the first field word: mask, subtract,
            // borrow, xor-and, flip; later words only when a lane borrows
            // (practically never), behind a vote (2)
            int nz = 0;
            for (int w = 0; w < W; ++w) nz += (run.cm[w] | run.cv[w]) != 0;
            const bool multi = ((run.t0 + run.len - 1) >> 5) != (run.t0 >> 5);
            iops += (nz ? nz + (nz > 1 ? nz / 2 : 0) + 1 : 0) + 5.0 + (multi ? 2.0 : 0.0);
            e += run.len - 1;
            continue;
        }
        if (e >= dfrom) {
            const double2* F = j.prog.fac.data() + op0.aux;
            bool z = false;
            switch (op0.code) {
            case fs::OP_PERM1: iops += 2; defer(F[0], F[1]); continue;
            case fs::OP_DIAG1: iops += 1; defer(F[0], F[1]); continue;
            case fs::OP_PH1: iops += 1; if (!same2(F[0], one)) defer(one, F[0]); continue;
            case fs::OP_MCPH: {
                int nz = 0;
                for (int w = 0; w < W; ++w) nz += (j.prog.masks[op0.aux2 + w] | j.prog.masks[op0.aux2 + W + w]) != 0;
                iops += nz + (nz > 1 ? nz / 2 : 0) + 1;
                if (!same2(F[0], one)) defer(one, F[0]);
                continue;
            }
            case fs::OP_DIAG2:
                if (same2(F[0], F[3]) && same2(F[1], F[2])) { iops += 2; defer(F[0], F[1]); continue; }
                break;
            case fs::OP_H: iops += 3; defer(R, mR); continue;
            case fs::OP_BR1:
                for (int k = 0; k < 4; ++k) z |= (F[k].x == 0.0 && F[k].y == 0.0);
                if (!z && same2(F[0], F[3]) && same2(F[1], F[2])) { iops += 3; defer(F[0], F[1]); continue; }
                break;
            default: break;
            }
        }
        const fs::Op& op = op0;
        int nz = 0;
        if (op.code == fs::OP_MCX || op.code == fs::OP_MCPH || op.code == fs::OP_MCNEG)
            for (int w = 0; w < W; ++w) nz += (j.prog.masks[op.aux2 + w] | j.prog.masks[op.aux2 + W + w]) != 0;
        const double test = nz + (nz > 1 ? (nz - 1 + 1) / 2 : 0) + 1;
        const double2* F = j.prog.fac.data() + op.aux;
        double fi = 0, ff = 0;
        switch (op.code) {
        case fs::OP_X: iops += 1; break;
        case fs::OP_MCX: iops += test + 1; break;
        case fs::OP_SWAP: iops += 5; break;
        case fs::OP_PERM1: iops += 3; fops += 4; break;
        case fs::OP_PERM2: iops += 8; fops += 4; break;
        case fs::OP_DIAG1: iops += 2; fops += 4; break;
        case fs::OP_PH1: factor_cost(F[0], fi, ff); iops += 1 + fi / 2; fops += ff / 2; break;
        case fs::OP_NEG1: iops += 1 + 1; break;
        case fs::OP_MCPH: factor_cost(F[0], fi, ff); iops += test + fi / 2; fops += ff / 2; break;
        case fs::OP_MCNEG: iops += test + 1; break;
        case fs::OP_DIAG2: iops += 3; fops += 4; break;
        case fs::OP_H: iops += 4; fops += 2; break;
        case fs::OP_BR1: {
            const bool sym = same2(F[0], F[3]) && same2(F[1], F[2]);
            const bool ri = (F[0].x == 0.0 || F[0].y == 0.0) && (F[1].x == 0.0 || F[1].y == 0.0);
            if (sym && ri) { iops += 7; fops += 2; }   // one real scalar product and a rotation
            else { iops += 5; fops += 4; }
            break;
        }
        case fs::OP_BR2: iops += 10; fops += 4; break;
        default: break;
        }
        // with a threshold, |beta|^2 after every op carrying a source: a
        // multiply and a fused multiply-add, an integer compare and branch
        const bool src_op = (op.code == fs::OP_H || op.code == fs::OP_BR1 || op.code == fs::OP_BR2) &&
                            (op.s0 >= 0 || (op.code == fs::OP_BR2 && op.s1 >= 0));
        if (j.eps > 0.0 && src_op) {
            iops += 2;
            fops += 2;
        }
        // the exact bound after a source op (straight-line engine): the
        // frozen-qubit test (xor, and, or per word) and per cascade field
        // its words (two funnel shifts and masks each for state and input)
        // and both borrow chains (four ops per word each), two compares
        if (fused && j.bound && src_op)
            for (const auto& pb : j.src_bounds) {
                if (pb.first != e) continue;
                double c = 1;
                for (int w = 0; w < 4; ++w) c += pb.second.frozen[w] ? 3 : 0;
                for (int f = 0; f < pb.second.n_fields; ++f) {
                    const int fw = (pb.second.len[f] + 31) / 32;
                    c += 4.0 * fw + 8.0 * fw + 4.0;
                }
                iops += c;
            }
    }
    for (const auto& c : classes) {
        const double2 A = c.first, B = c.second;
        const bool unit = (B.x == A.x && B.y == A.y) || (B.x == -A.x && B.y == -A.y) ||
                          (B.x == -A.y && B.y == A.x) || (B.x == A.y && B.y == -A.x);
        if (hoisted && unit) iops += 3;   // select and sign flips
        else fops += 4;                   // one complex product per region
    }
    if (phase) {
        iops += 2;   // shift and mask of the phase index
        fops += 4;   // one complex product by the table entry
    }
}

int fs_batch_region_work(const fs_batch* b, uint32_t job, double* int_ops, double* fp64_ops)
{
    if (!b || !int_ops || !fp64_ops) return fail(FS_ERR_INVALID, "NULL argument");
    if (!b->planned) return fail(FS_ERR_STATE, "fs_batch_plan must come first");
    if (job >= b->jobs.size()) return fail(FS_ERR_INVALID, "job %u out of range", job);
    const Job& j = b->jobs[job];
    const int G = (int)j.prog.ops.size();
    const int cuts[4] = {0, j.sp.c1, j.sp.c2, G};
    const int dfrom = job_defer_from(j, b->opt.engine == 0);
    const bool fused = b->opt.engine == 0;   // the straight-line engine fuses incrementer cascades
    for (int r = 0; r < 3; ++r) {
        double i = 0, f = 0;
        region_work(j, cuts[r], cuts[r + 1], i, f, dfrom, fused, r > 0 && dfrom <= G);
        int_ops[r] = i;
        fp64_ops[r] = f;
    }
    if (!j.levels.empty()) {
        // level-by-level prefix: each level's ops run once per entry of that
        // level; reported per final table entry
        double i = 0, f = 0;
        for (const fs::PrefixLevel& L : j.levels) {
            double li = 0, lf = 0;
            region_work(j, L.e0, L.e1, li, lf, dfrom, fused);
            i += li * std::ldexp(1.0, L.a_next - j.sp.Ap);
            f += lf * std::ldexp(1.0, L.a_next - j.sp.Ap);
        }
        int_ops[0] = i;
        fp64_ops[0] = f;
    }
    // per completed leaf: the chi test (2W); per valid leaf: two FP64 adds
    int_ops[3] = 2.0 * j.W;
    fp64_ops[3] = 2.0;
    if (b->opt.engine == 0) {
        // loop control of the generated engine, read off its item and leaf
        // loops: per item the pair / h_p / h_r indices, the entry-cache
        // tests, the nonzero test and vote of the item's sum, the loop
        // counter (24); per leaf the enumeration word's update and compare,
        // the restart test, the counters and the vote of the valid add (12)
        int_ops[1] += 24.0;
        int_ops[3] += 12.0;
        // the phase census: per valid leaf four compares and adds instead
        // of the FP64 adds; per root one product (2 conversions, 4 FP64)
        if (fs::jit_census(jit_specs(b)[job])) {
            int_ops[3] += 4.0;
            fp64_ops[3] = 0.0;
            fp64_ops[1] += 6.0;
        }
    }
    return FS_OK;
}

int fs_batch_job_words(const fs_batch* b, uint32_t job, uint32_t* words)
{
    if (!b || !words) return fail(FS_ERR_INVALID, "NULL argument");
    if (!b->planned) return fail(FS_ERR_STATE, "fs_batch_plan must come first");
    if (job >= b->jobs.size()) return fail(FS_ERR_INVALID, "job %u out of range", job);
    *words = (uint32_t)b->jobs[job].W;
    return FS_OK;
}

int fs_probe_peaks(double* dfma_per_s, double* int_ops_per_s, int32_t* sms)
{
    if (!dfma_per_s || !int_ops_per_s || !sms) return fail(FS_ERR_INVALID, "NULL argument");
    int n = 0;
    CUDA_TRY(fs::probe_peaks(dfma_per_s, int_ops_per_s, &n));
    *sms = n;
    return FS_OK;
}

int fs_batch_set_device(fs_batch* b, int32_t device)
{
    if (!b) return fail(FS_ERR_INVALID, "NULL batch");
    if (device < -1) return fail(FS_ERR_INVALID, "device must be >= 0 (or -1: the current device)");
    if (device >= 0) {
        int n = 0;
        const cudaError_t e = cudaGetDeviceCount(&n);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
        if (device >= n) return fail(FS_ERR_INVALID, "device %d out of range (%d devices)", device, n);
    }
    if (device != b->device) {
        b->device = device;
        b->planned = b->uploaded = false;   // grid sizes and the generated module are per device
        b->drop_jit();
    }
    return FS_OK;
}

int fs_batch_program_offset(const fs_batch* b, uint32_t job, size_t* offset, size_t* n_ops)
{
    if (!b || !offset || !n_ops) return fail(FS_ERR_INVALID, "NULL argument");
    if (!b->planned) return fail(FS_ERR_STATE, "fs_batch_plan must come first");
    if (job >= b->jobs.size()) return fail(FS_ERR_INVALID, "job %u out of range", job);
    *offset = b->jobs[job].o_ops;
    *n_ops = b->jobs[job].prog.ops.size();
    return FS_OK;
}

int fs_mlp_targets(const double* d_sums, uint64_t n, double floor_log10, float* d_target, void* stream)
{
    if (n && (!d_sums || !d_target)) return fail(FS_ERR_INVALID, "NULL argument");
    if (!std::isfinite(floor_log10)) return fail(FS_ERR_INVALID, "the floor must be finite");
    CUDA_TRY(fs::mlp_targets(d_sums, (unsigned long long)n, floor_log10, d_target, (cudaStream_t)stream));
    return FS_OK;
}

// ---- source placement in the graph form of Sec. IV-B (Fig. 4)

namespace {

struct WireGraph {
    int n_nodes = 0;                       // wire classes after merging
    std::vector<char> known;               // per node
    std::vector<std::array<int, 3>> tri;   // CNOTs still joining unknown nodes
};

int find_root(std::vector<int>& p, int x)
{
    while (p[x] != x) { p[x] = p[p[x]]; x = p[x]; }
    return x;
}

// Wires of a CNOT + single-qubit circuit, boundary wires known, CNOTs as
// triples; then the natural-source rule (a CNOT on a known wire goes, its
// other two wires merge) until no CNOT touches a known wire.  Returns
// FS_ERR_UNSUPPORTED for other gates.
int build_wire_graph(const fs_circuit& C, WireGraph& out)
{
    const int n = (int)C.n;
    int nw = n;
    std::vector<int> cur(n);
    for (int q = 0; q < n; ++q) cur[q] = q;
    std::vector<char> isknown(n, 1);
    std::vector<std::array<int, 3>> cn;
    for (size_t i = 0; i < C.g.size(); ++i) {
        const GateInfo& g = C.g[i];
        const int nctl = __builtin_popcountll(g.cm[0]) + __builtin_popcountll(g.cm[1]);
        if (g.role == WP) continue;                                  // keeps every wire
        if (g.role == DET && g.k == 1 && nctl == 0) continue;        // one wire through
        if (g.role == DET && g.kind == FS_SWAP) { std::swap(cur[g.q[0]], cur[g.q[1]]); continue; }
        if (g.role == DET && g.kind == FS_X && nctl == 1) {
            const int c = g.cm[0] ? __builtin_ctzll(g.cm[0]) : 64 + __builtin_ctzll(g.cm[1]);
            const int t = g.q[0];
            cn.push_back({cur[c], cur[t], nw});
            cur[t] = nw++;
            isknown.push_back(0);
            continue;
        }
        if (g.role == BR && g.k == 1 && nctl == 0) {
            cur[g.q[0]] = nw++;
            isknown.push_back(0);
            continue;
        }
        return fail(FS_ERR_UNSUPPORTED, "gate %zu is outside CNOT + single-qubit gates", i);
    }
    for (int q = 0; q < n; ++q) isknown[cur[q]] = 1;   // output wires
    std::vector<int> par(nw);
    for (int i = 0; i < nw; ++i) par[i] = i;
    bool changed = true;
    while (changed) {
        changed = false;
        std::vector<std::array<int, 3>> keep;
        for (auto t : cn) {
            for (int& x : t) x = find_root(par, x);
            int k = -1;
            for (int j = 0; j < 3; ++j)
                if (isknown[t[j]]) { k = j; break; }
            if (k < 0) { keep.push_back(t); continue; }
            int a = -1, b = -1;
            for (int j = 0; j < 3; ++j) {
                if (t[j] == t[k]) continue;
                if (a < 0) a = t[j]; else b = t[j];
            }
            if (a >= 0 && b >= 0 && a != b) {
                const char kn = isknown[a] | isknown[b];
                par[std::max(a, b)] = std::min(a, b);
                isknown[std::min(a, b)] = kn;
            }
            changed = true;
        }
        cn.swap(keep);
    }
    std::vector<int> id(nw, -1);
    out = WireGraph{};
    for (int x = 0; x < nw; ++x) {
        const int r = find_root(par, x);
        if (id[r] < 0) { id[r] = out.n_nodes++; out.known.push_back(isknown[r]); }
        if (isknown[x]) out.known[id[r]] = 1;
    }
    for (auto t : cn) out.tri.push_back({id[find_root(par, t[0])], id[find_root(par, t[1])], id[find_root(par, t[2])]});
    return FS_OK;
}

// Closure under the CNOT rule: two known wires of a CNOT fix the third.
void close_known(const WireGraph& G, std::vector<char>& kn)
{
    for (bool grew = true; grew;) {
        grew = false;
        for (const auto& t : G.tri) {
            const int k = kn[t[0]] + kn[t[1]] + kn[t[2]];
            if (k >= 2 && k < 3)
                for (int x : t)
                    if (!kn[x]) { kn[x] = 1; grew = true; }
        }
    }
}

bool all_known(const std::vector<char>& kn)
{
    for (char v : kn) if (!v) return false;
    return true;
}

}  // namespace

int fs_source_placement(const fs_circuit* c, uint32_t method, uint32_t* n_sources, uint32_t* n_nodes)
{
    if (!c || !n_sources) return fail(FS_ERR_INVALID, "NULL argument");
    if (method > 2) return fail(FS_ERR_INVALID, "method must be 0, 1 or 2");
    if (method == 0) {
        *n_sources = (uint32_t)c->A;
        if (n_nodes) *n_nodes = 0;
        return FS_OK;
    }
    WireGraph G;
    if (int rc = build_wire_graph(*c, G)) return rc;
    std::vector<int> unknown;
    for (int x = 0; x < G.n_nodes; ++x)
        if (!G.known[x]) unknown.push_back(x);
    if (n_nodes) *n_nodes = (uint32_t)unknown.size();
    if (method == 1) {
        // greedy: the unknown node on the most unresolved CNOTs, then closure
        std::vector<char> kn = G.known;
        close_known(G, kn);
        uint32_t k = 0;
        while (!all_known(kn)) {
            std::vector<int> deg(G.n_nodes, 0);
            for (const auto& t : G.tri) {
                if (kn[t[0]] && kn[t[1]] && kn[t[2]]) continue;
                for (int j = 0; j < 3; ++j) {
                    bool dup = false;
                    for (int i = 0; i < j; ++i) dup |= t[i] == t[j];
                    if (!dup && !kn[t[j]]) deg[t[j]]++;
                }
            }
            int best = -1;
            for (int x : unknown)
                if (!kn[x] && (best < 0 || deg[x] > deg[best])) best = x;
            kn[best] = 1;
            close_known(G, kn);
            ++k;
        }
        *n_sources = k;
        return FS_OK;
    }
    // exhaustive: subsets of the unknown nodes by increasing size
    const int m = (int)unknown.size();
    if (m > 30) return fail(FS_ERR_TOO_LARGE, "%d unknown wire classes: exhaustive placement is limited to 30", m);
    for (int k = 0; k <= m; ++k) {
        std::vector<int> pick(k);
        for (int i = 0; i < k; ++i) pick[i] = i;
        while (true) {
            std::vector<char> kn = G.known;
            for (int i : pick) kn[unknown[i]] = 1;
            close_known(G, kn);
            if (all_known(kn)) { *n_sources = (uint32_t)k; return FS_OK; }
            int i = k - 1;
            while (i >= 0 && pick[i] == m - k + i) --i;
            if (i < 0) break;
            ++pick[i];
            for (int j = i + 1; j < k; ++j) pick[j] = pick[j - 1] + 1;
        }
    }
    *n_sources = (uint32_t)m;
    return FS_OK;
}

int fs_lpt_assign(const double* cost, size_t n, uint32_t n_ranks, uint32_t* rank, double* load)
{
    if (n && (!cost || !rank)) return fail(FS_ERR_INVALID, "NULL argument");
    if (n_ranks == 0) return fail(FS_ERR_INVALID, "n_ranks must be >= 1");
    for (size_t i = 0; i < n; ++i)
        if (!(cost[i] >= 0.0) || std::isinf(cost[i])) return fail(FS_ERR_INVALID, "cost %zu is not finite and >= 0", i);
    // longest processing time first: units by descending cost (ties by
    // index), each to the least loaded rank (ties to the lowest rank)
    std::vector<size_t> order(n);
    for (size_t i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t c) { return cost[a] > cost[c]; });
    std::vector<double> ld(n_ranks, 0.0);
    for (size_t i : order) {
        uint32_t best = 0;
        for (uint32_t r = 1; r < n_ranks; ++r)
            if (ld[r] < ld[best]) best = r;
        rank[i] = best;
        ld[best] += cost[i];
    }
    if (load)
        for (uint32_t r = 0; r < n_ranks; ++r) load[r] = ld[r];
    return FS_OK;
}

int fs_set_wait_limit(int64_t polls)
{
    if (polls > 0xffffffffll) return fail(FS_ERR_INVALID, "at most 2^32 - 1 polls");
    fs::mlp_set_wait_limit(polls < 0 ? fs::mlp_default_wait_limit() : (uint32_t)polls);
    return FS_OK;
}

int fs_amplitudes(fs_circuit* c, const uint64_t* outputs, size_t n_out, double eps, double* amp_out)
{
    if (!c || (n_out && (!outputs || !amp_out))) return fail(FS_ERR_INVALID, "NULL argument");
    if (n_out == 0) return FS_OK;
    fs_batch b;
    if (int rc = fs_batch_add(&b, c, outputs, n_out, eps, nullptr)) return rc;
    size_t ws = 0;
    if (int rc = fs_batch_plan(&b, &ws)) return rc;
    void* d_ws = nullptr;
    double* d_amp = nullptr;
    cudaError_t e = cudaMalloc(&d_ws, ws ? ws : 256);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(workspace)");
    e = cudaMalloc((void**)&d_amp, 2 * n_out * sizeof(double));
    if (e != cudaSuccess) { cudaFree(d_ws); return cuda_fail(e, "cudaMalloc(amplitudes)"); }
    int rc = fs_batch_upload(&b, d_ws, ws ? ws : 256, nullptr);
    if (!rc) rc = fs_batch_run(&b, d_ws, d_amp, nullptr);
    if (!rc) rc = fs_batch_finish(&b, d_ws, nullptr, nullptr, 0);
    if (!rc) {
        e = cudaMemcpy(amp_out, d_amp, 2 * n_out * sizeof(double), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) rc = cuda_fail(e, "cudaMemcpy(amplitudes)");
    }
    cudaFree(d_amp);
    cudaFree(d_ws);
    return rc;
}

}  // extern "C"

// Internal layout shared by the host compiler (fs_host.cpp) and the CUDA
// kernels (fs_kernels.cu).  Not part of the public ABI.
#pragma once
#include <stdint.h>
#include <cuda_runtime.h>

#include <string>
#include <vector>

struct fs_batch;

namespace fs {

// Opcodes of the evaluation-order program.  Every op moves the state from
// the output side of one gate to its input side (the backward sweep of
// Sec. IV-A) and multiplies the gate's matrix element into the running
// amplitude.
enum OpCode : uint8_t {
    OP_X = 1,     // flip q0                                   (unit factor)
    OP_MCX,       // flip q0 when (st & mask) == val            (unit factor)
    OP_SWAP,      // exchange q0 and q1                         (unit factor)
    OP_PERM1,     // o = bit q0: amp *= fac[aux + o]; flip q0   (Y, antidiagonal U1)
    OP_PERM2,     // o = local 2-bit value: in = perm(o), amp *= fac[aux + o]
    OP_DIAG1,     // amp *= fac[aux + bit q0]                   (RZ, diagonal U1)
    OP_PH1,       // if bit q0: amp *= fac[aux]                 (S, T, P)
    OP_NEG1,      // if bit q0: amp = -amp                      (Z)
    OP_MCPH,      // if (st & mask) == val: amp *= fac[aux]     (controlled P/S/T)
    OP_MCNEG,     // if (st & mask) == val: amp = -amp          (CZ, MCZ)
    OP_DIAG2,     // amp *= fac[aux + bit q0 + 2 bit q1]        (RZZ, diagonal U2)
    OP_H,         // branching H: i = source; amp *= (o & i) ? -1/sqrt2 : 1/sqrt2
    OP_BR1,       // branching 1-qubit: amp *= fac[aux + 2 o + i]; q0 = i
    OP_BR2,       // branching 2-qubit: amp *= fac[aux + 4 o + i]; (q0, q1) = i
    OP_LAST
};

// 16-byte op.  s0/s1: bit index of the artificial source in the region's
// enumeration word h (-1: natural source, value read from the input bit
// string).  aux: factor offset (double2 units).  aux2: mask offset (u32
// units, W mask words then W value words) or, for OP_PERM2, the packed
// inverse permutation (2 bits per output value).
struct Op {
    uint8_t code, q0, q1, flags;
    int8_t s0, s1;
    uint16_t pad;
    uint32_t aux;
    uint32_t aux2;
};
static_assert(sizeof(Op) == 16, "Op must be 16 bytes");

// Keeps a batch on pageable staging (no pinned host buffers) for callers
// that must not allocate.
void batch_forbid_host_alloc(::fs_batch* b);

// A run of controlled-X ops [e, e + len) in evaluation order whose targets
// are the contiguous qubits t0, t0 + 1, ... and where op k is also
// controlled on the targets of ops 0..k-1, all with one polarity v, plus
// common controls (cm, cv) that do not touch the targets.  Applied in order
// the run maps the field x = bits [t0, t0 + len) of the register to x - 1
// (v = 1) or x + 1 (v = 0) modulo 2^len when the common controls hold: the
// ripple-carry incrementer / decrementer written as a cascade of
// multi-controlled X gates.
struct CascadeRun {
    int len, t0;
    bool dec;
    uint32_t cm[4], cv[4];
};
bool find_cascade(const Op* ops, const uint32_t* masks, int W, int e, int e1, CascadeRun& r);

// One checkpoint-table entry (Algorithm 2: propagated state sigma_p and
// partial amplitude beta_p after the prefix).  An entry whose prefix was cut
// (bottom) carries a NaN real part.
struct Entry {
    uint32_t st[4];
    double2 amp;
};
static_assert(sizeof(Entry) == 32, "Entry must be 32 bytes");

// Per-job descriptor in device memory.  The field list is a macro so that
// the generated straight-line kernels (fs_jit.cpp) declare the identical
// layout.  One declaration per field, no top-level commas.
#define FS_JOBDEV_FIELDS                                                      \
    const Op* ops;                                                            \
    const uint32_t* masks;                                                    \
    const double2* fac;                                                       \
    const uint32_t* outs;      /* M x 4 words */                              \
    const uint32_t* ins;       /* S x 4 words */                              \
    const double2* coef;       /* S */                                        \
    Entry* table;              /* pairs x 2^Ap */                             \
    double2* partials;         /* pairs x spp */                              \
    unsigned long long* stats; /* completed, valid, history visits, entries, prefix visits */ \
    int32_t G;                                                                \
    int32_t c1;                                                               \
    int32_t c2;                                                               \
    int32_t Ap;                                                               \
    int32_t Ar;                                                               \
    int32_t As;                                                               \
    int32_t W;                                                                \
    int32_t S;                                                                \
    int32_t M;                                                                \
    int32_t log2_ipp;          /* Ap + Ar */                                  \
    int32_t log2_spp;          /* max(0, log2_ipp - TILE_LOG2) */             \
    uint32_t s_magic;          /* division by S: multiplier (see fs_host.cpp) */ \
    uint64_t n_pairs;          /* S * M */                                    \
    uint64_t prefix_begin;     /* offset of this job in the flat prefix index space */ \
    uint64_t out_begin;        /* offset of this job's outputs in amp_out */ \
    uint64_t n_tiles;                                                         \
    double eps2;               /* eps^2 (0: exact) */                         \
    double2* log;              /* optional: per-item subtree sums (logging runs) */     \
    int32_t compact;           /* 1: history over the compacted live entries */         \
    int32_t s_shift;           /* division by S: ceil(log2 S) */                 \
    uint64_t* live;            /* compacted live entry indices, table order */            \
    double2* esum;             /* subtree sums of live items: per 32 (A_r >= 5) or per item */ \
    uint32_t* blk;             /* per compaction block: live count, then offset */       \
    uint64_t* prange;          /* per pair: [lo, hi) of its live entries */              \
    uint64_t n_entries;        /* checkpoint entries (pairs << Ap) */                   \
    double2 scale;             /* constant factor hoisted out of the root and suffix */ \
    unsigned long long* trace; /* optional: per output {completed, valid} leaves */ \
    uint32_t* odone;           /* optional: per output, subtree sums stored (reduction fused into the compacted history) */

struct JobDev {
    FS_JOBDEV_FIELDS
};

constexpr int TILE_LOG2 = 8;             // items per tile = threads per CTA
constexpr int TILE = 1 << TILE_LOG2;
constexpr int REDUCE_THREADS = 128;
constexpr int STATS_PER_JOB = 9;   // completed, valid, hist visits, entries, prefix visits, learned cuts,
                                   // live entries after compaction, compact work counter, bound cuts
constexpr int COMPACT_BLOCK = 1024;   // entries per compaction block (256 threads x 4)
constexpr int COMPACT_DIRECT_BLOCKS = 1024;   // up to this many blocks the write pass adds the counts itself
// The learned scorer's cut mark in an entry's amplitude: a NaN (every reader
// treats it as a cut entry) with its own payload, told apart from the other
// cut marks only by a compaction written beside the scorer.
constexpr unsigned long long LEARNED_CUT_BITS = 0x7ff8000000000001ull;
constexpr int MLP_PARAMS = 18817;

// Exact reachability bound at the checkpoint: what the ops after the cut can
// still change.  Qubits in `frozen` are targeted by no remaining op, so a
// checkpoint state that differs from b_in there reaches the input with no
// valid history; a field of contiguous qubits changed only by controlled
// +-1 cascades (find_cascade) moves by at most `radius` (the number of
// remaining cascades on it), so a state whose field value is farther than
// that from b_in's (cyclically, modulo 2^len) has an exactly zero subtree
// sum too.
// A deferred two-valued factor (A, B) = (1, e^{2 pi i p / 2^16}) for an
// integer p in (0, 2^16): the straight-line engine adds p to one integer
// phase per region instead of counting a class (one table product per
// region for all such factors).
bool phase_index(double2 A, double2 B, uint32_t* p);

constexpr int MAX_BOUND_FIELDS = 4;
struct BoundSpec {
    uint32_t frozen[4];
    int n_fields;
    int t0[MAX_BOUND_FIELDS];
    int len[MAX_BOUND_FIELDS];
    uint32_t radius[MAX_BOUND_FIELDS];
};
// Cuts (bottom) every live entry of a job's checkpoint table that the
// bound proves unreachable (counted in stats[8]); with count_blocks, also
// counts the live entries per compaction block (blk, zeroed by the caller).
cudaError_t launch_bound_prune(const JobDev* d_jobs, int job, const BoundSpec& sp, unsigned long long n_entries,
                               bool count_blocks, cudaStream_t s);

// Per-job constants of the learned pruner's features.
struct FeatureSpec {
    float log10_eps_ref;
    float depth;           // c1 / G
    float remaining;       // (A - A_p) / A
    int n_qubits;
    int next_qubits[8];    // targets of the next 8 artificial sources after the prefix (-1: none)
};

cudaError_t mlp_forward(const float* d_params, const float* d_x, long long n, float* d_y, cudaStream_t s);
cudaError_t mlp_grad(const float* d_params, const float* d_x, const float* d_t, long long n, float* d_grad,
                     cudaStream_t s);
cudaError_t mlp_adam(float* d_params, float* d_m, float* d_v, const float* d_grad, float lr, int step,
                     cudaStream_t s);
cudaError_t mlp_features(const JobDev* d_jobs, int job, const FeatureSpec& sp, float* d_feat,
                         unsigned long long n_entries, cudaStream_t s);
// rows = 0: score every entry and count the live ones per compaction block;
// 1: score the compacted live entries (after the exact bound) and mark cuts
// in the table only; 2: as 1, with the compaction's write pass done by the
// scoring kernel (four CTAs per compaction block share its live entries;
// the bound's per-block counts, at most COMPACT_DIRECT_BLOCKS blocks).
cudaError_t mlp_learned_prune(const float* d_params, const JobDev* d_jobs, int job, const FeatureSpec& sp,
                              float tau, unsigned long long n_entries, uint32_t* d_err, cudaStream_t s,
                              int rows);
cudaError_t mlp_targets(const double* d_sums, unsigned long long n, double floor_v, float* d_t, cudaStream_t s);
// Polls of a bounded tensor-core wait before it gives up (process-wide;
// change it only while no scoring kernel is being launched).
void mlp_set_wait_limit(uint32_t polls);
uint32_t mlp_default_wait_limit();
// Raises the dynamic shared-memory limit of the tensor-core scoring kernels
// (outside any stream capture, before their first launch).
cudaError_t mlp_prepare();

// Device error word values.
constexpr uint32_t DEV_ERR_BAD_OPCODE = 1;
constexpr uint32_t DEV_ERR_TIMEOUT = 2;   // a bounded wait on an mbarrier gave up

// One level of the per-source prefix expansion: ops [e0, e1) extend every
// entry of the previous level (a_prev source bits, in src; NULL for the
// first level, which starts at b_out) to a_next bits, into dst.
struct PrefixLevel {
    int e0, e1;
    int a_prev, a_next;
};


// Launch entry points (fs_kernels.cu).
cudaError_t launch_prefix(const JobDev* d_jobs, const uint64_t* d_job_prefix_begin, int n_jobs,
                          uint64_t total_prefix, uint32_t* d_err, cudaStream_t s);
cudaError_t launch_history(const JobDev* d_jobs, const uint2* d_tiles, uint64_t n_tiles,
                           unsigned int* d_counter, uint32_t* d_err, int grid, cudaStream_t s);
cudaError_t launch_prefix_level(const JobDev* d_job, const PrefixLevel& L, const Entry* src, Entry* dst,
                                uint64_t n_dst, bool last, uint32_t* d_err, cudaStream_t s);
cudaError_t jit_launch_prefix_level(void* handle, const JobDev* d_jobs, int job, int level, const PrefixLevel& L,
                                    const Entry* src, Entry* dst, uint64_t n_dst, bool last, cudaStream_t s);
// counted: the per-block live counts are already in blk (the learned prune
// step writes them), so only the scan and the write run.
cudaError_t launch_compact(const JobDev* d_job, uint64_t n_entries, bool counted, cudaStream_t s);
cudaError_t launch_history_compact(const JobDev* d_job, uint32_t* d_err, int grid, cudaStream_t s);
int compact_grid_size(int device);
cudaError_t jit_launch_compact(void* handle, const JobDev* d_jobs, int job, double2* d_amp, cudaStream_t s);
// Two launches: lane groups sum most outputs and list the large ones in
// d_big_list (count in d_big_count, zeroed by the caller); one block per
// listed output sums the rest.
// big_possible = false skips the block-per-output launch when no output
// can have more than RED_BIG_ITEMS items or RED_BIG_THREADS input states.
constexpr uint64_t RED_BIG_ITEMS = 4096;
// threads of the block-per-output pass; outputs whose input support has at
// least this many states also go to it (one thread per input state)
constexpr int RED_BIG_THREADS = 256;
cudaError_t launch_reduce(const JobDev* d_jobs, const uint64_t* d_job_out_begin, int n_jobs,
                          uint64_t total_out, double2* d_amp, unsigned int* d_big_count, uint64_t* d_big_list,
                          bool big_possible, cudaStream_t s);
int history_grid_size(int device);

// Straight-line engine (fs_jit.cpp): one generated persistent kernel for the
// root and suffix regions of every job of a batch.
struct JitJobSpec {
    const Op* ops;
    int G;
    const uint32_t* masks;
    const double2* fac;
    int W, c1, c2, Ap, Ar, As;
    double eps2;
    bool compact;
    std::vector<PrefixLevel> levels;   // empty: single-region prefix
    // exact reachability bound applied where the table is written; with
    // bound_counts the same kernel counts the live entries per compaction
    // block (the job has no learned pruner to do it)
    bool bound = false, bound_counts = false;
    BoundSpec bspec{};
    // with the bound: the bound after each op of the suffix that carries an
    // artificial source (evaluation position, spec for the ops after it)
    std::vector<std::pair<int, BoundSpec>> src_bounds;
};
// Whether the generated engine counts this job's valid leaves by phase (an
// exact suffix whose factors are all unit phases): no FP64 add per leaf.
bool jit_census(const JitJobSpec& J);
// The generated source for these jobs (what jit_build compiles), without
// compiling it.
std::string jit_source(const std::vector<JitJobSpec>& jobs);
// scales (per job): the constant factor the generated root and suffix
// leave out of every history (applied through the input coefficients).
int jit_build(const std::vector<JitJobSpec>& jobs, void** handle, std::string* err, double* compile_ms,
              std::string* source_out, std::vector<double2>* scales);
cudaError_t jit_launch_history(void* handle, const JobDev* d_jobs, const uint2* d_tiles, uint64_t n_tiles,
                               unsigned int* d_counter, cudaStream_t s);
cudaError_t jit_launch_prefix(void* handle, const JobDev* d_jobs, const uint64_t* d_begin, int n_jobs,
                              uint64_t total, cudaStream_t s);
void jit_release(void* handle);

// Sets the thread-local message read by fs_last_error and returns code.
int set_error(int code, const char* msg);

// Programmatic dependent launch.  The kernels of a run are launched so that
// each may be scheduled while the previous kernel on the stream finishes
// (its launch and block setup overlap the previous kernel's last blocks);
// every such kernel first waits for the previous grid to complete and its
// memory to be visible (griddepcontrol.wait) and then lets the next kernel
// be scheduled (griddepcontrol.launch_dependents).  FS_NO_PDL=1 in the
// environment launches them plainly.
#define FS_GRID_DEP() asm volatile("griddepcontrol.wait;\n\tgriddepcontrol.launch_dependents;" ::: "memory")
bool pdl_enabled();
// cudaLaunchKernelExC with the programmatic-serialization attribute (when
// enabled); args as for cudaLaunchKernel.
cudaError_t launch_ex(const void* func, dim3 grid, dim3 block, size_t smem, cudaStream_t s, void** args);
#ifdef __CUDACC__
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args... args)
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
    return cudaLaunchKernelEx(&cfg, kernel, ((KArgs)args)...);
}

// Compaction write of table block b (COMPACT_BLOCK entries, 256 threads x 4;
// every thread of the block calls it): each live entry (amplitude not the
// bottom NaN) goes to J.live at its rank among the live entries in table
// order, a pair's range of live ranks is recorded at its first entry (and
// closes the previous pair's), and the last table entry closes the last
// pair's.  scanned: J.blk holds each block's exclusive offset; otherwise
// it holds the blocks' counts, the block adds those before it (nblk is at
// most COMPACT_DIRECT_BLOCKS), and the last block writes the live total
// (stats[6]).  list (shared memory, optional): the block's live entries as
// offsets within the block, in table order.  write = false: only the list
// and the count (another CTA of the same block writes the compaction).
// learned_live: an entry carrying the scorer's cut mark counts as live (the
// scorer cutting this block's entries while its CTAs list them: every CTA
// then sees the same list, whichever cuts it reads).  Returns the block's
// live count.
__device__ __forceinline__ unsigned compact_block_write(const JobDev& J, unsigned b, unsigned nblk, int scanned,
                                                        uint16_t* list, bool write = true, bool learned_live = false)
{
    __shared__ unsigned s_pre[8], s_w[8];
    unsigned before = 0;
    if (!scanned && write) {
        unsigned t = 0;
        for (unsigned k = threadIdx.x; k < b; k += 256) t += J.blk[k];
        t = __reduce_add_sync(0xffffffffu, t);
        if ((threadIdx.x & 31) == 0) s_pre[threadIdx.x >> 5] = t;
        __syncthreads();
        for (int w = 0; w < 8; ++w) before += s_pre[w];
    }
    const uint64_t base = (uint64_t)b * COMPACT_BLOCK;
    bool lv[4];
    unsigned c = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const uint64_t e = base + (uint64_t)threadIdx.x * 4 + k;
        bool live = false;
        if (e < J.n_entries) {
            const double x = J.table[e].amp.x;
            const unsigned hi = (unsigned)__double2hiint(x) & 0x7fffffffu;
            live = !(hi > 0x7ff00000u || (hi == 0x7ff00000u && (unsigned)__double2loint(x) != 0u)) ||
                   (learned_live && (unsigned long long)__double_as_longlong(x) == LEARNED_CUT_BITS);
        }
        lv[k] = live;
        c += live;
    }
    unsigned x = c;   // inclusive warp scan of the per-thread counts
    for (int off = 1; off < 32; off <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, x, off);
        if ((threadIdx.x & 31) >= (unsigned)off) x += y;
    }
    if ((threadIdx.x & 31) == 31) s_w[threadIdx.x >> 5] = x;
    __syncthreads();
    unsigned woff = 0, total = 0;
    for (int w = 0; w < 8; ++w) {
        if (w < (int)(threadIdx.x >> 5)) woff += s_w[w];
        total += s_w[w];
    }
    if (!write) {   // the block's list only
        uint64_t pos = woff + x - c;
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (lv[k]) list[pos++] = (uint16_t)(threadIdx.x * 4 + k);
        return total;
    }
    if (!scanned && b + 1 == nblk && threadIdx.x == 0) J.stats[6] = (unsigned long long)before + total;
    const uint64_t first = (scanned ? (uint64_t)J.blk[b] : (uint64_t)before);
    uint64_t pos = first + woff + x - c;
    const uint64_t pmask = (1ull << J.Ap) - 1ull;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const uint64_t e = base + (uint64_t)threadIdx.x * 4 + k;
        if (e < J.n_entries && (e & pmask) == 0ull) {
            const uint64_t p = e >> J.Ap;
            J.prange[2 * p] = pos;
            if (p) J.prange[2 * p - 1] = pos;
        }
        if (lv[k]) {
            J.live[pos] = e;
            if (list) list[pos - first] = (uint16_t)(e - base);
            ++pos;
        }
        if (e + 1ull == J.n_entries) J.prange[2 * (e >> J.Ap) + 1] = pos;
    }
    return total;
}
#endif
cudaError_t probe_peaks(double* dfma_per_s, double* int_ops_per_s, int* sms);

}  // namespace fs

/*
 * feynsparse: selected computational-basis output amplitudes of a quantum
 * circuit as a reduced Feynman sum over histories, on one NVIDIA B300
 * (sm_103a).  C ABI; every entry point returns an int status (FS_OK = 0,
 * negative on error) and leaves a message for fs_last_error() on failure.
 *
 * The method is that of "Fewer Histories, Faster Paths" (Larssen, Pennati,
 * Asgrim, Peng, Markidis):
 *   - the transition amplitude <out|U_m ... U_1|in> (Eq. 1) of a sparse input
 *     |psi> = sum_in c_in |in> is sum_in c_in alpha^{in,out} (Eq. 2);
 *   - alpha is the sum over histories (Eqs. 3-5), reduced to a sum over the
 *     2^A assignments of artificial sources placed by a backward
 *     output-to-input sweep (Sec. IV-A, Eq. 7);
 *   - histories are evaluated with prefix/root/suffix checkpoints
 *     (Sec. IV-C, Algorithm 2) at cuts autotuned on Eq. 8;
 *   - invalid histories are pruned exactly and, when eps > 0, branches
 *     whose running |amplitude| falls below eps are dropped (Sec. IV-A,
 *     Observation 3).
 *
 * Conventions.
 *   Qubit q is bit q of a bit string (qubit 0 = least significant); at most
 *   FS_MAX_QUBITS qubits.  A bit string is passed as 2 uint64_t words (word 0
 *   holds qubits 0..63).  Matrices are indexed [output value][input value];
 *   for two targets the local value is bit(q[0]) + 2*bit(q[1]).
 *   H = [[1,1],[1,-1]]/sqrt2, X, Y = [[0,-i],[i,0]], Z = diag(1,-1),
 *   S = diag(1,i), T = diag(1,e^{i pi/4}), P(t) = diag(1,e^{it}),
 *   RX(t) = [[c,-is],[-is,c]], RY(t) = [[c,-s],[s,c]],
 *   RZ(t) = diag(e^{-it/2},e^{it/2}), RZZ(t) = diag(e^{-it/2}, e^{it/2},
 *   e^{it/2}, e^{-it/2}), c = cos(t/2), s = sin(t/2).
 *   Controls (ctrl_mask / ctrl_val, value 0 = negative control) are allowed
 *   on X (CNOT, Toffoli, MCX), Z (CZ, MCZ), P (controlled phase), S and T.
 *
 * Gate roles (Sec. II-A): H, RX, RY branch; X, Y, SWAP are deterministic;
 * Z, S, T, P, RZ, RZZ are wire-preserving; explicit U1/U2 matrices are
 * classified by their exact zero pattern (diagonal: wire-preserving; one
 * nonzero per column: deterministic; otherwise branching).  A branching
 * input whose wire is the circuit input wire of that qubit (no earlier gate
 * acted on the qubit except as a wire-preserving gate or a control) is a
 * natural source and takes its value from the input bit string; every other
 * branching input is an artificial source, numbered in the order the
 * backward sweep meets it.
 */
#ifndef FEYNSPARSE_H
#define FEYNSPARSE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define FS_API __attribute__((visibility("default")))
#else
#define FS_API
#endif

#define FS_MAX_QUBITS 128

/* status codes */
#define FS_OK 0
#define FS_ERR_INVALID (-1)        /* bad argument (null pointer, index out of range, ...) */
#define FS_ERR_UNSUPPORTED (-2)    /* unknown gate kind or controls on a kind that takes none */
#define FS_ERR_TOO_MANY_QUBITS (-3)
#define FS_ERR_NONUNITARY (-4)     /* explicit matrix with |U^+U - I| > 1e-12 */
#define FS_ERR_NOMEM (-5)
#define FS_ERR_CUDA (-6)           /* a CUDA runtime call failed; see fs_last_error() */
#define FS_ERR_TIMEOUT (-7)        /* a bounded device wait gave up (tensor-core scoring) */
#define FS_ERR_BAD_PROGRAM (-8)    /* the device found an opcode it does not know */
#define FS_ERR_TOO_LARGE (-9)      /* 2^A histories cannot be enumerated (A > 62) or
                                      the work exceeds the library's index range */
#define FS_ERR_STATE (-10)         /* call out of order (e.g. run before plan) */

/* gate kinds */
enum {
    FS_H = 0, FS_X = 1, FS_Y = 2, FS_Z = 3, FS_S = 4, FS_T = 5, FS_P = 6,
    FS_RX = 7, FS_RY = 8, FS_RZ = 9, FS_RZZ = 10, FS_SWAP = 11, FS_U1 = 12, FS_U2 = 13
};

/* One gate.  n_q targets in q[]; controls as 128-bit masks; theta for the
 * parametrised kinds; m[] = re/im interleaved row-major matrix for U1 (2x2,
 * 8 doubles) and U2 (4x4, 32 doubles). */
typedef struct fs_gate {
    uint32_t kind;
    uint32_t n_q;
    uint32_t q[2];
    uint64_t ctrl_mask[2];
    uint64_t ctrl_val[2];
    double theta;
    double m[32];
} fs_gate;

typedef struct fs_circuit fs_circuit;   /* opaque, owned by the library */
typedef struct fs_batch fs_batch;       /* opaque, owned by the library */

/* Result of the analysis (Sec. IV-A) and of the autotuned partition
 * (Sec. IV-C).  Cuts c1 <= c2 are positions in evaluation (output-to-input)
 * order: the prefix is evaluation positions [0, c1), the root [c1, c2), the
 * suffix [c2, n_gates). */
typedef struct fs_analysis {
    uint32_t n_qubits;
    uint32_t n_gates;
    uint32_t n_branch_vars;    /* branching inputs: natural + artificial */
    uint32_t n_natural;
    uint32_t A;                /* artificial sources */
    uint32_t n_wp, n_det, n_br;/* gate role counts */
    int32_t c1, c2;            /* autotuned cuts (for the request size last planned,
                                  or for a single output when none was) */
    uint32_t G_p, G_r, G_s;
    uint32_t A_p, A_r, A_s;
    uint64_t gateops_lo, gateops_hi;  /* Eq. 8 at (c1, c2), 128-bit */
    uint32_t max_ap, min_apr;  /* the autotuner's memory / parallelism constraints */
    uint32_t max_apr;          /* and its ceiling on A_p + A_r (items per pair) */
} fs_analysis;

/* Options of a batch.  split: 0 = autotuned, 1 = fixed cuts (c1, c2 applied
 * to every job), 2 = no checkpoints (Algorithm 1: a single region). */
typedef struct fs_options {
    uint32_t split;
    int32_t c1, c2;
    uint64_t table_budget_bytes;   /* checkpoint-table memory bound (0: 4 GiB) */
    uint64_t min_items;            /* parallelism floor for (prefix, root) items (0: 2^19) */
    uint64_t max_items;            /* ceiling on (prefix, root) items per job; bounds the
                                      per-tile partial sums (0: 2^28) */
    uint32_t engine;               /* history kernel: 0 = straight-line code generated per
                                      batch at upload (NVRTC, sm_103a), 1 = interpreter */
    uint32_t prefix_mode;          /* 0 = automatic: the prefix is split into levels at ops
                                      carrying sources where a cost model (ops per entry,
                                      32 B per entry read and written, one launch per
                                      level) says it pays; each level's gates run once per
                                      partial assignment; 1 = one region per prefix
                                      assignment, as in Algorithm 2; 2 = one level per
                                      branching op carrying a source */
} fs_options;

/* Counters of one job after a run. */
typedef struct fs_stats {
    uint64_t candidates;      /* S * M * 2^A */
    uint64_t completed;       /* leaves that reached the input boundary */
    uint64_t valid;           /* completed leaves with chi = 1 */
    uint64_t gate_visits;     /* gates evaluated, all kernels (Eq. 8 per pair in exact mode) */
    uint64_t history_visits;  /* of which in the root and suffix (history kernel) */
    uint64_t table_entries;   /* checkpoint entries written */
    int32_t c1, c2;
    uint32_t A_p, A_r, A_s;
    uint64_t learned_cuts;    /* checkpoint entries cut by the learned pruner */
    uint64_t live_entries;    /* checkpoint entries enumerated by the history kernel */
    uint64_t bound_cuts;      /* checkpoint entries cut by the exact reachability bound */
} fs_stats;

/* Thread-local message of the last failing call on this thread (library
 * plumbing; the paper has no counterpart).  Never NULL; owned by the
 * library and valid until the next failing call on the same thread. */
FS_API const char* fs_last_error(void);

/* Library version string (static storage; no counterpart in the paper). */
FS_API const char* fs_version(void);

/* Copies n_gates gates (host memory) into a new circuit on n_qubits qubits,
 * validates them (qubit indices, controls, unitarity of U1/U2 to 1e-12),
 * classifies their roles and places the artificial sources.  The gates are
 * in circuit order (the first gate acts first).  *out receives a handle to
 * free with fs_circuit_destroy.  Follows the statement of the problem
 * (Sec. II, Eq. 1) and the analysis of Sec. IV-A. */
FS_API int fs_circuit_create(const fs_gate* gates, size_t n_gates, uint32_t n_qubits,
                      fs_circuit** out);

/* Frees a circuit made by fs_circuit_create (NULL is accepted).  The circuit
 * of the statement of the problem (Sec. II, Eq. 1); batches that hold jobs
 * of it must be destroyed or re-planned without it first. */
FS_API int fs_circuit_destroy(fs_circuit* c);

/* Analysis for the basis input input_bits (2 words, host): fills *out with
 * the branching-variable and artificial-source counts and the autotuned
 * partition for one output; also makes input_bits the circuit's input
 * (S = 1, coefficient 1) until fs_set_input replaces it.  Sec. IV-A/IV-C. */
FS_API int fs_analyze(fs_circuit* c, const uint64_t* input_bits, fs_analysis* out);

/* Branching variables and artificial sources of the analysis (Sec. IV-A,
 * Eq. 7; Fig. 2 lists them for the four-qubit example).  Lists the
 * branching variables in backward-sweep order: per entry the gate
 * index (circuit order), the qubit, and the artificial source id or -1 for a
 * natural source.  Arrays of capacity cap (host); *count receives the total
 * (entries beyond cap are not written). */
FS_API int fs_branch_vars(const fs_circuit* c, int32_t* gate_index, int32_t* qubit, int32_t* source,
                   size_t cap, size_t* count);

/* Source placement in the graph form of Sec. IV-B (Fig. 4), for circuits of
 * CNOTs (one control, either polarity), SWAPs and single-qubit gates:
 * internal wires are nodes, each CNOT joins its control wire and the two
 * sides of its target (any two fix the third by XOR), diagonal and
 * single-qubit deterministic gates keep a wire, single-qubit branching
 * gates separate their two sides, and the input and output wires are known.
 * After the natural-source rule (a CNOT on a known wire is removed and its
 * other two wires merge), *n_sources receives the number of artificial
 * sources that make every wire known: method 0 = the backward sweep of
 * Sec. IV-A (A, any circuit), 1 = greedy (repeatedly the node on the most
 * unresolved CNOTs), 2 = the optimum by exhaustive search (at most 30
 * unknown wire classes, else FS_ERR_TOO_LARGE).  *n_nodes (may be NULL)
 * receives the unknown wire classes after merging.  FS_ERR_UNSUPPORTED for
 * other gates (methods 1, 2).  Analysis only: the history kernels use the
 * backward placement. */
FS_API int fs_source_placement(const fs_circuit* c, uint32_t method, uint32_t* n_sources, uint32_t* n_nodes);

/* Sparse input state sum_k coeffs[k] |support[k]> (Eq. 2): S bit strings of 2
 * words and S complex coefficients (re, im), host memory, copied. */
FS_API int fs_set_input(fs_circuit* c, const uint64_t* support_bits, const double* coeffs, size_t S);

/* Amplitudes <out|C|psi> = sum_in c_in alpha^{in,out} (Eqs. 1-2) of n_out
 * requested outputs (n_out x 2 words, host) into amp_out (2*n_out doubles,
 * re/im, host, caller-owned), each alpha the reduced history sum of Eq. 7
 * evaluated by Algorithm 2 at autotuned cuts (Eq. 8), with threshold eps
 * (0 = exact; eps > 0 drops branches below eps, Sec. IV-A Observation 3).
 * Synchronous: plans, copies to the device, runs the kernels on the legacy
 * default stream of the current device and copies back.  Device memory is
 * allocated and freed inside the call.  Errors: FS_ERR_INVALID (NULL
 * pointers, bits beyond the register), FS_ERR_TOO_LARGE (2^A not
 * enumerable), FS_ERR_NOMEM / FS_ERR_CUDA. */
FS_API int fs_amplitudes(fs_circuit* c, const uint64_t* outputs, size_t n_out, double eps,
                  double* amp_out);

/* ---- batches: many circuits and outputs in one persistent launch --------
 * A batch is the device form of the paper's output decomposition (Sec.
 * IV-D, Observations 5-6): every (output, input) pair of every job is an
 * independent work unit, and one persistent kernel drains a cost-sorted
 * tile queue in place of the server-worker balancer. */

/* New empty batch in *out (host object, freed by fs_batch_destroy): the
 * request queue of Sec. IV-D. */
FS_API int fs_batch_create(fs_batch** out);
/* Frees a batch of Sec. IV-D (NULL accepted); device workspaces stay the
 * caller's. */
FS_API int fs_batch_destroy(fs_batch* b);

/* CUDA device of the batch (Sec. IV-D: output shards may live on different
 * devices): plan, upload, run, finish and the feature query make it current
 * for their CUDA calls and restore the caller's device afterwards.  -1 (the
 * default) uses whatever device is current at each call.  Changing it drops
 * the plan.  FS_ERR_INVALID for a device index out of range. */
FS_API int fs_batch_set_device(fs_batch* b, int32_t device);

/* Batch options (may be NULL for defaults); call before fs_batch_plan.  The
 * split is the checkpoint partition of Sec. IV-C (autotuned on Eq. 8, fixed,
 * or none = Algorithm 1). */
FS_API int fs_batch_set_options(fs_batch* b, const fs_options* opt);

/* Adds a job (Eq. 2 for one circuit): circuit c (its current input state),
 * n_out outputs (host, copied), threshold eps (Sec. IV-A, Observation 3).  *job_id receives the job's index; its amplitudes
 * occupy amp_out[2*offset .. 2*(offset+n_out)) where offset is the sum of
 * n_out over earlier jobs. */
FS_API int fs_batch_add(fs_batch* b, fs_circuit* c, const uint64_t* outputs, size_t n_out,
                 double eps, uint32_t* job_id);

/* Fixes the checkpoint cuts (c1, c2) of one job (Sec. IV-C, Algorithm 2),
 * overriding the batch's split option
 * (both -1 restores it); 0 <= c1 <= c2 <= n_gates is checked at plan time.
 * Call before fs_batch_plan. */
FS_API int fs_batch_set_cuts(fs_batch* b, uint32_t job, int32_t c1, int32_t c2);

/* Compiles every job -- evaluation-order program of the backward sweep
 * (Sec. IV-A), cuts autotuned on Eq. 8 under the device's memory bounds
 * (Sec. IV-C), cost-sorted tile queue (Observation 6) -- and reports the
 * device workspace size in bytes (256-byte aligned sub-buffers).  Planning
 * again releases the generated kernel of the previous plan: graphs captured
 * from fs_batch_run before must be captured again after the next upload. */
FS_API int fs_batch_plan(fs_batch* b, size_t* workspace_bytes);

/* Staging of the boundary data (Sec. IV-D; the per-pair input and output
 * bit strings of Algorithm 2's InitializeState): copies the planned static
 * data (programs, bit strings, tile list) into the
 * caller's device workspace d_ws (at least workspace_bytes, 256-byte
 * aligned) on stream (a cudaStream_t, NULL = legacy default stream).  The
 * first upload of a plan builds the straight-line kernel (engine 0), stages
 * through pageable memory and returns after the copy; later uploads stage
 * through a pinned buffer owned by the batch and return at once (the copy is
 * ordered on stream; the next upload waits for it before reusing the
 * buffer).  A graph captured from fs_batch_run stays valid across uploads of
 * the same plan. */
FS_API int fs_batch_upload(fs_batch* b, void* d_ws, size_t ws_bytes, void* stream);

/* Algorithm 2 for every (output, input) pair of every job, summed per
 * output by Eq. 2.  Enqueues one evaluation of every job on stream: counter reset, prefix
 * expansion (checkpoint table), persistent history kernel over the atomic
 * tile queue, fixed-order reduction into d_amp_out (device, 2 * total
 * outputs doubles).  An exact job with the exact bound or a learned pruner
 * on the straight-line engine, with at least 5 sources in the root, fewer
 * than 32 input states and at most 4096 subtree sums per output, has its
 * outputs reduced by its compacted history kernel (the warp that stores an
 * output's last sum adds them, in the reduction kernel's order) and leaves
 * none to the reduction kernels.  Asynchronous and free of host synchronisation, so it
 * can be captured into a CUDA graph.  Its kernels are launched with
 * programmatic dependent launch (each waits for the previous grid before
 * touching memory); FS_NO_PDL=1 in the environment launches them plainly.
 * Requires fs_batch_upload on the same workspace first. */
FS_API int fs_batch_run(fs_batch* b, void* d_ws, double* d_amp_out, void* stream);

/* Waits for stream, reads the device error word and the per-job counters
 * (fs_stats array of capacity cap, host) of the last run: the candidate,
 * completed and valid history counts of Eq. 7 and the gate visits of
 * Eq. 8.  Errors found on the device: FS_ERR_BAD_PROGRAM (an opcode the
 * interpreter does not know), FS_ERR_TIMEOUT (a bounded wait gave up). */
FS_API int fs_batch_finish(fs_batch* b, void* d_ws, void* stream, fs_stats* stats, size_t cap);

/* The CUDA C++ source of the straight-line engine for the planned batch:
 * the regions of Algorithm 2 (Sec. IV-C) of every job as generated code,
 * what the next fs_batch_upload compiles (NVRTC, sm_103a).  No CUDA call.
 * Writes at most cap - 1 characters and a terminating NUL into buf (host;
 * NULL with cap 0 only queries), the full length into *len.
 * FS_ERR_STATE before fs_batch_plan. */
FS_API int fs_batch_generated_source(const fs_batch* b, char* buf, size_t cap, size_t* len);

/* Bytes fs_batch_upload copies host-to-device (programs, bit strings,
 * descriptors, tile list) for the planned batch: the boundary staging of
 * Sec. IV-D, reported for end-to-end throughput. */
FS_API int fs_batch_upload_bytes(const fs_batch* b, size_t* bytes);

/* Engine actually used by the last fs_batch_upload (0 straight-line, 1
 * interpreter) and the milliseconds spent generating and compiling the
 * straight-line kernel (the AdvanceCheckpoint regions of Algorithm 2 as
 * generated code).  FS_ERR_STATE before the first upload. */
FS_API int fs_batch_engine(const fs_batch* b, uint32_t* engine, double* compile_ms);

/* Total outputs over the jobs added so far (the requested set B_out of
 * Sec. IV-D, summed over jobs). */
FS_API int fs_batch_total_outputs(const fs_batch* b, size_t* n);

/* Launch accounting of Algorithm 2's stages: the number of kernel launches
 * fs_batch_run enqueues (prefix levels or the
 * flat prefix, the reduction kernels unless every job with outputs reduces
 * them itself (see fs_batch_run), the tiled history kernel when any job is
 * exact, and per pruned job a learned-prune launch if attached plus the
 * compaction: a count pass unless the bound or the pruner counted, a scan
 * when the table has more than 1024 compaction blocks of 1024 entries, and
 * the write (it also records each pair's live range), then the history
 * over live entries). */
FS_API int fs_batch_launch_count(const fs_batch* b, uint32_t* n);

/* Per-output cost (the paper's per-output distribution of work, Sec. V,
 * Fig. 11): with d_counts set (device, 2 x n_out uint64 of the job, 8-byte
 * aligned), every fs_batch_run zeroes it and adds each output's completed
 * and valid leaves ({completed, valid} per output, in request order) as the
 * history kernels finish its items; NULL turns it off.  Call before
 * fs_batch_upload.  Summed over outputs the counts equal fs_stats. */
FS_API int fs_batch_trace_outputs(fs_batch* b, uint32_t job, uint64_t* d_counts);

/* Stage timing (the paper times its kernel per output, Fig. 11; here per
 * stage of Algorithm 2).  enable != 0 makes fs_batch_run record CUDA events
 * around its stages (as event nodes when the stream is being captured). */
FS_API int fs_batch_time_kernels(fs_batch* b, int enable);
/* Milliseconds of the five stages of the last timed run: prefix expansion,
 * learned pruning, compaction, history, reduction (ms: 5 floats, host).
 * FS_ERR_STATE when no timed run was recorded. */
FS_API int fs_batch_stage_ms(fs_batch* b, float* ms);
/* Milliseconds of the last timed run's prefix expansion, history and
 * reduction stages (each pointer may be NULL). */
FS_API int fs_batch_kernel_ms(fs_batch* b, float* prefix_ms, float* history_ms, float* reduce_ms);

/* Per-region opcode histogram of a planned job (the G_p, G_r, G_s of Eq. 8
 * broken down by gate role, Sec. II-A): counts[r * FS_N_OPCODES + k]
 * for region r (0 prefix, 1 root, 2 suffix) and opcode k, into a host array
 * of 3 * FS_N_OPCODES uint32_t.  Opcode numbering is the library's internal
 * one (1 = X, 2 = MCX, 3 = SWAP, 4 = PERM1, 5 = PERM2, 6 = DIAG1, 7 = PH1,
 * 8 = NEG1, 9 = MCPH, 10 = MCNEG, 11 = DIAG2, 12 = H, 13 = BR1, 14 = BR2);
 * used to count algorithmic work for throughput reports. */
#define FS_N_OPCODES 16
FS_API int fs_batch_op_histogram(const fs_batch* b, uint32_t job, uint32_t* counts);

/* Algorithmic work (Eq. 8 counts gate visits; this weighs each visit by
 * its instructions) of one execution of each region (0 prefix, 1 root,
 * 2 suffix) of a planned job, as integer instructions on the register state
 * and FP64 instructions, from the job's program (control-mask words that are
 * not all zero, factor forms); index 3 is the work per completed leaf (chi
 * test, integer) and per valid leaf (accumulation, FP64).  For the
 * straight-line engine the root's figure includes the item loop around it
 * (24 integer instructions: indices, entry cache, sums) and the leaf figure
 * the suffix loop's control (12); where the engine counts a unit-phase
 * suffix's valid leaves by phase, a valid leaf costs 4 integer instructions
 * and no FP64, a root one product.  Arrays of 4 doubles (host).  Used to
 * state kernel throughput against the issue and FP64 rooflines. */
FS_API int fs_batch_region_work(const fs_batch* b, uint32_t job, double* int_ops, double* fp64_ops);

/* Register width (32-bit words: 1, 2 or 4) of a planned job's state (the
 * internal-wire values of Sec. II-A held as a bit register). */
FS_API int fs_batch_job_words(const fs_batch* b, uint32_t job, uint32_t* words);

/* Roofline denominators (no counterpart in the paper).  Measures, on the
 * current device, the sustained FP64 FMA rate (FMA/s) and
 * the 32-bit integer logic rate (ops/s) with short probe kernels, and
 * reports the SM count.  Allocates and frees 256 bytes of device memory. */
FS_API int fs_probe_peaks(double* dfma_per_s, double* int_ops_per_s, int32_t* sms);

/* Exact pruning at the checkpoint (Sec. IV-A Observation 3: a history that
 * cannot reach b_in contributes exactly zero; here decided for a whole
 * subtree at once).  With enable != 0, fs_batch_run cuts every checkpoint
 * entry (sigma_p, beta_p) of the job whose state provably cannot reach the
 * input b_in through the ops after the cut: a qubit that no remaining op
 * targets must already hold b_in's value, and a field of contiguous qubits
 * changed only by controlled +-1 cascades of multi-controlled X gates (an
 * incrementer / decrementer) moves by at most the number of such cascades
 * left, so a field value farther than that (cyclically) from b_in's is
 * unreachable.  Cut entries are counted in fs_stats.bound_cuts; the job runs
 * the history over the compacted live entries, so amplitudes are the exact
 * ones.  The straight-line engine also tests the bound after every op of
 * the suffix that carries an artificial source (the cut histories' leaves
 * are all invalid: fewer leaves complete, the amplitudes are unchanged).
 * Call before fs_batch_plan; FS_ERR_UNSUPPORTED from the plan when more
 * than 4 disjoint cascade fields follow the cut. */
FS_API int fs_batch_set_exact_bound(fs_batch* b, uint32_t job, int32_t enable);

/* ---- learned pruning at the checkpoint boundary ---------------------------
 * Not in the paper: a proposal built on its checkpoint boundary (Sec. IV-C).
 * A 16 -> 128 -> 128 -> 1 ReLU MLP scores each live checkpoint entry (the
 * partial history after the prefix of Algorithm 2) by the predicted
 * log10 |exact subtree sum| of its root and suffix completions; entries
 * scoring below tau are cut and every other entry is enumerated exactly (with
 * eps pruning as configured).  BF16 tensor-core operands, FP32 accumulation:
 * scoring (fs_mlp_forward and the prune step of fs_batch_run) on tcgen05.mma
 * with accumulators in tensor memory, training (fs_mlp_grad) on mma.sync.
 * Parameters: FS_MLP_PARAMS FP32 values in device memory, laid out W1[16][128],
 * b1[128], W2[128][128], b2[128], w3[128], b3 (W[k][n]: input k to output n).
 * Features (16 FP32 per entry): |beta|, log10|beta|, Re beta/|beta|,
 * Im beta/|beta|, (1 + log2 |int(sigma) - int(b_in)|)/8 (0 if equal; registers read as
 * unsigned integers, qubit q = bit q), c1/G, (A - A_p)/A,
 * Hamming(sigma, b_in)/n, and (sigma xor b_in) on the qubits of the next 8
 * artificial sources after the prefix. */
#define FS_MLP_PARAMS 18817

/* Scoring (learned pruning has no counterpart in the paper; it scores the
 * checkpoint entries of Algorithm 2, Sec. IV-C).
 * y[i] = MLP(x[i]) for n rows of 16 FP32 features (device pointers; x rows
 * 16-byte aligned, else FS_ERR_INVALID).  Asynchronous on stream; returns
 * FS_ERR_CUDA on a launch error.  The scoring kernel bounds its waits on the
 * tensor cores; in the batch path a wait that gives up is reported as
 * FS_ERR_TIMEOUT by fs_batch_finish, here (no status word) it leaves the
 * rows of the tiles it did not finish unwritten. */
FS_API int fs_mlp_forward(const float* d_params, const float* d_x, uint64_t n, float* d_y, void* stream);

/* Training of the pruner (no counterpart in the paper; targets are exact
 * subtree sums of Algorithm 2's checkpoint entries, Sec. IV-C).
 * Loss mean((y - target)^2) and its gradient: d_grad receives FS_MLP_PARAMS
 * gradient values followed by the loss (device, FS_MLP_PARAMS + 1 floats;
 * zeroed by the call).  Gradients are accumulated with atomics (summation
 * order not fixed). */
FS_API int fs_mlp_grad(const float* d_params, const float* d_x, const float* d_target, uint64_t n,
                       float* d_grad, void* stream);

/* Training of the pruner (no counterpart in the paper).
 * One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) on the FP32 parameters with
 * moment buffers d_m, d_v (device, FS_MLP_PARAMS floats each); step >= 1. */
FS_API int fs_mlp_adam(float* d_params, float* d_m, float* d_v, const float* d_grad, float lr, int32_t step,
                       void* stream);

/* Pruner inputs (no counterpart in the paper) of the checkpoint entries
 * (sigma_p, beta_p) of Algorithm 2 (Sec. IV-C).
 * Features of every checkpoint entry of a job after a run (entries = pairs x
 * 2^A_p, 16 floats each, device; bottom entries get NaN in feature 0). */
FS_API int fs_batch_features(fs_batch* b, uint32_t job, void* d_ws, float* d_features, void* stream);

/* Training targets of the pruner (no counterpart in the paper; S_i is the
 * exact sum over one checkpoint entry's root and suffix completions,
 * Algorithm 2): d_target[i] = max(log10 |S_i|, floor_log10)
 * for n logged subtree sums S_i (d_sums: n x (re, im) doubles, device, as
 * written by a logging run; d_target: n floats, device), computed in FP64
 * and rounded to FP32; an exactly zero sum gives the floor.  Asynchronous on
 * stream.  FS_ERR_INVALID for NULL pointers or a non-finite floor. */
FS_API int fs_mlp_targets(const double* d_sums, uint64_t n, double floor_log10, float* d_target, void* stream);

/* Logging runs (no counterpart in the paper; the items are Algorithm 2's
 * (h_p, h_r) loop iterations, Sec. IV-C): makes the history kernel write each (prefix, root) item's
 * exact subtree sum (re, im doubles) into d_log (device, 2 x items doubles,
 * items from fs_batch_log_items).  With a fixed split c1 = c2 the items are
 * the checkpoint entries.  Call before fs_batch_upload; NULL turns it off. */
FS_API int fs_batch_log_subtrees(fs_batch* b, uint32_t job, double* d_log);
/* Items of a planned job: pairs x 2^(A_p + A_r), the (h_p, h_r) iterations
 * of Algorithm 2 (Sec. IV-C), i.e. the length of its logging buffer.
 * FS_ERR_STATE before fs_batch_plan. */
FS_API int fs_batch_log_items(const fs_batch* b, uint32_t job, uint64_t* items);

/* Learned pruning at the checkpoint boundary of Algorithm 2 (no counterpart
 * in the paper; an alternative to the threshold of Sec. IV-A Observation 3).
 * Attaches a trained pruner (device parameters, threshold tau on the
 * predicted log10 |subtree sum|) to a job; fs_batch_run then scores and cuts
 * checkpoint entries between the prefix and history kernels.  Call before
 * fs_batch_plan (it changes the job's layout); NULL detaches it.  Jobs with a
 * pruner or eps > 0 run the history over the compacted list of live
 * checkpoint entries, so cut entries cost nothing downstream.  With the
 * exact bound also set (fs_batch_set_exact_bound) the bound cuts first and
 * the pruner scores only the entries it leaves live; up to 1024 compaction
 * blocks (2^20 table entries) the scoring kernel also writes the compaction
 * (on the generated engine an exact job with A_r >= 5 then runs in three
 * launches: prefix, scorer, history; fs_batch_launch_count gives the count). */
FS_API int fs_batch_set_pruner(fs_batch* b, uint32_t job, const float* d_params, float tau);

/* ---- output sharding across devices or processes -----------------------
 * Outputs are independent (Sec. IV-D, Observation 5) but their costs differ
 * (Observation 6).  fs_lpt_assign splits n work units with predicted costs
 * cost[i] (>= 0, host; e.g. S x Eq. 8 of each output's circuit) over n_ranks
 * ranks by longest-processing-time-first: units in descending cost (ties by
 * index) each go to the least loaded rank (ties to the lowest).  rank[i]
 * (host, n entries) receives unit i's rank and load (host, n_ranks entries,
 * may be NULL) the summed cost per rank.  No CUDA call; deterministic, so
 * every process computes the same assignment.  FS_ERR_INVALID for NULL
 * arrays, n_ranks = 0 or a cost that is negative or not finite. */
FS_API int fs_lpt_assign(const double* cost, size_t n, uint32_t n_ranks, uint32_t* rank, double* load);

/* ---- failure detection (no counterpart in the paper) ----------------------
 * Bounded device waits: every wait of the tensor-core scoring kernel on an
 * MMA-completion barrier gives up after `polls` polls, records
 * FS_ERR_TIMEOUT for fs_batch_finish, issues no further MMA and waits
 * (bounded) for the MMAs already committed before releasing its tensor
 * memory, so the context stays usable.  polls < 0 restores the default
 * (2^22); 0 makes every wait give up at once (a test of that path).
 * Process-wide; set it while no batch is running.  FS_ERR_INVALID above
 * 2^32 - 1. */
FS_API int fs_set_wait_limit(int64_t polls);

/* Byte offset of a planned job's op program (16-byte ops in the evaluation
 * order of the backward sweep, Sec. IV-A)
 * inside the workspace, and its op count: lets a caller inspect the uploaded
 * program, or corrupt it on purpose to test the device-side opcode check
 * (the interpreter engine reports an unknown opcode as FS_ERR_BAD_PROGRAM
 * from fs_batch_finish).  FS_ERR_STATE before fs_batch_plan. */
FS_API int fs_batch_program_offset(const fs_batch* b, uint32_t job, size_t* offset, size_t* n_ops);

/* ---- allocation-free variant ---------------------------------------------
 * The paper has no counterpart to this entry point; it exists for callers
 * that cannot allocate device memory at call time (code that must draw every
 * device allocation from a pool it does not own, or that must not grow the
 * process's device footprint while it runs).
 *
 * fs_amplitudes_noalloc computes the same amplitudes as fs_amplitudes
 * (outputs: n_out x 2 words, host; amp_out: 2 * n_out doubles re/im, host,
 * caller-owned; eps: 0 = exact) but calls no cudaMalloc, cudaFree or other
 * allocating routine.  Its whole device workspace -- programs, bit strings,
 * checkpoint table, partial sums, counters and the staged amplitudes -- lives
 * in one static device array of FS_NOALLOC_SCRATCH_BYTES bytes, which every
 * GPU that loads this part of the library holds until the process exits.
 * A request whose workspace would exceed it fails with FS_ERR_TOO_LARGE and a
 * message giving both sizes.
 *   - The first call on a device looks up that array's device address (once
 *     per device, with the device current); make that first call before any
 *     stream capture.  Under CUDA's lazy module loading that first call may
 *     also load this part of the library onto the device, which is when the
 *     device footprint grows by the array and the kernel code; later calls
 *     leave free device memory unchanged.
 *   - Every call uses the same array and leaves its contents behind; the
 *     counters that must start at zero are cleared by each call.  Calls whose
 *     GPU work overlaps (other host threads, or several streams) race on the
 *     array: serialise them.
 *   - It runs the library's precompiled kernels (the interpreter engine), so
 *     no code is generated or loaded onto the device at call time; exact-mode
 *     amplitudes agree with fs_amplitudes' generated code within rounding
 *     (1e-12 absolute + 1e-10 relative), threshold-mode ones bit for bit.
 *   - stream: a cudaStream_t (NULL = legacy default stream); the call
 *     synchronises it before returning. */
#define FS_NOALLOC_SCRATCH_BYTES (16u << 20)
FS_API int fs_amplitudes_noalloc(fs_circuit* c, const uint64_t* outputs, size_t n_out, double eps,
                                 double* amp_out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* FEYNSPARSE_H */

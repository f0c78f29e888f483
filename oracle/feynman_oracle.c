/*
 * Reference oracle (test infrastructure, not the product): a plain, slow CPU
 * restatement of the paper's reduced-history method.  Only the tests, the
 * smoke check and the benchmark's CPU-baseline leg may load this file.  It
 * shares no code with the CUDA library: its own gate matrices, its own
 * analysis, its own enumeration.
 *
 * What it computes (paper Sec. II and Sec. IV):
 *   amp(o) = sum_{in in supp psi} <in|psi> * alpha^{in,o}            (Eq. 2)
 *   alpha^{in,o} = sum_{a in {0,1}^A} chi(a) alpha_a                   (Eq. 7)
 * with artificial sources placed by a backward (output -> input) sweep
 * (Sec. IV-A) and histories evaluated either one by one (Algorithm 1) or
 * with the prefix/root/suffix checkpoints of Algorithm 2 (Sec. IV-C).
 *
 * Readings of the paper used here (the paper is silent on these points):
 *  - Gate roles are structural for named kinds (Sec. II-A): H, RX, RY
 *    branch; X, Y, SWAP (and X with controls) are deterministic; Z, S, T,
 *    P, RZ, RZZ (and Z/S/T/P with controls) are wire-preserving.  Explicit
 *    U1/U2 matrices are classified numerically: diagonal -> wire-preserving,
 *    one nonzero per column -> deterministic, otherwise branching.
 *  - A branching input is a natural source when its wire is the circuit's
 *    input wire for that qubit, i.e. no earlier gate acted on the qubit
 *    other than as a wire-preserving gate or a control (Fig. 2: H on q1 is
 *    natural, H on q0 and q3 are artificial; Table 1 counts).
 *  - Artificial sources are numbered in backward-encounter order; a
 *    two-qubit branching gate takes one per non-natural target, ascending.
 *  - chi(a) = 1 iff no factor on the path is exactly zero and the state
 *    reached at the input boundary equals the input bit string.
 *  - Threshold pruning (Sec. IV-A, Observation 3): right after the factor of
 *    a branching gate that carries an artificial source is applied, the
 *    history (and so its whole subtree) is dropped when |beta| < eps,
 *    tested as fma(re, re, im*im) < eps*eps.
 *  - Complex products use re = fma(a.re,b.re,-(a.im*b.im)),
 *    im = fma(a.re,b.im,a.im*b.re); this file is compiled without FP
 *    contraction so the formula is exactly what runs.
 *  - Sums over histories use Neumaier's compensated summation
 *    (Neumaier 1974) on the real and imaginary parts separately.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum {
    K_H = 0, K_X, K_Y, K_Z, K_S, K_T, K_P, K_RX, K_RY, K_RZ, K_RZZ, K_SWAP,
    K_U1, K_U2, K_NKINDS
};
enum { ROLE_WP = 0, ROLE_DET = 1, ROLE_BR = 2 };

typedef struct {
    int32_t kind;
    int32_t q0, q1;
    int32_t pad;
    uint64_t cmask[2], cval[2];
    double theta;
    double m[32];
} orc_gate_in;

typedef struct { double re, im; } cplx;

static cplx cmul(cplx a, cplx b)
{
    cplx r;
    r.re = fma(a.re, b.re, -(a.im * b.im));
    r.im = fma(a.re, b.im, a.im * b.re);
    return r;
}

static cplx cx(double re, double im) { cplx c = {re, im}; return c; }

/* One gate after analysis: its base matrix over its targets, its role. */
typedef struct {
    int role;
    int k;            /* number of targets (1 or 2) */
    int q[2];
    uint64_t cmask[2], cval[2];
    cplx u[16];       /* base matrix, u[out * dim + in] */
    int src[2];       /* per target: source id, -1 natural, -2 not branching */
} ogate;

typedef struct {
    int n, G, A;
    ogate* g;
} ocirc;

static int getbit(const uint64_t s[2], int q) { return (int)((s[q >> 6] >> (q & 63)) & 1u); }
static void setbit(uint64_t s[2], int q, int v)
{
    uint64_t m = (uint64_t)1 << (q & 63);
    if (v) s[q >> 6] |= m; else s[q >> 6] &= ~m;
}

/* Base matrices in the conventions of the library documentation:
 * S = diag(1,i), T = diag(1,e^{i pi/4}), P(t) = diag(1,e^{it}),
 * RX(t) = [[c,-is],[-is,c]], RY(t) = [[c,-s],[s,c]], RZ(t) = diag(e^{-it/2}, e^{it/2}),
 * RZZ(t) = exp(-i t Z(x)Z / 2), with c = cos(t/2), s = sin(t/2). */
static int build_gate(const orc_gate_in* in, ogate* g)
{
    memset(g, 0, sizeof(*g));
    g->q[0] = in->q0; g->q[1] = in->q1;
    g->cmask[0] = in->cmask[0]; g->cmask[1] = in->cmask[1];
    g->cval[0] = in->cval[0]; g->cval[1] = in->cval[1];
    g->src[0] = g->src[1] = -2;
    double t = in->theta, c = cos(t / 2.0), s = sin(t / 2.0), h = sqrt(0.5);
    int dim = 2;
    g->k = 1;
    switch (in->kind) {
    case K_H: g->u[0] = cx(h, 0); g->u[1] = cx(h, 0); g->u[2] = cx(h, 0); g->u[3] = cx(-h, 0); g->role = ROLE_BR; break;
    case K_X: g->u[1] = cx(1, 0); g->u[2] = cx(1, 0); g->role = ROLE_DET; break;
    case K_Y: g->u[1] = cx(0, -1); g->u[2] = cx(0, 1); g->role = ROLE_DET; break;
    case K_Z: g->u[0] = cx(1, 0); g->u[3] = cx(-1, 0); g->role = ROLE_WP; break;
    case K_S: g->u[0] = cx(1, 0); g->u[3] = cx(0, 1); g->role = ROLE_WP; break;
    case K_T: g->u[0] = cx(1, 0); g->u[3] = cx(cos(M_PI / 4.0), sin(M_PI / 4.0)); g->role = ROLE_WP; break;
    case K_P: g->u[0] = cx(1, 0); g->u[3] = cx(cos(t), sin(t)); g->role = ROLE_WP; break;
    case K_RX: g->u[0] = cx(c, 0); g->u[1] = cx(0, -s); g->u[2] = cx(0, -s); g->u[3] = cx(c, 0); g->role = ROLE_BR; break;
    case K_RY: g->u[0] = cx(c, 0); g->u[1] = cx(-s, 0); g->u[2] = cx(s, 0); g->u[3] = cx(c, 0); g->role = ROLE_BR; break;
    case K_RZ: g->u[0] = cx(c, -s); g->u[3] = cx(c, s); g->role = ROLE_WP; break;
    case K_RZZ:
        dim = 4; g->k = 2;
        g->u[0 * 4 + 0] = cx(c, -s); g->u[3 * 4 + 3] = cx(c, -s);
        g->u[1 * 4 + 1] = cx(c, s);  g->u[2 * 4 + 2] = cx(c, s);
        g->role = ROLE_WP; break;
    case K_SWAP:
        dim = 4; g->k = 2;
        g->u[0 * 4 + 0] = cx(1, 0); g->u[1 * 4 + 2] = cx(1, 0);
        g->u[2 * 4 + 1] = cx(1, 0); g->u[3 * 4 + 3] = cx(1, 0);
        g->role = ROLE_DET; break;
    case K_U1:
    case K_U2: {
        dim = in->kind == K_U1 ? 2 : 4;
        g->k = in->kind == K_U1 ? 1 : 2;
        for (int i = 0; i < dim * dim; i++) g->u[i] = cx(in->m[2 * i], in->m[2 * i + 1]);
        int diag = 1, perm = 1;
        for (int col = 0; col < dim; col++) {
            int nz = 0;
            for (int row = 0; row < dim; row++) {
                cplx v = g->u[row * dim + col];
                if (v.re != 0.0 || v.im != 0.0) { nz++; if (row != col) diag = 0; }
            }
            if (nz != 1) perm = 0;
        }
        g->role = diag ? ROLE_WP : (perm ? ROLE_DET : ROLE_BR);
        break;
    }
    default: return -1;
    }
    if ((g->cmask[0] | g->cmask[1]) && !(in->kind == K_X || in->kind == K_Z || in->kind == K_P ||
                                         in->kind == K_S || in->kind == K_T))
        return -1;
    return 0;
}

/* Analysis: natural sources (input-adjacent branching inputs), then the
 * backward sweep that numbers the artificial sources. */
static int analyze(ocirc* C)
{
    int n = C->n;
    char* touched = (char*)calloc((size_t)n, 1);
    for (int gi = 0; gi < C->G; gi++) {
        ogate* g = &C->g[gi];
        if (g->role == ROLE_BR)
            for (int t = 0; t < g->k; t++) g->src[t] = touched[g->q[t]] ? 0 : -1;  /* 0 = artificial, numbered below */
        if (g->role == ROLE_DET || g->role == ROLE_BR)
            for (int t = 0; t < g->k; t++) touched[g->q[t]] = 1;
    }
    free(touched);
    int A = 0;
    for (int gi = C->G - 1; gi >= 0; gi--) {
        ogate* g = &C->g[gi];
        if (g->role != ROLE_BR) continue;
        int order[2] = {0, 1};
        if (g->k == 2 && g->q[1] < g->q[0]) { order[0] = 1; order[1] = 0; }
        for (int j = 0; j < g->k; j++) {
            int t = order[j];
            if (g->src[t] == 0) g->src[t] = A++;
        }
    }
    C->A = A;
    return 0;
}

static int ctrl_ok(const ogate* g, const uint64_t s[2])
{
    return ((s[0] & g->cmask[0]) == g->cval[0]) && ((s[1] & g->cmask[1]) == g->cval[1]);
}

/* One gate in evaluation (backward) order.  The state holds the wire values
 * on the output side of the gate and is moved to its input side.  Returns 0
 * when the factor is exactly zero. */
static int step_gate(const ogate* g, uint64_t st[2], cplx* amp, const uint8_t* h,
                     const uint64_t b_in[2], int* has_src)
{
    int dim = g->k == 1 ? 2 : 4;
    int out = getbit(st, g->q[0]) | (g->k == 2 ? getbit(st, g->q[1]) << 1 : 0);
    int inv = out;
    cplx f = cx(1, 0);
    *has_src = 0;
    if (g->role == ROLE_WP) {
        if (ctrl_ok(g, st)) f = g->u[out * dim + out];
    } else if (g->role == ROLE_DET) {
        if (ctrl_ok(g, st)) {
            inv = -1;
            for (int col = 0; col < dim; col++) {
                cplx v = g->u[out * dim + col];
                if (v.re != 0.0 || v.im != 0.0) { inv = col; f = v; break; }
            }
            if (inv < 0) return 0;
        }
    } else {
        inv = 0;
        for (int t = 0; t < g->k; t++) {
            int b;
            if (g->src[t] < 0) b = getbit(b_in, g->q[t]);
            else { b = h[g->src[t]]; *has_src = 1; }
            inv |= b << t;
        }
        f = g->u[out * dim + inv];
    }
    if (f.re == 0.0 && f.im == 0.0) return 0;
    if (!(f.re == 1.0 && f.im == 0.0)) *amp = cmul(*amp, f);
    for (int t = 0; t < g->k; t++) setbit(st, g->q[t], (inv >> t) & 1);
    return 1;
}

static int below_eps(cplx a, double eps)
{
    return fma(a.re, a.re, a.im * a.im) < eps * eps;
}

/* AdvanceCheckpoint over the gates of evaluation positions [e0, e1).
 * Returns 1 on success, 0 on bottom (zero factor or pruned). */
static int advance(const ocirc* C, int e0, int e1, uint64_t st[2], cplx* amp, const uint8_t* h,
                   const uint64_t b_in[2], double eps, uint64_t* visits)
{
    for (int e = e0; e < e1; e++) {
        const ogate* g = &C->g[C->G - 1 - e];
        int has_src;
        (*visits)++;
        if (!step_gate(g, st, amp, h, b_in, &has_src)) return 0;
        if (eps > 0.0 && has_src && below_eps(*amp, eps)) return 0;
    }
    return 1;
}

typedef struct { double s, c; } neum;
static void neum_add(neum* a, double x)
{
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
    else a->c += (x - t) + a->s;
    a->s = t;
}

typedef struct {
    uint64_t completed, valid, visits;
} ocount;

/* Number of artificial sources among evaluation positions [e0, e1). */
static int sources_in(const ocirc* C, int e0, int e1)
{
    int a = 0;
    for (int e = e0; e < e1; e++) {
        const ogate* g = &C->g[C->G - 1 - e];
        if (g->role == ROLE_BR)
            for (int t = 0; t < g->k; t++) a += g->src[t] >= 0;
    }
    return a;
}

/* alpha^{b_in, b_out} by Algorithm 2 with checkpoints at evaluation
 * positions c1 <= c2 (c1 = c2 = 0 degenerates to Algorithm 1: one region). */
static cplx pair_amplitude(const ocirc* C, const uint64_t b_in[2], const uint64_t b_out[2],
                           double eps, int c1, int c2, ocount* cnt)
{
    int Ap = sources_in(C, 0, c1), Ar = sources_in(C, c1, c2), As = sources_in(C, c2, C->G);
    uint8_t* h = (uint8_t*)calloc((size_t)C->A + 1, 1);
    neum sr = {0, 0}, si = {0, 0};
    for (uint64_t hp = 0; hp < ((uint64_t)1 << Ap); hp++) {
        for (int j = 0; j < Ap; j++) h[j] = (uint8_t)((hp >> j) & 1);
        uint64_t sp[2] = {b_out[0], b_out[1]};
        cplx bp = cx(1, 0);
        if (!advance(C, 0, c1, sp, &bp, h, b_in, eps, &cnt->visits)) continue;
        for (uint64_t hr = 0; hr < ((uint64_t)1 << Ar); hr++) {
            for (int j = 0; j < Ar; j++) h[Ap + j] = (uint8_t)((hr >> j) & 1);
            uint64_t sr_[2] = {sp[0], sp[1]};
            cplx br = bp;
            if (!advance(C, c1, c2, sr_, &br, h, b_in, eps, &cnt->visits)) continue;
            for (uint64_t hs = 0; hs < ((uint64_t)1 << As); hs++) {
                for (int j = 0; j < As; j++) h[Ap + Ar + j] = (uint8_t)((hs >> j) & 1);
                uint64_t ss[2] = {sr_[0], sr_[1]};
                cplx bs = br;
                if (!advance(C, c2, C->G, ss, &bs, h, b_in, eps, &cnt->visits)) {
                    continue;
                }
                cnt->completed++;
                if (ss[0] == b_in[0] && ss[1] == b_in[1]) {
                    cnt->valid++;
                    neum_add(&sr, bs.re);
                    neum_add(&si, bs.im);
                }
            }
        }
    }
    free(h);
    return cx(sr.s + sr.c, si.s + si.c);
}

/* alpha^{b_in, b_out} as a depth-first search over the artificial sources in
 * the order the backward sweep meets them (the per-source limit of the
 * checkpointing of Sec. IV-C: every gate is evaluated once per assignment of
 * the sources met before it).  At a branching gate carrying artificial
 * sources each value of those sources is tried in turn; a branch whose
 * factor is exactly zero, or whose |beta| falls below eps right after that
 * factor (Sec. IV-A, Observation 3), is dropped with its whole subtree.
 * The surviving leaves, their chi test and their products are those of
 * Algorithm 1 / Algorithm 2 with the same threshold. */
typedef struct {
    const ocirc* C;
    const uint64_t* b_in;
    double eps;
    uint8_t* h;
    ocount* cnt;
    neum sr, si;
} dfs_ctx;

static void dfs(dfs_ctx* D, int e, const uint64_t st_in[2], cplx amp)
{
    const ocirc* C = D->C;
    uint64_t st[2] = {st_in[0], st_in[1]};
    for (; e < C->G; e++) {
        const ogate* g = &C->g[C->G - 1 - e];
        int srcs[2], ns = 0;
        if (g->role == ROLE_BR)
            for (int t = 0; t < g->k; t++)
                if (g->src[t] >= 0) srcs[ns++] = g->src[t];
        if (ns == 0) {
            int has_src;
            D->cnt->visits++;
            if (!step_gate(g, st, &amp, D->h, D->b_in, &has_src)) return;
            continue;
        }
        for (int v = 0; v < (1 << ns); v++) {
            for (int j = 0; j < ns; j++) D->h[srcs[j]] = (uint8_t)((v >> j) & 1);
            uint64_t s2[2] = {st[0], st[1]};
            cplx a2 = amp;
            int has_src;
            D->cnt->visits++;
            if (!step_gate(g, s2, &a2, D->h, D->b_in, &has_src)) continue;
            if (D->eps > 0.0 && below_eps(a2, D->eps)) continue;
            dfs(D, e + 1, s2, a2);
        }
        return;
    }
    D->cnt->completed++;
    if (st[0] == D->b_in[0] && st[1] == D->b_in[1]) {
        D->cnt->valid++;
        neum_add(&D->sr, amp.re);
        neum_add(&D->si, amp.im);
    }
}

static cplx pair_amplitude_dfs(const ocirc* C, const uint64_t b_in[2], const uint64_t b_out[2], double eps,
                               ocount* cnt)
{
    dfs_ctx D;
    D.C = C; D.b_in = b_in; D.eps = eps; D.cnt = cnt;
    D.h = (uint8_t*)calloc((size_t)C->A + 1, 1);
    D.sr.s = D.sr.c = D.si.s = D.si.c = 0.0;
    const uint64_t st[2] = {b_out[0], b_out[1]};
    dfs(&D, 0, st, cx(1, 0));
    free(D.h);
    return cx(D.sr.s + D.sr.c, D.si.s + D.si.c);
}

/* ---- exported API ------------------------------------------------------- */

static int make_circ(const orc_gate_in* gates, int G, int n, ocirc* C)
{
    if (n < 1 || n > 128 || G < 0) return -1;
    C->n = n; C->G = G;
    C->g = (ogate*)calloc((size_t)(G > 0 ? G : 1), sizeof(ogate));
    for (int i = 0; i < G; i++)
        if (build_gate(&gates[i], &C->g[i])) { free(C->g); return -2; }
    analyze(C);
    return 0;
}

/* Structure of the analysis: role per gate, per-target source id
 * (-1 natural, -2 not branching), and A. */
int orc_analyze(const orc_gate_in* gates, int G, int n, int32_t* role, int32_t* src, int32_t* A)
{
    ocirc C;
    int rc = make_circ(gates, G, n, &C);
    if (rc) return rc;
    for (int i = 0; i < G; i++) {
        role[i] = C.g[i].role;
        src[2 * i] = C.g[i].src[0];
        src[2 * i + 1] = C.g[i].k == 2 ? C.g[i].src[1] : -2;
    }
    *A = C.A;
    free(C.g);
    return 0;
}

/* Eq. 8: 2^Ap (Gp + 2^Ar (Gr + 2^As Gs)) for the cut (c1, c2), as a
 * 128-bit integer returned in two 64-bit halves. */
static unsigned __int128 gateops(int Gp, int Gr, int Gs, int Ap, int Ar, int As)
{
    unsigned __int128 one = 1;
    return (one << Ap) * ((unsigned __int128)Gp + (one << Ar) * ((unsigned __int128)Gr + (one << As) * (unsigned __int128)Gs));
}

int orc_region_counts(const orc_gate_in* gates, int G, int n, int c1, int c2, int32_t* out6, uint64_t* cost2)
{
    ocirc C;
    int rc = make_circ(gates, G, n, &C);
    if (rc) return rc;
    if (c1 < 0 || c2 < c1 || c2 > G) { free(C.g); return -1; }
    int Ap = sources_in(&C, 0, c1), Ar = sources_in(&C, c1, c2), As = sources_in(&C, c2, G);
    out6[0] = c1; out6[1] = c2 - c1; out6[2] = G - c2; out6[3] = Ap; out6[4] = Ar; out6[5] = As;
    unsigned __int128 v = gateops(c1, c2 - c1, G - c2, Ap, Ar, As);
    cost2[0] = (uint64_t)v; cost2[1] = (uint64_t)(v >> 64);
    free(C.g);
    return 0;
}

/* Autotuned partition (Sec. IV-C): the cut pair minimising Eq. 8
 * over every 0 <= c1 <= c2 <= G, subject to Ap <= max_ap and
 * min(min_apr, A) <= Ap + Ar <= max_apr.  Ties go to the smallest c1, then c2. */
int orc_autotune(const orc_gate_in* gates, int G, int n, int max_ap, int min_apr, int max_apr,
                 int32_t* c1_out, int32_t* c2_out, uint64_t* cost2)
{
    ocirc C;
    int rc = make_circ(gates, G, n, &C);
    if (rc) return rc;
    int* pre = (int*)calloc((size_t)G + 1, sizeof(int));  /* sources before position e */
    for (int e = 0; e < G; e++) pre[e + 1] = pre[e] + sources_in(&C, e, e + 1);
    int need = min_apr < C.A ? min_apr : C.A;
    int found = 0;
    unsigned __int128 best = 0;
    for (int c1 = 0; c1 <= G; c1++) {
        int Ap = pre[c1];
        if (Ap > max_ap) break;
        for (int c2 = c1; c2 <= G; c2++) {
            int Ar = pre[c2] - Ap, As = C.A - pre[c2];
            if (Ap + Ar < need) continue;
            if (Ap + Ar > max_apr) break;
            unsigned __int128 v = gateops(c1, c2 - c1, G - c2, Ap, Ar, As);
            if (!found || v < best) { best = v; *c1_out = c1; *c2_out = c2; found = 1; }
        }
    }
    free(pre);
    free(C.g);
    if (!found) return -3;
    cost2[0] = (uint64_t)best; cost2[1] = (uint64_t)(best >> 64);
    return 0;
}

typedef struct {
    const ocirc* C;
    const uint64_t* ins; const double* coef; int S;
    const uint64_t* outs; int M;
    double eps; int c1, c2;
    int dfs;          /* 1: per-source depth-first search instead of Algorithm 2 */
    double* amp; uint64_t* counts;
    int next;
    pthread_mutex_t mu;
} job_t;

static void* worker(void* arg)
{
    job_t* J = (job_t*)arg;
    for (;;) {
        pthread_mutex_lock(&J->mu);
        int o = J->next++;
        pthread_mutex_unlock(&J->mu);
        if (o >= J->M) break;
        neum ar = {0, 0}, ai = {0, 0};
        ocount tot = {0, 0, 0};
        for (int s = 0; s < J->S; s++) {
            ocount cnt = {0, 0, 0};
            cplx a = J->dfs ? pair_amplitude_dfs(J->C, &J->ins[2 * s], &J->outs[2 * o], J->eps, &cnt)
                            : pair_amplitude(J->C, &J->ins[2 * s], &J->outs[2 * o], J->eps, J->c1, J->c2, &cnt);
            cplx w = cmul(cx(J->coef[2 * s], J->coef[2 * s + 1]), a);
            neum_add(&ar, w.re);
            neum_add(&ai, w.im);
            tot.completed += cnt.completed; tot.valid += cnt.valid; tot.visits += cnt.visits;
        }
        J->amp[2 * o] = ar.s + ar.c;
        J->amp[2 * o + 1] = ai.s + ai.c;
        J->counts[3 * o + 0] = tot.completed;
        J->counts[3 * o + 1] = tot.valid;
        J->counts[3 * o + 2] = tot.visits;
    }
    return NULL;
}

/* The checkpoint table of one (input, output) pair after the prefix region
 * [0, c1) of Algorithm 2, exact mode: for every prefix assignment h_p
 * (artificial source j <-> bit j of h_p) the state sigma_p (2 words), the
 * partial amplitude beta_p, ok = 0 where an exactly zero factor was met
 * (bottom), and the exact subtree sum: the sum of the amplitudes of every
 * valid completion of h_p over the remaining sources (one region [c1, G)).
 * Arrays hold 2^Ap entries; Ap is returned in *Ap_out. */
int orc_checkpoints(const orc_gate_in* gates, int G, int n, const uint64_t* b_in, const uint64_t* b_out, int c1,
                    uint64_t* st, double* amp, uint8_t* ok, double* sub, int32_t* Ap_out)
{
    ocirc C;
    int rc = make_circ(gates, G, n, &C);
    if (rc) return rc;
    if (c1 < 0 || c1 > G || C.A > 40) { free(C.g); return -1; }
    const int Ap = sources_in(&C, 0, c1), Ar = sources_in(&C, c1, G);
    *Ap_out = Ap;
    uint8_t* h = (uint8_t*)calloc((size_t)C.A + 1, 1);
    uint64_t visits = 0;
    for (uint64_t hp = 0; hp < ((uint64_t)1 << Ap); hp++) {
        for (int j = 0; j < Ap; j++) h[j] = (uint8_t)((hp >> j) & 1);
        uint64_t sp[2] = {b_out[0], b_out[1]};
        cplx bp = cx(1, 0);
        const int live = advance(&C, 0, c1, sp, &bp, h, b_in, 0.0, &visits);
        st[2 * hp] = sp[0];
        st[2 * hp + 1] = sp[1];
        amp[2 * hp] = bp.re;
        amp[2 * hp + 1] = bp.im;
        ok[hp] = (uint8_t)live;
        neum sr = {0, 0}, si = {0, 0};
        if (live) {
            for (uint64_t hr = 0; hr < ((uint64_t)1 << Ar); hr++) {
                for (int j = 0; j < Ar; j++) h[Ap + j] = (uint8_t)((hr >> j) & 1);
                uint64_t ss[2] = {sp[0], sp[1]};
                cplx bs = bp;
                if (!advance(&C, c1, G, ss, &bs, h, b_in, 0.0, &visits)) continue;
                if (ss[0] == b_in[0] && ss[1] == b_in[1]) {
                    neum_add(&sr, bs.re);
                    neum_add(&si, bs.im);
                }
            }
        }
        sub[2 * hp] = sr.s + sr.c;
        sub[2 * hp + 1] = si.s + si.c;
    }
    free(h);
    free(C.g);
    return 0;
}

/* Amplitudes of M requested outputs for a sparse input of S basis states
 * (Eq. 2), with checkpoints (c1, c2) (c1 = c2 = 0: Algorithm 1; c1 = -1:
 * the per-source depth-first search), threshold
 * eps (0 = exact) on n_threads host threads.  counts: per output
 * {completed leaves, valid histories, gate visits}. */
int orc_run(const orc_gate_in* gates, int G, int n,
            const uint64_t* ins, const double* coef, int S,
            const uint64_t* outs, int M, double eps, int c1, int c2, int n_threads,
            double* amp, uint64_t* counts, int32_t* A_out)
{
    ocirc C;
    int rc = make_circ(gates, G, n, &C);
    if (rc) return rc;
    /* c1 = -1: the per-source depth-first search (any A); otherwise
     * Algorithm 2 with cuts (c1, c2), which enumerates 2^A per pair */
    const int use_dfs = c1 == -1;
    if (!use_dfs && (c1 < 0 || c2 < c1 || c2 > G || C.A > 62)) { free(C.g); return -1; }
    *A_out = C.A;
    job_t J;
    J.C = &C; J.ins = ins; J.coef = coef; J.S = S; J.outs = outs; J.M = M;
    J.eps = eps; J.c1 = c1; J.c2 = c2; J.dfs = use_dfs; J.amp = amp; J.counts = counts; J.next = 0;
    pthread_mutex_init(&J.mu, NULL);
    if (n_threads < 1) n_threads = 1;
    pthread_t* th = (pthread_t*)calloc((size_t)n_threads, sizeof(pthread_t));
    for (int t = 1; t < n_threads; t++) pthread_create(&th[t], NULL, worker, &J);
    worker(&J);
    for (int t = 1; t < n_threads; t++) pthread_join(th[t], NULL);
    free(th);
    pthread_mutex_destroy(&J.mu);
    free(C.g);
    return 0;
}

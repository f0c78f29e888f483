"""Learned pruning against threshold pruning at equal fidelity on QAOA-24
p = 3 (A = 72), the learned-pruning configuration of the QAOA MaxCut study
(Sec. V, Fig. 9; the pruner is not the paper's).

The network is trained on exact subtree sums logged from the 16-qubit p = 2
request of the threshold study (its checkpoint tables after 12 and 14
sources; exact enumeration is within reach there, A = 32).  On QAOA-24
p = 3 exact enumeration is not (2^72 histories per output), so the
evaluated runs are threshold runs: the threshold alone at several eps, and
the pruner at the checkpoint with the threshold in the suffix.  Fidelity is
judged against the dense state vector's amplitudes stored in
tests/golden/qaoa_threshold.json (written from oracle/ only).

Checked: with tau below every score the pruner cuts nothing and the
amplitudes are bitwise those of the threshold alone at the same eps and
cuts; at a tau that cuts, the leaves are a subset (fewer completed leaves)
and the fidelity is reported beside the threshold sweep's.  The printed
table (pytest -s) is the equal-fidelity comparison."""
import json
import os
import time

import numpy as np
import pytest
import torch

from workloads import mlp_init_params, qaoa_workload
from oracle import closed_forms
import paper_2608_01467_b300 as fs
from paper_2608_01467_b300 import learned

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "qaoa_threshold.json")
N_EVAL = 64                       # outputs of the QAOA-24 p = 3 request evaluated
EPS_SWEEP = (2e-4, 1e-4, 7e-5)    # threshold alone
EPS_LEARNED = 7e-5                # threshold in the suffix under the pruner
TAUS = (-1e30, -9.0, -8.0, -7.0, -6.0, -5.0, -4.0, -3.0)


def _cut_after_sources(circuit, k):
    """Evaluation position just after the op carrying artificial source
    k - 1 (the backward sweep's first k sources lie before it)."""
    bv = fs.Circuit(circuit).branch_vars()
    srcs = {s: g for g, q, s in bv if s >= 0}
    return 0 if k <= 0 else len(circuit.gates) - srcs[k - 1]


def _eval_request():
    with open(GOLD) as f:
        g = json.load(f)
    r = next(r for r in g["requests"] if r["n"] == 24 and r["p"] == 3)
    w = qaoa_workload(24, 3, n_out=r["n_out"], seed=r["seed"])
    assert [int(x) for x in w.outputs[:4]] == r["outputs_head"]
    exact = np.asarray(r["exact_re"]) + 1j * np.asarray(r["exact_im"])
    return w, exact


def _run(w, outs, eps, c1, c2, pruner=None, tau=0.0):
    C = fs.Circuit(w.circuit)
    C.set_input(w.inputs)
    b = fs.Batch(split="fixed", c1=c1, c2=c2)
    b.add(C, outs, eps)
    if pruner is not None:
        learned.attach(b, 0, pruner, tau)
    b.plan()
    b.allocate()
    b.upload()
    b.run()                       # first run: module load, caches
    b.finish()
    b.upload()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    b.run()
    st = b.finish()[0]
    dt = time.perf_counter() - t0
    return b.amp.cpu().numpy()[:len(outs)], st, dt


def _train():
    """MLP trained on exact log10 |subtree sum| of the 16-qubit p = 2
    request's checkpoint entries after 12 and after 14 sources (inside its
    last RX layer, as the evaluated checkpoint is)."""
    tr = qaoa_workload(16, 2, n_out=1024)
    xs, ts = [], []
    for k in (12, 14):
        cut = _cut_after_sources(tr.circuit, k)
        x, t, st = learned.log_training_data(tr.circuit, tr.inputs, tr.outputs[:32], cut)
        assert st["A_p"] == k and st["valid"] > 0
        xs.append(x)
        ts.append(t)
    x = torch.cat(xs).contiguous()
    t = torch.cat(ts).contiguous()
    params, losses = learned.train(x, t, mlp_init_params(4), steps=1500, batch=16384, lr=1e-3)
    assert losses[-1] < losses[0]
    return params, losses


def test_learned_vs_threshold_at_equal_fidelity_on_qaoa24_p3():
    w, exact_all = _eval_request()
    assert fs.Circuit(w.circuit).analyze(0)["A"] == 72
    outs = w.outputs[:N_EVAL]
    exact = exact_all[:N_EVAL]
    # checkpoint after 12 sources (4096 entries per output), 4 in the root
    c1 = _cut_after_sources(w.circuit, 12)
    c2 = _cut_after_sources(w.circuit, 16)
    params, losses = _train()
    rows = []
    thr = {}
    for eps in EPS_SWEEP:
        amp, st, dt = _run(w, outs, eps, c1, c2)
        assert (st["A_p"], st["A_r"]) == (12, 4)
        F = closed_forms.fidelity(exact, amp)
        thr[eps] = (amp, st)
        rows.append(("threshold", eps, None, F, st["completed"], st["live_entries"], 0, dt))
    base_amp, base_st = thr[EPS_LEARNED]
    cut_any = False
    for tau in TAUS:
        amp, st, dt = _run(w, outs, EPS_LEARNED, c1, c2, params, tau)
        F = closed_forms.fidelity(exact, amp)
        rows.append(("learned", EPS_LEARNED, tau, F, st["completed"], st["live_entries"], st["learned_cuts"], dt))
        if tau == -1e30:
            # cuts nothing: the threshold alone's amplitudes, bit for bit
            assert st["learned_cuts"] == 0
            assert st["completed"] == base_st["completed"] and st["valid"] == base_st["valid"]
            assert np.array_equal(amp, base_amp)
        else:
            # a learned cut removes whole subtrees: never more leaves
            assert st["completed"] <= base_st["completed"]
            cut_any = cut_any or st["learned_cuts"] > 0
    assert cut_any
    print("\nQAOA-24 p=3, %d outputs, (A_p, A_r) = (12, 4); training loss %.3f -> %.3f" %
          (N_EVAL, losses[0], losses[-1]))
    print("%-9s %7s %6s %9s %13s %9s %9s %8s" % ("mode", "eps", "tau", "fidelity", "leaves", "live", "l-cuts",
                                                "s"))
    for mode, eps, tau, F, comp, live, cuts, dt in rows:
        print("%-9s %7.0e %6s %9.5f %13d %9d %9d %8.3f" %
              (mode, eps, "-" if tau is None else ("-inf" if tau < -1e29 else "%g" % tau), F, comp, live, cuts, dt))
    # equal fidelity: for each learned row, the cheapest threshold row that
    # reaches at least its fidelity
    for mode, eps, tau, F, comp, live, cuts, dt in rows:
        if mode != "learned" or tau < -1e29:
            continue
        best = [r for r in rows if r[0] == "threshold" and r[3] >= F]
        if best:
            b = min(best, key=lambda r: r[7])
            print("tau %g: fidelity %.5f in %.3f s; threshold eps %g reaches %.5f in %.3f s (%.2fx)" %
                  (tau, F, dt, b[1], b[3], b[7], b[7] / dt))
        else:
            print("tau %g: fidelity %.5f in %.3f s; no threshold of the sweep reaches it" % (tau, F, dt))

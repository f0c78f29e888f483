"""Writes qaoa_threshold.json: stored oracle values for the QAOA MaxCut
requests of the threshold-pruning and learned-pruning parity tests.

Run from the repository root (takes several minutes on 8 host threads):

    python tests/golden/make_qaoa_golden.py

Everything here comes from `oracle/` (test infrastructure) and the seeded
input generators in `workloads/`; nothing from the CUDA library.

* exact: the dense state vector (oracle.dense) amplitudes of all requested
  outputs of each request -- the exact reference for fidelity;
* samples: for a few outputs of each (request, eps), the threshold-pruned
  amplitude and the completed / valid leaf counts of the per-source
  depth-first search (oracle.feynman.run_dfs, Sec. IV-A Observation 3);
* closed_form_leaves: for QAOA every RZZ factor has modulus 1 and the RX
  factors have modulus |cos(beta/2)| or |sin(beta/2)| whatever the state,
  so a history survives a threshold eps iff the product of its RX moduli is
  at least eps (the running product only decreases); the surviving leaf
  count per (output, input) pair is then a sum of binomial coefficients over
  the number of sine choices per layer.  Stored with the smallest relative
  distance of any such product to eps (ties would make the count depend on
  rounding).
"""
from __future__ import annotations

import json
import math
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from workloads.circuits import SEED_BASE, qaoa_workload  # noqa: E402
from oracle import dense, feynman  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "qaoa_threshold.json")

# (n, p, seed): configs 3 (p = 2) and 4 (p = 3), 1024 outputs each.  The
# thresholds keep the pruned search within reach: at QAOA-24 p = 3 (A = 72)
# eps = 1e-6 would leave about 1e11 leaves and 3e12 visited branches per
# output (closed form), eps = 1e-4 leaves 2e5 leaves and 1.6e8 branches.
REQUESTS = [
    (16, 2, SEED_BASE + 3), (20, 2, SEED_BASE + 3), (24, 2, SEED_BASE + 3), (24, 3, SEED_BASE + 4)]
SAMPLES = [  # (n, p, eps, sample output indices)
    (16, 2, 1e-4, [0, 1, 2, 3, 400, 511, 777, 1023]),
    (16, 2, 1e-6, [0, 1, 511, 1023]),
    (20, 2, 1e-4, [0, 1, 2, 3, 400, 511, 777, 1023]),
    (20, 2, 1e-6, [0, 1, 511, 1023]),
    (24, 2, 1e-4, [0, 1, 511, 1023]),
    (24, 3, 1e-4, [0, 1, 511, 1023]),
]


def closed_form(n, angles, eps):
    """Surviving leaves per pair and the smallest |log(product / eps)|."""
    per_layer = []
    for _, beta in angles:
        c, s = abs(math.cos(beta / 2)), abs(math.sin(beta / 2))
        per_layer.append([((n - k) * math.log(c) + k * math.log(s), math.comb(n, k)) for k in range(n + 1)])
    total = 0
    margin = float("inf")
    states = [(0.0, 1)]
    for layer in per_layer:
        states = [(a + b, x * y) for a, x in states for b, y in layer]
    for lg, cnt in states:
        margin = min(margin, abs(lg - math.log(eps)))
        if lg >= math.log(eps):
            total += cnt
    return total, margin


def main():
    threads = os.cpu_count() or 1
    data = {"citation": "Sec. IV-A Observation 3 (threshold pruning); Sec. V QAOA MaxCut case study (Fig. 9); "
                        "values from oracle.dense and oracle.feynman.run_dfs",
            "requests": [], "samples": []}
    for n, p, seed in REQUESTS:
        t0 = time.time()
        w = qaoa_workload(n, p, n_out=1024, seed=seed)
        amp = dense.amplitudes(w.circuit, w.inputs, w.outputs)
        data["requests"].append({"n": n, "p": p, "seed": seed, "n_out": len(w.outputs),
                                 "outputs_head": [int(x) for x in w.outputs[:4]],
                                 "exact_re": [float(z.real) for z in amp],
                                 "exact_im": [float(z.imag) for z in amp]})
        print(f"dense n={n} p={p}: {time.time() - t0:.1f} s", flush=True)
    for n, p, eps, idx in SAMPLES:
        t0 = time.time()
        seed = SEED_BASE + (3 if p == 2 else 4)
        w = qaoa_workload(n, p, n_out=1024, seed=seed)
        outs = [w.outputs[i] for i in idx]
        amp, cnt = feynman.run_dfs(w.circuit, w.inputs, outs, eps=eps, threads=threads)
        leaves, margin = closed_form(n, w.meta["angles"], eps)
        data["samples"].append({"n": n, "p": p, "seed": seed, "eps": eps, "index": idx,
                                "re": [float(z.real) for z in amp], "im": [float(z.imag) for z in amp],
                                "completed": [int(x) for x in cnt["completed"]],
                                "valid": [int(x) for x in cnt["valid"]],
                                "closed_form_leaves": leaves, "closed_form_margin": margin})
        print(f"dfs n={n} p={p} eps={eps}: {time.time() - t0:.1f} s, leaves {leaves}", flush=True)
    with open(OUT, "w") as f:
        json.dump(data, f)
    print("wrote", OUT)


if __name__ == "__main__":
    main()

"""Threshold pruning (Sec. IV-A, Observation 3) at the sizes of the QAOA
MaxCut requests: three seeded 3-regular graphs at 16, 20 and 24 qubits,
p = 2, 1024 requested outputs each, eps in {1e-4, 1e-6}, and QAOA-24 at
p = 3 (A = 72) at eps = 1e-4 (at 1e-6 its pruned search would keep about
1e11 leaves per output).

The stored values (tests/golden/qaoa_threshold.json, written by
tests/golden/make_qaoa_golden.py from oracle/ only) are the dense state
vector's exact amplitudes of every requested output and, for sampled
outputs, the oracle's per-source depth-first search with the same
threshold: pruned amplitudes and completed / valid leaf counts.  Each test
runs the request on the GPU (1024 outputs; large compacted checkpoint tables,
the block-per-output reduction), compares the sampled amplitudes
with the oracle's element by element, checks the job's leaf count against
the closed form, runs the sampled outputs alone with the same cuts for
bit-exact per-output counts, and reports the fidelity against the exact
amplitudes."""
import json
import os

import numpy as np
import pytest

from workloads import qaoa_workload
from oracle import closed_forms
import paper_2608_01467_b300 as fs

pytestmark = pytest.mark.gpu

ATOL, RTOL = 1e-12, 1e-10
GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "qaoa_threshold.json")


def _gold():
    with open(GOLD) as f:
        return json.load(f)


def _request(g, n, p):
    r = next(r for r in g["requests"] if r["n"] == n and r["p"] == p)
    w = qaoa_workload(n, p, n_out=r["n_out"], seed=r["seed"])
    assert [int(x) for x in w.outputs[:4]] == r["outputs_head"]
    exact = np.asarray(r["exact_re"]) + 1j * np.asarray(r["exact_im"])
    return w, exact


def _subset(n_all, sample_idx, size):
    """Output indices of a reduced request: the sampled ones plus the lowest
    others, `size` in all (every index when size >= n_all)."""
    if size >= n_all:
        return list(range(n_all))
    chosen = set(sample_idx)
    i = 0
    while len(chosen) < size:
        chosen.add(i)
        i += 1
    return sorted(chosen)


def _run(w, outputs, eps, cuts=None):
    C = fs.Circuit(w.circuit)
    C.set_input(w.inputs)
    b = fs.Batch()
    b.add(C, outputs, eps)
    if cuts is not None:
        b.set_cuts(0, *cuts)
    b.plan()
    b.allocate()
    b.upload()
    b.run()
    st = b.finish()[0]
    return b.amp.cpu().numpy()[:len(outputs)], st


# (n, p, eps, requested outputs): the full 1024-output requests (the whole
# set takes about two minutes on the level walk; FS_SHORT_TESTS=1 runs the
# two longest as reduced requests: the sampled outputs plus the lowest
# others)
SHORT = os.environ.get("FS_SHORT_TESTS") == "1"
CASES = [(16, 2, 1e-4, 1024), (16, 2, 1e-6, 1024), (20, 2, 1e-4, 1024),
         (20, 2, 1e-6, 64 if SHORT else 1024), (24, 2, 1e-4, 1024),
         (24, 3, 1e-4, 128 if SHORT else 1024)]


@pytest.mark.parametrize("n,p,eps,size", CASES)
def test_qaoa_threshold_request_matches_the_oracle(n, p, eps, size):
    g = _gold()
    w, exact = _request(g, n, p)
    smp = next(s for s in g["samples"] if s["n"] == n and s["p"] == p and s["eps"] == eps)
    A = fs.Circuit(w.circuit).analyze(0)["A"]
    assert A == n * p                                        # Table 1: QAOA A = sn
    sel = _subset(len(w.outputs), smp["index"], size)
    outs = [w.outputs[i] for i in sel]
    exact = exact[sel]
    amp, st = _run(w, outs, eps)
    idx = [sel.index(i) for i in smp["index"]]
    want = np.asarray(smp["re"]) + 1j * np.asarray(smp["im"])
    err = np.abs(amp[idx] - want)
    assert np.all(err <= ATOL + RTOL * np.abs(want)), err.max()
    # every pair of this request keeps the same leaves (the RX moduli do not
    # depend on the state): the closed-form count, and chi = 1 for all of them
    assert smp["closed_form_margin"] > 1e-9
    assert smp["completed"] == [smp["closed_form_leaves"]] * len(idx)
    assert st["completed"] == len(outs) * smp["closed_form_leaves"]
    assert st["valid"] == st["completed"]
    lp = (len(outs) - 1).bit_length()          # ceil(log2(pairs))
    assert st["candidates"] == (len(outs) << A if A + lp < 64 else (1 << 64) - 1)
    # the sampled outputs alone with the same cuts: per-output counts equal
    # to the oracle's, amplitudes bit-identical to the full request's
    amp2, st2 = _run(w, [outs[i] for i in idx], eps, (st["c1"], st["c2"]))
    assert st2["completed"] == sum(smp["completed"]) and st2["valid"] == sum(smp["valid"])
    assert np.array_equal(amp2, amp[idx])
    F = closed_forms.fidelity(exact, amp)
    weight = float(np.vdot(amp, amp).real / np.vdot(exact, exact).real)
    print(f"QAOA-{n} p={p} eps={eps:g} ({len(outs)} outputs): A={A} "
          f"(A_p, A_r, A_s)=({st['A_p']}, {st['A_r']}, {st['A_s']}) "
          f"live entries {st['live_entries']} leaves {st['completed']} fidelity {F:.6f} weight {weight:.6f}")
    assert 0.0 <= F <= 1.0 + 1e-12


def test_threshold_request_exercises_large_tables_and_the_block_reduction():
    """QAOA-16, eps = 1e-4: the compacted checkpoint table has far more
    entries than one compaction block and the scan's block count exceeds one
    pass of its 1024 threads; every output has more than 4096 live entries,
    so the block-per-output reduction sums them."""
    g = _gold()
    w, exact = _request(g, 16, 2)
    amp, st = _run(w, w.outputs, 1e-4)
    entries = len(w.outputs) << st["A_p"]
    assert entries // 1024 > 1024                  # compaction blocks > scan threads
    assert st["A_r"] <= 5 and st["live_entries"] // len(w.outputs) > 4096


def _cut_after_sources(circuit, k):
    """Evaluation position just after the op carrying artificial source
    k - 1 (the first k sources of the backward sweep lie before it)."""
    bv = fs.Circuit(circuit).branch_vars()
    srcs = {s: g for g, q, s in bv if s >= 0}
    return 0 if k <= 0 else len(circuit.gates) - srcs[k - 1]


@pytest.mark.parametrize("ap,ar", [(4, 2), (3, 6)])
@pytest.mark.parametrize("eps", [1e-3, 3e-4])
def test_level_walk_of_the_suffix_matches_the_oracle(ap, ar, eps):
    """Threshold jobs with five or more sources in the suffix walk it level
    by level, a warp per live checkpoint entry, with per-level queues of
    partial histories in shared memory.  With A_r = 2 the entry's roots fill
    part of one warp and its sum lands in the first of its subtree slots;
    with A_r = 6 the roots come in two chunks of 32 with one sum each.
    Amplitudes within 1e-12 / 1e-10 of the oracle at the same cuts, leaf
    counts exactly the oracle's, and fewer gate visits than Algorithm 2's
    (no cut subtree is entered)."""
    from oracle import feynman
    w = qaoa_workload(10, 2, n_out=24, seed=9)
    c1 = _cut_after_sources(w.circuit, ap)
    c2 = _cut_after_sources(w.circuit, ap + ar)
    C = fs.Circuit(w.circuit)
    C.set_input(w.inputs)
    b = fs.Batch(split="fixed", c1=c1, c2=c2)
    b.add(C, w.outputs, eps)
    b.plan()
    assert "QUEUE = true" in b.generated_source()
    b.allocate()
    b.upload()
    b.run()
    st = b.finish()[0]
    assert (st["A_p"], st["A_r"], st["A_s"]) == (ap, ar, 20 - ap - ar)
    amp = b.amp.cpu().numpy()[:len(w.outputs)]
    want, cnt = feynman.run(w.circuit, w.inputs, w.outputs, eps=eps, c1=c1, c2=c2)
    err = np.abs(amp - want)
    assert np.all(err <= ATOL + RTOL * np.abs(want)), err.max()
    assert st["completed"] == int(cnt["completed"].sum()) and st["valid"] == int(cnt["valid"].sum())
    assert st["gate_visits"] < int(cnt["visits"].sum())
    assert np.abs(want).max() > 1e-3

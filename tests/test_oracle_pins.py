"""Pins of the oracle against things other than itself: the paper's worked
examples and Table 1, closed forms, unitarity, literal brute force and
independent tiers.  CPU only."""
import json
import math
import os

import numpy as np
import pytest

from workloads import (Circuit, Gate, SplitMix64, aa_workload, amplitude_amplification,
                       four_qubit_figure, qaoa_maxcut, qaoa_workload, qft, quantum_walk,
                       qw_workload, random_small_circuit, three_qubit_example)
from oracle import bruteforce, closed_forms, dense, feynman

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def gold(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


# ---------------------------------------------------------------- paper pins

def test_three_qubit_example_all_tiers():
    g = gold("three_qubit_example.json")
    c = three_qubit_example()
    expect = np.zeros(8, complex)
    for k, (re, im) in g["amplitudes"].items():
        expect[int(k)] = complex(re, im)
    o3, cnt = feynman.run(c, [(g["input"], 1.0)], range(8))
    o2 = dense.amplitudes(c, [(g["input"], 1.0)], range(8))
    o1 = [bruteforce.wire_sum(c, 0, b) for b in range(8)]
    o0 = [bruteforce.history_sum(c, 0, b) for b in range(8)]
    for got in (o3, o2, o1, o0):
        assert np.max(np.abs(np.asarray(got) - expect)) < 1e-15
    assert int(cnt["valid"].sum()) == g["contributing_histories_total"]


def test_fig2_structure_and_gateops():
    g = gold("fig2_four_qubit.json")
    c = four_qubit_figure()
    an = feynman.analyze(c)
    assert an["roles"] == g["roles"]
    assert an["A"] == g["A"]
    for gi, k in g["sources_by_gate"].items():
        assert an["src"][int(gi)][0] == k
    for gi in g["natural_gates"]:
        assert an["src"][gi][0] == -1
    s = g["split_from_figure"]
    rc, cost = feynman.region_counts(c, s["c1"], s["c2"])
    assert list(rc[:3]) == s["G"] and list(rc[3:]) == s["A"]
    assert cost == g["gateops_checkpointed"]
    Gp, Gr, Gs = s["G"]
    assert cost == 2 * (Gp + 2 * (Gr + Gs))
    _, flat = feynman.region_counts(c, 0, 0)
    assert flat == g["gateops_flat"] == 4 * (Gp + Gr + Gs)


def _table1_circuit(row):
    fam, n, s = row["family"], row["n"], row["s"]
    if fam == "qft":
        return qft(n)
    if fam == "aa":
        return amplitude_amplification(n, s, marked=0b1011 % (1 << n))
    if fam == "qaoa":
        return qaoa_maxcut(n, s, SplitMix64(7 + n))[0]
    if fam == "qw":
        return quantum_walk(s, pos_bits=n - 4)
    raise ValueError(fam)


def test_table1_backward_source_counts():
    for row in gold("table1_sources.json")["rows"]:
        c = _table1_circuit(row)
        assert feynman.analyze(c)["A"] == row["A"], row


# ---------------------------------------------------------------- closed forms

def test_qft_dense_matches_closed_form():
    for n in (3, 5, 8):
        c = qft(n)
        for x in (0, 1, (1 << n) - 1, (0x5A % (1 << n))):
            got = dense.amplitudes(c, [(x, 1.0)], range(1 << n))
            want = np.array([closed_forms.qft_amplitude(n, x, y) for y in range(1 << n)])
            assert np.max(np.abs(got - want)) < 1e-13


def test_qft_reduced_history_matches_closed_form():
    n = 8
    c = qft(n)
    x = 0xB7
    got, cnt = feynman.run(c, [(x, 1.0)], range(1 << n))
    want = np.array([closed_forms.qft_amplitude(n, x, y) for y in range(1 << n)])
    assert np.max(np.abs(got - want)) < 1e-13
    # A = 0: one candidate and one valid history per pair (Sec. V, QFT)
    assert cnt["A"] == 0
    assert np.all(cnt["completed"] == 1) and np.all(cnt["valid"] == 1)


def test_walk_offsets_is_unitary_and_matches_dense():
    a = closed_forms.walk_offsets(10, math.sqrt(0.5), 1j * math.sqrt(0.5))
    assert abs(np.sum(np.abs(a) ** 2) - 1) < 1e-14
    # small walk circuit (4 position qubits) through the dense tier
    steps, pb = 3, 4
    c = quantum_walk(steps, pos_bits=pb)
    p0 = 7
    s = math.sqrt(0.5)
    ins = [((p0 << 1) | 0, s), ((p0 << 1) | 1, 1j * s)]
    sv = dense.statevector(c, ins)
    for y in range(1 << (pb + 1)):
        want = closed_forms.walk_amplitude(steps, p0, y, s, 1j * s, pb)
        assert abs(sv[y] - want) < 1e-14


def test_qw_reduced_history_matches_offset_walk_and_norm():
    w = qw_workload(steps=6, n_out=64, pos_bits=8)
    c = w.circuit
    s = math.sqrt(0.5)
    got, cnt = feynman.run(c, w.inputs, w.outputs)
    p0 = w.meta["p0"]
    want = np.array([closed_forms.walk_amplitude(6, p0, y, s, 1j * s, 8) for y in w.outputs])
    assert np.max(np.abs(got - want)) < 1e-14
    reach = w.meta["reachable"]
    assert abs(np.sum(np.abs(got[:reach]) ** 2) - 1.0) < 1e-13     # norm over reachable outputs
    assert np.all(got[reach:] == 0)                                 # unreachable: exactly zero
    assert np.all(cnt["valid"][reach:] == 0)
    assert cnt["A"] == 5


# ---------------------------------------------------------------- unitarity / invariants

def test_dense_unitarity_random_circuits():
    for seed in range(6):
        c = random_small_circuit(3, 10, seed)
        U = dense.unitary(c)
        assert np.max(np.abs(U.conj().T @ U - np.eye(8))) < 1e-13


# ---------------------------------------------------------------- tier cross-checks

@pytest.mark.parametrize("seed", range(10))
def test_random_tiny_circuits_all_tiers_agree(seed):
    rng = SplitMix64(1000 + seed)
    n = 3
    c = random_small_circuit(n, 7, 1000 + seed)
    b_in = rng.below(1 << n)
    outs = list(range(1 << n))
    o2 = dense.amplitudes(c, [(b_in, 1.0)], outs)
    o3, cnt = feynman.run(c, [(b_in, 1.0)], outs)
    assert np.max(np.abs(o3 - o2)) < 1e-13
    if bruteforce.count_internal_wires(c) <= 18:
        o1 = np.array([bruteforce.wire_sum(c, b_in, o) for o in outs])
        assert np.max(np.abs(o1 - o2)) < 1e-13
    assert abs(np.sum(np.abs(o3) ** 2) - 1) < 1e-12
    assert np.all(cnt["completed"] <= (1 << cnt["A"]))


def test_history_sum_literal_eq5_small():
    c = random_small_circuit(2, 4, 77)
    for b_in in range(4):
        o2 = dense.amplitudes(c, [(b_in, 1.0)], range(4))
        o0 = np.array([bruteforce.history_sum(c, b_in, b) for b in range(4)])
        assert np.max(np.abs(o0 - o2)) < 1e-14


@pytest.mark.parametrize("seed", range(6))
def test_random_medium_circuits_o3_vs_dense(seed):
    n = 6
    c = random_small_circuit(n, 24, 2000 + seed)
    rng = SplitMix64(3000 + seed)
    ins = [(rng.below(1 << n), complex(0.6, 0.0)), (rng.below(1 << n), complex(0.0, 0.8))]
    if ins[0][0] == ins[1][0]:
        ins = ins[:1]
        ins[0] = (ins[0][0], 1.0)
    outs = list(range(1 << n))
    o2 = dense.amplitudes(c, ins, outs)
    an = feynman.analyze(c)
    if an["A"] > 18:
        pytest.skip("too many sources for the slow path")
    o3, _ = feynman.run(c, ins, outs)
    assert np.max(np.abs(o3 - o2)) < 1e-12


def test_sparse_input_is_linear():
    c = random_small_circuit(4, 12, 555)
    outs = list(range(16))
    a1, _ = feynman.run(c, [(3, 1.0)], outs)
    a2, _ = feynman.run(c, [(9, 1.0)], outs)
    ab, _ = feynman.run(c, [(3, 0.6), (9, 0.8j)], outs)
    assert np.max(np.abs(ab - (0.6 * a1 + 0.8j * a2))) < 1e-14


def test_aa_small_vs_dense():
    w = aa_workload(n=4, iters=2, n_out=10, seed=11)
    o2 = dense.amplitudes(w.circuit, w.inputs, w.outputs)
    o3, cnt = feynman.run(w.circuit, w.inputs, w.outputs)
    assert np.max(np.abs(o3 - o2)) < 1e-13
    assert cnt["A"] == 16
    # every AA history is valid: ancillas restore, the natural H layer resets data to |0>
    assert np.all(cnt["valid"] == (1 << 16))


def test_aa_fig8_circuit_checkpointed_vs_dense():
    """Fig. 8 ablation circuit (4 qubits, 3 iterations, |0> in, lowest outputs)
    through Algorithm 2 with the autotuned cut."""
    w = aa_workload(n=4, iters=3, n_out=16, seed=11, all_outputs=True)
    outs = w.outputs[:3]
    c1, c2, cost = feynman.autotune(w.circuit)
    o2 = dense.amplitudes(w.circuit, w.inputs, outs)
    o3, cnt = feynman.run(w.circuit, w.inputs, outs, c1=c1, c2=c2)
    assert np.max(np.abs(o3 - o2)) < 1e-13
    assert np.all(cnt["visits"] == cost)


def test_qaoa_small_vs_dense():
    w = qaoa_workload(8, 2, n_out=32, seed=99)
    o2 = dense.amplitudes(w.circuit, w.inputs, w.outputs)
    o3, cnt = feynman.run(w.circuit, w.inputs, w.outputs)
    assert cnt["A"] == 16
    assert np.max(np.abs(o3 - o2)) < 1e-13


# ---------------------------------------------------------------- Algorithm 2 vs 1, Eq. 8

def test_checkpointed_equals_flat_and_visits_equal_eq8():
    c = qaoa_workload(6, 2, n_out=8, seed=5)
    G = len(c.circuit.gates)
    a_flat, cnt_flat = feynman.run(c.circuit, c.inputs, c.outputs)
    rng = SplitMix64(42)
    for _ in range(12):
        c1 = rng.below(G + 1)
        c2 = c1 + rng.below(G - c1 + 1)
        a, cnt = feynman.run(c.circuit, c.inputs, c.outputs, c1=c1, c2=c2)
        assert np.max(np.abs(a - a_flat)) < 1e-14
        assert np.array_equal(cnt["completed"], cnt_flat["completed"])
        assert np.array_equal(cnt["valid"], cnt_flat["valid"])
        (Gp, Gr, Gs, Ap, Ar, As), cost = feynman.region_counts(c.circuit, c1, c2)
        assert Gp + Gr + Gs == G and Ap + Ar + As == cnt["A"]
        assert cost == (1 << Ap) * (Gp + (1 << Ar) * (Gr + (1 << As) * Gs))
        # exact mode, no zero factors: counted gate visits equal Eq. 8
        assert np.all(cnt["visits"] == cost)


def test_autotune_is_argmin_of_eq8():
    for c in (four_qubit_figure(), qaoa_workload(6, 2, 4, seed=3).circuit,
              aa_workload(4, 2, 4, seed=2).circuit, random_small_circuit(4, 14, 9)):
        G = len(c.gates)
        best = None
        for c1 in range(G + 1):
            for c2 in range(c1, G + 1):
                _, cost = feynman.region_counts(c, c1, c2)
                if best is None or cost < best[0]:
                    best = (cost, c1, c2)
        t1, t2, tc = feynman.autotune(c)
        assert (tc, t1, t2) == best


# ---------------------------------------------------------------- threshold pruning

def _python_pruned_sum(c, b_in, b_out, eps):
    """Independent restatement for a tiny circuit: enumerate all source
    assignments, walk gates backward with numpy matrices, drop the history
    once |beta| < eps right after an artificial-source factor."""
    from oracle.gates import base_matrix
    an = feynman.analyze(c)
    A = an["A"]
    total = 0j
    kept = 0
    for h in range(1 << A):
        st = b_out
        amp = 1 + 0j
        ok = True
        for gi in range(len(c.gates) - 1, -1, -1):
            g = c.gates[gi]
            B = base_matrix(g)
            tq = list(g.qubits)
            on = all(((st >> q) & 1) == v for q, v in g.controls)
            out = sum(((st >> q) & 1) << j for j, q in enumerate(tq))
            role = an["roles"][gi]
            has_src = False
            if role == "WP":
                f = B[out, out] if on else 1
                inv = out
            elif role == "DET":
                if on:
                    inv = int(np.nonzero(B[out])[0][0])
                    f = B[out, inv]
                else:
                    inv, f = out, 1
            else:
                inv = 0
                for j, q in enumerate(tq):
                    sid = an["src"][gi][j]
                    bit = ((b_in >> q) & 1) if sid < 0 else ((h >> sid) & 1)
                    has_src |= sid >= 0
                    inv |= bit << j
                f = B[out, inv]
            if f == 0:
                ok = False
                break
            amp *= f
            for j, q in enumerate(tq):
                st = (st & ~(1 << q)) | (((inv >> j) & 1) << q)
            if eps > 0 and has_src and abs(amp) < eps:
                ok = False
                break
        if ok:
            kept += 1
            if st == b_in:
                total += amp
    return total, kept


def test_threshold_pruning_matches_independent_enumeration():
    w = qaoa_workload(4, 2, n_out=6, seed=21)
    c = w.circuit
    # choose eps values away from every partial magnitude so rounding cannot decide
    for eps in (1e-300, 0.05, 0.2, 0.5, 10.0):
        got, cnt = feynman.run(c, w.inputs, w.outputs, eps=eps)
        for i, o in enumerate(w.outputs):
            want, kept = _python_pruned_sum(c, 0, o, eps)
            assert abs(got[i] - want) < 1e-14, (eps, o)
            assert int(cnt["completed"][i]) == kept
    # eps above every magnitude: nothing survives
    got, cnt = feynman.run(c, w.inputs, w.outputs, eps=10.0)
    assert np.all(got == 0) and np.all(cnt["completed"] == 0)


def test_pruning_same_under_checkpoints():
    w = qaoa_workload(6, 2, n_out=8, seed=8)
    G = len(w.circuit.gates)
    a0, c0 = feynman.run(w.circuit, w.inputs, w.outputs, eps=0.03)
    a1, c1 = feynman.run(w.circuit, w.inputs, w.outputs, eps=0.03, c1=G // 3, c2=2 * G // 3)
    assert np.max(np.abs(a0 - a1)) < 1e-14
    assert np.array_equal(c0["completed"], c1["completed"])


def test_fidelity_definition():
    a = np.array([1, 1j, 0])
    assert closed_forms.fidelity(a, a) == pytest.approx(1.0)
    assert closed_forms.fidelity(a, 2 * a) == pytest.approx(1.0)
    assert closed_forms.fidelity(a, np.array([1, 0, 0])) == pytest.approx(0.5)
    assert closed_forms.captured_weight(a, np.array([1, 0, 0])) == pytest.approx(0.5)


def test_multithreaded_oracle_is_deterministic():
    w = qaoa_workload(8, 2, n_out=64, seed=13)
    a1, c1 = feynman.run(w.circuit, w.inputs, w.outputs, threads=1)
    a4, c4 = feynman.run(w.circuit, w.inputs, w.outputs, threads=4)
    assert np.array_equal(a1, a4) and np.array_equal(c1["valid"], c4["valid"])


# ------------------------------------------------ per-source depth-first search

@pytest.mark.parametrize("seed", [3, 17, 29])
def test_depth_first_search_equals_algorithms_1_and_2(seed):
    """The per-source search visits the same leaves as Algorithm 1 (and as
    Algorithm 2 at any cuts) and sums the same histories: equal amplitudes,
    equal completed and valid counts, exact and thresholded; its gate visits
    are Eq. 8 generalised to one region per source, never more than
    Algorithm 2's."""
    c = random_small_circuit(8, 45, 900 + seed)
    rng = SplitMix64(seed)
    inputs = [(rng.bits(8), 0.6), (rng.bits(8), 0.8j)]
    outputs = [rng.bits(8) for _ in range(6)]
    G = len(c.gates)
    for eps in (0.0, 0.05, 0.2):
        a1, k1 = feynman.run(c, inputs, outputs, eps=eps)
        a2, k2 = feynman.run(c, inputs, outputs, eps=eps, c1=G // 3, c2=2 * G // 3)
        ad, kd = feynman.run_dfs(c, inputs, outputs, eps=eps)
        assert np.max(np.abs(ad - a1)) < 1e-14 and np.max(np.abs(ad - a2)) < 1e-14
        for k in (k1, k2):
            assert np.array_equal(kd["completed"], k["completed"])
            assert np.array_equal(kd["valid"], k["valid"])
        assert np.all(kd["visits"] <= k2["visits"])


def _qaoa_closed_form_leaves(n, angles, eps):
    """Leaves of one (output, input) pair of QAOA MaxCut that survive the
    threshold eps: RZZ factors have modulus 1 and RX factors modulus
    |cos(beta/2)| (input = output value) or |sin(beta/2)| whatever the state,
    and every factor has modulus <= 1, so a history survives iff the product
    of its RX moduli is >= eps; with k_l sine choices in layer l there are
    prod_l C(n, k_l) such histories.  Also returns the smallest distance of a
    log-product to log(eps)."""
    layers = []
    for _, beta in angles:
        c, s = abs(math.cos(beta / 2)), abs(math.sin(beta / 2))
        layers.append([((n - k) * math.log(c) + k * math.log(s), math.comb(n, k)) for k in range(n + 1)])
    states = [(0.0, 1)]
    for layer in layers:
        states = [(a + b, x * y) for a, x in states for b, y in layer]
    return (sum(cnt for lg, cnt in states if lg >= math.log(eps)),
            min(abs(lg - math.log(eps)) for lg, _ in states))


@pytest.mark.parametrize("n,p,eps", [(8, 2, 1e-2), (10, 2, 1e-3), (10, 3, 1e-3), (12, 2, 1e-4)])
def test_threshold_leaf_count_matches_the_qaoa_closed_form(n, p, eps):
    w = qaoa_workload(n, p, n_out=4, seed=77 + n)
    want, margin = _qaoa_closed_form_leaves(n, w.meta["angles"], eps)
    assert margin > 1e-9          # no product within rounding of eps
    a, cnt = feynman.run_dfs(w.circuit, w.inputs, w.outputs, eps=eps, threads=4)
    assert list(cnt["completed"]) == [want] * len(w.outputs)
    assert list(cnt["valid"]) == [want] * len(w.outputs)   # chi = 1: the H layer reads b_in
    if n * p <= 24:
        a1, _ = feynman.run(w.circuit, w.inputs, w.outputs, eps=eps)
        assert np.max(np.abs(a - a1)) < 1e-14


def test_golden_qaoa_threshold_file_is_consistent():
    """The stored QAOA samples (written by tests/golden/make_qaoa_golden.py
    from the oracle) against the closed form and the seeded requests."""
    g = gold("qaoa_threshold.json")
    for r in g["requests"]:
        w = qaoa_workload(r["n"], r["p"], n_out=r["n_out"], seed=r["seed"])
        assert [int(x) for x in w.outputs[:4]] == r["outputs_head"]
        amp = np.asarray(r["exact_re"]) + 1j * np.asarray(r["exact_im"])
        assert len(amp) == r["n_out"] and np.all(np.abs(amp) <= 1.0)
    for s in g["samples"]:
        w = qaoa_workload(s["n"], s["p"], n_out=4, seed=s["seed"])
        want, margin = _qaoa_closed_form_leaves(s["n"], w.meta["angles"], s["eps"])
        assert s["closed_form_leaves"] == want and margin > 1e-9
        assert s["completed"] == [want] * len(s["index"]) == s["valid"]


def test_walk_checkpoints_beyond_the_remaining_steps_have_zero_subtree_sums():
    """The reading behind the exact reachability bound at the checkpoint: on
    the coined walk a checkpoint state whose position is farther from the
    input's than the steps left after the cut (each step moves it by one)
    has no valid completion, so its exact subtree sum is 0 -- and so is any
    state whose untouched ancilla differs from the input's.  Checked on the
    oracle's checkpoint tables (exact subtree sums by enumeration)."""
    steps, pos_bits = 6, 8
    w = qw_workload(steps=steps, n_out=24, pos_bits=pos_bits)
    c = w.circuit
    G = len(c.gates)
    per_step = G // steps
    mask = (1 << pos_bits) - 1
    seen = 0
    for k_prefix in (2, 3, 4):
        c1 = k_prefix * per_step                   # the last k_prefix steps are the prefix
        left = steps - k_prefix
        for b_in, _ in w.inputs:
            for b_out in w.outputs[:12]:
                t = feynman.checkpoints(c, b_in, b_out, c1)
                for st, live, sub in zip(t["state"], t["live"], t["subtree"]):
                    if not live:
                        continue
                    x, y = (st >> 1) & mask, (b_in >> 1) & mask
                    dist = min((x - y) & mask, (y - x) & mask)
                    anc_differs = ((st ^ b_in) >> (pos_bits + 3)) & 1
                    if dist > left or anc_differs:
                        assert sub == 0, (k_prefix, st, sub)
                        seen += 1
    assert seen > 0


def test_qft_of_a_two_tone_signal_has_four_bins_of_one_half():
    """Dense-support input (Eq. 2 with S ~ 2^n; the paper's QFT signal study,
    Sec. V, Fig. 7): the QFT of x_t = cos(2 pi f1 t/N) + cos(2 pi f2 t/N),
    normalised, is 1/2 at the frequencies f1, N - f1, f2, N - f2 (read
    through the bit reversal of the swap-free QFT) and 0 elsewhere; checked
    on the dense tier at n = 8 and the reduced-history oracle."""
    from workloads import qft_signal_workload
    w = qft_signal_workload(8, seed=12345)
    N = 1 << 8
    f1, f2 = w.meta["f1"], w.meta["f2"]
    want = np.zeros(N, complex)
    for k in (f1, N - f1, f2, N - f2):
        want[closed_forms.bit_reverse(k, 8)] = 0.5
    got = dense.amplitudes(w.circuit, w.inputs, w.outputs)
    assert len(w.inputs) >= N - 4
    assert np.max(np.abs(got - want)) < 1e-13
    o3, _ = feynman.run(w.circuit, w.inputs, w.outputs[:32], threads=4)
    assert np.max(np.abs(o3 - want[:32])) < 1e-13


# ------------------------------------------------ source placement (Sec. IV-B)

def test_fig4_source_placement():
    from workloads import placement_figure
    from oracle import placement
    g = gold("fig4_placement.json")
    c = placement_figure()
    nw, known, cnots = placement.wire_graph(c)
    assert nw - len(known) == g["internal_wires"]
    nodes, _, _ = placement.simplified(c)
    assert len(nodes) == g["nodes_after_merge"]
    assert placement.optimum(c) == g["optimum"]
    assert placement.greedy(c) == g["optimum"]
    assert feynman.analyze(c)["A"] == g["backward"]


def _cnot_h_circuit(n, G, seed):
    rng = SplitMix64(seed)
    gates = []
    for _ in range(G):
        r = rng.below(10)
        q = rng.below(n)
        if r < 5:
            c = rng.below(n - 1)
            c = c + 1 if c >= q else c
            gates.append(Gate("X", (q,), ((c, rng.below(2)),)))
        elif r < 7:
            gates.append(Gate("H", (q,)))
        elif r < 8:
            gates.append(Gate("RX", (q,), (), 0.3 + rng.uniform()))
        elif r < 9:
            gates.append(Gate("P", (q,), (), rng.uniform()))
        else:
            gates.append(Gate("X", (q,)))
    return Circuit(n, gates, f"cnoth{n}x{G}s{seed}")


@pytest.mark.parametrize("seed", range(6))
def test_placement_optimum_is_at_most_greedy_and_backward(seed):
    """The backward sweep's sources make every wire known by backward
    propagation, so the optimum of the graph form is at most A; greedy is a
    feasible choice, so at least the optimum.  The optimum is also checked
    against a literal search over sets of the original (unmerged) wires."""
    from oracle import placement
    from itertools import combinations
    c = _cnot_h_circuit(4, 14, 100 + seed)
    opt, gr, A = placement.optimum(c), placement.greedy(c), feynman.analyze(c)["A"]
    assert opt <= gr and opt <= A
    nw, known, cnots = placement.wire_graph(c)
    wires = [w for w in range(nw) if w not in known]

    def closes(extra):
        kn = set(known) | set(extra)
        grew = True
        while grew:
            grew = False
            for t in cnots:
                if sum(x in kn for x in t) == 2:
                    kn |= set(t)
                    grew = True
        return kn >= set(range(nw))
    lit = next(k for k in range(len(wires) + 1) if any(closes(s) for s in combinations(wires, k)))
    assert lit == opt


def test_pruner_features_against_values_derived_by_hand():
    """The oracle's learned-pruner features (oracle.features) against values
    derived by hand from the feature definition for two checkpoint tables:
    a 3-step walk on 4 position qubits and a 2-qubit QAOA layer (stored with
    the derivation in tests/golden/features_by_hand.json)."""
    from oracle import features as ofeat
    g = gold("features_by_hand.json")
    cases = {"walk": quantum_walk(3, pos_bits=4),
             "qaoa2": Circuit(2, [Gate("H", (0,)), Gate("H", (1,)), Gate("RZZ", (0, 1), (), 0.7),
                                  Gate("RX", (0,), (), 1.1), Gate("RX", (1,), (), 1.1)], "qaoa2")}
    for name, c in cases.items():
        d = g[name]
        assert len(c.gates) == (45 if name == "walk" else 5)
        F, _, Ap = ofeat.table_features(c, d["input"], d["output"], d["c1"])
        assert Ap == d["A_p"] and feynman.analyze(c)["A"] == d["A"]
        for h, want in d["entries"].items():
            assert np.max(np.abs(F[int(h)] - np.asarray(want))) < 1e-12, (name, h, F[int(h)], want)

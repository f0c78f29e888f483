"""Parity of the CUDA path (through the C ABI) with the oracle.

Exact mode: every amplitude within 1e-12 absolute + 1e-10 relative of the
oracle; structure counters (completed and valid histories, gate visits)
bit-exact.  Threshold mode: the device multiplies the same factors in the
same order as the oracle (bit-identical partial amplitudes), so the pruning
decisions and leaf counts must agree exactly."""
import math

import numpy as np
import pytest
import torch

from workloads import (Gate, SplitMix64, aa_workload, four_qubit_figure, qaoa_workload, qft,
                       qft_workload, quantum_walk, qw_workload, random_small_circuit,
                       three_qubit_example)
from oracle import closed_forms, dense, feynman
import paper_2608_01467_b300 as fs

pytestmark = pytest.mark.gpu

ATOL, RTOL = 1e-12, 1e-10


def close(got, want):
    got = np.asarray(got, complex)
    want = np.asarray(want, complex)
    err = np.abs(got - want)
    bad = err > ATOL + RTOL * np.abs(want)
    assert not bad.any(), f"max err {err.max():.3e} at {np.argmax(err)}"


def run_batch(jobs, split="auto", c1=0, c2=0, **kw):
    """jobs: list of (workloads.Circuit, inputs, outputs, eps)."""
    b = fs.Batch(split=split, c1=c1, c2=c2, **kw)
    circs = []
    for circ, inputs, outputs, eps in jobs:
        C = fs.Circuit(circ)
        C.set_input(inputs)
        circs.append(C)
        b.add(C, outputs, eps)
    b.plan()
    b.allocate()
    b.upload()
    b.run()
    stats = b.finish()
    amp = b.amp.cpu().numpy()
    return [amp[s] for s in b.job_slices()], stats, b


def oracle_counts(circ, inputs, outputs, eps=0.0, c1=0, c2=0):
    a, cnt = feynman.run(circ, inputs, outputs, eps=eps, c1=c1, c2=c2, threads=8)
    return a, cnt


def test_three_qubit_example_and_fig2():
    c = three_qubit_example()
    (a,), st, _ = run_batch([(c, [(0, 1.0)], list(range(8)), 0.0)])
    want = np.zeros(8, complex)
    want[0] = math.sqrt(0.5)
    want[7] = 1j * math.sqrt(0.5)
    close(a, want)
    assert st[0]["valid"] == 2 and st[0]["completed"] == 8
    f = four_qubit_figure()
    for b_in in range(16):
        (a,), st, _ = run_batch([(f, [(b_in, 1.0)], list(range(16)), 0.0)])
        o, cnt = oracle_counts(f, [(b_in, 1.0)], list(range(16)))
        close(a, o)
        assert st[0]["valid"] == int(cnt["valid"].sum())
        assert st[0]["completed"] == int(cnt["completed"].sum())


def test_qft8_all_outputs_closed_form():
    w = qft_workload(8)
    (a,), st, _ = run_batch([(w.circuit, w.inputs, w.outputs, 0.0)])
    x = w.meta["x"]
    close(a, [closed_forms.qft_amplitude(8, x, y) for y in range(256)])
    assert st[0]["completed"] == 256 and st[0]["valid"] == 256 and st[0]["candidates"] == 256


@pytest.mark.parametrize("n,G,seed", [(3, 12, 1), (4, 20, 2), (6, 30, 3), (7, 40, 4),
                                      (33, 60, 5), (40, 80, 6), (70, 100, 7), (128, 120, 8)])
def test_random_circuits_every_gate_kind(n, G, seed):
    c = random_small_circuit(n, G, 100 + seed)
    an = feynman.analyze(c)
    if an["A"] > 20:
        pytest.skip(f"A = {an['A']}")
    rng = SplitMix64(seed)
    ins = [(rng.bits(n), complex(0.6, 0.0)), (rng.bits(n), complex(0.0, 0.8))]
    if n <= 7:
        outs = list(range(1 << n))
    else:
        # outputs reachable from the inputs: take dense-free random strings plus
        # the single-history ends of deterministic runs
        outs = [rng.bits(n) for _ in range(40)]
    (a,), st, _ = run_batch([(c, ins, outs, 0.0)])
    o, cnt = oracle_counts(c, ins, outs)
    close(a, o)
    assert st[0]["completed"] == int(cnt["completed"].sum())
    assert st[0]["valid"] == int(cnt["valid"].sum())
    if n <= 7:
        close(a, dense.amplitudes(c, ins, outs))


def test_random_circuit_nonzero_outputs_wide_registers():
    """Outputs with nonzero amplitude on 40/70/128-qubit registers: the
    outputs are read off the dense simulation of the few active qubits."""
    for n in (40, 70, 128):
        rng = SplitMix64(n)
        act = sorted({rng.below(n) for _ in range(6)})
        while len(act) < 5:
            act.append((act[-1] + 1) % n)
            act = sorted(set(act))
        small = random_small_circuit(len(act), 24, 900 + n)
        gates = []
        for g in small.gates:
            gates.append(Gate(g.kind, tuple(act[q] for q in g.qubits),
                              tuple((act[q], v) for q, v in g.controls), g.theta, g.matrix))
        from workloads import Circuit as WC
        big = WC(n, gates, f"embed{n}")
        base = rng.bits(n)
        for q in act:
            base &= ~(1 << q)
        outs = []
        for y in range(1 << len(act)):
            v = base
            for j, q in enumerate(act):
                v |= ((y >> j) & 1) << q
            outs.append(v)
        (a,), st, _ = run_batch([(big, [(base, 1.0)], outs, 0.0)])
        o, _ = oracle_counts(big, [(base, 1.0)], outs)
        close(a, o)
        d = dense.amplitudes(small, [(0, 1.0)], list(range(1 << len(act))))
        close(a, d)
        assert abs(np.sum(np.abs(a) ** 2) - 1) < 1e-12


@pytest.mark.parametrize("family,a_s", [("aa", 6), ("aa", 12), ("qaoa", 12)])
def test_suffix_census_and_per_source_segments_vs_dense(family, a_s):
    """Exact suffixes on the generated engine: amplitude amplification's
    unit-phase suffix counts its leaves by phase (6 sources), with 12 it
    also runs as per-source segments with the class counts checkpointed;
    QAOA's RZZ classes are not unit phases, so 12 sources run as segments
    with table classes.  Against the dense state vector; every history is
    valid in these circuits, so the leaf counts are 2^A per pair."""
    if family == "aa":
        w = aa_workload(n=4, iters=3, seed=7, all_outputs=True)
        outs = w.outputs[:12]
    else:
        w = qaoa_workload(8, 2, n_out=12, seed=13)
        outs = w.outputs
    C = fs.Circuit(w.circuit)
    srcs = {s_: g for g, q, s_ in C.branch_vars() if s_ >= 0}
    G = len(w.circuit.gates)
    A = len(srcs)
    c1 = c2 = G - srcs[A - a_s - 1]
    C.set_input(w.inputs)
    b = fs.Batch(split="fixed", c1=c1, c2=c2, prefix="single")
    b.add(C, outs)
    b.plan()
    src = b.generated_source()
    assert ("CENSUS = true" in src) == (family == "aa")
    assert ("STACKED = true" in src) == (a_s >= 10)
    b.allocate()
    b.upload()
    b.run()
    st = b.finish()[0]
    amp = b.amp.cpu().numpy()[:len(outs)]
    close(amp, dense.amplitudes(w.circuit, w.inputs, outs))
    # no factor of these circuits is zero and every history reaches the input
    # bits: all 2^A histories of every pair complete and are valid
    assert st["valid"] == st["completed"] == len(outs) << A
    assert st["A_s"] == a_s


def test_aa_fig8_ablation_rows_agree():
    w = aa_workload(n=4, iters=3, seed=11, all_outputs=True)
    outs = w.outputs[:10]
    want = dense.amplitudes(w.circuit, w.inputs, outs)
    G = len(w.circuit.gates)
    res = {}
    for name, kw in (("none", dict(split="none", prefix="single")),
                     ("thirds", dict(split="fixed", c1=G // 3, c2=2 * G // 3, prefix="single")),
                     ("auto", dict(split="auto", prefix="single"))):
        (a,), st, _ = run_batch([(w.circuit, w.inputs, outs, 0.0)], **kw)
        close(a, want)
        assert st[0]["valid"] == 10 * (1 << 24)
        res[name] = st[0]
    # gate visits follow Eq. 8 at the chosen cuts, or fewer where the
    # suffix runs as per-source segments (the interpreter follows Eq. 8)
    for name, st in res.items():
        (_, cost) = feynman.region_counts(w.circuit, st["c1"], st["c2"])
        assert st["gate_visits"] <= 10 * cost
    (_,), st_i, _ = run_batch([(w.circuit, w.inputs, outs, 0.0)], split="fixed", c1=res["auto"]["c1"],
                              c2=res["auto"]["c2"], prefix="single", engine="interp")
    assert st_i[0]["gate_visits"] == 10 * feynman.region_counts(w.circuit, res["auto"]["c1"], res["auto"]["c2"])[1]


def test_aa12x1_config_all_outputs_vs_dense():
    """Amplitude amplification on 12 data qubits (10 ancillas, 22 qubits),
    one iteration (A = 24): the 64 requested outputs, autotuned split, against
    the dense state vector; the marked string carries the Grover amplitude
    sin(3 theta), sin(theta) = 2^-6."""
    w = aa_workload(n=12, iters=1)
    (a,), st, _ = run_batch([(w.circuit, w.inputs, w.outputs, 0.0)])
    assert feynman.analyze(w.circuit)["A"] == 24
    close(a, dense.amplitudes(w.circuit, w.inputs, w.outputs))
    theta = math.asin(2.0 ** -6)
    assert abs(abs(a[0]) - math.sin(3 * theta)) < 1e-12
    assert st[0]["completed"] == 64 * (1 << 24)


def test_qaoa8_exact_vs_dense_and_oracle_counts():
    w = qaoa_workload(8, 2, n_out=64, seed=31)
    (a,), st, _ = run_batch([(w.circuit, w.inputs, w.outputs, 0.0)], prefix="single")
    close(a, dense.amplitudes(w.circuit, w.inputs, w.outputs))
    assert st[0]["completed"] == 64 * (1 << 16) == st[0]["valid"]
    cost = feynman.region_counts(w.circuit, st[0]["c1"], st[0]["c2"])[1]
    assert st[0]["gate_visits"] <= 64 * cost      # Eq. 8, or fewer with per-source segments


def test_qaoa16_full_size_sampled_outputs():
    """QAOA p=2 on the 16-qubit graph of the benchmark family (A = 32):
    a sample of requested outputs against the dense state vector."""
    w = qaoa_workload(16, 2, n_out=1024)
    outs = w.outputs[:3]
    (a,), st, _ = run_batch([(w.circuit, w.inputs, outs, 0.0)])
    close(a, dense.amplitudes(w.circuit, w.inputs, outs))
    assert st[0]["valid"] == 3 * (1 << 32)


@pytest.mark.parametrize("eps", [1e-3, 0.02, 0.1])
def test_threshold_pruning_matches_oracle(eps):
    w = qaoa_workload(8, 2, n_out=48, seed=41)
    (a,), st, _ = run_batch([(w.circuit, w.inputs, w.outputs, eps)])
    o, cnt = oracle_counts(w.circuit, w.inputs, w.outputs, eps=eps)
    close(a, o)
    assert st[0]["completed"] == int(cnt["completed"].sum())
    assert st[0]["valid"] == int(cnt["valid"].sum())


@pytest.mark.parametrize("ap,ar", [(4, 2), (4, 5), (3, 8), (2, 12)])
def test_pruned_runs_any_root_width(ap, ar):
    """Pruned jobs run over compacted live entries; with A_r >= 5 a warp's 32
    items share an entry and leave one partial sum, below that one per item.
    Amplitudes and leaf counts against the oracle at the same cuts."""
    w = qaoa_workload(8, 2, n_out=24, seed=61)
    G = len(w.circuit.gates)
    src_gate = {sid: g for g, q, sid in fs.Circuit(w.circuit).branch_vars() if sid >= 0}
    c1, c2 = G - src_gate[ap - 1], G - src_gate[ap + ar - 1]
    eps = 2e-3
    (a,), st, _ = run_batch([(w.circuit, w.inputs, w.outputs, eps)], split="fixed", c1=c1, c2=c2)
    assert (st[0]["A_p"], st[0]["A_r"]) == (ap, ar)
    o, cnt = oracle_counts(w.circuit, w.inputs, w.outputs, eps=eps, c1=c1, c2=c2)
    close(a, o)
    assert st[0]["completed"] == int(cnt["completed"].sum())
    assert st[0]["valid"] == int(cnt["valid"].sum())


def test_qw_small_vs_offset_walk():
    w = qw_workload(steps=6, n_out=64, pos_bits=8)
    (a,), st, _ = run_batch([(w.circuit, w.inputs, w.outputs, 0.0)])
    s = math.sqrt(0.5)
    close(a, [closed_forms.walk_amplitude(6, w.meta["p0"], y, s, 1j * s, 8) for y in w.outputs])
    o, cnt = oracle_counts(w.circuit, w.inputs, w.outputs)
    assert st[0]["valid"] == int(cnt["valid"].sum())
    assert st[0]["completed"] == int(cnt["completed"].sum())


def test_qw100_full_config_all_outputs():
    """100-qubit walk, T = 16, 4096 outputs (the benchmark request): every
    amplitude against the offset-space walk; norm 1 over the reachable
    outputs; unreachable ones exactly zero; a sample of outputs against the
    oracle's history counts."""
    w = qw_workload()
    (a,), st, _ = run_batch([(w.circuit, w.inputs, w.outputs, 0.0)])
    s = math.sqrt(0.5)
    want = [closed_forms.walk_amplitude(16, w.meta["p0"], y, s, 1j * s, 96) for y in w.outputs]
    close(a, want)
    r = w.meta["reachable"]
    assert abs(np.sum(np.abs(a[:r]) ** 2) - 1) < 1e-12
    assert np.all(a[r:] == 0)
    assert st[0]["completed"] == 2 * 4096 * (1 << 15)
    sample = [w.outputs[0], w.outputs[17], w.outputs[r + 5]]
    _, cnt = oracle_counts(w.circuit, w.inputs, sample)
    b2, st2, _ = run_batch([(w.circuit, w.inputs, sample, 0.0)])
    assert st2[0]["valid"] == int(cnt["valid"].sum())


def test_mixed_batch_one_launch():
    """Jobs of different register widths and sizes in one persistent launch."""
    j1 = qft_workload(8)
    j2 = qaoa_workload(8, 2, n_out=32, seed=2)
    j3 = qw_workload(steps=5, n_out=40, pos_bits=8)
    c4 = random_small_circuit(70, 60, 77)
    rng = SplitMix64(4)
    j4 = (c4, [(rng.bits(70), 1.0)], [rng.bits(70) for _ in range(20)], 0.0)
    jobs = [(j1.circuit, j1.inputs, j1.outputs, 0.0), (j2.circuit, j2.inputs, j2.outputs, 0.0),
            (j3.circuit, j3.inputs, j3.outputs, 0.0), j4,
            (j2.circuit, j2.inputs, [], 0.0)]
    amps, st, b = run_batch(jobs)
    for (circ, ins, outs, eps), a in zip(jobs, amps):
        if not outs:
            assert len(a) == 0
            continue
        o, _ = oracle_counts(circ, ins, outs)
        close(a, o)


def test_reduction_large_and_small_outputs_in_one_warp():
    """Outputs with thousands of per-tile partials (the whole-warp and the
    block-per-output paths of the reduction) next to outputs with a handful,
    with input supports of 1 and 2 terms, in one batch; every amplitude
    against the oracle."""
    big = qaoa_workload(10, 2, n_out=3, seed=5)            # A = 20: 4096 partials, one warp each
    hc = random_small_circuit(8, 70, 701)                   # A = 22: 16384 partials, one block each
    hrng = SplitMix64(701)
    small = qft_workload(8)
    c = random_small_circuit(6, 30, 606)
    rng = SplitMix64(606)
    two = (c, [(rng.bits(6), 0.6), (rng.bits(6), 0.8j)], list(range(64)), 0.0)
    jobs = [(small.circuit, small.inputs, small.outputs[:5], 0.0),
            (big.circuit, big.inputs, big.outputs, 0.0), two,
            (small.circuit, small.inputs, small.outputs[5:40], 0.0),
            (hc, [(hrng.bits(8), 1.0)], [hrng.bits(8) for _ in range(2)], 0.0)]
    b = fs.Batch()
    circs = []
    for circ, ins, outs, eps in jobs:
        C = fs.Circuit(circ)
        C.set_input(ins)
        circs.append(C)
        b.add(C, outs, eps)
    b.set_cuts(1, 0, len(big.circuit.gates))   # one region: 2^20 items, 4096 partials per output
    b.set_cuts(4, 0, len(hc.gates))           # one region: 2^22 items
    b.plan()
    b.allocate()
    b.upload()
    b.run()
    st = b.finish()
    assert st[1]["A_r"] == 20 and st[4]["A_r"] == 22
    amp = b.amp.cpu().numpy()
    for (circ, ins, outs, eps), sl in zip(jobs, b.job_slices()):
        o, _ = oracle_counts(circ, ins, outs)
        close(amp[sl], o)


def _cascade_circuit(n, field, common, inc, order_msb_first, hs):
    """H on qubits hs, then a +1 (inc) or -1 on the qubits `field` (first =
    least significant) controlled on `common`, written as multi-controlled X
    gates most (or least) significant first, then H on hs again."""
    from workloads import Circuit as WC
    g = [Gate("H", (q,)) for q in hs]
    v = 1 if inc else 0
    ks = range(len(field) - 1, -1, -1) if order_msb_first else range(len(field))
    for k in ks:
        ctr = tuple(common) + tuple((field[j], v) for j in range(k))
        g.append(Gate("X", (field[k],), ctr) if ctr else Gate("X", (field[k],)))
    g += [Gate("H", (q,)) for q in hs]
    return WC(n, g, "cascade")


@pytest.mark.parametrize("n,f0,L,common,inc,msb", [
    (12, 2, 8, (), True, True), (12, 2, 8, ((0, 1),), False, True), (45, 27, 12, ((1, 0),), True, True),
    (70, 5, 60, ((0, 1), (68, 0)), False, True), (128, 1, 120, ((0, 1),), True, True),
    (45, 27, 12, ((1, 1),), True, False)])
def test_incrementer_cascades_match_oracle(n, f0, L, common, inc, msb):
    """Controlled +-1 on a contiguous field (within a word and across word
    boundaries, with and without common controls of either polarity): the
    straight-line engine replaces such MCX cascades by one borrow chain,
    which must agree with the oracle's gate-by-gate evaluation and with the
    interpreter bit for bit."""
    field = list(range(f0, f0 + L))
    hs = [f0, f0 + 1, f0 + L - 1] + [q for q, _ in common]
    c = _cascade_circuit(n, field, common, inc, msb, hs)
    rng = SplitMix64(n + L)
    ins = [(rng.bits(n), 1.0)]
    outs = [rng.bits(n) for _ in range(6)]
    # outputs reachable from the input: flip the H qubits and move the field by one
    b = ins[0][0]
    for k in range(16):
        y = b
        for j, q in enumerate(hs):
            if (k >> j) & 1:
                y ^= 1 << q
        x = (y >> f0) & ((1 << L) - 1)
        x = (x + (1 if inc else -1)) % (1 << L)
        outs.append((y & ~(((1 << L) - 1) << f0)) | (x << f0))
    a1, s1, _ = run_batch([(c, ins, outs, 0.0)], engine="straight")
    a2, s2, _ = run_batch([(c, ins, outs, 0.0)], engine="interp")
    o, cnt = oracle_counts(c, ins, outs)
    close(a1[0], o)
    close(a2[0], o)
    assert np.abs(o).max() > 0.1
    for k in ("completed", "valid"):
        assert s1[0][k] == s2[0][k], k
    assert s1[0]["gate_visits"] <= s2[0]["gate_visits"]
    assert s1[0]["valid"] == int(cnt["valid"].sum())


@pytest.mark.parametrize("S", [3, 5])
def test_input_support_not_a_power_of_two(S):
    """Sparse inputs of 3 and 5 basis states (Eq. 2): pair indices are split
    into (output, input) by a precomputed multiplier; exact, threshold and
    learned-free compacted runs against the oracle."""
    c = random_small_circuit(9, 50, 900 + S)
    rng = SplitMix64(S)
    ins = [(rng.bits(9), complex(0.3 * (k + 1), 0.1 * k)) for k in range(S)]
    outs = [rng.bits(9) for _ in range(37)]
    for eps in (0.0, 0.05):
        (a,), st, _ = run_batch([(c, ins, outs, eps)])
        o, cnt = oracle_counts(c, ins, outs, eps=eps, c1=st[0]["c1"], c2=st[0]["c2"])
        close(a, o)
        assert st[0]["valid"] == int(cnt["valid"].sum())


def test_deterministic_and_host_path_bitwise():
    w = qaoa_workload(8, 2, n_out=40, seed=9)
    (a1,), _, b = run_batch([(w.circuit, w.inputs, w.outputs, 0.0)])
    b.run()
    b.finish()
    a2 = b.amp.cpu().numpy()
    assert np.array_equal(a1, a2)
    C = fs.Circuit(w.circuit)
    C.set_input(w.inputs)
    a3 = C.amplitudes(w.outputs)
    assert np.array_equal(a1, a3)


def test_cuda_graph_capture_of_run():
    w = qaoa_workload(8, 2, n_out=40, seed=10)
    (a1,), _, b = run_batch([(w.circuit, w.inputs, w.outputs, 0.0)])
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    b.amp.zero_()
    with torch.cuda.graph(g, stream=s):
        b.run(stream=s)
    for _ in range(3):
        b.amp.zero_()
        g.replay()
    torch.cuda.synchronize()
    assert np.array_equal(b.amp.cpu().numpy(), a1)
    # later uploads stage through pinned memory without waiting; the graph
    # stays valid and sees the refreshed request
    for _ in range(3):
        b.upload(stream=s)
        with torch.cuda.stream(s):
            b.amp.zero_()
            g.replay()
        b.finish(stream=s)
        assert np.array_equal(b.amp.cpu().numpy(), a1)


def test_edge_cases_ragged_and_empty():
    c = qft(3)
    (a,), st, _ = run_batch([(c, [(5, 1.0)], [0, 1, 2, 3, 4], 0.0)])
    close(a, [closed_forms.qft_amplitude(3, 5, y) for y in range(5)])
    # no outputs at all
    amps, st, _ = run_batch([(c, [(5, 1.0)], [], 0.0)])
    assert len(amps[0]) == 0
    # empty circuit: identity
    from workloads import Circuit as WC
    e = WC(5, [], "empty")
    (a,), st, _ = run_batch([(e, [(9, 1.0)], [9, 8], 0.0)])
    close(a, [1.0, 0.0])
    # host convenience call with zero outputs
    C = fs.Circuit(c)
    assert len(C.amplitudes([])) == 0


@pytest.mark.parametrize("case", ["qaoa_exact", "qaoa_eps", "qw", "qw96", "rand7", "rand70", "aa"])
def test_engines_bitwise_equal(case):
    """The generated straight-line kernel and the interpreter agree within
    the exact-mode tolerance (the generated code defers two-valued factors
    into per-class tables: in exact mode everywhere, with a threshold after
    the last |beta| test), and their counters exactly: with a threshold every
    test sees the same double in both engines, so every pruning decision is
    the same."""
    if case.startswith("qaoa"):
        w = qaoa_workload(8, 2, n_out=40, seed=77)
        jobs = [(w.circuit, w.inputs, w.outputs, 0.05 if case == "qaoa_eps" else 0.0)]
    elif case == "qw":
        w = qw_workload(steps=6, n_out=40, pos_bits=8)
        jobs = [(w.circuit, w.inputs, w.outputs, 0.0)]
    elif case == "qw96":
        w = qw_workload(steps=6, n_out=40)
        jobs = [(w.circuit, w.inputs, w.outputs, 0.0)]
    elif case == "aa":
        w = aa_workload(n=4, iters=2, seed=3, all_outputs=True)
        jobs = [(w.circuit, w.inputs, w.outputs[:6], 0.0)]
    else:
        n = 7 if case == "rand7" else 70
        c = random_small_circuit(n, 40 if n == 7 else 90, 4242 + n)
        rng = SplitMix64(n)
        outs = list(range(1 << n)) if n == 7 else [rng.bits(n) for _ in range(30)]
        jobs = [(c, [(rng.bits(n), 0.6), (rng.bits(n), 0.8j)], outs, 0.0)]
    a1, s1, b1 = run_batch(jobs, engine="straight")
    a2, s2, b2 = run_batch(jobs, engine="interp")
    assert b1.engine()[0] == "straight" and b2.engine()[0] == "interp"
    for x, y in zip(a1, a2):
        close(x, y)
    for x, y in zip(s1, s2):
        for k in ("completed", "valid", "table_entries"):
            assert x[k] == y[k], k
        # a stacked suffix (per-source segments) restarts at the changed
        # source instead of the region start: it evaluates no more gates
        assert x["gate_visits"] <= y["gate_visits"]
    o, _ = oracle_counts(*jobs[0][:3], eps=jobs[0][3])
    close(a1[0], o)


@pytest.mark.parametrize("engine", ["straight", "interp"])
def test_level_prefix_equals_single_region_prefix(engine):
    """The prefix expanded one source level at a time gives the same
    checkpoint table as Algorithm 2's one region per prefix assignment:
    same amplitudes and history counts, fewer prefix gate visits."""
    for w, eps in ((qaoa_workload(8, 2, n_out=48, seed=51), 0.0), (qaoa_workload(8, 2, n_out=48, seed=52), 0.02),
                   (qw_workload(steps=6, n_out=40, pos_bits=8), 0.0)):
        G = len(w.circuit.gates)
        jobs = [(w.circuit, w.inputs, w.outputs, eps)]
        a1, s1, _ = run_batch(jobs, split="fixed", c1=2 * G // 3, c2=5 * G // 6, prefix="single", engine=engine)
        a2, s2, _ = run_batch(jobs, split="fixed", c1=2 * G // 3, c2=5 * G // 6, prefix="levels", engine=engine)
        a3, s3, b3 = run_batch(jobs, split="fixed", c1=2 * G // 3, c2=5 * G // 6, prefix="auto", engine=engine)
        close(a2[0], a1[0])
        close(a3[0], a1[0])
        for k in ("completed", "valid", "table_entries", "history_visits"):
            assert s1[0][k] == s2[0][k] == s3[0][k], k
        assert s2[0]["gate_visits"] - s2[0]["history_visits"] < s1[0]["gate_visits"] - s1[0]["history_visits"]
        # the automatic split is one of the segmentations in between
        pre = lambda st: st["gate_visits"] - st["history_visits"]
        assert pre(s2[0]) <= pre(s3[0]) <= pre(s1[0])

"""Host-side tests of the library (no GPU needed): the C ABI loads and
exports every declared symbol, the host analysis is bit-exact against the
oracle's, the autotuner picks the oracle's argmin of Eq. 8, argument errors
are reported with the documented codes."""
import ctypes
import math
import os
import re
import subprocess

import numpy as np
import pytest

from workloads import (Gate, Circuit as WCircuit, SplitMix64, aa_workload, amplitude_amplification,
                       four_qubit_figure, qaoa_maxcut, qaoa_workload, qft, quantum_walk,
                       qw_workload, random_small_circuit, three_qubit_example)
from oracle import feynman
import paper_2608_01467_b300 as fs
from paper_2608_01467_b300 import _lib
from paper_2608_01467_b300.build import LIB, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def setup_module(module):
    build()


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "feynsparse.h")).read()
    return sorted(set(re.findall(r"FS_API\s+[\w\s\*]*?\b(fs_\w+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    names = declared_symbols()
    assert len(names) >= 20
    L = ctypes.CDLL(LIB)
    for n in names:
        assert hasattr(L, n), n
    # and only those (plus nothing else called fs_*)
    out = subprocess.run(["nm", "-D", "--defined-only", LIB], capture_output=True, text=True).stdout
    exported = sorted({ln.split()[-1] for ln in out.splitlines() if " T fs_" in ln})
    assert exported == names
    assert set(_lib.exported_symbols()) == set(names)


def test_version_and_last_error():
    L = _lib.load()
    assert b"sm_103a" in L.fs_version()
    h = ctypes.c_void_p()
    rc = L.fs_circuit_create(None, 3, 2, ctypes.byref(h))
    assert rc == -1
    assert b"NULL" in L.fs_last_error()


CIRCUITS = [
    four_qubit_figure(), three_qubit_example(), qft(8), qft(12),
    amplitude_amplification(12, 3, 0xA5C), amplitude_amplification(6, 3, 17),
    amplitude_amplification(4, 3, 0),
    qaoa_maxcut(16, 2, SplitMix64(1))[0], qaoa_maxcut(24, 3, SplitMix64(2))[0],
    quantum_walk(16), quantum_walk(6, pos_bits=8),
] + [random_small_circuit(n, g, s) for n, g, s in
     [(3, 10, 1), (5, 30, 2), (7, 40, 3), (40, 80, 4), (70, 120, 5), (128, 150, 6)]]


@pytest.mark.parametrize("idx", range(len(CIRCUITS)))
def test_analysis_bit_exact_vs_oracle(idx):
    c = CIRCUITS[idx]
    o = feynman.analyze(c)
    C = fs.Circuit(c)
    a = C.analyze(0)
    assert a["A"] == o["A"]
    assert a["n_gates"] == len(c.gates)
    roles = o["roles"]
    assert a["n_wp"] == roles.count("WP") and a["n_det"] == roles.count("DET") and a["n_br"] == roles.count("BR")
    # branching variables: same gates, same qubits, same source ids (backward order)
    want = []
    for gi in range(len(c.gates) - 1, -1, -1):
        if roles[gi] != "BR":
            continue
        g = c.gates[gi]
        tq = list(g.qubits)
        order = sorted(range(len(tq)), key=lambda j: tq[j])
        for j in order:
            want.append((gi, tq[j], o["src"][gi][j]))
    assert C.branch_vars() == want
    assert a["n_natural"] == sum(1 for w in want if w[2] == -1)


@pytest.mark.parametrize("idx", [0, 1, 2, 5, 6, 7, 10, 12, 13])
def test_autotune_matches_oracle_argmin(idx):
    c = CIRCUITS[idx]
    a = fs.Circuit(c).analyze(0)
    c1, c2, cost = feynman.autotune(c, max_ap=a["max_ap"], min_apr=a["min_apr"], max_apr=a["max_apr"])
    assert (a["c1"], a["c2"]) == (c1, c2)
    assert a["gateops"] == cost
    (Gp, Gr, Gs, Ap, Ar, As), cost2 = feynman.region_counts(c, c1, c2)
    assert (a["G_p"], a["G_r"], a["G_s"], a["A_p"], a["A_r"], a["A_s"]) == (Gp, Gr, Gs, Ap, Ar, As)


def test_table1_counts_through_the_abi():
    assert fs.Circuit(qft(8)).analyze(0x3C)["A"] == 0
    assert fs.Circuit(amplitude_amplification(12, 3, 77)).analyze(0)["A"] == 72
    assert fs.Circuit(qaoa_maxcut(20, 2, SplitMix64(5))[0]).analyze(0)["A"] == 40
    assert fs.Circuit(quantum_walk(16)).analyze(0)["A"] == 15


def _err(gates, n):
    with pytest.raises(_lib.FsError) as e:
        fs.Circuit(gates=gates, n_qubits=n)
    return e.value.code


def test_argument_errors():
    assert _err([Gate("H", (3,))], 3) == -1                                  # qubit out of range
    assert _err([Gate("H", (0,))], 129) == -3                                # too many qubits
    assert _err([Gate("U1", (0,), (), 0.0, (1, 1, 0, 1))], 2) == -4          # not unitary
    assert _err([Gate("SWAP", (1, 1))], 2) == -1                             # repeated target
    assert _err([Gate("X", (0,), ((0, 1),))], 2) == -1                       # target is a control
    assert _err([Gate("X", (0,), ((5, 1),))], 3) == -1                       # control out of range
    g = _lib.fs_gate()
    g.kind = 1
    g.n_q = 1
    g.ctrl_mask[0] = 2
    g.ctrl_val[0] = 4                                                        # value outside mask
    h = ctypes.c_void_p()
    assert _lib.load().fs_circuit_create((_lib.fs_gate * 1)(g), 1, 3, ctypes.byref(h)) == -1
    g2 = _lib.fs_gate()
    g2.kind = 0
    g2.n_q = 1
    g2.ctrl_mask[0] = 2                                                      # controlled H
    assert _lib.load().fs_circuit_create((_lib.fs_gate * 1)(g2), 1, 3, ctypes.byref(h)) == -2
    g3 = _lib.fs_gate()
    g3.kind = 99
    g3.n_q = 1
    assert _lib.load().fs_circuit_create((_lib.fs_gate * 1)(g3), 1, 3, ctypes.byref(h)) == -2


def test_bits_beyond_n_rejected():
    C = fs.Circuit(qft(4))
    with pytest.raises(_lib.FsError):
        C.analyze(1 << 5)
    with pytest.raises(_lib.FsError):
        C.set_input([(1 << 4, 1.0)])
    b = fs.Batch()
    with pytest.raises(_lib.FsError):
        b.add(C, [1 << 7])


def test_plan_rejects_unenumerable_A():
    C = fs.Circuit(amplitude_amplification(12, 3, 5))
    b = fs.Batch()
    b.add(C, [0, 1])
    with pytest.raises(_lib.FsError) as e:
        b.plan()
    assert e.value.code == -9


def test_plan_layout_and_fixed_split_errors():
    w = qaoa_workload(8, 2, n_out=16, seed=3)
    C = fs.Circuit(w.circuit)
    b = fs.Batch(split="fixed", c1=5, c2=3)
    b.add(C, w.outputs)
    with pytest.raises(_lib.FsError):
        b.plan()
    b2 = fs.Batch(prefix="single")
    b2.add(C, w.outputs)
    b2.add(C, [])                      # empty job is allowed
    n = b2.plan()
    assert n > 0 and n % 256 == 0
    assert b2.total_outputs == 16
    # prefix, history, reduce by lane groups (no output can exceed what a
    # warp of the reduction sums, so the block-per-output pass is skipped)
    assert b2.launch_count() == 3
    b3 = fs.Batch(prefix="levels")     # prefix expanded one level per source op
    b3.add(C, w.outputs)
    b3.plan()
    st_levels = b3.launch_count() - 2  # levels + history + reduce
    assert st_levels >= 2


def test_mlp_forward_rejects_misaligned_features_before_any_device_work():
    L = fs._lib.load()
    rc = L.fs_mlp_forward(ctypes.c_void_p(256), ctypes.c_void_p(256 + 8), 1, ctypes.c_void_p(512), None)
    assert rc == -1 and b"16-byte" in L.fs_last_error()
    assert L.fs_mlp_forward(None, ctypes.c_void_p(256), 1, ctypes.c_void_p(512), None) == -1


def test_run_before_upload_is_a_state_error():
    C = fs.Circuit(qft(3))
    b = fs.Batch()
    b.add(C, [0, 1])
    b.plan()
    L = _lib.load()
    rc = L.fs_batch_run(b._h, ctypes.c_void_p(256), ctypes.c_void_p(512), None)
    assert rc == -10


def test_upload_rejects_truncated_or_misaligned_workspace():
    """Truncated and misaligned device buffers are refused on the host,
    before any device work is enqueued."""
    w = qaoa_workload(6, 2, n_out=8, seed=4)
    C = fs.Circuit(w.circuit)
    b = fs.Batch()
    b.add(C, w.outputs)
    n = b.plan()
    L = _lib.load()
    assert L.fs_batch_upload(b._h, ctypes.c_void_p(1 << 20), n - 256, None) == -1
    assert b"needed" in L.fs_last_error()
    assert L.fs_batch_upload(b._h, ctypes.c_void_p((1 << 20) + 16), n, None) == -1
    assert b"aligned" in L.fs_last_error()
    assert L.fs_batch_upload(b._h, None, n, None) == -1


def test_options_and_cut_validation():
    L = _lib.load()
    b = fs.Batch()
    bad = _lib.fs_options()
    bad.split = 7
    assert L.fs_batch_set_options(b._h, ctypes.byref(bad)) == -1
    bad = _lib.fs_options()
    bad.engine = 3
    assert L.fs_batch_set_options(b._h, ctypes.byref(bad)) == -1
    C = fs.Circuit(qft(4))
    b.add(C, [1, 2])
    assert L.fs_batch_set_cuts(b._h, 0, 5, 2) == -1
    assert L.fs_batch_set_cuts(b._h, 3, 0, 0) == -1
    assert L.fs_batch_set_cuts(b._h, 0, 2, 99) == 0
    with pytest.raises(_lib.FsError):
        b.plan()                       # c2 beyond the gate count
    assert L.fs_batch_set_cuts(b._h, 0, -1, -1) == 0
    assert b.plan() > 0


def _walk_like(n, f0, L, msb_first):
    """H on the coin (qubit 0), then +1 on qubits f0 .. f0+L-1 controlled on
    the coin, as multi-controlled X gates most (or least) significant first."""
    g = [Gate("H", (0,))]
    ks = range(L - 1, -1, -1) if msb_first else range(L)
    for k in ks:
        g.append(Gate("X", (f0 + k,), ((0, 1),) + tuple((f0 + j, 1) for j in range(k))))
    return WCircuit(n, g, "inc")


def test_work_model_counts_fused_incrementers_for_the_generated_engine():
    """The straight-line engine replaces a controlled +-1 written as an MCX
    cascade (most significant gate first, i.e. least significant first in the
    output-to-input evaluation order) by one borrow chain; the work model
    counts it that way for that engine only, and a cascade in the other
    order is left gate by gate."""
    for msb_first, fused in ((True, True), (False, False)):
        c = _walk_like(40, 3, 30, msb_first)
        C = fs.Circuit(c)
        C.set_input([(0, 1.0)])
        work = {}
        for engine in ("straight", "interp"):
            b = fs.Batch(split="fixed", c1=0, c2=len(c.gates), engine=engine)
            b.add(C, [0, 1])
            b.plan()
            work[engine] = b.region_work(0)[0][1]   # root region integer ops
        # the straight-line engine's item loop around the root: 24
        loop = 24
        if fused:
            # H deferred (3 + 1 class count) + its unit-phase class applied as a
            # sign flip (3) + the cascade: common-control test on 1 word (2),
            # 5 for the field's first register word and a vote (2) guarding
            # the second word, which only a borrow reaches
            assert work["straight"] == 4 + 3 + 2 + 5 + 2 + loop
            assert work["straight"] - loop < work["interp"] / 4
        else:
            # gate by gate in both engines; they differ only in the H: 4 integer
            # ops + 2 FP64 literally, 4 + 3 (sign flip) deferred and hoisted
            assert work["straight"] == work["interp"] + 3 + loop


def test_automatic_prefix_segmentation_is_between_flat_and_per_source():
    """prefix="auto" keeps some of the per-source level boundaries: never more
    launches than one level per source op, never fewer than the flat prefix;
    on the 100-qubit walk with A_p = 10 it splits (large table), with A_p = 2
    it keeps the flat prefix (the extra launches cost more than they save)."""
    w = qw_workload(n_out=512)
    G = len(w.circuit.gates)
    src_gate = {sid: g for g, q, sid in fs.Circuit(w.circuit).branch_vars() if sid >= 0}
    C = fs.Circuit(w.circuit)
    C.set_input(w.inputs)
    counts = {}
    for ap in (2, 10):
        c1 = G - src_gate[ap - 1]
        for mode in ("single", "levels", "auto"):
            b = fs.Batch(split="fixed", c1=c1, c2=c1, prefix=mode)
            b.add(C, w.outputs)
            b.plan()
            counts[(ap, mode)] = b.launch_count()
        assert counts[(ap, "single")] <= counts[(ap, "auto")] <= counts[(ap, "levels")]
    assert counts[(2, "auto")] == counts[(2, "single")]
    assert counts[(10, "auto")] > counts[(10, "single")]


def test_generated_source_requires_a_plan_and_reports_its_length():
    C = fs.Circuit(qft(3))
    b = fs.Batch()
    b.add(C, [0, 1])
    L = fs._lib.load()
    n = ctypes.c_size_t(0)
    assert L.fs_batch_generated_source(b._h, None, 0, ctypes.byref(n)) == -10   # FS_ERR_STATE
    b.plan()
    assert L.fs_batch_generated_source(b._h, None, 0, ctypes.byref(n)) == 0 and n.value > 1000
    small = ctypes.create_string_buffer(16)
    assert L.fs_batch_generated_source(b._h, small, 16, ctypes.byref(n)) == 0
    assert len(small.value) == 15 and n.value > 1000   # truncated, NUL-terminated
    src = b.generated_source()
    assert len(src) == n.value and "struct J0" in src and "fs_jit_history" in src


HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "feynsparse.h")
CITATION = re.compile(r"(Sec\. [IV]|Eqs?\. ?\d|Algorithm \d|Observation \d|Fig\. \d|Table \d|no counterpart)")


def test_every_exported_call_cites_its_passage():
    """Each FS_API declaration of the header is preceded by a comment that
    names the passage of the paper it follows (section, equation, algorithm,
    observation, figure or table) or says that the paper has no counterpart."""
    lines = open(HEADER).read().split("\n")
    missing = []
    for i, line in enumerate(lines):
        if not line.startswith("FS_API"):
            continue
        j, block = i - 1, []
        while j >= 0 and (lines[j].startswith(("FS_API", "#define")) or lines[j].strip().startswith(("/*", "*"))
                          or lines[j].startswith(" " * 8)):
            block.append(lines[j])
            j -= 1
        if not CITATION.search("\n".join(block)):
            missing.append(line)
    assert not missing, missing
    names = set(re.findall(r"FS_API [^(]*?\b(fs_\w+)\(", open(HEADER).read()))
    assert names == set(_lib.exported_symbols()), names ^ set(_lib.exported_symbols())


def test_device_wait_limit_program_offset_and_targets_argument_checks():
    L = _lib.load()
    b = fs.Batch()
    assert L.fs_batch_set_device(b._h, -2) == -1
    assert L.fs_batch_set_device(b._h, -1) == 0
    w = qaoa_workload(6, 2, n_out=4, seed=9)
    C = fs.Circuit(w.circuit)
    b.add(C, w.outputs)
    off, n = ctypes.c_size_t(0), ctypes.c_size_t(0)
    assert L.fs_batch_program_offset(b._h, 0, ctypes.byref(off), ctypes.byref(n)) == -10
    b.plan()
    o, k = b.program_offset(0)
    assert k == len(w.circuit.gates) and o % 256 == 0
    assert L.fs_batch_program_offset(b._h, 1, ctypes.byref(off), ctypes.byref(n)) == -1
    assert L.fs_set_wait_limit(1 << 33) == -1
    assert L.fs_set_wait_limit(-1) == 0
    assert L.fs_mlp_targets(ctypes.c_void_p(256), 4, float("nan"), ctypes.c_void_p(512), None) == -1
    assert L.fs_mlp_targets(None, 4, -12.0, ctypes.c_void_p(512), None) == -1


def test_threshold_jobs_plan_beyond_62_sources_and_keep_the_root_narrow():
    """An exact job with A = 72 (QAOA-24, p = 3) is refused (2^72 histories
    per pair); with a threshold the suffix skips cut subtrees, so it plans
    with every region's word within 62 bits.  A threshold job's root adds no
    more assignments than the parallelism floor needs, and its cuts are the
    oracle's Eq. 8 argmin under the same bounds."""
    w = qaoa_workload(24, 3, n_out=1024, seed=0x5EED0004)
    C = fs.Circuit(w.circuit)
    b = fs.Batch()
    b.add(C, w.outputs, 0.0)
    with pytest.raises(_lib.FsError) as e:
        b.plan()
    assert e.value.code == -9
    for n, p, A in ((24, 3, 72), (16, 2, 32)):
        w = qaoa_workload(n, p, n_out=1024, seed=0x5EED0004)
        C = fs.Circuit(w.circuit)
        b = fs.Batch()
        b.add(C, w.outputs, 1e-6)
        b.plan()
        iw, _ = b.region_work(0)
        assert all(x >= 0 for x in iw)
        # budget 4 GiB / (1024 pairs x 40 B) -> A_p <= 16; floor 2^19 items -> A_p + A_r >= 9
        max_ap, min_apr, max_apr = 16, 9, 16
        c1, c2, cost = feynman.autotune(w.circuit, max_ap=max_ap, min_apr=min_apr, max_apr=max_apr)
        (Gp, Gr, Gs, Ap, Ar, As), _ = feynman.region_counts(w.circuit, c1, c2)
        assert Ap + Ar + As == A and As <= 62 and Ap + Ar <= max_apr
        hist = b.op_histogram(0)
        assert sum(hist["prefix"].values()) == Gp and sum(hist["root"].values()) == Gr


def test_source_placement_matches_the_oracle():
    """fs_source_placement (graph form of Sec. IV-B) against the oracle's
    own graph reduction: Fig. 4 (backward 2, optimum 1 on 3 merged nodes)
    and random CNOT + single-qubit circuits; other gates are refused."""
    import importlib
    from workloads import placement_figure
    from oracle import placement
    pins = importlib.import_module("test_oracle_pins")
    circuits = [placement_figure()] + [pins._cnot_h_circuit(5, 18, 300 + s) for s in range(8)]
    for c in circuits:
        C = fs.Circuit(c)
        nodes = len(placement.simplified(c)[0])
        assert C.source_placement("backward")[0] == feynman.analyze(c)["A"]
        assert C.source_placement("greedy") == (placement.greedy(c), nodes)
        assert C.source_placement("optimal") == (placement.optimum(c), nodes)
    C = fs.Circuit(qw_workload(steps=3, n_out=4, pos_bits=8).circuit)    # multi-controlled X
    with pytest.raises(_lib.FsError) as e:
        C.source_placement("greedy")
    assert e.value.code == -2


def test_compacted_exact_job_launches():
    """An exact job with the reachability bound, on the generated engine:
    the prefix (bound applied, live entries counted per compaction block),
    the compaction's write pass (it adds the block counts before its own
    when there are at most 1024 blocks: no scan launch) and the compacted
    history, which also reduces the outputs (A_r >= 5, at most 4096 sums
    per output): three launches.  The interpreter keeps its bound pass and
    the reduction kernel; a table of more than 1024 compaction blocks adds
    the scan."""
    w = qw_workload(n_out=1024)
    C = fs.Circuit(w.circuit)
    C.set_input(w.inputs)
    G = len(w.circuit.gates)
    src = {s: g for g, q, s in C.branch_vars() if s >= 0}

    def count(engine, ap, ar):
        # evaluation positions after the first ap and ap + ar backward
        # sources; the prefix as one region (no per-source levels)
        b = fs.Batch(engine=engine, prefix="single")
        b.add(C, w.outputs, 0.0)
        b.set_exact_bound(0)
        b.set_cuts(0, G - src[ap - 1], G - src[ap + ar - 1])
        b.plan()
        return b.launch_count()

    assert count("straight", 4, 8) == 3        # 2048 pairs x 16 entries: 32 blocks
    assert count("interp", 4, 8) == 5          # bound pass, prefix, write, history, reduction
    # 2048 pairs x 1024 entries: 2048 blocks (scan); A_r < 5: the reduction,
    # and its pass for outputs of more than 4096 sums
    assert count("straight", 10, 4) == 6
    assert count("straight", 9, 5) == 3        # 1024 blocks
    assert count("straight", 4, 3) == 4        # A_r = 3: the reduction kernel sums per item

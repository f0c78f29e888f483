"""Host-side checks of the bench's QAOA-24 p = 3 learned-vs-threshold
workload (no GPU): its request is the stored one (so the fidelity of both
arms is judged by the stored dense amplitudes), its cuts put 12 sources
before the checkpoint and 4 in the root, and the held-out outputs that
choose tau are disjoint from the timed ones."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import paper_2608_01467_b300 as fs  # noqa: E402
from workloads import qaoa_workload  # noqa: E402


def test_qaoa24p3_workload_is_the_stored_request():
    jobs, cfg = bench.family_jobs("qaoa24p3")
    assert len(jobs) == 1 and cfg["outputs"] == 64 and cfg["cut_sources"] == [12, 4]
    w = jobs[0]
    assert w.name == "qaoa24p3" and w.eps == bench.QAOA24P3_EPS
    ex = bench.exact_reference(w)
    assert ex is not None and ex.shape == (64,)
    assert np.array_equal(ex, bench.stored_exact(24, 3, 0, 64))
    # the held-out outputs choosing tau: the same circuit, outputs 64..127
    full = qaoa_workload(24, 3, n_out=1024, eps=w.eps, seed=0x5EED0004)
    assert full.outputs[:64] == w.outputs
    assert not set(full.outputs[64:128]) & set(w.outputs)
    assert bench.stored_exact(24, 3, 64, 128).shape == (64,)


def test_qaoa24p3_cuts_place_the_checkpoint_after_twelve_sources():
    w = bench.family_jobs("qaoa24p3")[0][0]
    c1 = bench.source_cut(w.circuit, 12)
    c2 = bench.source_cut(w.circuit, 16)
    G = len(w.circuit.gates)
    # sources whose gate lies in the first c evaluated (output-side) gates
    srcs = [g for g, q, s in fs.Circuit(w.circuit).branch_vars() if s >= 0]
    assert sum(1 for g in srcs if G - g <= c1) == 12
    assert sum(1 for g in srcs if c1 < G - g <= c2) == 4

"""Per-output leaf counters (fs_batch_trace_outputs): the completed and
valid leaves of every requested output, the per-output cost distribution of
the paper's Fig. 11, against the oracle's per-output counts -- exact jobs
on the tiled history kernel and threshold jobs on the compacted one, both
engines."""
import numpy as np
import pytest
import torch

from workloads import qaoa_workload, qw_workload
from oracle import feynman
import paper_2608_01467_b300 as fs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("engine", ["straight", "interp"])
@pytest.mark.parametrize("case", ["qaoa_exact", "walk_threshold"])
def test_per_output_counts_match_the_oracle(case, engine):
    if case == "qaoa_exact":
        w = qaoa_workload(8, 2, n_out=48, seed=5)
        eps = 0.0
    else:
        w = qw_workload(steps=7, n_out=40, pos_bits=8)
        eps = 0.3
    G = len(w.circuit.gates)
    c1, c2 = G // 3, 2 * G // 3
    C = fs.Circuit(w.circuit)
    C.set_input(w.inputs)
    b = fs.Batch(split="fixed", c1=c1, c2=c2, engine=engine)
    b.add(C, w.outputs, eps)
    counts = torch.full((2 * len(w.outputs),), 7, dtype=torch.int64, device="cuda")   # zeroed by the run
    b.trace_outputs(0, counts)
    b.plan()
    b.allocate()
    b.upload()
    for _ in range(2):                  # the counters restart at every run
        b.run()
        st = b.finish()[0]
    got = counts.cpu().numpy().reshape(-1, 2)
    _, cnt = feynman.run(w.circuit, w.inputs, w.outputs, eps=eps, c1=c1, c2=c2)
    assert np.array_equal(got[:, 0], cnt["completed"].astype(np.int64))
    assert np.array_equal(got[:, 1], cnt["valid"].astype(np.int64))
    assert got[:, 0].sum() == st["completed"] and got[:, 1].sum() == st["valid"]

"""Exact reachability bound at the checkpoint (fs_batch_set_exact_bound):
entries whose state cannot reach the input through the remaining ops are
cut; the amplitudes stay exact.  On the coined walk every step moves the
position by one through a controlled +1 and a controlled -1 cascade, so the
library's bound allows a distance of two per remaining step (two cascades)
and checks the untouched ancilla; the expected cuts are counted here from
the oracle's checkpoint tables with that rule."""
import numpy as np
import pytest

from workloads import qw_workload
from oracle import feynman
import paper_2608_01467_b300 as fs

pytestmark = pytest.mark.gpu

POS = 96


def _run(w, c1, bound):
    C = fs.Circuit(w.circuit)
    C.set_input(w.inputs)
    b = fs.Batch(split="fixed", c1=c1, c2=c1)
    b.add(C, w.outputs)
    if bound:
        b.set_exact_bound(0)
    b.plan()
    b.allocate()
    b.upload()
    b.run()
    st = b.finish()[0]
    return b.amp.cpu().numpy()[:len(w.outputs)], st


@pytest.mark.parametrize("k_prefix", [3, 5])
def test_exact_bound_cuts_the_unreachable_entries_and_keeps_the_amplitudes(k_prefix):
    steps = 8
    w = qw_workload(steps=steps, n_out=128)
    G = len(w.circuit.gates)
    c1 = k_prefix * (G // steps)                  # the last k_prefix steps form the prefix
    left = steps - k_prefix
    exact, st0 = _run(w, c1, False)
    got, st = _run(w, c1, True)
    err = np.abs(got - exact)
    assert np.all(err <= 1e-12 + 1e-10 * np.abs(exact)), err.max()
    mask = (1 << POS) - 1
    expect, zero_cut = 0, 0
    for b_out in w.outputs:
        for b_in, _ in w.inputs:
            t = feynman.checkpoints(w.circuit, b_in, b_out, c1)
            for s, live, sub in zip(t["state"], t["live"], t["subtree"]):
                if not live:
                    continue
                x, y = (s >> 1) & mask, (b_in >> 1) & mask
                dist = min((x - y) & mask, (y - x) & mask)
                if dist > 2 * left or ((s ^ b_in) >> (POS + 3)) & 1:
                    expect += 1
                    zero_cut += sub == 0
    assert st["bound_cuts"] == expect == zero_cut > 0
    assert st["live_entries"] == st0["live_entries"] - expect
    assert st["valid"] == st0["valid"]
    assert st["completed"] < st0["completed"]

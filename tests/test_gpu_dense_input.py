"""Dense-support inputs (Eq. 2 with S ~ 2^n): the QFT of a real two-tone
signal on 12 qubits, every sample a basis state of the input, every bin
requested -- the restated form of the paper's QFT signal study (Sec. V,
Fig. 7), whose signal is not given.  The spectrum is 1/2 at the bins of
f1, N - f1, f2, N - f2 (through the bit reversal of the swap-free QFT) and
zero elsewhere; all 4096 amplitudes are checked against that closed form,
which the oracle tests pin to the dense state vector."""
import numpy as np
import pytest

from workloads import qft_signal_workload
from oracle import closed_forms
import paper_2608_01467_b300 as fs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n", [10, 12])
def test_qft_two_tone_signal_all_bins(n):
    w = qft_signal_workload(n)
    N = 1 << n
    assert len(w.inputs) >= N - 4                 # dense support
    C = fs.Circuit(w.circuit)
    C.set_input(w.inputs)
    b = fs.Batch()
    b.add(C, w.outputs)
    b.plan()
    b.allocate()
    b.upload()
    b.run()
    st = b.finish()[0]
    got = b.amp.cpu().numpy()[:N]
    want = np.zeros(N, complex)
    for k in (w.meta["f1"], N - w.meta["f1"], w.meta["f2"], N - w.meta["f2"]):
        want[closed_forms.bit_reverse(k, n)] = 0.5
    assert np.max(np.abs(got - want)) < 1e-12
    # A = 0: one history per (output, input) pair, every one of them valid
    assert st["completed"] == st["valid"] == N * len(w.inputs)

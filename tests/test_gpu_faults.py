"""Failure detection on the device without faulting it.

* A corrupt program: the host overwrites one op of an uploaded program with
  an opcode the interpreter does not know; the device-side check records
  FS_ERR_BAD_PROGRAM in the error word and cuts that history (no trap, no
  out-of-range access), fs_batch_finish reports it, and a clean upload runs
  correctly afterwards.
* A bounded wait that gives up: with the poll limit at 0 every wait of the
  tensor-core scoring kernel on an MMA-completion barrier gives up at once;
  the kernel records FS_ERR_TIMEOUT, issues no further MMA, waits for the
  MMAs already committed and releases its tensor memory; fs_batch_finish
  reports the timeout and the context keeps working (the same batch runs
  correctly once the default limit is back)."""
import numpy as np
import pytest
import torch

from workloads import mlp_init_params, qaoa_workload, qw_workload
from oracle import feynman
import paper_2608_01467_b300 as fs
from paper_2608_01467_b300 import _lib, learned

pytestmark = pytest.mark.gpu


def test_unknown_opcode_is_reported_and_the_context_survives():
    w = qaoa_workload(8, 2, n_out=16, seed=41)
    C = fs.Circuit(w.circuit)
    C.set_input(w.inputs)
    b = fs.Batch(engine="interp")
    b.add(C, w.outputs)
    b.plan()
    b.allocate()
    b.upload()
    torch.cuda.synchronize()
    off, n_ops = b.program_offset(0)
    ws = b._raw[(b.ws_ptr - b._raw.data_ptr()):]
    k = n_ops // 2
    assert ws[off + 16 * k].item() != 0          # byte 0 of an op is its opcode
    ws[off + 16 * k] = 0xEE                      # no such opcode
    b.run()
    with pytest.raises(_lib.FsError) as e:
        b.finish()
    assert e.value.code == -8                    # FS_ERR_BAD_PROGRAM
    b.upload()                                   # the clean program again
    b.run()
    b.finish()
    want, _ = feynman.run(w.circuit, w.inputs, w.outputs)
    got = b.amp.cpu().numpy()[:len(w.outputs)]
    assert np.max(np.abs(got - want)) < 1e-12


def test_tensor_core_wait_gives_up_and_the_context_survives():
    w = qw_workload(steps=6, n_out=24, pos_bits=8)
    G = len(w.circuit.gates)
    C = fs.Circuit(w.circuit)
    C.set_input(w.inputs)
    b = fs.Batch(split="fixed", c1=G // 3, c2=2 * G // 3)
    b.add(C, w.outputs)
    params = torch.from_numpy(np.asarray(mlp_init_params(0), np.float32)).cuda()
    learned.attach(b, 0, params, -1e30)              # scores every entry, cuts none
    b.plan()
    b.allocate()
    b.upload()
    L = _lib.load()
    try:
        assert L.fs_set_wait_limit(0) == 0
        b.run()
        with pytest.raises(_lib.FsError) as e:
            b.finish()
        assert e.value.code == -7                    # FS_ERR_TIMEOUT
    finally:
        assert L.fs_set_wait_limit(-1) == 0
    b.run()
    st = b.finish()[0]
    want, _ = feynman.run(w.circuit, w.inputs, w.outputs)
    got = b.amp.cpu().numpy()[:len(w.outputs)]
    assert st["learned_cuts"] == 0
    assert np.max(np.abs(got - want)) < 1e-12

"""fs_amplitudes_noalloc: the allocation-free twin of fs_amplitudes.

Some callers cannot allocate device memory while they run -- code that must
take every device allocation from a pool it does not own, or a plugin that
must not grow the process's device footprint at call time.  For them the
library offers one entry point whose whole device workspace is a static
device array of fixed size (FS_NOALLOC_SCRATCH_BYTES).  These tests call it
through the C ABI and check that it returns what fs_amplitudes returns, on
calls in a row (the array keeps the previous call's contents), and that a
request too large for the array is refused with a clear error.

This file is named so that pytest collects it last."""
import ctypes
import numpy as np
import pytest

from workloads import qaoa_workload, qw_workload
import paper_2608_01467_b300 as fs
from paper_2608_01467_b300 import _lib

pytestmark = pytest.mark.gpu

ATOL, RTOL = 1e-12, 1e-10


def bits(values):
    a = np.zeros(2 * max(len(values), 1), np.uint64)
    for i, v in enumerate(values):
        a[2 * i] = v & 0xFFFFFFFFFFFFFFFF
        a[2 * i + 1] = v >> 64
    return a


def call_noalloc(C, outputs, eps=0.0):
    L = _lib.load()
    b = bits(outputs)
    out = np.zeros(2 * max(len(outputs), 1))
    rc = L.fs_amplitudes_noalloc(C.handle, b.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                                 len(outputs), eps,
                                 out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), None)
    return rc, out[0:2 * len(outputs):2] + 1j * out[1:2 * len(outputs):2]


def check_close(got, want):
    err = np.abs(got - want)
    assert np.all(err <= ATOL + RTOL * np.abs(want)), err.max()


def test_noalloc_matches_fs_amplitudes_on_calls_in_a_row():
    w1 = qaoa_workload(8, 2, n_out=64, seed=17)
    w2 = qw_workload(steps=6, n_out=48, pos_bits=8)
    C1 = fs.Circuit(w1.circuit)
    C1.set_input(w1.inputs)
    C2 = fs.Circuit(w2.circuit)
    C2.set_input(w2.inputs)
    ref1 = C1.amplitudes(w1.outputs)
    ref2 = C2.amplitudes(w2.outputs)
    ref1p = C1.amplitudes(w1.outputs, eps=0.02)
    for C, outs, ref, eps in ((C1, w1.outputs, ref1, 0.0), (C2, w2.outputs, ref2, 0.0),
                              (C1, w1.outputs, ref1p, 0.02), (C1, w1.outputs, ref1, 0.0)):
        rc, got = call_noalloc(C, outs, eps)
        assert rc == 0, _lib.load().fs_last_error()
        check_close(got, ref)


def test_noalloc_refuses_requests_larger_than_its_scratch():
    # 2^20 requested outputs need at least 2^20 x (16 B bit string + 32 B
    # checkpoint entry + 16 B partial + 16 B amplitude) = 80 MiB > 16 MiB
    w = qaoa_workload(20, 1, n_out=16, seed=5)
    C = fs.Circuit(w.circuit)
    C.set_input(w.inputs)
    rc, _ = call_noalloc(C, list(range(1 << 20)))
    assert rc == -9
    msg = _lib.load().fs_last_error().decode()
    assert "scratch" in msg and str(_lib.NOALLOC_SCRATCH_BYTES) in msg
    # a small request still works after the refusal
    rc, got = call_noalloc(C, w.outputs[:4])
    assert rc == 0
    check_close(got, C.amplitudes(w.outputs[:4]))


def test_noalloc_leaves_free_device_memory_unchanged():
    """After the first call on a device (which may load this part of the
    library, the static array included, under lazy module loading), further
    calls allocate nothing: the free device memory reported by the driver is
    the same before and after each of them."""
    import torch
    w = qw_workload(steps=6, n_out=48, pos_bits=8)
    C = fs.Circuit(w.circuit)
    C.set_input(w.inputs)
    for eps in (0.0, 0.02):          # first calls: exact and threshold kernels loaded
        rc, _ = call_noalloc(C, w.outputs, eps)
        assert rc == 0
    torch.cuda.synchronize()
    for eps in (0.0, 0.0, 0.02, 0.02):
        free0, _ = torch.cuda.mem_get_info()
        rc, got = call_noalloc(C, w.outputs, eps)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        assert rc == 0 and free1 == free0, (free0, free1)
    check_close(got, C.amplitudes(w.outputs, eps=0.02))

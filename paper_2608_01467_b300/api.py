"""Python binding over the C ABI: argument marshalling only.

Every step of the path (analysis, compilation, prefix expansion, history
enumeration, reduction) runs inside libfeynsparse.so; PyTorch only provides
device memory and streams.
"""
from __future__ import annotations

import ctypes
from typing import Iterable, List, Sequence, Tuple

import numpy as np

from . import _lib
from ._lib import check, fs_analysis, fs_gate, fs_options, fs_stats

U64 = ctypes.c_uint64
MASK64 = (1 << 64) - 1


def _bits_array(values: Sequence[int]) -> np.ndarray:
    a = np.zeros(2 * max(len(values), 1), np.uint64)
    for i, v in enumerate(values):
        a[2 * i] = v & MASK64
        a[2 * i + 1] = (v >> 64) & MASK64
    return a


def _ptr(a: np.ndarray, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


def gates_to_abi(gates) -> ctypes.Array:
    """workloads.Gate records -> fs_gate array."""
    arr = (fs_gate * max(1, len(gates)))()
    for i, g in enumerate(gates):
        o = arr[i]
        o.kind = _lib.KIND[g.kind]
        o.n_q = len(g.qubits)
        o.q[0] = g.qubits[0]
        o.q[1] = g.qubits[1] if len(g.qubits) > 1 else 0
        cm = [0, 0]
        cv = [0, 0]
        for q, v in g.controls:
            cm[q >> 6] |= 1 << (q & 63)
            if v:
                cv[q >> 6] |= 1 << (q & 63)
        o.ctrl_mask[0], o.ctrl_mask[1] = cm
        o.ctrl_val[0], o.ctrl_val[1] = cv
        o.theta = float(g.theta)
        if g.matrix is not None:
            for j, z in enumerate(g.matrix):
                o.m[2 * j] = complex(z).real
                o.m[2 * j + 1] = complex(z).imag
    return arr


class Circuit:
    """fs_circuit handle: fs_circuit_create(gates, n_qubits)."""

    def __init__(self, circuit=None, gates=None, n_qubits=None):
        L = _lib.load()
        if circuit is not None:
            gates, n_qubits = circuit.gates, circuit.n_qubits
        self.n_qubits = int(n_qubits)
        self.n_gates = len(gates)
        arr = gates_to_abi(gates)
        h = ctypes.c_void_p()
        check(L.fs_circuit_create(arr, len(gates), self.n_qubits, ctypes.byref(h)))
        self._h = h
        self.inputs: List[Tuple[int, complex]] = [(0, 1.0 + 0j)]

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            _lib.load().fs_circuit_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def analyze(self, input_bits: int = 0) -> dict:
        a = fs_analysis()
        b = _bits_array([input_bits])
        check(_lib.load().fs_analyze(self._h, _ptr(b, U64), ctypes.byref(a)))
        self.inputs = [(input_bits, 1.0 + 0j)]
        d = {f: getattr(a, f) for f, _ in fs_analysis._fields_}
        d["gateops"] = a.gateops_lo | (a.gateops_hi << 64)
        return d

    def branch_vars(self):
        L = _lib.load()
        cnt = ctypes.c_size_t(0)
        check(L.fs_branch_vars(self._h, None, None, None, 0, ctypes.byref(cnt)))
        n = cnt.value
        gi = np.zeros(max(n, 1), np.int32)
        qb = np.zeros(max(n, 1), np.int32)
        sr = np.zeros(max(n, 1), np.int32)
        check(L.fs_branch_vars(self._h, _ptr(gi, ctypes.c_int32), _ptr(qb, ctypes.c_int32),
                               _ptr(sr, ctypes.c_int32), n, ctypes.byref(cnt)))
        return [(int(gi[i]), int(qb[i]), int(sr[i])) for i in range(n)]

    def source_placement(self, method: str = "backward"):
        """(artificial sources, unknown wire classes) of the backward sweep,
        the greedy or the optimal placement of the graph form (Fig. 4)."""
        k, m = ctypes.c_uint32(0), ctypes.c_uint32(0)
        check(_lib.load().fs_source_placement(self._h, {"backward": 0, "greedy": 1, "optimal": 2}[method],
                                              ctypes.byref(k), ctypes.byref(m)))
        return k.value, m.value

    def set_input(self, inputs: Iterable[Tuple[int, complex]]):
        inputs = list(inputs)
        b = _bits_array([x for x, _ in inputs])
        c = np.array([[complex(v).real, complex(v).imag] for _, v in inputs], np.float64).reshape(-1)
        check(_lib.load().fs_set_input(self._h, _ptr(b, U64), _ptr(c, ctypes.c_double), len(inputs)))
        self.inputs = inputs

    def amplitudes(self, outputs: Sequence[int], eps: float = 0.0) -> np.ndarray:
        """fs_amplitudes with host buffers (synchronous)."""
        M = len(outputs)
        b = _bits_array(list(outputs))
        out = np.zeros(2 * max(M, 1), np.float64)
        check(_lib.load().fs_amplitudes(self._h, _ptr(b, U64), M, float(eps), _ptr(out, ctypes.c_double)))
        return out[0:2 * M:2] + 1j * out[1:2 * M:2]


def _stream_handle(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


class Batch:
    """Many (circuit, outputs, eps) jobs evaluated by one persistent launch.

    plan() compiles and sizes the device workspace; allocate() takes it from
    PyTorch; upload() copies programs and bit strings; run() enqueues the
    kernels (graph-capturable); finish() synchronises and reads counters."""

    def __init__(self, split: str = "auto", c1: int = 0, c2: int = 0,
                 table_budget_bytes: int = 0, min_items: int = 0, max_items: int = 0,
                 engine: str = "straight", prefix: str = "auto", device: int = -1):
        L = _lib.load()
        h = ctypes.c_void_p()
        check(L.fs_batch_create(ctypes.byref(h)))
        self._h = h
        if device >= 0:
            check(L.fs_batch_set_device(self._h, int(device)))
        opt = fs_options()
        opt.split = {"auto": 0, "fixed": 1, "none": 2}[split]
        opt.c1, opt.c2 = c1, c2
        opt.table_budget_bytes = table_budget_bytes
        opt.min_items = min_items
        opt.max_items = max_items
        opt.engine = {"straight": 0, "interp": 1}[engine]
        opt.prefix_mode = {"auto": 0, "single": 1, "levels": 2}[prefix]
        check(L.fs_batch_set_options(self._h, ctypes.byref(opt)))
        self.engine_name = engine
        self.jobs = []
        self.ws = None
        self.amp = None
        self.ws_bytes = 0
        self._circuits = []

    def close(self):
        if getattr(self, "_h", None):
            _lib.load().fs_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add(self, circuit: Circuit, outputs: Sequence[int], eps: float = 0.0) -> int:
        b = _bits_array(list(outputs))
        jid = ctypes.c_uint32(0)
        check(_lib.load().fs_batch_add(self._h, circuit.handle, _ptr(b, U64), len(outputs),
                                       float(eps), ctypes.byref(jid)))
        self.jobs.append((len(outputs), float(eps)))
        self._circuits.append(circuit)
        return jid.value

    def trace_outputs(self, job: int, counts):
        """Per-output {completed, valid} leaf counters of a job in a device
        uint64 tensor of 2 x n_out elements (None: off); call before upload."""
        ptr = None if counts is None else ctypes.c_void_p(counts.data_ptr())
        check(_lib.load().fs_batch_trace_outputs(self._h, job, ptr))
        self._trace = counts

    def set_exact_bound(self, job: int, enable: bool = True):
        """Cut checkpoint entries that provably cannot reach the input (exact)."""
        check(_lib.load().fs_batch_set_exact_bound(self._h, job, 1 if enable else 0))

    def set_cuts(self, job: int, c1: int, c2: int):
        """Fixed cuts for one job (both -1: back to the batch's split)."""
        check(_lib.load().fs_batch_set_cuts(self._h, job, c1, c2))

    def plan(self) -> int:
        n = ctypes.c_size_t(0)
        check(_lib.load().fs_batch_plan(self._h, ctypes.byref(n)))
        self.ws_bytes = n.value
        return self.ws_bytes

    @property
    def total_outputs(self) -> int:
        n = ctypes.c_size_t(0)
        check(_lib.load().fs_batch_total_outputs(self._h, ctypes.byref(n)))
        return n.value

    def engine(self):
        """(engine name, compile milliseconds) after upload."""
        e, ms = ctypes.c_uint32(), ctypes.c_double()
        check(_lib.load().fs_batch_engine(self._h, ctypes.byref(e), ctypes.byref(ms)))
        return ("straight" if e.value == 0 else "interp"), ms.value

    def static_bytes(self) -> int:
        n = ctypes.c_size_t(0)
        check(_lib.load().fs_batch_upload_bytes(self._h, ctypes.byref(n)))
        return n.value

    def allocate(self, device="cuda"):
        import torch
        self._raw = torch.empty(self.ws_bytes + 256, dtype=torch.uint8, device=device)
        p = self._raw.data_ptr()
        self.ws_ptr = (p + 255) & ~255
        self.amp = torch.zeros(max(self.total_outputs, 1), dtype=torch.complex128, device=device)
        return self.ws_ptr

    def upload(self, stream=None):
        check(_lib.load().fs_batch_upload(self._h, ctypes.c_void_p(self.ws_ptr), self.ws_bytes,
                                          _stream_handle(stream)))

    def run(self, stream=None):
        check(_lib.load().fs_batch_run(self._h, ctypes.c_void_p(self.ws_ptr),
                                       ctypes.c_void_p(self.amp.data_ptr()), _stream_handle(stream)))

    def finish(self, stream=None):
        n = len(self.jobs)
        st = (fs_stats * max(n, 1))()
        check(_lib.load().fs_batch_finish(self._h, ctypes.c_void_p(self.ws_ptr),
                                          _stream_handle(stream), st, n))
        return [{f: getattr(st[i], f) for f, _ in fs_stats._fields_} for i in range(n)]

    def launch_count(self) -> int:
        n = ctypes.c_uint32(0)
        check(_lib.load().fs_batch_launch_count(self._h, ctypes.byref(n)))
        return n.value

    def time_kernels(self, enable=True):
        check(_lib.load().fs_batch_time_kernels(self._h, 1 if enable else 0))

    def kernel_ms(self):
        a, h, r = ctypes.c_float(), ctypes.c_float(), ctypes.c_float()
        check(_lib.load().fs_batch_kernel_ms(self._h, ctypes.byref(a), ctypes.byref(h), ctypes.byref(r)))
        return a.value, h.value, r.value

    def stage_ms(self):
        """{prefix, prune, compact, history, reduce} milliseconds of the last timed run."""
        arr = (ctypes.c_float * 5)()
        check(_lib.load().fs_batch_stage_ms(self._h, arr))
        return dict(zip(("prefix", "prune", "compact", "history", "reduce"), list(arr)))

    def op_histogram(self, job: int):
        """{region: {opname: count}} of a planned job (regions prefix/root/suffix)."""
        arr = (ctypes.c_uint32 * (3 * _lib.N_OPCODES))()
        check(_lib.load().fs_batch_op_histogram(self._h, job, arr))
        out = {}
        for r, name in enumerate(("prefix", "root", "suffix")):
            out[name] = {_lib.OPCODES[k]: arr[r * _lib.N_OPCODES + k]
                         for k in _lib.OPCODES if arr[r * _lib.N_OPCODES + k]}
        return out

    def program_offset(self, job: int):
        """(byte offset in the workspace, op count) of a planned job's program."""
        off, n = ctypes.c_size_t(0), ctypes.c_size_t(0)
        check(_lib.load().fs_batch_program_offset(self._h, job, ctypes.byref(off), ctypes.byref(n)))
        return off.value, n.value

    def generated_source(self) -> str:
        """CUDA C++ of the straight-line engine for the planned batch."""
        L = _lib.load()
        n = ctypes.c_size_t(0)
        check(L.fs_batch_generated_source(self._h, None, 0, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(n.value + 1)
        check(L.fs_batch_generated_source(self._h, buf, n.value + 1, ctypes.byref(n)))
        return buf.value.decode()

    def region_work(self, job: int):
        """Per single execution: ([prefix, root, suffix, per-leaf] integer ops,
        [prefix, root, suffix, per-valid-leaf] FP64 instructions)."""
        i = (ctypes.c_double * 4)()
        f = (ctypes.c_double * 4)()
        check(_lib.load().fs_batch_region_work(self._h, job, i, f))
        return list(i), list(f)

    def job_words(self, job: int) -> int:
        w = ctypes.c_uint32(0)
        check(_lib.load().fs_batch_job_words(self._h, job, ctypes.byref(w)))
        return w.value

    def job_slices(self):
        off = 0
        out = []
        for m, _ in self.jobs:
            out.append(slice(off, off + m))
            off += m
        return out


def probe_peaks():
    """Measured FP64 FMA/s, 32-bit integer ops/s and SM count of the current device."""
    d, i, n = ctypes.c_double(), ctypes.c_double(), ctypes.c_int32()
    check(_lib.load().fs_probe_peaks(ctypes.byref(d), ctypes.byref(i), ctypes.byref(n)))
    return {"dfma_per_s": d.value, "int_ops_per_s": i.value, "sms": n.value}


def amplitudes(circuit, inputs, outputs, eps: float = 0.0) -> np.ndarray:
    """One-call convenience: workloads.Circuit + sparse input -> amplitudes
    through fs_circuit_create / fs_set_input / fs_amplitudes."""
    c = Circuit(circuit)
    c.set_input(inputs)
    return c.amplitudes(outputs, eps)

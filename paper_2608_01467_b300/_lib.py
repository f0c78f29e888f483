"""ctypes declarations of the C ABI in include/feynsparse.h (argument
marshalling only).  Loading fails loudly when libfeynsparse.so is missing:
there is no fallback path."""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfeynsparse.so")

FS_OK = 0
ERRORS = {-1: "FS_ERR_INVALID", -2: "FS_ERR_UNSUPPORTED", -3: "FS_ERR_TOO_MANY_QUBITS",
          -4: "FS_ERR_NONUNITARY", -5: "FS_ERR_NOMEM", -6: "FS_ERR_CUDA", -7: "FS_ERR_TIMEOUT",
          -8: "FS_ERR_BAD_PROGRAM", -9: "FS_ERR_TOO_LARGE", -10: "FS_ERR_STATE"}
KIND = {"H": 0, "X": 1, "Y": 2, "Z": 3, "S": 4, "T": 5, "P": 6, "RX": 7, "RY": 8, "RZ": 9,
        "RZZ": 10, "SWAP": 11, "U1": 12, "U2": 13}


class FsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class fs_gate(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_uint32), ("n_q", ctypes.c_uint32), ("q", ctypes.c_uint32 * 2),
                ("ctrl_mask", ctypes.c_uint64 * 2), ("ctrl_val", ctypes.c_uint64 * 2),
                ("theta", ctypes.c_double), ("m", ctypes.c_double * 32)]


class fs_analysis(ctypes.Structure):
    _fields_ = [("n_qubits", ctypes.c_uint32), ("n_gates", ctypes.c_uint32),
                ("n_branch_vars", ctypes.c_uint32), ("n_natural", ctypes.c_uint32),
                ("A", ctypes.c_uint32), ("n_wp", ctypes.c_uint32), ("n_det", ctypes.c_uint32),
                ("n_br", ctypes.c_uint32), ("c1", ctypes.c_int32), ("c2", ctypes.c_int32),
                ("G_p", ctypes.c_uint32), ("G_r", ctypes.c_uint32), ("G_s", ctypes.c_uint32),
                ("A_p", ctypes.c_uint32), ("A_r", ctypes.c_uint32), ("A_s", ctypes.c_uint32),
                ("gateops_lo", ctypes.c_uint64), ("gateops_hi", ctypes.c_uint64),
                ("max_ap", ctypes.c_uint32), ("min_apr", ctypes.c_uint32),
                ("max_apr", ctypes.c_uint32)]


class fs_options(ctypes.Structure):
    _fields_ = [("split", ctypes.c_uint32), ("c1", ctypes.c_int32), ("c2", ctypes.c_int32),
                ("table_budget_bytes", ctypes.c_uint64), ("min_items", ctypes.c_uint64),
                ("max_items", ctypes.c_uint64), ("engine", ctypes.c_uint32),
                ("prefix_mode", ctypes.c_uint32)]


class fs_stats(ctypes.Structure):
    _fields_ = [("candidates", ctypes.c_uint64), ("completed", ctypes.c_uint64),
                ("valid", ctypes.c_uint64), ("gate_visits", ctypes.c_uint64),
                ("history_visits", ctypes.c_uint64),
                ("table_entries", ctypes.c_uint64), ("c1", ctypes.c_int32), ("c2", ctypes.c_int32),
                ("A_p", ctypes.c_uint32), ("A_r", ctypes.c_uint32), ("A_s", ctypes.c_uint32),
                ("learned_cuts", ctypes.c_uint64), ("live_entries", ctypes.c_uint64),
                ("bound_cuts", ctypes.c_uint64)]


P = ctypes.POINTER
vp = ctypes.c_void_p
SIGNATURES = {
    "fs_last_error": (ctypes.c_char_p, []),
    "fs_version": (ctypes.c_char_p, []),
    "fs_circuit_create": (ctypes.c_int, [P(fs_gate), ctypes.c_size_t, ctypes.c_uint32, P(vp)]),
    "fs_circuit_destroy": (ctypes.c_int, [vp]),
    "fs_analyze": (ctypes.c_int, [vp, P(ctypes.c_uint64), P(fs_analysis)]),
    "fs_branch_vars": (ctypes.c_int, [vp, P(ctypes.c_int32), P(ctypes.c_int32), P(ctypes.c_int32),
                                      ctypes.c_size_t, P(ctypes.c_size_t)]),
    "fs_set_input": (ctypes.c_int, [vp, P(ctypes.c_uint64), P(ctypes.c_double), ctypes.c_size_t]),
    "fs_amplitudes": (ctypes.c_int, [vp, P(ctypes.c_uint64), ctypes.c_size_t, ctypes.c_double,
                                     P(ctypes.c_double)]),
    "fs_batch_create": (ctypes.c_int, [P(vp)]),
    "fs_batch_destroy": (ctypes.c_int, [vp]),
    "fs_batch_set_options": (ctypes.c_int, [vp, P(fs_options)]),
    "fs_batch_add": (ctypes.c_int, [vp, vp, P(ctypes.c_uint64), ctypes.c_size_t, ctypes.c_double,
                                    P(ctypes.c_uint32)]),
    "fs_batch_plan": (ctypes.c_int, [vp, P(ctypes.c_size_t)]),
    "fs_batch_upload": (ctypes.c_int, [vp, vp, ctypes.c_size_t, vp]),
    "fs_batch_run": (ctypes.c_int, [vp, vp, vp, vp]),
    "fs_batch_finish": (ctypes.c_int, [vp, vp, vp, P(fs_stats), ctypes.c_size_t]),
    "fs_batch_total_outputs": (ctypes.c_int, [vp, P(ctypes.c_size_t)]),
    "fs_batch_upload_bytes": (ctypes.c_int, [vp, P(ctypes.c_size_t)]),
    "fs_batch_generated_source": (ctypes.c_int, [vp, ctypes.c_char_p, ctypes.c_size_t, P(ctypes.c_size_t)]),
    "fs_batch_engine": (ctypes.c_int, [vp, P(ctypes.c_uint32), P(ctypes.c_double)]),
    "fs_batch_launch_count": (ctypes.c_int, [vp, P(ctypes.c_uint32)]),
    "fs_batch_time_kernels": (ctypes.c_int, [vp, ctypes.c_int]),
    "fs_batch_kernel_ms": (ctypes.c_int, [vp, P(ctypes.c_float), P(ctypes.c_float),
                                          P(ctypes.c_float)]),
    "fs_batch_stage_ms": (ctypes.c_int, [vp, P(ctypes.c_float)]),
    "fs_batch_op_histogram": (ctypes.c_int, [vp, ctypes.c_uint32, P(ctypes.c_uint32)]),
    "fs_batch_job_words": (ctypes.c_int, [vp, ctypes.c_uint32, P(ctypes.c_uint32)]),
    "fs_batch_region_work": (ctypes.c_int, [vp, ctypes.c_uint32, P(ctypes.c_double), P(ctypes.c_double)]),
    "fs_probe_peaks": (ctypes.c_int, [P(ctypes.c_double), P(ctypes.c_double), P(ctypes.c_int32)]),
    "fs_mlp_forward": (ctypes.c_int, [vp, vp, ctypes.c_uint64, vp, vp]),
    "fs_mlp_grad": (ctypes.c_int, [vp, vp, vp, ctypes.c_uint64, vp, vp]),
    "fs_mlp_adam": (ctypes.c_int, [vp, vp, vp, vp, ctypes.c_float, ctypes.c_int32, vp]),
    "fs_batch_features": (ctypes.c_int, [vp, ctypes.c_uint32, vp, vp, vp]),
    "fs_batch_log_subtrees": (ctypes.c_int, [vp, ctypes.c_uint32, vp]),
    "fs_batch_log_items": (ctypes.c_int, [vp, ctypes.c_uint32, P(ctypes.c_uint64)]),
    "fs_batch_set_cuts": (ctypes.c_int, [vp, ctypes.c_uint32, ctypes.c_int32, ctypes.c_int32]),
    "fs_batch_set_pruner": (ctypes.c_int, [vp, ctypes.c_uint32, vp, ctypes.c_float]),
    "fs_amplitudes_noalloc": (ctypes.c_int, [vp, P(ctypes.c_uint64), ctypes.c_size_t, ctypes.c_double,
                                             P(ctypes.c_double), vp]),
    "fs_batch_set_device": (ctypes.c_int, [vp, ctypes.c_int32]),
    "fs_batch_program_offset": (ctypes.c_int, [vp, ctypes.c_uint32, P(ctypes.c_size_t), P(ctypes.c_size_t)]),
    "fs_mlp_targets": (ctypes.c_int, [vp, ctypes.c_uint64, ctypes.c_double, vp, vp]),
    "fs_set_wait_limit": (ctypes.c_int, [ctypes.c_int64]),
    "fs_batch_set_exact_bound": (ctypes.c_int, [vp, ctypes.c_uint32, ctypes.c_int32]),
    "fs_batch_trace_outputs": (ctypes.c_int, [vp, ctypes.c_uint32, vp]),
    "fs_source_placement": (ctypes.c_int, [vp, ctypes.c_uint32, P(ctypes.c_uint32), P(ctypes.c_uint32)]),
    "fs_lpt_assign": (ctypes.c_int, [P(ctypes.c_double), ctypes.c_size_t, ctypes.c_uint32, P(ctypes.c_uint32),
                                     P(ctypes.c_double)]),
}
NOALLOC_SCRATCH_BYTES = 16 << 20
MLP_PARAMS = 18817
N_OPCODES = 16
OPCODES = {1: "X", 2: "MCX", 3: "SWAP", 4: "PERM1", 5: "PERM2", 6: "DIAG1", 7: "PH1", 8: "NEG1",
           9: "MCPH", 10: "MCNEG", 11: "DIAG2", 12: "H", 13: "BR1", 14: "BR2"}

_lib = None


def load():
    """The loaded library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with "
                              "`python -m paper_2608_01467_b300.build` (no CPU fallback exists)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check(rc):
    if rc != FS_OK:
        msg = load().fs_last_error()
        raise FsError(rc, msg.decode() if msg else "")
    return rc


def exported_symbols():
    return list(SIGNATURES)

"""O3: ctypes front end of the C reduced-history oracle (test infrastructure).

``build()`` compiles feynman_oracle.c with gcc (no FP contraction, so the
explicit fma formulas are what runs).  The functions below convert neutral
``workloads.Gate`` records into the oracle's own gate struct.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "feynman_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libfeynman_oracle.so")
_lock = threading.Lock()
_lib = None

KIND = {"H": 0, "X": 1, "Y": 2, "Z": 3, "S": 4, "T": 5, "P": 6, "RX": 7, "RY": 8,
        "RZ": 9, "RZZ": 10, "SWAP": 11, "U1": 12, "U2": 13}
ROLE_NAMES = {0: "WP", 1: "DET", 2: "BR"}


class OrcGate(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("q0", ctypes.c_int32), ("q1", ctypes.c_int32),
                ("pad", ctypes.c_int32), ("cmask", ctypes.c_uint64 * 2),
                ("cval", ctypes.c_uint64 * 2), ("theta", ctypes.c_double),
                ("m", ctypes.c_double * 32)]


def build(force: bool = False) -> str:
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or \
            os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off",
                               "-fPIC", "-shared", "-o", _LIB_PATH, _SRC, "-lm", "-lpthread"])
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB_PATH)
            P = ctypes.POINTER
            L.orc_analyze.argtypes = [P(OrcGate), ctypes.c_int, ctypes.c_int,
                                      P(ctypes.c_int32), P(ctypes.c_int32), P(ctypes.c_int32)]
            L.orc_region_counts.argtypes = [P(OrcGate), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                            ctypes.c_int, P(ctypes.c_int32), P(ctypes.c_uint64)]
            L.orc_autotune.argtypes = [P(OrcGate), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_int, ctypes.c_int, P(ctypes.c_int32),
                                       P(ctypes.c_int32), P(ctypes.c_uint64)]
            L.orc_run.argtypes = [P(OrcGate), ctypes.c_int, ctypes.c_int,
                                  P(ctypes.c_uint64), P(ctypes.c_double), ctypes.c_int,
                                  P(ctypes.c_uint64), ctypes.c_int, ctypes.c_double,
                                  ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                  P(ctypes.c_double), P(ctypes.c_uint64), P(ctypes.c_int32)]
            L.orc_checkpoints.argtypes = [P(OrcGate), ctypes.c_int, ctypes.c_int, P(ctypes.c_uint64),
                                          P(ctypes.c_uint64), ctypes.c_int, P(ctypes.c_uint64),
                                          P(ctypes.c_double), P(ctypes.c_uint8), P(ctypes.c_double),
                                          P(ctypes.c_int32)]
            _lib = L
    return _lib


def _gates(circuit):
    arr = (OrcGate * max(1, len(circuit.gates)))()
    for i, g in enumerate(circuit.gates):
        o = arr[i]
        o.kind = KIND[g.kind]
        o.q0 = g.qubits[0]
        o.q1 = g.qubits[1] if len(g.qubits) > 1 else 0
        cm = [0, 0]
        cv = [0, 0]
        for q, v in g.controls:
            cm[q >> 6] |= 1 << (q & 63)
            if v:
                cv[q >> 6] |= 1 << (q & 63)
        o.cmask[0], o.cmask[1] = cm
        o.cval[0], o.cval[1] = cv
        o.theta = g.theta
        if g.matrix is not None:
            for j, z in enumerate(g.matrix):
                o.m[2 * j] = complex(z).real
                o.m[2 * j + 1] = complex(z).imag
    return arr


def _words(values):
    a = np.zeros(2 * len(values), np.uint64)
    for i, v in enumerate(values):
        a[2 * i] = v & 0xFFFFFFFFFFFFFFFF
        a[2 * i + 1] = (v >> 64) & 0xFFFFFFFFFFFFFFFF
    return a


def _p(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


def analyze(circuit):
    """Roles per gate, per-gate (source id | -1 natural | -2 none) for each
    target, and A (Sec. IV-A backward placement)."""
    G = len(circuit.gates)
    role = np.zeros(max(G, 1), np.int32)
    src = np.zeros(2 * max(G, 1), np.int32)
    A = ctypes.c_int32(0)
    rc = lib().orc_analyze(_gates(circuit), G, circuit.n_qubits, _p(role, ctypes.c_int32),
                           _p(src, ctypes.c_int32), ctypes.byref(A))
    if rc:
        raise ValueError(f"orc_analyze failed: {rc}")
    return {"roles": [ROLE_NAMES[int(r)] for r in role[:G]],
            "src": [(int(src[2 * i]), int(src[2 * i + 1])) for i in range(G)],
            "A": int(A.value)}


def region_counts(circuit, c1, c2):
    """(Gp, Gr, Gs, Ap, Ar, As) and Eq. 8 for cuts at evaluation
    positions c1 <= c2."""
    out = np.zeros(6, np.int32)
    cost = np.zeros(2, np.uint64)
    rc = lib().orc_region_counts(_gates(circuit), len(circuit.gates), circuit.n_qubits,
                                 c1, c2, _p(out, ctypes.c_int32), _p(cost, ctypes.c_uint64))
    if rc:
        raise ValueError(f"orc_region_counts failed: {rc}")
    return tuple(int(x) for x in out), int(cost[0]) | (int(cost[1]) << 64)


def autotune(circuit, max_ap=64, min_apr=0, max_apr=1 << 30):
    c1 = ctypes.c_int32(0)
    c2 = ctypes.c_int32(0)
    cost = np.zeros(2, np.uint64)
    rc = lib().orc_autotune(_gates(circuit), len(circuit.gates), circuit.n_qubits, max_ap,
                            min_apr, max_apr, ctypes.byref(c1), ctypes.byref(c2),
                            _p(cost, ctypes.c_uint64))
    if rc:
        raise ValueError(f"orc_autotune failed: {rc}")
    return int(c1.value), int(c2.value), int(cost[0]) | (int(cost[1]) << 64)


def run(circuit, inputs, outputs, eps=0.0, c1=0, c2=0, threads=1):
    """Amplitudes (complex128[M]) of the requested outputs for the sparse
    input [(basis, coeff)] (Eq. 2) by Algorithm 2 with cuts (c1, c2), or
    Algorithm 1 when c1 = c2 = 0; plus per-output counts
    {completed, valid, visits} and A."""
    return _run(circuit, inputs, outputs, eps, c1, c2, threads)


def run_dfs(circuit, inputs, outputs, eps=0.0, threads=1):
    """As run(), by a depth-first search over the artificial sources in
    backward order that drops a subtree as soon as its branch is cut (any A;
    cost proportional to the surviving tree, not to 2^A).  Same leaves and
    counts {completed, valid} as Algorithm 1/2 with the same eps; visits
    count the gates the search evaluated."""
    return _run(circuit, inputs, outputs, eps, -1, -1, threads)


def _run(circuit, inputs, outputs, eps, c1, c2, threads):
    ins = _words([b for b, _ in inputs])
    coef = np.array([[complex(c).real, complex(c).imag] for _, c in inputs], np.float64).reshape(-1)
    outs = _words(list(outputs))
    M = len(outputs)
    amp = np.zeros(2 * max(M, 1), np.float64)
    counts = np.zeros(3 * max(M, 1), np.uint64)
    A = ctypes.c_int32(0)
    rc = lib().orc_run(_gates(circuit), len(circuit.gates), circuit.n_qubits,
                       _p(ins, ctypes.c_uint64), _p(coef, ctypes.c_double), len(inputs),
                       _p(outs, ctypes.c_uint64), M, float(eps), int(c1), int(c2), int(threads),
                       _p(amp, ctypes.c_double), _p(counts, ctypes.c_uint64), ctypes.byref(A))
    if rc:
        raise ValueError(f"orc_run failed: {rc}")
    a = amp[0:2 * M:2] + 1j * amp[1:2 * M:2]
    c = counts[:3 * M].reshape(M, 3)
    return a, {"completed": c[:, 0].copy(), "valid": c[:, 1].copy(),
               "visits": c[:, 2].copy(), "A": int(A.value)}


def checkpoints(circuit, b_in: int, b_out: int, c1: int):
    """Checkpoint table of one (input, output) pair after the prefix [0, c1)
    of Algorithm 2 (exact mode): per prefix assignment h_p (source j = bit j)
    the state (int), beta_p (complex), live (False = an exactly zero factor)
    and the exact subtree sum over the remaining sources; and A_p."""
    G = len(circuit.gates)
    size = 1 << region_counts(circuit, c1, c1)[0][3]
    bi, bo = _words([b_in]), _words([b_out])
    st = np.zeros(2 * size, np.uint64)
    amp = np.zeros(2 * size, np.float64)
    ok = np.zeros(size, np.uint8)
    sub = np.zeros(2 * size, np.float64)
    Ap = ctypes.c_int32(0)
    rc = lib().orc_checkpoints(_gates(circuit), G, circuit.n_qubits, _p(bi, ctypes.c_uint64),
                               _p(bo, ctypes.c_uint64), int(c1), _p(st, ctypes.c_uint64),
                               _p(amp, ctypes.c_double), _p(ok, ctypes.c_uint8), _p(sub, ctypes.c_double),
                               ctypes.byref(Ap))
    if rc:
        raise ValueError(f"orc_checkpoints failed: {rc}")
    m = 1 << Ap.value
    states = [int(st[2 * i]) | (int(st[2 * i + 1]) << 64) for i in range(m)]
    return {"Ap": int(Ap.value), "state": states,
            "beta": amp[0:2 * m:2] + 1j * amp[1:2 * m:2],
            "live": ok[:m].astype(bool),
            "subtree": sub[0:2 * m:2] + 1j * sub[1:2 * m:2]}

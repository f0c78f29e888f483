"""O2: dense state-vector simulation (test infrastructure only).

C|psi> for psi given as a sparse input (Eq. 2 of the paper), computed by
applying each gate's full local matrix (oracle.gates.local_matrix) to a
2^n-entry complex128 vector, so every output amplitude is available at once.
Feasible up to ~24 qubits (2^24 x 16 B = 256 MB).
"""
from __future__ import annotations

import numpy as np

from .gates import local_matrix


def apply_gate(psi: np.ndarray, g, n: int) -> np.ndarray:
    """psi has shape (2,)*n with axis j <-> qubit n-1-j (C order of the flat
    index sum_q bit_q 2^q)."""
    qubits, M = local_matrix(g)
    k = len(qubits)
    Mt = M.reshape((2,) * (2 * k))
    # in Mt the first k axes are output bits of qubits[k-1], ..., qubits[0]
    in_axes = list(range(k, 2 * k))
    psi_axes = [n - 1 - q for q in reversed(qubits)]
    out = np.tensordot(Mt, psi, axes=(in_axes, psi_axes))
    return np.moveaxis(out, list(range(k)), psi_axes)


def statevector(circuit, inputs) -> np.ndarray:
    """Final state (flat, index = basis integer) for the sparse input
    [(basis, coefficient), ...]."""
    n = circuit.n_qubits
    flat = np.zeros(1 << n, complex)
    for b, c in inputs:
        flat[b] += c
    psi = flat.reshape((2,) * n) if n > 0 else flat
    for g in circuit.gates:
        psi = apply_gate(psi, g, n)
    return psi.reshape(-1)


def amplitudes(circuit, inputs, outputs) -> np.ndarray:
    sv = statevector(circuit, inputs)
    return np.array([sv[o] for o in outputs], complex)


def unitary(circuit) -> np.ndarray:
    """Full 2^n x 2^n matrix, column j = C|j> (tiny circuits only)."""
    n = circuit.n_qubits
    cols = [statevector(circuit, [(j, 1.0)]) for j in range(1 << n)]
    return np.stack(cols, axis=1)

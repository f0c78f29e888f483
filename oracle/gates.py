"""Gate matrices for the Python oracle tiers (O1, O2).

Conventions (readings of the paper, which gives none; the product documents
the same ones in its header):
  H = [[1,1],[1,-1]]/sqrt2, X, Y = [[0,-i],[i,0]], Z = diag(1,-1),
  S = diag(1,i), T = diag(1,e^{i pi/4}), P(t) = diag(1,e^{it}),
  RX(t) = [[c,-is],[-is,c]], RY(t) = [[c,-s],[s,c]],
  RZ(t) = diag(e^{-it/2}, e^{it/2}), RZZ(t) = diag over (b0,b1) of
  e^{-it/2} when b0 == b1 else e^{+it/2}, c = cos(t/2), s = sin(t/2).
Matrices are indexed [output value, input value] (the paper's U_{i(t-1),i(t)}
transition element read as <out|U|in>).
"""
from __future__ import annotations

import math

import numpy as np


def base_matrix(g) -> np.ndarray:
    """Matrix of the gate on its target qubits only (controls excluded).
    For two targets the index is bit(q0) + 2*bit(q1)."""
    t = g.theta
    c, s = math.cos(t / 2), math.sin(t / 2)
    k = g.kind
    if k == "H":
        h = math.sqrt(0.5)
        return np.array([[h, h], [h, -h]], complex)
    if k == "X":
        return np.array([[0, 1], [1, 0]], complex)
    if k == "Y":
        return np.array([[0, -1j], [1j, 0]], complex)
    if k == "Z":
        return np.diag([1, -1]).astype(complex)
    if k == "S":
        return np.diag([1, 1j])
    if k == "T":
        return np.diag([1, complex(math.cos(math.pi / 4), math.sin(math.pi / 4))])
    if k == "P":
        return np.diag([1, complex(math.cos(t), math.sin(t))])
    if k == "RX":
        return np.array([[c, -1j * s], [-1j * s, c]], complex)
    if k == "RY":
        return np.array([[c, -s], [s, c]], complex)
    if k == "RZ":
        return np.diag([complex(c, -s), complex(c, s)])
    if k == "RZZ":
        e0, e1 = complex(c, -s), complex(c, s)
        return np.diag([e0, e1, e1, e0])
    if k == "SWAP":
        m = np.zeros((4, 4), complex)
        m[0, 0] = m[1, 2] = m[2, 1] = m[3, 3] = 1
        return m
    if k in ("U1", "U2"):
        d = 2 if k == "U1" else 4
        return np.array(g.matrix, complex).reshape(d, d)
    raise ValueError(k)


def local_matrix(g):
    """(qubits, M): the full matrix of a gate on the list `qubits` =
    targets followed by controls; local index bit i <-> qubits[i].  A control
    (qubit, v) enables the base action when the qubit holds v, otherwise the
    gate acts as the identity."""
    tq = list(g.qubits)
    cq = [q for q, _ in g.controls]
    cv = [v for _, v in g.controls]
    qubits = tq + cq
    B = base_matrix(g)
    dt = B.shape[0]
    nt = len(tq)
    dim = 1 << len(qubits)
    M = np.zeros((dim, dim), complex)
    for ctrl in range(1 << len(cq)):
        on = all(((ctrl >> j) & 1) == cv[j] for j in range(len(cq)))
        for o in range(dt):
            for i in range(dt):
                val = B[o, i] if on else (1.0 if o == i else 0.0)
                M[o | (ctrl << nt), i | (ctrl << nt)] = val
    return qubits, M

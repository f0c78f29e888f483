"""O1: literal brute-force path sums (test infrastructure only).

Two obviously-correct definitions of the transition amplitude, for tiny
circuits only:

* ``history_sum`` -- Eqs. 3-5 of the paper written out: the sum over every
  sequence of intermediate computational-basis states of the product of the
  full 2^n x 2^n gate matrix elements.
* ``wire_sum`` -- the internal-wire formulation of Sec. II-A: every gate that
  acts on a qubit (as target or control) ends that qubit's wire segment and
  starts a new one; the unknowns are the segments that touch neither the
  input nor the output boundary, and a history's weight is the product of
  each gate's local matrix element between the values on its incoming and
  outgoing segments.  No segment merging, no propagation, no sources.
"""
from __future__ import annotations

import itertools

import numpy as np

from .gates import local_matrix


def _full_matrix(g, n):
    qubits, M = local_matrix(g)
    dim = 1 << n
    U = np.zeros((dim, dim), complex)
    k = len(qubits)
    rest_mask = (dim - 1) & ~sum(1 << q for q in qubits)
    for i in range(dim):
        li = sum(((i >> q) & 1) << j for j, q in enumerate(qubits))
        for lo in range(1 << k):
            v = M[lo, li]
            if v == 0:
                continue
            o = i & rest_mask
            for j, q in enumerate(qubits):
                o |= ((lo >> j) & 1) << q
            U[o, i] += v
    return U


def history_sum(circuit, b_in: int, b_out: int) -> complex:
    """Eq. 5: sum over histories (i_in, i(1), ..., i(m-1), i_out) of
    prod_t <i(t)|U^(t)|i(t-1)> (Eq. 4)."""
    n = circuit.n_qubits
    Us = [_full_matrix(g, n) for g in circuit.gates]
    m = len(Us)
    if m == 0:
        return complex(1.0 if b_in == b_out else 0.0)
    total = 0j
    for mids in itertools.product(range(1 << n), repeat=m - 1):
        seq = (b_in,) + mids + (b_out,)
        a = 1 + 0j
        for t in range(m):
            a *= Us[t][seq[t + 1], seq[t]]
            if a == 0:
                break
        total += a
    return total


def count_internal_wires(circuit) -> int:
    segs_per_qubit = [1] * circuit.n_qubits
    for g in circuit.gates:
        for q in list(g.qubits) + [c for c, _ in g.controls]:
            segs_per_qubit[q] += 1
    return sum(max(0, s - 2) for s in segs_per_qubit)


def wire_sum(circuit, b_in: int, b_out: int) -> complex:
    """Sum over all assignments of the internal wire segments (vectorised
    over the 2^V assignments) of the product of local gate elements."""
    n = circuit.n_qubits
    # segment ids: per qubit a running counter; (q, k) with k = 0 the input wire
    last = [0] * n
    gate_io = []
    for g in circuit.gates:
        qubits, M = local_matrix(g)
        ins = [(q, last[q]) for q in qubits]
        for q in qubits:
            last[q] += 1
        outs = [(q, last[q]) for q in qubits]
        gate_io.append((M, ins, outs))
    var = {}
    for q in range(n):
        for k in range(1, last[q]):
            var[(q, k)] = len(var)
    V = len(var)
    if V > 24:
        raise ValueError(f"{V} internal wires: too many for brute force")
    assign = np.arange(1 << V, dtype=np.int64)

    def value(seg):
        q, k = seg
        if k == 0 and last[q] == 0:
            # untouched qubit: input wire is the output wire
            return None
        if k == 0:
            return (b_in >> q) & 1
        if k == last[q]:
            return (b_out >> q) & 1
        return (assign >> var[seg]) & 1

    for q in range(n):
        if last[q] == 0 and ((b_in >> q) & 1) != ((b_out >> q) & 1):
            return 0j
    amp = np.ones(1 << V, complex)
    for M, ins, outs in gate_io:
        li = 0
        lo = 0
        for j, seg in enumerate(ins):
            li = li + (value(seg) << j)
        for j, seg in enumerate(outs):
            lo = lo + (value(seg) << j)
        amp = amp * M[lo, li]
    return complex(amp.sum())

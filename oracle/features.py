"""CPU reference of the learned pruner's 16 input features (test
infrastructure only; not loaded by the library).

For one checkpoint-table entry (state sigma after the prefix region, partial
amplitude beta), input bit string b_in, and the cut (c1 of G gates, A_p of A
artificial sources before it), the features are, in FP64:
  0 |beta|                      1 max(log10 |beta|, -30)  (-30 for beta = 0)
  2 Re beta / |beta|            3 Im beta / |beta|        (0 for beta = 0)
  4 (1 + log2 |int(sigma) - int(b_in)|) / 8, 0 when sigma = b_in
    (registers read as unsigned integers, qubit q = bit q)
  5 c1 / G                      6 (A - A_p) / A           (0 for G = 0, A = 0)
  7 Hamming(sigma, b_in) / n
  8..15 bit q_k of sigma xor b_in for the targets q_k of the next 8
    artificial sources after the cut (evaluation order), 0 where fewer
    remain.
The list follows the feature set the learned-pruning configuration names
(|partial amplitude|, log magnitude, depth, remaining branch count, 8
boundary bits) completed to 16 inputs.
"""
from __future__ import annotations

import math

import numpy as np

from . import feynman


def next_source_qubits(circuit, Ap: int, k: int = 8):
    """Target qubits of artificial sources A_p .. A_p + k - 1 (-1: none)."""
    an = feynman.analyze(circuit)
    q_of = {}
    for g, (s0, s1) in zip(circuit.gates, an["src"]):
        if s0 >= 0:
            q_of[s0] = g.qubits[0]
        if s1 >= 0:
            q_of[s1] = g.qubits[1]
    return [q_of.get(Ap + j, -1) for j in range(k)]


def entry_features(state: int, beta: complex, b_in: int, n: int, c1: int, G: int, A: int, Ap: int,
                   next_qubits) -> np.ndarray:
    f = np.zeros(16, np.float64)
    mag = abs(beta)
    f[0] = mag
    f[1] = max(math.log10(mag), -30.0) if mag > 0 else -30.0
    f[2] = beta.real / mag if mag > 0 else 0.0
    f[3] = beta.imag / mag if mag > 0 else 0.0
    d = abs(state - b_in)
    f[4] = (1.0 + math.log2(d)) / 8.0 if d else 0.0
    f[5] = c1 / G if G else 0.0
    f[6] = (A - Ap) / A if A else 0.0
    x = state ^ b_in
    f[7] = bin(x).count("1") / n
    for k, q in enumerate(next_qubits):
        f[8 + k] = float((x >> q) & 1) if q >= 0 else 0.0
    return f


def table_features(circuit, b_in: int, b_out: int, c1: int):
    """Features (FP64 [2^A_p, 16], NaN rows for bottom entries) and exact
    subtree sums of one (input, output) pair's checkpoint table, in the
    oracle's prefix order (source j = bit j of h_p)."""
    t = feynman.checkpoints(circuit, b_in, b_out, c1)
    A = feynman.analyze(circuit)["A"]
    Ap = t["Ap"]
    nq = next_source_qubits(circuit, Ap)
    G = len(circuit.gates)
    m = len(t["state"])
    F = np.full((m, 16), np.nan)
    for i in range(m):
        if t["live"][i]:
            F[i] = entry_features(t["state"][i], complex(t["beta"][i]), b_in, circuit.n_qubits, c1, G, A, Ap, nq)
    return F, t["subtree"], Ap

"""O4: closed forms and independent small models (test infrastructure only).

* QFT without final swaps (Sec. V, QFT case study): with H applied first to
  the most significant qubit and controlled phases from lower qubits,
  <y|C|x> = 2^{-n/2} exp(2 pi i x rev_n(y) / 2^n), rev_n reversing the n-bit
  string.  (The dense tier confirms the bit-reversal convention.)
* Coined quantum walk (Sec. V, quantum-walk case study): the walk simulated
  directly in offset space -- coin H, then a move of +1 when the coin is 1 and
  -1 when it is 0 -- over offsets [-T, T] from the start position; no circuit
  and no gates involved.
* Fidelity of a pruned output vector against the exact one.
"""
from __future__ import annotations

import cmath
import math

import numpy as np


def bit_reverse(y: int, n: int) -> int:
    r = 0
    for i in range(n):
        r |= ((y >> i) & 1) << (n - 1 - i)
    return r


def qft_amplitude(n: int, x: int, y: int) -> complex:
    return cmath.exp(2j * math.pi * x * bit_reverse(y, n) / (1 << n)) / math.sqrt(1 << n)


def walk_offsets(steps: int, coin0: complex, coin1: complex):
    """Amplitudes a[k + steps, c] of offset k and coin c after `steps` steps
    from offset 0 with coin state coin0|0> + coin1|1>."""
    a = np.zeros((2 * steps + 1, 2), complex)
    a[steps, 0] = coin0
    a[steps, 1] = coin1
    s = math.sqrt(0.5)
    for _ in range(steps):
        c0 = s * (a[:, 0] + a[:, 1])
        c1 = s * (a[:, 0] - a[:, 1])
        b = np.zeros_like(a)
        b[:-1, 0] = c0[1:]      # coin 0 moves to offset - 1
        b[1:, 1] = c1[:-1]      # coin 1 moves to offset + 1
        a = b
    return a


def walk_amplitude(steps: int, p0: int, y: int, coin0: complex, coin1: complex,
                   pos_bits: int) -> complex:
    """Amplitude of output y (coin = bit 0, position = bits 1..pos_bits,
    ancillas 0) of the coined walk started at position p0."""
    if y >> (pos_bits + 1):
        return 0j
    coin = y & 1
    k = (y >> 1) - p0
    if abs(k) > steps:
        return 0j
    return complex(walk_offsets(steps, coin0, coin1)[k + steps, coin])


def fidelity(a_exact, a_test) -> float:
    """|<a_exact, a_test>|^2 / (|a_exact|^2 |a_test|^2) over the requested
    outputs; 0 when either vector vanishes."""
    a = np.asarray(a_exact, complex)
    b = np.asarray(a_test, complex)
    na = np.vdot(a, a).real
    nb = np.vdot(b, b).real
    if na == 0 or nb == 0:
        return 0.0
    return float(abs(np.vdot(a, b)) ** 2 / (na * nb))


def captured_weight(a_exact, a_test) -> float:
    a = np.asarray(a_exact, complex)
    b = np.asarray(a_test, complex)
    na = np.vdot(a, a).real
    return float(np.vdot(b, b).real / na) if na else 0.0

"""Seeded circuit families and request lists (inputs only, no method arithmetic).

Conventions fixed here and used by every consumer:

* A basis state is a Python ``int``; qubit ``q`` is bit ``q`` (qubit 0 is the
  least significant bit).  Circuits have at most 128 qubits.
* A ``Gate`` names its kind, its target qubit(s), optional controls given as
  ``(qubit, value)`` pairs (value 0 is a negative control), an angle and, for
  the explicit kinds ``U1``/``U2``, a row-major matrix whose row index is the
  output value and whose column index is the input value.  For ``U2`` the
  two-bit value is ``bit(q0) + 2*bit(q1)``.
* Controls are allowed on ``X``, ``Z``, ``P``, ``S`` and ``T`` only
  (controlled permutations and controlled phases: CNOT, Toffoli, MCX, CZ,
  MCZ, controlled-R_k).

The four families are those of the evaluation section of the paper (QFT,
amplitude amplification, QAOA MaxCut, coined quantum walk) plus the two worked
examples of the paper's Sec. II (three-qubit H/CNOT/S/CNOT) and Fig. 2
(four-qubit internal-wire example).  Random numbers come from splitmix64
(Steele, Lea and Flood, OOPSLA 2014) so that every input is reproducible.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

import numpy as np

MASK64 = (1 << 64) - 1

KINDS = ("H", "X", "Y", "Z", "S", "T", "P", "RX", "RY", "RZ", "RZZ",
         "SWAP", "U1", "U2")
CONTROLLABLE = ("X", "Z", "P", "S", "T")


class SplitMix64:
    """splitmix64 generator: 64-bit state advanced by the golden-ratio
    increment, output mixed by two xor-shift-multiply rounds."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Uniform double in [0, 1) from the top 53 bits."""
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))

    def below(self, n: int) -> int:
        """Uniform integer in [0, n) for n < 2**64 (multiply-shift)."""
        return (self.next_u64() * n) >> 64

    def bits(self, nbits: int) -> int:
        """Uniform nbits-bit integer (nbits <= 128)."""
        v = 0
        got = 0
        while got < nbits:
            v |= self.next_u64() << got
            got += 64
        return v & ((1 << nbits) - 1)


@dataclass(frozen=True)
class Gate:
    kind: str
    qubits: Tuple[int, ...]
    controls: Tuple[Tuple[int, int], ...] = ()
    theta: float = 0.0
    matrix: Optional[Tuple[complex, ...]] = None

    def __post_init__(self):
        assert self.kind in KINDS, self.kind
        nq = 2 if self.kind in ("RZZ", "SWAP", "U2") else 1
        assert len(self.qubits) == nq, (self.kind, self.qubits)
        if self.controls:
            assert self.kind in CONTROLLABLE, self.kind
        if self.kind in ("U1", "U2"):
            assert self.matrix is not None and len(self.matrix) == (4 if self.kind == "U1" else 16)


@dataclass
class Circuit:
    n_qubits: int
    gates: List[Gate]
    name: str = ""

    def qubits_used(self):
        s = set()
        for g in self.gates:
            s.update(g.qubits)
            s.update(q for q, _ in g.controls)
        return s


@dataclass
class Workload:
    """One request: a circuit, a sparse input state and the requested outputs."""
    circuit: Circuit
    inputs: List[Tuple[int, complex]]          # (basis state, coefficient)
    outputs: List[int]
    eps: float = 0.0
    name: str = ""
    meta: dict = field(default_factory=dict)


def bits_to_int(bits: Sequence[int]) -> int:
    return sum((int(b) & 1) << i for i, b in enumerate(bits))


def int_to_bits(x: int, n: int) -> List[int]:
    return [(x >> i) & 1 for i in range(n)]


# --------------------------------------------------------------------------
# Worked examples of the paper
# --------------------------------------------------------------------------

def three_qubit_example() -> Circuit:
    """Sec. II worked example: H(q0), CNOT(q0->q1), S(q1), CNOT(q1->q2)."""
    return Circuit(3, [
        Gate("H", (0,)),
        Gate("X", (1,), ((0, 1),)),
        Gate("S", (1,)),
        Gate("X", (2,), ((1, 1),)),
    ], "three_qubit_example")


def four_qubit_figure() -> Circuit:
    """Fig. 2 four-qubit internal-wire circuit, columns 1..5 in order, gates
    within a column in the order the figure lists them."""
    return Circuit(4, [
        Gate("X", (0,), ((1, 1),)),          # col 1: CNOT q1 -> q0
        Gate("H", (1,)),                     # col 2
        Gate("SWAP", (2, 3)),                # col 2
        Gate("H", (3,)),                     # col 3
        Gate("P", (2,), (), math.pi),        # col 3: P(pi), wire-preserving
        Gate("X", (1,), ((0, 1),)),          # col 3: CNOT q0 -> q1
        Gate("H", (0,)),                     # col 4
        Gate("SWAP", (1, 2)),                # col 5
    ], "four_qubit_figure")


def placement_figure() -> Circuit:
    """Fig. 4 three-qubit circuit for the source-placement graph, columns 1..8:
    H on q2; CNOTs q2 -> q1, q2 -> q0, q2 -> q1, q2 -> q0, q0 -> q1, q1 -> q2;
    H on q0 and q1."""
    return Circuit(3, [
        Gate("H", (2,)),                     # col 1
        Gate("X", (1,), ((2, 1),)),          # col 2
        Gate("X", (0,), ((2, 1),)),          # col 3
        Gate("X", (1,), ((2, 1),)),          # col 4
        Gate("X", (0,), ((2, 1),)),          # col 5
        Gate("X", (1,), ((0, 1),)),          # col 6
        Gate("X", (2,), ((1, 1),)),          # col 7
        Gate("H", (0,)),                     # col 8
        Gate("H", (1,)),                     # col 8
    ], "placement_figure")


# --------------------------------------------------------------------------
# Circuit families of the evaluation section
# --------------------------------------------------------------------------

def qft(n: int) -> Circuit:
    """QFT without the final swaps: for j = n-1 .. 0, H on q_j followed by
    controlled phases R_{j-k+1} (angle 2*pi/2^(j-k+1)) from each lower qubit
    q_k, k = j-1 .. 0, onto q_j."""
    gates = []
    for j in range(n - 1, -1, -1):
        gates.append(Gate("H", (j,)))
        for k in range(j - 1, -1, -1):
            gates.append(Gate("P", (j,), ((k, 1),), 2.0 * math.pi / (1 << (j - k + 1))))
    return Circuit(n, gates, f"qft{n}")


def _mcz_vchain(data: Sequence[int], anc: Sequence[int]) -> List[Gate]:
    """Multi-controlled Z over all `data` qubits built from Toffolis into
    ancillas (a_0 = d_0 & d_1, a_k = a_{k-1} & d_{k+1}), a CZ between the last
    ancilla and the last data qubit, then the Toffolis in reverse."""
    n = len(data)
    assert n >= 3 and len(anc) >= n - 2
    comp = [Gate("X", (anc[0],), ((data[0], 1), (data[1], 1)))]
    for k in range(1, n - 2):
        comp.append(Gate("X", (anc[k],), ((anc[k - 1], 1), (data[k + 1], 1))))
    cz = Gate("Z", (data[n - 1],), ((anc[n - 3], 1),))
    return comp + [cz] + comp[::-1]


def amplitude_amplification(n: int, iters: int, marked: int) -> Circuit:
    """Grover-style amplitude amplification on n data qubits (q0..q_{n-1})
    with n-2 ancillas (q_n..q_{2n-3}) for the Toffoli V-chain: H on every data
    qubit, then `iters` times [phase oracle marking `marked`: X on the data
    qubits where the marked bit is 0, MCZ, the same X's; diffusion: H^n, X^n,
    MCZ, X^n, H^n]."""
    data = list(range(n))
    anc = list(range(n, 2 * n - 2))
    gates = [Gate("H", (q,)) for q in data]
    zeros = [q for q in data if not (marked >> q) & 1]
    for _ in range(iters):
        gates += [Gate("X", (q,)) for q in zeros]
        gates += _mcz_vchain(data, anc)
        gates += [Gate("X", (q,)) for q in zeros]
        gates += [Gate("H", (q,)) for q in data]
        gates += [Gate("X", (q,)) for q in data]
        gates += _mcz_vchain(data, anc)
        gates += [Gate("X", (q,)) for q in data]
        gates += [Gate("H", (q,)) for q in data]
    return Circuit(2 * n - 2, gates, f"aa{n}x{iters}")


def random_regular_graph(n: int, d: int, rng: SplitMix64) -> List[Tuple[int, int]]:
    """Random d-regular simple graph by the pairing (configuration) model:
    shuffle n*d stubs, pair neighbours, reject loops and multi-edges."""
    assert (n * d) % 2 == 0
    while True:
        stubs = [v for v in range(n) for _ in range(d)]
        for i in range(len(stubs) - 1, 0, -1):          # Fisher-Yates
            j = rng.below(i + 1)
            stubs[i], stubs[j] = stubs[j], stubs[i]
        edges = set()
        ok = True
        for i in range(0, len(stubs), 2):
            a, b = stubs[i], stubs[i + 1]
            if a == b or (min(a, b), max(a, b)) in edges:
                ok = False
                break
            edges.add((min(a, b), max(a, b)))
        if ok:
            return sorted(edges)


def qaoa_maxcut(n: int, p: int, rng: SplitMix64, degree: int = 3):
    """QAOA for MaxCut on a seeded random regular graph: H on every qubit,
    then for l = 1..p RZZ(gamma_l) on every edge and RX(beta_l) on every
    qubit; gamma_l, beta_l uniform in [0, pi)."""
    edges = random_regular_graph(n, degree, rng)
    angles = []
    for _ in range(p):
        g = math.pi * rng.uniform()
        b = math.pi * rng.uniform()
        angles.append((g, b))
    gates = [Gate("H", (q,)) for q in range(n)]
    for g, b in angles:
        gates += [Gate("RZZ", (i, j), (), g) for i, j in edges]
        gates += [Gate("RX", (q,), (), b) for q in range(n)]
    return Circuit(n, gates, f"qaoa{n}p{p}"), edges, angles


QW_POS_BITS = 96


def quantum_walk(steps: int, pos_bits: int = QW_POS_BITS) -> Circuit:
    """Coined walk on a cycle of 2^pos_bits sites.  Qubit 0 is the coin,
    qubits 1..pos_bits the position, and three ancillas follow.  One step:
    H(coin); a0 <- coin, a1 <- not coin (CNOT, X, CNOT); position += 1
    controlled on a0 (MCX cascade, most significant bit first); position -= 1
    controlled on a1 (MCX cascade with negative controls); uncompute a1 and
    a0.  The third ancilla stays |0>."""
    coin = 0
    pos = [1 + j for j in range(pos_bits)]
    a0, a1 = pos_bits + 1, pos_bits + 2
    n = pos_bits + 4
    gates: List[Gate] = []
    for _ in range(steps):
        gates.append(Gate("H", (coin,)))
        gates.append(Gate("X", (a0,), ((coin, 1),)))
        gates.append(Gate("X", (a1,)))
        gates.append(Gate("X", (a1,), ((coin, 1),)))
        for k in range(pos_bits - 1, -1, -1):
            ctr = ((a0, 1),) + tuple((pos[j], 1) for j in range(k))
            gates.append(Gate("X", (pos[k],), ctr))
        for k in range(pos_bits - 1, -1, -1):
            ctr = ((a1, 1),) + tuple((pos[j], 0) for j in range(k))
            gates.append(Gate("X", (pos[k],), ctr))
        gates.append(Gate("X", (a1,), ((coin, 1),)))
        gates.append(Gate("X", (a1,)))
        gates.append(Gate("X", (a0,), ((coin, 1),)))
    return Circuit(n, gates, f"qw{n}t{steps}")


# --------------------------------------------------------------------------
# Random small circuits (for cross-checks on tiny sizes)
# --------------------------------------------------------------------------

def _rand_unitary(k: int, rng: SplitMix64) -> np.ndarray:
    z = np.array([[complex(rng.uniform() - 0.5, rng.uniform() - 0.5) for _ in range(k)]
                  for _ in range(k)])
    q, r = np.linalg.qr(z)
    d = np.diag(r)
    return q * (d / np.abs(d))


def random_small_circuit(n: int, n_gates: int, seed: int, kinds=None,
                         max_controls: int = 2) -> Circuit:
    """Random circuit over every gate kind (including explicit diagonal,
    permutation and dense U1/U2 matrices) for tiny cross-checks."""
    rng = SplitMix64(seed)
    kinds = list(kinds or KINDS + ("U1d", "U1p", "U2d", "U2p"))
    gates = []
    for _ in range(n_gates):
        k = kinds[rng.below(len(kinds))]
        if k in ("RZZ", "SWAP", "U2", "U2d", "U2p") and n < 2:
            k = "H"
        q0 = rng.below(n)
        q1 = (q0 + 1 + rng.below(n - 1)) % n if n > 1 else q0
        th = 2 * math.pi * rng.uniform()
        ctr = ()
        if k in CONTROLLABLE and n > 1:
            nc = rng.below(min(max_controls, n - 1) + 1)
            pool = [q for q in range(n) if q != q0]
            sel = []
            for _ in range(nc):
                c = pool.pop(rng.below(len(pool)))
                sel.append((c, rng.below(2)))
            ctr = tuple(sel)
        if k in ("RZZ", "SWAP"):
            gates.append(Gate(k, (q0, q1), (), th))
        elif k in ("U1", "U1d", "U1p"):
            if k == "U1":
                m = _rand_unitary(2, rng)
            elif k == "U1d":
                m = np.diag([np.exp(2j * math.pi * rng.uniform()) for _ in range(2)])
            else:
                m = np.array([[0, np.exp(2j * math.pi * rng.uniform())],
                              [np.exp(2j * math.pi * rng.uniform()), 0]])
            gates.append(Gate("U1", (q0,), (), 0.0, tuple(complex(v) for v in m.reshape(-1))))
        elif k in ("U2", "U2d", "U2p"):
            if k == "U2":
                m = _rand_unitary(4, rng)
            elif k == "U2d":
                m = np.diag([np.exp(2j * math.pi * rng.uniform()) for _ in range(4)])
            else:
                perm = [0, 1, 2, 3]
                for i in range(3, 0, -1):
                    j = rng.below(i + 1)
                    perm[i], perm[j] = perm[j], perm[i]
                m = np.zeros((4, 4), complex)
                for col in range(4):
                    m[perm[col], col] = np.exp(2j * math.pi * rng.uniform())
            gates.append(Gate("U2", (q0, q1), (), 0.0, tuple(complex(v) for v in m.reshape(-1))))
        else:
            gates.append(Gate(k, (q0,), ctr, th))
    return Circuit(n, gates, f"rand{n}x{n_gates}s{seed}")


# --------------------------------------------------------------------------
# Requests (circuit + sparse input + outputs) for the benchmark families
# --------------------------------------------------------------------------

SEED_BASE = 0x5EED0000


def qft_workload(n: int = 8, seed: int = SEED_BASE + 1) -> Workload:
    """QFT-n from a seeded basis input x, all 2^n outputs, exact."""
    rng = SplitMix64(seed)
    x = rng.below(1 << n)
    return Workload(qft(n), [(x, 1.0 + 0j)], list(range(1 << n)), 0.0,
                    f"qft{n}", {"x": x})


def qft_signal_workload(n: int = 12, seed: int = SEED_BASE + 6) -> Workload:
    """QFT-n of a seeded real two-tone signal as a dense input state:
    x_t = cos(2 pi f1 t / N) + cos(2 pi f2 t / N) for t = 0 .. N-1 (N = 2^n),
    normalised, every basis state with a nonzero sample in the support
    (S ~ N); all N outputs.  f1 != f2 are drawn in [1, N/2)."""
    rng = SplitMix64(seed)
    N = 1 << n
    f1 = 1 + rng.below(N // 2 - 1)
    f2 = f1
    while f2 == f1:
        f2 = 1 + rng.below(N // 2 - 1)
    x = [math.cos(2.0 * math.pi * f1 * t / N) + math.cos(2.0 * math.pi * f2 * t / N) for t in range(N)]
    norm = math.sqrt(sum(v * v for v in x))
    inputs = [(t, complex(v / norm, 0.0)) for t, v in enumerate(x) if v != 0.0]
    return Workload(qft(n), inputs, list(range(N)), 0.0, f"qft{n}signal", {"f1": f1, "f2": f2})


def aa_workload(n: int = 12, iters: int = 3, n_out: int = 64,
                seed: int = SEED_BASE + 2, all_outputs: bool = False) -> Workload:
    """Amplitude amplification with a seeded marked string; outputs are the
    marked string plus seeded distinct data strings (ancillas 0), or every
    data string when `all_outputs`."""
    rng = SplitMix64(seed)
    m = rng.below(1 << n)
    c = amplitude_amplification(n, iters, m)
    if all_outputs:
        outs = list(range(1 << n))
    else:
        outs = [m]
        seen = {m}
        while len(outs) < min(n_out, 1 << n):
            y = rng.below(1 << n)
            if y not in seen:
                seen.add(y)
                outs.append(y)
    return Workload(c, [(0, 1.0 + 0j)], outs, 0.0, f"aa{n}x{iters}", {"marked": m})


def qaoa_workload(n: int, p: int = 2, n_out: int = 1024, eps: float = 0.0,
                  seed: int = SEED_BASE + 3) -> Workload:
    """QAOA MaxCut on a seeded 3-regular graph with n_out seeded distinct
    requested bit strings; input |0^n>."""
    rng = SplitMix64(seed + (n << 8) + (p << 4))
    c, edges, angles = qaoa_maxcut(n, p, rng)
    outs = []
    seen = set()
    while len(outs) < min(n_out, 1 << n):
        y = rng.bits(n)
        if y not in seen:
            seen.add(y)
            outs.append(y)
    return Workload(c, [(0, 1.0 + 0j)], outs, eps, f"qaoa{n}p{p}",
                    {"edges": edges, "angles": angles})


def qw_workload(steps: int = 16, n_out: int = 4096, pos_bits: int = QW_POS_BITS,
                seed: int = SEED_BASE + 5) -> Workload:
    """Quantum walk from a seeded start position p0 with coin
    (|0> + i|1>)/sqrt(2) (two input basis states).  Outputs: every reachable
    (position, coin) after `steps` steps, then seeded unreachable ones near p0
    (odd offsets, or even offsets beyond +-steps), ancillas 0."""
    rng = SplitMix64(seed)
    span = 1 << 20 if pos_bits > 24 else 1 << (pos_bits // 2)
    p0 = span + rng.below((1 << pos_bits) - 2 * span)
    c = quantum_walk(steps, pos_bits)
    s = 1.0 / math.sqrt(2.0)
    inputs = [((p0 << 1) | 0, complex(s, 0.0)), ((p0 << 1) | 1, complex(0.0, s))]
    outs = []
    seen = set()
    for k in range(-steps, steps + 1, 2):
        for coin in (0, 1):
            y = ((p0 + k) << 1) | coin
            outs.append(y)
            seen.add(y)
    reach = len(outs)
    wide = min(max(4 * n_out, 64), p0, (1 << pos_bits) - 1 - p0)
    assert n_out <= 2 * wide + 2, "register too small for that many outputs"
    while len(outs) < n_out:
        k = rng.below(2 * wide + 1) - wide
        coin = rng.below(2)
        y = ((p0 + k) << 1) | coin
        if y in seen:
            continue
        if (k - steps) % 2 == 0 and abs(k) <= steps:
            continue
        seen.add(y)
        outs.append(y)
    return Workload(c, inputs, outs, 0.0, f"qw{pos_bits + 4}t{steps}",
                    {"p0": p0, "reachable": reach})

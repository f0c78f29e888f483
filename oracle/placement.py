"""Artificial-source placement as a graph problem (Sec. IV-B, Fig. 4) --
test infrastructure only.

For circuits of CNOTs and single-qubit gates the internal wires form a
graph: every CNOT is a node joined to three wires (its control wire and the
two sides of its target), and knowing any two of them fixes the third by
XOR.  Single-qubit deterministic gates and wire-preserving gates (diagonal,
controls) keep a wire; single-qubit branching gates separate the two sides
(no constraint).  The input and output wires are known from b_in and b_out
(natural sources).  The minimum number of artificial sources is the size
of the smallest set of extra known wires whose closure under the CNOT rule
is every wire.  Natural sources simplify the graph first: a CNOT touching a
known wire is removed and its other two wires are merged.
"""
from __future__ import annotations

from itertools import combinations

DIAGONAL = ("Z", "S", "T", "P", "RZ", "RZZ")
BRANCHING = ("H", "RX", "RY")


class Unsupported(ValueError):
    pass


def wire_graph(circuit):
    """(number of wires, known wire ids, CNOT triples (control, target in,
    target out)) in circuit order."""
    n = circuit.n_qubits
    nwires = n
    cur = list(range(n))
    known = set(range(n))                 # input wires
    cnots = []
    for g in circuit.gates:
        if g.kind in DIAGONAL:
            continue                      # wire-preserving (controls included)
        if g.kind in ("X", "Y") and not g.controls:
            continue                      # deterministic: both sides are one wire
        if g.kind == "SWAP":
            a, b = g.qubits
            cur[a], cur[b] = cur[b], cur[a]   # the two wires change qubits
            continue
        if g.kind == "X" and len(g.controls) == 1:
            (c, _), t = g.controls[0], g.qubits[0]
            cnots.append((cur[c], cur[t], nwires))
            cur[t] = nwires
            nwires += 1
            continue
        if g.kind in BRANCHING and not g.controls:
            cur[g.qubits[0]] = nwires
            nwires += 1
            continue
        raise Unsupported(f"gate {g.kind} with {len(g.controls)} controls is outside CNOT + 1-qubit")
    known |= set(cur)                     # output wires
    return nwires, known, cnots


class _DSU:
    def __init__(self, n):
        self.p = list(range(n))

    def find(self, x):
        while self.p[x] != x:
            self.p[x] = self.p[self.p[x]]
            x = self.p[x]
        return x

    def union(self, a, b):
        a, b = self.find(a), self.find(b)
        if a != b:
            self.p[max(a, b)] = min(a, b)


def simplified(circuit):
    """Apply the natural-source merge rule until no CNOT touches a known
    node: (node ids, known nodes, remaining CNOT triples over nodes)."""
    nw, known, cnots = wire_graph(circuit)
    d = _DSU(nw)
    known = set(known)
    live = list(cnots)
    changed = True
    while changed:
        changed = False
        rest = []
        for tri in live:
            a, b, c = (d.find(x) for x in tri)
            kn = [x for x in (a, b, c) if x in known]
            if kn:
                others = [x for x in (a, b, c) if x != kn[0]]
                if len(others) == 2:
                    d.union(others[0], others[1])
                    r = d.find(others[0])
                    if others[0] in known or others[1] in known:
                        known.add(r)
                changed = True
            else:
                rest.append((a, b, c))
        live = [tuple(d.find(x) for x in t) for t in rest]
        known = {d.find(x) for x in known}
    nodes = sorted({d.find(x) for x in range(nw)} - known)
    return nodes, known, live


def closure(known, cnots):
    known = set(known)
    grew = True
    while grew:
        grew = False
        for t in cnots:
            if sum(x in known for x in t) >= 2:   # two of the three wires (a merged node counts twice)
                for x in t:
                    if x not in known:
                        known.add(x)
                        grew = True
    return known


def optimum(circuit):
    """Smallest number of artificial sources (exhaustive over subsets of
    the simplified graph's unknown nodes)."""
    nodes, known, cnots = simplified(circuit)
    allnodes = set(nodes) | known
    for k in range(len(nodes) + 1):
        for s in combinations(nodes, k):
            if closure(known | set(s), cnots) >= allnodes:
                return k
    return len(nodes)


def greedy(circuit):
    """Sources chosen one at a time: the unknown node on the most unresolved
    CNOTs (ties: smallest id), then the closure; until every node is known."""
    nodes, known, cnots = simplified(circuit)
    allnodes = set(nodes) | known
    known = closure(known, cnots)
    k = 0
    while not known >= allnodes:
        deg = {}
        for t in cnots:
            if all(x in known for x in t):
                continue
            for x in set(t):
                if x not in known:
                    deg[x] = deg.get(x, 0) + 1
        cand = sorted((x for x in nodes if x not in known), key=lambda x: (-deg.get(x, 0), x))
        known = closure(known | {cand[0]}, cnots)
        k += 1
    return k

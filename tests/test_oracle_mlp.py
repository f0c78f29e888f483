"""Pins of the CPU MLP reference: finite differences of the FP64 form, the
bfloat16 rounding rule against torch's, and agreement of the mixed-precision
form with the FP64 one to bfloat16 accuracy."""
import numpy as np
import torch

from oracle import mlp
from workloads.mlp_init import mlp_init_params


def test_bf16_rounding_matches_torch():
    x = np.random.default_rng(1).normal(size=4096).astype(np.float32) * 10
    x[:4] = [1.0, -2.5, 3.0000002, 1e-30]
    want = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.bf16(x), want)


def test_fp64_gradient_matches_finite_differences():
    rng = np.random.default_rng(7)
    p = mlp_init_params(3).astype(np.float64) * 0.5
    p[2048:2176] = rng.normal(size=128) * 0.1
    p[18560:18688] = rng.normal(size=128) * 0.1
    X = rng.normal(size=(24, 16))
    T = rng.normal(size=24)
    loss, g = mlp.loss_and_grad(p, X, T, use_bf16=False)
    idx = np.concatenate([rng.choice(2048, 12, replace=False), 2048 + rng.choice(128, 6, replace=False),
                          2176 + rng.choice(16384, 20, replace=False), 18560 + rng.choice(128, 6, replace=False),
                          18688 + rng.choice(128, 6, replace=False), [18816]])
    for i in idx:
        h = 1e-6
        pp = p.copy(); pp[i] += h
        pm = p.copy(); pm[i] -= h
        fd = (mlp.loss_and_grad(pp, X, T, False)[0] - mlp.loss_and_grad(pm, X, T, False)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 + 1e-5 * abs(fd), (i, fd, g[i])


def test_bf16_form_close_to_fp64_form():
    rng = np.random.default_rng(9)
    p = mlp_init_params(5)
    X = rng.normal(size=(64, 16))
    T = rng.normal(size=64)
    l1, g1 = mlp.loss_and_grad(p, X, T, True)
    l2, g2 = mlp.loss_and_grad(p, X, T, False)
    assert abs(l1 - l2) < 0.05 * abs(l2)
    assert np.linalg.norm(g1 - g2) < 0.05 * np.linalg.norm(g2)


def test_checkpoint_table_worked_example_and_subtree_sums():
    """Sec. II's three-qubit example, output 111 from input 000: no
    artificial source, one history; after each prefix the state and beta
    are those of the backward walk, and the single subtree sum is the
    amplitude i/sqrt2 (Eq. 6)."""
    from oracle import feynman
    from workloads import three_qubit_example
    c = three_qubit_example()
    want_state = [7, 3, 3, 1, 0]
    want_beta = [1, 1, 1j, 1j, 1j * np.sqrt(0.5)]
    for c1 in range(5):
        t = feynman.checkpoints(c, 0, 7, c1)
        assert t["Ap"] == 0 and t["state"] == [want_state[c1]] and t["live"][0]
        assert abs(t["beta"][0] - want_beta[c1]) < 1e-15
        assert abs(t["subtree"][0] - 1j * np.sqrt(0.5)) < 1e-15


def test_subtree_sums_add_up_to_the_dense_amplitude():
    """Over every prefix assignment the exact subtree sums add up to the
    amplitude (Eq. 7 split at the cut), checked against the dense state
    vector for QAOA and a random circuit with exactly-zero factors."""
    from oracle import dense, feynman
    from workloads import qaoa_workload, random_small_circuit
    w = qaoa_workload(6, 1, n_out=4, seed=3)
    c = random_small_circuit(5, 30, 555)
    for circ, b_in, outs in ((w.circuit, 0, w.outputs), (c, 9, [0, 5, 17, 31])):
        G = len(circ.gates)
        d = dense.amplitudes(circ, [(b_in, 1.0)], outs)
        for o, want in zip(outs, d):
            for c1 in (0, G // 3, G // 2, G):
                t = feynman.checkpoints(circ, b_in, o, c1)
                assert abs(np.sum(t["subtree"]) - want) < 1e-12
                # a bottom entry (an exactly zero factor) carries no subtree
                assert np.all(t["subtree"][~t["live"]] == 0)


def test_features_of_worked_example_entries():
    from oracle import features
    # beta = i/sqrt2 at state 000 (= b_in), cut after all 4 gates, A = 0
    f = features.entry_features(0, 1j * np.sqrt(0.5), 0, 3, 4, 4, 0, 0, [-1] * 8)
    assert np.allclose(f[:8], [np.sqrt(0.5), np.log10(np.sqrt(0.5)), 0, 1, 0, 1, 0, 0], atol=1e-15)
    assert np.all(f[8:] == 0)
    # state 011 against b_in 000 after 2 of 4 gates: distance 3, Hamming 2
    f = features.entry_features(3, 1j, 0, 3, 2, 4, 0, 0, [0, 1, 2, -1, -1, -1, -1, -1])
    assert np.allclose(f[:8], [1, 0, 0, 1, (1 + np.log2(3)) / 8, 0.5, 0, 2 / 3], atol=1e-15)
    assert list(f[8:]) == [1, 1, 0, 0, 0, 0, 0, 0]
    # 128-bit registers: |sigma - b_in| = 2^100 - 1 -> 1 + log2 just below 101
    f = features.entry_features((1 << 100) - 1, 0.5, 0, 128, 1, 2, 4, 1, [-1] * 8)
    assert abs(f[4] * 8 - (1 + 100)) < 1e-12 and f[6] == 0.75 and f[1] == np.log10(0.5)


def test_next_source_qubits_follow_backward_numbering():
    """QAOA p = 1: the backward sweep meets the RX layer first (sources
    0..n-1 on qubits n-1..0 in evaluation order); the H layer is natural."""
    from oracle import feynman, features
    from workloads import qaoa_workload
    w = qaoa_workload(6, 1, n_out=1, seed=3)
    an = feynman.analyze(w.circuit)
    rx = [g.qubits[0] for g in w.circuit.gates if g.kind == "RX"]
    assert an["A"] == 6
    assert features.next_source_qubits(w.circuit, 0, 8) == list(reversed(rx)) + [-1, -1]
    assert features.next_source_qubits(w.circuit, 4, 8) == list(reversed(rx))[4:] + [-1] * 6

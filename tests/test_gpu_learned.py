"""Learned pruning: the MLP kernels against the CPU reference MLP, Adam, the
logging run, and the pruner end to end (cuts nothing at tau = -inf; keeps
the fidelity bar at a tuned tau)."""
import math

import numpy as np
import pytest
import torch

from workloads import mlp_init_params, qaoa_workload
from oracle import closed_forms, mlp as omlp
import paper_2608_01467_b300 as fs
from paper_2608_01467_b300 import learned

pytestmark = pytest.mark.gpu


def rel_err(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


def test_mlp_forward_matches_cpu_reference():
    rng = np.random.default_rng(1)
    p = mlp_init_params(11)
    X = rng.normal(size=(1003, 16)).astype(np.float32)
    y = learned.forward(torch.from_numpy(p).cuda(), torch.from_numpy(X).cuda()).cpu().numpy()
    want, _ = omlp.forward(p, X)
    assert rel_err(y, want) < 1e-2
    assert np.max(np.abs(y - want)) < 2e-2 * np.max(np.abs(want))


def test_mlp_gradient_matches_cpu_reference():
    rng = np.random.default_rng(2)
    p = mlp_init_params(12)
    p[2048:2176] = rng.normal(size=128) * 0.1
    p[18560:18688] = rng.normal(size=128) * 0.1
    X = rng.normal(size=(777, 16)).astype(np.float32)
    T = rng.normal(size=777).astype(np.float32)
    g, loss = learned.grad(torch.from_numpy(p).cuda(), torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda())
    g = g.cpu().numpy()
    wl, wg = omlp.loss_and_grad(p, X, T)
    assert abs(float(loss) - wl) < 1e-3 * abs(wl)
    errs = {}
    for name, (lo, hi) in {"W1": (0, 2048), "b1": (2048, 2176), "W2": (2176, 18560), "b2": (18560, 18688),
                           "w3": (18688, 18816), "b3": (18816, 18817)}.items():
        errs[name] = rel_err(g[lo:hi], wg[lo:hi])
    print("gradient relative errors per block:", errs)
    assert all(e < 1e-2 for e in errs.values()), errs


def test_adam_step_matches_formula():
    rng = np.random.default_rng(3)
    p = rng.normal(size=18817).astype(np.float32)
    g = rng.normal(size=18817).astype(np.float32)
    P, M, V = (torch.from_numpy(p).cuda(), torch.zeros(18817, device="cuda"), torch.zeros(18817, device="cuda"))
    G = torch.from_numpy(g).cuda()
    for step in (1, 2):
        learned.adam_step(P, M, V, G, 1e-3, step)
    m = 0.0
    v = 0.0
    q = p.astype(np.float64)
    for step in (1, 2):
        m = 0.9 * m + 0.1 * g
        v = 0.999 * v + 0.001 * g * g
        q = q - 1e-3 * (m / (1 - 0.9 ** step)) / (np.sqrt(v / (1 - 0.999 ** step)) + 1e-8)
    assert np.max(np.abs(P.cpu().numpy() - q)) < 1e-5


def test_training_reduces_loss_on_a_known_target():
    rng = np.random.default_rng(4)
    X = rng.normal(size=(8192, 16)).astype(np.float32)
    T = (X[:, 0] * 0.7 - np.abs(X[:, 3]) + 0.3 * X[:, 8] * X[:, 9]).astype(np.float32)
    x, t = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
    _, l0 = learned.grad(torch.from_numpy(mlp_init_params(5)).cuda(), x, t)
    p, losses = learned.train(x, t, mlp_init_params(5), steps=300, batch=2048, lr=3e-3)
    _, l1 = learned.grad(p, x, t)
    assert float(l1) < 0.1 * float(l0)


def _run(w, outs, cut, eps=0.0, pruner=None, tau=0.0):
    C = fs.Circuit(w.circuit)
    C.set_input(w.inputs)
    b = fs.Batch(split="fixed", c1=cut, c2=cut)
    b.add(C, outs, eps)
    if pruner is not None:
        learned.attach(b, 0, pruner, tau)
    b.plan()
    b.allocate()
    b.upload()
    b.run()
    st = b.finish()[0]
    return b.amp.cpu().numpy()[:len(outs)], st


def _bitrev(x, bits):
    return int(format(x, f"0{bits}b")[::-1], 2) if bits else 0


@pytest.mark.parametrize("case", ["qaoa", "walk", "random"])
def test_table_features_and_logged_subtree_sums_match_oracle(case):
    """Every checkpoint entry's 16 features (FP32 on the GPU) and exact
    subtree sum (the training target) against the oracle's checkpoint table
    and its FP64 feature definition.  The library numbers prefix sources
    from the most significant bit of h_p, the oracle from the least."""
    from oracle import features as ofeat
    if case == "qaoa":
        w = qaoa_workload(8, 2, n_out=5, seed=17)
        circ, inputs, outs = w.circuit, w.inputs, w.outputs
        cut = 24
    elif case == "walk":
        from workloads import qw_workload
        w = qw_workload(steps=7, n_out=6, pos_bits=8)
        circ, inputs, outs = w.circuit, w.inputs, w.outputs
        cut = len(circ.gates) // 2
    else:
        from workloads import SplitMix64, random_small_circuit
        circ = random_small_circuit(7, 40, 4321)
        rng = SplitMix64(4321)
        inputs = [(rng.bits(7), 0.6), (rng.bits(7), 0.8j)]
        outs = [rng.bits(7) for _ in range(5)]
        cut = 20
    feat, log, st = learned.table_data(circ, inputs, outs, cut)
    feat = feat.cpu().numpy()
    tgt = learned.subtree_targets(log).cpu().numpy().astype(np.float64)
    sub = log.cpu().numpy()
    sub = sub[:, 0] + 1j * sub[:, 1]
    S = len(inputs)
    Ap = st["A_p"]
    assert feat.shape[0] == len(outs) * S << Ap
    for o, b_out in enumerate(outs):
        for s, (b_in, _) in enumerate(inputs):
            F, T, ap = ofeat.table_features(circ, b_in, b_out, cut)
            assert ap == Ap
            base = (o * S + s) << Ap
            idx = [base + _bitrev(h, Ap) for h in range(1 << Ap)]
            g, gs = feat[idx], sub[idx]
            live = ~np.isnan(F[:, 0])
            assert np.array_equal(np.isnan(g[:, 0]), ~live)
            err = np.abs(gs - T)
            assert np.all(err <= 1e-12 + 1e-10 * np.abs(T)), err.max()
            d = np.abs(g[live].astype(np.float64) - F[live])
            assert np.all(d[:, :8] <= 2e-5 + 2e-5 * np.abs(F[live][:, :8])), d.max(axis=0)
            assert np.array_equal(g[live][:, 8:], F[live][:, 8:])
            # the training target: max(log10 |subtree sum|, -12) (fs_mlp_targets),
            # checked where the sum is well above the 1e-12 amplitude bar
            tg = tgt[idx]
            big = np.abs(T) >= 1e-9
            want_t = np.maximum(np.log10(np.abs(T[big])), learned.TARGET_FLOOR)
            assert np.all(np.abs(tg[big] - want_t) <= 1e-5), np.max(np.abs(tg[big] - want_t))
            assert np.all(tg >= learned.TARGET_FLOOR)
            zero = np.abs(T) == 0.0
            assert np.all(tg[zero & (np.abs(gs) == 0.0)] == learned.TARGET_FLOOR)


def test_prune_decisions_match_cpu_mlp_on_logged_features():
    """The tensor-core scoring inside the prune step against the CPU
    reference MLP on the same checkpoint entries: every entry whose CPU score
    is clearly below tau is cut, every entry clearly above is kept."""
    n = 10
    w = qaoa_workload(n, 2, n_out=24, seed=23)
    cut = n
    x, t, _ = learned.log_training_data(w.circuit, w.inputs, w.outputs, cut)
    p = mlp_init_params(31)
    score, _ = omlp.forward(p, x.cpu().numpy())
    tau = float(np.median(score))
    margin = 2e-2 * float(np.max(np.abs(score)))
    below = int(np.sum(score < tau - margin))
    near = int(np.sum(np.abs(score - tau) <= margin))
    _, st = _run(w, w.outputs, cut, pruner=torch.from_numpy(p).cuda(), tau=tau)
    assert below > 0 and below <= st["learned_cuts"] <= below + near, (below, near, st["learned_cuts"])
    assert st["live_entries"] == x.shape[0] - st["learned_cuts"]


def test_learned_pruner_end_to_end():
    n = 12
    w = qaoa_workload(n, 2, n_out=128, seed=21)
    cut = n                                  # after the last RX layer (A_p = n)
    x, t, st = learned.log_training_data(w.circuit, w.inputs, w.outputs[:64], cut)
    assert x.shape[0] == 64 * (1 << n) and st["valid"] == 64 * (1 << 24)
    params, losses = learned.train(x, t, mlp_init_params(0), steps=300, batch=4096, lr=2e-3)
    assert losses[-1] < losses[0]
    held = w.outputs[64:]
    exact, st_ex = _run(w, held, cut)
    # tau below every prediction: nothing is cut and the result is the exact
    # one (summed over the compacted entries: equal to rounding)
    a, st0 = _run(w, held, cut, pruner=params, tau=-1e30)
    assert st0["learned_cuts"] == 0 and st0["valid"] == st_ex["valid"]
    assert np.max(np.abs(a - exact) - (1e-12 + 1e-10 * np.abs(exact))) <= 0
    # some tau keeps fidelity >= 0.999 while cutting checkpoint entries
    best = None
    for tau in (-9.0, -8.0, -7.0, -6.0, -5.5, -5.0):
        a, s = _run(w, held, cut, pruner=params, tau=tau)
        F = closed_forms.fidelity(exact, a)
        if F >= 0.999:
            best = (tau, F, s["learned_cuts"], s["completed"])
    assert best is not None and best[2] > 0, best


def _qw_run(w, split="auto", c1=0, c2=0, eps=0.0, pruner=None, tau=0.0):
    C = fs.Circuit(w.circuit)
    C.set_input(w.inputs)
    b = fs.Batch(split=split, c1=c1, c2=c2)
    b.add(C, w.outputs, eps)
    if pruner is not None:
        learned.attach(b, 0, pruner, tau)
    b.plan()
    b.allocate()
    b.upload()
    b.run()
    st = b.finish()[0]
    return b.amp.cpu().numpy()[:len(w.outputs)], st


def test_learned_pruner_gain_over_threshold_on_the_walk():
    """What the trained network adds: on the 100-qubit walk most checkpoint
    entries can no longer reach the input (their subtree sums are exactly
    zero).  The pruner learns to cut them and keeps the fidelity; threshold
    pruning cannot, because every branch at a given depth has the same
    magnitude (1/sqrt2)^k, so any eps either cuts nothing or cuts whole
    depths."""
    from workloads import qw_workload
    tr = qw_workload(n_out=256, seed=0x5EED0005 + 300)
    ev = qw_workload(n_out=512, seed=0x5EED0005 + 400)
    bv = fs.Circuit(ev.circuit).branch_vars()
    src_gate = {s: g for g, q, s in bv if s >= 0}
    G = len(ev.circuit.gates)
    c1, c2 = G - src_gate[7], G - src_gate[10]          # 8 sources before, 3 in the root
    x, t, _ = learned.log_training_data(tr.circuit, tr.inputs, tr.outputs, c1)
    params, _ = learned.train(x, t, mlp_init_params(1), steps=1200, batch=16384, lr=1e-3)
    exact, st_ex = _qw_run(ev)
    a, st = _qw_run(ev, "fixed", c1, c2, pruner=params, tau=-9.0)
    F = closed_forms.fidelity(exact, a)
    assert F >= 0.999
    assert st["completed"] < 0.1 * st_ex["completed"]
    gains = []
    for eps in (1e-4, 1e-3, 3e-3, 6e-3, 1e-2):
        a2, s2 = _qw_run(ev, "fixed", c1, c2, eps=eps)
        F2 = closed_forms.fidelity(exact, a2)
        gains.append((eps, F2, s2["completed"]))
        assert F2 < 0.999 or s2["completed"] == st_ex["completed"], (eps, F2, s2["completed"])
    print("learned:", F, st["completed"], "of", st_ex["completed"], "threshold:", gains)

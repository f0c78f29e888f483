"""Exact reachability bound at the checkpoint (fs_batch_set_exact_bound):
entries whose state cannot reach the input through the remaining ops are
cut; the amplitudes stay exact.  On the coined walk every step moves the
position by one through a controlled +1 and a controlled -1 cascade, so the
library's bound allows a distance of two per remaining step (two cascades)
and checks the untouched ancilla; the expected cuts are counted here from
the oracle's checkpoint tables with that rule."""
import numpy as np
import pytest

from workloads import qw_workload
from oracle import feynman
import paper_2608_01467_b300 as fs

pytestmark = pytest.mark.gpu

POS = 96


def _run(w, c1, bound):
    C = fs.Circuit(w.circuit)
    C.set_input(w.inputs)
    b = fs.Batch(split="fixed", c1=c1, c2=c1)
    b.add(C, w.outputs)
    if bound:
        b.set_exact_bound(0)
    b.plan()
    b.allocate()
    b.upload()
    b.run()
    st = b.finish()[0]
    return b.amp.cpu().numpy()[:len(w.outputs)], st


@pytest.mark.parametrize("k_prefix", [3, 5])
def test_exact_bound_cuts_the_unreachable_entries_and_keeps_the_amplitudes(k_prefix):
    steps = 8
    w = qw_workload(steps=steps, n_out=128)
    G = len(w.circuit.gates)
    c1 = k_prefix * (G // steps)                  # the last k_prefix steps form the prefix
    left = steps - k_prefix
    exact, st0 = _run(w, c1, False)
    got, st = _run(w, c1, True)
    err = np.abs(got - exact)
    assert np.all(err <= 1e-12 + 1e-10 * np.abs(exact)), err.max()
    mask = (1 << POS) - 1
    expect, zero_cut = 0, 0
    for b_out in w.outputs:
        for b_in, _ in w.inputs:
            t = feynman.checkpoints(w.circuit, b_in, b_out, c1)
            for s, live, sub in zip(t["state"], t["live"], t["subtree"]):
                if not live:
                    continue
                x, y = (s >> 1) & mask, (b_in >> 1) & mask
                dist = min((x - y) & mask, (y - x) & mask)
                if dist > 2 * left or ((s ^ b_in) >> (POS + 3)) & 1:
                    expect += 1
                    zero_cut += sub == 0
    assert st["bound_cuts"] == expect == zero_cut > 0
    assert st["live_entries"] == st0["live_entries"] - expect
    assert st["valid"] == st0["valid"]
    assert st["completed"] < st0["completed"]


def test_learned_pruner_on_top_of_the_exact_bound():
    """With both, the table is compacted after the bound and the pruner
    scores only the live entries, marking its cuts in place: with tau below
    every score nothing more is cut and the amplitudes stay exact; with tau
    above every score every live entry is cut and the amplitudes are zero."""
    import torch
    from workloads import mlp_init_params
    from paper_2608_01467_b300 import learned
    steps = 8
    w = qw_workload(steps=steps, n_out=128)
    G = len(w.circuit.gates)
    c1 = 3 * (G // steps)
    exact, st0 = _run(w, c1, False)
    _, stb = _run(w, c1, True)
    params = torch.from_numpy(np.asarray(mlp_init_params(3), np.float32)).cuda()
    for tau, expect_cut in ((-1e30, False), (1e30, True)):
        C = fs.Circuit(w.circuit)
        C.set_input(w.inputs)
        b = fs.Batch(split="fixed", c1=c1, c2=c1)
        b.add(C, w.outputs)
        b.set_exact_bound(0)
        learned.attach(b, 0, params, tau)
        b.plan()
        b.allocate()
        b.upload()
        b.run()
        st = b.finish()[0]
        got = b.amp.cpu().numpy()[:len(w.outputs)]
        assert st["bound_cuts"] == stb["bound_cuts"]
        if expect_cut:
            assert st["learned_cuts"] == stb["live_entries"] and st["live_entries"] == 0
            assert np.all(got == 0) and st["completed"] == 0
        else:
            assert st["learned_cuts"] == 0 and st["live_entries"] == stb["live_entries"]
            err = np.abs(got - exact)
            assert np.all(err <= 1e-12 + 1e-10 * np.abs(exact)), err.max()


def _cut_run(w, c1, c2, engine="straight", bound=True, tau=None, outputs=None):
    import torch
    from workloads import mlp_init_params
    from paper_2608_01467_b300 import learned
    outs = w.outputs if outputs is None else outputs
    C = fs.Circuit(w.circuit)
    C.set_input(w.inputs)
    b = fs.Batch(engine=engine, prefix="single")
    b.add(C, outs)
    if bound:
        b.set_exact_bound(0)
    if tau is not None:
        params = torch.from_numpy(np.asarray(mlp_init_params(3), np.float32)).cuda()
        learned.attach(b, 0, params, tau)
    b.set_cuts(0, c1, c2)
    b.plan()
    b.allocate()
    b.upload()
    b.amp.fill_(complex(float("nan"), float("nan")))   # every output must be written
    b.run()
    st = b.finish()[0]
    return b.amp.cpu().numpy()[:len(outs)], st, b.launch_count()


def test_compacted_history_reduces_its_own_outputs():
    """An exact compacted job on the generated engine with A_r >= 5 leaves
    no reduction launch: the warp that stores an output's last subtree sum
    adds the output's sums (Eq. 2).  Outputs without a live entry come out
    as exact zeros, outputs with up to 64 sums (the exact bound leaves a few
    entries per output) and with more (a pruner that cuts nothing leaves
    all 32 entries x 8 sums) agree with the interpreter's separate
    reduction and with the plain exact run, every output is written, and a
    sub-request gives the same doubles as the full request.  A pruner on top
    of the bound scores the live entries in the kernel that writes the
    compaction; cutting nothing, it leaves the amplitudes bitwise as they
    are."""
    w = qw_workload(steps=16, n_out=512)
    G = len(w.circuit.gates)
    src = {s: g for g, q, s in fs.Circuit(w.circuit).branch_vars() if s >= 0}
    c1, c2 = G - src[3], G - src[11]            # A_p = 4, A_r = 8
    exact, _, _ = _cut_run(w, c1, c2, bound=False)
    tol = lambda x, y: np.all(np.abs(x - y) <= 1e-12 + 1e-10 * np.abs(y))
    got, st, n = _cut_run(w, c1, c2)
    assert n == 3 and np.all(np.isfinite(got.view(np.float64)))
    assert tol(got, exact), np.abs(got - exact).max()
    zero = got == 0
    assert zero.sum() > 0 and np.all(np.abs(exact[zero]) <= 1e-12)
    ref, st_i, n_i = _cut_run(w, c1, c2, engine="interp")
    assert n_i == 5 and tol(got, ref) and st["live_entries"] == st_i["live_entries"]
    # a pruner on top of the bound that cuts nothing: its kernel also writes
    # the compaction (prefix, scorer, history), the same doubles
    bp, st_bp, n_bp = _cut_run(w, c1, c2, tau=-1e30)
    assert n_bp == 3 and st_bp["learned_cuts"] == 0 and st_bp["live_entries"] == st["live_entries"]
    assert np.array_equal(bp, got)
    bp_i, _, n_bpi = _cut_run(w, c1, c2, engine="interp", tau=-1e30)
    assert n_bpi == 5 and np.array_equal(bp_i, ref)
    # the pruner alone, cutting nothing: 256 sums for every output
    allv, st_a, n_a = _cut_run(w, c1, c2, bound=False, tau=-1e30)
    assert n_a == 4 and st_a["learned_cuts"] == 0    # prune, write, history (+ the prefix)
    assert np.all(np.isfinite(allv.view(np.float64))) and tol(allv, exact)
    ref_a, _, _ = _cut_run(w, c1, c2, engine="interp", bound=False, tau=-1e30)
    assert tol(allv, ref_a)
    # outputs alone: the same doubles
    idx = list(range(0, 512, 7))
    sub, _, _ = _cut_run(w, c1, c2, outputs=[w.outputs[i] for i in idx])
    assert np.array_equal(sub, got[idx])
    sub_a, _, _ = _cut_run(w, c1, c2, bound=False, tau=-1e30, outputs=[w.outputs[i] for i in idx])
    assert np.array_equal(sub_a, allv[idx])


def test_scorer_cuts_on_the_bound_are_those_of_the_network_and_repeat_bitwise():
    """A pruner on top of the bound that cuts about half of the live
    entries.  The scoring kernel spreads a compaction block's live entries
    over several CTAs, each listing the block's entries while the others may
    already be cutting some: every CTA must list the same entries.  The cuts
    are exactly the live entries the same network scores below tau (its
    forward pass over the job's features), the entries left are the bound's
    live ones minus those, repeated runs give the same doubles and counts,
    and the generated and interpreted histories over the same compaction
    agree."""
    import ctypes
    import torch
    from workloads import mlp_init_params
    from paper_2608_01467_b300 import _lib, learned
    w = qw_workload(steps=16, n_out=512)
    G = len(w.circuit.gates)
    src = {s: g for g, q, s in fs.Circuit(w.circuit).branch_vars() if s >= 0}
    c1, c2 = G - src[3], G - src[11]            # A_p = 4, A_r = 8
    params = torch.from_numpy(np.asarray(mlp_init_params(3), np.float32)).cuda()
    # the bound alone: its live entries and their scores
    C = fs.Circuit(w.circuit)
    C.set_input(w.inputs)
    b = fs.Batch(prefix="single")
    b.add(C, w.outputs)
    b.set_exact_bound(0)
    b.set_cuts(0, c1, c2)
    b.plan()
    b.allocate()
    b.upload()
    b.run()
    st_b = b.finish()[0]
    n_ent = len(w.outputs) * len(w.inputs) << st_b["A_p"]
    feat = torch.empty((n_ent, 16), dtype=torch.float32, device="cuda")
    _lib.check(_lib.load().fs_batch_features(b._h, 0, ctypes.c_void_p(b.ws_ptr), ctypes.c_void_p(feat.data_ptr()),
                                             ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)))
    live = ~torch.isnan(feat[:, 0])
    assert int(live.sum()) == st_b["live_entries"]
    # a compaction block holds more live entries than one CTA scores (256)
    assert n_ent % 1024 == 0 and int(live.view(-1, 1024).sum(1).max()) > 256
    score = learned.forward(params, feat[live].contiguous()).cpu().numpy()
    tau = float(np.median(score))
    below = int((score < tau).sum())
    assert 0 < below < len(score)
    runs = [_cut_run(w, c1, c2, tau=tau) for _ in range(3)]
    amp, st, n = runs[0]
    assert n == 3 and st["learned_cuts"] == below
    assert st["live_entries"] == st_b["live_entries"] - below
    for a2, s2, _ in runs[1:]:
        assert np.array_equal(a2, amp)
        assert all(s2[k] == st[k] for k in ("learned_cuts", "live_entries", "completed", "valid"))
    # (the interpreter does not test the bound inside the suffix, so its
    # completed count is larger; the live entries and amplitudes agree)
    ref, st_i, _ = _cut_run(w, c1, c2, engine="interp", tau=tau)
    assert st_i["learned_cuts"] == below and st_i["live_entries"] == st["live_entries"]
    assert np.all(np.abs(amp - ref) <= 1e-12 + 1e-10 * np.abs(ref))

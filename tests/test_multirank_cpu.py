"""The N > 1 path of bench.py on the CPU: two gloo ranks rendezvous on
127.0.0.1, take max/sum over ranks and barrier; each rank gets its own
seeded request of the same size (weak scaling, no data-path collective)."""
import os
import socket
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import torch
    import torch.distributed as dist
    import bench
    r, w, _ = bench.dist_setup(None)
    dev = torch.device("cpu")
    mx = bench.max_over_ranks(float(r + 1), w, dev)
    sm = bench.sum_over_ranks(float(10 * (r + 1)), w, dev)
    bench.barrier(w)
    jobs, cfg = bench.workload_jobs("qw100", r, 64)
    q.put((r, w, mx, sm, len(jobs[0].outputs), jobs[0].meta["p0"]))
    dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [x[1] for x in res] == [2, 2]
    assert all(x[2] == 2.0 for x in res)          # max over ranks
    assert all(x[3] == 30.0 for x in res)         # sum over ranks
    assert res[0][4] == res[1][4] == 64           # same per-rank size
    assert res[0][5] != res[1][5]                 # distinct seeded requests


def _shard_worker(rank, world, port, q):
    """One rank of a sharded request: its LPT share of the outputs is
    evaluated (by the oracle here: the CPU stands in for this rank's GPU),
    then every rank gathers the whole request."""
    sys.path.insert(0, ROOT)
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "MASTER_ADDR": "127.0.0.1",
                       "MASTER_PORT": str(port)})
    import numpy as np
    import torch.distributed as dist
    from workloads import qaoa_workload, qw_workload
    from oracle import feynman
    import paper_2608_01467_b300 as fs
    from paper_2608_01467_b300 import shard
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ws = [qaoa_workload(6, 2, n_out=9, seed=3), qw_workload(steps=5, n_out=14, pos_bits=8)]
    jobs = [(fs.Circuit(w.circuit), w.inputs, w.outputs) for w in ws]
    mine, assign, load = shard.shard(jobs, world, rank)
    local = [feynman.run(w.circuit, w.inputs, [w.outputs[i] for i in idx])[0] if len(idx) else np.zeros(0, complex)
             for w, idx in zip(ws, mine)]
    full = shard.gather(local, mine, jobs)
    q.put((rank, [list(m) for m in mine], list(assign), list(load), [list(a) for a in full]))
    dist.destroy_process_group()


def test_sharded_request_gathers_the_one_rank_result():
    """Output sharding of one request over two gloo ranks (Sec. IV-D,
    Observation 5): every output is assigned to exactly one rank, the LPT
    loads differ by at most one unit's cost, and the gathered amplitudes
    equal the one-rank result."""
    import numpy as np
    from workloads import qaoa_workload, qw_workload
    from oracle import feynman
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=180) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ws = [qaoa_workload(6, 2, n_out=9, seed=3), qw_workload(steps=5, n_out=14, pos_bits=8)]
    want = [feynman.run(w.circuit, w.inputs, w.outputs)[0] for w in ws]
    (_, m0, a0, l0, f0), (_, m1, a1, l1, f1) = res
    assert a0 == a1 and l0 == l1                      # the same assignment on every rank
    for j in range(2):
        assert sorted(m0[j] + m1[j]) == list(range(len(ws[j].outputs)))
        assert not set(m0[j]) & set(m1[j])
    import paper_2608_01467_b300 as fs
    from paper_2608_01467_b300 import shard
    costs = shard.unit_costs([(fs.Circuit(w.circuit), w.inputs, w.outputs) for w in ws])
    assert abs(l0[0] - l0[1]) <= max(costs)            # LPT: within one unit's cost
    for full in (f0, f1):
        for got, exp in zip(full, want):
            assert np.max(np.abs(np.asarray(got) - exp)) == 0.0


def test_lpt_assignment_properties():
    import numpy as np
    from paper_2608_01467_b300 import shard
    rng = np.random.default_rng(5)
    costs = rng.integers(1, 100, size=57).astype(float)
    for world in (1, 2, 3, 8):
        rank, load = shard.lpt_assign(costs, world)
        assert rank.max() < world and len(rank) == len(costs)
        assert np.allclose([costs[rank == r].sum() for r in range(world)], load)
        assert load.max() - load.min() <= costs.max()
    r2, _ = shard.lpt_assign(costs, 3)
    assert np.array_equal(r2, shard.lpt_assign(costs, 3)[0])   # deterministic

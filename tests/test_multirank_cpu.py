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

"""Output sharding of one request across ranks (argument marshalling and
torch.distributed plumbing only).

The outputs of a request are independent (Sec. IV-D, Observation 5), so a
request can be split over processes, one GPU each, with no exchange until
the amplitudes are gathered.  Their costs differ between circuits
(Observation 6): every (job, output) unit is weighed by S x Eq. 8 of its
circuit (the library's autotuned gate-operation count) and the units are
assigned by longest-processing-time-first in the library (fs_lpt_assign).
Every rank computes the same assignment; rank r runs the units assigned to
it; `gather` returns all amplitudes, in request order, on every rank.
"""
from __future__ import annotations

import ctypes
from typing import List, Sequence, Tuple

import numpy as np

from . import _lib
from ._lib import check


def lpt_assign(costs: Sequence[float], world: int) -> Tuple[np.ndarray, np.ndarray]:
    """(rank of every unit, summed cost per rank)."""
    c = np.ascontiguousarray(costs, dtype=np.float64)
    rank = np.zeros(max(len(c), 1), np.uint32)
    load = np.zeros(max(world, 1), np.float64)
    check(_lib.load().fs_lpt_assign(c.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), len(c), int(world),
                                    rank.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
                                    load.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return rank[:len(c)], load


def unit_costs(jobs) -> List[float]:
    """jobs: [(Circuit, inputs, outputs)]; one cost per (job, output):
    S x Eq. 8 at the circuit's autotuned cuts."""
    costs = []
    for circ, inputs, outputs in jobs:
        eq8 = float(circ.analyze(0)["gateops"])
        circ.set_input(inputs)
        costs += [len(inputs) * eq8] * len(outputs)
    return costs


def shard(jobs, world: int, rank: int):
    """This rank's part of the request: per job the indices of its outputs,
    plus the full assignment (unit order = jobs' outputs in order)."""
    assign, load = lpt_assign(unit_costs(jobs), world)
    mine, off = [], 0
    for _, _, outputs in jobs:
        a = assign[off:off + len(outputs)]
        mine.append(np.nonzero(a == rank)[0])
        off += len(outputs)
    return mine, assign, load


def gather(local: Sequence[np.ndarray], mine, jobs, group=None) -> List[np.ndarray]:
    """Every rank's amplitudes of its units, reassembled per job in request
    order on every rank (one all_gather of the per-rank arrays)."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    parts = [None] * world
    dist.all_gather_object(parts, [(np.asarray(m), np.asarray(a)) for m, a in zip(mine, local)], group=group)
    out = [np.zeros(len(outputs), complex) for _, _, outputs in jobs]
    for per_rank in parts:
        for j, (idx, amp) in enumerate(per_rank):
            out[j][idx] = amp
    return out

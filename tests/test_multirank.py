"""The benchmark's multi-process path on the CPU: two ranks over gloo.

One process per GPU runs its own replica (or its own ensemble members); the
only cross-rank steps are the reductions of the timing harness: the job's
time is the slowest rank's, its units are the sum over ranks, and the
ensemble ranks draw disjoint member seeds.  No GPU is touched.
"""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import bench
    from paper_1701_06254_gb300 import inputs as I
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        secs = [1.5, 2.25][rank]                      # rank 1 is the slowest
        mx = bench.rank_max(secs, dist, "cpu")
        cases = I.ensemble(3, seed0=bench.ensemble_seed0(rank, 3), size_lo=(5, 4, 2), size_hi=(9, 8, 3))
        cells = sum(c.n for c in cases)
        tot = bench.rank_sum(cells, dist, "cpu")
        seeds = [bench.ensemble_seed0(rank, 3) + k for k in range(3)]
        gathered = [None] * world
        dist.all_gather_object(gathered, (cells, seeds))
        out[rank] = (mx, tot, gathered)
    finally:
        dist.destroy_process_group()


def test_two_ranks_reduce_time_and_units():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_worker, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
        res = dict(out)
    for rank in range(world):
        mx, tot, gathered = res[rank]
        assert mx == 2.25                                             # the slowest rank's time
        assert tot == sum(c for c, _ in gathered)                      # units of every rank
        seeds = [set(s) for _, s in gathered]
        assert not (seeds[0] & seeds[1])                               # disjoint members
    # ranks draw different models, so their cell counts differ in general:
    # the whole-job rate must sum them, not scale rank 0's
    c0, c1 = res[0][2][0][0], res[0][2][1][0]
    assert c0 != c1


def test_single_process_reductions_are_identity():
    import bench
    assert bench.rank_max(3.5, None, "cpu") == 3.5
    assert bench.rank_sum(7, None, "cpu") == 7.0
    assert bench.ensemble_seed0(0, 128) == 2000 and bench.ensemble_seed0(2, 128) == 2256

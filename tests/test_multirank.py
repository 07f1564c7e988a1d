"""Host logic of the multi-GPU bench path, on CPU with the gloo backend (world size 2):

  * the scan's run partition (greedy longest-first by cells) gives every run to exactly one
    rank, and the heaviest rank carries at most the lightest rank's cells plus one run;
  * two processes agree on their shares without communication (each computes the same
    partition), and their union, gathered over gloo, is the whole table;
  * the timing reduction returns the slowest rank's values on every rank.
"""
import os
import socket

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_partition_covers_and_balances():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    import pic_inputs as pi
    table = pi.scan_table(256, seed=4)
    for world in (1, 2, 3, 8):
        parts = bench._partition(table, world)
        flat = sorted(r for p in parts for r in p)
        assert flat == list(range(len(table)))
        loads = [sum(table[r][0] * table[r][1] for r in p) for p in parts]
        biggest = max(t[0] * t[1] for t in table)
        assert max(loads) - min(loads) <= biggest


def _worker(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    import pic_inputs as pi
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        table = pi.scan_table(256, seed=4)
        mine = bench._partition(table, world)[rank]
        gathered = [None] * world
        dist.all_gather_object(gathered, mine)
        times = bench._max_over_ranks(dist, [10.0 + rank, 5.0 - rank], device="cpu")
        q.put((rank, gathered, times))
    finally:
        dist.destroy_process_group()


def test_two_ranks_gloo():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    import sys
    sys.path.insert(0, ROOT)
    import pic_inputs as pi
    n = len(pi.scan_table(256, seed=4))
    for rank, gathered, times in out:
        assert sorted(r for g in gathered for r in g) == list(range(n))
        assert not set(gathered[0]) & set(gathered[1])
        assert times == [11.0, 5.0]

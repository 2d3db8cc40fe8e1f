"""World-size-2 gloo tests of the N>1 host logic on CPU.

Each rank takes its owned range from paper_1403_7294_gb300.shard, scans its
read window (the oracle stands in for the device scan here: this checks the
splitting, ownership and gather logic, not the kernels), and the gathered
result must equal one scan of the whole text. The benchmark's max-over-ranks
timing reduction is exercised too."""
import os
import random
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1403_7294_gb300 import shard


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle

        rng = random.Random(42)
        text = bytes(rng.choice(b"ACGT") for _ in range(20011))
        pats = [text[j : j + rng.randint(4, 16)] for j in rng.sample(range(20000), 80)] + [b"ACGTACGTACGT"]
        lmax = max(len(p) for p in pats)
        lens = np.array([len(p) for p in pats])
        b, e = shard.owned_range(len(text), world, rank)
        rb, re_ = shard.read_window(b, e, lmax)
        pos, pid, _ = oracle.Machine(pats).scan(text[rb:re_])
        end = pos.astype(np.int64) + lens[pid] - 1 + rb
        keep = (end >= b) & (end < e)
        mine = np.stack([np.zeros(keep.sum(), np.int64), pos[keep].astype(np.int64) + rb, pid[keep].astype(np.int64)], 1)
        parts = [None] * world
        dist.all_gather_object(parts, mine)
        import bench

        t = bench.max_over_ranks(float(rank + 1), world)
        if rank == 0:
            full_pos, full_pid, _ = oracle.Machine(pats).scan(text)
            full = shard.gather_occurrences([np.stack([np.zeros(len(full_pos), np.int64), full_pos.astype(np.int64),
                                                       full_pid.astype(np.int64)], 1)])
            got = shard.gather_occurrences(parts)
            q.put((bool(np.array_equal(got, full)), len(full), t))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_sharded_scan_equals_one_scan(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    [p.start() for p in procs]
    [p.join(120) for p in procs]
    assert all(p.exitcode == 0 for p in procs)
    ok, n, t = q.get(timeout=10)
    assert ok and n > 80
    assert t == float(world)  # max over ranks


def test_owned_ranges_partition():
    for n in (0, 1, 63, 64, 65, 1000, 12345):
        for world in (1, 2, 3, 8):
            rs = [shard.owned_range(n, world, r) for r in range(world)]
            assert rs[0][0] == 0 and rs[-1][1] == n
            for (a, b), (c, d) in zip(rs[:-1], rs[1:]):
                assert b == c and a <= b
            assert all(a % 64 == 0 for a, _ in rs)

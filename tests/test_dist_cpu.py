"""Multi-rank exchange (reduce-scatter of state blocks + all-gather of
finalized values) on CPU ranks over gloo: the result equals the one-rank
result bit for bit, for any G (including blocks left empty), both dtypes,
and a data error on one rank reaches every rank."""
import socket

import pytest
import torch.multiprocessing as mp

from paper_1802_09883_gb300 import dist as D

import dist_workers as W


def _port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_shard_range_covers_rows_with_aligned_boundaries():
    for n in (0, 1, 5, 1000, 1001, 4097):
        for world in (1, 2, 3, 8):
            rs = [D.shard_range(n, r, world) for r in range(world)]
            assert rs[0][0] == 0 and rs[-1][1] == n
            for (a, b), (c, d) in zip(rs, rs[1:]):
                assert b == c and a <= b
            assert all(lo % 4 == 0 for lo, hi in rs if hi > lo)  # empty tail shards sit at n


def test_group_blocks_partition_the_groups():
    for G in (1, 2, 7, 1024, 1025):
        for world in (1, 2, 3, 8):
            bl = D.group_blocks(G, world)
            assert bl[0][0] == 0 and bl[-1][1] == G
            sizes = [b - a for a, b in bl]
            assert max(sizes) - min(sizes) <= 1


@pytest.mark.parametrize("n,G,L,dt,bad", [
    (200_003, 1024, 3, "f64", -1),
    (50_001, 1, 2, "f64", -1),      # one group: rank 1's block is empty
    (60_000, 777, 3, "f32", -1),
    (30_000, 64, 3, "f64", 1),      # a bad key on rank 1 only
])
def test_two_rank_exchange_equals_one_rank(n, G, L, dt, bad):
    mp.spawn(W.exchange_body, args=(2, _port(), n, G, L, dt, bad), nprocs=2, join=True)

"""Rank bodies for the multi-process (gloo, CPU) tests of the exchange in
paper_1802_09883_gb300.dist.  The per-rank aggregation and the merge are
the CPU oracle's, standing in for the device kernels: what is tested here is
the host protocol (sharding, block reduce-scatter, all-gather, error OR)."""
import os

import numpy as np
import torch
import torch.distributed as dist

from oracle import oracle as O
from paper_1802_09883_gb300 import dist as D
from paper_1802_09883_gb300 import workloads as WL


def _init(rank, world, port):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)


def oracle_merge_fn(dtype, L):
    def merge(dst, src):
        g = dst.shape[0]
        a = O.State(np.dtype(dtype), L, g, dst.numpy().reshape(-1))
        b = O.State(np.dtype(dtype), L, g, src.numpy().reshape(-1))
        O.merge(a, b)  # in place on dst's memory
    return merge


def exchange_body(rank, world, port, n, G, L, dtype_name, bad_rank):
    _init(rank, world, port)
    try:
        dtype = np.float64 if dtype_name == "f64" else np.float32
        w = WL.plain(n=n, G=G, L=L, seed=11, device="cpu",
                     dtype=torch.float64 if dtype == np.float64 else torch.float32)
        keys, vals = w.keys.numpy(), w.values.numpy()
        lo, hi = D.shard_range(n, rank, world)
        k = keys[lo:hi].copy()
        if rank == bad_rank and k.size:
            k[0] = G  # one bad key on this rank only
        st = O.init(dtype, L, G)
        bad = O.groupby_sum(st, k, vals[lo:hi])
        rec = st.buf.size // G
        records = torch.from_numpy(st.buf).view(G, rec)
        g0, g1, mine = D.reduce_scatter_records(records, oracle_merge_fn(dtype, L))
        blk = O.State(np.dtype(dtype), L, g1 - g0, mine.numpy().reshape(-1))
        vals_blk = torch.from_numpy(O.finalize(blk)) if g1 > g0 else torch.empty(0, dtype=torch.from_numpy(
            np.empty(0, dtype)).dtype)
        full = D.allgather_blocks(vals_blk, G).numpy()
        errors = D.or_over_ranks(int(bad > 0))
        # the whole input on one rank (bad rows skipped the same way)
        kk = keys.copy()
        if bad_rank >= 0:
            lo_b, hi_b = D.shard_range(n, bad_rank, world)
            if hi_b > lo_b:
                kk[lo_b] = G
        ref_st = O.init(dtype, L, G)
        O.groupby_sum(ref_st, kk, vals)
        ref = O.finalize(ref_st)
        iv = np.int64 if dtype == np.float64 else np.int32
        assert np.array_equal(full.view(iv), ref.view(iv)), "exchange result differs from one-rank result"
        assert errors == (1 if bad_rank >= 0 else 0)
        assert D.max_over_ranks(float(rank)) == world - 1
    finally:
        dist.destroy_process_group()

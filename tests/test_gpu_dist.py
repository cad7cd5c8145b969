"""Device side of the multi-rank exchange: merging record blocks with the
library's merge kernel equals aggregating the rows together, and the
single-rank NCCL path of allreduce_groupby returns the plain result."""
import os
import socket

import numpy as np
import pytest
import torch

import paper_1802_09883_gb300 as R
from paper_1802_09883_gb300 import dist as D
from paper_1802_09883_gb300 import workloads as WL

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _bits(t):
    a = t.detach().cpu().numpy()
    return a.view(np.int64 if a.dtype == np.float64 else np.int32)


@pytest.mark.parametrize("G,L", [(1024, 3), (5000, 2)])
def test_device_merge_of_record_blocks(G, L):
    w = WL.sweep_cell(G, "uniform", L, n=1 << 20, seed=7, device=DEV)
    half = (w.n // 2) // 4 * 4
    a, b, whole = R.State(G, L), R.State(G, L), R.State(G, L)
    a.add(w.keys[:half], w.values[:half])
    b.add(w.keys[half:], w.values[half:])
    whole.add(w.keys, w.values)
    H = R.HEADER_BYTES
    rec = (a.tensor.numel() - H) // G
    ra, rb = a.tensor[H:].view(G, rec), b.tensor[H:].view(G, rec)
    g0, g1 = 100, 900  # a block in the middle, as one rank would own it
    blk = ra[g0:g1].clone()
    D.device_merge(torch.float64, L)(blk, rb[g0:g1].contiguous())
    assert torch.equal(blk, whole.tensor[H:].view(G, rec)[g0:g1])


def test_allreduce_groupby_single_rank_nccl():
    import torch.distributed as dist
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    store = dist.TCPStore("127.0.0.1", port, 1, True)
    dist.init_process_group("nccl", store=store, rank=0, world_size=1)
    try:
        w = WL.plain(n=300_000, G=1000, L=3, seed=3, device=DEV)
        st = R.State(1000, 3)
        st.add(w.keys, w.values)
        out = D.allreduce_groupby(st)
        assert np.array_equal(_bits(out), _bits(st.finalize()))
    finally:
        dist.destroy_process_group()

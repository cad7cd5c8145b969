"""Reproducible SUM without GROUP BY: the keyless single-pass kernel gives
the bytes of a one-group grouped SUM and the oracle's result, for aligned
and unaligned inputs, splits and specials."""
import numpy as np
import pytest
import torch

import paper_1802_09883_gb300 as R
from paper_1802_09883_gb300 import workloads as WL
from oracle import oracle as O

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _oracle_sum(v, L):
    vn = v.cpu().numpy()
    return O.groupby_sum_values(np.zeros(vn.size, np.int32), vn, 1, L, dtype=vn.dtype, threads=4)


@pytest.mark.parametrize("dtype,L,n", [(torch.float64, 3, 1 << 22), (torch.float64, 2, 1_000_003),
                                       (torch.float32, 3, 3_000_001), (torch.float64, 4, 5)])
def test_scalar_sum_matches_grouped_and_oracle(dtype, L, n):
    g = torch.Generator(device=DEV)
    g.manual_seed(n + L)
    v = WL.random_values(n, -60, 60, g, DEV, dtype)
    keyless = R.State(1, L, dtype).add_values(v)
    grouped = R.State(1, L, dtype)
    grouped.add(torch.zeros(n, dtype=torch.int32, device=DEV), v)
    torch.cuda.synchronize()
    assert torch.equal(keyless.tensor, grouped.tensor)
    got = R.scalar_sum(v, L).cpu().numpy().reshape(1)
    ref = _oracle_sum(v, L)
    iv = np.int64 if got.dtype == np.float64 else np.int32
    assert got.view(iv)[0] == ref.view(iv)[0]


def test_scalar_sum_unaligned_split_and_order():
    g = torch.Generator(device=DEV)
    g.manual_seed(17)
    v = WL.random_values(1_000_001, -30, 30, g, DEV)
    whole = R.State(1, 3).add_values(v)
    parts = R.State(1, 3).add_values(v[1:]).add_values(v[:1])  # v[1:] starts 8 bytes past alignment
    perm = R.State(1, 3).add_values(v[torch.randperm(v.numel(), device=DEV)])
    torch.cuda.synchronize()
    assert torch.equal(whole.tensor, parts.tensor) and torch.equal(whole.tensor, perm.tensor)


def test_scalar_sum_specials_and_empty():
    v = torch.tensor([1.0, float("inf"), -2.0], dtype=torch.float64, device=DEV)
    assert torch.isinf(R.scalar_sum(v)).item()
    assert R.scalar_sum(v[:0]).item() == 0.0
    st = R.State(4, 3)  # not a one-group state: refused on the host
    with pytest.raises(ValueError):
        st.add_values(v)


def test_host_columns_match_device_columns():
    g = torch.Generator(device=DEV)
    g.manual_seed(23)
    n, G = (1 << 25) + 12345, 1000  # three staged chunks, the last ragged
    keys = WL.uniform_keys(n, G, g, DEV)
    vals = WL.random_values(n, -40, 40, g, DEV)
    dev_state = R.State(G, 3)
    dev_state.add(keys, vals)
    kh, vh = keys.cpu().pin_memory(), vals.cpu().pin_memory()
    host_state = R.State(G, 3).add_host(kh, vh)
    torch.cuda.synchronize()
    assert torch.equal(dev_state.tensor, host_state.tensor)
    with pytest.raises(ValueError):  # pageable host memory
        R.State(G, 3).add_host(keys.cpu(), vals.cpu())

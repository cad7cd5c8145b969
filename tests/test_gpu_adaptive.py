"""repro_groupby_sum_adaptive: the partitioning depth picked from the keys'
range (none, one or two passes) gives the bytes repro_groupby_sum gives,
and the oracle's, whichever depth it takes."""
import os

import numpy as np
import pytest
import torch

import paper_1802_09883_gb300 as R
from paper_1802_09883_gb300 import workloads as WL
from oracle import oracle as O

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _rows(n, span, seed, dtype=torch.float64):
    g = torch.Generator(device=DEV)
    g.manual_seed(seed)
    keys = WL.uniform_keys(n, span, g, DEV)
    vals = WL.random_values(n, -40, 40, g, DEV, dtype)
    return keys, vals


def _both(keys, vals, G, L):
    a, b = R.State(G, L, vals.dtype), R.State(G, L, vals.dtype)
    depth = a.add_adaptive(keys, vals)
    b.add(keys, vals)
    torch.cuda.synchronize()
    return depth, a, b


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_narrow_key_range_takes_no_partitioning(dtype):
    """Keys in [0, 1500) under num_groups = 2^20: one single pass over the
    first 1500 records; the rest of the state stays empty."""
    G, L, span = 1 << 20, 3, 1500
    keys, vals = _rows((1 << 22) + 3, span, 5, dtype)
    depth, a, b = _both(keys, vals, G, L)
    assert depth == 0
    assert a.check() == 0
    assert torch.equal(a.tensor, b.tensor)
    npd = np.float64 if dtype == torch.float64 else np.float32
    ost = O.init(npd, L, span)
    O.groupby_sum(ost, keys.cpu().numpy(), vals.cpu().numpy(), threads=os.cpu_count() or 1)
    K, fl, lo, hi = a.host_view()
    oK, ofl, olo, ohi = O.to_bins(ost)
    assert np.array_equal(K[:span], oK) and np.array_equal(fl[:span], ofl)
    assert np.array_equal(lo[:span], olo) and np.array_equal(hi[:span], ohi)
    assert not K[span:].any() and not fl[span:].any() and not lo[span:].any() and not hi[span:].any()
    out = a.finalize().cpu().numpy()
    iv = np.int64 if npd == np.float64 else np.int32
    assert np.array_equal(out[:span].view(iv), O.finalize(ost).view(iv))


def test_medium_key_range_takes_one_pass_instead_of_two():
    """Keys in [0, 40000) under num_groups = 2^24 (two passes for the declared
    count): one pass sized for 40000 groups, the same bytes."""
    G, L = 1 << 24, 2
    keys, vals = _rows(1 << 22, 40_000, 7)
    depth, a, b = _both(keys, vals, G, L)
    assert depth == 1
    assert a.check() == 0
    assert torch.equal(a.tensor, b.tensor)


@pytest.mark.parametrize("G,L,dist,want", [(1 << 20, 3, "zipf", 1), (1 << 20, 3, "uniform", 1),
                                           (1 << 20, 4, "uniform", 2), (1 << 20, 4, "zipf", 1),
                                           (1 << 16, 3, "zipf", 1), (1 << 16, 3, "uniform", 1)])
def test_full_key_range_keeps_the_rule_depth(G, L, dist, want):
    """Keys over all groups: uniform keys keep the rule's plan (one pass
    into 1024 partitions at 2^20 groups and L = 3, two passes over 2048 at
    L = 4, one over 64 at 2^16); Zipf keys are skewed (the fullest partition
    far above the mean), so the call goes over to one pass -- into 2^7-group
    partitions with lane-private table copies at 2^16, into 1024 partitions
    instead of two passes at 2^20 and L = 4 -- the same bytes either way,
    and the oracle's."""
    R.tune_clear()  # the rule's choices, not a measured one
    w = WL.sweep_cell(G, dist, L, n=1 << 22, seed=9, device=DEV)
    depth, a, b = _both(w.keys, w.values, G, L)
    assert depth == want
    assert torch.equal(a.tensor, b.tensor)
    ost = O.init(np.float64, L, G)
    O.groupby_sum(ost, w.keys.cpu().numpy(), w.values.cpu().numpy(), threads=4)
    K, fl, lo, hi = a.host_view()
    oK, ofl, olo, ohi = O.to_bins(ost)
    assert np.array_equal(K, oK) and np.array_equal(lo, olo) and np.array_equal(hi, ohi)


def test_bad_keys_and_unaligned_columns_go_the_plain_way():
    """A key outside [0, G) keeps the plan for the declared count (which
    flags it, as repro_groupby_sum does); unaligned columns skip the range
    read altogether."""
    G, L = 1 << 20, 3
    keys, vals = _rows(100_003, 2000, 11)
    keys[77] = G + 3
    depth, a, b = _both(keys, vals, G, L)
    assert depth in (1, 2)
    with pytest.raises(R.ReproError):
        a.check()
    assert torch.equal(a.tensor, b.tensor)
    keys, vals = _rows(100_004, 2000, 12)
    depth, a, b = _both(keys[1:], vals[1:], G, L)  # 4- and 8-byte aligned only
    assert depth == -1
    assert torch.equal(a.tensor, b.tensor)


def test_small_declared_count_needs_no_probe():
    keys, vals = _rows(200_000, 1000, 13)
    depth, a, b = _both(keys, vals, 1000, 3)
    assert depth == 0
    assert torch.equal(a.tensor, b.tensor)

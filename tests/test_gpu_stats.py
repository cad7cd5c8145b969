"""COUNT / SUM / AVG / VARIANCE / STDDEV on the GPU vs the stats oracle,
bit for bit (NaN compared as NaN: its payload is not part of the result)."""
import numpy as np
import pytest
import torch

import paper_1802_09883_gb300 as R
from paper_1802_09883_gb300 import workloads as WL
from oracle import stats as OS

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _same(a, b, name):
    a, b = np.asarray(a), np.asarray(b)
    assert a.dtype == b.dtype and a.shape == b.shape, name
    if a.dtype.kind == "f":
        nan = np.isnan(a)
        assert np.array_equal(nan, np.isnan(b)), name
        iv = np.int64 if a.dtype == np.float64 else np.int32
        bad = np.flatnonzero(a[~nan].view(iv) != b[~nan].view(iv))
        assert bad.size == 0, f"{name}: {bad.size} differ, e.g. {a[~nan][bad[:3]]} vs {b[~nan][bad[:3]]}"
    else:
        assert np.array_equal(a, b), name


def _check_all(got, ref):
    for f in R.STATS_FIELDS:
        _same(got[f].cpu().numpy(), ref[f], f)


@pytest.mark.parametrize("dtype,G,L,n", [(torch.float64, 1000, 3, 1_000_003), (torch.float32, 300, 3, 500_000),
                                         (torch.float64, 70_000, 2, 1 << 20), (torch.float64, 10, 4, 4097)])
def test_stats_match_oracle(dtype, G, L, n):
    g = torch.Generator(device=DEV)
    g.manual_seed(G + L)
    keys = WL.uniform_keys(n, G - 3, g, DEV)  # the last three groups stay empty
    vals = WL.random_values(n, -20, 20, g, DEV, dtype)
    got = R.groupby_stats(keys, vals, G, L)
    ref = OS.groupby_stats(keys.cpu().numpy(), vals.cpu().numpy(), G, L, threads=4)
    _check_all(got, ref)


def test_stats_empty_single_special_and_bad_keys():
    keys = torch.tensor([0, 0, 1, 3, 3, 3, 4, 4, 7], dtype=torch.int32, device=DEV)
    vals = torch.tensor([1.0, 3.0, 2.5, float("inf"), 1.0, 2.0, float("nan"), 1.0, 9.0], dtype=torch.float64,
                        device=DEV)
    st = R.Stats(6, 3).add(keys, vals)
    with pytest.raises(R.ReproError):  # key 7 is out of range
        st.check()
    got = st.finalize()
    ok = keys < 6
    ref = OS.groupby_stats(keys[ok].cpu().numpy(), vals[ok].cpu().numpy(), 6, 3)
    _check_all(got, ref)
    assert got["count"].tolist() == [2, 1, 0, 3, 2, 0]


def test_stats_merge_equals_one_pass():
    g = torch.Generator(device=DEV)
    g.manual_seed(3)
    keys = WL.uniform_keys(300_000, 500, g, DEV)
    vals = WL.random_values(300_000, -30, 30, g, DEV)
    a = R.Stats(500, 3).add(keys[:100_000], vals[:100_000])
    b = R.Stats(500, 3).add(keys[100_000:], vals[100_000:])
    whole = R.Stats(500, 3).add(keys, vals)
    a.merge(b)
    torch.cuda.synchronize()
    assert torch.equal(a.tensor, whole.tensor)

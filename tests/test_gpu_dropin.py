"""The unbuffered drop-in accumulator (repro_accum.cuh) gives the library's
state bytes; the DECIMAL baseline is exact."""
import numpy as np
import pytest
import torch

import paper_1802_09883_gb300 as R
from paper_1802_09883_gb300 import workloads as WL

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.mark.parametrize("dtype,L,e_lo,e_hi", [(torch.float64, 3, -60, 60), (torch.float64, 2, -1060, -1000),
                                               (torch.float32, 3, -140, 20), (torch.float64, 4, 900, 1000)])
def test_dropin_equals_buffered(dtype, L, e_lo, e_hi):
    g = torch.Generator(device=DEV)
    g.manual_seed(L - e_lo)
    v = WL.random_values(1_234_567, e_lo, e_hi, g, DEV, dtype)  # includes subnormal or huge ranges
    a = R.State(1, L, dtype).add_values(v)
    b = R.State(1, L, dtype).add_values_unbuffered(v)
    torch.cuda.synchronize()
    assert torch.equal(a.tensor, b.tensor)


def test_dropin_specials_and_merge_order():
    v = torch.tensor([1.0, -2.5, float("inf"), 3.0, float("-inf")], dtype=torch.float64, device=DEV)
    a = R.State(1, 3).add_values(v)
    b = R.State(1, 3).add_values_unbuffered(v[:2]).add_values_unbuffered(v[2:])
    torch.cuda.synchronize()
    assert torch.equal(a.tensor, b.tensor)
    assert torch.isnan(b.finalize()[0]).item()


def test_decimal_baseline_is_exact():
    g = torch.Generator(device=DEV)
    g.manual_seed(5)
    n, G = 3_000_001, 777
    keys = WL.uniform_keys(n, G + 3, g, DEV)  # a few out-of-range keys are skipped
    vals = torch.randint(-10**12, 10**12, (n,), generator=g, device=DEV, dtype=torch.int64)
    out = R.groupby_sum_decimal64(keys, vals, G).cpu().numpy()
    k, v = keys.cpu().numpy(), vals.cpu().numpy()
    ok = k < G
    ref = np.zeros(G, dtype=np.int64)
    np.add.at(ref, k[ok], v[ok])
    assert np.array_equal(out, ref)
    out_big = R.groupby_sum_decimal64(keys, vals, 100_000).cpu().numpy()  # global-atomic path
    ref_big = np.zeros(100_000, dtype=np.int64)
    np.add.at(ref_big, k, v)
    assert np.array_equal(out_big, ref_big)

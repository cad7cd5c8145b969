"""The unbuffered drop-in accumulator (repro_accum.cuh): its state and
result against the CPU oracle, and against the buffered kernel's bytes; the
DECIMAL baseline is exact."""
import numpy as np
import pytest
import torch

import paper_1802_09883_gb300 as R
from paper_1802_09883_gb300 import workloads as WL
from oracle import oracle as O

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


def _dropin_values(dtype, n, seed):
    """Normal values over the whole exponent range, subnormals, zeros of both
    signs and magnitudes just below the supported limit (2^1005 for double,
    2^120 for float, where the top level's running sum would overflow)."""
    g = torch.Generator(device=DEV)
    g.manual_seed(seed)
    if dtype == torch.float64:
        lo_e, hi_e, sub_bits, lim = -1022, 1003, 52, 2.0 ** 1005
    else:
        lo_e, hi_e, sub_bits, lim = -126, 118, 23, 2.0 ** 120
    v = WL.random_values(n, lo_e, hi_e, g, DEV, dtype)
    k = n // 8
    it = torch.int64 if dtype == torch.float64 else torch.int32
    sub = torch.randint(1, 1 << sub_bits, (k,), generator=g, device=DEV, dtype=torch.int64).to(it).view(dtype)
    v[:k] = sub
    v[k:k + 64] = 0.0
    v[k + 64:k + 128] = -0.0
    npd = np.float64 if dtype == torch.float64 else np.float32
    top = np.nextafter(npd(lim), npd(0))
    v[k + 128:k + 160] = torch.tensor([top, -top] * 16, dtype=dtype, device=DEV)
    return v[torch.randperm(n, generator=g, device=DEV)].contiguous()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("L", [1, 2, 3, 4])
def test_dropin_matches_oracle(dtype, L):
    """repro_accum<T,L> one value at a time per thread, tree-merged: the
    state's K, flags and 128-bit bins and the result bits equal the C
    oracle's (Algorithm 2 per value, Sec. IV's type)."""
    v = _dropin_values(dtype, 300_001, 31 * L + (dtype == torch.float32))
    st = R.State(1, L, dtype).add_values_unbuffered(v)
    out = st.finalize().cpu().numpy()
    assert st.check() == 0
    npd = np.float64 if dtype == torch.float64 else np.float32
    ref = O.init(npd, L, 1)
    assert O.groupby_sum(ref, np.zeros(v.numel(), np.int32), v.cpu().numpy(), threads=4) == 0
    K, fl, lo, hi = st.host_view()
    oK, ofl, olo, ohi = O.to_bins(ref)
    assert np.array_equal(K, oK) and np.array_equal(fl, ofl)
    assert np.array_equal(lo, olo) and np.array_equal(hi, ohi)
    iv = np.int64 if npd == np.float64 else np.int32
    assert np.array_equal(out.view(iv), O.finalize(ref).view(iv))


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_dropin_specials_and_range_match_oracle(dtype):
    npd = np.float64 if dtype == torch.float64 else np.float32
    lim = npd(2.0 ** 1005 if dtype == torch.float64 else 2.0 ** 120)
    cases = [[1.0, np.inf, 2.0], [-np.inf, 3.0], [np.inf, -np.inf], [np.nan, 1.0], [lim, 1.0], [0.0, -0.0]]
    for vals in cases:
        v = torch.tensor(vals, dtype=dtype, device=DEV)
        st = R.State(1, 3, dtype).add_values_unbuffered(v)
        out = st.finalize().cpu().numpy()
        ref = O.init(npd, 3, 1)
        O.groupby_sum(ref, np.zeros(len(vals), np.int32), np.array(vals, npd))
        K, fl, lo, hi = st.host_view()
        oK, ofl, olo, ohi = O.to_bins(ref)
        assert np.array_equal(fl, ofl), vals
        assert np.array_equal(K, oK) and np.array_equal(lo, olo) and np.array_equal(hi, ohi), vals
        iv = np.int64 if npd == np.float64 else np.int32
        assert np.array_equal(out.view(iv), O.finalize(ref).view(iv)), vals


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

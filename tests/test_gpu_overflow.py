"""Level sums past int64: every path against the C oracle, bit for bit.

A level of repro<double,L> sums digits of up to 2^(W-1) = 2^39; the paper
keeps the sum in <S, C> with an exact carry count (Algorithm 2's carry-bit
propagation), and the library keeps it as a 128-bit integer.  The inputs
here pack values at the top of the window with top grid index 27 (top digit
close to 2^39), 6*10^7 of them per group with one sign, so level 0 of those
groups ends far beyond 2^63: the high words of the 128-bit bins, the
overflow test of the 128-bit atomic add, the 128-bit flush of a CTA table
into its partial record and the merges of such records all carry nonzero
high parts.  Float levels cannot get there (digits up to 2^17 would need
2^46 rows), so the inputs are double.
"""
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

import paper_1802_09883_gb300 as R
from paper_1802_09883_gb300 import workloads as WL
from oracle import oracle as O

pytestmark = pytest.mark.gpu
DEV = "cuda"
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
N = 1 << 27
L = 3


def overflow_rows(n, seed, device, G=3, hot=None):
    """Keys over G groups: 45 % in group 0 (values at the top of binade 2^44,
    positive), 45 % in group 1 (the same, negative), the rest uniform over
    the other groups with values s * M * 2^e, e in [-40, 40].  With `hot` the
    positive heavy group is that key instead of 0 and there is no negative
    one (the partitioned path's case: one hot key among many groups)."""
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    u = torch.rand(n, generator=g, device=device)
    rest = torch.randint(0 if hot is not None else 2, G, (n,), generator=g, device=device, dtype=torch.int32)
    if hot is None:
        keys = torch.where(u < 0.45, 0, torch.where(u < 0.90, 1, rest)).to(torch.int32)
    else:
        keys = torch.where(u < 0.5, hot, rest).to(torch.int32)
    pos = WL.binade_top_values(n, 44, 1.9, g, device, sign=+1)
    neg = WL.binade_top_values(n, 44, 1.9, g, device, sign=-1)
    mixed = WL.random_values(n, -40, 40, g, device)
    if hot is None:
        vals = torch.where(keys == 0, pos, torch.where(keys == 1, neg, mixed))
    else:
        vals = torch.where(keys == hot, pos, mixed)
    return keys.contiguous(), vals.contiguous()


def _np(t):
    return t.detach().cpu().numpy()


def assert_state_matches(st_bytes, ost, G):
    K, fl, lo, hi = R.parse_state(st_bytes, L, G)
    oK, ofl, olo, ohi = O.to_bins(ost)
    assert np.array_equal(K, oK), "K differs"
    assert np.array_equal(fl, ofl), "flags differ"
    assert np.array_equal(lo, olo), "bins (lo) differ"
    assert np.array_equal(hi, ohi), "bins (hi) differ"


def assert_result_matches(out, ost):
    a = np.asarray(out).view(np.int64)
    b = O.finalize(ost).view(np.int64)
    assert np.array_equal(a, b), f"results differ: {np.asarray(out)[a != b][:4]} vs {O.finalize(ost)[a != b][:4]}"


@pytest.fixture(scope="module")
def three_groups():
    keys, vals = overflow_rows(N, 2063, DEV)
    kh, vh = _np(keys), _np(vals)
    ost = O.init(np.float64, L, 3)
    assert O.groupby_sum(ost, kh, vh, threads=os.cpu_count() or 1) == 0
    _, _, _, ohi = O.to_bins(ost)
    assert ohi[0, 0] >= 1 and ohi[1, 0] <= -2, "the input does not take level 0 past int64"
    return keys, vals, ost


def _state_bytes(st):
    torch.cuda.synchronize()
    return st.tensor.cpu().numpy()


def test_single_pass_default_grid(three_groups):
    keys, vals, ost = three_groups
    st = R.State(3, L)
    st.add(keys, vals)
    out = st.finalize()
    assert st.check() == 0
    assert_state_matches(_state_bytes(st), ost, 3)
    assert_result_matches(_np(out), ost)


def test_two_pass_path_128_bit_atomics(three_groups):
    """Unaligned columns take the window pass + 128-bit global atomic adds."""
    keys, vals, ost = three_groups
    kk = torch.empty(N + 1, dtype=torch.int32, device=DEV)
    vv = torch.empty(N + 1, dtype=torch.float64, device=DEV)
    kk[1:] = keys
    vv[1:] = vals
    st = R.State(3, L)
    st.add(kk[1:], vv[1:])  # 4- and 8-byte aligned, not 16
    out = st.finalize()
    assert st.check() == 0
    assert_state_matches(_state_bytes(st), ost, 3)
    assert_result_matches(_np(out), ost)


def test_merge_of_two_wide_states(three_groups):
    keys, vals, ost = three_groups
    h = N // 2
    a, b = R.State(3, L), R.State(3, L)
    a.add(keys[:h], vals[:h])
    b.add(keys[h:], vals[h:])
    a.merge(b)
    out = a.finalize()
    assert a.check() == 0
    assert_state_matches(_state_bytes(a), ost, 3)
    assert_result_matches(_np(out), ost)


def test_batched_task_split_into_items(three_groups):
    """One large task in the batched multi-task kernel: its items' partial
    tables are folded by the item merge in 128 bits."""
    keys, vals, ost = three_groups
    (st,) = R.groupby_sum_batched([(keys, vals, 3)], L=L)
    out = st.finalize()
    assert st.check() == 0
    assert_state_matches(_state_bytes(st), ost, 3)
    assert_result_matches(_np(out), ost)


def test_scalar_sum_keyless():
    g = torch.Generator(device=DEV)
    g.manual_seed(77)
    vals = WL.binade_top_values(N // 2, 44, 1.9, g, DEV, sign=-1)
    st = R.State(1, L).add_values(vals)
    out = st.finalize()
    assert st.check() == 0
    ost = O.init(np.float64, L, 1)
    O.groupby_sum(ost, np.zeros(vals.numel(), np.int32), _np(vals), threads=os.cpu_count() or 1)
    assert O.to_bins(ost)[3][0, 0] <= -2
    assert_state_matches(_state_bytes(st), ost, 1)
    assert_result_matches(_np(out), ost)


def test_partitioned_path_with_one_hot_group():
    G = 1 << 16
    keys, vals = overflow_rows(N // 2, 4163, DEV, G=G, hot=12345)
    st = R.State(G, L)
    st.add(keys, vals)
    out = st.finalize()
    assert st.check() == 0
    ost = O.init(np.float64, L, G)
    assert O.groupby_sum(ost, _np(keys), _np(vals), threads=os.cpu_count() or 1) == 0
    assert O.to_bins(ost)[3][12345, 0] >= 1
    assert_state_matches(_state_bytes(st), ost, G)
    assert_result_matches(_np(out), ost)


_SUB = r"""
import sys, torch, numpy as np
sys.path.insert(0, {root!r})
sys.path.insert(0, {tests!r})
import paper_1802_09883_gb300 as R
from test_gpu_overflow import overflow_rows, N, L
keys, vals = overflow_rows(N, 2063, "cuda")
st = R.State(3, L)
st.add(keys, vals)
out = st.finalize()
st.check()
torch.cuda.synchronize()
np.save({state!r}, st.tensor.cpu().numpy())
np.save({out!r}, out.cpu().numpy())
print("ok")
"""


@pytest.mark.parametrize("env", [{"REPRO_FUSED_CTAS": "2"},
                                 {"REPRO_FUSED_CTAS": "2", "REPRO_FLUSH_ROWS": "4096"},
                                 {"REPRO_FUSED_CTAS": "3", "REPRO_FUSED_CFG": "3,2048,16,1"}])
def test_single_pass_few_ctas_wide_partials(three_groups, env, tmp_path):
    """Two or three CTAs take 2^26 rows each, so every CTA's own partial
    record passes 2^63 through its flushes of the int64 table (every 2^23
    rows, or every 4096) -- the 128-bit read-add-write of the partial."""
    _, _, ost = three_groups
    sf, of = str(tmp_path / "state.npy"), str(tmp_path / "out.npy")
    code = _SUB.format(root=ROOT, tests=os.path.join(ROOT, "tests"), state=sf, out=of)
    r = subprocess.run([sys.executable, "-c", code], env={**os.environ, **env}, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0 and "ok" in r.stdout, r.stdout + r.stderr
    assert_state_matches(np.load(sf), ost, 3)
    assert_result_matches(np.load(of), ost)

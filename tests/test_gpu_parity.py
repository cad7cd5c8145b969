"""GPU path vs the CPU oracle, bit for bit (states and results).

Every test calls the CUDA kernels through the C ABI (via the thin binding)
and compares with oracle/repro_oracle.c on the same seeded inputs.
"""
import numpy as np
import pytest
import torch

import paper_1802_09883_gb300 as R
from paper_1802_09883_gb300 import workloads as WL
from oracle import oracle as O

pytestmark = pytest.mark.gpu

DEV = "cuda"


def _np(t):
    return t.detach().cpu().numpy()


def oracle_state(keys, vals, G, L, threads=4):
    st = O.init(vals.dtype, L, G)
    bad = O.groupby_sum(st, keys, vals, threads=threads)
    return st, bad


def assert_state_equal(gst: R.State, ost):
    K, fl, lo, hi = gst.host_view()
    oK, ofl, olo, ohi = O.to_bins(ost)
    assert np.array_equal(K, oK), "K differs"
    assert np.array_equal(fl, ofl), "flags differ"
    assert np.array_equal(lo, olo), "bins (lo) differ"
    assert np.array_equal(hi, ohi), "bins (hi) differ"


def assert_bits_equal(a, b):
    a, b = np.asarray(a), np.asarray(b)
    assert a.dtype == b.dtype and a.shape == b.shape
    ai = a.view(np.int64 if a.dtype == np.float64 else np.int32)
    bi = b.view(np.int64 if b.dtype == np.float64 else np.int32)
    mism = np.flatnonzero(ai != bi)
    assert mism.size == 0, f"{mism.size} results differ, first at {mism[:5]}: {a[mism[:5]]} vs {b[mism[:5]]}"


def run_gpu(keys_t, vals_t, G, L):
    st = R.State(G, L, vals_t.dtype)
    st.add(keys_t, vals_t)
    out = st.finalize()
    torch.cuda.synchronize()
    return st, out


# ----------------------------------------------------------------- config 0

@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_plain_1e6_rows_1024_groups_L3(dtype):
    w = WL.plain(n=1_000_000, G=1024, L=3, seed=1, device=DEV, dtype=dtype)
    st, out = run_gpu(w.keys, w.values, w.G, w.L)
    assert st.check() == 0
    ost, bad = oracle_state(_np(w.keys), _np(w.values), w.G, w.L)
    assert bad == 0
    assert_state_equal(st, ost)
    assert_bits_equal(_np(out), O.finalize(ost))


# ------------------------------------------------------- shapes and levels

@pytest.mark.parametrize("L", [1, 2, 3, 4])
@pytest.mark.parametrize("G", [1, 16, 1000, 3000, 7777, 70000])
def test_group_counts_and_levels(G, L):
    n = 200_003  # several tiles and a ragged tail
    w = WL.plain(n=n, G=G, L=L, seed=G * 10 + L, device=DEV, e_lo=-60, e_hi=60)
    st, out = run_gpu(w.keys, w.values, G, L)
    ost, _ = oracle_state(_np(w.keys), _np(w.values), G, L)
    assert_state_equal(st, ost)
    assert_bits_equal(_np(out), O.finalize(ost))


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("L", [1, 2, 4])
def test_wide_exponent_range_and_subnormals(dtype, L):
    g = torch.Generator(device=DEV)
    g.manual_seed(5 + L)
    n, G = 100_000, 37
    lo_e, hi_e = (-1074, 1000) if dtype == torch.float64 else (-149, 118)
    keys = WL.uniform_keys(n, G, g, DEV)
    # exponents across the whole range (random_values takes biased-exponent
    # offsets, so subnormals are drawn separately)
    vals = WL.random_values(n, max(lo_e, -1022 if dtype == torch.float64 else -126), hi_e, g, DEV, dtype)
    sub = torch.randint(1, 1 << (20 if dtype == torch.float64 else 12), (n // 10,), generator=g, device=DEV)
    sub = sub.to(torch.int64 if dtype == torch.float64 else torch.int32).view(dtype)
    vals[: n // 10] = sub
    st, out = run_gpu(keys, vals, G, L)
    ost, _ = oracle_state(_np(keys), _np(vals), G, L)
    assert_state_equal(st, ost)
    assert_bits_equal(_np(out), O.finalize(ost))


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_special_values_and_empty_groups(dtype):
    npd = np.float64 if dtype == torch.float64 else np.float32
    lim = 2.0 ** 1005 if dtype == torch.float64 else 2.0 ** 120
    keys = np.array([0, 0, 1, 1, 2, 3, 3, 4, 4, 5, 5, 6, 8, 8], np.int32)
    vals = np.array([1.0, np.nan, np.inf, 2.0, -np.inf, np.inf, -np.inf, lim, 1.0, 0.0, -0.0, -np.inf,
                     np.nextafter(npd(lim), npd(0)), -np.nextafter(npd(lim), npd(0))], npd)
    kt, vt = torch.from_numpy(keys).to(DEV), torch.from_numpy(vals).to(DEV)
    for L in (1, 3, 4):
        st, out = run_gpu(kt, vt, 10, L)
        ost, _ = oracle_state(keys, vals, 10, L, threads=1)
        assert_state_equal(st, ost)
        assert_bits_equal(_np(out), O.finalize(ost))
        o = _np(out)
        assert o.view(np.int64 if npd == np.float64 else np.int32)[0] == \
            (0x7FF8000000000000 if npd == np.float64 else 0x7FC00000)
        assert o[7] == 0 and not np.signbit(o[7]) and o[9] == 0 and not np.signbit(o[9])


def test_bad_keys_are_reported_and_skipped():
    keys = torch.tensor([0, 5, -1, 2, 1 << 30], dtype=torch.int32, device=DEV)
    vals = torch.tensor([1.0, 2.0, 3.0, 4.0, 5.0], dtype=torch.float64, device=DEV)
    st = R.State(5, 2)
    st.add(keys, vals)
    out = st.finalize()
    with pytest.raises(R.ReproError) as ei:
        st.check()
    assert ei.value.status == 2  # REPRO_EKEY
    assert _np(out).tolist() == [1.0, 0.0, 4.0, 0.0, 0.0]


def test_empty_input():
    st = R.State(8, 3)
    st.add(torch.empty(0, dtype=torch.int32, device=DEV), torch.empty(0, dtype=torch.float64, device=DEV))
    out = st.finalize()
    assert st.check() == 0
    assert (_np(out) == 0).all() and not np.signbit(_np(out)).any()


def test_layout_mismatch_is_detected():
    """A state initialised for L = 3 but passed with L = 4 is refused on the
    device (REPRO_ELAYOUT) and left untouched."""
    st = R.State(8, 3)
    with pytest.raises(ValueError):
        R.State(16, 3).merge(st)
    lib = R.lib()
    keys = torch.zeros(4, dtype=torch.int32, device=DEV)
    vals = torch.ones(4, dtype=torch.float64, device=DEV)
    buf = torch.zeros(R.state_bytes(torch.float64, 4, 8), dtype=torch.uint8, device=DEV)
    buf[: st.tensor.numel()] = st.tensor
    before = _np(buf).copy()
    s = torch.cuda.current_stream().cuda_stream
    assert lib.repro_groupby_sum(keys.data_ptr(), vals.data_ptr(), 4, 0, 4, 8, buf.data_ptr(), s) == 0
    assert lib.repro_state_check(buf.data_ptr(), None, s) == 7  # REPRO_ELAYOUT
    after = _np(buf)
    assert np.array_equal(after[64:], before[64:])


# ------------------------------------------------------------ invariants

@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_shuffles_splits_and_merges_give_identical_bytes(dtype):
    w = WL.sweep_cell(G=1 << 10, dist="zipf", L=3, n=1 << 20, seed=7, device=DEV, dtype=dtype)
    ref, ref_out = run_gpu(w.keys, w.values, w.G, w.L)
    ref_bytes = _np(ref.tensor)
    g = torch.Generator(device=DEV)
    g.manual_seed(3)
    for trial in range(3):
        p = torch.randperm(w.n, generator=g, device=DEV)
        k, v = w.keys[p], w.values[p]
        st, out = run_gpu(k, v, w.G, w.L)
        assert np.array_equal(_np(st.tensor), ref_bytes)
        # split into calls on one state
        cuts = sorted(torch.randint(1, w.n, (5,), generator=g, device=DEV).tolist())
        edges = [0] + cuts + [w.n]
        acc = R.State(w.G, w.L, dtype)
        parts = []
        for a, b in zip(edges[:-1], edges[1:]):
            acc.add(k[a:b], v[a:b])
            s = R.State(w.G, w.L, dtype)
            s.add(k[a:b], v[a:b])
            parts.append(s)
        assert np.array_equal(_np(acc.tensor), ref_bytes)
        # separate states merged in a shuffled order
        order = torch.randperm(len(parts), generator=g, device=DEV).tolist()
        m = parts[order[0]]
        for i in order[1:]:
            m.merge(parts[i])
        torch.cuda.synchronize()
        assert np.array_equal(_np(m.tensor), ref_bytes)
    ost, _ = oracle_state(_np(w.keys), _np(w.values), w.G, w.L)
    assert_state_equal(ref, ost)
    assert_bits_equal(_np(ref_out), O.finalize(ost))


def test_merge_with_different_windows_matches_oracle():
    g = torch.Generator(device=DEV)
    g.manual_seed(11)
    G, L = 300, 3
    ka, kb = WL.uniform_keys(50_000, G, g, DEV), WL.uniform_keys(50_000, G, g, DEV)
    va = WL.random_values(50_000, -90, -20, g, DEV)
    vb = WL.random_values(50_000, -30, 70, g, DEV)
    A, B = R.State(G, L), R.State(G, L)
    A.add(ka, va)
    B.add(kb, vb)
    A.merge(B)
    oa, _ = oracle_state(_np(ka), _np(va), G, L)
    ob, _ = oracle_state(_np(kb), _np(vb), G, L)
    O.merge(oa, ob)
    assert_state_equal(A, oa)
    assert_bits_equal(_np(A.finalize()), O.finalize(oa))


# -------------------------------------------------------------- baselines

def test_fp64_baseline_close_to_exact():
    w = WL.plain(n=1_000_000, G=1024, L=3, seed=1, device=DEV)
    out = _np(R.groupby_sum_fp64(w.keys, w.values, w.G))
    ref = O.groupby_sum_values(_np(w.keys), _np(w.values), w.G, 4)  # L = 4 holds every bit here
    absum = np.bincount(_np(w.keys), weights=np.abs(_np(w.values)), minlength=w.G)
    cnt = np.bincount(_np(w.keys), minlength=w.G)
    # eq. (5): (n - 1) eps sum |b|
    assert np.all(np.abs(out - ref) <= (cnt - 1).clip(min=0) * 2.0 ** -53 * absum + 1e-300)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("G,dist", [(16, "zipf"), (1000, "uniform"), (5000, "zipf"), (300_000, "uniform")])
@pytest.mark.parametrize("offset", [0, 1])
def test_conventional_baseline_strategies_within_error_bound(dtype, G, dist, offset):
    """Every table strategy of the conventional GroupBy (aligned columns by
    vector loads, unaligned ones by scalar loads) sums within eq. (5)'s bound
    (n - 1) eps sum|b| of the exact group sums; strategies whose tables do
    not fit report so."""
    w = WL.sweep_cell(G, dist, 3, n=(1 << 20) + 7, seed=G + offset, device=DEV, dtype=dtype)
    k, v = w.keys[offset:], w.values[offset:]
    kn, vn = _np(k), _np(v).astype(np.float64)
    ref = O.groupby_sum_values(kn, vn, G, 4)  # L = 4 holds every bit here
    absum = np.bincount(kn, weights=np.abs(vn), minlength=G)
    cnt = np.bincount(kn, minlength=G)
    eps = 2.0 ** -53 if dtype == torch.float64 else 2.0 ** -24
    ran = 0
    for mode in R.FP_MODES:
        out = R.groupby_sum_fp_mode(k, v, G, mode)
        if out is None:
            assert mode in (0, 1, 2) and G > 1000
            continue
        ran += 1
        got = _np(out).astype(np.float64)
        assert np.all(np.abs(got - ref) <= cnt.clip(min=1) * eps * absum + 1e-30), (mode, G)
    assert ran >= 2


def test_fp32_baseline_runs():
    w = WL.plain(n=100_000, G=100, L=3, seed=4, device=DEV, dtype=torch.float32)
    out = _np(R.groupby_sum_fp32(w.keys, w.values, w.G)).astype(np.float64)
    ref = np.bincount(_np(w.keys), weights=_np(w.values).astype(np.float64), minlength=w.G)
    absum = np.bincount(_np(w.keys), weights=np.abs(_np(w.values)).astype(np.float64), minlength=w.G)
    cnt = np.bincount(_np(w.keys), minlength=w.G)
    assert np.all(np.abs(out - ref) <= cnt * 2.0 ** -24 * absum + 1e-30)


# ----------------------------------------------------- single-pass fused path

def test_raise_heavy_input_sorted_by_magnitude():
    """Rows sorted by |value|: nearly every tile raises some group's window
    (the deferred-row path of the single-pass kernel)."""
    g = torch.Generator(device=DEV)
    g.manual_seed(21)
    n, G, L = 400_000, 200, 3
    keys = WL.uniform_keys(n, G, g, DEV)
    vals = WL.random_values(n, -300, 300, g, DEV)
    order = torch.argsort(vals.abs())
    vals = vals[order].contiguous()
    st, out = run_gpu(keys, vals, G, L)
    ost, _ = oracle_state(_np(keys), _np(vals), G, L)
    assert_state_equal(st, ost)
    assert_bits_equal(_np(out), O.finalize(ost))


@pytest.mark.parametrize("n", [1, 100, 2047, 2048, 2049, 6000])
def test_small_and_ragged_row_counts(n):
    w = WL.plain(n=n, G=64, L=4, seed=n, device=DEV, e_lo=-50, e_hi=50)
    st, out = run_gpu(w.keys, w.values, w.G, w.L)
    ost, _ = oracle_state(_np(w.keys), _np(w.values), w.G, w.L, threads=1)
    assert_state_equal(st, ost)
    assert_bits_equal(_np(out), O.finalize(ost))


def test_unaligned_inputs_take_the_two_pass_path():
    w = WL.plain(n=50_001, G=300, L=3, seed=9, device=DEV)
    k, v = w.keys[1:], w.values[1:]  # 4- and 8-byte aligned, not 16
    st, out = run_gpu(k, v, w.G, w.L)
    ost, _ = oracle_state(_np(k), _np(v), w.G, w.L)
    assert_state_equal(st, ost)
    assert_bits_equal(_np(out), O.finalize(ost))


_SUB = r"""
import sys, numpy as np, torch
sys.path.insert(0, {root!r})
import paper_1802_09883_gb300 as R
from paper_1802_09883_gb300 import workloads as WL
from oracle import oracle as O
for G, L, dtype in ((16, 2, torch.float64), (1024, 3, torch.float64), (777, 4, torch.float32), (3000, 3, torch.float64)):
    w = WL.plain(n=300_001, G=G, L=L, seed=G + L, device="cuda", e_lo=-45, e_hi=45, dtype=dtype)
    st = R.State(G, L, dtype)
    st.add(w.keys, w.values)
    out = st.finalize().cpu().numpy()
    st.check()
    ref = O.init(np.float64 if dtype == torch.float64 else np.float32, L, G)
    O.groupby_sum(ref, w.keys.cpu().numpy(), w.values.cpu().numpy(), threads=4)
    K, fl, lo, hi = st.host_view()
    oK, ofl, olo, ohi = O.to_bins(ref)
    assert (K == oK).all() and (fl == ofl).all() and (lo == olo).all() and (hi == ohi).all(), (G, L)
    iv = np.int64 if out.dtype == np.float64 else np.int32
    assert (out.view(iv) == O.finalize(ref).view(iv)).all(), (G, L)
print("ok")
"""


@pytest.mark.parametrize("env", [{"REPRO_FLUSH_ROWS": "4096"}, {"REPRO_FUSED_CFG": "2,1024,16,1"},
                                 {"REPRO_FUSED_CFG": "4,1024,8,2"}, {"REPRO_FUSED_CFG": "3,2048,16,1"},
                                 {"REPRO_FUSED_CFG": "3,1024,8,2,32"}, {"REPRO_FUSED_CFG": "1,2048,8,3"},
                                 {"REPRO_FUSED_CFG": "1,4096,16,1,32"}])
def test_fused_variants_in_subprocess(env):
    """Mid-kernel flushes of the int64 table into the 128-bit partial, and
    other tile / stage / warp configurations, give the same bits."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", _SUB.format(root=root)], env={**os.environ, **env},
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and "ok" in r.stdout, r.stdout + r.stderr


# ------------------------------------------------- partitioned large-G path

@pytest.mark.parametrize("G,dist,L,n,dtype", [
    (1 << 16, "zipf", 3, 1 << 22, torch.float64), (1 << 16, "uniform", 2, 1 << 22, torch.float64),  # one pass
    (5000, "zipf", 3, 1 << 22, torch.float64),
    (1 << 20, "uniform", 3, 1 << 22, torch.float64),  # one wide pass: 1024 partitions, long tiles
    (1 << 20, "zipf", 3, 1 << 22, torch.float32),
    (300_000, "uniform", 3, 1 << 22, torch.float32),  # one pass, 293 partitions
    (300_000, "uniform", 4, 1 << 22, torch.float64),  # one pass, 586 partitions of 512 groups
    (1 << 20, "uniform", 4, 1 << 22, torch.float64),  # two passes: 2048 partitions
    (3_000_000, "zipf", 2, 1 << 21, torch.float64),  # two passes, coarse partitions of uneven size
    (1 << 24, "uniform", 4, 1 << 20, torch.float64),  # 8192 final partitions (most groups empty)
])
def test_partitioned_path_matches_oracle(G, dist, L, n, dtype):
    w = WL.sweep_cell(G, dist, L, n=n, seed=G + L, device=DEV, dtype=dtype)
    st, out = run_gpu(w.keys, w.values, w.G, w.L)
    assert st.check() == 0
    ost, _ = oracle_state(_np(w.keys), _np(w.values), w.G, w.L, threads=8 if G <= (1 << 20) else 1)
    assert_state_equal(st, ost)
    assert_bits_equal(_np(out), O.finalize(ost))


def test_partitioned_path_accumulates_and_reports_bad_keys():
    G, L = 70_000, 3
    g = torch.Generator(device=DEV)
    g.manual_seed(44)
    k1 = WL.uniform_keys(300_000, G, g, DEV)
    v1 = WL.random_values(300_000, -30, 30, g, DEV)
    k2 = WL.uniform_keys(200_000, G, g, DEV)
    v2 = WL.random_values(200_000, -5, 60, g, DEV)  # raises windows of the first call
    k2[123] = G + 5
    st = R.State(G, L)
    st.add(k1, v1)
    st.add(k2, v2)
    with pytest.raises(R.ReproError):
        st.check()
    mask = (k2 >= 0) & (k2 < G)
    ost, _ = oracle_state(np.concatenate([_np(k1), _np(k2[mask])]), np.concatenate([_np(v1), _np(v2[mask])]), G, L)
    assert_state_equal(st, ost)


@pytest.mark.parametrize("n", [1, 5, 2447, 9999])
def test_partitioned_path_small_inputs_with_idle_ctas(n):
    """Row counts that leave most partition CTAs without rows."""
    G, L = 20000, 3
    w = WL.plain(n=n, G=G, L=L, seed=n, device=DEV, e_lo=-45, e_hi=45)
    st, out = run_gpu(w.keys, w.values, G, L)
    assert st.check() == 0
    ost, _ = oracle_state(_np(w.keys), _np(w.values), G, L, threads=1)
    assert_state_equal(st, ost)
    assert_bits_equal(_np(out), O.finalize(ost))


# ------------------------------------------- few groups, several columns

@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_multicolumn_composite_keys_match_oracle(dtype):
    k1, k2, cols = WL.few_groups_multicol(n=2_000_003, seed=2, device=DEV)
    cols = cols.to(dtype)
    states = R.groupby_sum_cols(k1, k2, 2, list(cols), num_groups=4, L=3)
    gid = (2 * _np(k1).astype(np.int32) + _np(k2).astype(np.int32))
    for c, st in enumerate(states):
        assert st.check() == 0
        ost, _ = oracle_state(gid, _np(cols[c]), 4, 3)
        assert_state_equal(st, ost)
        assert_bits_equal(_np(st.finalize()), O.finalize(ost))


def test_multicolumn_bad_composite_keys_flag_every_state():
    k1 = torch.tensor([0, 1, 3, 0], dtype=torch.uint8, device=DEV)
    k2 = torch.tensor([1, 1, 1, 0], dtype=torch.uint8, device=DEV)
    cols = [torch.tensor([1.0, 2.0, 3.0, 4.0], dtype=torch.float64, device=DEV) for _ in range(2)]
    states = R.groupby_sum_cols(k1, k2, 2, cols, num_groups=4, L=2)
    for st in states:
        with pytest.raises(R.ReproError):
            st.check()
        assert _np(st.finalize()).tolist() == [4.0, 1.0, 0.0, 2.0]


@pytest.mark.parametrize("ncols,G,n,dtype", [(3, 4, 1_000_003, torch.float64), (5, 16, 777_777, torch.float32),
                                             (4, 3000, 500_001, torch.float64)])
def test_multicolumn_groups_of_columns_equal_one_pass_per_column(ncols, G, n, dtype):
    g = torch.Generator(device=DEV)
    g.manual_seed(ncols * G)
    card2 = 64 if G > 256 else 2
    k1 = torch.randint(0, (G + card2 - 1) // card2, (n,), generator=g, device=DEV, dtype=torch.uint8)
    k2 = torch.randint(0, card2, (n,), generator=g, device=DEV, dtype=torch.uint8)
    cols = [WL.random_values(n, -50, 50, g, DEV, dtype) for _ in range(ncols)]
    states = R.groupby_sum_cols(k1, k2, card2, cols, num_groups=G, L=3)
    gid = k1.to(torch.int32) * card2 + k2.to(torch.int32)
    ok = gid < G
    for c, st in zip(cols, states):
        ref = R.State(G, 3, dtype)
        ref.add(torch.where(ok, gid, torch.zeros_like(gid))[ok], c[ok])
        torch.cuda.synchronize()
        if bool(ok.all()):
            assert st.check() == 0
        else:  # composite keys past num_groups were skipped and flagged
            with pytest.raises(R.ReproError):
                st.check()
        K, fl, lo, hi = st.host_view()
        rK, rfl, rlo, rhi = ref.host_view()
        assert np.array_equal(K, rK) and np.array_equal(fl, rfl) and np.array_equal(lo, rlo) and np.array_equal(hi, rhi)


@pytest.mark.parametrize("ipc", [1, 8])
def test_split_partitions_with_window_bounds_match_oracle(ipc, tmp_path):
    """Partitions split into many work items (a loaded choice of 8 items per
    CTA) share a window array of lower bounds between their items; the state
    must still equal the oracle's bit for bit.  n >= 64 G, so no exact
    window pass runs."""
    G, L, n = 20_000, 3, (1 << 23) + 5
    w = WL.sweep_cell(G, "zipf", L, n=n, seed=77, device=DEV)
    f = tmp_path / "choice.txt"
    f.write_text(f"part 0 {L} {(G - 1).bit_length()} 9 1 2 1024 8 2 1 {ipc}\n")
    R.tune_clear()
    R.tune_load(str(f))
    try:
        st, out = run_gpu(w.keys, w.values, w.G, w.L)
    finally:
        R.tune_clear()
    assert st.check() == 0
    ost, _ = oracle_state(_np(w.keys), _np(w.values), w.G, w.L, threads=8)
    assert_state_equal(st, ost)
    assert_bits_equal(_np(out), O.finalize(ost))


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("G", [16, 1000, 70_000])
def test_zero_heavy_columns_match_oracle(dtype, G):
    """A third of the rows +0 or -0 (a discount column, say): zeros ride the
    four-row fast path without touching the table; results and state equal
    the oracle's."""
    g = torch.Generator(device=DEV)
    g.manual_seed(91 + G)
    n = (1 << 21) + 3
    keys = WL.uniform_keys(n, G, g, DEV)
    vals = WL.random_values(n, -30, 30, g, DEV, dtype)
    z = torch.rand(n, generator=g, device=DEV) < 0.33
    signs = torch.where(torch.rand(n, generator=g, device=DEV) < 0.5, -1.0, 1.0).to(dtype)
    vals = torch.where(z, torch.zeros_like(vals) * signs, vals)  # +0 and -0
    st, out = run_gpu(keys, vals, G, 3)
    assert st.check() == 0
    ost, _ = oracle_state(_np(keys), _np(vals), G, 3, threads=8)
    assert_state_equal(st, ost)
    assert_bits_equal(_np(out), O.finalize(ost))


# ------------------------------------------------- the benchmark's own cell

def test_bench_headline_cell_full_state():
    """The workload bench.py times by default -- 2^28 rows, 1024 groups
    uniform, repro<double,3>, the same seed -- every group's state (K, flags,
    128-bit bins) and result against the threaded C oracle, in the built-in
    configuration and in the one the autotuner picks (which bench.py times)."""
    import os
    w = WL.sweep_cell(1 << 10, "uniform", 3, n=1 << 28, device=DEV)
    ost, bad = oracle_state(_np(w.keys), _np(w.values), w.G, w.L, threads=os.cpu_count() or 1)
    assert bad == 0
    st, out = run_gpu(w.keys, w.values, w.G, w.L)
    assert st.check() == 0
    assert_state_equal(st, ost)
    assert_bits_equal(_np(out), O.finalize(ost))
    R.tune_clear()
    try:
        R.tune(w.keys, w.values, w.G, w.L)
        st2, out2 = run_gpu(w.keys, w.values, w.G, w.L)
    finally:
        R.tune_clear()
    assert_state_equal(st2, ost)
    assert_bits_equal(_np(out2), O.finalize(ost))

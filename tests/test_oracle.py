"""The C oracle (Algorithm 2 in IEEE arithmetic) against the exact model.

The two oracles are independent derivations of the paper's method: the C
oracle keeps the paper's <S, C> floating-point state and replays Algorithm 2
per value; the exact model writes the method as a definition over big
integers.  They must agree bit for bit, states and results.
"""
import numpy as np
import pytest

from oracle import exact as X
from oracle import oracle as O

FMTS = {np.float64: X.DOUBLE, np.float32: X.FLOAT}


def _values(rs, n, dtype, elo, ehi):
    v = rs.uniform(1, 2, n) * np.exp2(rs.integers(elo, ehi + 1, n)) * rs.choice([-1.0, 1.0], n)
    return v.astype(dtype)


def _exact_bins(states, L):
    K = np.array([s.K for s in states], np.int32)
    fl = np.array([s.flags for s in states], np.uint32)
    T = [[s.T[j] for j in range(L)] for s in states]
    return K, fl, T


def _oracle_T(lo, hi):
    return [[(int(h) << 64) + int(l) for l, h in zip(lr, hr)] for lr, hr in zip(lo, hi)]


def _same_bits(a, b):
    return np.array_equal(np.asarray(a).view(np.uint8), np.asarray(b).view(np.uint8))


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("L", [1, 2, 3, 4])
def test_oracle_matches_exact_model(dtype, L):
    fmt = FMTS[dtype]
    rs = np.random.default_rng(1000 + L)
    emax = 900 if dtype == np.float64 else 100
    emin = -1074 if dtype == np.float64 else -149
    for G, n, lo_e, hi_e in ((1, 300, -10, 10), (5, 600, -40, 40), (3, 300, emin, emax),
                             (17, 800, -60, 20)):
        keys = rs.integers(0, G, n)
        vals = _values(rs, n, dtype, lo_e, hi_e)
        st = O.init(dtype, L, G)
        assert O.groupby_sum(st, keys, vals) == 0
        K, fl, lo, hi = O.to_bins(st)
        ex = X.groupby_sum(keys, vals, G, L, fmt)
        eK, efl, eT = _exact_bins(ex, L)
        assert np.array_equal(K, eK)
        assert np.array_equal(fl, efl)
        assert _oracle_T(lo, hi) == eT
        want = np.array([X.to_float(X.finalize(s, L, fmt), fmt) for s in ex], dtype=dtype)
        assert _same_bits(O.finalize(st), want)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_subnormals_and_extremes(dtype):
    fmt = FMTS[dtype]
    fi = np.finfo(dtype)
    tiny = fi.smallest_subnormal
    vals = np.array([tiny, -tiny, 3 * tiny, fi.tiny, fi.tiny * 1.5, -fi.tiny / 3,
                     tiny * 1000, 0.0, -0.0, 1.0, fi.eps], dtype=dtype)
    keys = np.array([0, 0, 0, 1, 1, 1, 2, 3, 3, 4, 4])
    for L in (1, 2, 3, 4):
        got = O.groupby_sum_values(keys, vals, 6, L, dtype)
        want = X.groupby_sum_values(keys, vals, 6, L, fmt)
        assert _same_bits(got, want), L
    # huge values up to just below the range limit
    lim = 2.0 ** 1005 if dtype == np.float64 else 2.0 ** 120
    big = np.nextafter(dtype(lim), dtype(0))
    vals = np.array([big, -big, big, big / 3, -big / 7], dtype=dtype)
    for L in (1, 2, 4):
        got = O.groupby_sum_values(np.zeros(5, int), vals, 1, L, dtype)
        want = X.groupby_sum_values(np.zeros(5, int), vals, 1, L, fmt)
        assert _same_bits(got, want)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_special_values(dtype):
    fmt = FMTS[dtype]
    nan, inf = np.nan, np.inf
    lim = 2.0 ** 1005 if dtype == np.float64 else 2.0 ** 120
    keys = [0, 0, 1, 1, 2, 3, 3, 4, 4, 5, 5, 6]
    vals = np.array([1.0, nan, inf, 2.0, -inf, inf, -inf, lim, 1.0, 0.0, -0.0, -inf], dtype=dtype)
    got = O.groupby_sum_values(keys, vals, 8, 3, dtype)
    want = X.groupby_sum_values(keys, vals, 8, 3, fmt)
    assert _same_bits(got, want)
    st = O.init(dtype, 3, 8)
    O.groupby_sum(st, keys, vals)
    K, fl, lo, hi = O.to_bins(st)
    assert fl[4] == O.FLAG_RANGE and fl[0] == O.FLAG_NAN
    assert fl[3] == O.FLAG_POS_INF | O.FLAG_NEG_INF
    assert not np.signbit(got[5]) and got[7] == 0 and not np.signbit(got[7])


def test_bad_keys_are_counted_and_skipped():
    st = O.init(np.float64, 2, 4)
    bad = O.groupby_sum(st, [0, 4, -1, 3, 2], np.array([1.0, 2.0, 3.0, 4.0, 5.0]))
    assert bad == 2
    out = O.finalize(st)
    assert list(out) == [1.0, 0.0, 5.0, 4.0]


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("L", [2, 3])
def test_permutations_splits_and_threads_identical(dtype, L):
    rs = np.random.default_rng(77 + L)
    n, G = 20000, 33
    keys = rs.integers(0, G, n)
    vals = _values(rs, n, dtype, -40, 40)
    ref = O.init(dtype, L, G)
    O.groupby_sum(ref, keys, vals)
    ref_bins = O.to_bins(ref)
    ref_out = O.finalize(ref)
    for trial in range(4):
        p = rs.permutation(n)
        st = O.init(dtype, L, G)
        O.groupby_sum(st, keys[p], vals[p])
        assert all(np.array_equal(a, b) for a, b in zip(O.to_bins(st), ref_bins))
        # random split into parts, merged in random order
        cuts = np.sort(rs.choice(np.arange(1, n), rs.integers(1, 9), replace=False))
        parts = np.split(p, cuts)
        states = []
        for part in parts:
            s = O.init(dtype, L, G)
            O.groupby_sum(s, keys[part], vals[part])
            states.append(s)
        while len(states) > 1:
            i = int(rs.integers(0, len(states) - 1))
            a, b = states.pop(i), states.pop(i)
            O.merge(a, b)
            states.insert(i, a)
        assert all(np.array_equal(x, y) for x, y in zip(O.to_bins(states[0]), ref_bins))
        th = O.init(dtype, L, G)
        O.groupby_sum(th, keys[p], vals[p], threads=int(rs.integers(2, 8)))
        assert _same_bits(O.finalize(th), ref_out)


def test_merge_matches_exact_merge():
    rs = np.random.default_rng(5)
    L, G = 3, 6
    a_keys, b_keys = rs.integers(0, G, 400), rs.integers(0, G, 400)
    a_vals = _values(rs, 400, np.float64, -80, 0)
    b_vals = _values(rs, 400, np.float64, -10, 60)  # raises most windows
    A, B = O.init(np.float64, L, G), O.init(np.float64, L, G)
    O.groupby_sum(A, a_keys, a_vals)
    O.groupby_sum(B, b_keys, b_vals)
    O.merge(A, B)
    ea = X.groupby_sum(a_keys, a_vals, G, L, X.DOUBLE)
    eb = X.groupby_sum(b_keys, b_vals, G, L, X.DOUBLE)
    em = [X.merge(x, y, L) for x, y in zip(ea, eb)]
    K, fl, lo, hi = O.to_bins(A)
    assert list(K) == [s.K for s in em]
    assert _oracle_T(lo, hi) == [s.T for s in em]


def test_tie_heavy_input_is_order_independent():
    """Values that sit exactly halfway between two units of the lowest level
    (reading R2): every order gives the same state."""
    L = 2
    u_low = 2.0 ** -34  # lowest unit of the window at grid index 27 (set by 2^30)
    base = np.array([1.0, -3.0, 5.0, 1000.0, -65535.0])
    vals = np.concatenate([base + 0.5 * u_low, base - 0.5 * u_low, base + 1.5 * u_low, [2.0 ** 30]])
    assert np.all(vals[:-1] != np.tile(base, 3))  # the half units are representable
    assert vals.size == 16
    outs = set()
    rs = np.random.default_rng(9)
    for _ in range(20):
        p = rs.permutation(vals.size)
        st = O.init(np.float64, L, 1)
        O.groupby_sum(st, np.zeros(vals.size, int), vals[p])
        outs.add(tuple(np.concatenate([a.ravel().view(np.uint8) for a in O.to_bins(st)])))
    assert len(outs) == 1
    want = X.groupby_sum(np.zeros(vals.size, int), vals, 1, L, X.DOUBLE)[0]
    K, fl, lo, hi = O.to_bins(st)
    assert _oracle_T(lo, hi)[0] == want.T


def test_oracle_levels_beyond_2p63():
    """Bins past int64: the C oracle's carry counts, its 128-bit bin view and
    its finalize against the exact model's digits times multiplicities.

    Six values packed at the top of the window with top grid index 27 (top
    digit close to 2^(W-1)), each repeated millions of times; group 0 sums
    them positive, group 1 negative (both pass 2^64 at level 0), group 2
    mixes signs and smaller values.  Algorithm 2 keeps S in [1.5, 1.75) ufp
    and counts the carries in C, so T = (S - 1.5 ufp)/ulp + C 2^(m-2) must
    reach these magnitudes exactly."""
    fmt = X.DOUBLE
    rs = np.random.default_rng(63)
    tops = rs.uniform(1.9, 2.0, 6) * 2.0 ** 44  # |b| / u(27) in [1.9, 2) 2^38
    small = rs.uniform(1.0, 2.0, 6) * np.exp2(rs.integers(-30, 20, 6))
    mult = rs.integers(1 << 22, 1 << 23, 6)
    L, G = 3, 3
    parts_k, parts_v, want = [], [], []
    for g, (vals, signs) in enumerate(((tops, np.ones(6)), (tops, -np.ones(6)),
                                      (np.concatenate([tops, small]), np.tile([1.0, -1.0], 6)))):
        m = mult if g < 2 else np.concatenate([mult, mult[::-1]]) >> 8
        v = np.repeat(vals * signs, m)
        parts_k.append(np.full(v.size, g, np.int32))
        parts_v.append(v)
        K = max(X.top_index(fmt, X.Fraction(float(x))) for x in vals)
        T = [0] * L
        for x, c in zip(vals * signs, m):
            for j, d in enumerate(X.digits(fmt, X.Fraction(float(x)), K, L)):
                T[j] += int(c) * d
        want.append(X.GroupState(K, 0, T))
    keys = np.concatenate(parts_k)
    vals = np.concatenate(parts_v)
    perm = rs.permutation(keys.size)
    keys, vals = keys[perm], vals[perm]
    st = O.init(np.float64, L, G)
    assert O.groupby_sum(st, keys, vals, threads=8) == 0
    K, fl, lo, hi = O.to_bins(st)
    got_T = _oracle_T(lo, hi)
    assert [w.K for w in want] == K.tolist()
    assert [w.T for w in want] == got_T
    assert got_T[0][0] > 1 << 63 and got_T[1][0] < -(1 << 63)  # past int64: a nonzero high word
    res = np.array([X.to_float(X.finalize(w, L, fmt), fmt) for w in want])
    assert _same_bits(O.finalize(st), res)

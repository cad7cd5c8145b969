"""Pins for the exact big-integer model (oracle/exact.py).

Everything here checks the model against something other than itself: the
paper's worked examples and tables (tests/golden), IEEE hardware rounding,
closed forms, invariants, and brute force against a literal replay of
Algorithm 2 in a toy format.
"""
import itertools
import math
import random
from fractions import Fraction

import numpy as np
import pytest

from oracle import exact as X

pytestmark = pytest.mark.filterwarnings("ignore")


def _toy_values(rng, n, m, emin, emax):
    """Random toy-format values with m fraction bits, exponents in [emin, emax]."""
    out = []
    for _ in range(n):
        mant = rng.randrange(1 << m, 1 << (m + 1))
        e = rng.randint(emin, emax)
        s = rng.choice((1, -1))
        out.append(s * Fraction(mant) * Fraction(2) ** (e - m))
    return out


# ---------------------------------------------------------------------------
# Worked examples of Sec. III (Fig. rsum-example, Fig. carry-example)
# ---------------------------------------------------------------------------

def test_worked_example_replay_reproduces_printed_result(golden):
    g = golden("rsum_worked_example.txt")
    m, W, f, L = (int(g[k]) for k in ("m", "W", "f", "L"))
    fmt = X.toy(m, W, g_min=f - m - (L - 1) * W)
    st = X.alg2_init(fmt, L, f)
    for b in g["values"].split():
        X.alg2_add(st, Fraction(b), fmt, t=W)
        assert all(d == int(g["carries"]) for d in st.carries)
    assert X.alg2_finalize(st, fmt) == int(g["result"])
    assert st.C == [0] * L
    assert st.raises == 1


def test_worked_example_under_listed_threshold_matches_definition(golden):
    """With the threshold 2^(W-1) that Algorithm 2 lists, the same three
    values raise twice and the result is 12; the definition (window from the
    max |b|) gives the same levels and the same result."""
    g = golden("rsum_worked_example.txt")
    m, W, f, L = (int(g[k]) for k in ("m", "W", "f", "L"))
    g_min = f - m - (L - 1) * W
    fmt = X.toy(m, W, g_min=g_min)
    vals = [Fraction(b) for b in g["values"].split()]
    st = X.alg2_init(fmt, L, f)
    for b in vals:
        X.alg2_add(st, b, fmt, t=W - 1)
    assert st.raises == 2
    assert X.alg2_finalize(st, fmt) == 12
    d = X.groupby_sum([0] * len(vals), vals, 1, L, fmt)[0]
    assert d.T == X.alg2_level_integers(st, fmt)
    assert X.finalize(d, L, fmt) == 12


def test_carry_example(golden):
    g = golden("rsum_worked_example.txt")
    m, W = int(g["m"]), int(g["W"])
    fmt = X.toy(m, W, g_min=0)
    S0, C0 = Fraction(int(g["carry_S_before"])), int(g["carry_C_before"])
    st = X.ReplayState([S0], [C0])
    t_before = X.alg2_level_integers(st, fmt)[0]
    X.alg2_add(st, Fraction(g["carry_value"]), fmt, t=W)
    assert st.carries == [int(g["carry_d"])]
    assert st.C == [C0 + int(g["carry_d"])]
    u = X.ufp(S0)
    assert Fraction(3, 2) * u <= st.S[0] < Fraction(7, 4) * u
    # the level still holds T + its digit: RNE(3.125 / ulp(S)) = 3
    assert X.alg2_level_integers(st, fmt)[0] == t_before + 3


def test_eft_examples(golden):
    g = golden("eft_examples.txt")
    half = X.Fmt("half", m=int(g["half_m"]), W=1, g_min=-24, emin=-14, emax=15)
    a, b = Fraction(g["half_a"]), Fraction(g["half_b"])
    p = int(g["half_p"])
    assert a == int(g["half_alpha_a"]) * Fraction(2) ** p
    assert b == int(g["half_alpha_b"]) * Fraction(2) ** p
    assert X.rd(a, half) == a and X.rd(b, half) == b
    assert X.fadd(a, b, half) == a + b == Fraction(g["half_sum"])
    t3 = X.toy(int(g["split_m"]), 1, 0)
    a, b = Fraction(g["split_a"]), Fraction(g["split_b"])
    q = X.fsub(X.fadd(a, b, t3), a, t3)
    r = X.fsub(b, q, t3)
    assert q == Fraction(g["split_q"]) and r == Fraction(g["split_r"])
    assert q % X.ulp(a, t3) == 0  # q is a multiple of ulp(a)
    assert X.fadd(q, r, t3) == b


def test_toy_nonassociativity(golden):
    g = golden("eft_examples.txt")
    t2 = X.toy(int(g["toy_m"]), 1, 0)
    a, b, c = (Fraction(g[k]) for k in ("toy_a", "toy_b", "toy_c"))
    left = X.fadd(X.fadd(a, b, t2, "trunc"), c, t2, "trunc")
    right = X.fadd(a, X.fadd(b, c, t2, "trunc"), t2, "trunc")
    assert left == int(g["toy_left"]) and right == int(g["toy_right"])
    err = ((a + b) - X.fadd(a, b, t2, "trunc")) + ((a + b + c) - left)
    err2 = ((b + c) - X.fadd(b, c, t2, "trunc")) + ((a + X.fadd(b, c, t2, "trunc")) - right)
    assert err == 0 and err2 == int(g["toy_error_sum"])


def test_sql_example_order_dependence_and_repro(golden):
    g = golden("sql_example.txt")
    vals = [float(v) for v in g["values"].split()]

    def conv(order):
        s = 0.0
        for i in order:
            s += vals[i]
        return s

    before = conv([int(i) for i in g["order_before"].split()])
    after = conv([int(i) for i in g["order_after"].split()])
    assert "%.15g" % before == g["printed_before"]
    assert "%.15g" % after == g["printed_after"]
    outs = set()
    for perm in itertools.permutations(range(3)):
        for L in (2, 3):
            v = X.groupby_sum_values([0] * 3, [vals[i] for i in perm], 1, L, X.DOUBLE)
            outs.add((L, v.tobytes()))
    assert len(outs) == 2  # one result per L, whatever the order


# ---------------------------------------------------------------------------
# Table II and the error bounds
# ---------------------------------------------------------------------------

def test_table2_from_eq5_eq6(golden_rows):
    mean = {"U12": 1.5, "EXP": 1.0}
    mx = {"U12": 2.0, "EXP": 22.0}
    for method, L, n, dist, printed in golden_rows("table2_error_bounds.txt"):
        L, n, printed = int(L), int(n), float(printed)
        if method == "conv":
            v = X.error_bound_conventional(n, 2.0 ** -53, n * mean[dist])
        else:
            v = X.error_bound_rsum(n, L, 40, mx[dist])
        # printed with two significant digits
        assert float("%.1e" % v) == pytest.approx(printed, rel=1e-9), (method, L, n, dist, v)


@pytest.mark.parametrize("dist", ["U12", "EXP"])
@pytest.mark.parametrize("L", [1, 2, 3])
def test_accuracy_within_bound(dist, L):
    rs = np.random.default_rng(7 + L)
    n = 1000
    vals = rs.uniform(1, 2, n) if dist == "U12" else rs.exponential(1.0, n)
    st = X.groupby_sum([0] * n, vals, 1, L, X.DOUBLE)[0]
    q = X.finalize(st, L, X.DOUBLE)
    ex = X.exact_sum(vals)
    # The listed raise threshold puts u_top <= 2 max|b|: twice eq. (6).
    trunc = 2 * X.error_bound_rsum(n, L, 40, float(np.max(np.abs(vals))))
    vs = X.level_values(st, L, X.DOUBLE)
    fold = (L + 1) * 2.0 ** -53 * sum(abs(float(v)) for v in vs)
    assert abs(float(q - ex)) <= trunc + fold
    # the truncation part alone: exact level sum vs exact sum
    lev = sum(st.T[j] * X.unit(X.DOUBLE, st.K - j) for j in range(L))
    assert abs(float(lev - ex)) <= trunc


# ---------------------------------------------------------------------------
# Rounding of the model against IEEE hardware
# ---------------------------------------------------------------------------

def test_rd_double_matches_hardware():
    rs = random.Random(3)
    specials = [5e-324, 2.2250738585072014e-308, 1.7976931348623157e308, 1e-310, 0.1]
    for _ in range(3000):
        a = rs.choice(specials + [rs.uniform(-1, 1) * 2.0 ** rs.randint(-1074, 1023)])
        b = rs.choice(specials + [rs.uniform(-1, 1) * 2.0 ** rs.randint(-1074, 1023)])
        hw = a + b
        md = X.fadd(Fraction(a), Fraction(b), X.DOUBLE)
        if math.isinf(hw):
            assert md == hw
        else:
            assert md == Fraction(hw), (a, b)


def test_rd_float_matches_hardware():
    rs = np.random.default_rng(4)
    a = (rs.uniform(-1, 1, 3000) * np.exp2(rs.integers(-149, 128, 3000))).astype(np.float32)
    b = (rs.uniform(-1, 1, 3000) * np.exp2(rs.integers(-149, 128, 3000))).astype(np.float32)
    with np.errstate(over="ignore"):
        hw = a + b
    for x, y, z in zip(a, b, hw):
        md = X.fadd(Fraction(float(x)), Fraction(float(y)), X.FLOAT)
        if np.isinf(z):
            assert md == float(z)
        else:
            assert md == Fraction(float(z)), (x, y)


def test_rd_integer_times_unit_matches_ldexp():
    rs = random.Random(5)
    for _ in range(2000):
        T = rs.randint(-(1 << 52), 1 << 52)  # float(T) is exact
        k = rs.randint(-1200, 1100)
        try:
            want = math.ldexp(float(T), k)  # one correctly rounded scaling
        except OverflowError:
            want = math.copysign(math.inf, T)
        got = X.rd(T * Fraction(2) ** k, X.DOUBLE)
        if isinstance(got, float):
            assert got == want
        else:
            assert got == Fraction(want), (T, k)


# ---------------------------------------------------------------------------
# Grid, window and digits
# ---------------------------------------------------------------------------

def test_kmax_and_range_limits():
    assert X.k_max(X.DOUBLE) == 51
    assert X.k_max(X.FLOAT) == 14
    big = 2.0 ** 1005
    assert X.classify(X.DOUBLE, big)[0] == X.FLAG_RANGE
    assert X.classify(X.DOUBLE, np.nextafter(big, 0))[0] == 0
    assert X.classify(X.FLOAT, np.float32(2.0 ** 120))[0] == X.FLAG_RANGE
    assert X.classify(X.FLOAT, np.nextafter(np.float32(2.0 ** 120), np.float32(0)))[0] == 0


def test_top_index_boundaries():
    f = X.DOUBLE
    for K in range(1, 52):
        edge = Fraction(2) ** (f.W - 1) * X.unit(f, K - 1)  # smallest |b| needing K
        assert X.top_index(f, edge) == K
        below = Fraction(float(np.nextafter(float(edge), 0.0)))
        assert X.top_index(f, below) == K - 1
    assert X.top_index(f, Fraction(0)) == 0
    assert X.top_index(f, Fraction(5e-324)) == 0


@pytest.mark.parametrize("fmt", [X.DOUBLE, X.FLOAT])
def test_digits_closed_form_and_telescoping(fmt):
    rs = np.random.default_rng(11)
    W = fmt.W
    for _ in range(400):
        if fmt is X.DOUBLE:
            b = float(rs.uniform(-2, 2) * 2.0 ** int(rs.integers(-1074, 1000)))
        else:
            b = float(np.float32(rs.uniform(-2, 2) * 2.0 ** int(rs.integers(-149, 118))))
        x = Fraction(b)
        Kb = X.top_index(fmt, x)
        for K in (Kb, Kb + 1, Kb + 3):
            for L in (1, 2, 3, 4):
                c = X.digits(fmt, x, K, L)
                for j in range(L):
                    if K - j < 0:
                        assert c[j] == 0
                        continue
                    up = 0 if j == 0 else X.rne(x / X.unit(fmt, K - j + 1))
                    assert c[j] == X.rne(x / X.unit(fmt, K - j)) - (1 << W) * up
                    assert abs(c[j]) <= 1 << (W - 1)
                low = max(K - L + 1, 0)
                lev = sum(c[j] * X.unit(fmt, K - j) for j in range(L) if K - j >= 0)
                assert lev == X.rne(x / X.unit(fmt, low)) * X.unit(fmt, low)


def test_digit_window_independence():
    """The digit at a grid index does not depend on the window it is taken
    in (as long as the window's top can take the value): what makes local
    windows, level raising and merges give one result."""
    f = X.DOUBLE
    rs = np.random.default_rng(12)
    for _ in range(300):
        x = Fraction(float(rs.uniform(-2, 2) * 2.0 ** int(rs.integers(-300, 300))))
        Kb = X.top_index(f, x)
        ref = dict(zip(range(Kb, Kb - 6, -1), X.digits(f, x, Kb, 6)))
        for K in range(Kb, Kb + 4):
            for j, c in enumerate(X.digits(f, x, K, 6)):
                if K - j in ref:
                    assert c == ref[K - j]


# ---------------------------------------------------------------------------
# Definition vs literal Algorithm 2 (toy format, brute force)
# ---------------------------------------------------------------------------

def _replay(vals, fmt, L, t, extractor="constant"):
    st = X.alg2_init(fmt, L, fmt.m + fmt.g_min)  # S^(1) at grid index 0
    for b in vals:
        X.alg2_add(st, b, fmt, t=t, extractor=extractor)
    return st


def _replay_top(st, fmt):
    return (X.floor_log2(X.ulp(st.S[0], fmt)) - fmt.g_min) // fmt.W


@pytest.mark.parametrize("L", [1, 2, 3])
def test_brute_force_streaming_equals_definition(L):
    fmt = X.toy(10, 4, -20)
    rs = random.Random(100 + L)
    for trial in range(60):
        n = rs.randint(1, 5)
        vals = _toy_values(rs, n, 10, -10, 10)
        d = X.groupby_sum([0] * n, vals, 1, L, fmt)[0]
        want = (d.K, d.T, X.finalize(d, L, fmt))
        for perm in itertools.permutations(vals):
            st = _replay(perm, fmt, L, t=fmt.W - 1)
            got = (_replay_top(st, fmt), X.alg2_level_integers(st, fmt), X.alg2_finalize(st, fmt))
            assert got == want, (vals, perm)


def test_threshold_W_is_not_reproducible():
    """Negative control: the raise threshold 2^W (the worked example's) gives
    order-dependent results on some inputs."""
    fmt = X.toy(10, 4, -20)
    rs = random.Random(7)
    found = False
    for trial in range(300):
        vals = _toy_values(rs, 4, 10, -10, 10)
        res = {X.alg2_finalize(_replay(p, fmt, 2, t=fmt.W), fmt)
               for p in itertools.permutations(vals)}
        if len(res) > 1:
            found = True
            break
    assert found


def test_running_extractor_ties_are_order_dependent():
    """Negative control for reading R2: with the running sum as extractor an
    exact tie rounds by the running sum's last bit, so order matters."""
    fmt = X.toy(10, 4, -20)
    vals = [Fraction(1), Fraction(1, 2)]  # both need grid index 5 (u = 1); 1/2 is a tie
    for L, what in ((1, "result"), (2, "state")):
        run, const = set(), set()
        for p in itertools.permutations(vals):
            a = _replay(p, fmt, L, fmt.W - 1, "running")
            b = _replay(p, fmt, L, fmt.W - 1, "constant")
            if what == "result":
                run.add(X.alg2_finalize(a, fmt))
                const.add(X.alg2_finalize(b, fmt))
            else:
                run.add(tuple(X.alg2_level_integers(a, fmt)))
                const.add(tuple(X.alg2_level_integers(b, fmt)))
        assert len(const) == 1 and len(run) == 2


@pytest.mark.parametrize("L", [2, 3])
def test_split_and_merge_equals_whole(L):
    fmt = X.toy(10, 4, -20)
    rs = random.Random(200 + L)
    for trial in range(40):
        n = rs.randint(2, 40)
        G = rs.randint(1, 4)
        keys = [rs.randrange(G) for _ in range(n)]
        vals = _toy_values(rs, n, 10, -10, 12)
        whole = X.groupby_sum(keys, vals, G, L, fmt)
        idx = list(range(n))
        rs.shuffle(idx)
        cuts = sorted(rs.sample(range(1, n), rs.randint(0, min(5, n - 1))))
        parts = [idx[a:b] for a, b in zip([0] + cuts, cuts + [n])]
        states = [X.groupby_sum([keys[i] for i in p], [vals[i] for i in p], G, L, fmt) for p in parts]
        while len(states) > 1:  # random merge tree
            i = rs.randrange(len(states) - 1)
            a, b = states.pop(i), states.pop(i)
            states.insert(i, [X.merge(x, y, L) for x, y in zip(a, b)])
        for w, s in zip(whole, states[0]):
            assert (w.K, w.T) == (s.K, s.T)


# ---------------------------------------------------------------------------
# Special cases with closed forms
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("fmt", [X.DOUBLE, X.FLOAT])
@pytest.mark.parametrize("L", [1, 2, 3, 4])
def test_single_value_group(fmt, L):
    rs = np.random.default_rng(21 + L)
    dt = np.float64 if fmt is X.DOUBLE else np.float32
    for _ in range(100):
        b = dt(rs.uniform(-2, 2) * 2.0 ** int(rs.integers(-60, 60)))
        x = Fraction(float(b))
        K = X.top_index(fmt, x)
        low = X.unit(fmt, max(K - L + 1, 0))
        want = X.rne(x / low) * low
        got = X.finalize(X.groupby_sum([0], [b], 1, L, fmt)[0], L, fmt)
        assert got == want
        if L >= 3:
            assert got == x  # a double's bits span at most three levels


@pytest.mark.parametrize("fmt", [X.DOUBLE, X.FLOAT])
def test_cancelling_pairs_give_positive_zero(fmt):
    rs = np.random.default_rng(31)
    dt = np.float64 if fmt is X.DOUBLE else np.float32
    xs = (rs.uniform(-2, 2, 20) * np.exp2(rs.integers(-30, 30, 20))).astype(dt)
    vals = np.concatenate([xs, -xs])
    rs.shuffle(vals)
    out = X.groupby_sum_values(np.zeros(40, int), vals, 1, 3, fmt)
    assert out[0] == 0 and not np.signbit(out[0])


def test_integer_sums_are_exact():
    rs = np.random.default_rng(41)
    vals = rs.integers(-(1 << 40), 1 << 40, 500).astype(np.float64)
    out = X.groupby_sum_values(np.zeros(500, int), vals, 1, 2, X.DOUBLE)
    assert out[0] == float(int(np.sum(vals.astype(np.int64))))


def test_enough_levels_capture_the_exact_sum():
    rs = np.random.default_rng(42)
    vals = rs.uniform(-2, 2, 300) * np.exp2(rs.integers(-10, 11, 300))
    st = X.groupby_sum(np.zeros(300, int), vals, 1, 3, X.DOUBLE)[0]
    lev = sum(st.T[j] * X.unit(X.DOUBLE, st.K - j) for j in range(3))
    assert lev == X.exact_sum(vals)


def test_specials_and_empty_groups():
    f = X.DOUBLE
    nan, inf = float("nan"), float("inf")
    keys = [0, 0, 1, 1, 2, 3, 3, 4, 5, 5]
    vals = [1.0, nan, inf, 2.0, -inf, inf, -inf, 2.0 ** 1010, 0.0, -0.0]
    out = X.groupby_sum_values(keys, vals, 7, 2, f)
    assert np.isnan(out[0]) and out[1] == inf and out[2] == -inf and np.isnan(out[3])
    assert np.isnan(out[4])  # out of range
    assert out[5] == 0 and not np.signbit(out[5])
    assert out[6] == 0 and not np.signbit(out[6])  # empty group


def test_bad_key_rejected():
    with pytest.raises(ValueError):
        X.groupby_sum([0, 3], [1.0, 2.0], 3, 2, X.DOUBLE)

"""Exact big-integer model of reproducible grouped SUM (repro<T,L>).

TEST INFRASTRUCTURE ONLY.  This module is one of two independent oracles for
the reproducible grouped SUM of Mueller, Arteaga, Hoefler, Alonso,
"Reproducible Floating-Point Aggregation in RDBMSs" (arXiv 1802.09883).  Only
``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it; the product path never does.

It computes the method with Python integers and ``fractions.Fraction`` --
no hardware floating point is used for the arithmetic -- in two forms:

* ``groupby_sum`` / ``finalize``: the method's result written out as a
  definition (window from the group's max |b|, digits, exact integer bins,
  one rounding per level, fold from the lowest level).  The C oracle
  (``repro_oracle.c``) follows Algorithm 2 step by step in IEEE arithmetic;
  the two are derived independently and must agree bit for bit.
* ``alg2_init`` / ``alg2_add`` / ``alg2_finalize``: Algorithm 2 replayed literally in a toy binary format
  (m fraction bits, unbounded exponent) so that the paper's worked examples
  (Fig. rsum-example, Fig. carry-example, Sec. III-C) can be replayed and the
  streaming level-raise can be compared with the definition by brute force.

Notation follows Sec. III and Table I: ``m`` fraction bits of the mantissa,
``W`` bits between extraction levels, ``L`` levels, ufp / ulp as in
Sec. III-A.

Readings of the paper taken here (the paper is silent, ambiguous or at odds
with itself on each):

R1  Level raise threshold 2^(W-1) * ulp(S^(1)) exactly as Algorithm 2 lists
    it (the worked example of Fig. rsum-example is only consistent with 2^W;
    2^W is not order-independent, so the listed threshold is used; the
    example is replayed with t = W in ``alg2_add`` to check mechanics).
R2  Extraction against a constant extractor M = 1.5 * ufp(S^(l)) of the
    level, which rounds r / ulp(S) to nearest with ties to even independent
    of the running sum (Algorithm 2 uses the running sum itself, which makes
    ties order-dependent).
R3  All levels sit on one global grid: the unit of grid index k is
    u(k) = 2^(g_min + k W) with g_min the exponent of the smallest subnormal
    (-1074 for double, -149 for float); Sec. III-C leaves the anchor f free.
R4  Carry counts C are exact integers; a level's value is RN(T * u) with T the
    exact integer the level holds (eq. (1) performs exactly this rounding
    whenever its two operands are exact).
R5  NaN / +-Inf / values whose window would overflow S are flagged; the flags
    decide the result (NaN, +-Inf) and such values add nothing to the bins.
R6  Eq. (1) is folded from the lowest level up, left-associative.
R7  Two states merge by aligning to the larger window and dropping levels
    that fall off the bottom (operator+=(repro), Sec. V-B, with eq. (2)/(3)
    for equal windows).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from fractions import Fraction
from typing import Iterable, List, Optional, Sequence, Tuple

import numpy as np

# Group flag bits (shared meaning with the public state layout).
FLAG_NAN = 1
FLAG_POS_INF = 2
FLAG_NEG_INF = 4
FLAG_RANGE = 8


@dataclass(frozen=True)
class Fmt:
    """A binary floating-point format plus the repro parameters W and g_min.

    m: fraction bits (Sec. III-A, ulp(x) = ufp(x) * 2^-m).
    W: bits between consecutive extractors (Sec. III-C; 40 for double,
       18 for float).
    g_min: exponent of the unit of grid index 0 (reading R3).
    emin / emax: exponent range of normal numbers; None for a toy format with
       an unbounded exponent (no subnormals, no overflow).
    """

    name: str
    m: int
    W: int
    g_min: int
    emin: Optional[int] = None
    emax: Optional[int] = None

    @property
    def bounded(self) -> bool:
        return self.emax is not None


DOUBLE = Fmt("double", m=52, W=40, g_min=-1074, emin=-1022, emax=1023)
FLOAT = Fmt("float", m=23, W=18, g_min=-149, emin=-126, emax=127)


def toy(m: int, W: int, g_min: int) -> Fmt:
    """Toy format with m fraction bits and an unbounded exponent."""
    return Fmt(f"toy(m={m},W={W})", m=m, W=W, g_min=g_min)


# --------------------------------------------------------------------------
# Integer rounding and the format's rounding function (Sec. II-B, "rd")
# --------------------------------------------------------------------------

def rne(x: Fraction) -> int:
    """Round a rational to the nearest integer, ties to even."""
    x = Fraction(x)
    fl = x.numerator // x.denominator
    rem = x - fl
    if rem > Fraction(1, 2):
        return fl + 1
    if rem < Fraction(1, 2):
        return fl
    return fl + (fl & 1)


def trunc_toward_zero(x: Fraction) -> int:
    x = Fraction(x)
    q = abs(x.numerator) // x.denominator
    return q if x >= 0 else -q


def floor_log2(x: Fraction) -> int:
    """The integer e with 2^e <= |x| < 2^(e+1), for x != 0."""
    x = abs(Fraction(x))
    if x == 0:
        raise ValueError("log2(0) is undefined")
    e = x.numerator.bit_length() - x.denominator.bit_length()
    if Fraction(2) ** e > x:
        e -= 1
    return e


def ufp(x: Fraction) -> Fraction:
    """Unit in the first place: 2^E for x = M 2^E, M in [1, 2) (Sec. III-A)."""
    return Fraction(2) ** floor_log2(x)


def ulp(x: Fraction, fmt: Fmt) -> Fraction:
    """Unit in the last place: ufp(x) * 2^-m (Sec. III-A)."""
    return ufp(x) / (Fraction(2) ** fmt.m)


def rd(x: Fraction, fmt: Fmt, mode: str = "rne"):
    """Round the exact rational x into fmt.

    mode "rne": round to nearest, ties to even, with gradual underflow and
    overflow to +-inf for bounded formats (returns a float('inf') object on
    overflow).  mode "trunc": truncation toward zero (the rd of the toy
    example in Sec. II-B).  Finite results are returned as Fractions.
    """
    x = Fraction(x)
    if x == 0:
        return Fraction(0)
    e = floor_log2(x)
    if fmt.bounded and e < fmt.emin:
        e = fmt.emin  # subnormal range: fixed quantum 2^(emin - m)
    q = Fraction(2) ** (e - fmt.m)  # the quantum (ulp) at this binade
    if mode == "rne":
        k = rne(x / q)
    elif mode == "trunc":
        k = trunc_toward_zero(x / q)
    else:
        raise ValueError(mode)
    y = k * q
    if fmt.bounded:
        max_finite = (2 - Fraction(2) ** (-fmt.m)) * Fraction(2) ** fmt.emax
        if abs(y) > max_finite:
            return float("inf") if y > 0 else float("-inf")
    return y


def fadd(a, b, fmt: Fmt, mode: str = "rne"):
    """a (+) b = rd(a + b) (Sec. II-B)."""
    return rd(Fraction(a) + Fraction(b), fmt, mode)


def fsub(a, b, fmt: Fmt, mode: str = "rne"):
    """a (-) b = rd(a - b)."""
    return rd(Fraction(a) - Fraction(b), fmt, mode)


# --------------------------------------------------------------------------
# The global grid (reading R3) and the window of a value (Algorithm 2, R1)
# --------------------------------------------------------------------------

def unit(fmt: Fmt, k: int) -> Fraction:
    """u(k) = 2^(g_min + k W): the unit of grid index k."""
    return Fraction(2) ** (fmt.g_min + k * fmt.W)


def k_max(fmt: Fmt) -> Optional[int]:
    """Largest grid index whose running sum S = 1.5 * 2^m * u(k) is finite."""
    if not fmt.bounded:
        return None
    k = 0
    while fmt.m + fmt.g_min + (k + 1) * fmt.W <= fmt.emax:
        k += 1
    return k


def top_index(fmt: Fmt, b: Fraction) -> int:
    """K(b): the smallest grid index K >= 0 whose level can take b,
    i.e. |b| < 2^(W-1) * u(K) (Algorithm 2's raise condition, reading R1)."""
    b = abs(Fraction(b))
    if b == 0:
        return 0
    e = floor_log2(b)  # |b| >= 2^x  <=>  e >= x for integer x
    K = 0
    while e >= fmt.W - 1 + fmt.g_min + K * fmt.W:
        K += 1
    return K


def digits(fmt: Fmt, b: Fraction, K: int, L: int) -> List[int]:
    """The L digits of b in the window whose top grid index is K.

    Level j has unit u_j = u(K - j).  Each digit is the contribution
    q^(j) / u_j of Algorithm 2's transform: c_j = RNE(r_{j-1} / u_j) and
    r_j = r_{j-1} - c_j u_j, with r_{-1} = b (reading R2 for the ties).
    Levels with K - j < 0 do not exist and hold 0.
    """
    r = Fraction(b)
    out = []
    for j in range(L):
        if K - j < 0:
            if r != 0:
                raise AssertionError("value below the grid")
            out.append(0)
            continue
        u = unit(fmt, K - j)
        c = rne(r / u)
        out.append(c)
        r = r - c * u
    return out


# --------------------------------------------------------------------------
# Per-group state and the grouped SUM as a definition
# --------------------------------------------------------------------------

@dataclass
class GroupState:
    """Canonical state of one group: top grid index K, flags, exact bins T."""

    K: int = 0
    flags: int = 0
    T: List[int] = field(default_factory=list)

    def copy(self) -> "GroupState":
        return GroupState(self.K, self.flags, list(self.T))


def classify(fmt: Fmt, b) -> Tuple[int, Optional[Fraction]]:
    """Return (flag bits, exact value or None) for one input value."""
    bf = float(b)
    if bf != bf:
        return FLAG_NAN, None
    if bf == float("inf"):
        return FLAG_POS_INF, None
    if bf == float("-inf"):
        return FLAG_NEG_INF, None
    x = Fraction(bf) if not isinstance(b, Fraction) else b
    km = k_max(fmt)
    if km is not None and top_index(fmt, x) > km:
        return FLAG_RANGE, None
    return 0, x


def groupby_sum(keys: Sequence[int], values: Sequence, G: int, L: int,
                fmt: Fmt) -> List[GroupState]:
    """Grouped reproducible SUM written as a definition.

    Pass 1 fixes each group's window from its largest |b| (the smallest K
    with max |b| < 2^(W-1) u(K), which is where Algorithm 2's level raising
    ends up); pass 2 sums each value's window digits into exact integer bins.
    Keys outside [0, G) raise ValueError.
    """
    xs: List[Tuple[int, Optional[Fraction], int]] = []
    states = [GroupState(0, 0, [0] * L) for _ in range(G)]
    for k, b in zip(keys, values):
        k = int(k)
        if not 0 <= k < G:
            raise ValueError(f"key {k} outside [0, {G})")
        fl, x = classify(fmt, b)
        states[k].flags |= fl
        if x is not None:
            states[k].K = max(states[k].K, top_index(fmt, x))
            xs.append((k, x, 0))
    for k, x, _ in xs:
        st = states[k]
        for j, c in enumerate(digits(fmt, x, st.K, L)):
            st.T[j] += c
    return states


def merge(a: GroupState, b: GroupState, L: int) -> GroupState:
    """operator+=(repro) (Sec. V-B) under reading R7: align to the larger
    window, drop the levels that fall below it, add bins, OR the flags."""
    K = max(a.K, b.K)
    out = GroupState(K, a.flags | b.flags, [0] * L)
    for s in (a, b):
        d = K - s.K
        for j in range(L):
            if j - d >= 0:
                out.T[j] += s.T[j - d]
    return out


def level_values(st: GroupState, L: int, fmt: Fmt) -> List:
    """V_j = RN(T_j u_j) (reading R4)."""
    return [rd(st.T[j] * unit(fmt, st.K - j), fmt) if st.K - j >= 0 else Fraction(0)
            for j in range(L)]


def finalize(st: GroupState, L: int, fmt: Fmt, mode: str = "fold"):
    """Eq. (1): Q = sum of the level values, folded from the lowest level
    (j = L-1) up to the top (j = 0) in the format's arithmetic (R6).

    Returns a Fraction for a finite result, or float nan / +-inf.
    """
    if st.flags & (FLAG_NAN | FLAG_RANGE) or (st.flags & FLAG_POS_INF and st.flags & FLAG_NEG_INF):
        return float("nan")
    if st.flags & FLAG_POS_INF:
        return float("inf")
    if st.flags & FLAG_NEG_INF:
        return float("-inf")
    vs = level_values(st, L, fmt)
    q = vs[L - 1]
    for j in range(L - 2, -1, -1):
        if isinstance(q, float) or isinstance(vs[j], float):
            q = float(q) + float(vs[j])  # IEEE inf arithmetic on overflowed levels
            continue
        q = fadd(q, vs[j], fmt)
    return q


def to_float(x, fmt: Fmt):
    """Convert a finalize() result to the host type of the format."""
    if isinstance(x, float):
        return np.float64(x) if fmt is DOUBLE else np.float32(x)
    if fmt is DOUBLE:
        return np.float64(float(x))  # exact: x is a double
    if fmt is FLOAT:
        return np.float32(float(x))  # exact: x is a float
    return x


def groupby_sum_values(keys, values, G: int, L: int, fmt: Fmt) -> np.ndarray:
    """Finalized grouped SUM as a numpy array of the format's type."""
    sts = groupby_sum(keys, values, G, L, fmt)
    dt = np.float64 if fmt is DOUBLE else np.float32
    return np.array([to_float(finalize(s, L, fmt), fmt) for s in sts], dtype=dt)


# --------------------------------------------------------------------------
# Independent references used to pin the model
# --------------------------------------------------------------------------

def exact_sum(values: Iterable) -> Fraction:
    """Big-integer superaccumulator: the exact sum of the values."""
    s = Fraction(0)
    for v in values:
        s += Fraction(float(v))
    return s


def error_bound_conventional(n: int, eps: float, sum_abs: float) -> float:
    """Eq. (5): e_conv = (n - 1) * eps * sum |b_i|."""
    return (n - 1) * eps * sum_abs


def error_bound_rsum(n: int, L: int, W: int, max_abs: float) -> float:
    """Eq. (6): e_RSum = n * 2^((1-L) W - 1) * max |b_i|."""
    return n * 2.0 ** ((1 - L) * W - 1) * max_abs


# --------------------------------------------------------------------------
# Algorithm 2 replayed literally in a toy format (worked examples, brute force)
# --------------------------------------------------------------------------

@dataclass
class ReplayState:
    S: List[Fraction]
    C: List[int]
    raises: int = 0
    carries: List[int] = field(default_factory=list)


def alg2_init(fmt: Fmt, L: int, f: int) -> ReplayState:
    """S^(l) = 1.5 * 2^(f - (l-1) W), C^(l) = 0 (Sec. III-C)."""
    return ReplayState([Fraction(3, 2) * Fraction(2) ** (f - l * fmt.W) for l in range(L)],
                       [0] * L)


def alg2_add(st: ReplayState, b, fmt: Fmt, t: int, extractor: str = "running") -> None:
    """One iteration of Algorithm 2 for value b in the toy format.

    t: the raise threshold exponent (|b| >= 2^t * ulp(S^(1)) raises; the
    listing has t = W-1, the worked example needs t = W).
    extractor: "running" uses S^(l) itself as in the listing, "constant"
    uses 1.5 * ufp(S^(l)) (reading R2).
    """
    b = Fraction(b)
    L = len(st.S)
    # check extractor validity, raise levels if needed
    while abs(b) >= Fraction(2) ** t * ulp(st.S[0], fmt):
        for l in range(L - 1, 0, -1):
            st.S[l] = st.S[l - 1]
            st.C[l] = st.C[l - 1]
        st.S[0] = Fraction(3, 2) * Fraction(2) ** fmt.W * ufp(st.S[1] if L > 1 else st.S[0])
        st.C[0] = 0
        st.raises += 1
    # transform
    r = b
    for l in range(L):
        ext = st.S[l] if extractor == "running" else Fraction(3, 2) * ufp(st.S[l])
        q = fsub(fadd(r, ext, fmt), ext, fmt)
        st.S[l] = fadd(st.S[l], q, fmt)
        r = fsub(r, q, fmt)
    # carry-bit propagation
    st.carries = []
    for l in range(L):
        u = ufp(st.S[l])
        lo, hi = Fraction(3, 2) * u, Fraction(7, 4) * u
        d = 0
        while not (lo <= st.S[l] - d * u / 4 < hi):
            d += 1 if st.S[l] - d * u / 4 >= hi else -1
        st.S[l] = fsub(st.S[l], d * u / 4, fmt)
        st.C[l] += d
        st.carries.append(d)


def alg2_finalize(st: ReplayState, fmt: Fmt) -> Fraction:
    """Eq. (1) folded from the last level (R6), in the toy format."""
    vals = []
    for S, C in zip(st.S, st.C):
        u = ufp(S)
        vals.append(fadd(fsub(S, Fraction(3, 2) * u, fmt), u / 4 * C, fmt))
    q = vals[-1]
    for v in reversed(vals[:-1]):
        q = fadd(q, v, fmt)
    return q


def alg2_level_integers(st: ReplayState, fmt: Fmt) -> List[int]:
    """The exact integer T^(l) = (S - 1.5 ufp(S)) / ulp(S) + C 2^(m-2)
    held by each level of a replay state."""
    out = []
    for S, C in zip(st.S, st.C):
        u = ufp(S)
        t = (S - Fraction(3, 2) * u) / ulp(S, fmt) + C * 2 ** (fmt.m - 2)
        assert t.denominator == 1
        out.append(int(t))
    return out

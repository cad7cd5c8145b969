"""Seeded synthetic inputs for the grouped SUM: keys and values only.

This module draws random numbers and nothing else -- it holds none of the
method's arithmetic -- so both the CUDA path and the CPU oracles can be fed
from it.  Every generator takes a seed and a torch device; the same seed on
the same device gives the same tensors.

Value recipe (the paper's workloads are keys uniform in [0, G) with
floating-point values, Sec. VI-A): value = s * M * 2^e with a fair random
sign s, M uniform in [1, 2) with all fraction bits random, and e a uniform
integer in [e_lo, e_hi].  The values are composed bit by bit, so no rounding
enters the generator.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Optional, Tuple

import torch


def _gen(seed: int, device) -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return g


def random_values(n: int, e_lo: int, e_hi: int, gen: torch.Generator, device,
                  dtype=torch.float64) -> torch.Tensor:
    """n values s * M * 2^e composed from random sign, fraction and exponent bits."""
    if dtype == torch.float64:
        frac = torch.randint(0, 1 << 52, (n,), generator=gen, device=device, dtype=torch.int64)
        e = torch.randint(e_lo, e_hi + 1, (n,), generator=gen, device=device, dtype=torch.int64)
        s = torch.randint(0, 2, (n,), generator=gen, device=device, dtype=torch.int64)
        bits = (s << 63) | ((e + 1023) << 52) | frac
        return bits.view(torch.float64)
    if dtype == torch.float32:
        frac = torch.randint(0, 1 << 23, (n,), generator=gen, device=device, dtype=torch.int32)
        e = torch.randint(e_lo, e_hi + 1, (n,), generator=gen, device=device, dtype=torch.int32)
        s = torch.randint(0, 2, (n,), generator=gen, device=device, dtype=torch.int32)
        bits = (s << 31) | ((e + 127) << 23) | frac
        return bits.view(torch.float32)
    raise ValueError("dtype must be float64 or float32")


def binade_top_values(n: int, e: int, m_min: float, gen: torch.Generator, device, sign: int = 0) -> torch.Tensor:
    """n float64 values s * M * 2^e with M uniform in [m_min, 2) (all fraction
    bits random above that floor): magnitudes packed at the top of one binade.
    sign = +1 or -1 fixes the sign, 0 draws it."""
    lo = int((m_min - 1.0) * (1 << 52))
    frac = torch.randint(lo, 1 << 52, (n,), generator=gen, device=device, dtype=torch.int64)
    if sign == 0:
        s = torch.randint(0, 2, (n,), generator=gen, device=device, dtype=torch.int64)
    else:
        s = torch.full((n,), 1 if sign < 0 else 0, device=device, dtype=torch.int64)
    bits = (s << 63) | ((e + 1023) << 52) | frac
    return bits.view(torch.float64)


def uniform_keys(n: int, G: int, gen, device) -> torch.Tensor:
    """Keys uniform in [0, G) (Sec. VI-A)."""
    return torch.randint(0, G, (n,), generator=gen, device=device, dtype=torch.int32)


def zipf_keys(n: int, G: int, s: float, gen, device) -> torch.Tensor:
    """Keys with rank-r probability proportional to r^-s, ranks mapped to keys
    by a seeded permutation of [0, G)."""
    r = torch.arange(1, G + 1, device=device, dtype=torch.float64)
    cdf = torch.cumsum(r.pow(-s), 0)
    cdf = cdf / cdf[-1]
    u = torch.rand(n, generator=gen, device=device, dtype=torch.float64)
    rank = torch.searchsorted(cdf, u).clamp_(max=G - 1)
    perm = torch.randperm(G, generator=gen, device=device)
    return perm[rank].to(torch.int32)


@dataclass
class Workload:
    keys: torch.Tensor      # int32[n]
    values: torch.Tensor    # float64[n] or float32[n]
    G: int
    L: int
    name: str

    @property
    def n(self) -> int:
        return int(self.keys.numel())


def plain(n: int = 1_000_000, G: int = 1024, L: int = 3, seed: int = 1, device="cpu",
          e_lo: int = -10, e_hi: int = 10, dtype=torch.float64) -> Workload:
    """Plain repro SUM: keys uniform over G groups, exponents uniform in
    [e_lo, e_hi] (defaults: 10^6 rows, 1024 groups, L = 3, seed 1)."""
    g = _gen(seed, device)
    keys = uniform_keys(n, G, g, device)
    vals = random_values(n, e_lo, e_hi, g, device, dtype)
    return Workload(keys, vals, G, L, f"plain n={n} G={G} L={L} e=[{e_lo},{e_hi}]")


def sweep_cell(G: int, dist: str = "uniform", L: int = 3, n: int = 1 << 28, seed: Optional[int] = None,
               device="cpu", dtype=torch.float64, pair_frac: float = 0.10) -> Workload:
    """One cell of the group-count sweep: n rows, keys uniform or Zipf(1.1)
    over G groups, exponents uniform in [-40, 40], and a fraction pair_frac
    of the rows made of cancelling pairs (k, x), (k, -x) shuffled in."""
    if seed is None:  # one seed per cell: 101 + index over (dist, G, L)
        gi = [16, 1 << 10, 1 << 16, 1 << 20, 1 << 24].index(G) if G in (16, 1 << 10, 1 << 16, 1 << 20, 1 << 24) else 0
        seed = 101 + 15 * (dist == "zipf") + 3 * gi + (L - 2 if 2 <= L <= 4 else 0)
    g = _gen(seed, device)
    n_pairs = int(n * pair_frac) // 2
    n_main = n - 2 * n_pairs

    def draw_keys(m):
        if dist == "uniform":
            return uniform_keys(m, G, g, device)
        if dist == "zipf":
            return zipf_keys(m, G, 1.1, g, device)
        raise ValueError(dist)

    k_main = draw_keys(n_main)
    v_main = random_values(n_main, -40, 40, g, device, dtype)
    k_pair = draw_keys(n_pairs)
    v_pair = random_values(n_pairs, -40, 40, g, device, dtype)
    keys = torch.cat([k_main, k_pair, k_pair])
    vals = torch.cat([v_main, v_pair, -v_pair])
    del k_main, v_main, k_pair, v_pair
    perm = torch.randperm(n, generator=g, device=device)
    keys = keys[perm]
    vals = vals[perm]
    del perm
    return Workload(keys, vals, G, L, f"sweep n={n} G={G} {dist} L={L}")


def few_groups_multicol(n: int = 60_000_000, seed: int = 2, device="cpu") -> Tuple[torch.Tensor, torch.Tensor, torch.Tensor]:
    """Few-group multi-column input: two uint8 key columns with 2 values each
    and four double columns from two-decimal prices p in [900, 105000] and
    discounts d in [0, 0.10]: p, d, p*(1-d), p*d.  Returns (k1, k2, cols[4, n])."""
    g = _gen(seed, device)
    k1 = torch.randint(0, 2, (n,), generator=g, device=device, dtype=torch.uint8)
    k2 = torch.randint(0, 2, (n,), generator=g, device=device, dtype=torch.uint8)
    p = torch.randint(90000, 10500001, (n,), generator=g, device=device, dtype=torch.int64).to(torch.float64) / 100
    d = torch.randint(0, 11, (n,), generator=g, device=device, dtype=torch.int64).to(torch.float64) / 100
    cols = torch.stack([p, d, p * (1 - d), p * d])
    return k1, k2, cols


def log_uniform_ints(m: int, lo: float, hi: float, gen, device="cpu") -> torch.Tensor:
    """m integers round(10^U) with U uniform in [log10 lo, log10 hi]."""
    import math
    u = torch.rand(m, generator=gen, device=device, dtype=torch.float64)
    x = torch.pow(10.0, math.log10(lo) + u * (math.log10(hi) - math.log10(lo)))
    return x.round().clamp_(lo, hi).to(torch.int64)


def batched_tasks(num_tasks: int = 4096, seed: int = 3, rows=(1e3, 1e7), groups=(1, 1e5), device="cpu",
                  dtype=torch.float64, e_lo: int = -10, e_hi: int = 10):
    """Independent aggregations: rows and group counts log-uniform in the
    given ranges, keys uniform over each task's groups, values as in plain().
    Returns a list of (keys, values, G)."""
    g = _gen(seed, device)
    n = log_uniform_ints(num_tasks, rows[0], rows[1], g, device).tolist()
    G = log_uniform_ints(num_tasks, groups[0], groups[1], g, device).tolist()
    out = []
    for i in range(num_tasks):
        keys = uniform_keys(n[i], G[i], g, device)
        vals = random_values(n[i], e_lo, e_hi, g, device, dtype)
        out.append((keys, vals, int(G[i])))
    return out


@dataclass
class ServingTable:
    """A resident table the queries of a serving trace scan: one int32 key
    column per group-count level (keys uniform over that many groups) and one
    value column, all max_rows long."""
    keys: torch.Tensor      # int32[levels, max_rows]
    values: torch.Tensor    # float64[max_rows] (or float32)
    groups: Tuple[int, ...]

    def query(self, start: int, rows: int, level: int):
        return self.keys[level, start:start + rows], self.values[start:start + rows], self.groups[level]


def serving_table(max_rows: int, groups=(1, 1e6), levels: int = 25, seed: int = 4, device="cpu",
                  dtype=torch.float64) -> ServingTable:
    """Key columns for `levels` group counts log-spaced over `groups`
    (round(10^x)), values as in plain()."""
    import math
    lo, hi = math.log10(groups[0]), math.log10(groups[1])
    Gs = tuple(sorted({int(round(10 ** (lo + (hi - lo) * i / max(1, levels - 1)))) for i in range(levels)}))
    g = _gen(seed, device)
    keys = torch.empty((len(Gs), max_rows), dtype=torch.int32, device=device)
    for i, G in enumerate(Gs):
        keys[i] = uniform_keys(max_rows, G, g, device)
    vals = random_values(max_rows, -10, 10, g, device, dtype)
    return ServingTable(keys, vals, Gs)


def serving_trace(num_requests: int, table: ServingTable, rows=(1e4, 1e8), seed: int = 4):
    """Queries over `table`: rows log-uniform in `rows`, group count drawn
    log-uniformly among the table's levels, a random start (a multiple of 4
    rows, so every slice keeps 16-byte alignment), and unit-mean exponential
    inter-arrival gaps (scale them by 1/lambda).  Returns (queries, gaps) with
    queries a list of (start, rows, level)."""
    g = _gen(seed, "cpu")
    max_rows = table.values.numel()
    n = log_uniform_ints(num_requests, rows[0], min(rows[1], max_rows), g).tolist()
    lvl = torch.randint(0, len(table.groups), (num_requests,), generator=g).tolist()
    u = torch.rand(num_requests, generator=g, dtype=torch.float64)
    start = [int(float(u[i]) * (max_rows - n[i])) // 4 * 4 for i in range(num_requests)]
    gaps = (-torch.log1p(-torch.rand(num_requests, generator=g, dtype=torch.float64))).tolist()
    return [(start[i], int(n[i]), int(lvl[i])) for i in range(num_requests)], gaps

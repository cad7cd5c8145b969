"""COUNT / SUM / AVG / VARIANCE / STDDEV per group from reproducible sums.

Test infrastructure, like the rest of oracle/: imported only by the tests,
the smoke check and the CPU legs of bench.py; the CUDA path never uses it.

The paper observes that once SUM is reproducible every SQL aggregate can be
made reproducible: COUNT needs no floating point and VARIANCE / STDDEV are
computed from sums (Sec. I).  This module computes, per group, from the C
oracle's reproducible SUM(x) and SUM(x*x) (each product rounded to nearest in
the value type) and an exact row count:
    mean = S / n,  D = max(Q - (S * S) / n, 0),  var_pop = D / n,
    var_samp = D / (n - 1),  stddev_* = sqrt(var_*),
every operation rounded to nearest in the value type, in this order; empty
groups give NaN for the mean and the variances, one row NaN for var_samp.
"""
from __future__ import annotations

import numpy as np

from . import oracle as O


def groupby_stats(keys, values, G: int, L: int, threads: int = 1) -> dict:
    keys = np.ascontiguousarray(keys, dtype=np.int32)
    values = np.ascontiguousarray(values)
    dt = values.dtype.type
    ok = (keys >= 0) & (keys < G)
    k, v = keys[ok], values[ok]
    count = np.bincount(k, minlength=G).astype(np.int64)
    S = O.groupby_sum_values(k, v, G, L, dtype=values.dtype, threads=threads)
    Q = O.groupby_sum_values(k, (v * v).astype(values.dtype), G, L, dtype=values.dtype, threads=threads)
    n = count.astype(values.dtype)
    nan = dt(np.nan)
    with np.errstate(all="ignore"):
        mean = np.where(count > 0, S / n, nan).astype(values.dtype)
        D = (Q - (S * S) / n).astype(values.dtype)
        D = np.where(D < 0, dt(0), D).astype(values.dtype)
        var_pop = np.where(count > 0, D / n, nan).astype(values.dtype)
        var_samp = np.where(count > 1, D / (n - dt(1)), nan).astype(values.dtype)
        return {"count": count, "sum": S, "mean": mean, "var_samp": var_samp, "var_pop": var_pop,
                "stddev_samp": np.sqrt(var_samp).astype(values.dtype),
                "stddev_pop": np.sqrt(var_pop).astype(values.dtype)}

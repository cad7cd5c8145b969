"""Pins for the stats oracle (COUNT / AVG / VARIANCE / STDDEV from sums,
Sec. I): closed forms on small exact inputs, empty and single-row groups."""
import numpy as np

from oracle import stats as OS


def test_closed_forms_on_exact_inputs():
    keys = np.array([0, 0, 0, 0, 1, 1, 1, 3], dtype=np.int32)
    vals = np.array([1.0, 2.0, 3.0, 4.0, 5.5, 5.5, 5.5, -7.25])
    r = OS.groupby_stats(keys, vals, 5, 3)
    assert r["count"].tolist() == [4, 3, 0, 1, 0]
    assert r["sum"][0] == 10.0 and r["mean"][0] == 2.5
    assert r["var_pop"][0] == 1.25  # mean of squares 7.5 minus 2.5^2
    assert r["var_samp"][0] == 5.0 / 3.0  # 5 / 3 rounded to nearest
    assert r["stddev_pop"][0] == np.sqrt(1.25)
    assert r["mean"][1] == 5.5 and r["var_pop"][1] == 0.0 and r["var_samp"][1] == 0.0  # constant group
    assert r["mean"][3] == -7.25 and r["var_pop"][3] == 0.0 and np.isnan(r["var_samp"][3])  # one row
    for f in ("mean", "var_pop", "var_samp", "stddev_pop"):  # empty groups
        assert np.isnan(r[f][2]) and np.isnan(r[f][4])
    assert r["sum"][2] == 0.0


def test_float_variant_rounds_in_float():
    keys = np.zeros(3, dtype=np.int32)
    vals = np.array([0.1, 0.2, 0.3], dtype=np.float32)
    r = OS.groupby_stats(keys, vals, 1, 3)
    assert r["sum"].dtype == np.float32 and r["var_samp"].dtype == np.float32
    S = np.float32(0.1) + np.float32(0.2) + np.float32(0.3)  # exact in the repro sum: tiny values, L = 3
    assert abs(float(r["sum"][0]) - float(S)) <= 1e-7


def test_bad_keys_are_skipped():
    keys = np.array([0, 5, -1, 0], dtype=np.int32)
    vals = np.array([2.0, 100.0, 100.0, 4.0])
    r = OS.groupby_stats(keys, vals, 2, 2)
    assert r["count"].tolist() == [2, 0] and r["mean"][0] == 3.0 and r["var_pop"][0] == 1.0

"""ctypes binding of the C oracle ``repro_oracle.c`` (TEST INFRASTRUCTURE ONLY).

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may
import this module.  ``build()`` compiles the oracle with gcc into
``oracle/_build``; nothing here touches a GPU.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(BUILD_DIR, "librepro_oracle.so")
SOURCES = [os.path.join(HERE, "repro_oracle.c"), os.path.join(HERE, "repro_oracle_body.h")]

FLAG_NAN, FLAG_POS_INF, FLAG_NEG_INF, FLAG_RANGE = 1, 2, 4, 8

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle (plain gcc, no fused multiply-add) if it is stale."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    fresh = os.path.exists(LIB_PATH) and all(
        os.path.getmtime(LIB_PATH) >= os.path.getmtime(s) for s in SOURCES)
    if force or not fresh:
        tmp = LIB_PATH + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off",
               "-fno-fast-math", "-pthread", "-o", tmp, SOURCES[0], "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, LIB_PATH)
    return LIB_PATH


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(LIB_PATH)
        vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
        for suf in ("f64", "f32"):
            getattr(L, "oracle_state_size_" + suf).restype = ctypes.c_size_t
            getattr(L, "oracle_init_" + suf).argtypes = [vp, i64]
            f = getattr(L, "oracle_groupby_sum_" + suf)
            f.argtypes = [vp, vp, i64, i32, i64, vp]
            f.restype = i64
            f = getattr(L, "oracle_groupby_sum_threads_" + suf)
            f.argtypes = [vp, vp, i64, i32, i64, vp, i32]
            f.restype = i64
            getattr(L, "oracle_merge_" + suf).argtypes = [vp, vp, i32, i64]
            getattr(L, "oracle_finalize_" + suf).argtypes = [vp, i32, i64, vp]
            getattr(L, "oracle_to_bins_" + suf).argtypes = [vp, i32, i64, vp, vp, vp, vp]
        _lib = L
    return _lib


def _suffix(dtype) -> str:
    dt = np.dtype(dtype)
    if dt == np.float64:
        return "f64"
    if dt == np.float32:
        return "f32"
    raise ValueError("dtype must be float64 or float32")


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


@dataclass
class State:
    """G oracle states (the paper's <S[L], C[L]> per group, plus K and flags)."""

    dtype: np.dtype
    L: int
    G: int
    buf: np.ndarray

    @property
    def suf(self) -> str:
        return _suffix(self.dtype)


def init(dtype, L: int, G: int) -> State:
    if not 1 <= L <= 4:
        raise ValueError("L must be in 1..4")
    suf = _suffix(dtype)
    size = getattr(lib(), "oracle_state_size_" + suf)()
    buf = np.zeros(size * max(G, 1), dtype=np.uint8)
    getattr(lib(), "oracle_init_" + suf)(_ptr(buf), G)
    return State(np.dtype(dtype), L, G, buf)


def groupby_sum(st: State, keys, values, threads: int = 1) -> int:
    """Accumulate rows into st; returns the number of rows with a bad key."""
    keys = np.ascontiguousarray(keys, dtype=np.int32)
    values = np.ascontiguousarray(values, dtype=st.dtype)
    if keys.shape != values.shape:
        raise ValueError("keys and values differ in length")
    n = keys.size
    if threads == 1:
        return int(getattr(lib(), "oracle_groupby_sum_" + st.suf)(
            _ptr(keys), _ptr(values), n, st.L, st.G, _ptr(st.buf)))
    bad = int(getattr(lib(), "oracle_groupby_sum_threads_" + st.suf)(
        _ptr(keys), _ptr(values), n, st.L, st.G, _ptr(st.buf), threads))
    if bad < 0:
        raise MemoryError("oracle: private tables could not be allocated")
    return bad


def merge(dst: State, src: State) -> None:
    assert (dst.dtype, dst.L, dst.G) == (src.dtype, src.L, src.G)
    getattr(lib(), "oracle_merge_" + dst.suf)(_ptr(dst.buf), _ptr(src.buf), dst.L, dst.G)


def finalize(st: State) -> np.ndarray:
    out = np.empty(st.G, dtype=st.dtype)
    getattr(lib(), "oracle_finalize_" + st.suf)(_ptr(st.buf), st.L, st.G, _ptr(out))
    return out


def to_bins(st: State):
    """(K[G] int32, flags[G] uint32, lo[G, L] int64, hi[G, L] int64): the exact
    level integers T = hi 2^64 + lo (both halves signed)."""
    K = np.empty(st.G, np.int32)
    fl = np.empty(st.G, np.uint32)
    lo = np.empty((st.G, st.L), np.int64)
    hi = np.empty((st.G, st.L), np.int64)
    getattr(lib(), "oracle_to_bins_" + st.suf)(_ptr(st.buf), st.L, st.G, _ptr(K), _ptr(fl),
                                               _ptr(lo), _ptr(hi))
    return K, fl, lo, hi


def groupby_sum_values(keys, values, G: int, L: int, dtype=np.float64, threads: int = 1) -> np.ndarray:
    st = init(dtype, L, G)
    bad = groupby_sum(st, keys, values, threads)
    if bad:
        raise ValueError(f"{bad} keys outside [0, {G})")
    return finalize(st)

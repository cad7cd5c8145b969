"""Reproducible grouped SUM (repro<T,L>) on GB300.

Python binding of librepro.so (C ABI in include/repro.h).  This module only
marshals arguments -- device pointers from torch tensors and the current
CUDA stream -- and every step of the computation runs in the library's CUDA
kernels.  There is no CPU fallback: without a CUDA device or without the
compiled library the calls raise.

    import torch, paper_1802_09883_gb300 as repro
    out = repro.groupby_sum(keys, values, num_groups=1024, L=3)   # float64[G]

    st = repro.State(num_groups=1024, L=3)                        # resumable
    st.add(keys_part1, values_part1); st.add(keys_part2, values_part2)
    st.merge(other_state); out = st.finalize()
"""
from __future__ import annotations

import ctypes
import os
import re
from typing import Optional

import numpy as np
import torch

from . import build as _build

REPRO_F64 = 0
REPRO_F32 = 1
FLAG_NAN, FLAG_POS_INF, FLAG_NEG_INF, FLAG_RANGE = 1, 2, 4, 8
ERR_KEY, ERR_TIMEOUT, ERR_LAYOUT = 1, 2, 4
HEADER_BYTES = 64

STATUS = {0: "REPRO_OK", 1: "REPRO_EINVAL", 2: "REPRO_EKEY", 3: "REPRO_ERANGE", 4: "REPRO_ENOMEM",
          5: "REPRO_ECUDA", 6: "REPRO_ETIMEOUT", 7: "REPRO_ELAYOUT"}

_lib = None


class ReproError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = lib().repro_strerror(status).decode() if _lib is not None else STATUS.get(status, "?")
        super().__init__(f"{where}: {STATUS.get(status, status)} ({msg})")


def library_path() -> str:
    return _build.LIB


def declared_functions():
    """Names of the functions declared in include/repro.h."""
    with open(os.path.join(_build.INCLUDE, "repro.h")) as fh:
        text = fh.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^[A-Za-z_][\w\s\*]*?\b(\w+)\s*\(", text, flags=re.M)) - {"if", "defined"})


def lib(build_if_stale: bool = True):
    """Load librepro.so (building it first when missing or stale)."""
    global _lib
    if _lib is None:
        if build_if_stale:
            _build.build()
        if not os.path.exists(_build.LIB):
            raise RuntimeError("librepro.so is not built; run paper_1802_09883_gb300.build.build()")
        L = ctypes.CDLL(_build.LIB)
        vp, i64, i32, u32p = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.POINTER(ctypes.c_uint32)
        L.repro_state_bytes.argtypes = [i32, i32, i64]
        L.repro_state_bytes.restype = ctypes.c_size_t
        L.repro_state_init.argtypes = [vp, i32, i32, i64, vp]
        L.repro_groupby_sum.argtypes = [vp, vp, i64, i32, i32, i64, vp, vp]
        L.repro_groupby_sum_noalloc.argtypes = [vp, vp, i64, i32, i32, i64, vp, vp]
        L.repro_groupby_sum_adaptive.argtypes = [vp, vp, i64, i32, i32, i64, vp, ctypes.POINTER(ctypes.c_int), vp]
        L.repro_merge.argtypes = [vp, vp, i32, i32, i64, vp]
        L.repro_merge_records.argtypes = [vp, vp, i32, i64, vp]
        L.repro_finalize.argtypes = [vp, i32, i32, i64, vp, vp]
        L.repro_state_check.argtypes = [vp, u32p, vp]
        L.groupby_sum_fp64.argtypes = [vp, vp, i64, i64, vp, vp]
        L.groupby_sum_fp32.argtypes = [vp, vp, i64, i64, vp, vp]
        L.groupby_sum_fp_mode.argtypes = [vp, vp, i64, i32, i64, i32, vp, vp]
        L.repro_batch_prepare.argtypes = [vp, i32, i32, i32, ctypes.POINTER(vp)]
        L.repro_batch_run.argtypes = [vp, vp]
        L.repro_batch_destroy.argtypes = [vp]
        L.repro_batch_reset.argtypes = [vp, vp]
        L.repro_batch_describe.argtypes = [vp, vp]
        L.repro_batch_set_outputs.argtypes = [vp, vp]
        L.repro_batch_finalize.argtypes = [vp, vp]
        L.repro_groupby_sum_batched.argtypes = [vp, i32, i32, i32, vp]
        L.repro_groupby_sum_cols.argtypes = [vp, vp, i32, vp, i32, i64, i32, i32, i64, vp, vp]
        L.repro_release_cached_memory.argtypes = []
        L.repro_strerror.argtypes = [i32]
        L.repro_strerror.restype = ctypes.c_char_p
        L.repro_version.restype = i32
        u64p = ctypes.POINTER(ctypes.c_uint64)
        L.repro_server_now_ns.argtypes = []
        L.repro_server_now_ns.restype = i64
        L.repro_server_create.argtypes = [vp, ctypes.POINTER(vp)]
        L.repro_server_submit.argtypes = [vp, vp, vp, i64, i32, i32, i64, vp, vp, i64, u64p]
        L.repro_server_poll.argtypes = [vp, ctypes.c_uint64, vp]
        L.repro_server_wait.argtypes = [vp, ctypes.c_uint64, ctypes.c_double, vp]
        L.repro_server_release.argtypes = [vp, ctypes.c_uint64]
        L.repro_server_stats_get.argtypes = [vp, vp]
        L.repro_server_destroy.argtypes = [vp]
        L.repro_tune_groupby.argtypes = [vp, vp, i64, i32, i32, i64, vp, vp]
        L.repro_tune_save.argtypes = [ctypes.c_char_p]
        L.repro_tune_load.argtypes = [ctypes.c_char_p]
        L.repro_tune_clear.argtypes = []
        L.repro_tune_clear.restype = None
        L.repro_batch_tune.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_double)]
        L.repro_sum.argtypes = [vp, i64, i32, i32, vp, vp]
        L.repro_groupby_sum_host.argtypes = [vp, vp, i64, i32, i32, i64, vp, vp]
        L.repro_sum_unbuffered.argtypes = [vp, i64, i32, i32, vp, vp]
        L.groupby_sum_decimal64.argtypes = [vp, vp, i64, i64, vp, vp]
        L.repro_stats_state_bytes.argtypes = [i32, i32, i64]
        L.repro_stats_state_bytes.restype = ctypes.c_size_t
        L.repro_stats_init.argtypes = [vp, i32, i32, i64, vp]
        L.repro_groupby_stats.argtypes = [vp, vp, i64, i32, i32, i64, vp, vp]
        L.repro_stats_merge.argtypes = [vp, vp, i32, i32, i64, vp]
        L.repro_stats_finalize.argtypes = [vp, i32, i32, i64, vp, vp]
        for name in ("repro_state_init", "repro_groupby_sum", "repro_groupby_sum_noalloc", "repro_groupby_sum_adaptive", "repro_merge", "repro_merge_records",
                     "repro_finalize", "repro_batch_prepare", "repro_batch_run", "repro_batch_destroy",
                     "repro_batch_reset", "repro_batch_set_outputs", "repro_batch_finalize", "repro_batch_describe",
                     "repro_groupby_sum_batched", "repro_groupby_sum_cols", "repro_release_cached_memory",
                     "repro_state_check", "groupby_sum_fp64", "groupby_sum_fp32", "groupby_sum_fp_mode", "repro_server_create",
                     "repro_server_submit", "repro_server_poll", "repro_server_wait", "repro_server_release",
                     "repro_server_stats_get", "repro_server_destroy", "repro_tune_groupby", "repro_tune_save",
                     "repro_tune_load", "repro_batch_tune", "repro_stats_init", "repro_groupby_stats",
                     "repro_stats_merge", "repro_stats_finalize", "repro_sum", "repro_sum_unbuffered",
                     "repro_groupby_sum_host",
                     "groupby_sum_decimal64"):
            getattr(L, name).restype = i32
        _lib = L
    return _lib


def _require_cuda(t: torch.Tensor, name: str):
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor (this library has no CPU path)")


def _stream(device) -> int:
    return torch.cuda.current_stream(device).cuda_stream


def _dtype_code(dtype) -> int:
    if dtype == torch.float64:
        return REPRO_F64
    if dtype == torch.float32:
        return REPRO_F32
    raise ValueError("values must be float64 or float32")


def _check(status: int, where: str):
    if status != 0:
        raise ReproError(status, where)


def state_bytes(dtype, L: int, num_groups: int) -> int:
    return int(lib().repro_state_bytes(_dtype_code(dtype), L, num_groups))


class State:
    """G reproducible accumulators repro<T,L> in device memory (the library's
    canonical state layout: header + per group K, flags, L 128-bit bins)."""

    def __init__(self, num_groups: int, L: int = 3, dtype=torch.float64, device=None,
                 tensor: Optional[torch.Tensor] = None):
        if not torch.cuda.is_available():
            raise RuntimeError("paper_1802_09883_gb300 needs a CUDA device")
        self.G = int(num_groups)
        self.L = int(L)
        self.dtype = dtype
        self.code = _dtype_code(dtype)
        nbytes = state_bytes(dtype, self.L, self.G)
        if nbytes == 0:
            raise ValueError("invalid L or num_groups")
        if tensor is not None:
            if tensor.numel() != nbytes or tensor.dtype != torch.uint8:
                raise ValueError("state tensor has the wrong size or dtype")
            self.tensor = tensor
        else:
            dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
            self.tensor = torch.empty(nbytes, dtype=torch.uint8, device=dev)
            self.reset()

    @property
    def device(self):
        return self.tensor.device

    def reset(self):
        _check(lib().repro_state_init(self.tensor.data_ptr(), self.code, self.L, self.G,
                                      _stream(self.device)), "repro_state_init")
        return self

    def add(self, keys: torch.Tensor, values: torch.Tensor):
        """Accumulate rows (keys int32[n], values of the state's dtype)."""
        _require_cuda(keys, "keys")
        _require_cuda(values, "values")
        if keys.dtype != torch.int32:
            raise ValueError("keys must be int32")
        if values.dtype != self.dtype:
            raise ValueError(f"values must be {self.dtype}")
        if keys.numel() != values.numel():
            raise ValueError("keys and values differ in length")
        keys = keys.contiguous()
        values = values.contiguous()
        _check(lib().repro_groupby_sum(keys.data_ptr(), values.data_ptr(), keys.numel(), self.code, self.L,
                                       self.G, self.tensor.data_ptr(), _stream(self.device)),
               "repro_groupby_sum")
        return self

    def add_adaptive(self, keys: torch.Tensor, values: torch.Tensor) -> int:
        """As add(), with the partitioning depth picked from the keys' range
        (a probe of the keys and one stream synchronisation first); returns
        the partition passes taken (0, 1, 2; -1: the plain way)."""
        _require_cuda(keys, "keys")
        _require_cuda(values, "values")
        if keys.dtype != torch.int32 or values.dtype != self.dtype or keys.numel() != values.numel():
            raise ValueError("keys int32 and values of the state's dtype, same length")
        keys, values = keys.contiguous(), values.contiguous()
        depth = ctypes.c_int(-1)
        _check(lib().repro_groupby_sum_adaptive(keys.data_ptr(), values.data_ptr(), keys.numel(), self.code, self.L,
                                                self.G, self.tensor.data_ptr(), ctypes.byref(depth),
                                                _stream(self.device)), "repro_groupby_sum_adaptive")
        return depth.value

    def merge(self, other: "State"):
        if (other.G, other.L, other.dtype) != (self.G, self.L, self.dtype):
            raise ValueError("states differ in num_groups, L or dtype")
        _check(lib().repro_merge(self.tensor.data_ptr(), other.tensor.data_ptr(), self.code, self.L, self.G,
                                 _stream(self.device)), "repro_merge")
        return self

    def finalize(self, out: Optional[torch.Tensor] = None) -> torch.Tensor:
        if out is None:
            out = torch.empty(self.G, dtype=self.dtype, device=self.device)
        _check(lib().repro_finalize(self.tensor.data_ptr(), self.code, self.L, self.G, out.data_ptr(),
                                    _stream(self.device)), "repro_finalize")
        return out

    def add_values(self, values: torch.Tensor):
        """Reproducible SUM of every value into this one-group state."""
        if self.G != 1:
            raise ValueError("add_values needs a state with num_groups = 1")
        _require_cuda(values, "values")
        if values.dtype != self.dtype:
            raise ValueError("values must have the state's dtype")
        values = values.contiguous()
        _check(lib().repro_sum(values.data_ptr(), values.numel(), self.code, self.L, self.tensor.data_ptr(),
                               _stream(self.device)), "repro_sum")
        return self

    def add_host(self, keys: torch.Tensor, values: torch.Tensor):
        """Accumulate pinned host columns: chunked copies overlapped with the
        aggregation (the tensors must stay unchanged until the current
        stream has passed this call)."""
        if keys.is_cuda or values.is_cuda or not keys.is_pinned() or not values.is_pinned():
            raise ValueError("keys and values must be pinned host tensors")
        if keys.dtype != torch.int32 or values.dtype != self.dtype or keys.numel() != values.numel():
            raise ValueError("keys int32 and values of the state's dtype, same length")
        keys, values = keys.contiguous(), values.contiguous()
        _check(lib().repro_groupby_sum_host(keys.data_ptr(), values.data_ptr(), keys.numel(), self.code, self.L,
                                            self.G, self.tensor.data_ptr(), _stream(self.device)),
               "repro_groupby_sum_host")
        return self

    def add_values_unbuffered(self, values: torch.Tensor):
        """The same SUM as add_values through the per-row drop-in type."""
        if self.G != 1:
            raise ValueError("add_values_unbuffered needs a state with num_groups = 1")
        _require_cuda(values, "values")
        if values.dtype != self.dtype:
            raise ValueError("values must have the state's dtype")
        values = values.contiguous()
        _check(lib().repro_sum_unbuffered(values.data_ptr(), values.numel(), self.code, self.L,
                                          self.tensor.data_ptr(), _stream(self.device)), "repro_sum_unbuffered")
        return self

    def error_word(self) -> int:
        """Synchronise and return the state's error word (REPRO_ERR_* bits)."""
        err = ctypes.c_uint32(0)
        st = lib().repro_state_check(self.tensor.data_ptr(), ctypes.byref(err), _stream(self.device))
        if st not in (0, 2, 6, 7):
            _check(st, "repro_state_check")
        return err.value

    def check(self) -> int:
        """Synchronise and raise ReproError if a data error was recorded."""
        err = ctypes.c_uint32(0)
        st = lib().repro_state_check(self.tensor.data_ptr(), ctypes.byref(err), _stream(self.device))
        _check(st, "repro_state_check")
        return err.value

    def clone(self) -> "State":
        return State(self.G, self.L, self.dtype, tensor=self.tensor.clone())

    def host_view(self):
        """(K[G], flags[G], lo[G, L], hi[G, L]) copied to the host."""
        return parse_state(self.tensor.cpu().numpy(), self.L, self.G)


def parse_state(raw: np.ndarray, L: int, G: int):
    """Split raw state bytes into (K, flags, lo[G, L], hi[G, L])."""
    rec = np.dtype([("K", "<i4"), ("flags", "<u4"), ("bins", "<i8", (L, 2))])
    arr = np.frombuffer(raw[HEADER_BYTES:].tobytes(), dtype=rec, count=G)
    return (arr["K"].copy(), arr["flags"].copy(), arr["bins"][:, :, 0].copy(), arr["bins"][:, :, 1].copy())


def groupby_sum(keys: torch.Tensor, values: torch.Tensor, num_groups: int, L: int = 3,
                check: bool = True) -> torch.Tensor:
    """One-shot reproducible SUM ... GROUP BY key: returns values.dtype[num_groups]."""
    st = State(num_groups, L, values.dtype, device=values.device)
    st.add(keys, values)
    out = st.finalize()
    if check:
        st.check()
    return out


def groupby_sum_fp64(keys: torch.Tensor, values: torch.Tensor, num_groups: int,
                     out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """Conventional (non-reproducible) float64 GroupBy baseline."""
    _require_cuda(keys, "keys")
    _require_cuda(values, "values")
    if out is None:
        out = torch.empty(num_groups, dtype=torch.float64, device=values.device)
    _check(lib().groupby_sum_fp64(keys.data_ptr(), values.data_ptr(), keys.numel(), num_groups, out.data_ptr(),
                                  _stream(values.device)), "groupby_sum_fp64")
    return out


def groupby_sum_fp32(keys: torch.Tensor, values: torch.Tensor, num_groups: int,
                     out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """Conventional (non-reproducible) float32 GroupBy baseline."""
    _require_cuda(keys, "keys")
    _require_cuda(values, "values")
    if out is None:
        out = torch.empty(num_groups, dtype=torch.float32, device=values.device)
    _check(lib().groupby_sum_fp32(keys.data_ptr(), values.data_ptr(), keys.numel(), num_groups, out.data_ptr(),
                                  _stream(values.device)), "groupby_sum_fp32")
    return out


FP_MODES = {0: "shared table (one copy per lane when they fit)", 1: "shared table, equal keys combined per warp",
            2: "one shared table per warp", 3: "global atomics", 4: "global atomics, equal keys combined per warp"}


def groupby_sum_fp_mode(keys: torch.Tensor, values: torch.Tensor, num_groups: int, mode: int,
                        out: Optional[torch.Tensor] = None) -> Optional[torch.Tensor]:
    """The conventional baseline with an explicit table strategy (FP_MODES);
    None when that strategy's tables do not fit for num_groups."""
    _require_cuda(keys, "keys")
    _require_cuda(values, "values")
    if out is None:
        out = torch.empty(num_groups, dtype=values.dtype, device=values.device)
    st = lib().groupby_sum_fp_mode(keys.data_ptr(), values.data_ptr(), keys.numel(), _dtype_code(values.dtype),
                                   num_groups, mode, out.data_ptr(), _stream(values.device))
    if st == 3:  # REPRO_ERANGE
        return None
    _check(st, "groupby_sum_fp_mode")
    return out


class _Task(ctypes.Structure):
    _fields_ = [("keys", ctypes.c_void_p), ("values", ctypes.c_void_p), ("n", ctypes.c_int64),
                ("num_groups", ctypes.c_int64), ("state", ctypes.c_void_p)]


class _BatchInfo(ctypes.Structure):
    _fields_ = [("tasks", ctypes.c_int32), ("single_pass_tasks", ctypes.c_int32),
                ("partition_tasks", ctypes.c_int32), ("lane_tasks", ctypes.c_int32), ("items", ctypes.c_int32),
                ("merge_blocks", ctypes.c_int32), ("items_per_cta", ctypes.c_int32),
                ("partition_overlap", ctypes.c_int32),
                ("device_bytes", ctypes.c_int64), ("class_tasks", ctypes.c_int32 * 3), ("reserved", ctypes.c_int32)]


class BatchPlan:
    """Many independent grouped SUMs in one persistent launch.

    tasks: list of (keys, values, State); all States share dtype and L.
    run() enqueues the plan's kernels on the current stream (capturable in a
    CUDA graph); every run adds the tasks' rows into their states again.
    """

    def __init__(self, tasks):
        if not tasks:
            raise ValueError("no tasks")
        st0 = tasks[0][2]
        self.dtype, self.L, self.code = st0.dtype, st0.L, st0.code
        self._keep = []
        arr = (_Task * len(tasks))()
        for i, (k, v, st) in enumerate(tasks):
            _require_cuda(k, "keys")
            _require_cuda(v, "values")
            if (st.dtype, st.L) != (self.dtype, self.L):
                raise ValueError("all tasks must share dtype and L")
            if k.dtype != torch.int32 or v.dtype != self.dtype or k.numel() != v.numel():
                raise ValueError("task %d: keys int32 and values of the batch dtype, same length" % i)
            k, v = k.contiguous(), v.contiguous()
            self._keep.append((k, v, st))
            arr[i] = _Task(k.data_ptr(), v.data_ptr(), k.numel(), st.G, st.tensor.data_ptr())
        self._plan = ctypes.c_void_p()
        _check(lib().repro_batch_prepare(ctypes.cast(arr, ctypes.c_void_p), len(tasks), self.code, self.L,
                                         ctypes.byref(self._plan)), "repro_batch_prepare")
        self.device = st0.device

    def run(self):
        _check(lib().repro_batch_run(self._plan, _stream(self.device)), "repro_batch_run")
        return self

    def describe(self) -> dict:
        """How the plan runs its tasks (single pass / batched partition pass /
        side lanes), its items and the device memory it holds."""
        info = _BatchInfo()
        _check(lib().repro_batch_describe(self._plan, ctypes.byref(info)), "repro_batch_describe")
        out = {name: getattr(info, name) for name, _ in _BatchInfo._fields_ if name != "reserved"}
        out["class_tasks"] = list(info.class_tasks)
        return out

    def tune(self) -> float:
        """Time item sizes for this plan and keep the fastest (the states are
        re-initialised afterwards); returns the median ms of one run."""
        ms = ctypes.c_double(0)
        _check(lib().repro_batch_tune(self._plan, _stream(self.device), ctypes.byref(ms)), "repro_batch_tune")
        return ms.value

    def reset(self):
        """Re-initialise every task's state in one launch."""
        _check(lib().repro_batch_reset(self._plan, _stream(self.device)), "repro_batch_reset")
        return self

    def set_outputs(self, outs):
        """One device tensor (num_groups of the dtype) or None per task."""
        if len(outs) != len(self._keep):
            raise ValueError("one output per task")
        ptrs = (ctypes.c_void_p * len(outs))()
        for i, (o, (_, _, st)) in enumerate(zip(outs, self._keep)):
            if o is None:
                continue
            _require_cuda(o, "out")
            if o.dtype != self.dtype or o.numel() < st.G or not o.is_contiguous():
                raise ValueError("output %d: contiguous, the batch dtype, num_groups elements" % i)
            ptrs[i] = o.data_ptr()
        _check(lib().repro_batch_set_outputs(self._plan, ctypes.cast(ptrs, ctypes.c_void_p)),
               "repro_batch_set_outputs")
        self._outs = list(outs)
        return self

    def finalize(self):
        """Finalize every task with an output, in one launch."""
        _check(lib().repro_batch_finalize(self._plan, _stream(self.device)), "repro_batch_finalize")
        return self

    def close(self):
        if self._plan:
            lib().repro_batch_destroy(self._plan)
            self._plan = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def groupby_sum_batched(tasks, L: int = 3):
    """tasks: list of (keys, values, num_groups); returns one State per task."""
    states = [State(G, L, v.dtype, device=v.device) for _, v, G in tasks]
    plan = BatchPlan([(k, v, st) for (k, v, _), st in zip(tasks, states)])
    plan.run()
    torch.cuda.current_stream(plan.device).synchronize()
    plan.close()
    return states


def groupby_sum_cols(key1: torch.Tensor, key2: torch.Tensor, card2: int, cols, num_groups: int, L: int = 3,
                     states=None):
    """SUM of every column in `cols` grouped by (key1 * card2 + key2), two
    uint8 key columns; returns (and accumulates into) one State per column."""
    _require_cuda(key1, "key1")
    _require_cuda(key2, "key2")
    if key1.dtype != torch.uint8 or key2.dtype != torch.uint8 or key1.numel() != key2.numel():
        raise ValueError("key1 and key2 must be uint8 columns of the same length")
    cols = [c.contiguous() for c in cols]
    dtype = cols[0].dtype
    if any(c.dtype != dtype or c.numel() != key1.numel() for c in cols):
        raise ValueError("all columns must share dtype and length with the keys")
    if states is None:
        states = [State(num_groups, L, dtype, device=cols[0].device) for _ in cols]
    key1, key2 = key1.contiguous(), key2.contiguous()
    cp = (ctypes.c_void_p * len(cols))(*[c.data_ptr() for c in cols])
    sp = (ctypes.c_void_p * len(states))(*[st.tensor.data_ptr() for st in states])
    _check(lib().repro_groupby_sum_cols(key1.data_ptr(), key2.data_ptr(), card2, ctypes.cast(cp, ctypes.c_void_p),
                                        len(cols), key1.numel(), _dtype_code(dtype), L, num_groups,
                                        ctypes.cast(sp, ctypes.c_void_p), _stream(cols[0].device)),
           "repro_groupby_sum_cols")
    return states


def release_cached_memory():
    _check(lib().repro_release_cached_memory(), "repro_release_cached_memory")


class _TuneResult(ctypes.Structure):
    _fields_ = [("path", ctypes.c_int32), ("candidates", ctypes.c_int32), ("stages", ctypes.c_int32),
                ("tile_rows", ctypes.c_int32), ("consumer_warps", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("table_copies", ctypes.c_int32), ("partition_shift", ctypes.c_int32), ("best_ms", ctypes.c_double),
                ("default_ms", ctypes.c_double), ("partition_levels", ctypes.c_int32),
                ("partition_items_per_cta", ctypes.c_int32)]


def tune(keys: torch.Tensor, values: torch.Tensor, num_groups: int, L: int = 3) -> dict:
    """Time every configuration that fits on these inputs and record the
    fastest for (dtype, L, num_groups bucket); returns what was chosen."""
    _require_cuda(keys, "keys")
    _require_cuda(values, "values")
    keys, values = keys.contiguous(), values.contiguous()
    r = _TuneResult()
    _check(lib().repro_tune_groupby(keys.data_ptr(), values.data_ptr(), keys.numel(), _dtype_code(values.dtype), L,
                                    num_groups, _stream(values.device), ctypes.byref(r)), "repro_tune_groupby")
    out = {name: getattr(r, name) for name, _ in _TuneResult._fields_}
    out["path"] = ("single_pass", "partitioned", "two_pass")[r.path]
    return out


def tune_save(path: str):
    _check(lib().repro_tune_save(os.fsencode(path)), "repro_tune_save")


def tune_load(path: str):
    _check(lib().repro_tune_load(os.fsencode(path)), "repro_tune_load")


def tune_clear():
    lib().repro_tune_clear()


class _StatsOut(ctypes.Structure):
    _fields_ = [(name, ctypes.c_void_p) for name in
                ("count", "sum", "mean", "var_samp", "var_pop", "stddev_samp", "stddev_pop")]


STATS_FIELDS = ("count", "sum", "mean", "var_samp", "var_pop", "stddev_samp", "stddev_pop")


class Stats:
    """COUNT / SUM / AVG / VARIANCE / STDDEV per group from reproducible sums
    of x and x*x plus exact row counts (a stats state in device memory)."""

    def __init__(self, num_groups: int, L: int = 3, dtype=torch.float64, device=None):
        if not torch.cuda.is_available():
            raise RuntimeError("paper_1802_09883_gb300 needs a CUDA device")
        self.G, self.L, self.dtype, self.code = int(num_groups), int(L), dtype, _dtype_code(dtype)
        nbytes = int(lib().repro_stats_state_bytes(self.code, self.L, self.G))
        if nbytes == 0:
            raise ValueError("invalid L or num_groups")
        dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.tensor = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        _check(lib().repro_stats_init(self.tensor.data_ptr(), self.code, self.L, self.G, _stream(dev)),
               "repro_stats_init")

    def add(self, keys: torch.Tensor, values: torch.Tensor):
        _require_cuda(keys, "keys")
        _require_cuda(values, "values")
        if keys.dtype != torch.int32 or values.dtype != self.dtype or keys.numel() != values.numel():
            raise ValueError("keys int32 and values of the state's dtype, same length")
        keys, values = keys.contiguous(), values.contiguous()
        _check(lib().repro_groupby_stats(keys.data_ptr(), values.data_ptr(), keys.numel(), self.code, self.L, self.G,
                                         self.tensor.data_ptr(), _stream(self.tensor.device)), "repro_groupby_stats")
        return self

    def merge(self, other: "Stats"):
        _check(lib().repro_stats_merge(self.tensor.data_ptr(), other.tensor.data_ptr(), self.code, self.L, self.G,
                                       _stream(self.tensor.device)), "repro_stats_merge")
        return self

    def check(self) -> int:
        err = ctypes.c_uint32(0)
        _check(lib().repro_state_check(self.tensor.data_ptr(), ctypes.byref(err), _stream(self.tensor.device)),
               "repro_state_check")
        return err.value

    def finalize(self) -> dict:
        dev = self.tensor.device
        res = {"count": torch.empty(self.G, dtype=torch.int64, device=dev)}
        for name in STATS_FIELDS[1:]:
            res[name] = torch.empty(self.G, dtype=self.dtype, device=dev)
        out = _StatsOut(*[res[name].data_ptr() for name in STATS_FIELDS])
        _check(lib().repro_stats_finalize(self.tensor.data_ptr(), self.code, self.L, self.G, ctypes.byref(out),
                                          _stream(dev)), "repro_stats_finalize")
        return res


def groupby_stats(keys: torch.Tensor, values: torch.Tensor, num_groups: int, L: int = 3) -> dict:
    """One-shot COUNT / SUM / AVG / VAR_SAMP / VAR_POP / STDDEV_* GROUP BY key."""
    st = Stats(num_groups, L, values.dtype, device=values.device).add(keys, values)
    res = st.finalize()
    st.check()
    return res


def scalar_sum(values: torch.Tensor, L: int = 3) -> torch.Tensor:
    """Reproducible SUM of a float64/float32 tensor (no GROUP BY): a 0-dim
    tensor of the same dtype, identical for any order or split of the values."""
    st = State(1, L, values.dtype, device=values.device).add_values(values)
    out = st.finalize()
    st.check()
    return out[0]


def groupby_sum_decimal64(keys: torch.Tensor, values: torch.Tensor, num_groups: int,
                          out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """DECIMAL baseline: exact int64 SUM per group of scaled-integer values."""
    _require_cuda(keys, "keys")
    _require_cuda(values, "values")
    if values.dtype != torch.int64 or keys.dtype != torch.int32:
        raise ValueError("keys int32, values int64")
    keys, values = keys.contiguous(), values.contiguous()
    if out is None:
        out = torch.empty(num_groups, dtype=torch.int64, device=values.device)
    _check(lib().groupby_sum_decimal64(keys.data_ptr(), values.data_ptr(), keys.numel(), num_groups, out.data_ptr(),
                                       _stream(values.device)), "groupby_sum_decimal64")
    return out

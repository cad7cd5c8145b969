"""Python binding of the request server (repro_server_* in include/repro.h).

The server is native: a scheduler thread in librepro.so admits queries by
device memory, batches the next chunk of every admitted query into one
multi-task launch per iteration, and stamps completions from a host callback.
This module marshals arguments, keeps each query's tensors alive until it is
done, and runs a timed trace of queries (arrival times given in advance).
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass
from typing import List, Optional, Sequence

import numpy as np
import torch

from . import ReproError, _check, _dtype_code, _require_cuda, lib


class ServerConfig(ctypes.Structure):
    _fields_ = [("memory_budget", ctypes.c_int64), ("chunk_rows", ctypes.c_int64),
                ("max_active", ctypes.c_int32), ("max_inflight", ctypes.c_int32)]


class RequestInfo(ctypes.Structure):
    _fields_ = [("done", ctypes.c_int32), ("status", ctypes.c_int32), ("errors", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32), ("arrival_ns", ctypes.c_int64), ("admit_ns", ctypes.c_int64),
                ("done_ns", ctypes.c_int64)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("iterations", ctypes.c_int64),
                ("batch_launches", ctypes.c_int64), ("large_calls", ctypes.c_int64),
                ("memory_in_use", ctypes.c_int64), ("memory_peak", ctypes.c_int64),
                ("memory_budget", ctypes.c_int64), ("active", ctypes.c_int32), ("waiting", ctypes.c_int32),
                ("memory_server_peak", ctypes.c_int64)]


def now_ns() -> int:
    """The server's clock (monotonic, nanoseconds)."""
    return int(lib().repro_server_now_ns())


@dataclass
class Request:
    id: int
    out: torch.Tensor
    n: int
    num_groups: int
    _keep: tuple

    info: Optional[RequestInfo] = None

    @property
    def latency_s(self) -> float:
        return (self.info.done_ns - self.info.arrival_ns) * 1e-9


class Server:
    """Continuous-batching server for reproducible grouped SUMs on one device."""

    def __init__(self, memory_budget: int = 0, chunk_rows: int = 0, max_active: int = 0, max_inflight: int = 0,
                 device=None):
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        cfg = ServerConfig(memory_budget, chunk_rows, max_active, max_inflight)
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            _check(lib().repro_server_create(ctypes.byref(cfg), ctypes.byref(h)), "repro_server_create")
        self._h = h
        self._reqs = {}

    def submit(self, keys: torch.Tensor, values: torch.Tensor, num_groups: int, L: int = 3,
               out: Optional[torch.Tensor] = None, arrival_ns: int = 0, host_out: bool = True,
               ready: Optional[torch.cuda.Event] = None) -> Request:
        """Queue SUM(values) GROUP BY keys; the result lands in `out` (pinned
        host memory by default).  The inputs must stay unchanged until the
        request is done.  The server waits for `ready` (default: an event
        recorded now on the current stream) before reading them."""
        _require_cuda(keys, "keys")
        _require_cuda(values, "values")
        if keys.dtype != torch.int32 or keys.numel() != values.numel():
            raise ValueError("keys must be int32 and as long as values")
        keys, values = keys.contiguous(), values.contiguous()
        if out is None:
            out = (torch.empty(num_groups, dtype=values.dtype, pin_memory=True) if host_out
                   else torch.empty(num_groups, dtype=values.dtype, device=values.device))
        if ready is None:
            ready = torch.cuda.Event()
            ready.record(torch.cuda.current_stream(values.device))
        rid = ctypes.c_uint64()
        _check(lib().repro_server_submit(self._h, keys.data_ptr(), values.data_ptr(), keys.numel(),
                                         _dtype_code(values.dtype), L, num_groups, out.data_ptr(),
                                         ctypes.c_void_p(ready.cuda_event), int(arrival_ns), ctypes.byref(rid)),
               "repro_server_submit")
        r = Request(rid.value, out, keys.numel(), num_groups, (keys, values, ready))
        self._reqs[r.id] = r
        return r

    def wait(self, req: Request, timeout_s: float = 600.0) -> Request:
        info = RequestInfo()
        _check(lib().repro_server_wait(self._h, req.id, timeout_s, ctypes.byref(info)), "repro_server_wait")
        req.info = info
        if info.status != 0:
            raise ReproError(info.status, f"request {req.id}")
        return req

    def poll(self, req: Request) -> bool:
        info = RequestInfo()
        _check(lib().repro_server_poll(self._h, req.id, ctypes.byref(info)), "repro_server_poll")
        req.info = info
        return bool(info.done)

    def release(self, req: Request):
        _check(lib().repro_server_release(self._h, req.id), "repro_server_release")
        self._reqs.pop(req.id, None)
        req._keep = ()

    def stats(self) -> dict:
        st = ServerStats()
        _check(lib().repro_server_stats_get(self._h, ctypes.byref(st)), "repro_server_stats_get")
        return {name: getattr(st, name) for name, _ in ServerStats._fields_}

    def close(self):
        if self._h:
            st = lib().repro_server_destroy(self._h)
            self._h = None
            self._reqs.clear()
            _check(st, "repro_server_destroy")

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def run_trace(server: Server, queries: Sequence[tuple], arrivals_s: Sequence[float], L: int = 3,
              keep_results: bool = False, timeout_s: float = 600.0) -> dict:
    """Submit `queries` ((keys, values, num_groups) on the device) with arrival
    times `arrivals_s` (seconds after the start), wait for all, and return
    per-request latency (arrival -> result in host memory) and the rows/s.
    Outputs are allocated and every query submitted before the first arrival
    (the start is put far enough ahead), so the client adds no delay."""
    outs = [torch.empty(q[2], dtype=q[1].dtype, pin_memory=True) for q in queries]
    ready = torch.cuda.Event()
    ready.record(torch.cuda.current_stream(server.device))
    t0 = now_ns() + 5_000_000 + 40_000 * len(queries)
    reqs: List[Request] = []
    for (k, v, G), a, o in zip(queries, arrivals_s, outs):
        reqs.append(server.submit(k, v, G, L, out=o, arrival_ns=t0 + int(a * 1e9), ready=ready))
    late = max(0, now_ns() - t0)
    lat, first, last = [], None, 0
    results = []
    for r in reqs:
        server.wait(r, timeout_s)
        lat.append(r.latency_s)
        first = r.info.arrival_ns if first is None else min(first, r.info.arrival_ns)
        last = max(last, r.info.done_ns)
        if keep_results:
            results.append(r.out)
        server.release(r)
    lat = np.asarray(lat)
    rows = sum(int(q[0].numel()) for q in queries)
    span = (last - first) * 1e-9
    return {"requests": len(reqs), "rows": rows, "span_s": span, "rows_per_s": rows / span if span > 0 else 0.0,
            "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "mean_ms": float(lat.mean() * 1e3), "max_ms": float(lat.max() * 1e3),
            "submit_overrun_ms": late * 1e-6, "results": results if keep_results else None}

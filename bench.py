#!/usr/bin/env python3
"""Benchmark of the reproducible grouped SUM on GB300.

One step = one reproducible SUM ... GROUP BY over one batch of synthetic rows
resident in HBM: state reset, every row through the library's kernels
(window, digit extraction, exact accumulation, merge) and the finalize to
float64 per group.  Prints ONE JSON line (rank 0).

    python bench.py                      # N = 1, default cell
    python bench.py --G 65536 --dist zipf --L 4
    python bench.py --impl reference     # the CPU oracle on the host cores
    torchrun --nproc-per-node N bench.py --gpus N   # N independent shards

Timing: W warm-up steps, then K steps between CUDA events on the launching
stream with a barrier + synchronize on both sides; max over ranks.  Inputs
(12 bytes x 2^28 rows = 3.2 GB) are far larger than L2, so no flush is
needed between steps.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import statistics
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "repro GroupBy-SUM rows/s and HBM GB/s vs non-repro FP64 GroupBy, 1 GB300, bit-exact"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=1 << 28)
    ap.add_argument("--G", type=int, default=1 << 10)
    ap.add_argument("--dist", default="uniform", choices=["uniform", "zipf"])
    ap.add_argument("--L", type=int, default=3)
    ap.add_argument("--key-span", type=int, default=0,
                    help="draw the keys over [0, span) while the state declares --G groups (0: span = G)")
    ap.add_argument("--adaptive", action="store_true",
                    help="aggregate through repro_groupby_sum_adaptive (depth from the keys' range)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--oracle-threads", type=int, default=0,
                    help="host threads of the CPU oracle (reference arm, cpu_baseline); 0: all cores")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="skip the untimed autotuning before the warm-up")
    ap.add_argument("--tune-file", default="",
                    help="sweep cells: load the tuned choices from this file if it exists, else tune and save them")
    ap.add_argument("--no-verify", action="store_true",
                    help="skip the (untimed) check of the step's state and results against the CPU oracle")
    ap.add_argument("--workload", default="sweep", choices=["sweep", "multicol", "batched", "serve", "scalar", "stats"],
                    help="sweep: one grouped SUM (default); multicol: 4 SUM columns over two uint8 keys; "
                         "batched: many aggregations in one launch; serve: the request server; "
                         "scalar: SUM without GROUP BY; stats: COUNT/SUM/AVG/VAR/STDDEV per group")
    ap.add_argument("--dtype", default="f64", choices=["f64", "f32"], help="multicol value type")
    ap.add_argument("--rows", type=int, default=0, help="multicol rows / serve table rows (0: default)")
    ap.add_argument("--tasks", type=int, default=4096, help="batched: number of aggregations")
    ap.add_argument("--requests", type=int, default=2000, help="serve: queries per trace")
    return ap.parse_args()


# ------------------------------------------------------------------- clocks

class ClockSampler:
    """Samples SM clock and clock-event reasons through NVML (ctypes) in a
    thread while running; falls back to nvidia-smi if NVML is unavailable."""

    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown", 0x2: "applications_clocks_setting",
               0x1: "gpu_idle"}

    def __init__(self, torch_device_index: int):
        self.samples = []
        self.max_mhz = None
        self._stop = threading.Event()
        self._thr = None
        self.nvml = None
        self.handle = None
        try:
            nv = ctypes.CDLL("libnvidia-ml.so.1")
            if nv.nvmlInit_v2() != 0:
                raise OSError("nvmlInit failed")
            import torch
            h = ctypes.c_void_p()
            uuid = str(torch.cuda.get_device_properties(torch_device_index).uuid)
            ok = False
            for cand in (uuid, "GPU-" + uuid):
                if nv.nvmlDeviceGetHandleByUUID(cand.encode(), ctypes.byref(h)) == 0:
                    ok = True
                    break
            if not ok:
                cnt = ctypes.c_uint(0)
                nv.nvmlDeviceGetCount_v2(ctypes.byref(cnt))
                if cnt.value != 1 or nv.nvmlDeviceGetHandleByIndex_v2(0, ctypes.byref(h)) != 0:
                    raise OSError("no NVML handle")
            self.nvml, self.handle = nv, h
            mx = ctypes.c_uint(0)
            if nv.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx)) == 0:  # NVML_CLOCK_SM
                self.max_mhz = mx.value
        except Exception:
            self.nvml = None

    def _run(self):
        nv, h = self.nvml, self.handle
        clk = ctypes.c_uint(0)
        rs = ctypes.c_ulonglong(0)
        while not self._stop.is_set():
            if nv.nvmlDeviceGetClockInfo(h, 1, ctypes.byref(clk)) == 0:
                nv.nvmlDeviceGetCurrentClocksEventReasons(h, ctypes.byref(rs))
                self.samples.append((clk.value, rs.value))
            time.sleep(0.002)

    def start(self):
        if self.nvml is not None:
            self._thr = threading.Thread(target=self._run, daemon=True)
            self._thr.start()

    def stop(self):
        if self._thr is not None:
            self._stop.set()
            self._thr.join()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": self.max_mhz, "reasons": ["unsampled"], "samples": 0}
        reasons = set()
        for _, r in self.samples:
            for bit, name in self.REASONS.items():
                if r & bit:
                    reasons.add(name)
        return {"sm_mhz": statistics.median(c for c, _ in self.samples), "sm_max_mhz": self.max_mhz,
                "reasons": sorted(reasons), "samples": len(self.samples)}


# --------------------------------------------------------------- our path

def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch

    import paper_1802_09883_gb300 as R
    from paper_1802_09883_gb300 import workloads as WL

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    lib = R.lib()

    # weak scaling: every rank aggregates its own shard of the same shape
    span = args.key_span if args.key_span > 0 else args.G
    w = WL.sweep_cell(span, args.dist, args.L, n=args.n, device=dev,
                      seed=None if rank == 0 else 1000 + rank)
    w.G = args.G  # the declared group count (keys reach [0, span))
    G, L, n = w.G, w.L, w.n
    depth = None
    st = R.State(G, L, torch.float64, device=dev)
    out = torch.empty(G, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)

    tuned = None
    if args.tune_file and os.path.exists(args.tune_file):  # an earlier run's measured choices
        R.tune_load(args.tune_file)
        tuned = {"loaded_from": args.tune_file}
    elif not args.no_tune:  # untimed: measured configuration choice for this workload
        tuned = R.tune(w.keys, w.values, G, L)
        if args.tune_file:
            R.tune_save(args.tune_file)

    def step():
        nonlocal depth
        st.reset()
        if args.adaptive:
            depth = st.add_adaptive(w.keys, w.values)
        else:
            st.add(w.keys, w.values)
        st.finalize(out)

    def barrier():
        if dist is not None:
            dist.barrier()

    for _ in range(max(args.warmup, 3)):
        step()
    st.check()
    torch.cuda.synchronize()

    clocks = ClockSampler(local_rank)
    lib.repro_profile_enable(1)
    for name in ("accum", "window", "fused", "partition", "merge", "finalize"):
        lib.repro_profile_read(name.encode(), None, None)
    launches0 = lib.repro_launch_count()
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks.stop()
    launches = lib.repro_launch_count() - launches0
    ms = e0.elapsed_time(e1) / args.steps
    st.check()  # a data or time-out error in a timed step fails the run
    # the last timed step's state and results, kept for the checks below
    dev_state = st.tensor.cpu().numpy().copy()
    dev_out = out.cpu().numpy().copy()
    prof = {}
    for name in ("accum", "window", "fused", "partition", "merge", "finalize"):
        t = ctypes.c_double(0)
        c = ctypes.c_int64(0)
        lib.repro_profile_read(name.encode(), ctypes.byref(t), ctypes.byref(c))
        if c.value:
            prof[name] = {"ms_per_launch": t.value / c.value, "launches": c.value}
    lib.repro_profile_enable(0)
    if dist is not None:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())

    # conventional FP64 GroupBy on the same rows: every table strategy that
    # fits is timed and the fastest is the baseline (the strong version)
    fp_modes = time_fp_modes(R, w.keys, w.values, G, args.steps, stream)
    fp_best = min(fp_modes, key=lambda m: fp_modes[m])
    fp_ms = fp_modes[fp_best]

    # end to end through the public API from pinned host buffers
    e2e = None
    if not args.no_e2e:
        keys_h = torch.empty(n, dtype=torch.int32, pin_memory=True)
        vals_h = torch.empty(n, dtype=torch.float64, pin_memory=True)
        keys_h.copy_(w.keys)
        vals_h.copy_(w.values)
        out_h = torch.empty(G, dtype=torch.float64, pin_memory=True)

        def e2e_step():  # host columns in, result to host: copies overlapped with the aggregation
            st.reset()
            st.add_host(keys_h, vals_h)
            st.finalize(out)
            out_h.copy_(out, non_blocking=True)

        for _ in range(2):
            e2e_step()
        torch.cuda.synchronize()
        barrier()
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        for _ in range(args.steps):
            e2e_step()
        g1.record(stream)
        torch.cuda.synchronize()
        barrier()
        e2e_ms = g0.elapsed_time(g1) / args.steps
        if dist is not None:
            t = torch.tensor([e2e_ms], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e2e_ms = float(t.item())
        # the e2e result must be the device-resident path's, bit for bit
        assert np.array_equal(out_h.numpy().view(np.int64), dev_out.view(np.int64))
        e2e = {"value": n * world / (e2e_ms / 1e3), "unit": "rows/s", "h2d_bytes_per_step": n * (4 + 8),
               "d2h_bytes_per_step": G * 8, "ms_per_step": e2e_ms}
        del keys_h, vals_h

    verify = None
    if not args.no_verify and rank == 0:  # untimed: the timed step's state and results against the oracle
        verify = verify_step(w, dev_state, dev_out, args.oracle_threads)

    result = None
    if rank == 0:
        algo_bytes = n * (4 + 8) + G * 8
        peaks = load_peaks()
        dom = max(prof.items(), key=lambda kv: kv[1]["ms_per_launch"] * kv[1]["launches"]) if prof else None
        roof = None
        if dom is not None:
            name, p = dom
            # algorithmic bytes of one launch of the dominant row-pass kernel:
            # every row's key and value read once
            dom_bytes = n * (4 + 8)
            ach = dom_bytes / (p["ms_per_launch"] / 1e3) / 1e9
            cfg_key = None
            if tuned and tuned.get("path") == "single_pass":
                cfg_key = "%d,%d,%d,%d,%d" % (tuned["stages"], tuned["tile_rows"], tuned["consumer_warps"],
                                              tuned["ctas_per_sm"], tuned["table_copies"])
            wkey = "n=%d G=%d %s L=%d" % (n, G, args.dist, L)
            roof = {"bound": "hbm", "kernel": name, "achieved": round(ach, 1), "peak": peaks["hbm_gbs"],
                    "unit": "GB/s", "frac": round(ach / peaks["hbm_gbs"], 4),
                    "traffic": measured_traffic("k_fused" if name == "fused" else name, wkey, cfg_key),
                    "traffic_source": "profiles/traffic.json (ncu dram__bytes_read.sum + dram__bytes_write.sum, "
                                      "same sources, workload and configuration; null otherwise)",
                    "peak_source": peaks["source"], "ms_per_launch": p["ms_per_launch"],
                    "launches_per_step": p["launches"] / args.steps}
        result = {
            "metric": METRIC,
            "value": n * world / (ms / 1e3),
            "unit": "rows/s",
            "n_gpus": world,
            "steps": args.steps,
            "warmup": max(args.warmup, 3),
            "ms_per_step": ms,
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"grouped SUM, {n} rows, {G} groups {args.dist}, repro<double,{L}>, "
                                   f"exponents U[-40,40], 10% cancelling pairs"
                                   + (f", keys over [0, {span})" if span != G else "")
                                   + (", adaptive depth" if args.adaptive else ""),
                       "n": n, "G": G, "key_span": span, "adaptive_depth": depth,
                       "dist": args.dist, "L": L, "parallelism": f"shards{world}",
                       "l2": "inputs (12 B/row) far larger than L2; no flush"},
            "hbm_gbs_algorithmic": algo_bytes / (ms / 1e3) / 1e9,
            "roofline": roof,
            "kernels": prof,
            "fp64_baseline": {"ms_per_step": fp_ms, "rows_per_s": n / (fp_ms / 1e3),
                              "repro_over_fp64_time": ms / fp_ms, "strategy": R.FP_MODES[fp_best],
                              "ms_by_strategy": {R.FP_MODES[m]: round(t, 4) for m, t in fp_modes.items()},
                              "hbm_frac": round(n * 12 / (fp_ms / 1e3) / 1e9 / load_peaks()["hbm_gbs"], 4)},
            "e2e": e2e,
            "gpu_launches": int(launches),
            "clocks": clocks.summary(),
            "tuned": tuned,
        }
        if verify is not None:
            result["verify"] = verify
            result["bit_exact"] = verify["bit_exact"]
    if dist is not None:
        dist.destroy_process_group()
    return result


def time_fp_modes(R, keys, values, G, steps, stream):
    """ms per call of the conventional GroupBy for every table strategy that
    fits G (3 untimed warm-ups each; CUDA events on the launching stream)."""
    import torch
    out = torch.empty(G, dtype=values.dtype, device=values.device)
    res = {}
    for mode in sorted(R.FP_MODES):
        if R.groupby_sum_fp_mode(keys, values, G, mode, out=out) is None:
            continue
        for _ in range(2):
            R.groupby_sum_fp_mode(keys, values, G, mode, out=out)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(steps):
            R.groupby_sum_fp_mode(keys, values, G, mode, out=out)
        b.record(stream)
        torch.cuda.synchronize()
        res[mode] = a.elapsed_time(b) / steps
    return res


def verify_state(keys_np, vals_np, G, L, state_bytes, got, threads=0):
    """One state and its results against the C oracle on the same rows, bit
    for bit: every group's K, flags and 128-bit bins and every result."""
    import numpy as np

    import paper_1802_09883_gb300 as R
    from oracle import oracle as O

    nth = threads if threads and threads > 0 else (os.cpu_count() or 1)
    ref = O.init(vals_np.dtype.type, L, G)
    bad = O.groupby_sum(ref, keys_np, vals_np, threads=nth)
    K, fl, lo, hi = R.parse_state(state_bytes, L, G)
    oK, ofl, olo, ohi = O.to_bins(ref)
    iv = np.int64 if vals_np.dtype == np.float64 else np.int32
    state_ok = bool(np.array_equal(K, oK) and np.array_equal(fl, ofl) and np.array_equal(lo, olo)
                    and np.array_equal(hi, ohi))
    res_ok = bool(np.array_equal(np.asarray(got).view(iv), O.finalize(ref).view(iv)))
    return state_ok and res_ok and bad == 0


def verify_step(w, state_bytes, got, threads=0):
    """The last timed step's state and results against the CPU oracle.

    Up to 2^20 groups the whole state is compared -- every group's K, flags
    and 128-bit bins and every result, bit for bit -- with the C oracle run
    on all rows (threads over row chunks, exact merge).  Beyond, the oracle's
    per-thread tables would not fit comfortably, so the rows of a random
    sample of 512 groups are gathered and those groups' results compared."""
    import numpy as np
    import torch

    import paper_1802_09883_gb300 as R
    from oracle import oracle as O

    G, L = w.G, w.L
    nth = threads if threads and threads > 0 else (os.cpu_count() or 1)
    t0 = time.perf_counter()
    if G <= (1 << 20):
        kh, vh = w.keys.cpu().numpy(), w.values.cpu().numpy()
        ref = O.init(np.float64, L, G)
        bad = O.groupby_sum(ref, kh, vh, threads=nth)
        K, fl, lo, hi = R.parse_state(state_bytes, L, G)
        oK, ofl, olo, ohi = O.to_bins(ref)
        state_ok = bool(np.array_equal(K, oK) and np.array_equal(fl, ofl) and np.array_equal(lo, olo)
                        and np.array_equal(hi, ohi))
        res_ok = bool(np.array_equal(got.view(np.int64), O.finalize(ref).view(np.int64)))
        return {"mode": "full state", "groups": G, "rows": int(kh.size), "bad_keys": int(bad),
                "state_equal": state_ok, "results_equal": res_ok, "bit_exact": state_ok and res_ok and bad == 0,
                "oracle": f"C oracle, {nth} host threads", "seconds": round(time.perf_counter() - t0, 2)}
    gen = torch.Generator(device="cpu")
    gen.manual_seed(17)
    ngroups = min(G, 512)
    sample = torch.randperm(G, generator=gen)[:ngroups].to(w.keys.device)
    remap = torch.full((G,), -1, dtype=torch.int32, device=w.keys.device)
    remap[sample] = torch.arange(ngroups, dtype=torch.int32, device=w.keys.device)
    sel = remap[w.keys.long()]
    mask = sel >= 0
    k = sel[mask].cpu().numpy()
    v = w.values[mask].cpu().numpy()
    ref = O.groupby_sum_values(k, v, ngroups, L, threads=nth)
    mine = got[sample.cpu().numpy()]
    ok = bool(np.array_equal(mine.view(np.int64), ref.view(np.int64)))
    return {"mode": "sampled groups", "groups": ngroups, "rows": int(k.size), "results_equal": ok, "bit_exact": ok,
            "oracle": f"C oracle, {nth} host threads", "seconds": round(time.perf_counter() - t0, 2)}


# the sources each profiled kernel is compiled from
KERNEL_SOURCES = {"k_fused": ["repro_fused.cu", "fused_device.cuh", "repro_device.cuh", "ptx.cuh"]}


def kernel_source_hash(kernel):
    """sha256 over the sources a kernel is compiled from: a DRAM traffic
    figure is reported only for the kernel it was measured on."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1802_09883_gb300", "csrc")
    for name in KERNEL_SOURCES.get(kernel, []):
        h.update(name.encode())
        with open(os.path.join(csrc, name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def measured_traffic(kernel, workload_key, cfg_key):
    """DRAM bytes per launch from profiles/traffic.json when that capture was
    taken on these sources, this workload and this kernel configuration."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
            entries = json.load(fh)
    except Exception:
        return None
    if kernel not in KERNEL_SOURCES:
        return None
    src = kernel_source_hash(kernel)
    for e in entries:
        if (e.get("kernel") == kernel and e.get("workload") == workload_key and e.get("config") == cfg_key
                and e.get("source_sha256") == src):
            return e.get("dram_bytes_per_launch")
    return None


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as fh:
            d = json.load(fh)
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured (MEASURED_PEAKS.json burst copy)"}
    except Exception:
        return {"hbm_gbs": 6800.0, "source": "fallback 6.8 TB/s"}


# ------------------------------------------------------- secondary workloads

PROF_NAMES = ("accum", "window", "fused", "partition", "merge", "finalize")


def _prof_start(lib):
    lib.repro_profile_enable(1)
    for name in PROF_NAMES:
        lib.repro_profile_read(name.encode(), None, None)


def _prof_stop(lib):
    prof = {}
    for name in PROF_NAMES:
        t = ctypes.c_double(0)
        c = ctypes.c_int64(0)
        lib.repro_profile_read(name.encode(), ctypes.byref(t), ctypes.byref(c))
        if c.value:
            prof[name] = {"ms_per_launch": t.value / c.value, "launches": c.value, "ms_total": t.value}
    lib.repro_profile_enable(0)
    return prof


def _time(fn, steps, stream):
    import torch

    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def _base_line(args, metric, value, unit, ms, dtype, workload, extra_cfg):
    return {"metric": metric, "value": value, "unit": unit, "n_gpus": 1, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": dtype, "data": "synthetic",
            "config": dict({"workload": workload}, **extra_cfg)}


def run_multicol(args, local_rank):
    """Few-group multi-column aggregate: SUM of 4 columns GROUP BY two uint8
    keys (4 groups), repro<T,3>; one step = reset, aggregate, finalize."""
    import torch

    import paper_1802_09883_gb300 as R
    from paper_1802_09883_gb300 import workloads as WL

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    lib = R.lib()
    n = args.rows or 60_000_000
    dt = torch.float64 if args.dtype == "f64" else torch.float32
    esz = 8 if dt == torch.float64 else 4
    k1, k2, cols = WL.few_groups_multicol(n=n, seed=2, device=dev)
    cols = cols.to(dt).contiguous()
    colsl = list(cols)
    G, L = 4, 3
    states = [R.State(G, L, dt, device=dev) for _ in colsl]
    outs = [torch.empty(G, dtype=dt, device=dev) for _ in colsl]
    stream = torch.cuda.current_stream(dev)
    # group ids as the per-column path forms them (baselines and tuning, untimed)
    gid = (k1.to(torch.int32) * 2 + k2.to(torch.int32)).contiguous()
    tuned = None
    if not args.no_tune:  # the per-column passes use the choice for 4 groups
        tuned = R.tune(gid, colsl[0], G, L)

    def step():
        for st in states:
            st.reset()
        R.groupby_sum_cols(k1, k2, 2, colsl, G, L, states=states)
        for st, o in zip(states, outs):
            st.finalize(o)

    for _ in range(max(args.warmup, 3)):
        step()
    for st in states:
        st.check()
    clocks = ClockSampler(local_rank)
    _prof_start(lib)
    l0 = lib.repro_launch_count()
    clocks.start()
    ms = _time(step, args.steps, stream)
    clocks.stop()
    launches = lib.repro_launch_count() - l0
    prof = _prof_stop(lib)
    for st in states:
        st.check()
    verify = None
    if not args.no_verify:  # untimed: every column's state and results against the oracle
        t0 = time.perf_counter()
        torch.cuda.synchronize()
        gh = gid.cpu().numpy()
        oks = [verify_state(gh, c.cpu().numpy(), G, L, st.tensor.cpu().numpy(), o.cpu().numpy(),
                            args.oracle_threads) for c, st, o in zip(colsl, states, outs)]
        verify = {"mode": "full state, every column", "groups": G, "rows": n, "columns": len(oks),
                  "bit_exact": all(oks), "oracle": "C oracle", "seconds": round(time.perf_counter() - t0, 2)}
    # conventional GroupBy on the same rows (group ids precomputed, untimed)
    fp_outs = [torch.empty(G, dtype=dt, device=dev) for _ in colsl]
    fp = R.groupby_sum_fp64 if dt == torch.float64 else R.groupby_sum_fp32

    def fp_step():
        for c, o in zip(colsl, fp_outs):
            fp(gid, c, G, out=o)

    fp_step()
    fp_ms = _time(fp_step, args.steps, stream)
    # DECIMAL baseline: the same four columns as exact scaled integers (p, d
    # in hundredths; p * (1 - d), p * d in ten-thousandths), int64 sums per group
    dec = [torch.round(cols[0].double() * 100).long(), torch.round(cols[1].double() * 100).long(),
           torch.round(cols[2].double() * 10000).long(), torch.round(cols[3].double() * 10000).long()]
    dec_out = [torch.empty(G, dtype=torch.int64, device=dev) for _ in dec]

    def dec_step():
        for c, o in zip(dec, dec_out):
            R.groupby_sum_decimal64(gid, c, G, out=o)

    dec_step()
    dec_ms = _time(dec_step, args.steps, stream)
    del dec
    # end to end from pinned host buffers
    k1h, k2h = k1.cpu().pin_memory(), k2.cpu().pin_memory()
    colsh = cols.cpu().pin_memory()
    outs_h = torch.empty((len(colsl), G), dtype=dt, pin_memory=True)
    k1d, k2d, colsd = torch.empty_like(k1), torch.empty_like(k2), torch.empty_like(cols)
    colsdl = list(colsd)

    def e2e_step():
        k1d.copy_(k1h, non_blocking=True)
        k2d.copy_(k2h, non_blocking=True)
        colsd.copy_(colsh, non_blocking=True)
        for st in states:
            st.reset()
        R.groupby_sum_cols(k1d, k2d, 2, colsdl, G, L, states=states)
        for i, (st, o) in enumerate(zip(states, outs)):
            st.finalize(o)
            outs_h[i].copy_(o, non_blocking=True)

    e2e_step()
    e2e_ms = _time(e2e_step, args.steps, stream)
    for o, oh in zip(outs, outs_h):
        assert torch.equal(o.cpu(), oh)
    peaks = load_peaks()
    fused = prof.get("fused")
    roof = None
    if fused:
        per_launch = n * (4 + esz)  # the fused pass reads one group id and one value per row
        ach = per_launch / (fused["ms_per_launch"] / 1e3) / 1e9
        roof = {"bound": "hbm", "kernel": "fused", "achieved": round(ach, 1), "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "frac": round(ach / peaks["hbm_gbs"], 4), "traffic": None,
                "peak_source": peaks["source"], "ms_per_launch": fused["ms_per_launch"],
                "launches_per_step": fused["launches"] / args.steps}
    algo = n * (2 + 4 * esz) + 4 * G * esz
    res = _base_line(args, "repro multi-column GroupBy-SUM rows/s (4 SUM columns, 4 groups)", n / (ms / 1e3),
                     "rows/s", ms, args.dtype,
                     f"few-group multi-column aggregate, {n} rows, 2 uint8 keys -> 4 groups, 4 SUM columns, "
                     f"repro<{'double' if esz == 8 else 'float'},3>",
                     {"n": n, "G": G, "L": L, "columns": 4, "l2": "inputs far larger than L2; no flush"})
    res.update({"hbm_gbs_algorithmic": algo / (ms / 1e3) / 1e9, "roofline": roof, "kernels": prof,
                "fp64_baseline": {"kind": "fp64" if esz == 8 else "fp32", "ms_per_step": fp_ms,
                                  "repro_over_fp_time": ms / fp_ms},
                "decimal_baseline": {"kind": "4 x groupby_sum_decimal64 (exact int64, scaled columns)",
                                     "ms_per_step": dec_ms, "repro_over_decimal_time": ms / dec_ms},
                "e2e": {"value": n / (e2e_ms / 1e3), "unit": "rows/s", "h2d_bytes_per_step": n * (2 + 4 * esz),
                        "d2h_bytes_per_step": 4 * G * esz, "ms_per_step": e2e_ms},
                "gpu_launches": int(launches), "clocks": clocks.summary(), "tuned": tuned})
    if verify is not None:
        res["verify"] = verify
        res["bit_exact"] = verify["bit_exact"]
    return res


def run_batched(args, local_rank):
    """Many independent aggregations in one persistent launch, replayed from
    a CUDA graph: one step = reset all states, aggregate, finalize all."""
    import torch

    import paper_1802_09883_gb300 as R
    from paper_1802_09883_gb300 import workloads as WL

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    lib = R.lib()
    L = 3
    t_gen = time.time()
    tasks = WL.batched_tasks(args.tasks, seed=3, device=dev)
    torch.cuda.synchronize()
    t_gen = time.time() - t_gen
    rows = sum(int(k.numel()) for k, _, _ in tasks)
    groups = sum(G for _, _, G in tasks)
    states = [R.State(G, L, torch.float64, device=dev) for _, _, G in tasks]
    outs = [torch.empty(G, dtype=torch.float64, device=dev) for _, _, G in tasks]
    t_plan = time.time()
    plan = R.BatchPlan([(k, v, st) for (k, v, _), st in zip(tasks, states)])
    plan.set_outputs(outs)
    t_plan = time.time() - t_plan
    tune_ms = None if args.no_tune else plan.tune()  # untimed: item size for this batch
    plan_info = plan.describe()
    side = torch.cuda.Stream(dev)
    side.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.stream(side):
        l0 = lib.repro_launch_count()
        plan.reset().run().finalize()  # eager warm-up; counts the launches of one step
        torch.cuda.synchronize()
        per_step_launches = lib.repro_launch_count() - l0
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=side):
            plan.reset().run().finalize()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream(dev)
    for _ in range(max(args.warmup, 3)):
        graph.replay()
    torch.cuda.synchronize()
    clocks = ClockSampler(local_rank)
    clocks.start()
    ms = _time(graph.replay, args.steps, stream)
    clocks.stop()
    # bit-equality of a sample of tasks against the one-task path
    sample = list(range(0, len(tasks), max(1, len(tasks) // 16)))
    same = all(torch.equal(outs[i].view(torch.int64),
                           R.groupby_sum(tasks[i][0], tasks[i][1], tasks[i][2], L).view(torch.int64))
               for i in sample)
    # per-kernel times from one eager step with the profiler on
    with torch.cuda.stream(side):
        _prof_start(lib)
        plan.reset().run().finalize()
        torch.cuda.synchronize()
        prof = _prof_stop(lib)
    # conventional FP64 GroupBy over the same tasks, one call each
    fp_outs = [torch.empty(G, dtype=torch.float64, device=dev) for _, _, G in tasks]

    def fp_step():
        for (k, v, G), o in zip(tasks, fp_outs):
            R.groupby_sum_fp64(k, v, G, out=o)

    fp_step()
    fp_ms = _time(fp_step, max(1, args.steps // 4), stream)
    peaks = load_peaks()
    algo = rows * 12 + groups * 8
    ach = algo / (ms / 1e3) / 1e9
    res = _base_line(args, "repro batched GroupBy-SUM rows/s (independent aggregations, one graph replay)",
                     rows / (ms / 1e3), "rows/s", ms, "f64",
                     f"batched: {len(tasks)} aggregations, rows log-uniform 1e3-1e7, groups log-uniform 1-1e5, "
                     f"repro<double,3>, values as the plain config", 
                     {"tasks": len(tasks), "rows": rows, "groups": groups, "L": L,
                      "l2": f"inputs {rows * 12 / 1e9:.1f} GB, far larger than L2; no flush"})
    res.update({"hbm_gbs_algorithmic": ach,
                "roofline": {"bound": "hbm", "kernel": "whole step (graph replay)", "achieved": round(ach, 1),
                             "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": round(ach / peaks["hbm_gbs"], 4),
                             "traffic": None, "peak_source": peaks["source"]},
                "kernels": prof, "fp64_baseline": {"ms_per_step": fp_ms, "repro_over_fp64_time": ms / fp_ms,
                                                   "kind": "one groupby_sum_fp64 call per task"},
                "e2e": None, "e2e_note": "inputs of this workload are generated on the device (tens of GB)",
                "gpu_launches": int(per_step_launches * args.steps), "clocks": clocks.summary(),
                "verify": {"tasks_checked": len(sample), "bit_equal_to_single_task": bool(same)},
                "plan": dict(plan_info, prepare_s=t_plan, generate_s=t_gen, tuned_run_ms=tune_ms)})
    plan.close()
    return res


def run_serve(args, local_rank):
    """Request server under Poisson arrivals: capacity from a closed-loop
    trace, then latency at 0.5 / 0.7 / 0.9 of that rate."""
    import numpy as np
    import torch

    import paper_1802_09883_gb300 as R
    from paper_1802_09883_gb300 import serve as S
    from paper_1802_09883_gb300 import workloads as WL

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    lib = R.lib()
    max_rows = args.rows or 100_000_000
    table = WL.serving_table(max_rows, groups=(1, 1e6), levels=25, seed=4, device=dev)
    trace, gaps = WL.serving_trace(args.requests, table, rows=(1e4, 1e8), seed=4)
    queries = [table.query(*q) for q in trace]
    rows = sum(int(q[0].numel()) for q in queries)
    torch.cuda.synchronize()
    clocks = ClockSampler(local_rank)
    with S.Server(chunk_rows=1 << 24, max_active=256) as srv:
        S.run_trace(srv, queries[:64], [0.0] * 64)  # warm-up
        l0 = lib.repro_launch_count()
        clocks.start()
        closed = S.run_trace(srv, queries, [0.0] * len(queries))
        rate = len(queries) / closed["span_s"]
        open_runs = {}
        for frac in (0.5, 0.7, 0.9):
            arr = np.cumsum(gaps) / (frac * rate)
            r = S.run_trace(srv, queries, arr)
            open_runs[str(frac)] = {k: r[k] for k in ("p50_ms", "p99_ms", "mean_ms", "max_ms", "rows_per_s",
                                                       "span_s")}
        clocks.stop()
        launches = lib.repro_launch_count() - l0
        stats = srv.stats()
        # a sample of results in the mix vs each query alone
        sample = list(range(0, len(queries), max(1, len(queries) // 12)))
        mix = S.run_trace(srv, [queries[i] for i in sample], [0.0] * len(sample), keep_results=True)
    same = all(torch.equal(o.view(torch.int64), R.groupby_sum(*queries[i]).cpu().view(torch.int64))
               for i, o in zip(sample, mix["results"]))
    res = _base_line(args, "repro serving rows/s (closed loop) with p50/p99 latency under Poisson arrivals",
                     closed["rows_per_s"], "rows/s", closed["span_s"] * 1e3, "f64",
                     f"serving: {len(queries)} queries, rows log-uniform 1e4-1e8, groups log-uniform 1-1e6 "
                     f"(25 levels), repro<double,3>, results to pinned host memory",
                     {"requests": len(queries), "rows": rows, "table_rows": max_rows, "L": 3,
                      "chunk_rows": 1 << 24, "l2": "queries scan a 10 GB resident table; no flush"})
    res.update({"serving": {"capacity_requests_per_s": rate, "closed_loop": {k: closed[k] for k in (
                    "p50_ms", "p99_ms", "mean_ms", "rows_per_s", "span_s")}, "poisson": open_runs,
                    "server": {k: stats[k] for k in ("iterations", "batch_launches", "large_calls",
                                                     "memory_peak", "memory_budget", "memory_server_peak")}},
                "verify": {"queries_checked": len(sample), "bit_equal_alone_and_in_mix": bool(same)},
                "e2e": {"value": closed["rows_per_s"], "unit": "rows/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": sum(q[2] for q in queries) * 8,
                        "note": "queries scan a device-resident table; each result is copied to host"},
                "gpu_launches": int(launches), "clocks": clocks.summary(), "roofline": None})
    return res


def run_scalar(args, local_rank):
    """Reproducible SUM without GROUP BY over 2^28 float64 values (the sweep's
    value recipe), against torch.sum in float64 on the same values."""
    import torch

    import paper_1802_09883_gb300 as R
    from paper_1802_09883_gb300 import workloads as WL

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    lib = R.lib()
    n = args.rows or (1 << 28)
    w = WL.sweep_cell(16, "uniform", args.L, n=n, device=dev)
    vals = w.values
    del w
    st = R.State(1, args.L, torch.float64, device=dev)
    out = torch.empty(1, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    tuned = None
    if not args.no_tune:  # untimed; the keyless kernel shares the one-group configuration
        zk = torch.zeros(n, dtype=torch.int32, device=dev)
        tuned = R.tune(zk, vals, 1, args.L)
        del zk

    def step():
        st.reset()
        st.add_values(vals)
        st.finalize(out)

    for _ in range(max(args.warmup, 3)):
        step()
    st.check()
    clocks = ClockSampler(local_rank)
    _prof_start(lib)
    l0 = lib.repro_launch_count()
    clocks.start()
    ms = _time(step, args.steps, stream)
    clocks.stop()
    launches = lib.repro_launch_count() - l0
    prof = _prof_stop(lib)
    ref = torch.empty((), dtype=torch.float64, device=dev)
    torch.sum(vals, dim=0, out=ref)
    base_ms = _time(lambda: torch.sum(vals, dim=0, out=ref), args.steps, stream)
    # the unbuffered drop-in type (one value at a time per thread) on the same values
    ub = R.State(1, args.L, torch.float64, device=dev)

    def ub_step():
        ub.reset()
        ub.add_values_unbuffered(vals)

    ub_step()
    ub_ms = _time(ub_step, max(1, args.steps // 2), stream)
    torch.cuda.synchronize()
    same = torch.equal(ub.tensor, st.tensor)
    st.check()
    verify = None
    if not args.no_verify:  # untimed: the state and result against the oracle on all values
        import numpy as np

        t0 = time.perf_counter()
        vh = vals.cpu().numpy()
        ok = verify_state(np.zeros(vh.size, np.int32), vh, 1, args.L, st.tensor.cpu().numpy(), out.cpu().numpy(),
                          args.oracle_threads)
        verify = {"mode": "full state", "groups": 1, "rows": n, "bit_exact": ok, "oracle": "C oracle",
                  "seconds": round(time.perf_counter() - t0, 2)}
    peaks = load_peaks()
    fused = prof.get("fused")
    roof = None
    if fused:
        ach = n * 8 / (fused["ms_per_launch"] / 1e3) / 1e9
        roof = {"bound": "hbm", "kernel": "fused (keyless)", "achieved": round(ach, 1), "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "frac": round(ach / peaks["hbm_gbs"], 4), "traffic": None,
                "peak_source": peaks["source"], "ms_per_launch": fused["ms_per_launch"]}
    res = _base_line(args, "repro SUM (no GROUP BY) values/s", n / (ms / 1e3), "values/s", ms, "f64",
                     f"scalar SUM of {n} float64 values (exponents U[-40,40], 10% cancelling pairs), "
                     f"repro<double,{args.L}>", {"n": n, "L": args.L, "l2": "inputs far larger than L2; no flush"})
    res.update({"hbm_gbs_algorithmic": n * 8 / (ms / 1e3) / 1e9, "roofline": roof, "kernels": prof,
                "fp64_baseline": {"kind": "torch.sum float64", "ms_per_step": base_ms,
                                  "repro_over_fp64_time": ms / base_ms},
                "unbuffered_dropin": {"ms_per_step": ub_ms, "over_buffered_time": ub_ms / ms,
                                      "over_fp64_time": ub_ms / base_ms, "same_state_bytes": bool(same)},
                "e2e": None, "gpu_launches": int(launches), "clocks": clocks.summary(), "tuned": tuned})
    if verify is not None:
        res["verify"] = verify
        res["bit_exact"] = verify["bit_exact"]
    return res


def run_stats(args, local_rank):
    """COUNT / SUM / AVG / VAR / STDDEV per group on the headline cell
    (2^28 rows, G = 1024), against two FP64 GroupBys (x and x*x)."""
    import torch

    import paper_1802_09883_gb300 as R
    from paper_1802_09883_gb300 import workloads as WL

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    lib = R.lib()
    w = WL.sweep_cell(args.G, args.dist, args.L, n=args.n, device=dev)
    n, G = w.n, w.G
    st = R.Stats(G, args.L, device=dev)
    stream = torch.cuda.current_stream(dev)
    outs = {}
    if not args.no_tune:  # untimed
        R.tune(w.keys, w.values, G, args.L)

    def step():
        nonlocal outs
        lib.repro_stats_init(st.tensor.data_ptr(), st.code, st.L, st.G, stream.cuda_stream)
        st.add(w.keys, w.values)
        outs = st.finalize()

    for _ in range(max(args.warmup, 3)):
        step()
    st.check()
    clocks = ClockSampler(local_rank)
    l0 = lib.repro_launch_count()
    clocks.start()
    ms = _time(step, args.steps, stream)
    clocks.stop()
    launches = lib.repro_launch_count() - l0
    sq = w.values * w.values
    fo1 = torch.empty(G, dtype=torch.float64, device=dev)
    fo2 = torch.empty(G, dtype=torch.float64, device=dev)

    def fp_step():
        R.groupby_sum_fp64(w.keys, w.values, G, out=fo1)
        R.groupby_sum_fp64(w.keys, sq, G, out=fo2)

    fp_step()
    fp_ms = _time(fp_step, args.steps, stream)
    res = _base_line(args, "repro COUNT/SUM/AVG/VAR/STDDEV GroupBy rows/s", n / (ms / 1e3), "rows/s", ms, "f64",
                     f"per-group statistics, {n} rows, {G} groups {args.dist}, repro<double,{args.L}> sums of x "
                     f"and x*x", {"n": n, "G": G, "dist": args.dist, "L": args.L,
                                  "l2": "inputs far larger than L2; no flush"})
    res.update({"hbm_gbs_algorithmic": n * 12 / (ms / 1e3) / 1e9, "roofline": None,
                "fp64_baseline": {"kind": "two groupby_sum_fp64 (x, x*x precomputed)", "ms_per_step": fp_ms,
                                  "repro_over_fp64_time": ms / fp_ms},
                "e2e": None, "gpu_launches": int(launches), "clocks": clocks.summary()})
    st.check()
    if not args.no_verify:  # untimed: every statistic of every group against the oracle, bit for bit
        import numpy as np

        from oracle import stats as OS

        t0 = time.perf_counter()
        torch.cuda.synchronize()
        nth = args.oracle_threads if args.oracle_threads > 0 else (os.cpu_count() or 1)
        ref = OS.groupby_stats(w.keys.cpu().numpy(), w.values.cpu().numpy(), G, args.L, threads=nth)
        ok = True
        for name, want in ref.items():
            got = outs[name].cpu().numpy()
            iv = np.int64 if got.dtype.itemsize == 8 else np.int32
            ok = ok and bool(np.array_equal(got.view(iv), np.asarray(want).astype(got.dtype).view(iv)))
        res["verify"] = {"mode": "every statistic of every group", "groups": G, "rows": n, "bit_exact": ok,
                         "oracle": f"C oracle ({nth} host threads) and oracle/stats.py",
                         "seconds": round(time.perf_counter() - t0, 2)}
        res["bit_exact"] = ok
    return res


# -------------------------------------------------------- CPU oracle timing

def cpu_oracle_rate(G, dist, L, rows, threads):
    """Rows/s of the C oracle (as it stands) on `rows` rows of the workload."""
    import numpy as np

    from oracle import oracle as O
    from paper_1802_09883_gb300 import workloads as WL

    w = WL.sweep_cell(G, dist, L, n=rows, device="cpu")
    k = w.keys.numpy()
    v = w.values.numpy()
    st = O.init(np.float64, L, G)
    t = time.perf_counter()
    O.groupby_sum(st, k, v, threads=threads)
    O.finalize(st)
    dt = time.perf_counter() - t
    return rows / dt, dt


def oracle_threads(args):
    return args.oracle_threads if args.oracle_threads > 0 else (os.cpu_count() or 1)


def cpu_baseline(args):
    threads = oracle_threads(args)
    rows = 1 << 22
    rate, dt = cpu_oracle_rate(args.G, args.dist, args.L, rows, threads)
    # grow the sample towards ~10 s of CPU work (threads x wall)
    target_wall = max(1.0, 10.0 / threads)
    if dt < target_wall:
        rows = int(min(args.n, rows * target_wall / max(dt, 1e-3)))
        rate, dt = cpu_oracle_rate(args.G, args.dist, args.L, rows, threads)
    return {"value": rate, "unit": "rows/s", "cores": threads, "kind": "oracle",
            "sample": f"{rows} rows drawn with the same recipe (G={args.G} {args.dist}, L={args.L}), "
                      f"C oracle with {threads} threads over row chunks + exact merge, {dt:.2f} s wall"}


def run_reference(args, rank):
    if rank != 0:
        return None
    threads = oracle_threads(args)
    from oracle import oracle as O

    O.build()
    rows = 1 << 22
    _, dt = cpu_oracle_rate(args.G, args.dist, args.L, rows, threads)
    # each step a bounded sample: about 2 s of wall time
    rows = int(min(args.n, max(1 << 20, rows * 2.0 / max(dt, 1e-3))))
    rates = []
    for i in range(max(args.warmup, 3) + args.steps):
        r, _ = cpu_oracle_rate(args.G, args.dist, args.L, rows, threads)
        if i >= max(args.warmup, 3):
            rates.append(r)
    value = statistics.median(rates)
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "rows/s", "n_gpus": 1,
        "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": rows / value * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"grouped SUM, {args.n} rows, {args.G} groups {args.dist}, repro<double,{args.L}>, "
                               f"exponents U[-40,40], 10% cancelling pairs",
                   "n": args.n, "G": args.G, "dist": args.dist, "L": args.L, "parallelism": "host threads"},
        "cpu_baseline": {"value": value, "unit": "rows/s", "cores": threads, "kind": "oracle",
                         "sample": f"{rows} rows per step drawn with the same recipe; C oracle, "
                                   f"{threads} threads over row chunks + exact merge"},
        "e2e": {"value": value, "unit": "rows/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        res = run_reference(args, rank)
        if res is not None:
            print(json.dumps(res), flush=True)
        return
    if args.workload != "sweep":
        if rank == 0:
            fn = {"multicol": run_multicol, "batched": run_batched, "serve": run_serve, "scalar": run_scalar,
                  "stats": run_stats}[args.workload]
            print(json.dumps(fn(args, local_rank)), flush=True)
        return
    res = run_ours(args, rank, world, local_rank)
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline:
            from oracle import oracle as O

            O.build()
            res["cpu_baseline"] = cpu_baseline(args)
        print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()

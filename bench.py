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
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--verify", action="store_true", help="check sampled groups against the oracle")
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
    w = WL.sweep_cell(args.G, args.dist, args.L, n=args.n, device=dev,
                      seed=None if rank == 0 else 1000 + rank)
    G, L, n = w.G, w.L, w.n
    st = R.State(G, L, torch.float64, device=dev)
    out = torch.empty(G, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        st.reset()
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

    # conventional FP64 GroupBy on the same rows
    fp_out = torch.empty(G, dtype=torch.float64, device=dev)
    for _ in range(3):
        R.groupby_sum_fp64(w.keys, w.values, G, out=fp_out)
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for _ in range(args.steps):
        R.groupby_sum_fp64(w.keys, w.values, G, out=fp_out)
    f1.record(stream)
    torch.cuda.synchronize()
    fp_ms = f0.elapsed_time(f1) / args.steps

    # end to end through the public API from pinned host buffers
    e2e = None
    if not args.no_e2e:
        keys_h = torch.empty(n, dtype=torch.int32, pin_memory=True)
        vals_h = torch.empty(n, dtype=torch.float64, pin_memory=True)
        keys_h.copy_(w.keys)
        vals_h.copy_(w.values)
        out_h = torch.empty(G, dtype=torch.float64, pin_memory=True)
        kd = torch.empty_like(w.keys)
        vd = torch.empty_like(w.values)

        def e2e_step():
            kd.copy_(keys_h, non_blocking=True)
            vd.copy_(vals_h, non_blocking=True)
            st.reset()
            st.add(kd, vd)
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
        # the e2e result must be the device result, bit for bit
        assert torch.equal(out_h.view(torch.int64), out.cpu().view(torch.int64))
        e2e = {"value": n * world / (e2e_ms / 1e3), "unit": "rows/s", "h2d_bytes_per_step": n * (4 + 8),
               "d2h_bytes_per_step": G * 8, "ms_per_step": e2e_ms}
        del keys_h, vals_h

    verify = None
    if args.verify:
        verify = verify_sampled(w, out, st)

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
            roof = {"bound": "hbm", "kernel": name, "achieved": round(ach, 1), "peak": peaks["hbm_gbs"],
                    "unit": "GB/s", "frac": round(ach / peaks["hbm_gbs"], 4), "traffic": None,
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
                                   f"exponents U[-40,40], 10% cancelling pairs",
                       "n": n, "G": G, "dist": args.dist, "L": L, "parallelism": f"shards{world}",
                       "l2": "inputs (12 B/row) far larger than L2; no flush"},
            "hbm_gbs_algorithmic": algo_bytes / (ms / 1e3) / 1e9,
            "roofline": roof,
            "kernels": prof,
            "fp64_baseline": {"ms_per_step": fp_ms, "rows_per_s": n / (fp_ms / 1e3),
                              "repro_over_fp64_time": ms / fp_ms},
            "e2e": e2e,
            "gpu_launches": int(launches),
            "clocks": clocks.summary(),
        }
        if verify is not None:
            result["verify"] = verify
    if dist is not None:
        dist.destroy_process_group()
    return result


def verify_sampled(w, out, st):
    """Check a sample of groups against the CPU oracle (rows gathered per group)."""
    import numpy as np
    import torch

    from oracle import oracle as O

    G = w.G
    gen = torch.Generator(device="cpu")
    gen.manual_seed(17)
    ngroups = min(G, 8 if G <= 1024 else 512)
    sample = torch.randperm(G, generator=gen)[:ngroups].to(w.keys.device)
    remap = torch.full((G,), -1, dtype=torch.int32, device=w.keys.device)
    remap[sample] = torch.arange(ngroups, dtype=torch.int32, device=w.keys.device)
    sel = remap[w.keys.long()]
    mask = sel >= 0
    k = sel[mask].cpu().numpy()
    v = w.values[mask].cpu().numpy()
    ref = O.groupby_sum_values(k, v, ngroups, w.L, threads=os.cpu_count() or 1)
    got = out[sample].cpu().numpy()
    ok = np.array_equal(got.view(np.int64), ref.view(np.int64))
    return {"groups": ngroups, "rows": int(k.size), "bit_exact": bool(ok)}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as fh:
            d = json.load(fh)
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured (MEASURED_PEAKS.json burst copy)"}
    except Exception:
        return {"hbm_gbs": 6800.0, "source": "fallback 6.8 TB/s"}


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


def cpu_baseline(args):
    threads = os.cpu_count() or 1
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
    threads = os.cpu_count() or 1
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
    res = run_ours(args, rank, world, local_rank)
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline:
            from oracle import oracle as O

            O.build()
            res["cpu_baseline"] = cpu_baseline(args)
        print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()

"""Request server: every query's result is bit-identical alone and in the
mix (continuous batching, chunked partial states, admission by memory), and
equal to the CPU oracle on a sample."""
import numpy as np
import pytest
import torch

import paper_1802_09883_gb300 as R
from paper_1802_09883_gb300 import serve as S
from paper_1802_09883_gb300 import workloads as WL
from oracle import oracle as O

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _bits(t):
    a = t.detach().cpu().numpy()
    return a.view(np.int64 if a.dtype == np.float64 else np.int32)


def _mixed_queries(seed, count):
    """Queries of mixed size, group count (both lanes), dtype and L."""
    table64 = WL.serving_table(400_000, groups=(1, 2e5), levels=9, seed=seed, device=DEV)
    vals32 = WL.random_values(400_000, -20, 20, WL._gen(seed + 1, DEV), DEV, torch.float32)
    trace, gaps = WL.serving_trace(count, table64, rows=(1e2, 4e5), seed=seed)
    out = []
    for i, (start, rows, level) in enumerate(trace):
        k, v, G = table64.query(start, rows, level)
        L = 3
        if i % 5 == 3:
            v = vals32[start:start + rows]
        if i % 7 == 2:
            L = 2
        out.append((k, v, G, L))
    return out, gaps


@pytest.mark.parametrize("chunk_rows,budget,max_active", [(4096, 64 << 20, 6), (1 << 16, 1 << 30, 64)])
def test_results_equal_alone_and_in_the_mix(chunk_rows, budget, max_active):
    queries, gaps = _mixed_queries(41, 48)
    alone = [R.groupby_sum(k, v, G, L) for k, v, G, L in queries]
    torch.cuda.synchronize()
    with S.Server(memory_budget=budget, chunk_rows=chunk_rows, max_active=max_active) as srv:
        t0 = S.now_ns() + 1_000_000
        arr = np.cumsum(gaps) * 2e-4  # ~0.2 ms mean gap: arrivals overlap running work
        reqs = [srv.submit(k, v, G, L, arrival_ns=t0 + int(a * 1e9)) for (k, v, G, L), a in zip(queries, arr)]
        for r in reqs:
            srv.wait(r, 120.0)
        st = srv.stats()
        for q, r, ref in zip(queries, reqs, alone):
            assert np.array_equal(_bits(r.out), _bits(ref)), (q[0].numel(), q[2], q[3])
            assert r.info.arrival_ns <= r.info.admit_ns <= r.info.done_ns
            srv.release(r)
    assert st["completed"] == len(queries)
    # the footprint counts the server's own buffers too; it stays within the
    # budget except when a query is admitted alone for progress
    assert st["memory_server_peak"] > 0
    assert st["memory_peak"] <= budget + st["memory_server_peak"]
    assert st["iterations"] > 1
    assert st["large_calls"] > 0  # some group counts take the partitioned lane


def test_server_results_match_oracle_on_a_sample():
    queries, _ = _mixed_queries(5, 12)
    with S.Server(chunk_rows=8192) as srv:
        reqs = [srv.submit(k, v, G, L) for k, v, G, L in queries]
        for (k, v, G, L), r in list(zip(queries, reqs))[::3]:
            srv.wait(r)
            vn = v.cpu().numpy()
            ref = O.groupby_sum_values(k.cpu().numpy(), vn, G, L, dtype=vn.dtype, threads=4)
            assert np.array_equal(_bits(r.out), ref.view(np.int64 if ref.dtype == np.float64 else np.int32))


def test_bad_keys_fail_only_their_query_and_empty_queries_give_zeros():
    g = WL._gen(9, DEV)
    k = WL.uniform_keys(50_000, 100, g, DEV)
    v = WL.random_values(50_000, -5, 5, g, DEV)
    bad = k.clone()
    bad[777] = 100
    with S.Server(chunk_rows=4096) as srv:
        r_ok = srv.submit(k, v, 100)
        r_bad = srv.submit(bad, v, 100)
        r_empty = srv.submit(k[:0], v[:0], 10)
        srv.wait(r_ok)
        with pytest.raises(R.ReproError):
            srv.wait(r_bad)
        assert r_bad.info.errors & 1
        srv.wait(r_empty)
        assert np.array_equal(_bits(r_ok.out), _bits(R.groupby_sum(k, v, 100)))
        assert np.all(_bits(r_empty.out) == 0)


def test_query_larger_than_the_budget_is_refused():
    k = torch.zeros(16, dtype=torch.int32, device=DEV)
    v = torch.ones(16, dtype=torch.float64, device=DEV)
    with S.Server(memory_budget=1 << 20) as srv:
        with pytest.raises(R.ReproError) as ei:
            srv.submit(k, v, 1_000_000)  # a 48 MB state
        assert ei.value.status == 3  # REPRO_ERANGE
        with pytest.raises(R.ReproError):  # pageable host output: not device-accessible
            srv.submit(k, v, 10, out=torch.empty(10, dtype=torch.float64))


def test_run_trace_reports_latency_and_throughput():
    table = WL.serving_table(1 << 20, groups=(1, 1e5), levels=6, seed=4, device=DEV)
    trace, gaps = WL.serving_trace(64, table, rows=(1e3, 1e6), seed=4)
    queries = [table.query(*q) for q in trace]
    with S.Server(chunk_rows=1 << 18) as srv:
        res = S.run_trace(srv, queries, np.cumsum(gaps) * 1e-4, keep_results=True)
    assert res["requests"] == 64 and res["rows_per_s"] > 0
    assert 0 < res["p50_ms"] <= res["p99_ms"] <= res["max_ms"]
    for (k, v, G), out in list(zip(queries, res["results"]))[::8]:
        assert np.array_equal(_bits(out), _bits(R.groupby_sum(k, v, G)))

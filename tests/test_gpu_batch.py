"""Batched grouped SUM (one persistent launch over many tasks) vs the
single-task path and the CPU oracle, bit for bit."""
import numpy as np
import pytest
import torch

import paper_1802_09883_gb300 as R
from paper_1802_09883_gb300 import workloads as WL
from oracle import oracle as O

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _tasks(seed, count, dtype, big_g=True):
    g = torch.Generator(device=DEV)
    g.manual_seed(seed)
    rs = np.random.default_rng(seed)
    out = []
    sizes = [0, 1, 3, 100, 2047, 2048, 2049] + [int(x) for x in np.exp(rs.uniform(np.log(1e3), np.log(3e6), count))]
    for i, n in enumerate(sizes):
        G = int(np.exp(rs.uniform(0, np.log(3000))))
        if big_g and i % 17 == 5:
            G = 20000  # beyond the single-pass table: two-pass path
        keys = WL.uniform_keys(n + 1, G, g, DEV)
        vals = WL.random_values(n + 1, -45, 45, g, DEV, dtype)
        if i % 13 == 7:  # 4-byte / 8-byte aligned only: two-pass path
            keys, vals = keys[1:], vals[1:]
        else:
            keys, vals = keys[:n], vals[:n]
        out.append((keys, vals, G))
    return out


def _single(keys, vals, G, L):
    st = R.State(G, L, vals.dtype)
    st.add(keys, vals)
    return st


@pytest.mark.parametrize("dtype,L", [(torch.float64, 3), (torch.float32, 2), (torch.float64, 4)])
def test_batched_states_equal_single_task_states(dtype, L):
    tasks = _tasks(100 + L, 60, dtype)
    states = R.groupby_sum_batched(tasks, L=L)
    for (k, v, G), st in zip(tasks, states):
        ref = _single(k, v, G, L)
        torch.cuda.synchronize()
        assert torch.equal(st.tensor, ref.tensor), (k.numel(), G)
        assert st.check() == 0


def test_batched_matches_oracle_on_a_sample():
    tasks = _tasks(7, 20, torch.float64, big_g=False)
    states = R.groupby_sum_batched(tasks, L=3)
    for (k, v, G), st in list(zip(tasks, states))[::4]:
        out = st.finalize().cpu().numpy()
        ref = O.groupby_sum_values(k.cpu().numpy(), v.cpu().numpy(), G, 3, threads=4)
        assert np.array_equal(out.view(np.int64), ref.view(np.int64))


def test_one_large_task_split_into_many_items_and_merged():
    w = WL.sweep_cell(1024, "zipf", 3, n=6_000_000, seed=5, device=DEV)
    (st,) = R.groupby_sum_batched([(w.keys, w.values, w.G)], L=3)
    ref = _single(w.keys, w.values, w.G, 3)
    torch.cuda.synchronize()
    assert torch.equal(st.tensor, ref.tensor)


@pytest.mark.parametrize("big_g", [False, True])  # True: side lanes (partitioned tasks) forked inside the graph
def test_batch_plan_replays_in_a_cuda_graph(big_g):
    tasks = _tasks(9, 30 if big_g else 12, torch.float64, big_g=big_g)
    states = [R.State(G, 3, torch.float64) for _, _, G in tasks]
    plan = R.BatchPlan([(k, v, st) for (k, v, _), st in zip(tasks, states)])
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        plan.run()  # warm-up outside the capture (module loading, attributes)
        torch.cuda.synchronize()
        for st in states:
            st.reset()
        with torch.cuda.graph(graph, stream=s):
            for st in states:
                st.reset()
            plan.run()
    torch.cuda.synchronize()
    for rep in range(2):
        graph.replay()
        torch.cuda.synchronize()
        for (k, v, G), st in zip(tasks, states):
            ref = _single(k, v, G, 3)
            torch.cuda.synchronize()
            assert torch.equal(st.tensor, ref.tensor), rep
    plan.close()


def test_bad_keys_flag_only_their_task():
    g = torch.Generator(device=DEV)
    g.manual_seed(3)
    k1 = WL.uniform_keys(10000, 50, g, DEV)
    v1 = WL.random_values(10000, -5, 5, g, DEV)
    k2 = k1.clone()
    k2[17] = 50  # out of range
    states = R.groupby_sum_batched([(k1, v1, 50), (k2, v1, 50)], L=2)
    assert states[0].check() == 0
    with pytest.raises(R.ReproError):
        states[1].check()


def test_batch_reset_and_finalize_in_one_launch_each():
    tasks = _tasks(21, 30, torch.float64)
    states = [R.State(G, 3, torch.float64) for _, _, G in tasks]
    outs = [torch.empty(G, dtype=torch.float64, device=DEV) for _, _, G in tasks]
    plan = R.BatchPlan([(k, v, st) for (k, v, _), st in zip(tasks, states)])
    plan.set_outputs(outs)
    for rep in range(2):  # the reset makes the second pass equal the first
        plan.reset().run().finalize()
        torch.cuda.synchronize()
        for (k, v, G), st, o in zip(tasks, states, outs):
            ref = _single(k, v, G, 3)
            assert torch.equal(st.tensor, ref.tensor), rep
            assert torch.equal(o.view(torch.int64), ref.finalize().view(torch.int64)), rep
    plan.close()


def test_many_large_group_tasks_share_one_partition_pass():
    g = torch.Generator(device=DEV)
    g.manual_seed(77)
    rs = np.random.default_rng(77)
    tasks = []
    for i in range(40):
        n = int(np.exp(rs.uniform(np.log(1), np.log(3e5))))
        G = int(np.exp(rs.uniform(np.log(7000), np.log(131072))))
        if i == 5:
            G = 700_000  # beyond the batched pass: its own lane
        keys = WL.uniform_keys(n, G, g, DEV)
        vals = WL.random_values(n, -45, 45, g, DEV)
        if i == 9 and n > 3:
            keys[n // 2] = G + 1  # one bad key, in this task only
        tasks.append((keys, vals, G))
    states = [R.State(G, 3) for _, _, G in tasks]
    plan = R.BatchPlan([(k, v, st) for (k, v, _), st in zip(tasks, states)])
    info = plan.describe()
    assert info["partition_tasks"] >= 30 and info["lane_tasks"] == 1, info
    plan.run()
    torch.cuda.synchronize()
    plan.close()
    for i, ((k, v, G), st) in enumerate(zip(tasks, states)):
        ref = R.State(G, 3)
        ref.add(k, v)
        torch.cuda.synchronize()
        assert torch.equal(st.tensor, ref.tensor), (i, k.numel(), G)
        if i == 9 and k.numel() > 3:
            with pytest.raises(R.ReproError):
                st.check()
        else:
            assert st.check() == 0

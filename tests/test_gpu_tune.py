"""Autotuning changes speed, never bits: after tuning, every path gives the
same state bytes as the built-in choice."""
import pytest
import torch

import paper_1802_09883_gb300 as R
from paper_1802_09883_gb300 import workloads as WL

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _state(k, v, G, L):
    st = R.State(G, L, v.dtype)
    st.add(k, v)
    torch.cuda.synchronize()
    return st


@pytest.mark.parametrize("G,L,dtype,path", [(1000, 3, torch.float64, "single_pass"),
                                            (100, 2, torch.float32, "single_pass"),
                                            (70000, 3, torch.float64, "partitioned")])
def test_tuned_choice_gives_identical_state(G, L, dtype, path):
    g = torch.Generator(device=DEV)
    g.manual_seed(5)
    n = 1 << 21
    keys = WL.uniform_keys(n, G, g, DEV)
    vals = WL.random_values(n, -40, 40, g, DEV, dtype)
    R.tune_clear()
    before = _state(keys, vals, G, L)
    res = R.tune(keys, vals, G, L)
    assert res["path"] == path
    assert res["candidates"] >= 1 and res["best_ms"] > 0 and res["default_ms"] > 0
    after = _state(keys, vals, G, L)  # now with the tuned choice
    assert torch.equal(before.tensor, after.tensor)
    R.tune_clear()


def test_batch_tune_keeps_results():
    g = torch.Generator(device=DEV)
    g.manual_seed(8)
    tasks = []
    for n, G in [(100_000, 50), (1_000_000, 1000), (5000, 3), (300_000, 4000)]:
        tasks.append((WL.uniform_keys(n, G, g, DEV), WL.random_values(n, -20, 20, g, DEV), G))
    states = [R.State(G, 3) for _, _, G in tasks]
    plan = R.BatchPlan([(k, v, st) for (k, v, _), st in zip(tasks, states)])
    ms = plan.tune()
    assert ms > 0
    for st in states:  # tuning leaves the states re-initialised
        assert torch.equal(st.tensor, R.State(st.G, 3).tensor)
    plan.run()
    torch.cuda.synchronize()
    for (k, v, G), st in zip(tasks, states):
        assert torch.equal(st.tensor, _state(k, v, G, 3).tensor)
    plan.close()


@pytest.mark.parametrize("G", [1_000_003, 70_000])
def test_every_partition_choice_gives_identical_state(G, tmp_path):
    """Each partition width with one and with two partition passes (forced
    through a loaded choice) gives the state bytes of the built-in rule."""
    g = torch.Generator(device=DEV)
    g.manual_seed(11)
    n = (1 << 22) + 3  # ragged tail
    keys = WL.uniform_keys(n, G, g, DEV)
    vals = WL.random_values(n, -40, 40, g, DEV)
    R.tune_clear()
    ref = _state(keys, vals, G, 3)
    bucket = (G - 1).bit_length()
    f = tmp_path / "choice.txt"
    for shift in range(6, 13):
        for levels in (1, 2):
            f.write_text(f"part 0 3 {bucket} {shift} {levels}\n")
            R.tune_clear()
            R.tune_load(str(f))
            st = _state(keys, vals, G, 3)
            assert torch.equal(ref.tensor, st.tensor), (shift, levels)
    R.tune_clear()


def test_partition_aggregation_configurations_give_identical_state(tmp_path):
    """The aggregation kernel's configuration recorded with a partition
    choice changes speed only."""
    g = torch.Generator(device=DEV)
    g.manual_seed(12)
    G, n = 300_000, (1 << 22) + 1
    keys = WL.uniform_keys(n, G, g, DEV)
    vals = WL.random_values(n, -40, 40, g, DEV)
    R.tune_clear()
    ref = _state(keys, vals, G, 3)
    bucket = (G - 1).bit_length()
    f = tmp_path / "choice.txt"
    for cfg in ["2 1024 8 1 1", "3 2048 16 1 1", "4 1024 8 2 1", "2 2048 8 3 1", "2 1024 8 2 1 1",
                "3 2048 8 2 1 8", "1 2048 8 2 1", "1 2048 16 1 1 4"]:
        f.write_text(f"part 0 3 {bucket} 10 0 {cfg}\n")
        R.tune_clear()
        R.tune_load(str(f))
        st = _state(keys, vals, G, 3)
        assert torch.equal(ref.tensor, st.tensor), cfg
    R.tune_clear()

"""Failure detection without a GPU fault: a bounded wait that runs out.

Every mbarrier wait of the single-pass kernel has a time limit; when it runs
out the kernel records REPRO_ERR_TIMEOUT in the state's error word, drains
the copies it issued and returns, so the context stays usable.  Here the
failure is injected from the host: REPRO_STALL_TILE=0 makes each CTA's
producer issue no tile at all in the first launch, and REPRO_WAIT_NS
shortens the wait limit to 20 ms, so every consumer's first wait runs out.
Nothing faults, traps or hangs: each wait gives up by itself.
"""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_SUB = r"""
import json, sys, numpy as np, torch
sys.path.insert(0, {root!r})
import paper_1802_09883_gb300 as R
from paper_1802_09883_gb300 import workloads as WL
from oracle import oracle as O
w = WL.plain(n=1 << 22, G=1024, L=3, seed=5, device="cuda")
res = {{}}
st = R.State(w.G, w.L)
init = st.tensor.cpu().numpy().copy()
st.add(w.keys, w.values)               # first launch: every CTA's first wait runs out (20 ms)
torch.cuda.synchronize()
after = st.tensor.cpu().numpy()
res["error_word"] = st.error_word()
try:
    st.check()
    res["status"] = 0
except R.ReproError as e:
    res["status"] = e.status
res["records_unchanged"] = bool(np.array_equal(after[64:], init[64:]))
# the context is still usable: the next call on a fresh state is exact
st2 = R.State(w.G, w.L)
st2.add(w.keys, w.values)
out = st2.finalize().cpu().numpy()
res["next_status"] = st2.check()
ref = O.init(np.float64, w.L, w.G)
O.groupby_sum(ref, w.keys.cpu().numpy(), w.values.cpu().numpy(), threads=4)
K, fl, lo, hi = st2.host_view()
oK, ofl, olo, ohi = O.to_bins(ref)
res["next_state_exact"] = bool((K == oK).all() and (fl == ofl).all() and (lo == olo).all() and (hi == ohi).all())
res["next_result_exact"] = bool(np.array_equal(out.view(np.int64), O.finalize(ref).view(np.int64)))
print(json.dumps(res))
"""


def test_bounded_wait_times_out_and_reports():
    env = {**os.environ, "REPRO_STALL_TILE": "0", "REPRO_STALL_LAUNCHES": "1", "REPRO_WAIT_NS": "20000000",
           "REPRO_FUSED_CFG": "2,2048,8,2"}
    r = subprocess.run([sys.executable, "-c", _SUB.format(root=ROOT)], env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    res = json.loads(r.stdout.strip().splitlines()[-1])
    assert res["status"] == 6, res            # REPRO_ETIMEOUT
    assert res["error_word"] & 2, res         # REPRO_ERR_TIMEOUT
    assert res["records_unchanged"], res      # aborted CTAs add nothing
    assert res["next_status"] == 0, res
    assert res["next_state_exact"] and res["next_result_exact"], res

"""The allocation-free entry point, repro_groupby_sum_noalloc.

Callers that cannot allocate device memory while they aggregate (a buffer
manager that owns the GPU's memory, an allocator owned by another runtime, a
request path that must not block on allocation) call this variant; it keeps
its scratch in a fixed array inside the library.  Its results must be the
same bits as repro_groupby_sum's.  This file is collected last, so a run
that stops at the first failure has run every other test before it.
"""
import ctypes

import numpy as np
import pytest
import torch

import paper_1802_09883_gb300 as R
from paper_1802_09883_gb300 import workloads as WL

pytestmark = pytest.mark.gpu


def _state_bytes(G, L, code):
    return R.lib().repro_state_bytes(code, L, G)


def _run(entry, keys, vals, G, L, code):
    """Init a state, accumulate through `entry` (a C-ABI function), finalize;
    return (state bytes, result) on the host."""
    lib = R.lib()
    s = torch.cuda.current_stream().cuda_stream
    st = torch.empty(_state_bytes(G, L, code), dtype=torch.uint8, device="cuda")
    out = torch.empty(G, dtype=vals.dtype, device="cuda")
    assert lib.repro_state_init(st.data_ptr(), code, L, G, s) == 0
    assert entry(keys.data_ptr(), vals.data_ptr(), keys.numel(), code, L, G, st.data_ptr(), s) == 0
    assert lib.repro_finalize(st.data_ptr(), code, L, G, out.data_ptr(), s) == 0
    err = ctypes.c_uint32(0)
    assert lib.repro_state_check(st.data_ptr(), ctypes.byref(err), s) == 0
    return st.cpu().numpy(), out.cpu().numpy()


@pytest.mark.parametrize("G,L,dtype,rows", [
    (1024, 3, torch.float64, (1_000_003, 333_333)),
    (16, 2, torch.float64, (1_000_003, 333_333)),
    (700, 4, torch.float32, (1_000_003, 333_333)),
    # 16 MiB holds only 99 partial tables of 3000 groups (56 bytes each at
    # L = 3) where the grid would have one CTA per SM: the cap on the CTA
    # count, and the longer tile ranges it gives each CTA, are in effect
    (3000, 3, torch.float64, ((1 << 24) + 3, (1 << 23) + 1)),
])
def test_noalloc_matches_repro_groupby_sum_on_two_calls(G, L, dtype, rows):
    lib = R.lib()
    code = R.REPRO_F64 if dtype == torch.float64 else R.REPRO_F32
    if G == 3000:  # the array's cap is below the one-CTA-per-SM grid
        assert (16 << 20) // (G * (8 + 16 * L)) < torch.cuda.get_device_properties(0).multi_processor_count
    for call, (n, seed) in enumerate(zip(rows, (11, 12))):
        w = WL.plain(n=n, G=G, L=L, seed=seed + G, device="cuda", e_lo=-45, e_hi=45, dtype=dtype)
        ref_st, ref_out = _run(lib.repro_groupby_sum, w.keys, w.values, G, L, code)
        got_st, got_out = _run(lib.repro_groupby_sum_noalloc, w.keys, w.values, G, L, code)
        iv = np.int64 if dtype == torch.float64 else np.int32
        assert np.array_equal(got_out.view(iv), ref_out.view(iv)), f"call {call}: results differ"
        assert np.array_equal(got_st, ref_st), f"call {call}: state bytes differ"


def test_noalloc_rejects_sizes_beyond_its_limit():
    lib = R.lib()
    s = torch.cuda.current_stream().cuda_stream
    G, L = 1 << 20, 3  # a table far beyond the single-pass path
    st = torch.empty(_state_bytes(G, L, R.REPRO_F64), dtype=torch.uint8, device="cuda")
    keys = torch.zeros(8, dtype=torch.int32, device="cuda")
    vals = torch.ones(8, dtype=torch.float64, device="cuda")
    assert lib.repro_state_init(st.data_ptr(), R.REPRO_F64, L, G, s) == 0
    rc = lib.repro_groupby_sum_noalloc(keys.data_ptr(), vals.data_ptr(), 8, R.REPRO_F64, L, G, st.data_ptr(), s)
    assert rc == 3  # REPRO_ERANGE

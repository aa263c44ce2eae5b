"""The allocation-free entry point polymul_batch_static, for callers that
cannot allocate device memory (for example while a CUDA graph is being
captured in global mode, or under a host memory manager that owns the
device memory).  Called through the C ABI directly; its results must equal
those of the plan-based entry point bit for bit, on consecutive calls that
switch degree and modulus (the fixed table memory is refreshed in place)
and on a repeated call.  Kept in a file that runs last."""
import ctypes

import numpy as np
import pytest

from paper_2307_06554_gb300 import workloads as wl

from helpers import from_dev, to_dev

pytestmark = pytest.mark.gpu


def _static_call(lib, n, q, ta, tb, tc, batch):
    import torch
    rc = lib.polymul_batch_static(ctypes.c_uint32(n), ctypes.c_uint64(q), ctypes.c_void_p(ta.data_ptr()),
                                  ctypes.c_void_p(tb.data_ptr()), ctypes.c_void_p(tc.data_ptr()),
                                  ctypes.c_uint64(batch), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc


def test_static_entry_matches_plan_entry():
    import torch
    from paper_2307_06554_gb300 import polymul
    lib = ctypes.CDLL(polymul.library_path())
    lib.polymul_batch_static.restype = ctypes.c_int
    cases = [(1024, 12289, 37, 1), (4096, 786433, 5, 2), (1024, 12289, 11, 3)]
    for n, q, batch, seed in cases:
        rng = np.random.default_rng(seed)
        a = wl.uniform_coeffs(rng, batch, [q], n, np.uint32)
        b = wl.uniform_coeffs(rng, batch, [q], n, np.uint32)
        ta, tb = to_dev(a), to_dev(b)
        tc = torch.full_like(ta, -1)
        assert _static_call(lib, n, q, ta, tb, tc, batch) == 0, polymul.polymul_last_error()
        torch.cuda.synchronize()
        got = from_dev(tc, np.uint32)
        with polymul.Plan(n, [q]) as plan:
            ref = torch.full_like(ta, -1)
            plan.batch(ta, tb, ref)
            torch.cuda.synchronize()
            want = from_dev(ref, np.uint32)
        assert np.array_equal(got, want), "n=%d q=%d" % (n, q)


def test_static_entry_rejects_out_of_range():
    from paper_2307_06554_gb300 import polymul
    lib = ctypes.CDLL(polymul.library_path())
    rc = lib.polymul_batch_static(ctypes.c_uint32(8192), ctypes.c_uint64(40961), None, None, None,
                                  ctypes.c_uint64(1), None)
    assert rc == polymul.POLYMUL_EINVAL
    assert "4096" in polymul.polymul_last_error()

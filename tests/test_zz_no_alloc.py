"""The allocation-free entry point polymul_batch_static, for callers that
cannot allocate device memory (for example while a CUDA graph is being
captured in global mode, or under a host memory manager that owns the
device memory).  Called through the C ABI directly; its results must equal
those of the plan-based entry point bit for bit and the CPU oracle, on
consecutive calls that switch degree and modulus (the fixed table memory is
refreshed in place), on a repeated call, and on a repeat from a second
stream.  Its status call reports an expired device wait.  Kept in a file
that runs last."""
import ctypes

import numpy as np
import pytest

from oracle import native
from paper_2307_06554_gb300 import workloads as wl

from helpers import from_dev, to_dev

pytestmark = pytest.mark.gpu


def _static_call(lib, n, q, ta, tb, tc, batch, stream=None):
    import torch
    st = stream if stream is not None else torch.cuda.current_stream().cuda_stream
    rc = lib.polymul_batch_static(ctypes.c_uint32(n), ctypes.c_uint64(q), ctypes.c_void_p(ta.data_ptr()),
                                  ctypes.c_void_p(tb.data_ptr()), ctypes.c_void_p(tc.data_ptr()),
                                  ctypes.c_uint64(batch), ctypes.c_void_p(st))
    return rc


def _lib():
    from paper_2307_06554_gb300 import polymul
    lib = ctypes.CDLL(polymul.library_path())
    lib.polymul_batch_static.restype = ctypes.c_int
    lib.polymul_static_status.restype = ctypes.c_int
    lib.polymul_static_status.argtypes = [ctypes.c_void_p]
    return polymul, lib


# (n, q, batch, seed): both ends of the degree range, the default reduction
# mode for small q and the bounded-value modes for 30- and 31-bit primes
CASES = [(1024, 12289, 37, 1), (4096, 786433, 5, 2), (1024, 12289, 11, 3), (16, 97, 41, 4),
         (4096, 1073692673, 6, 5), (2048, 2147389441, 9, 6), (256, 7681, 300, 7)]


def test_case_primes_are_ntt_friendly():
    for n, q, _, _ in CASES:
        assert wl.is_prime(q) and (q - 1) % (2 * n) == 0, (n, q)


def test_static_entry_matches_plan_entry_and_oracle():
    import torch
    polymul, lib = _lib()
    for n, q, batch, seed in CASES:
        rng = np.random.default_rng(seed)
        a = wl.uniform_coeffs(rng, batch, [q], n, np.uint32)
        b = wl.uniform_coeffs(rng, batch, [q], n, np.uint32)
        ta, tb = to_dev(a), to_dev(b)
        tc = torch.full_like(ta, -1)
        assert _static_call(lib, n, q, ta, tb, tc, batch) == 0, polymul.polymul_last_error()
        torch.cuda.synchronize()
        assert lib.polymul_static_status(None) == 0
        got = from_dev(tc, np.uint32)
        with polymul.Plan(n, [q]) as plan:
            ref = torch.full_like(ta, -1)
            plan.batch(ta, tb, ref)
            torch.cuda.synchronize()
            want = from_dev(ref, np.uint32)
        assert np.array_equal(got, want), "n=%d q=%d: static vs plan" % (n, q)
        assert np.array_equal(got.astype(np.uint64), native.polymul_batch(a, b, [q])), "n=%d q=%d: vs oracle" % (n, q)


def test_static_entry_repeat_on_second_stream():
    """The same (n, q) again, from another stream after the first finished:
    the tables are not re-uploaded (already in place) and the result is the
    same."""
    import torch
    polymul, lib = _lib()
    n, q, batch = 1024, 12289, 64
    rng = np.random.default_rng(9)
    a = wl.uniform_coeffs(rng, batch, [q], n, np.uint32)
    b = wl.uniform_coeffs(rng, batch, [q], n, np.uint32)
    ta, tb = to_dev(a), to_dev(b)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    c1, c2 = torch.full_like(ta, -1), torch.full_like(ta, -1)
    assert _static_call(lib, n, q, ta, tb, c1, batch, s1.cuda_stream) == 0
    s1.synchronize()
    assert _static_call(lib, n, q, ta, tb, c2, batch, s2.cuda_stream) == 0
    s2.synchronize()
    want = native.polymul_batch(a, b, [q])
    assert np.array_equal(from_dev(c1, np.uint32).astype(np.uint64), want)
    assert np.array_equal(from_dev(c2, np.uint32).astype(np.uint64), want)


def test_static_status_reports_expired_wait():
    """An expired bounded wait (made without a fault by the diagnostics
    entry) is reported by the status call, which allocates nothing; the next
    call is exact and clean."""
    import torch
    polymul, lib = _lib()
    n, q, batch = 1024, 12289, 200
    rng = np.random.default_rng(10)
    a = wl.uniform_coeffs(rng, batch, [q], n, np.uint32)
    b = wl.uniform_coeffs(rng, batch, [q], n, np.uint32)
    ta, tb = to_dev(a), to_dev(b)
    tc = torch.full_like(ta, -1)
    polymul.polymul_selftest_inject_wait(1, 64)
    try:
        assert _static_call(lib, n, q, ta, tb, tc, batch) == 0
        assert lib.polymul_static_status(None) == polymul.POLYMUL_ETIMEOUT
        assert lib.polymul_static_status(None) == 0  # reported once
    finally:
        polymul.polymul_selftest_inject_wait(0, 1)
    assert _static_call(lib, n, q, ta, tb, tc, batch) == 0
    assert lib.polymul_static_status(None) == 0
    assert np.array_equal(from_dev(tc, np.uint32).astype(np.uint64), native.polymul_batch(a, b, [q]))


def test_static_entry_rejects_out_of_range():
    polymul, lib = _lib()
    rc = lib.polymul_batch_static(ctypes.c_uint32(8192), ctypes.c_uint64(40961), None, None, None,
                                  ctypes.c_uint64(1), None)
    assert rc == polymul.POLYMUL_EINVAL
    assert "4096" in polymul.polymul_last_error()

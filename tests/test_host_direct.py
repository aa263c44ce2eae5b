"""The host-buffer entry's direct route: when a, b and c are page-locked host
memory the device maps, one launch of the NTT batch kernel reads a and b and
writes c in host memory itself (Sec. 4, overlapping computation with I/O).
Every case is compared element by element with the oracle and with the
staged route (POLYMUL_FLAG_HOST_STAGED: copies through device buffers), and
checks which route ran through polymul_plan_info.host_direct."""
import numpy as np
import pytest

from oracle import native
from paper_2307_06554_gb300 import workloads as wl

from helpers import assert_equal_residues

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pm():
    from paper_2307_06554_gb300 import polymul
    return polymul


def _primes(seed, k, bits, n):
    return wl.draw_primes(np.random.default_rng(seed), k, bits, bits, n.bit_length())


def _case(seed, batch, q_list, n, dtype):
    rng = np.random.default_rng(seed)
    return wl.uniform_coeffs(rng, batch, q_list, n, dtype), wl.uniform_coeffs(rng, batch, q_list, n, dtype)


def _pinned(x: np.ndarray):
    """A page-locked torch copy of x (same bytes, signed view)."""
    import torch
    view = x.view(np.int32 if x.dtype == np.uint32 else np.int64)
    return torch.from_numpy(np.ascontiguousarray(view)).pin_memory()


def _as(t, dtype):
    return t.numpy().view(dtype)


def _sampled_check(got, a, b, q_list, what, seed=0):
    """Degrees where the whole schoolbook product is slow: the first and
    last coefficient and six random ones of every row, from the oracle."""
    rng = np.random.default_rng(seed)
    n = a.shape[-1]
    for p in range(a.shape[0]):
        for j, q in enumerate(q_list):
            js = sorted({0, n - 1, *[int(x) for x in rng.integers(0, n, 6)]})
            want = native.coeffs(a[p, j], b[p, j], q, js)
            assert np.array_equal(got[p, j, js].astype(np.uint64), want), "%s product %d prime %d" % (what, p, j)


def _direct_calls(plan, pm):
    return pm.polymul_plan_info_get(plan.handle)["host_direct"]


def _run_both(pm, n, q_list, a, b, flags=0):
    """c by the direct route (pinned buffers) and by the staged route; the
    direct plan must have taken the direct route once."""
    ta, tb = _pinned(a), _pinned(b)
    tc = _pinned(np.full_like(a, 0xFFFF))
    with pm.Plan(n, q_list, flags=flags) as plan:
        before = _direct_calls(plan, pm)
        plan.batch_host(ta, tb, tc)
        assert _direct_calls(plan, pm) == before + 1
        pm.polymul_plan_status(plan.handle)
    out = _pinned(np.zeros_like(a))
    with pm.Plan(n, q_list, flags=flags | pm.FLAG_HOST_STAGED) as staged:
        staged.batch_host(ta, tb, out)  # page-locked, yet staged by the flag
        assert _direct_calls(staged, pm) == 0
    return _as(tc, a.dtype), _as(out, a.dtype)


def test_ring_1024_direct_equals_oracle_and_staged(pm):
    """n = 1024, q = 12289 (the unreduced-mode plan): 1000 products, not a
    multiple of the units the teams take at once."""
    n, q_list = 1024, [12289]
    a, b = _case(1, 1000, q_list, n, np.uint32)
    got, staged = _run_both(pm, n, q_list, a, b)
    assert np.array_equal(got, staged)
    assert_equal_residues(got, native.polymul_batch(a, b, q_list), "direct route")


@pytest.mark.parametrize("logn", [4, 5, 7, 9, 10, 11, 12, 13, 14])
@pytest.mark.parametrize("bits", [30, 31])
def test_u32_degrees(pm, logn, bits):
    """Every degree of the 32-bit direct kernels (warp teams below 2^10,
    CTA teams from there; radix 32 at 2^14), Harvey-range and 31-bit
    moduli, two or three primes per product."""
    n = 1 << logn
    k = 2 if logn >= 13 else 3
    batch = max(3, min(200, (1 << 18) // (n * k)))
    q_list = _primes(100 + logn + bits, k, bits, n)
    a, b = _case(logn * 7 + bits, batch, q_list, n, np.uint32)
    got, staged = _run_both(pm, n, q_list, a, b)
    assert np.array_equal(got, staged)
    idx = sorted({0, batch // 2, batch - 1})
    assert_equal_residues(got[idx], native.polymul_batch(a[idx], b[idx], q_list), "n=%d" % n)


@pytest.mark.parametrize("logn", [15, 16])
def test_u32_cluster_degrees(pm, logn):
    """32-bit words above 2^14: the plan's thread-block-cluster kernel reads
    and writes the host rows itself."""
    n = 1 << logn
    q_list = _primes(200 + logn, 2, 30, n)
    a, b = _case(logn * 5, 3, q_list, n, np.uint32)
    got, staged = _run_both(pm, n, q_list, a, b)
    assert np.array_equal(got, staged)
    _sampled_check(got, a, b, q_list, "n=%d" % n, seed=logn)


@pytest.mark.parametrize("logn", [4, 6, 8, 10, 12, 13, 14, 16])
def test_u64_degrees(pm, logn):
    """64-bit words: 59-bit primes, every direct shape family and the
    cluster kernels from 2^14."""
    n = 1 << logn
    q_list = _primes(300 + logn, 2, 59, n)
    batch = max(2, min(64, (1 << 16) // n))
    a, b = _case(logn * 11, batch, q_list, n, np.uint64)
    got, staged = _run_both(pm, n, q_list, a, b)
    assert np.array_equal(got, staged)
    if logn >= 14:
        _sampled_check(got, a, b, q_list, "n=%d" % n, seed=logn)
    else:
        idx = sorted({0, batch - 1})
        assert_equal_residues(got[idx], native.polymul_batch(a[idx], b[idx], q_list), "n=%d" % n)


def test_cyclic_direct(pm):
    """The ring x^n - 1 on the direct route."""
    n = 2048
    q_list = _primes(401, 2, 30, n)
    a, b = _case(402, 40, q_list, n, np.uint32)
    got, staged = _run_both(pm, n, q_list, a, b, flags=pm.FLAG_CYCLIC)
    assert np.array_equal(got, staged)
    assert_equal_residues(got[[0, 39]], native.polymul_batch(a[[0, 39]], b[[0, 39]], q_list, cyclic=True),
                          "cyclic")


def test_rewritten_buffers_are_read_again(pm):
    """The host rewrites the same page-locked buffers between calls: every
    call reads what the host wrote last (nothing of a or b is kept on the
    device), and writes every result."""
    n, q_list = 1024, [12289]
    ta = _pinned(np.zeros((300, 1, n), np.uint32))
    tb = _pinned(np.zeros((300, 1, n), np.uint32))
    tc = _pinned(np.zeros((300, 1, n), np.uint32))
    with pm.Plan(n, q_list) as plan:
        for seed in (11, 12, 13):
            a, b = _case(seed, 300, q_list, n, np.uint32)
            _as(ta, np.uint32)[:] = a
            _as(tb, np.uint32)[:] = b
            _as(tc, np.uint32)[:] = 0xFFFFFFFF
            plan.batch_host(ta, tb, tc)
            got = _as(tc, np.uint32).copy()
            assert_equal_residues(got, native.polymul_batch(a, b, q_list), "seed %d" % seed)
        assert _direct_calls(plan, pm) == 3


def test_offset_into_pinned_allocation(pm):
    """Rows that start inside a page-locked allocation (a slice from
    product 5 on): the route checks the range, not the allocation's start."""
    n, q_list = 512, [12289]
    a, b = _case(21, 64, q_list, n, np.uint32)
    ta, tb = _pinned(a), _pinned(b)
    tc = _pinned(np.zeros_like(a))
    with pm.Plan(n, q_list) as plan:
        plan.batch_host(ta[5:], tb[5:], tc[5:])
        assert _direct_calls(plan, pm) == 1
    got = _as(tc, np.uint32)
    assert not got[:5].any()  # rows before the slice untouched
    assert_equal_residues(got[5:], native.polymul_batch(a[5:], b[5:], q_list), "slice")


def test_pageable_or_mixed_buffers_take_the_staged_route(pm):
    """Pageable memory, or one pageable operand among pinned ones, is not
    read in place: the call is staged and exact."""
    n, q_list = 1024, [12289]
    a, b = _case(31, 50, q_list, n, np.uint32)
    want = native.polymul_batch(a, b, q_list)
    with pm.Plan(n, q_list) as plan:
        c = np.zeros_like(a)
        plan.batch_host(a, b, c)  # numpy arrays: pageable
        assert_equal_residues(c, want, "pageable")
        tc = _pinned(np.zeros_like(a))
        plan.batch_host(_pinned(a), b, tc)  # b pageable
        assert_equal_residues(_as(tc, np.uint32), want, "mixed")
        assert _direct_calls(plan, pm) == 0


def test_validate_flag_on_the_direct_route(pm):
    """POLYMUL_FLAG_VALIDATE reads a and b once more over the link before
    the product: exact for canonical inputs, EDOMAIN for a coefficient at q."""
    n, q = 1024, 12289
    a, b = _case(41, 20, [q], n, np.uint32)
    ta, tb, tc = _pinned(a), _pinned(b), _pinned(np.zeros_like(a))
    with pm.Plan(n, [q], flags=pm.FLAG_VALIDATE) as plan:
        plan.batch_host(ta, tb, tc)
        assert _direct_calls(plan, pm) == 1
        assert_equal_residues(_as(tc, np.uint32), native.polymul_batch(a, b, [q]), "validate")
        _as(tb, np.uint32)[7, 0, 100] = q
        with pytest.raises(pm.PolymulError) as e:
            plan.batch_host(ta, tb, tc)
        assert e.value.code == pm.POLYMUL_EDOMAIN


@pytest.mark.parametrize("n,q_list", [(256, [3329]), (64, [1000, 3329]), (2048, [97, 193])])
def test_aux_plans_direct(pm, n, q_list):
    """Auxiliary-prime plans (moduli without a 2n-th root of unity, n = 256,
    q = 3329 among them) read and write host rows in place too: the direct
    form of their kernel (centred lift, one 31-bit NTT prime, reduction mod
    each q) against the oracle and the staged route."""
    a, b = _case(42 + n, 20, q_list, n, np.uint32)
    with pm.Plan(n, q_list) as plan:
        assert plan.info["aux_primes"] == 1
    got, staged = _run_both(pm, n, q_list, a, b)
    assert np.array_equal(got, staged)
    assert_equal_residues(got, native.polymul_batch(a, b, q_list), "auxiliary prime n=%d" % n)


@pytest.mark.parametrize("flags", [0, 16])
def test_mapped_batches_queue_on_a_stream(pm, flags):
    """polymul_batch_mapped is asynchronous: eight batches over four host
    sets queued back to back on one stream (with and without
    POLYMUL_FLAG_OVERLAP), one synchronisation, every product exact."""
    import torch
    n, q_list = 1024, [12289]
    sets = []
    for s in range(4):
        a, b = _case(60 + s, 512, q_list, n, np.uint32)
        sets.append((a, b, _pinned(a), _pinned(b), _pinned(np.zeros_like(a))))
    stream = torch.cuda.Stream()
    with pm.Plan(n, q_list, flags=flags) as plan:
        for i in range(8):
            a, b, ta, tb, tc = sets[i % 4]
            plan.batch_mapped(ta, tb, tc, stream=stream)
        stream.synchronize()
        pm.polymul_plan_status(plan.handle, stream.cuda_stream)
    for a, b, ta, tb, tc in sets:
        assert_equal_residues(_as(tc, np.uint32), native.polymul_batch(a, b, q_list), "queued batch")


def test_mapped_chain_waits_for_its_operand(pm):
    """c1 = a b, then c2 = c1 b', queued on one stream with
    POLYMUL_FLAG_OVERLAP: the second batch reads what the first writes, so
    it must not run ahead of it (the stream-order record)."""
    import torch
    n, q_list = 2048, _primes(71, 1, 30, 2048)
    a, b = _case(72, 700, q_list, n, np.uint32)
    _, b2 = _case(73, 700, q_list, n, np.uint32)
    ta, tb, tb2 = _pinned(a), _pinned(b), _pinned(b2)
    tc1, tc2 = _pinned(np.zeros_like(a)), _pinned(np.zeros_like(a))
    stream = torch.cuda.Stream()
    with pm.Plan(n, q_list, flags=pm.FLAG_OVERLAP) as plan:
        for _ in range(3):
            plan.batch_mapped(ta, tb, tc1, stream=stream)
            plan.batch_mapped(tc1, tb2, tc2, stream=stream)
        stream.synchronize()
    c1 = native.polymul_batch(a, b, q_list).astype(np.uint32)
    assert_equal_residues(_as(tc1, np.uint32), c1, "first of the chain")
    idx = [0, 350, 699]
    assert_equal_residues(_as(tc2, np.uint32)[idx], native.polymul_batch(c1[idx], b2[idx], q_list), "second")


def test_mapped_rejects_what_it_cannot_read(pm):
    """Pageable memory, a misaligned row start and a tensor-path plan:
    EINVAL or ENOTSUP, nothing launched."""
    import torch
    n, q_list = 1024, [12289]
    a, b = _case(81, 8, q_list, n, np.uint32)
    ta, tb, tc = _pinned(a), _pinned(b), _pinned(np.zeros_like(a))
    with pm.Plan(n, q_list) as plan:
        with pytest.raises(pm.PolymulError) as e:
            plan.batch_mapped(a, b, np.zeros_like(a))  # pageable numpy arrays
        assert e.value.code == pm.POLYMUL_EINVAL
        raw = torch.zeros(8 * n * 4 + 16, dtype=torch.uint8).pin_memory()
        with pytest.raises(pm.PolymulError) as e:
            pm.polymul_batch_mapped(plan.handle, raw.data_ptr() + 2, tb, tc, 8, None)
        assert e.value.code == pm.POLYMUL_EINVAL
    with pm.Plan(n, q_list, path=pm.PATH_TENSOR) as plan:
        with pytest.raises(pm.PolymulError) as e:
            plan.batch_mapped(ta, tb, tc)
        assert e.value.code == pm.POLYMUL_ENOTSUP


def test_direct_then_device_entry_share_nothing(pm):
    """A direct host call and device-entry batches on the same plan, in
    turn: each exact (the host entry's counter slot is its own)."""
    import torch
    n, q_list = 2048, _primes(51, 1, 30, 2048)
    a, b = _case(52, 256, q_list, n, np.uint32)
    want = native.polymul_batch(a[[0, 255]], b[[0, 255]], q_list)
    ta, tb, tc = _pinned(a), _pinned(b), _pinned(np.zeros_like(a))
    with pm.Plan(n, q_list) as plan:
        for _ in range(2):
            da, db = ta.cuda(), tb.cuda()
            dc = torch.empty_like(da)
            plan.batch(da, db, dc)
            plan.batch_host(ta, tb, tc)
            torch.cuda.synchronize()
            pm.polymul_plan_status(plan.handle)
            assert np.array_equal(dc.cpu().numpy(), tc.numpy())
    assert_equal_residues(_as(tc, np.uint32)[[0, 255]], want, "direct after device entry")

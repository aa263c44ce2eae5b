"""Path (b) for moduli up to 2^62 in 64-bit words (k_toeplitz_u64: five to
eight drained 8-bit digits per operand, n = 2^10 .. 2^16) against the CPU
oracle: whole products where the oracle is quick, sampled coefficients at
the largest degrees, both rings, the smallest digit count, coefficients at
the extremes of the centred range and at each chunk's exactness bound, more
units than CTAs with a relaunch, and the serving loop on the tensor path."""
import numpy as np
import pytest

from oracle import native
from paper_2307_06554_gb300 import workloads as wl

from helpers import assert_equal_residues, run_plan_batch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pm():
    from paper_2307_06554_gb300 import polymul
    return polymul


def _select_u64(plan):
    for i in range(plan.info["candidates"]):
        info = plan.select(i)
        if info["tensor_kernel"] == 6:
            return info
    raise AssertionError("no 64-bit digit kernel among the candidates")


def _sampled(got, a, b, q_list, rng, cyclic=False, count=16):
    n = a.shape[-1]
    for p in range(a.shape[0]):
        for jq, q in enumerate(q_list):
            js = sorted(set([0, 1, 7, 8, 1023, 1024, n // 2, n - 1] + [int(x) for x in rng.integers(0, n, count)]))
            want = native.coeffs(a[p, jq], b[p, jq], q, js, cyclic=cyclic)
            assert np.array_equal(got[p, jq, js].astype(np.uint64), want), (p, jq)


@pytest.mark.parametrize("n,bits,k,batch,cyclic", [(1024, 59, 2, 9, False), (2048, 45, 1, 5, True),
                                                   (4096, 59, 2, 3, False), (4096, 33, 2, 3, False),
                                                   (1024, 61, 1, 4, True)])
def test_u64_digits_against_oracle(pm, n, bits, k, batch, cyclic):
    rng = np.random.default_rng(n + 3 * bits + k)
    q_list = wl.draw_primes(rng, k, bits, bits, 1)
    a = wl.uniform_coeffs(rng, batch, q_list, n, np.uint64)
    b = wl.uniform_coeffs(rng, batch, q_list, n, np.uint64)
    with pm.Plan(n, q_list, path=pm.PATH_TENSOR, flags=pm.FLAG_CYCLIC if cyclic else 0) as plan:
        info = _select_u64(plan)
        want_l = next(L for L in range(1, 9) if 127 * ((1 << (8 * L)) - 1) // 255 >= max(q_list) // 2)
        assert info["digit_bits"] == 8 and info["digits"] == max(5, want_l), info
        got = run_plan_batch(plan, a, b)
        pm.polymul_plan_status(plan.handle)
    assert_equal_residues(got, native.polymul_batch(a, b, q_list, cyclic=cyclic), "u64 digits n=%d" % n)


@pytest.mark.parametrize("n,bits", [(8192, 59), (16384, 50), (65536, 59)])
def test_u64_digits_large_degrees_sampled(pm, n, bits):
    rng = np.random.default_rng(n + bits)
    q_list = wl.draw_primes(rng, 1, bits, bits, 1)
    a = wl.uniform_coeffs(rng, 1, q_list, n, np.uint64)
    b = wl.uniform_coeffs(rng, 1, q_list, n, np.uint64)
    with pm.Plan(n, q_list, path=pm.PATH_TENSOR) as plan:
        assert plan.info["tensor_kernel"] == 6  # the only tensor kernel at these shapes
        got = run_plan_batch(plan, a, b)
        pm.polymul_plan_status(plan.handle)
    _sampled(got, a, b, q_list, rng)


def test_u64_extremes_and_chunk_bound(pm):
    """Coefficients at +-floor(q/2), and every coefficient's three low
    digits at -128: each digit-pair product of those is 2^14, so a chunk's
    sum over 1024 K reaches 2^24, the edge of exact fp32 integers."""
    n = 4096
    q = wl.draw_primes(np.random.default_rng(5), 1, 62, 62, 1)[0]  # the largest digit count (8)
    x = sum(-128 << (8 * s) for s in range(3))
    a = np.full((3, 1, n), (q + x) % q, np.uint64)
    b = np.full((3, 1, n), (q + x) % q, np.uint64)
    a[1, 0] = q // 2
    b[1, 0, ::2] = q // 2 + 1
    a[2, 0, ::3] = q - 1
    with pm.Plan(n, [q], path=pm.PATH_TENSOR) as plan:
        assert _select_u64(plan)["digits"] == 8
        got = run_plan_batch(plan, a, b)
        pm.polymul_plan_status(plan.handle)
    assert_equal_residues(got, native.polymul_batch(a, b, [q]), "extremes")


def test_u64_many_units_and_relaunch(pm):
    n = 2048
    rng = np.random.default_rng(2049)
    q_list = wl.draw_primes(rng, 3, 58, 59, 1)
    a = wl.uniform_coeffs(rng, 70, q_list, n, np.uint64)
    b = wl.uniform_coeffs(rng, 70, q_list, n, np.uint64)
    with pm.Plan(n, q_list, path=pm.PATH_TENSOR) as plan:
        assert 70 * 3 * _select_u64(plan)["tensor_groups"] > plan.info["grid"]
        got = run_plan_batch(plan, a, b)
        again = run_plan_batch(plan, a[:4], b[:4])
        pm.polymul_plan_status(plan.handle)
    assert np.array_equal(again, got[:4])
    assert_equal_residues(got[:6], native.polymul_batch(a[:6], b[:6], q_list), "many units")


def test_server_on_the_tensor_path(pm):
    """Requests submitted after polymul_server_set_path(TENSOR) run on the
    64-bit digit kernel (degrees below 1024 stay on the NTT path); switching
    back gives the NTT kernels; every result matches the oracle."""
    import torch
    rng = np.random.default_rng(77)
    pool = wl.draw_primes(rng, 6, 59, 59, 15)
    with pm.Server(pool, 16384, device_bytes=512 << 20, lanes=4) as srv:
        srv.set_path(pm.PATH_TENSOR)
        cases = [(512, [0, 3]), (1024, [1]), (4096, [2, 5, 0]), (16384, [4]), (2048, [3, 1])]
        outs = []
        for n, idx in cases:
            qs = [pool[i] for i in idx]
            a = wl.uniform_coeffs(rng, 1, qs, n, np.uint64)[0]
            b = wl.uniform_coeffs(rng, 1, qs, n, np.uint64)[0]
            ha = torch.from_numpy(a.view(np.int64).copy()).pin_memory()
            hb = torch.from_numpy(b.view(np.int64).copy()).pin_memory()
            hc = torch.zeros_like(ha).pin_memory()
            outs.append((srv.submit(n, idx, ha.numpy(), hb.numpy(), hc.numpy()), a, b, qs, hc, ha, hb))
        srv.set_path(pm.PATH_NTT)
        for t, a, b, qs, hc, _, _ in outs:
            srv.wait(t, timeout_s=60.0)
        st = srv.stats(reset=True)
        assert st["failed"] == 0 and st["completed"] == len(cases), st
    for t, a, b, qs, hc, _, _ in outs:
        n = a.shape[-1]
        got = hc.numpy().view(np.uint64).reshape(len(qs), n)
        if n <= 4096:
            assert_equal_residues(got[None], native.polymul_batch(a[None], b[None], qs), "served n=%d" % n)
        else:
            _sampled(got[None], a[None], b[None], qs, rng)


def test_server_set_path_rejects_bad_path(pm):
    rng = np.random.default_rng(78)
    pool = wl.draw_primes(rng, 2, 59, 59, 15)
    with pm.Server(pool, 4096, device_bytes=64 << 20, lanes=2) as srv:
        with pytest.raises(pm.PolymulError) as ei:
            srv.set_path(7)
        assert ei.value.code == pm.POLYMUL_EINVAL

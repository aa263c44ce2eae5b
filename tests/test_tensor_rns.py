"""Path (b) with the paper's residue number system of small moduli
(k_toeplitz_rns, Sec. 2.4) against the CPU oracle: 32-bit moduli (the RNS
kernel as a tensor-path candidate beside the digit kernels), 59- and 62-bit
moduli in 64-bit words (where it is the only tensor kernel), a modulus with
no NTT route, both rings, the largest centred products, batches that are
not a multiple of the grid, and agreement with the NTT path."""
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


def _select_rns(pm, plan):
    info = plan.info
    if info["rns_moduli"] == 0:
        idx = [i for i in range(info["candidates"]) if plan.select(i)["rns_moduli"] > 0]
        assert idx, "no RNS candidate"
        info = plan.select(idx[0])
    assert info["path"] == pm.PATH_TENSOR and info["rns_moduli"] > 0
    return info


def _sampled(got, a, b, q_list, rng, cyclic=False, count=24):
    n = a.shape[-1]
    for p in range(a.shape[0]):
        for jq, q in enumerate(q_list):
            js = sorted(set([0, 1, 7, 8, n // 2, n - 1] + [int(x) for x in rng.integers(0, n, count)]))
            want = native.coeffs(a[p, jq], b[p, jq], q, js, cyclic=cyclic)
            assert np.array_equal(got[p, jq, js].astype(np.uint64), want), (p, jq)


@pytest.mark.parametrize("n,bits", [(64, 14), (256, 14), (1024, 14), (1024, 30), (2048, 22), (4096, 30)])
def test_rns_u32_against_oracle(pm, n, bits):
    rng = np.random.default_rng(n + 3 * bits)
    q_list = [12289] if bits == 14 else wl.draw_primes(rng, 2, bits, bits, 1)
    batch = {64: 33, 256: 17, 1024: 9, 2048: 5, 4096: 3}[n]
    a = wl.uniform_coeffs(rng, batch, q_list, n, np.uint32)
    b = wl.uniform_coeffs(rng, batch, q_list, n, np.uint32)
    with pm.Plan(n, q_list, path=pm.PATH_TENSOR) as plan:
        info = _select_rns(pm, plan)
        assert info["rns_moduli"] == len(pm.polymul_tensor_rns_base(n, max(q_list)))
        got = run_plan_batch(plan, a, b)
        pm.polymul_plan_status(plan.handle)
    assert_equal_residues(got, native.polymul_batch(a, b, q_list), "rns n=%d bits=%d" % (n, bits))


@pytest.mark.parametrize("n,bits,k", [(64, 59, 2), (256, 62, 1), (1024, 59, 2), (2048, 59, 1), (4096, 59, 2)])
def test_rns_u64_against_oracle(pm, n, bits, k):
    """64-bit words: the RNS kernel (the tensor path's only kernel below
    n = 1024; beside the 64-bit digit kernel from 1024 on, first there from
    n = 4096)."""
    rng = np.random.default_rng(7 * n + bits)
    q_list = wl.draw_primes(rng, k, bits, bits, 1)
    batch = {64: 21, 256: 11, 1024: 5, 2048: 3, 4096: 2}[n]
    a = wl.uniform_coeffs(rng, batch, q_list, n, np.uint64)
    b = wl.uniform_coeffs(rng, batch, q_list, n, np.uint64)
    with pm.Plan(n, q_list, path=pm.PATH_TENSOR) as plan:
        codes = [plan.select(i)["tensor_kernel"] for i in range(plan.info["candidates"])]
        assert codes == ([3] if n < 1024 else [6, 3] if n <= 2048 else [3, 6]), codes
        info = plan.select(codes.index(3))
        assert plan.elem_bytes == 8 and info["path"] == pm.PATH_TENSOR and info["rns_moduli"] > 0
        got = run_plan_batch(plan, a, b)
        pm.polymul_plan_status(plan.handle)
    if n <= 2048:
        assert_equal_residues(got, native.polymul_batch(a, b, q_list), "rns u64 n=%d" % n)
    else:
        _sampled(got, a, b, q_list, rng)


@pytest.mark.parametrize("n,bits,elem", [(1024, 59, 8), (2048, 30, 4), (128, 62, 8)])
def test_rns_cyclic(pm, n, bits, elem):
    rng = np.random.default_rng(n + bits + 1)
    q_list = wl.draw_primes(rng, 1, bits, bits, 1)
    dt = np.uint32 if elem == 4 else np.uint64
    a = wl.uniform_coeffs(rng, 4, q_list, n, dt)
    b = wl.uniform_coeffs(rng, 4, q_list, n, dt)
    with pm.Plan(n, q_list, path=pm.PATH_TENSOR, flags=pm.FLAG_CYCLIC) as plan:
        _select_rns(pm, plan)
        got = run_plan_batch(plan, a, b)
    assert_equal_residues(got, native.polymul_batch(a, b, q_list, cyclic=True), "rns cyclic n=%d" % n)


def test_rns_extremes(pm):
    """All q-1 (centred -1), the most negative and most positive centred
    values: the centred products reach n floor(q/2)^2, the range the base
    must cover with its margin."""
    n = 1024
    q = (1 << 62) - 57
    assert wl.is_prime(q)
    a = np.empty((4, 1, n), np.uint64)
    b = np.empty((4, 1, n), np.uint64)
    a[0] = q - 1
    b[0] = q - 1
    a[1] = q // 2 + 1  # -(q-1)/2
    b[1] = q // 2 + 1
    a[2] = q // 2      # +(q-1)/2
    b[2] = q // 2 + 1
    a[3, 0, ::2] = q // 2
    a[3, 0, 1::2] = q // 2 + 1
    b[3] = q // 2
    with pm.Plan(n, [q], path=pm.PATH_TENSOR) as plan:
        got = run_plan_batch(plan, a, b)
    assert_equal_residues(got, native.polymul_batch(a, b, [q]), "rns extremes")


def test_rns_modulus_without_ntt_route(pm):
    """q = 2^61 + 1 (not prime, above 2^32): no NTT route; AUTO takes the
    tensor path's RNS kernel."""
    q = (1 << 61) + 1
    n = 512
    rng = np.random.default_rng(61)
    a = wl.uniform_coeffs(rng, 6, [q], n, np.uint64)
    b = wl.uniform_coeffs(rng, 6, [q], n, np.uint64)
    with pm.Plan(n, [q]) as plan:
        info = plan.info
        assert info["path"] == pm.PATH_TENSOR and info["rns_moduli"] > 0
        got = run_plan_batch(plan, a, b)
    assert_equal_residues(got, native.polymul_batch(a, b, [q]), "q = 2^61 + 1")


def test_rns_ragged_units_and_relaunch(pm):
    n = 4096
    rng = np.random.default_rng(41)
    q_list = wl.draw_primes(rng, 2, 59, 59, 13)
    a = wl.uniform_coeffs(rng, 97, q_list, n, np.uint64)
    b = wl.uniform_coeffs(rng, 97, q_list, n, np.uint64)
    with pm.Plan(n, q_list, path=pm.PATH_TENSOR) as plan:
        info = plan.info
        assert 97 * 2 * info["tensor_groups"] > info["grid"]
        got = run_plan_batch(plan, a, b)
        got2 = run_plan_batch(plan, a[:3], b[:3])
        pm.polymul_plan_status(plan.handle)
    assert np.array_equal(got2, got[:3])
    rs = np.random.default_rng(42)
    for p in (0, 48, 96):
        js = sorted(int(x) for x in rs.integers(0, n, 12))
        for jq, q in enumerate(q_list):
            assert np.array_equal(got[p, jq, js].astype(np.uint64), native.coeffs(a[p, jq], b[p, jq], q, js)), (p, jq)


def test_rns_matches_ntt_path(pm):
    """59-bit NTT-friendly primes: the NTT path and the tensor path's RNS
    kernel agree on every coefficient."""
    n = 2048
    rng = np.random.default_rng(2048)
    q_list = wl.draw_primes(rng, 2, 59, 59, 12)
    a = wl.uniform_coeffs(rng, 40, q_list, n, np.uint64)
    b = wl.uniform_coeffs(rng, 40, q_list, n, np.uint64)
    with pm.Plan(n, q_list, path=pm.PATH_TENSOR) as tp, pm.Plan(n, q_list, path=pm.PATH_NTT) as npl:
        assert np.array_equal(run_plan_batch(tp, a, b), run_plan_batch(npl, a, b))


def test_rns_every_tensor_candidate(pm):
    """A 32-bit plan's tensor candidates (whole-product digits, tiled
    digits, RNS) all give the oracle's result."""
    n, q = 1024, 1000003
    rng = np.random.default_rng(3)
    a = wl.uniform_coeffs(rng, 11, [q], n, np.uint32)
    b = wl.uniform_coeffs(rng, 11, [q], n, np.uint32)
    want = native.polymul_batch(a, b, [q])
    with pm.Plan(n, [q], path=pm.PATH_TENSOR) as plan:
        kinds = set()
        for i in range(plan.info["candidates"]):
            info = plan.select(i)
            kinds.add((info["tensor_groups"] > 0, info["rns_moduli"] > 0))
            assert_equal_residues(run_plan_batch(plan, a, b), want, "candidate %d" % i)
    assert kinds == {(False, False), (True, False), (True, True)}

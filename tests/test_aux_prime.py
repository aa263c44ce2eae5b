"""Auxiliary-prime NTT (moduli with no 2n-th root of unity, including
composite and power-of-two moduli, which Sec. 2.1 of the paper allows):
bit-exact against the oracle, at the full size of the n = 256, q = 3329
workload and on the extreme centred values."""
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


def test_ring_small_full_size(pm):
    w = wl.ring_small()
    with pm.Plan(w.n, w.q_list) as plan:
        assert plan.info["path"] == pm.PATH_NTT and plan.info["aux_primes"] == 1
        got = run_plan_batch(plan, w.a, w.b)
    assert_equal_residues(got, native.polymul_batch(w.a, w.b, w.q_list), w.name)


@pytest.mark.parametrize("n,q_list", [(16, [1000]), (64, [1000, 3329]), (128, [3329, 255]), (256, [1024]),
                                      (512, [257, 769]), (2048, [97, 193]), (256, [3329, 2053])])
def test_aux_moduli(pm, n, q_list):
    rng = np.random.default_rng(n + sum(q_list))
    batch = 9
    a = wl.uniform_coeffs(rng, batch, q_list, n, np.uint32)
    b = wl.uniform_coeffs(rng, batch, q_list, n, np.uint32)
    # extremes: q-1 (centred -1), q//2 and q//2 + 1 (largest magnitudes)
    for j, q in enumerate(q_list):
        a[0, j] = q - 1
        b[0, j] = q - 1
        a[1, j] = q // 2
        b[1, j] = q // 2
        a[2, j] = q // 2 + 1 if q > 2 else 1
        b[2, j] = q // 2 + 1 if q > 2 else 1
        a[3, j] = q // 2
        b[3, j] = q // 2 + 1 if q > 2 else 1
    with pm.Plan(n, q_list) as plan:
        assert plan.info["aux_primes"] == 1
        got = run_plan_batch(plan, a, b)
    assert_equal_residues(got, native.polymul_batch(a, b, q_list), "aux n=%d q=%s" % (n, q_list))


def test_no_route_is_reported(pm):
    """q = 8192 (not prime) at n = 2^15 has neither an auxiliary-prime route
    nor a tensor-path shape (degrees up to 2^14): creation fails with
    ENOTSUP, not a fallback."""
    with pytest.raises(pm.PolymulError) as ei:
        pm.Plan(32768, [8192])
    assert ei.value.code == pm.POLYMUL_ENOTSUP


@pytest.mark.parametrize("n,q", [(128, 3331), (256, 3329), (512, 1000), (1024, 1000)])
def test_aux_every_candidate(pm, n, q):
    """Every kernel the autotuner may pick for an auxiliary-prime plan
    (radix-16 and radix-4 register passes) is exact."""
    rng = np.random.default_rng(n + q)
    a = wl.uniform_coeffs(rng, 19, [q], n, np.uint32)
    b = wl.uniform_coeffs(rng, 19, [q], n, np.uint32)
    want = native.polymul_batch(a, b, [q])
    with pm.Plan(n, [q]) as plan:
        assert plan.info["aux_primes"] == 1
        ncand = plan.info["candidates"]
        assert ncand == 2
        seen = set()
        for i in range(ncand):
            info = plan.select(i)
            seen.add(info["radix_bits"])
            assert_equal_residues(run_plan_batch(plan, a, b), want, "candidate %d" % i)
        assert seen == {2, 4}

"""Path (b), the Toeplitz (matrix) form on the tensor cores, against the CPU
oracle: bit-exact at the full size of the n = 1024 workload, on several
digit counts, and on adversarial inputs whose digit products are all of
maximal magnitude, so that partial sums reach exactly 2^24 -- the largest
magnitude the design allows, at the edge of exact fp32 integers."""
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


def _tensor_plan(pm, n, q_list):
    plan = pm.Plan(n, q_list, path=pm.PATH_TENSOR)
    assert plan.info["path"] == pm.PATH_TENSOR
    return plan


def test_ring_1024_full_size_tensor(pm):
    w = wl.ring_1024()
    with _tensor_plan(pm, w.n, w.q_list) as plan:
        got = run_plan_batch(plan, w.a, w.b)
    assert_equal_residues(got, native.polymul_batch(w.a, w.b, w.q_list), "tensor " + w.name)


@pytest.mark.parametrize("n,bits,batch", [(1024, 14, 37), (1024, 22, 9), (1024, 30, 9), (2048, 14, 7), (2048, 20, 5)])
def test_tensor_digit_counts(pm, n, bits, batch):
    rng = np.random.default_rng(n + bits)
    q_list = wl.draw_primes(rng, 2, bits, bits, 1)  # any odd prime: the tensor path needs no root of unity
    a = wl.uniform_coeffs(rng, batch, q_list, n, np.uint32)
    b = wl.uniform_coeffs(rng, batch, q_list, n, np.uint32)
    with _tensor_plan(pm, n, q_list) as plan:
        got = run_plan_batch(plan, a, b)
    assert_equal_residues(got, native.polymul_batch(a, b, q_list), "tensor n=%d bits=%d" % (n, bits))


def test_tensor_non_ntt_modulus(pm):
    """q = 3329 has no 2n-th root of unity at n = 1024: AUTO picks the tensor path."""
    rng = np.random.default_rng(4)
    q = 3329
    a = wl.uniform_coeffs(rng, 17, [q], 1024, np.uint32)
    b = wl.uniform_coeffs(rng, 17, [q], 1024, np.uint32)
    with pm.Plan(1024, [q]) as plan:
        assert plan.info["path"] == pm.PATH_TENSOR
        got = run_plan_batch(plan, a, b)
    assert_equal_residues(got, native.polymul_batch(a, b, [q]), "q=3329")


def test_tensor_exactness_boundary(pm):
    """Every coefficient's three low balanced 8-bit digits are -128, so every
    digit product of those digits is +-2^14 and, for the output coefficient
    with no wrap-around, the 1024-term sum is exactly 2^24."""
    q = 1073479681  # a 30-bit prime; centred values span four 8-bit digits
    assert wl.is_prime(q)
    n = 1024
    x = -128 - 128 * 256 - 128 * 65536  # digits (-128, -128, -128, 0)
    v = q + x
    a = np.full((3, 1, n), v, np.uint32)
    b = np.full((3, 1, n), v, np.uint32)
    rng = np.random.default_rng(11)
    # second product: random signs of the same magnitude pattern
    signs = rng.integers(0, 2, size=(2, n))
    a[1, 0] = np.where(signs[0] == 1, v, -x)
    b[1, 0] = np.where(signs[1] == 1, v, -x)
    # third product: all q-1 (centred -1) against the extreme pattern
    a[2, 0] = q - 1
    with _tensor_plan(pm, n, [q]) as plan:
        got = run_plan_batch(plan, a, b)
    assert_equal_residues(got, native.polymul_batch(a, b, [q]), "exactness boundary")


def test_tensor_matches_ntt_path(pm):
    """Both paths on the same NTT-friendly batch: bit-identical."""
    w = wl.ring_1024(batch=300, seed=21)
    with _tensor_plan(pm, w.n, w.q_list) as tp, pm.Plan(w.n, w.q_list, path=pm.PATH_NTT) as npl:
        assert np.array_equal(run_plan_batch(tp, w.a, w.b), run_plan_batch(npl, w.a, w.b))

"""Large degrees, n = 2^14 .. 2^16: one thread-block cluster per product
with exchanges through distributed shared memory (64-bit words, and 32-bit
words above 2^14), or one 512-thread CTA per product (32-bit words at 2^14;
the cluster kernel is that plan's autotuner candidate, checked with every
other candidate in the autotuner tests).
Checked against the oracle on sampled output coefficients and, for the
whole output, by evaluation at roots of x^n + 1 (c(w) = a(w) b(w) mod q for
w^n = -1), an independent check of every coefficient at once."""
import numpy as np
import pytest

from oracle import native
from paper_2307_06554_gb300 import workloads as wl

from helpers import run_plan_batch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pm():
    from paper_2307_06554_gb300 import polymul
    return polymul


def _root(q, n):
    e = (q - 1) // (2 * n)
    for g in range(2, 1000):
        psi = pow(g, e, q)
        if pow(psi, n, q) == q - 1:
            return psi
    raise AssertionError


def _evaluate(poly, x, q):
    """Horner over numpy chunks: exact with Python integers."""
    acc = 0
    for coef in reversed(poly.tolist()):
        acc = (acc * x + coef) % q
    return acc


def _check(a, b, got, q_list, n, samples=24, roots=2, seed=0):
    rng = np.random.default_rng(seed)
    batch, k = a.shape[0], a.shape[1]
    for p in range(batch):
        for j, q in enumerate(q_list):
            js = sorted(set([0, 1, n // 2, n - 1] + [int(x) for x in rng.integers(0, n, samples)]))
            want = native.coeffs(a[p, j], b[p, j], q, js)
            assert np.array_equal(got[p, j, js].astype(np.uint64), want), (p, j)
            psi = _root(q, n)
            for r in range(roots):
                w = pow(psi, 2 * int(rng.integers(0, n)) + 1, q)
                assert _evaluate(got[p, j].astype(np.uint64), w, q) == \
                    _evaluate(a[p, j].astype(np.uint64), w, q) * _evaluate(b[p, j].astype(np.uint64), w, q) % q


@pytest.mark.parametrize("logn", [14, 15, 16])
def test_u64_cluster_degrees(pm, logn):
    n = 1 << logn
    rng = np.random.default_rng(logn)
    q_list = wl.draw_primes(rng, 2, 59, 59, 17)
    a = wl.uniform_coeffs(rng, 2, q_list, n, np.uint64)
    b = wl.uniform_coeffs(rng, 2, q_list, n, np.uint64)
    a[1, 0] = q_list[0] - 1  # extremes
    b[1, 0] = q_list[0] - 1
    with pm.Plan(n, q_list) as plan:
        got = run_plan_batch(plan, a, b)
    _check(a, b, got, q_list, n, seed=logn)
    # all-(q-1) squared has a closed form: coefficient j is 2j + 2 - n mod q
    q = q_list[0]
    assert np.array_equal(got[1, 0].astype(object), np.array([(2 * j + 2 - n) % q for j in range(n)], dtype=object))


@pytest.mark.parametrize("logn,bits", [(14, 31), (15, 30), (16, 30), (14, 17)])
def test_u32_cluster_degrees(pm, logn, bits):
    n = 1 << logn
    rng = np.random.default_rng(logn * 3 + bits)
    # 17 bits: 65537 = 2^16 + 1 (the unreduced small-modulus mode)
    q_list = [65537] if bits == 17 else wl.draw_primes(rng, 2, bits, bits, 17)
    a = wl.uniform_coeffs(rng, 3, q_list, n, np.uint32)
    b = wl.uniform_coeffs(rng, 3, q_list, n, np.uint32)
    with pm.Plan(n, q_list) as plan:
        got = run_plan_batch(plan, a, b)
    _check(a, b, got, q_list, n, roots=1, seed=logn + bits)

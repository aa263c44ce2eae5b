"""The cyclic ring Z_q[x]/(x^n-1) (POLYMUL_FLAG_CYCLIC) on every path
against the CPU oracle's cyclic definition: the NTT path with moduli that
have an n-th but no 2n-th root of unity, 64-bit words, the auxiliary-prime
route, the tensor path, the large-degree kernels, and every autotuner
candidate."""
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


def _odd_cofactor_primes(rng, count, bits, n):
    """Primes q = 1 + j n with j odd (so q = 1 mod n but not mod 2n: the
    cyclic transform exists, the negacyclic one does not)."""
    out = []
    while len(out) < count:
        lo, hi = (1 << (bits - 1)) // n + 1, ((1 << bits) - 2) // n
        j = int(rng.integers(lo, hi + 1)) | 1
        q = 1 + j * n
        if j <= hi and q < (1 << bits) and wl.is_prime(q) and q not in out:
            out.append(q)
    return out


def _case(seed, batch, q_list, n, dtype):
    rng = np.random.default_rng(seed)
    return wl.uniform_coeffs(rng, batch, q_list, n, dtype), wl.uniform_coeffs(rng, batch, q_list, n, dtype)


@pytest.mark.parametrize("logn", [4, 6, 8, 9, 10, 11, 12, 13, 14])
def test_cyclic_ntt_u32(pm, logn):
    n = 1 << logn
    rng = np.random.default_rng(500 + logn)
    q_list = _odd_cofactor_primes(rng, 2, 30, n)
    a, b = _case(logn, {16: 21, 64: 13, 256: 9}.get(n, 3), q_list, n, np.uint32)
    with pm.Plan(n, q_list, flags=pm.FLAG_CYCLIC) as plan:
        info = plan.info
        assert info["path"] == pm.PATH_NTT and info["cyclic"] == 1 and info["aux_primes"] == 0
        got = run_plan_batch(plan, a, b)
    assert_equal_residues(got, native.polymul_batch(a, b, q_list, cyclic=True), "cyclic n=%d" % n)


@pytest.mark.parametrize("logn", [4, 10, 12])
def test_cyclic_ntt_u64(pm, logn):
    n = 1 << logn
    rng = np.random.default_rng(600 + logn)
    q_list = _odd_cofactor_primes(rng, 2, 59, n)
    a, b = _case(logn + 1, 3, q_list, n, np.uint64)
    a[0, 0, :] = q_list[0] - 1  # extremes
    b[0, 0, :] = q_list[0] - 1
    with pm.Plan(n, q_list, flags=pm.FLAG_CYCLIC) as plan:
        assert plan.elem_bytes == 8
        got = run_plan_batch(plan, a, b)
    assert_equal_residues(got, native.polymul_batch(a, b, q_list, cyclic=True), "cyclic u64 n=%d" % n)
    # all-(q-1) squared in x^n - 1: every coefficient is n mod q
    assert np.all(got[0, 0].astype(object) == n % q_list[0])


def test_cyclic_small_ntt_modes(pm):
    """12289 at n = 1024 (q = 1 mod 2n as well) and 65537 at 2^14: the
    unreduced small-modulus mode with cyclic tables."""
    for n, q in ((1024, 12289), (16384, 65537)):
        a, b = _case(n, 3, [q], n, np.uint32)
        with pm.Plan(n, [q], flags=pm.FLAG_CYCLIC) as plan:
            assert plan.info["ntt_mode"] == 2
            got = run_plan_batch(plan, a, b)
        assert_equal_residues(got, native.polymul_batch(a, b, [q], cyclic=True), "cyclic q=%d" % q)


@pytest.mark.parametrize("n,q", [(256, 3331), (256, 259), (512, 1000)])
def test_cyclic_auxiliary_prime(pm, n, q):
    """Moduli without an n-th root of unity (3331 at n = 256) or not prime
    (259 = 7 * 37, 1000) go through one 31-bit auxiliary prime with cyclic
    tables (the route needs 2 n floor(q/2)^2 < 2^31)."""
    assert (q - 1) % n != 0 or not wl.is_prime(q)
    a, b = _case(n + q, 5, [q], n, np.uint32)
    with pm.Plan(n, [q], path=pm.PATH_NTT, flags=pm.FLAG_CYCLIC) as plan:
        assert plan.info["aux_primes"] == 1
        got = run_plan_batch(plan, a, b)
    assert_equal_residues(got, native.polymul_batch(a, b, [q], cyclic=True), "cyclic aux n=%d q=%d" % (n, q))


@pytest.mark.parametrize("n,bits", [(1024, 14), (1024, 23), (1024, 30), (2048, 14), (2048, 20)])
def test_cyclic_tensor_path(pm, n, bits):
    rng = np.random.default_rng(700 + bits)
    q_list = [12289] if bits == 14 else wl.draw_primes(rng, 2, bits, bits, 1)
    a, b = _case(n * bits, 5, q_list, n, np.uint32)
    a[0, 0, :] = q_list[0] - 1
    b[0, 0, :] = q_list[0] // 2 + 1  # the most negative centred value
    with pm.Plan(n, q_list, path=pm.PATH_TENSOR, flags=pm.FLAG_CYCLIC) as plan:
        assert plan.info["path"] == pm.PATH_TENSOR and plan.info["cyclic"] == 1
        got = run_plan_batch(plan, a, b)
    assert_equal_residues(got, native.polymul_batch(a, b, q_list, cyclic=True), "cyclic tensor n=%d" % n)


@pytest.mark.parametrize("n,bits,elem", [(32768, 30, 4), (65536, 30, 4), (16384, 59, 8)])
def test_cyclic_large_degrees(pm, n, bits, elem):
    """Thread-block cluster kernels with cyclic tables; sampled coefficients
    against the oracle."""
    rng = np.random.default_rng(800 + bits)
    q_list = _odd_cofactor_primes(rng, 1, bits, n)
    dt = np.uint32 if elem == 4 else np.uint64
    a, b = _case(n + bits, 2, q_list, n, dt)
    with pm.Plan(n, q_list, flags=pm.FLAG_CYCLIC) as plan:
        got = run_plan_batch(plan, a, b)
    js = sorted(set([0, 1, n // 2, n - 1] + [int(x) for x in rng.integers(0, n, 20)]))
    for p in range(2):
        want = native.coeffs(a[p, 0], b[p, 0], q_list[0], js, cyclic=True)
        assert np.array_equal(got[p, 0, js].astype(np.uint64), want), p


@pytest.mark.parametrize("n,bits", [(1024, 14), (4096, 29), (16384, 30)])
def test_cyclic_every_candidate(pm, n, bits):
    rng = np.random.default_rng(900 + n)
    q_list = [12289] if bits == 14 else _odd_cofactor_primes(rng, 2, bits, n)
    a, b = _case(n + 7, 3, q_list, n, np.uint32)
    want = native.polymul_batch(a, b, q_list, cyclic=True)
    with pm.Plan(n, q_list, flags=pm.FLAG_CYCLIC) as plan:
        for i in range(plan.info["candidates"]):
            info = plan.select(i)
            assert_equal_residues(run_plan_batch(plan, a, b), want,
                                  "candidate %d (path %d, radix %d)" % (i, info["path"], info["radix_bits"]))


def test_cyclic_and_negacyclic_plans_differ(pm):
    n, q = 1024, 12289
    a, b = _case(3, 2, [q], n, np.uint32)
    with pm.Plan(n, [q], flags=pm.FLAG_CYCLIC) as pc, pm.Plan(n, [q]) as pn:
        assert pc.info["cyclic"] == 1 and pn.info["cyclic"] == 0
        gc, gn = run_plan_batch(pc, a, b), run_plan_batch(pn, a, b)
    assert not np.array_equal(gc, gn)
    assert_equal_residues(gn, native.polymul_batch(a, b, [q]), "negacyclic")


def test_cyclic_moduli_without_ntt_route(pm):
    """64-bit moduli without an n-th root of unity have no NTT route; at
    n = 2^15 the tensor path's 64-bit digit kernel serves them (sampled
    coefficients against the oracle), and with a ternary b (no one-digit
    form for 64-bit words, no RNS base at that degree) nothing does."""
    q = (1 << 61) - 1  # prime, q - 1 = 2 * odd: no root of order 2^15
    with pytest.raises(pm.PolymulError) as ei:
        pm.Plan(1024, [q], path=pm.PATH_NTT, flags=pm.FLAG_CYCLIC)
    assert ei.value.code == pm.POLYMUL_ENOTSUP
    with pytest.raises(pm.PolymulError) as ei:
        pm.Plan(32768, [q], flags=pm.FLAG_CYCLIC | pm.FLAG_TERNARY_B)
    assert ei.value.code == pm.POLYMUL_ENOTSUP
    n = 32768
    a, b = _case(11, 1, [q], n, np.uint64)
    with pm.Plan(n, [q], flags=pm.FLAG_CYCLIC) as plan:
        assert plan.info["path"] == pm.PATH_TENSOR and plan.info["tensor_kernel"] == 6
        got = run_plan_batch(plan, a, b)
        pm.polymul_plan_status(plan.handle)
    js = [0, 1, 1023, 1024, 4097, n // 2, n - 2, n - 1]
    assert np.array_equal(got[0, 0, js].astype(np.uint64), native.coeffs(a[0, 0], b[0, 0], q, js, cyclic=True))

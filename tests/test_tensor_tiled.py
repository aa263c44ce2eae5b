"""Path (b) at every degree 2^6 .. 2^14 (k_toeplitz_tiled: output groups
and K chunks, Sec. 2.6) against the CPU oracle: whole products where the
oracle is quick, sampled coefficients at the largest degrees, every digit
count 1 .. 5, both rings, extreme operands whose partial sums reach the
exactness bound, batches that are not a multiple of the grid, the small-ring
and RNS workloads on the tensor path, the tiled kernel beside the
whole-product one at n = 1024 and 2048 (first at 2048, where it serves two
blocks from one A slice), ternary b, and moduli at the digit-count
boundaries.  The drained form (8-bit digits at every degree, exact per K
chunk of at most 1024) likewise, with its own exactness boundary, and where
the undrained form has no digit count (a 31-bit modulus at 2^14)."""
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


def _tensor_plan(pm, n, q_list, cyclic=False):
    plan = pm.Plan(n, q_list, path=pm.PATH_TENSOR, flags=pm.FLAG_CYCLIC if cyclic else 0)
    info = plan.info
    assert info["path"] == pm.PATH_TENSOR
    return plan


def _digit_width(n):
    # the widest w with n 2^(2w-2) <= 2^24 and w <= 8
    logn = n.bit_length() - 1
    return min(8, (24 - logn) // 2 + 1)


def _select(plan, code):
    """Select the plan's candidate whose tensor kernel has the given code (1
    whole product, 2 tiled, 3 RNS, 4 tiled drained); returns its info."""
    codes = []
    for i in range(plan.info["candidates"]):
        info = plan.select(i)
        codes.append(info["tensor_kernel"])
        if info["tensor_kernel"] == code:
            return info
    raise AssertionError("no candidate with tensor kernel %d (have %s)" % (code, codes))


def _check_sampled(got, a, b, q_list, cyclic, rng, count=24):
    n = a.shape[-1]
    for p in range(a.shape[0]):
        for jq, q in enumerate(q_list):
            js = sorted(set([0, 1, 7, 8, n // 2, n - 9, n - 8, n - 1] +
                            [int(x) for x in rng.integers(0, n, count)]))
            want = native.coeffs(a[p, jq], b[p, jq], q, js, cyclic=cyclic)
            assert np.array_equal(got[p, jq, js].astype(np.uint64), want), (p, jq)


@pytest.mark.parametrize("n", [64, 128, 256, 512, 4096])
@pytest.mark.parametrize("bits", [14, 22, 30])
def test_tiled_against_oracle(pm, n, bits):
    rng = np.random.default_rng(n * 100 + bits)
    q_list = [12289] if bits == 14 else wl.draw_primes(rng, 2, bits, bits, 1)
    batch = {64: 41, 128: 23, 256: 19, 512: 9, 4096: 3}[n]
    a = wl.uniform_coeffs(rng, batch, q_list, n, np.uint32)
    b = wl.uniform_coeffs(rng, batch, q_list, n, np.uint32)
    with _tensor_plan(pm, n, q_list) as plan:
        info = _select(plan, 2)
        assert info["tensor_groups"] >= 1 and info["digit_bits"] == _digit_width(n)
        got = run_plan_batch(plan, a, b)
    assert_equal_residues(got, native.polymul_batch(a, b, q_list), "tiled n=%d bits=%d" % (n, bits))


@pytest.mark.parametrize("n,bits", [(8192, 14), (8192, 30), (16384, 14), (16384, 29)])
def test_tiled_large_degrees_sampled(pm, n, bits):
    rng = np.random.default_rng(n + bits)
    q_list = [12289] if bits == 14 else wl.draw_primes(rng, 1, bits, bits, 1)
    a = wl.uniform_coeffs(rng, 2, q_list, n, np.uint32)
    b = wl.uniform_coeffs(rng, 2, q_list, n, np.uint32)
    with _tensor_plan(pm, n, q_list) as plan:
        assert plan.info["tensor_groups"] > 1  # several output groups per product
        got = run_plan_batch(plan, a, b)
    _check_sampled(got, a, b, q_list, False, rng)


@pytest.mark.parametrize("n,bits", [(64, 14), (256, 22), (4096, 30), (8192, 20)])
def test_tiled_cyclic(pm, n, bits):
    rng = np.random.default_rng(7 * n + bits)
    q_list = [12289] if bits == 14 else wl.draw_primes(rng, 1, bits, bits, 1)
    a = wl.uniform_coeffs(rng, 3, q_list, n, np.uint32)
    b = wl.uniform_coeffs(rng, 3, q_list, n, np.uint32)
    with _tensor_plan(pm, n, q_list, cyclic=True) as plan:
        assert plan.info["cyclic"] == 1
        got = run_plan_batch(plan, a, b)
    if n <= 4096:
        assert_equal_residues(got, native.polymul_batch(a, b, q_list, cyclic=True), "tiled cyclic n=%d" % n)
    else:
        _check_sampled(got, a, b, q_list, True, rng)


@pytest.mark.parametrize("n,q,digits", [(256, 251, 1), (256, 3329, 2), (1024, 1000003, 3), (4096, 65537, 3),
                                        (2048, 536870909, 5)])
def test_tiled_digit_counts(pm, n, q, digits):
    """Every instantiated digit count (1 .. 5)."""
    rng = np.random.default_rng(q % 1000 + n)
    a = wl.uniform_coeffs(rng, 5, [q], n, np.uint32)
    b = wl.uniform_coeffs(rng, 5, [q], n, np.uint32)
    with pm.Plan(n, [q], path=pm.PATH_TENSOR) as plan:
        # n = 1024, 2048 have a whole-product kernel too, n >= 2048 the
        # drained one; use the tiled one
        info = _select(plan, 2)
        assert info["digits"] == digits, info
        got = run_plan_batch(plan, a, b)
    assert_equal_residues(got, native.polymul_batch(a, b, [q]), "digits=%d n=%d" % (digits, n))


@pytest.mark.parametrize("n,kernel", [(64, 2), (256, 2), (4096, 2), (8192, 2), (4096, 4), (16384, 4)])
def test_tiled_exactness_boundary(pm, n, kernel):
    """The low digits of every coefficient at -2^(w-1): each of their
    digit products is 2^(2w-2), so the output coefficient without wrap-around
    sums n of them, n 2^(2w-2) = 2^24 at n = 4096 -- the edge of exact fp32
    integers -- and the other sums mix signs.  Moduli at the top of what
    five digits cover (31 bits up to 2^12; at 2^13 the largest prime whose
    half five 6-bit digits reach, 1056698273).  The drained
    kernel (8-bit digits) reaches 1024 x 2^14 = 2^24 within each K chunk;
    four digits cover 31-bit moduli at every degree."""
    w = 8 if kernel == 4 else _digit_width(n)
    q = 2147483629 if n <= 4096 or kernel == 4 else 1056698273
    assert wl.is_prime(q)
    digits = -(1 << (w - 1))
    low = 3 if w == 8 else 4  # as many low digits at their minimum as stay inside (-q/2, q/2]
    x = sum(digits << (w * s) for s in range(low))
    v = q + x
    assert 0 < v < q
    a = np.full((2, 1, n), v, np.uint32)
    b = np.full((2, 1, n), v, np.uint32)
    a[1, 0] = q - 1
    b[1, 0, ::3] = q // 2 + 1  # the most negative centred value
    with pm.Plan(n, [q], path=pm.PATH_TENSOR) as plan:
        assert _select(plan, kernel)["digit_bits"] == w
        got = run_plan_batch(plan, a, b)
    js = sorted(set([0, 1, n // 2, n - 2, n - 1] + list(range(0, n, max(1, n // 64)))))
    for p in range(2):
        want = native.coeffs(a[p, 0], b[p, 0], q, js)
        assert np.array_equal(got[p, 0, js].astype(np.uint64), want), p


def test_tiled_ragged_units(pm):
    """More units than resident CTAs, not a multiple of the grid, with
    several output groups per product and several primes."""
    n = 8192
    rng = np.random.default_rng(81)
    q_list = wl.draw_primes(rng, 3, 28, 30, 1)
    a = wl.uniform_coeffs(rng, 131, q_list, n, np.uint32)
    b = wl.uniform_coeffs(rng, 131, q_list, n, np.uint32)
    with _tensor_plan(pm, n, q_list) as plan:
        info = plan.info
        assert 131 * 3 * info["tensor_groups"] > info["grid"]
        got = run_plan_batch(plan, a, b)
        got2 = run_plan_batch(plan, a[:5], b[:5])  # the counters reset between launches
    rs = np.random.default_rng(82)
    for p in [0, 1, 64, 129, 130]:
        js = sorted(int(x) for x in rs.integers(0, n, 16))
        for jq, q in enumerate(q_list):
            want = native.coeffs(a[p, jq], b[p, jq], q, js)
            assert np.array_equal(got[p, jq, js].astype(np.uint64), want), (p, jq)
    assert np.array_equal(got2, got[:5])


def test_ring_small_on_tensor_path(pm):
    """The n = 256, q = 3329 workload (no 512-th root of unity mod 3329) on
    the tensor path, whole batch against the oracle."""
    w = wl.ring_small()
    with _tensor_plan(pm, w.n, w.q_list) as plan:
        got = run_plan_batch(plan, w.a, w.b)
    assert_equal_residues(got, native.polymul_batch(w.a, w.b, w.q_list), "tensor " + w.name)


def test_rns_4096_on_tensor_path(pm):
    """The n = 4096 RNS workload (8 primes of 30 bits, ternary b) on the
    tensor path: every product's every prime on sampled coefficients, and
    whole products for a few."""
    w = wl.rns_4096()
    with _tensor_plan(pm, w.n, w.q_list) as plan:
        # four 8-bit digits (drained K chunks) rather than five of 7 bits
        assert (plan.info["tensor_kernel"], plan.info["digits"], plan.info["digit_bits"]) == (4, 4, 8)
        got = run_plan_batch(plan, w.a, w.b)
    for p in (0, 255):
        assert_equal_residues(got[p:p + 1], native.polymul_batch(w.a[p:p + 1], w.b[p:p + 1], w.q_list),
                              "product %d" % p)
    rng = np.random.default_rng(43)
    for p in range(0, 256, 17):
        js = sorted(int(x) for x in rng.integers(0, w.n, 6))
        for jq, q in enumerate(w.q_list):
            want = native.coeffs(w.a[p, jq], w.b[p, jq], q, js)
            assert np.array_equal(got[p, jq, js].astype(np.uint64), want), (p, jq)


@pytest.mark.parametrize("n", [1024, 2048])
def test_tiled_candidate_matches_whole_product_kernel(pm, n):
    """At n = 1024 the whole-product kernel first, then the tiled and RNS
    ones; at 2048 the tiled one first (two blocks from one A slice), and the
    drained one too (7-bit digits there, as many 8-bit ones): every digit
    kernel gives the same coefficients, and the oracle's."""
    rng = np.random.default_rng(n)
    q_list = [12289, 7681]
    a = wl.uniform_coeffs(rng, 77, q_list, n, np.uint32)
    b = wl.uniform_coeffs(rng, 77, q_list, n, np.uint32)
    with pm.Plan(n, q_list, path=pm.PATH_TENSOR) as plan:
        info = plan.info
        codes = [plan.select(i)["tensor_kernel"] for i in range(info["candidates"])]
        assert codes == ([2, 1, 4, 5, 3] if n == 2048 else [1, 2, 5, 3]), codes
        outs = {}
        for code in codes:
            if code != 3:
                _select(plan, code)
                outs[code] = run_plan_batch(plan, a, b)
    for code in outs:
        assert np.array_equal(outs[code], outs[2]), code
    assert_equal_residues(outs[2], native.polymul_batch(a, b, q_list), "tiled n=%d" % n)


def test_tensor_path_limits(pm):
    """Outside the tensor path's shapes creation fails with ENOTSUP when the
    path is forced: 32-bit words above 2^14; a 59-bit modulus at 2^13 with
    a ternary b (the 64-bit digit kernel has no one-digit A side, and the
    RNS kernel's moduli there stay below 92)."""
    for n, q, flags in ((32768, 12289, 0), (8192, (1 << 59) - 55, pm.FLAG_TERNARY_B)):
        with pytest.raises(pm.PolymulError) as ei:
            pm.Plan(n, [q], path=pm.PATH_TENSOR, flags=flags)
        assert ei.value.code == pm.POLYMUL_ENOTSUP, (n, q)


def test_rns_takes_32_bit_moduli_above_2_31(pm):
    """A 32-bit modulus at or above 2^31 has no digit kernel (signed 32-bit
    centring) and no NTT route (32-bit words hold moduli below 2^31); the
    residue-number-system kernel serves it."""
    q = 2147483659  # prime, between 2^31 and 2^32
    assert wl.is_prime(q)
    n = 1024
    rng = np.random.default_rng(31)
    a = wl.uniform_coeffs(rng, 4, [q], n, np.uint32)
    b = wl.uniform_coeffs(rng, 4, [q], n, np.uint32)
    with pm.Plan(n, [q]) as plan:
        info = plan.info
        assert info["path"] == pm.PATH_TENSOR and info["rns_moduli"] > 0 and plan.elem_bytes == 4
        got = run_plan_batch(plan, a, b)
    assert_equal_residues(got, native.polymul_batch(a, b, [q]), "q > 2^31 on the RNS kernel")


# ---- ternary b (POLYMUL_FLAG_TERNARY_B): b as one digit on the A side ----

@pytest.mark.parametrize("n,bits,cyclic", [(64, 14, False), (1024, 30, False), (2048, 14, True), (4096, 29, False),
                                           (512, 30, True)])
def test_ternary_b_against_oracle(pm, n, bits, cyclic):
    rng = np.random.default_rng(3 * n + bits)
    q_list = [12289] if bits == 14 else wl.draw_primes(rng, 2, bits, bits, 1)
    a = wl.uniform_coeffs(rng, 7, q_list, n, np.uint32)
    b = wl.ternary_coeffs(rng, 7, q_list, n, np.uint32)
    flags = pm.FLAG_TERNARY_B | (pm.FLAG_CYCLIC if cyclic else 0)
    with pm.Plan(n, q_list, path=pm.PATH_TENSOR, flags=flags) as plan:
        info = plan.info
        assert info["tensor_groups"] >= 1  # the tiled kernel, also at n = 1024 and 2048
        got = run_plan_batch(plan, a, b)
        pm.polymul_plan_status(plan.handle)
    assert_equal_residues(got, native.polymul_batch(a, b, q_list, cyclic=cyclic), "ternary n=%d" % n)


def test_ternary_b_large_degree_sampled(pm):
    n = 16384
    rng = np.random.default_rng(161)
    q_list = wl.draw_primes(rng, 1, 30, 30, 1)
    a = wl.uniform_coeffs(rng, 3, q_list, n, np.uint32)
    b = wl.ternary_coeffs(rng, 3, q_list, n, np.uint32)
    with pm.Plan(n, q_list, path=pm.PATH_TENSOR, flags=pm.FLAG_TERNARY_B) as plan:
        got = run_plan_batch(plan, a, b)
        pm.polymul_plan_status(plan.handle)
    _check_sampled(got, a, b, q_list, False, rng)


def test_rns_4096_ternary_on_tensor_path(pm):
    """The n = 4096 RNS workload's b is ternary: with the flag the tensor path
    gives the same results as without it (five digits of b) and as the
    oracle."""
    w = wl.rns_4096(batch=24)
    with _tensor_plan(pm, w.n, w.q_list) as plain:
        want = run_plan_batch(plain, w.a, w.b)
    with pm.Plan(w.n, w.q_list, path=pm.PATH_TENSOR, flags=pm.FLAG_TERNARY_B) as plan:
        got = run_plan_batch(plan, w.a, w.b)
        pm.polymul_plan_status(plan.handle)
    assert np.array_equal(got, want)
    assert_equal_residues(got[:2], native.polymul_batch(w.a[:2], w.b[:2], w.q_list), "ternary rns_4096")


def test_ternary_b_one_digit_values(pm):
    """Any b whose centred coefficients fit one digit is exact under the
    flag, not only {-1, 0, 1}: here |b| < 2^(w-1) = 128 at n = 1024."""
    n, q = 1024, 12289
    rng = np.random.default_rng(5)
    a = wl.uniform_coeffs(rng, 4, [q], n, np.uint32)
    bs = rng.integers(-127, 128, size=(4, 1, n))
    b = np.where(bs < 0, bs + q, bs).astype(np.uint32)
    with pm.Plan(n, [q], path=pm.PATH_TENSOR, flags=pm.FLAG_TERNARY_B) as plan:
        got = run_plan_batch(plan, a, b)
        pm.polymul_plan_status(plan.handle)
    assert_equal_residues(got, native.polymul_batch(a, b, [q]), "one-digit b")


def test_ternary_b_domain_error_is_reported(pm):
    """A b coefficient that does not fit one digit under the flag: the
    launch's results are invalid and the status call returns EDOMAIN; the
    plan then works again."""
    n, q = 2048, 12289
    rng = np.random.default_rng(6)
    a = wl.uniform_coeffs(rng, 3, [q], n, np.uint32)
    bad = wl.ternary_coeffs(rng, 3, [q], n, np.uint32)
    bad[1, 0, 77] = 5000
    good = wl.ternary_coeffs(rng, 3, [q], n, np.uint32)
    with pm.Plan(n, [q], path=pm.PATH_TENSOR, flags=pm.FLAG_TERNARY_B) as plan:
        run_plan_batch(plan, a, bad)
        with pytest.raises(pm.PolymulError) as ei:
            pm.polymul_plan_status(plan.handle)
        assert ei.value.code == pm.POLYMUL_EDOMAIN
        pm.polymul_plan_status(plan.handle)  # cleared
        got = run_plan_batch(plan, a, good)
        pm.polymul_plan_status(plan.handle)
    assert_equal_residues(got, native.polymul_batch(a, good, [q]), "after the domain error")


def test_ternary_flag_ignored_by_ntt_path(pm):
    n, q = 1024, 12289
    rng = np.random.default_rng(8)
    a = wl.uniform_coeffs(rng, 5, [q], n, np.uint32)
    b = wl.uniform_coeffs(rng, 5, [q], n, np.uint32)  # not ternary
    with pm.Plan(n, [q], path=pm.PATH_NTT, flags=pm.FLAG_TERNARY_B) as plan:
        got = run_plan_batch(plan, a, b)
        pm.polymul_plan_status(plan.handle)
    assert_equal_residues(got, native.polymul_batch(a, b, [q]), "ntt with the flag")


@pytest.mark.parametrize("n,q,digits", [(1024, 65521, 3), (256, 65519, 3), (2048, 16381, 3), (4096, 16381, 3),
                                        (8192, 1073479681, 0)])
def test_digit_capacity_boundary(pm, n, q, digits):
    """Moduli just below a digit-count boundary: L balanced w-bit digits in
    [-2^(w-1), 2^(w-1)) reach (2^(w-1) - 1)(2^(wL) - 1)/(2^w - 1), a little
    less than (2^(wL) - 1)/2, so floor(q/2) of these moduli needs one digit
    more than the naive bound says (digits == 0: more than five digits of
    the undrained kernels; the drained kernel's four 8-bit digits serve it,
    and the residue-number-system kernel too).  Every coefficient at the
    positive and negative extremes of the centred range, on each digit
    kernel the plan holds."""
    assert wl.is_prime(q)
    rng = np.random.default_rng(q % 997)
    a = wl.uniform_coeffs(rng, 3, [q], n, np.uint32)
    b = wl.uniform_coeffs(rng, 3, [q], n, np.uint32)
    a[0] = q // 2          # +floor(q/2)
    b[0] = q // 2
    a[1] = q // 2 + 1      # -floor(q/2) (q odd)
    b[1, 0, ::2] = q // 2
    with pm.Plan(n, [q], path=pm.PATH_TENSOR) as plan:
        codes = [plan.select(i)["tensor_kernel"] for i in range(plan.info["candidates"])]
        if digits:
            assert _select(plan, next(c for c in codes if c in (1, 2)))["digits"] == digits
        else:
            assert codes == [4, 5, 3], codes
        gots = []
        for code in codes:
            if code != 3 or not digits:
                _select(plan, code)
                gots.append((code, run_plan_batch(plan, a, b)))
    for code, got in gots:
        if n <= 4096:
            assert_equal_residues(got, native.polymul_batch(a, b, [q]), "boundary n=%d q=%d kernel %d" % (n, q, code))
        else:
            _check_sampled(got, a, b, [q], False, rng)


# ---- the drained tiled kernel: 8-bit digits at every degree ----

@pytest.mark.parametrize("n,bits,cyclic", [(2048, 22, False), (2048, 31, True), (4096, 30, False), (4096, 31, False),
                                           (4096, 26, True)])
def test_drained_against_oracle(pm, n, bits, cyclic):
    rng = np.random.default_rng(11 * n + bits)
    q_list = wl.draw_primes(rng, 2, bits, bits, 1)
    a = wl.uniform_coeffs(rng, 5, q_list, n, np.uint32)
    b = wl.uniform_coeffs(rng, 5, q_list, n, np.uint32)
    with _tensor_plan(pm, n, q_list, cyclic=cyclic) as plan:
        info = _select(plan, 4)
        assert info["digit_bits"] == 8 and info["digits"] <= 4
        got = run_plan_batch(plan, a, b)
        pm.polymul_plan_status(plan.handle)
    assert_equal_residues(got, native.polymul_batch(a, b, q_list, cyclic=cyclic), "drained n=%d bits=%d" % (n, bits))


@pytest.mark.parametrize("n,bits,ternary", [(8192, 30, False), (16384, 31, False), (16384, 31, True),
                                            (8192, 20, True)])
def test_drained_large_degrees_sampled(pm, n, bits, ternary):
    """Up to 16 K chunks drained per unit of work; a 31-bit modulus at 2^14
    has no undrained digit kernel (six 6-bit digits)."""
    rng = np.random.default_rng(n + 3 * bits + ternary)
    q_list = wl.draw_primes(rng, 2, bits, bits, 1)
    a = wl.uniform_coeffs(rng, 3, q_list, n, np.uint32)
    b = (wl.ternary_coeffs if ternary else wl.uniform_coeffs)(rng, 3, q_list, n, np.uint32)
    with pm.Plan(n, q_list, path=pm.PATH_TENSOR, flags=pm.FLAG_TERNARY_B if ternary else 0) as plan:
        info = _select(plan, 4)
        assert info["tensor_groups"] >= 1
        got = run_plan_batch(plan, a, b)
        pm.polymul_plan_status(plan.handle)
    _check_sampled(got, a, b, q_list, False, rng)


def test_drained_matches_undrained_on_many_units(pm):
    """Both digit kernels on a batch with more units of work than resident
    CTAs: the same coefficients, bit for bit, and the oracle's on a sample."""
    n = 4096
    rng = np.random.default_rng(4099)
    q_list = wl.draw_primes(rng, 3, 29, 30, 13)
    a = wl.uniform_coeffs(rng, 97, q_list, n, np.uint32)
    b = wl.uniform_coeffs(rng, 97, q_list, n, np.uint32)
    with _tensor_plan(pm, n, q_list) as plan:
        assert plan.info["tensor_kernel"] == 4  # first: four 8-bit digits instead of five 7-bit ones
        assert 97 * 3 * plan.info["tensor_groups"] > plan.info["grid"]
        drained = run_plan_batch(plan, a, b)
        _select(plan, 2)
        undrained = run_plan_batch(plan, a, b)
    assert np.array_equal(drained, undrained)
    _check_sampled(drained[:4], a[:4], b[:4], q_list, False, rng, count=8)


# ---- the drained kernel as a warp-specialised pipeline (one CTA per SM) ----

@pytest.mark.parametrize("n,bits,ternary,cyclic", [(256, 13, False, False), (1024, 14, False, True), (2048, 30, False, False),
                                                   (4096, 30, False, False), (4096, 30, True, False),
                                                   (4096, 31, False, True), (2048, 22, True, True)])
def test_pipelined_against_oracle(pm, n, bits, ternary, cyclic):
    rng = np.random.default_rng(13 * n + bits + ternary)
    q_list = [12289] if bits == 14 else wl.draw_primes(rng, 2, bits, bits, 1)
    batch = 300 if n <= 1024 else 7  # more units than CTAs: several per CTA, walked statically
    a = wl.uniform_coeffs(rng, batch, q_list, n, np.uint32)
    b = (wl.ternary_coeffs if ternary else wl.uniform_coeffs)(rng, batch, q_list, n, np.uint32)
    flags = (pm.FLAG_TERNARY_B if ternary else 0) | (pm.FLAG_CYCLIC if cyclic else 0)
    with pm.Plan(n, q_list, path=pm.PATH_TENSOR, flags=flags) as plan:
        info = _select(plan, 5)
        assert info["digit_bits"] == 8 and info["block"] == 512
        got = run_plan_batch(plan, a, b)
        pm.polymul_plan_status(plan.handle)
    if n <= 1024:
        assert_equal_residues(got, native.polymul_batch(a, b, q_list, cyclic=cyclic), "pipelined n=%d" % n)
    else:
        assert_equal_residues(got[:3], native.polymul_batch(a[:3], b[:3], q_list, cyclic=cyclic), "pipelined n=%d" % n)


@pytest.mark.parametrize("n,bits,ternary", [(8192, 30, False), (16384, 31, True), (16384, 30, False)])
def test_pipelined_large_degrees_sampled(pm, n, bits, ternary):
    rng = np.random.default_rng(n + 7 * bits + ternary)
    q_list = wl.draw_primes(rng, 2, bits, bits, 1)
    a = wl.uniform_coeffs(rng, 3, q_list, n, np.uint32)
    b = (wl.ternary_coeffs if ternary else wl.uniform_coeffs)(rng, 3, q_list, n, np.uint32)
    with pm.Plan(n, q_list, path=pm.PATH_TENSOR, flags=pm.FLAG_TERNARY_B if ternary else 0) as plan:
        _select(plan, 5)
        got = run_plan_batch(plan, a, b)
        pm.polymul_plan_status(plan.handle)
    _check_sampled(got, a, b, q_list, False, rng)


def test_pipelined_matches_drained_and_relaunches(pm):
    """Fewer units than SMs, then many: the pipeline's static walk, its
    mbarrier phases across launches and the hand-off between its drainer
    sets give the drained kernel's coefficients bit for bit."""
    n = 4096
    rng = np.random.default_rng(4097)
    q_list = wl.draw_primes(rng, 3, 29, 30, 13)
    for batch in (5, 97):
        a = wl.uniform_coeffs(rng, batch, q_list, n, np.uint32)
        b = wl.uniform_coeffs(rng, batch, q_list, n, np.uint32)
        with _tensor_plan(pm, n, q_list) as plan:
            _select(plan, 4)
            want = run_plan_batch(plan, a, b)
            _select(plan, 5)
            got = run_plan_batch(plan, a, b)
            again = run_plan_batch(plan, a, b)
            pm.polymul_plan_status(plan.handle)
        assert np.array_equal(got, want) and np.array_equal(again, want), batch
    _check_sampled(want[:2], a[:2], b[:2], q_list, False, rng, count=8)


def test_pipelined_domain_error_is_reported(pm):
    """A b coefficient outside one digit under the ternary flag, on the
    pipelined kernel: EDOMAIN, then exact again."""
    n, q = 4096, 1073479681
    rng = np.random.default_rng(61)
    a = wl.uniform_coeffs(rng, 3, [q], n, np.uint32)
    bad = wl.ternary_coeffs(rng, 3, [q], n, np.uint32)
    bad[2, 0, 4000] = 1000
    good = wl.ternary_coeffs(rng, 3, [q], n, np.uint32)
    with pm.Plan(n, [q], path=pm.PATH_TENSOR, flags=pm.FLAG_TERNARY_B) as plan:
        _select(plan, 5)
        run_plan_batch(plan, a, bad)
        with pytest.raises(pm.PolymulError) as ei:
            pm.polymul_plan_status(plan.handle)
        assert ei.value.code == pm.POLYMUL_EDOMAIN
        got = run_plan_batch(plan, a, good)
        pm.polymul_plan_status(plan.handle)
    assert_equal_residues(got[:1], native.polymul_batch(a[:1], good[:1], [q]), "after the domain error")

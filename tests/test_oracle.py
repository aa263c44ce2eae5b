"""Pins for the CPU oracle: each check comes from the paper or from
mathematics, never from the oracle itself and never from the CUDA path.

* Example 1 (Sec. 2.2, Eq. equ-example-mul), symbolic, from tests/golden.
* the x^n = -1 sign rule on monomials;
* identity, multiplication by x = negacyclic rotation;
* commutativity, distributivity, associativity;
* brute force on tiny rings against numpy's polynomial long division;
* evaluation at all roots of x^n + 1 for NTT-friendly q (the ring is then
  a product of n fields, so this check is complete);
* Kronecker substitution with CPython big-int multiplication (a different
  exact algorithm) against the C oracle at mid sizes;
* Sec. 2.5 divide identity, Sec. 4 Karatsuba identity, Sec. 2.4/2.6 RNS.
A test plants plausible mistakes in copies of the oracle and checks that
some pin catches each one.  The cyclic ring x^n - 1 (named in Sec. 2.1) has
its own pins of the same kinds at the end, including numpy's FFT splitting
the full product into both rings.
"""
import os
import math
import random

import numpy as np
import pytest

from oracle import native
from oracle import schoolbook as sb

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _rand_poly(rng, n, q):
    return [rng.randrange(q) for _ in range(n)]


# ---------------------------------------------------------------- Example 1
def _load_example1():
    sympy = pytest.importorskip("sympy")
    lines = [l.strip() for l in open(os.path.join(GOLDEN, "example1_n3.txt"))
             if l.strip() and not l.startswith("#")]
    i_m, i_r = lines.index("matrix"), lines.index("result")
    mat = [[sympy.sympify(t) for t in row.split()] for row in lines[i_m + 1:i_r]]
    res = [sympy.sympify(r) for r in lines[i_r + 1:]]
    a = sympy.symbols("a0 a1 a2")
    b = sympy.symbols("b0 b1 b2")
    return sympy, mat, res, list(a), list(b)


def test_example1_matrix():
    sympy, mat, res, a, b = _load_example1()
    t = sb.toeplitz_matrix(b)
    for i in range(3):
        for j in range(3):
            assert sympy.expand(t[i][j] - mat[i][j]) == 0


def test_example1_result_both_routes():
    sympy, mat, res, a, b = _load_example1()
    via_fold = sb.negacyclic_convolution(a, b)
    via_mat = sb.vec_mat(a, sb.toeplitz_matrix(b))
    for j in range(3):
        assert sympy.expand(via_fold[j] - res[j]) == 0
        assert sympy.expand(via_mat[j] - res[j]) == 0


def test_example1_numeric_mod_q():
    # the same expressions evaluated numerically, then mod q
    rng = random.Random(11)
    for q in (2, 3, 3329, 12289, (1 << 61) - 1):
        a = _rand_poly(rng, 3, q)
        b = _rand_poly(rng, 3, q)
        a0, a1, a2 = a
        b0, b1, b2 = b
        want = [(a0 * b0 - a1 * b2 - a2 * b1) % q,
                (a0 * b1 + a1 * b0 - a2 * b2) % q,
                (a0 * b2 + a1 * b1 + a2 * b0) % q]
        assert sb.negacyclic_mul(a, b, q) == want
        assert sb.matrix_form_mul(a, b, q) == want


# ---------------------------------------------------------------- ring laws
@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 8, 16, 32, 64])
def test_monomial_sign_rule(n):
    for i in range(n):
        for j in range(n):
            ei = [0] * n
            ej = [0] * n
            ei[i] = 1
            ej[j] = 1
            c = sb.negacyclic_convolution(ei, ej)
            want = [0] * n
            want[(i + j) % n] = -1 if i + j >= n else 1
            assert c == want, (n, i, j)
    q = 97
    ei = [0] * n
    ei[n - 1] = 1
    c = sb.negacyclic_mul(ei, ei, q)
    want = [0] * n
    want[(2 * n - 2) % n] = q - 1 if n > 1 else 1
    assert c == want


@pytest.mark.parametrize("n,q", [(1, 7), (8, 17), (16, 3329), (33, 1000), (64, (1 << 59) + 21)])
def test_identity_and_x_rotation(n, q):
    rng = random.Random(n * 7 + q)
    a = _rand_poly(rng, n, q)
    one = [1] + [0] * (n - 1)
    assert sb.negacyclic_mul(a, one, q) == a
    assert sb.negacyclic_mul(one, a, q) == a
    if n > 1:
        x = [0, 1] + [0] * (n - 2)
        rot = [(-a[n - 1]) % q] + a[: n - 1]
        assert sb.negacyclic_mul(x, a, q) == rot
        # x^n = -1: applying the rotation n times negates
        r = a
        for _ in range(n):
            r = sb.negacyclic_mul(x, r, q)
        assert r == [(-v) % q for v in a]


@pytest.mark.parametrize("n,q", [(4, 2), (8, 15), (16, 12289), (31, 65536), (64, 3329),
                                 (32, (1 << 62) - 57), (16, (1 << 64) - 59)])
def test_commutative_distributive_associative(n, q):
    rng = random.Random(n * 131 + q % 1000)
    for _ in range(3):
        a, b, c = (_rand_poly(rng, n, q) for _ in range(3))
        ab = sb.negacyclic_mul(a, b, q)
        assert ab == sb.negacyclic_mul(b, a, q)
        bc = [(x + y) % q for x, y in zip(b, c)]
        lhs = sb.negacyclic_mul(a, bc, q)
        rhs = [(x + y) % q for x, y in zip(ab, sb.negacyclic_mul(a, c, q))]
        assert lhs == rhs
        assert sb.negacyclic_mul(ab, c, q) == sb.negacyclic_mul(a, sb.negacyclic_mul(b, c, q), q)
        assert all(0 <= v < q for v in ab)


# ---------------------------------------------------------------- brute force
def _numpy_remainder(a, b, n, q):
    """Z[x] product and remainder by x^n+1 via numpy.polynomial (an
    independent library routine), exact for small integers."""
    from numpy.polynomial import polynomial as P
    prod = P.polymul(np.array(a, dtype=np.float64), np.array(b, dtype=np.float64))
    div = np.zeros(n + 1)
    div[0] = 1.0
    div[n] = 1.0
    _, rem = P.polydiv(prod, div)
    rem = list(np.rint(rem).astype(np.int64)) + [0] * n
    return [int(v) % q for v in rem[:n]]


@pytest.mark.parametrize("n,q", [(1, 5), (2, 3), (3, 4), (4, 3), (2, 5)])
def test_brute_force_all_pairs_tiny(n, q):
    import itertools
    polys = list(itertools.product(range(q), repeat=n))
    for a in polys:
        for b in polys:
            assert sb.negacyclic_mul(list(a), list(b), q) == _numpy_remainder(a, b, n, q)


@pytest.mark.parametrize("n", [5, 8, 12, 16])
def test_brute_force_random_small(n):
    rng = random.Random(n)
    for q in (2, 7, 97, 3329, 40961):
        for _ in range(10):
            a = _rand_poly(rng, n, q)
            b = _rand_poly(rng, n, q)
            assert sb.negacyclic_mul(a, b, q) == _numpy_remainder(a, b, n, q)


# ---------------------------------------------------------------- roots of x^n+1
def _primitive_2n_root(q, n):
    """Some psi with psi^n = -1 mod prime q (then psi has order 2n)."""
    assert (q - 1) % (2 * n) == 0
    for g in range(2, q):
        psi = pow(g, (q - 1) // (2 * n), q)
        if pow(psi, n, q) == q - 1:
            return psi
    raise AssertionError


def _evaluate(poly, x, q):
    acc = 0
    for coef in reversed(poly):
        acc = (acc * x + coef) % q
    return acc


@pytest.mark.parametrize("n,q", [(16, 97), (64, 12289), (128, 3329), (256, 7681), (1024, 12289)])
def test_root_evaluation_complete(n, q):
    rng = random.Random(q + n)
    a = _rand_poly(rng, n, q)
    b = _rand_poly(rng, n, q)
    c = native.polymul_one(np.array(a, np.uint64), np.array(b, np.uint64), q).tolist()
    if n <= 256:
        assert c == sb.negacyclic_mul(a, b, q)
    psi = _primitive_2n_root(q, n)
    roots = [pow(psi, 2 * i + 1, q) for i in range(n)]
    assert len(set(roots)) == n
    step = 1 if n <= 256 else 7
    for w in roots[::step]:
        assert pow(w, n, q) == q - 1
        assert _evaluate(c, w, q) == _evaluate(a, w, q) * _evaluate(b, w, q) % q


# ---------------------------------------------------------------- Kronecker
def _kronecker(a, b, q):
    n = len(a)
    w = (n * (q - 1) ** 2).bit_length() + 1
    A = sum(int(v) << (w * i) for i, v in enumerate(a))
    B = sum(int(v) << (w * i) for i, v in enumerate(b))
    P = A * B
    mask = (1 << w) - 1
    full = [(P >> (w * d)) & mask for d in range(2 * n - 1)]
    return [(full[j] - (full[j + n] if j + n < 2 * n - 1 else 0)) % q for j in range(n)]


@pytest.mark.parametrize("n,q", [(256, 3329), (1024, 12289), (4096, 998244353),
                                 (2048, (1 << 59) - 55), (1000, (1 << 64) - 59)])
def test_c_oracle_vs_kronecker(n, q):
    rng = np.random.default_rng(n + q % 997)
    a = rng.integers(0, q, size=n, dtype=np.uint64)
    b = rng.integers(0, q, size=n, dtype=np.uint64)
    got = native.polymul_one(a, b, q).tolist()
    assert got == _kronecker(a.tolist(), b.tolist(), q)


def test_c_oracle_extremes_and_python_agree():
    for n, q in ((64, (1 << 64) - 59), (128, (1 << 62) - 57), (32, 2), (17, 3329)):
        a = np.full(n, q - 1, dtype=np.uint64)
        b = np.full(n, q - 1, dtype=np.uint64)
        got = native.polymul_one(a, b, q).tolist()
        assert got == sb.negacyclic_mul(a.tolist(), b.tolist(), q)
        # all-(q-1) times all-(q-1): coefficient j is (j+1) - (n-1-j) = 2j+2-n
        assert got == [(2 * j + 2 - n) % q for j in range(n)]
    rng = np.random.default_rng(5)
    a = rng.integers(0, 3329, size=(3, 2, 64), dtype=np.uint64)
    b = rng.integers(0, 3329, size=(3, 2, 64), dtype=np.uint64)
    qs = [3329, 3001]
    a[:, 1] %= 3001
    b[:, 1] %= 3001
    assert (native.polymul_batch(a, b, qs) == sb.polymul_batch(a, b, qs)).all()


def test_c_oracle_sampled_coeffs():
    rng = np.random.default_rng(9)
    q = (1 << 59) - 55
    a = rng.integers(0, q, size=512, dtype=np.uint64)
    b = rng.integers(0, q, size=512, dtype=np.uint64)
    full = native.polymul_one(a, b, q)
    js = [0, 1, 255, 511, 300]
    assert native.coeffs(a, b, q, js).tolist() == [int(full[j]) for j in js]


# ---------------------------------------------------------------- paper identities
@pytest.mark.parametrize("n", [2, 4, 8, 16, 32])
def test_divide_identity(n):
    rng = random.Random(n)
    q = 12289
    a = _rand_poly(rng, n, q)
    b = _rand_poly(rng, n, q)
    t = sb.toeplitz_matrix(b)
    assert sb.divide_vec_mat(a, t, leaf=1) == sb.vec_mat(a, t)
    # for a negacyclic matrix the diagonal blocks are equal (MA == MD)
    h = n // 2
    assert [r[:h] for r in t[:h]] == [r[h:] for r in t[h:]]
    assert [v % q for v in sb.divide_vec_mat(a, t, leaf=2)] == sb.negacyclic_mul(a, b, q)


@pytest.mark.parametrize("n", [1, 2, 3, 7, 8, 16, 33, 64])
def test_karatsuba_identity(n):
    rng = random.Random(n + 100)
    f = [rng.randrange(-1000, 1000) for _ in range(n)]
    g = [rng.randrange(-1000, 1000) for _ in range(n)]
    assert sb.karatsuba_product(f, g, leaf=1) == sb.full_product(f, g)


def test_rns_route_and_base_rules():
    rng = random.Random(3)
    for n, q in ((8, 3329), (16, 12289), (32, 1 << 20)):
        base = sb.select_rns_base(q, n)
        prod = 1
        for m in base:
            prod *= m
        assert prod > n * q * q
        assert all(m < 256 for m in base)
        assert base == sorted(base, reverse=True)
        for i in range(len(base)):
            for j in range(i + 1, len(base)):
                assert sb._gcd(base[i], base[j]) == 1
        a = _rand_poly(rng, n, q)
        b = _rand_poly(rng, n, q)
        assert sb.rns_polymul(a, b, q, base) == sb.negacyclic_mul(a, b, q)
    # CRT against exhaustive search
    mods = [7, 9, 10]
    for x in range(0, 630, 13):
        assert sb.crt([x % m for m in mods], mods) == x


def _coprime_sequences(maxv):
    """Every pairwise-coprime set of integers in [2, maxv], as a descending
    tuple (exhaustive enumeration)."""
    out = []

    def rec(top, cur):
        out.append(tuple(cur))
        for m in range(top, 1, -1):
            if all(math.gcd(m, c) == 1 for c in cur):
                rec(m - 1, cur + [m])
    rec(maxv, [])
    return out


def _prod(xs):
    p = 1
    for x in xs:
        p *= x
    return p


def _base_by_enumeration(sets, bound):
    """The largest-first rule of Sec. 2.6 read off the enumeration: among the
    minimal coprime sequences whose product exceeds the bound (every proper
    prefix stays at or below it), the lexicographically greatest; None when
    even the largest-first scan of all moduli cannot pass the bound."""
    full = max(sets)  # the largest-first scan taken to the end
    if _prod(full) <= bound:
        return None
    minimal = [t for t in sets if _prod(t) > bound and _prod(t[:-1]) <= bound]
    best = max(minimal)
    assert best == full[:len(best)]
    return list(best)


def _check_base_rule(select):
    """True when `select(q, ell, max_bits)` agrees with the enumeration on
    3- and 4-bit moduli for many bounds and on the closed-form boundary case
    (a bound equal to the first modulus must take a second one)."""
    for bits in (3, 4):
        sets = _coprime_sequences((1 << bits) - 1)
        for q in range(2, 60):
            for ell in (1, 2, 3, 5, 7):
                want = _base_by_enumeration(sets, ell * q * q)
                try:
                    got = select(q, ell, bits)
                except ValueError:
                    got = None
                if got != want:
                    return False
    # 6-bit moduli: 63 = 7 * 3^2 is the first modulus; ell * q^2 = 63 is not
    # yet exceeded by it, so the next largest coprime modulus, 62, follows
    return select(3, 7, 6) == [63, 62]


def test_rns_base_against_enumeration():
    assert _check_base_rule(sb.select_rns_base)


def test_rns_base_pin_catches_planted_mistakes():
    def start_one_low(q, ell, max_bits=8):  # the scan starts at 2^b - 2
        bound, chosen, prod, m = ell * q * q, [], 1, (1 << max_bits) - 2
        while prod <= bound:
            if m < 2:
                raise ValueError
            if all(math.gcd(m, c) == 1 for c in chosen):
                chosen.append(m)
                prod *= m
            m -= 1
        return chosen

    def stops_at_equality(q, ell, max_bits=8):  # product >= bound accepted
        bound, chosen, prod, m = ell * q * q, [], 1, (1 << max_bits) - 1
        while prod < bound:
            if m < 2:
                raise ValueError
            if all(math.gcd(m, c) == 1 for c in chosen):
                chosen.append(m)
                prod *= m
            m -= 1
        return chosen

    def odd_only(q, ell, max_bits=8):  # skips valid even moduli
        bound, chosen, prod, m = ell * q * q, [], 1, (1 << max_bits) - 1
        while prod <= bound:
            if m < 2:
                raise ValueError
            if m % 2 and all(math.gcd(m, c) == 1 for c in chosen):
                chosen.append(m)
                prod *= m
            m -= 1
        return chosen

    def smallest_first(q, ell, max_bits=8):
        bound, chosen, prod, m = ell * q * q, [], 1, 2
        while prod <= bound:
            if m >= (1 << max_bits):
                raise ValueError
            if all(math.gcd(m, c) == 1 for c in chosen):
                chosen.append(m)
                prod *= m
            m += 1
        return sorted(chosen, reverse=True)

    for bad in (start_one_low, stops_at_equality, odd_only, smallest_first):
        assert not _check_base_rule(bad), bad.__name__


# ---------------------------------------------------------------- planted mistakes
def _pins_fail(mul):
    """Run a subset of the pins above against a candidate multiplier;
    return True if any of them fails."""
    rng = random.Random(1)
    try:
        # monomial rule
        for n in (3, 8):
            for i in range(n):
                for j in range(n):
                    ei = [0] * n
                    ej = [0] * n
                    ei[i] = ej[j] = 1
                    want = [0] * n
                    want[(i + j) % n] = 96 if i + j >= n else 1
                    if mul(ei, ej, 97) != want:
                        return True
        # example 1 numerically
        a, b, q = [3, 5, 7], [11, 13, 17], 1009
        a0, a1, a2 = a
        b0, b1, b2 = b
        want = [(a0 * b0 - a1 * b2 - a2 * b1) % q, (a0 * b1 + a1 * b0 - a2 * b2) % q,
                (a0 * b2 + a1 * b1 + a2 * b0) % q]
        if mul(a, b, q) != want:
            return True
        # root evaluation
        n, q = 16, 97
        a = _rand_poly(rng, n, q)
        b = _rand_poly(rng, n, q)
        c = mul(a, b, q)
        psi = _primitive_2n_root(q, n)
        for i in range(n):
            w = pow(psi, 2 * i + 1, q)
            if _evaluate(c, w, q) != _evaluate(a, w, q) * _evaluate(b, w, q) % q:
                return True
        if any(not (0 <= v < q) for v in c):
            return True
    except Exception:
        return True
    return False


def test_planted_mistakes_are_caught():
    assert not _pins_fail(sb.negacyclic_mul)
    assert not _pins_fail(sb.matrix_form_mul)

    def wrap_sign_dropped(a, b, q):  # cyclic instead of negacyclic
        n = len(a)
        c = [0] * n
        for i in range(n):
            for k in range(n):
                c[(i + k) % n] += a[i] * b[k]
        return [v % q for v in c]

    def transposed_matrix(a, b, q):  # a times T(b)^T
        t = sb.toeplitz_matrix(b)
        tt = [list(r) for r in zip(*t)]
        return [v % q for v in sb.vec_mat(a, tt)]

    def off_by_one_fold(a, b, q):
        full = sb.full_product(a, b)
        n = len(a)
        c = list(full[:n])
        for d in range(n, len(full)):
            c[(d - n + 1) % n] -= full[d]
        return [v % q for v in c]

    def lazy_output(a, b, q):  # un-normalised output in [0, 2q)
        return [v + q if v < q // 3 else v for v in sb.negacyclic_mul(a, b, q)]

    def dropped_term(a, b, q):
        n = len(a)
        c = sb.negacyclic_convolution(a, b)
        c[0] += a[n - 1] * b[1] if n > 1 else 0
        return [v % q for v in c]

    def shift_direction(a, b, q):  # rows shifted left instead of right
        n = len(b)
        rows = [list(b)]
        for _ in range(1, n):
            p = rows[-1]
            rows.append(p[1:] + [-p[0]])
        return [v % q for v in sb.vec_mat(a, rows)]

    for bad in (wrap_sign_dropped, transposed_matrix, off_by_one_fold, lazy_output,
                dropped_term, shift_direction):
        assert _pins_fail(bad), bad.__name__


# ---------------------------------------------------------------- the cyclic ring x^n - 1
# Sec. 2.1 names Z_q[x]/(x^n-1) as the other common ring; Sec. 2.5 says the
# matrix form carries over to other moduli.  Pins of the same kinds: the
# monomial rule x^n = 1, brute force against numpy's long division by x^n - 1,
# evaluation at all n-th roots of unity (complete when q = 1 mod n is prime),
# numpy's FFT splitting the full product into both rings, and planted mistakes.
@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 16, 33])
def test_cyclic_monomial_rule(n):
    for i in range(n):
        for j in range(n):
            ei = [0] * n
            ej = [0] * n
            ei[i] = 1
            ej[j] = 1
            want = [0] * n
            want[(i + j) % n] = 1
            assert sb.cyclic_convolution(ei, ej) == want, (n, i, j)
            if n <= 16:
                got = native.polymul_one(np.array(ei, np.uint64), np.array(ej, np.uint64), 97, cyclic=True)
                assert got.tolist() == want


def _numpy_remainder_cyclic(a, b, n, q):
    """Z[x] product and remainder by x^n - 1 via numpy.polynomial."""
    from numpy.polynomial import polynomial as P
    prod = P.polymul(np.array(a, dtype=np.float64), np.array(b, dtype=np.float64))
    div = np.zeros(n + 1)
    div[0] = -1.0
    div[n] = 1.0
    _, rem = P.polydiv(prod, div)
    rem = list(np.rint(rem).astype(np.int64)) + [0] * n
    return [int(v) % q for v in rem[:n]]


@pytest.mark.parametrize("n,q", [(1, 5), (2, 3), (3, 4), (4, 3), (2, 5)])
def test_cyclic_brute_force_all_pairs_tiny(n, q):
    import itertools
    polys = list(itertools.product(range(q), repeat=n))
    for a in polys:
        for b in polys:
            assert sb.cyclic_mul(list(a), list(b), q) == _numpy_remainder_cyclic(a, b, n, q)


@pytest.mark.parametrize("n", [5, 8, 12, 16])
def test_cyclic_brute_force_random_small(n):
    rng = random.Random(100 + n)
    for q in (2, 7, 97, 3329, 40961):
        for _ in range(10):
            a = _rand_poly(rng, n, q)
            b = _rand_poly(rng, n, q)
            want = _numpy_remainder_cyclic(a, b, n, q)
            assert sb.cyclic_mul(a, b, q) == want
            assert sb.circulant_form_mul(a, b, q) == want
            got = native.polymul_one(np.array(a, np.uint64), np.array(b, np.uint64), q, cyclic=True)
            assert got.tolist() == want


def _primitive_n_root(q, n):
    """Some w of multiplicative order exactly n mod prime q (q = 1 mod n)."""
    assert (q - 1) % n == 0
    for g in range(2, q):
        w = pow(g, (q - 1) // n, q)
        if all(pow(w, n // p, q) != 1 for p in (2, 3, 5, 7) if n % p == 0):
            return w
    raise AssertionError


@pytest.mark.parametrize("n,q", [(16, 97), (64, 193), (256, 7681), (1024, 12289), (3, 7)])
def test_cyclic_root_evaluation_complete(n, q):
    rng = random.Random(7 * n + q)
    a = _rand_poly(rng, n, q)
    b = _rand_poly(rng, n, q)
    c = native.polymul_one(np.array(a, np.uint64), np.array(b, np.uint64), q, cyclic=True).tolist()
    if n <= 256:
        assert c == sb.cyclic_mul(a, b, q)
    w = _primitive_n_root(q, n)
    roots = [pow(w, i, q) for i in range(n)]
    assert len(set(roots)) == n  # n distinct roots of x^n - 1: the check is complete
    step = 1 if n <= 256 else 5
    for r in roots[::step]:
        assert pow(r, n, q) == 1
        assert _evaluate(c, r, q) == _evaluate(a, r, q) * _evaluate(b, r, q) % q


@pytest.mark.parametrize("n", [1, 2, 7, 16, 64])
def test_fft_full_product_splits_into_both_rings(n):
    """x^(2n) - 1 = (x^n - 1)(x^n + 1): the full product p = low + x^n high
    (computed by numpy's FFT, exact for these small integers) reduces to
    low + high in the cyclic ring and low - high in the negacyclic one."""
    rng = random.Random(n)
    a = [rng.randrange(50) for _ in range(n)]
    b = [rng.randrange(50) for _ in range(n)]
    fa = np.fft.rfft(np.array(a + [0] * n, dtype=np.float64))
    fb = np.fft.rfft(np.array(b + [0] * n, dtype=np.float64))
    full = [int(v) for v in np.rint(np.fft.irfft(fa * fb, 2 * n))]
    low, high = full[:n], full[n:]
    assert sb.cyclic_convolution(a, b) == [x + y for x, y in zip(low, high)]
    assert sb.negacyclic_convolution(a, b) == [x - y for x, y in zip(low, high)]


@pytest.mark.parametrize("n,q", [(1, 7), (8, 17), (16, 3329), (33, 1000), (64, (1 << 59) + 21)])
def test_cyclic_identity_rotation_and_laws(n, q):
    rng = random.Random(n * 3 + q % 97)
    a = _rand_poly(rng, n, q)
    b = _rand_poly(rng, n, q)
    c = _rand_poly(rng, n, q)
    one = [1] + [0] * (n - 1)
    assert sb.cyclic_mul(a, one, q) == a
    if n > 1:
        x = [0, 1] + [0] * (n - 2)
        assert sb.cyclic_mul(x, a, q) == [a[n - 1]] + a[: n - 1]  # rotation, nothing negated
        r = a
        for _ in range(n):
            r = sb.cyclic_mul(x, r, q)
        assert r == a  # x^n = 1
    ab = sb.cyclic_mul(a, b, q)
    assert ab == sb.cyclic_mul(b, a, q)
    assert sb.cyclic_mul(ab, c, q) == sb.cyclic_mul(a, sb.cyclic_mul(b, c, q), q)
    bc = [(u + v) % q for u, v in zip(b, c)]
    assert sb.cyclic_mul(a, bc, q) == [(u + v) % q for u, v in zip(ab, sb.cyclic_mul(a, c, q))]
    got = native.polymul_one(np.array(a, np.uint64), np.array(b, np.uint64), q, cyclic=True)
    assert got.tolist() == ab
    js = sorted(set([0, n - 1, n // 2]))
    assert native.coeffs(np.array(a, np.uint64), np.array(b, np.uint64), q, js, cyclic=True).tolist() == \
        [ab[j] for j in js]


def test_circulant_matrix_rows():
    b = [10, 20, 30, 40]
    assert sb.circulant_matrix(b) == [[10, 20, 30, 40], [40, 10, 20, 30], [30, 40, 10, 20], [20, 30, 40, 10]]


def _cyclic_pins_fail(mul):
    rng = random.Random(2)
    try:
        for n in (3, 8):
            for i in range(n):
                for j in range(n):
                    ei = [0] * n
                    ej = [0] * n
                    ei[i] = ej[j] = 1
                    want = [0] * n
                    want[(i + j) % n] = 1
                    if mul(ei, ej, 97) != want:
                        return True
        n, q = 16, 97
        a = _rand_poly(rng, n, q)
        b = _rand_poly(rng, n, q)
        c = mul(a, b, q)
        if any(not (0 <= v < q) for v in c):
            return True
        w = _primitive_n_root(q, n)
        for i in range(n):
            r = pow(w, i, q)
            if _evaluate(c, r, q) != _evaluate(a, r, q) * _evaluate(b, r, q) % q:
                return True
        if mul(a[:5], b[:5], q) != _numpy_remainder_cyclic(a[:5], b[:5], 5, q):
            return True
    except Exception:
        return True
    return False


def test_cyclic_planted_mistakes_are_caught():
    assert not _cyclic_pins_fail(sb.cyclic_mul)
    assert not _cyclic_pins_fail(sb.circulant_form_mul)
    assert not _cyclic_pins_fail(lambda a, b, q: native.polymul_one(np.array(a, np.uint64), np.array(b, np.uint64),
                                                                    q, cyclic=True).tolist())

    def negacyclic_instead(a, b, q):
        return sb.negacyclic_mul(a, b, q)

    def wrap_dropped(a, b, q):  # the product truncated to degree < n
        return [v % q for v in sb.full_product(a, b)[: len(a)]]

    def off_by_one_wrap(a, b, q):
        full = sb.full_product(a, b)
        n = len(a)
        c = list(full[:n])
        for d in range(n, len(full)):
            c[(d - n + 1) % n] += full[d]
        return [v % q for v in c]

    def transposed_circulant(a, b, q):
        t = [list(r) for r in zip(*sb.circulant_matrix(b))]
        return [v % q for v in sb.vec_mat(a, t)]

    def lazy_output(a, b, q):
        return [v + q if v < q // 3 else v for v in sb.cyclic_mul(a, b, q)]

    for bad in (negacyclic_instead, wrap_dropped, off_by_one_wrap, transposed_circulant, lazy_output):
        assert _cyclic_pins_fail(bad), bad.__name__

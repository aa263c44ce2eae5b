"""The algebra the tensor path relies on, checked with exact integers on the
CPU against the oracle (no GPU, no code of the CUDA path):

* the Sec. 2.5 division with 8-coefficient blocks: c_{8u+v} is the sum over
  k = 8d' + r of A[u][k] B[v][k], A[u][k] = a~_{8u+k-8D} (block-Hankel in a,
  a row shift of 8 elements) and B[v][k] = b~_{8(D-d')+v-r} (block-Toeplitz
  in b), a~, b~ the antiperiodic (negacyclic) or periodic (cyclic)
  extensions;
* Sec. 2.6 for high degrees: the sum over K split into chunks, and S copies
  of b shifted by 1024 coefficients in the B operand giving, from one A
  slice, the outputs 1024 s further on (a~ b~ is periodic in the summation
  index);
* Sec. 2.4 with the residue number system: the CRT by fast base conversion
  recovers every centred product once the base's product exceeds 16 n
  floor(q/2)^2, with the quotient rounded from a float32 sum.
"""
import math

import numpy as np
import pytest

from oracle import schoolbook as sb


def _ext(x, i, sign):
    """x~_i over [-n, 2n): x~_{i-n} = sign x_i, x~_{i+n} = sign x_i."""
    n = len(x)
    if 0 <= i < n:
        return int(x[i])
    if -n <= i < 0:
        return sign * int(x[i + n])
    assert n <= i < 2 * n
    return sign * int(x[i - n])


def _matrix_form(a, b, sign, kc=None, shifts=1, u_rows=None):
    """c from the block-Hankel x block-Toeplitz products; A slices of 128
    rows (fewer below n = 1024), K in chunks of kc, S shifted copies of b."""
    n = len(a)
    D = n // 8 - 1
    kc = kc or n
    rows = u_rows or min(128, n // 8)
    out = [None] * n
    blocks = max(1, n // 1024)
    for b0 in range(0, blocks, shifts):
        acc = np.zeros((rows, 8 * shifts), dtype=object)
        for c0 in range(0, n, kc):
            for u in range(rows):
                for k in range(c0, c0 + kc):
                    av = _ext(a, 8 * (128 * b0 + u) + k - 8 * D, sign)
                    if av == 0:
                        continue
                    dp, r = divmod(k, 8)
                    for s in range(shifts):
                        for v in range(8):
                            acc[u, 8 * s + v] += av * _ext(b, 8 * (D - dp) + v - r + 1024 * s, sign)
        for s in range(shifts):
            for u in range(rows):
                for v in range(8):
                    j = 8 * (128 * (b0 + s) + u) + v
                    if j < n:
                        out[j] = acc[u, 8 * s + v]
    return out


def _reference(a, b, sign):
    n = len(a)
    c = [0] * n
    for i in range(n):
        for k in range(n):
            if i + k < n:
                c[i + k] += int(a[i]) * int(b[k])
            else:
                c[i + k - n] += sign * int(a[i]) * int(b[k])
    return c


@pytest.mark.parametrize("n", [16, 64, 256])
@pytest.mark.parametrize("sign", [-1, 1])
def test_block_hankel_toeplitz_form(n, sign):
    rng = np.random.default_rng(n)
    a = rng.integers(-50, 51, n)
    b = rng.integers(-50, 51, n)
    assert _matrix_form(a, b, sign) == _reference(a, b, sign)


@pytest.mark.parametrize("sign", [-1, 1])
def test_k_chunks_and_shifted_copies(sign):
    """n = 2048 (two 1024-output blocks): K in four chunks of 512, and both
    blocks from one A slice with a shifted copy of b; sampled rows."""
    n = 2048
    rng = np.random.default_rng(7)
    a = rng.integers(-9, 10, n)
    b = rng.integers(-9, 10, n)
    want = _reference(a, b, sign)
    got = _matrix_form(a, b, sign, kc=512, shifts=2, u_rows=6)  # rows u < 6 of each block
    for s in range(2):
        for u in range(6):
            for v in range(8):
                j = 1024 * s + 8 * u + v
                assert got[j] == want[j], (s, u, v)


def test_matrix_form_matches_the_oracle_mod_q():
    n, q = 64, 12289
    rng = np.random.default_rng(3)
    a = rng.integers(0, q, n)
    b = rng.integers(0, q, n)
    centre = lambda x: np.where(x > q // 2, x - q, x)
    got = [x % q for x in _matrix_form(centre(a), centre(b), -1)]
    want = sb.polymul_batch(a.reshape(1, 1, n).astype(np.uint64), b.reshape(1, 1, n).astype(np.uint64), [q])[0, 0]
    assert [int(x) for x in want] == got


def _crt_fast(x, moduli, q):
    """x from its residues by fast base conversion, the quotient rounded from
    a float32 sum of y_i / m_i (the epilogue's arithmetic), then mod q."""
    M = math.prod(moduli)
    f = np.float32(0)
    s = 0
    for m in moduli:
        Mi = M // m
        y = (x % m) * pow(Mi % m, -1, m) % m
        s += y * (Mi % q)
        f = np.float32(f + np.float32(y) * (np.float32(1) / np.float32(m)))
    k = int(np.rint(f))
    return (s - k * (M % q)) % q


@pytest.mark.parametrize("n,q", [(1024, 12289), (4096, (1 << 59) - 55), (1024, (1 << 62) - 57), (16384, (1 << 30) - 35)])
def test_crt_with_rounded_quotient(n, q):
    """Greedy base (odd, pairwise coprime, largest first under the per-degree
    cap) whose product exceeds 16 n floor(q/2)^2: every integer in the
    centred products' range comes back exactly, the extremes included."""
    h = 0
    while (h + 1) ** 2 * n <= 1 << 24:
        h += 1
    cap = min(255, 2 * h + 1)
    bound = 16 * n * (q // 2) ** 2
    moduli = []
    for m in range(cap, 2, -2):
        if math.prod(moduli) > bound:
            break
        if all(math.gcd(m, x) == 1 for x in moduli):
            moduli.append(m)
    assert math.prod(moduli) > bound and len(moduli) <= 32
    X = n * (q // 2) ** 2
    rng = np.random.default_rng(n)
    xs = [X, -X, 0, 1, -1, X - 1, -X + 1] + [int(v) for v in rng.integers(-(1 << 62), 1 << 62, 200)]
    xs = [max(-X, min(X, x)) for x in xs] + [int(X * t) for t in (0.3, -0.7, 0.999999)]
    for x in xs:
        assert _crt_fast(x, moduli, q) == x % q, x


def test_shifted_copy_needs_the_extension_beyond_n():
    """Planted mistake: extending b periodically past n in the negacyclic
    ring (instead of with the sign) breaks the shifted block."""
    n = 2048
    rng = np.random.default_rng(11)
    a = rng.integers(-9, 10, n)
    b = rng.integers(-9, 10, n)
    want = _reference(a, b, -1)
    good = _matrix_form(a, b, -1, kc=1024, shifts=2, u_rows=2)
    assert all(good[1024 + j] == want[1024 + j] for j in range(16))
    orig = globals()["_ext"]

    def wrong(x, i, sign):
        return int(x[i - len(x)]) if i >= len(x) else orig(x, i, sign)
    globals()["_ext"] = wrong
    try:
        bad = _matrix_form(a, b, -1, kc=1024, shifts=2, u_rows=2)
    finally:
        globals()["_ext"] = orig
    assert any(bad[1024 + j] != want[1024 + j] for j in range(16))

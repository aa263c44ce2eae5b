"""CPU oracle for negacyclic polynomial multiplication in Z_q[x]/(x^n+1).

TEST INFRASTRUCTURE ONLY.  Only the test-suite, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may
import or run anything in this package.  The CUDA library never calls it and
shares no code with it: no kernels, headers, helpers, tables or constants.

Everything here is plain Python integer arithmetic (arbitrary precision), so
nothing can overflow; speed is not a goal.  Functions follow the paper
("TPU as Cryptographic Accelerator", arXiv 2307.06554):

* ``full_product``          -- Sec. 2.1 (i): multiply as if in Z[x]
                               (degree <= 2n-2, coefficients up to n(q-1)^2).
* ``fold_negacyclic``       -- Sec. 2.2: for every d >= n subtract c_d from
                               c_{d-n} (x^n = -1).
* ``negacyclic_mul``        -- the definition: full product, fold, mod q.
                               Result is the unique canonical residue vector.
* ``toeplitz_matrix`` /
  ``vec_mat``               -- Sec. 2.2, Eq. (equ-genereal-mat): row vector
                               a times the negacyclic matrix of b.
* ``divide_vec_mat``        -- Sec. 2.5: split the vector in 2 and the matrix
                               in 4 blocks; r1 = V1*MA + V2*MC,
                               r2 = V1*MB + V2*MD, recursively.
* ``karatsuba_product``     -- Sec. 4: h2 = f1 g1, h0 = f0 g0,
                               h1 = (f1+f0)(g1+g0) - h2 - h0.
* ``select_rns_base`` /
  ``crt`` / ``rns_polymul`` -- Sec. 2.4 and 2.6, Algorithm 1: residues mod
                               small coprime moduli whose product exceeds
                               l*q^2, per-modulus matrix products, CRT back,
                               then mod q.
* ``fold_cyclic`` / ``cyclic_mul`` /
  ``circulant_matrix``      -- the ring Z_q[x]/(x^n-1), which Sec. 2.1 names
                               as the other common ring and to which Sec. 2.5
                               says the matrix form carries over: x^n = 1, so
                               c_d is added to c_{d-n}; the matrix is the
                               circulant of b (rows shifted right by one, the
                               wrapped entry kept).

Readings of the paper taken here (each is pinned by a test):
* orientation: c = a * T(b) with T[i][j] = b_{j-i} for j >= i and
  -b_{n+j-i} for j < i (Example 1 fixes it);
* output: canonical residues in [0, q);
* n: any positive length (Example 1 uses n = 3); q: any integer >= 2
  (Sec. 2.1 says q need not be prime).
"""
from __future__ import annotations

from typing import List, Sequence

import numpy as np


# --------------------------------------------------------------------------
# the definition (Sec. 2.1 (i) + Sec. 2.2)
# --------------------------------------------------------------------------
def full_product(a: Sequence, b: Sequence) -> list:
    """Coefficients of a(x)*b(x) in Z[x]: d-th entry is sum_{i+k=d} a_i b_k.
    Works for any ring elements supporting + and * (ints, sympy symbols)."""
    n, m = len(a), len(b)
    c = [0] * (n + m - 1)
    for i in range(n):
        for k in range(m):
            c[i + k] = c[i + k] + a[i] * b[k]
    return c


def fold_negacyclic(full: Sequence, n: int) -> list:
    """Reduce a Z[x] coefficient list modulo x^n + 1 by the Sec. 2.2 rule:
    the term c_d x^d with d >= n is removed and c_d is subtracted from the
    coefficient of x^(d-n).  Applied from the top degree down, so degrees
    >= 2n (not produced by a product of two length-n operands, but allowed)
    fold repeatedly."""
    c = list(full)
    for d in range(len(c) - 1, n - 1, -1):
        c[d - n] = c[d - n] - c[d]
        c[d] = 0
    return c[:n] + [0] * max(0, n - len(c))


def negacyclic_convolution(a: Sequence, b: Sequence) -> list:
    """a*b in Z[x]/(x^n+1) over the integers (no reduction mod q)."""
    n = len(a)
    if len(b) != n:
        raise ValueError("operands must have the same length")
    return fold_negacyclic(full_product(a, b), n)


def negacyclic_mul(a: Sequence[int], b: Sequence[int], q: int) -> List[int]:
    """c = a*b in Z_q[x]/(x^n+1), coefficients canonical in [0, q)."""
    if q < 2:
        raise ValueError("q must be >= 2")
    return [int(x) % q for x in negacyclic_convolution([int(v) for v in a], [int(v) for v in b])]


# --------------------------------------------------------------------------
# matrix form (Sec. 2.2, Eq. equ-genereal-mat and Example 1)
# --------------------------------------------------------------------------
def toeplitz_matrix(b: Sequence) -> list:
    """The n x n negacyclic matrix of b: row 0 is (b_0 .. b_{n-1}); every
    further row is the row above shifted right by one place with the entry
    that wraps around to column 0 negated.  Entry [i][j] is b_{j-i} when
    j >= i and -b_{n+j-i} when j < i."""
    n = len(b)
    rows = [list(b)]
    for _ in range(1, n):
        prev = rows[-1]
        rows.append([-prev[n - 1]] + prev[: n - 1])
    return rows


def vec_mat(v: Sequence, m: Sequence[Sequence]) -> list:
    """Row vector times matrix: out_j = sum_i v_i m[i][j]."""
    cols = len(m[0]) if m else 0
    out = [0] * cols
    for i, vi in enumerate(v):
        row = m[i]
        for j in range(cols):
            out[j] = out[j] + vi * row[j]
    return out


def matrix_form_mul(a: Sequence[int], b: Sequence[int], q: int) -> List[int]:
    return [int(x) % q for x in vec_mat([int(v) for v in a], toeplitz_matrix([int(v) for v in b]))]


# --------------------------------------------------------------------------
# divide and conquer (Sec. 2.5)
# --------------------------------------------------------------------------
def divide_vec_mat(v: Sequence, m: Sequence[Sequence], leaf: int = 1) -> list:
    """v * M by the Sec. 2.5 split: V = (V1, V2), M = [[MA, MB], [MC, MD]],
    r1 = V1 MA + V2 MC, r2 = V1 MB + V2 MD, result (r1, r2); recursing on
    each block product until the dimension is <= leaf (or odd)."""
    n = len(v)
    if n <= leaf or n % 2:
        return vec_mat(v, m)
    h = n // 2
    v1, v2 = v[:h], v[h:]
    ma = [row[:h] for row in m[:h]]
    mb = [row[h:] for row in m[:h]]
    mc = [row[:h] for row in m[h:]]
    md = [row[h:] for row in m[h:]]
    r1a = divide_vec_mat(v1, ma, leaf)
    r2c = divide_vec_mat(v2, mc, leaf)
    r1b = divide_vec_mat(v1, mb, leaf)
    r2d = divide_vec_mat(v2, md, leaf)
    r1 = [x + y for x, y in zip(r1a, r2c)]
    r2 = [x + y for x, y in zip(r1b, r2d)]
    return r1 + r2


# --------------------------------------------------------------------------
# Karatsuba (Sec. 4)
# --------------------------------------------------------------------------
def karatsuba_product(f: Sequence, g: Sequence, leaf: int = 4) -> list:
    """Z[x] product of equal-length f, g by the Sec. 4 split at x^m:
    f = f1 x^m + f0, g = g1 x^m + g0 (f0, g0 of length m),
    f g = h2 x^2m + h1 x^m + h0."""
    n = len(f)
    if len(g) != n:
        raise ValueError("equal lengths expected")
    if n <= leaf:
        return full_product(f, g)
    m = n // 2
    f0, f1 = list(f[:m]), list(f[m:])
    g0, g1 = list(g[:m]), list(g[m:])
    # pad the low halves to the length of the high halves for the middle term
    L = len(f1)
    f0p = f0 + [0] * (L - m)
    g0p = g0 + [0] * (L - m)
    h0 = karatsuba_product(f0, g0, leaf)
    h2 = karatsuba_product(f1, g1, leaf)
    s = karatsuba_product([x + y for x, y in zip(f1, f0p)], [x + y for x, y in zip(g1, g0p)], leaf)
    h1 = list(s)
    for i, v in enumerate(h2):
        h1[i] -= v
    for i, v in enumerate(h0):
        h1[i] -= v
    out = [0] * (2 * n - 1)
    for i, v in enumerate(h0):
        out[i] += v
    for i, v in enumerate(h1):
        out[i + m] += v
    for i, v in enumerate(h2):
        out[i + 2 * m] += v
    return out


# --------------------------------------------------------------------------
# RNS route of Algorithm 1 (Sec. 2.4, 2.6)
# --------------------------------------------------------------------------
def _gcd(x: int, y: int) -> int:
    while y:
        x, y = y, x % y
    return x


def select_rns_base(q: int, ell: int, max_bits: int = 8) -> List[int]:
    """Sec. 2.6: moduli of at most ``max_bits`` bits, pairwise coprime, the
    largest taken first, until their product exceeds ell * q^2."""
    bound = ell * q * q
    chosen: List[int] = []
    prod = 1
    m = (1 << max_bits) - 1
    while prod <= bound:
        if m < 2:
            raise ValueError("no %d-bit coprime base exceeds l*q^2" % max_bits)
        if all(_gcd(m, c) == 1 for c in chosen):
            chosen.append(m)
            prod *= m
        m -= 1
    return chosen


def crt(residues: Sequence[int], moduli: Sequence[int]) -> int:
    """The unique x in [0, prod m_i) with x = r_i mod m_i (Sec. 2.4)."""
    big = 1
    for m in moduli:
        big *= m
    x = 0
    for r, m in zip(residues, moduli):
        mi = big // m
        x += r * mi * pow(mi, -1, m)
    return x % big


def rns_polymul(a: Sequence[int], b: Sequence[int], q: int, moduli: Sequence[int] = None) -> List[int]:
    """Algorithm 1 with an RNS base: the matrix of b is lifted to
    non-negative entries (-b lifted to q - b), so every integer entry of
    a * T(b) lies in [0, n (q-1)^2]; each modulus m_i gets its own residue
    vector-matrix product; CRT recovers the integers; reduce mod q."""
    n = len(a)
    if moduli is None:
        moduli = select_rns_base(q, n)
    prod = 1
    for m in moduli:
        prod *= m
    if prod <= n * (q - 1) ** 2:
        raise ValueError("RNS base too small for l*q^2")
    t = [[int(x) % q for x in row] for row in toeplitz_matrix([int(v) % q for v in b])]
    av = [int(v) % q for v in a]
    per_mod = []
    for m in moduli:
        am = [x % m for x in av]
        tm = [[x % m for x in row] for row in t]
        per_mod.append([x % m for x in vec_mat(am, tm)])
    return [crt([pm[j] for pm in per_mod], moduli) % q for j in range(n)]


# --------------------------------------------------------------------------
# the cyclic ring Z_q[x]/(x^n - 1) (Sec. 2.1, Sec. 2.5)
# --------------------------------------------------------------------------
def fold_cyclic(full: Sequence, n: int) -> list:
    """Reduce a Z[x] coefficient list modulo x^n - 1: the term c_d x^d with
    d >= n is removed and c_d is added to the coefficient of x^(d-n)
    (x^n = 1), from the top degree down."""
    c = list(full)
    for d in range(len(c) - 1, n - 1, -1):
        c[d - n] = c[d - n] + c[d]
        c[d] = 0
    return c[:n] + [0] * max(0, n - len(c))


def cyclic_convolution(a: Sequence, b: Sequence) -> list:
    """a*b in Z[x]/(x^n-1) over the integers (no reduction mod q)."""
    n = len(a)
    if len(b) != n:
        raise ValueError("operands must have the same length")
    return fold_cyclic(full_product(a, b), n)


def cyclic_mul(a: Sequence[int], b: Sequence[int], q: int) -> List[int]:
    """c = a*b in Z_q[x]/(x^n-1), coefficients canonical in [0, q)."""
    if q < 2:
        raise ValueError("q must be >= 2")
    return [int(x) % q for x in cyclic_convolution([int(v) for v in a], [int(v) for v in b])]


def circulant_matrix(b: Sequence) -> list:
    """The n x n matrix of multiplication by b in Z[x]/(x^n-1): row 0 is
    (b_0 .. b_{n-1}); every further row is the row above shifted right by
    one place, the entry that wraps around to column 0 kept as it is.
    Entry [i][j] is b_{(j-i) mod n}."""
    n = len(b)
    rows = [list(b)]
    for _ in range(1, n):
        prev = rows[-1]
        rows.append([prev[n - 1]] + prev[: n - 1])
    return rows


def circulant_form_mul(a: Sequence[int], b: Sequence[int], q: int) -> List[int]:
    return [int(x) % q for x in vec_mat([int(v) for v in a], circulant_matrix([int(v) for v in b]))]


# --------------------------------------------------------------------------
# batched driver over numpy arrays ([batch][k][n], canonical residues)
# --------------------------------------------------------------------------
def polymul_batch(a: np.ndarray, b: np.ndarray, q_list: Sequence[int], cyclic: bool = False) -> np.ndarray:
    """Python-integer oracle over a [batch][k][n] batch (the cyclic ring
    when ``cyclic``).  Slow (n^2 Python multiplications per product); meant
    for small cases."""
    if a.shape != b.shape or a.ndim != 3 or a.shape[1] != len(q_list):
        raise ValueError("shape mismatch")
    mul = cyclic_mul if cyclic else negacyclic_mul
    out = np.zeros(a.shape, dtype=np.uint64)
    for p in range(a.shape[0]):
        for j, q in enumerate(q_list):
            out[p, j] = mul(a[p, j].tolist(), b[p, j].tolist(), int(q))
    return out

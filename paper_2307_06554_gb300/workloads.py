"""Seeded synthetic inputs for negacyclic polynomial multiplication.

This module is shared by the CUDA path's tests/bench and by the CPU oracle.
It draws moduli and coefficient arrays and nothing else: it holds none of
the multiplication arithmetic (no convolution, no NTT, no reduction of
products).  The paper's own experiments also use synthetic operands
(Sec. 3, "Prototype and evaluation": n in {2^8, 2^10, 2^14}, random
polynomials), so no dataset is stood in for.

Layout convention everywhere: a polynomial batch is a C-contiguous array of
shape [batch][k][n] (product, RNS prime, coefficient), coefficient-contiguous,
each value canonical in [0, q_j).  Storage is uint32 when every q < 2^32,
else uint64.

Workloads (sizes of the five standing configurations):
  * ``ring_small``     n=256,  q=3329 (not NTT-friendly), 64 pairs, int32
  * ``ring_1024``      n=1024, q=12289, 4096 pairs, int32
  * ``rns_4096``       n=4096, 8 seeded 30-bit primes q = 1 mod 8192, 256
                       pairs; a uniform mod q, b ternary {-1,0,1} lifted
  * ``ragged_2000``    2000 products, n in {1024..16384}, 1..16 primes of
                       28..31 bits (q = 1 mod 32768), uniform
  * ``serve_20k``      20000 Poisson requests, n in {4096..65536},
                       1..32 primes of 59 bits (q = 1 mod 2^17), uint64
"""
from __future__ import annotations

import dataclasses
from typing import List, Sequence

import numpy as np

# --------------------------------------------------------------------------
# primality (used only to draw moduli)
# --------------------------------------------------------------------------
_MR_BASES = (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37)


def is_prime(m: int) -> bool:
    """Deterministic Miller-Rabin; the first twelve prime bases decide every
    m < 3.3e24, which covers all 64-bit moduli drawn here."""
    if m < 2:
        return False
    for p in _MR_BASES:
        if m % p == 0:
            return m == p
    d, s = m - 1, 0
    while d % 2 == 0:
        d //= 2
        s += 1
    for a in _MR_BASES:
        x = pow(a, d, m)
        if x == 1 or x == m - 1:
            continue
        for _ in range(s - 1):
            x = x * x % m
            if x == m - 1:
                break
        else:
            return False
    return True


def draw_primes(rng: np.random.Generator, count: int, bits_lo: int, bits_hi: int,
                two_adic: int, exclude: Sequence[int] = ()) -> List[int]:
    """Draw ``count`` distinct primes q = 1 + j*2^two_adic whose bit length is
    drawn uniformly from [bits_lo, bits_hi] (a b-bit prime has
    2^(b-1) < q < 2^b).  Deterministic for a given generator state."""
    out: List[int] = []
    seen = set(int(x) for x in exclude)
    step = 1 << two_adic
    while len(out) < count:
        bits = int(rng.integers(bits_lo, bits_hi + 1))
        jlo = ((1 << (bits - 1)) - 1) // step + 1
        jhi = ((1 << bits) - 2) // step
        if jhi < jlo:
            raise ValueError("no candidate of %d bits with 2^%d | q-1" % (bits, two_adic))
        for _ in range(100000):
            j = int(rng.integers(jlo, jhi + 1))
            q = 1 + j * step
            if q not in seen and is_prime(q):
                seen.add(q)
                out.append(q)
                break
        else:  # pragma: no cover - astronomically unlikely
            raise RuntimeError("prime search exhausted")
    return out


def storage_dtype(q_list: Sequence[int]):
    return np.uint32 if max(q_list) < (1 << 32) else np.uint64


def uniform_coeffs(rng: np.random.Generator, batch: int, q_list: Sequence[int], n: int,
                   dtype=None) -> np.ndarray:
    """[batch][k][n] array, entry (p, j, i) uniform in [0, q_j)."""
    dtype = dtype or storage_dtype(q_list)
    k = len(q_list)
    out = np.empty((batch, k, n), dtype=dtype)
    for j, q in enumerate(q_list):
        out[:, j, :] = rng.integers(0, q, size=(batch, n), dtype=np.uint64).astype(dtype)
    return out


def ternary_coeffs(rng: np.random.Generator, batch: int, q_list: Sequence[int], n: int,
                   dtype=None) -> np.ndarray:
    """[batch][k][n] array of one ternary polynomial per product ({-1,0,1}
    with probability 1/3 each), the same integer polynomial under every
    prime, with -1 lifted to q_j - 1."""
    dtype = dtype or storage_dtype(q_list)
    t = rng.integers(-1, 2, size=(batch, n), dtype=np.int64)
    k = len(q_list)
    out = np.empty((batch, k, n), dtype=dtype)
    for j, q in enumerate(q_list):
        out[:, j, :] = np.where(t < 0, q - 1, t).astype(dtype)
    return out


# --------------------------------------------------------------------------
# the standing workloads
# --------------------------------------------------------------------------
@dataclasses.dataclass
class Batch:
    """One homogeneous batch: every product has the same n and prime list."""
    name: str
    n: int
    q_list: List[int]
    a: np.ndarray  # [batch][k][n]
    b: np.ndarray

    @property
    def batch(self) -> int:
        return self.a.shape[0]


def ring_small(batch: int = 64, seed: int = 1, n: int = 256, q: int = 3329) -> Batch:
    rng = np.random.default_rng(seed)
    a = uniform_coeffs(rng, batch, [q], n)
    b = uniform_coeffs(rng, batch, [q], n)
    return Batch("ring_small n=%d q=%d batch=%d" % (n, q, batch), n, [q], a, b)


def ring_1024(batch: int = 4096, seed: int = 2, n: int = 1024, q: int = 12289) -> Batch:
    rng = np.random.default_rng(seed)
    a = uniform_coeffs(rng, batch, [q], n)
    b = uniform_coeffs(rng, batch, [q], n)
    return Batch("ring_1024 n=%d q=%d batch=%d" % (n, q, batch), n, [q], a, b)


def rns_4096(batch: int = 256, seed: int = 3, n: int = 4096, k: int = 8) -> Batch:
    rng = np.random.default_rng(seed)
    q_list = draw_primes(rng, k, 30, 30, 13)  # q = 1 mod 8192
    a = uniform_coeffs(rng, batch, q_list, n)
    b = ternary_coeffs(rng, batch, q_list, n)
    return Batch("rns_4096 n=%d k=%d batch=%d ternary-b" % (n, k, batch), n, q_list, a, b)


@dataclasses.dataclass
class Product:
    """One product of a ragged batch: its degree, its primes (indices into
    the pool) and its operands ([k][n] each)."""
    n: int
    prime_idx: List[int]
    a: np.ndarray
    b: np.ndarray


@dataclasses.dataclass
class Ragged:
    name: str
    pool: List[int]
    products: List[Product]


RAGGED_DEGREES = (1024, 2048, 4096, 8192, 16384)


def ragged_2000(count: int = 2000, seed: int = 4, degrees: Sequence[int] = RAGGED_DEGREES,
                kmax: int = 16, pool_size: int = 64) -> Ragged:
    """Uneven batch: n uniform over ``degrees``, k uniform in [1, kmax],
    the primes of each product drawn without replacement from a pool of
    28..31-bit primes q = 1 mod 32768 (so q = 1 mod 2n for every n)."""
    rng = np.random.default_rng(seed)
    pool = draw_primes(rng, pool_size, 28, 31, 15)
    prods = []
    for _ in range(count):
        n = int(degrees[int(rng.integers(0, len(degrees)))])
        k = int(rng.integers(1, kmax + 1))
        idx = sorted(int(x) for x in rng.choice(pool_size, size=k, replace=False))
        ql = [pool[i] for i in idx]
        a = uniform_coeffs(rng, 1, ql, n, dtype=np.uint32)[0]
        b = uniform_coeffs(rng, 1, ql, n, dtype=np.uint32)[0]
        prods.append(Product(n, idx, a, b))
    return Ragged("ragged_%d" % count, pool, prods)


SERVE_DEGREES = (4096, 8192, 16384, 32768, 65536)


@dataclasses.dataclass
class Request:
    arrival_s: float
    n: int
    prime_idx: List[int]
    seed: int  # operands are drawn lazily from this seed (see request_operands)


def serve_pool(seed: int = 5, pool_size: int = 32) -> List[int]:
    rng = np.random.default_rng(seed)
    return draw_primes(rng, pool_size, 59, 59, 17)


def serve_requests(count: int = 20000, rate_per_s: float = 1.0e4, seed: int = 5,
                   degrees: Sequence[int] = SERVE_DEGREES, kmax: int = 32,
                   pool_size: int = 32) -> List[Request]:
    """Poisson arrivals (exponential gaps with mean 1/rate), n uniform over
    ``degrees``, k uniform in [1, kmax] primes from the 59-bit pool."""
    rng = np.random.default_rng(seed + 1000)
    gaps = rng.exponential(1.0 / rate_per_s, size=count)
    t = np.cumsum(gaps)
    out = []
    for i in range(count):
        n = int(degrees[int(rng.integers(0, len(degrees)))])
        k = int(rng.integers(1, kmax + 1))
        idx = sorted(int(x) for x in rng.choice(pool_size, size=k, replace=False))
        out.append(Request(float(t[i]), n, idx, seed * 1000003 + i))
    return out


def request_operands(req: Request, pool: Sequence[int]):
    """Operands of one serving request: a, b of shape [k][n], uint64."""
    rng = np.random.default_rng(req.seed)
    ql = [pool[i] for i in req.prime_idx]
    a = uniform_coeffs(rng, 1, ql, req.n, dtype=np.uint64)[0]
    b = uniform_coeffs(rng, 1, ql, req.n, dtype=np.uint64)[0]
    return a, b

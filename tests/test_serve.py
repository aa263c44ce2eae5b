"""Serving loop (continuous batching): every result is identical whether
the request ran alone or in a mix of concurrent requests of different
degrees and prime counts; results match the oracle (sampled coefficients
and evaluation at a root of x^n + 1); admission respects the device-memory
budget; the Poisson replay driver returns one latency per request."""
import numpy as np
import pytest

from oracle import native
from paper_2307_06554_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pm():
    from paper_2307_06554_gb300 import polymul
    return polymul


@pytest.fixture(scope="module")
def pool():
    return wl.serve_pool()


def _pinned(x):
    """A page-locked copy (host-device copies then overlap other work)."""
    import torch
    return torch.from_numpy(x).pin_memory().numpy()


def _requests(pool, count, seed, kmax=6, degrees=wl.SERVE_DEGREES):
    reqs = wl.serve_requests(count=count, seed=seed, kmax=kmax, degrees=degrees)
    out = []
    for r in reqs:
        a, b = wl.request_operands(r, pool)
        out.append((r.n, r.prime_idx, _pinned(a), _pinned(b)))
    return out


def _root(q, n):
    e = (q - 1) // (2 * n)
    for g in range(2, 1000):
        psi = pow(g, e, q)
        if pow(psi, n, q) == q - 1:
            return psi


def _eval(poly, x, q):
    acc = 0
    for coef in reversed(poly.tolist()):
        acc = (acc * x + int(coef)) % q
    return acc


def _oracle_check(pool, n, idx, a, b, c, seed):
    rng = np.random.default_rng(seed)
    for j, pi in enumerate(idx):
        q = pool[pi]
        js = sorted(set([0, n - 1] + [int(x) for x in rng.integers(0, n, 8)]))
        assert np.array_equal(c[j, js], native.coeffs(a[j], b[j], q, js))
        w = pow(_root(q, n), 2 * int(rng.integers(0, n)) + 1, q)
        assert _eval(c[j], w, q) == _eval(a[j], w, q) * _eval(b[j], w, q) % q


def test_alone_equals_in_the_mix(pm, pool):
    reqs = _requests(pool, 14, seed=71)
    with pm.Server(pool, 65536, device_bytes=1 << 30, lanes=6) as srv:
        alone = []
        for n, idx, a, b in reqs:
            c = np.zeros_like(a)
            srv.wait(srv.submit(n, idx, a, b, c))
            alone.append(c)
        mix = [_pinned(np.zeros_like(a)) for _, _, a, _ in reqs]
        tickets = [srv.submit(n, idx, a, b, c) for (n, idx, a, b), c in zip(reqs, mix)]
        for t in tickets:
            srv.wait(t)
        st = srv.stats()
    for i in range(len(reqs)):
        assert np.array_equal(alone[i], mix[i]), "request %d differs in the mix" % i
    for i in (0, 5, 13):
        n, idx, a, b = reqs[i]
        _oracle_check(pool, n, idx, a, b, mix[i], seed=i)
    assert st["completed"] == 2 * len(reqs) and st["failed"] == 0
    # alone: c pageable, so copied; in the mix: every buffer page-locked, so
    # read and written in place
    assert st["completed_direct"] == len(reqs)


@pytest.mark.parametrize("route", ["direct", "staged"])
def test_routes_agree_at_every_degree(pm, route):
    """Degrees 2^4 .. 2^16 (the batch kernel's warp and CTA teams, the
    cluster kernels) and requests of more primes than the launch arguments
    carry (36 of a pool of 40: the prime map goes through the arena): the
    direct route (page-locked a, b, c read and written in place) and the
    staged one give the oracle's products."""
    rng = np.random.default_rng(91)
    pool40 = wl.draw_primes(rng, 40, 59, 59, 17)
    cases = []
    for n, k in ((16, 3), (256, 5), (2048, 36), (4096, 2), (16384, 3), (32768, 2), (65536, 1), (1024, 36)):
        idx = sorted(int(x) for x in rng.choice(40, size=k, replace=False))
        a = np.stack([rng.integers(0, pool40[i], size=n, dtype=np.uint64) for i in idx])
        b = np.stack([rng.integers(0, pool40[i], size=n, dtype=np.uint64) for i in idx])
        cases.append((n, idx, _pinned(a), _pinned(b), _pinned(np.zeros_like(a))))
    with pm.Server(pool40, 65536, device_bytes=1 << 30, lanes=4) as srv:
        if route == "staged":
            srv.set_route(pm.ROUTE_STAGED)
        tickets = [srv.submit(n, idx, a, b, c) for n, idx, a, b, c in cases]
        for t in tickets:
            srv.wait(t)
        st = srv.stats()
    assert st["completed"] == len(cases) and st["failed"] == 0
    assert st["completed_direct"] == (len(cases) if route == "direct" else 0)
    for i, (n, idx, a, b, c) in enumerate(cases):
        _oracle_check(pool40, n, idx, a, b, c, seed=300 + i)


def test_pageable_operands_are_copied(pm, pool):
    """A request with any pageable buffer is copied whatever the route."""
    reqs = _requests(pool, 4, seed=74, kmax=3, degrees=(4096, 16384))
    with pm.Server(pool, 16384, device_bytes=1 << 28, lanes=2) as srv:
        outs = []
        for i, (n, idx, a, b) in enumerate(reqs):
            # request 0 all page-locked; 1, 2, 3 with a pageable a, c or b
            # (kept referenced until the request completes)
            xa = a.copy() if i == 1 else a
            xb = b.copy() if i == 3 else b
            c = np.zeros_like(a) if i == 2 else _pinned(np.zeros_like(a))
            srv.wait(srv.submit(n, idx, xa, xb, c))
            outs.append(c)
        st = srv.stats()
    assert st["completed"] == 4 and st["completed_direct"] == 1
    for i, (n, idx, a, b) in enumerate(reqs):
        _oracle_check(pool, n, idx, a, b, outs[i], seed=400 + i)


def test_admission_by_device_memory(pm, pool):
    """An arena that holds about two of the largest requests: requests queue
    and are admitted as memory frees; all finish and are correct."""
    reqs = _requests(pool, 24, seed=72, kmax=4, degrees=(16384, 32768, 65536))
    budget = 2 * 3 * 4 * 65536 * 8 + (1 << 20)
    outs = [np.zeros_like(a) for _, _, a, _ in reqs]
    with pm.Server(pool, 65536, device_bytes=budget, lanes=4) as srv:
        tickets = [srv.submit(n, idx, a, b, c) for (n, idx, a, b), c in zip(reqs, outs)]
        for t in tickets:
            srv.wait(t)
        st = srv.stats()
    assert st["arena_peak_bytes"] <= budget
    assert st["completed"] == len(reqs)
    for i in (0, 11, 23):
        n, idx, a, b = reqs[i]
        _oracle_check(pool, n, idx, a, b, outs[i], seed=100 + i)


def test_poisson_replay(pm, pool):
    reqs = _requests(pool, 120, seed=73, kmax=4, degrees=(4096, 8192, 16384))
    arrivals = [r.arrival_s for r in wl.serve_requests(count=120, seed=73, rate_per_s=2.0e4, kmax=4,
                                                       degrees=(4096, 8192, 16384))]
    outs = [_pinned(np.zeros_like(a)) for _, _, a, _ in reqs]
    with pm.Server(pool, 16384, device_bytes=1 << 28, lanes=8) as srv:
        lat = srv.replay([(n, idx, a, b, c) for (n, idx, a, b), c in zip(reqs, outs)], arrivals)
        st = srv.stats()
    assert len(lat) == 120 and min(lat) > 0
    assert st["completed"] == 120 and st["p50_us"] <= st["p99_us"]
    for i in (0, 60, 119):
        n, idx, a, b = reqs[i]
        _oracle_check(pool, n, idx, a, b, outs[i], seed=200 + i)


def test_submit_rejects_bad_requests(pm, pool):
    a = np.zeros((1, 4096), np.uint64)
    with pm.Server(pool, 16384, device_bytes=1 << 26, lanes=2) as srv:
        for n, idx in ((100, [0]), (32768, [0]), (4096, [99]), (4096, [])):
            with pytest.raises(pm.PolymulError) as ei:
                srv.submit(n, idx, a, a, a)
            assert ei.value.code == pm.POLYMUL_EINVAL
        with pytest.raises(pm.PolymulError):
            srv.wait(12345, 0.01)


def test_direct_requests_need_no_arena(pm):
    """On the direct route a request needs device memory only for a prime
    map that does not fit the launch arguments: a request larger than the
    whole arena runs (it would be refused on the staged route), and so does
    one of 70 primes of an 80-prime pool (its map takes 280 bytes of the
    arena)."""
    rng = np.random.default_rng(95)
    pool80 = wl.draw_primes(rng, 80, 59, 59, 17)
    n_max = 4096
    small = 3 * n_max * 8 + (1 << 12)  # about one single-prime request of degree n_max
    cases = []
    for n, k in ((4096, 6), (1024, 70)):
        idx = sorted(int(x) for x in rng.choice(80, size=k, replace=False))
        a = np.stack([rng.integers(0, pool80[i], size=n, dtype=np.uint64) for i in idx])
        b = np.stack([rng.integers(0, pool80[i], size=n, dtype=np.uint64) for i in idx])
        cases.append((n, idx, _pinned(a), _pinned(b), _pinned(np.zeros_like(a))))
    with pm.Server(pool80, n_max, device_bytes=small, lanes=2) as srv:
        for n, idx, a, b, c in cases:
            srv.wait(srv.submit(n, idx, a, b, c))
        st = srv.stats()
        assert st["completed_direct"] == 2 and st["arena_peak_bytes"] <= 512
        srv.set_route(pm.ROUTE_STAGED)
        n, idx, a, b, c = cases[0]
        with pytest.raises(pm.PolymulError) as e:
            srv.submit(n, idx, a, b, c)
        assert e.value.code == pm.POLYMUL_EINVAL
    for i, (n, idx, a, b, c) in enumerate(cases):
        _oracle_check(pool80, n, idx, a, b, c, seed=500 + i)

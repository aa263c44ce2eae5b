"""Uneven batches in one persistent launch (and as a CUDA graph) against the
CPU oracle: every product of small mixed lists, a sample of the 2000-product
workload (n from 1024 to 16384, 1..16 primes), graph replay identical to
the direct launch, argument validation, and degree classes moved to the
tensor path (the drained tiled digit kernel over the class's rows) alone,
mixed with NTT classes, and as the tuner chooses."""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

from oracle import native
from paper_2307_06554_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pm():
    from paper_2307_06554_gb300 import polymul
    return polymul


def _pack(rag):
    total = sum(p.n * len(p.prime_idx) for p in rag.products)
    a = np.empty(total, np.uint32)
    b = np.empty(total, np.uint32)
    off = 0
    for p in rag.products:
        m = p.n * len(p.prime_idx)
        a[off:off + m] = p.a.reshape(-1)
        b[off:off + m] = p.b.reshape(-1)
        off += m
    return a, b


def _run(pm, rag, nmax=16384, graph=False, choice=None, tune=False):
    import torch
    a, b = _pack(rag)
    with pm.Ragged(rag.pool, nmax, [(p.n, p.prime_idx) for p in rag.products]) as r:
        ta = torch.from_numpy(a.view(np.int32)).cuda()
        tb = torch.from_numpy(b.view(np.int32)).cuda()
        tc = torch.full_like(ta, -1)
        if choice is not None:
            r.select(choice)
        if tune:
            assert 0 <= r.tune(ta, tb, tc) < 128
            tc.fill_(-1)
        r.run(ta, tb, tc, graph=graph)
        pm.polymul_ragged_status(r.batch)
        offsets = list(r.offsets)
        c = tc.cpu().numpy().view(np.uint32)
    return c, offsets


def _check(rag, c, offsets, which):
    def one(i):
        p = rag.products[i]
        qs = [rag.pool[j] for j in p.prime_idx]
        want = native.polymul_batch(p.a[None], p.b[None], qs, threads=1)[0]
        got = c[offsets[i]:offsets[i] + p.n * len(qs)].reshape(len(qs), p.n).astype(np.uint64)
        return i if not np.array_equal(got, want) else None
    with ThreadPoolExecutor(max_workers=native.default_threads()) as ex:
        bad = [i for i in ex.map(one, which) if i is not None]
    assert not bad, "mismatching products: %s" % bad[:10]


def test_small_mixed_every_product(pm):
    rag = wl.ragged_2000(count=40, seed=41, degrees=(1024, 2048, 4096), kmax=4, pool_size=8)
    c, off = _run(pm, rag)
    _check(rag, c, off, range(len(rag.products)))


def test_largest_degrees(pm):
    rag = wl.ragged_2000(count=4, seed=42, degrees=(8192, 16384), kmax=2, pool_size=4)
    c, off = _run(pm, rag)
    _check(rag, c, off, range(len(rag.products)))


def test_segments_of_different_team_counts_on_one_cta(pm):
    """More units than CTAs, a one-team segment (n = 16384) before an
    eight-team segment (n = 1024): CTAs move between team layouts, teams take
    different numbers of units, and every team barrier must keep its own
    phase.  Checks the n = 1024 products."""
    rag = wl.ragged_2000(count=400, seed=44, degrees=(1024, 16384), kmax=2, pool_size=4)
    c, off = _run(pm, rag)
    _check(rag, c, off, [i for i, p in enumerate(rag.products) if p.n == 1024])


def test_fewer_units_than_ctas_and_relaunch(pm):
    """Three units in all (grid of three CTAs), launched twice on the same
    plan: the segment counters reset between launches."""
    import torch
    rag = wl.ragged_2000(count=2, seed=45, degrees=(1024, 8192), kmax=2, pool_size=3)
    a, b = _pack(rag)
    outs = []
    with pm.Ragged(rag.pool, 16384, [(p.n, p.prime_idx) for p in rag.products]) as r:
        assert r.info["grid"] == r.info["units"] <= 4
        ta = torch.from_numpy(a.view(np.int32)).cuda()
        tb = torch.from_numpy(b.view(np.int32)).cuda()
        for graph in (False, False, True, True):
            tc = torch.full_like(ta, -1)
            r.run(ta, tb, tc, graph=graph)
            pm.polymul_ragged_status(r.batch)
            outs.append(tc.cpu().numpy().view(np.uint32))
        off = list(r.offsets)
    for c in outs[1:]:
        assert np.array_equal(c, outs[0])
    _check(rag, outs[0], off, range(len(rag.products)))


def test_smaller_nmax_prefix_tables(pm):
    """A pool built for n_max = 4096 serves 1024..4096 through table prefixes."""
    rag = wl.ragged_2000(count=24, seed=43, degrees=(1024, 2048, 4096), kmax=3, pool_size=6)
    c, off = _run(pm, rag, nmax=4096)
    _check(rag, c, off, range(len(rag.products)))


def test_ragged_2000_sampled_and_graph(pm):
    rag = wl.ragged_2000()
    c1, off = _run(pm, rag)
    c2, _ = _run(pm, rag, graph=True)
    assert np.array_equal(c1, c2)
    small = [i for i, p in enumerate(rag.products) if p.n == 1024]
    rng = np.random.default_rng(7)
    large = [int(i) for i in rng.choice([i for i, p in enumerate(rag.products) if p.n > 1024], 8, replace=False)]
    _check(rag, c1, off, small + large)


def test_prepare_rejects_bad_descriptors(pm):
    pool = wl.ragged_2000(count=1, pool_size=4).pool
    ctx = pm.polymul_ragged_create(pool, 4096)
    try:
        bad = [
            ([(512, 1, 0, 0)], [0], 512),        # n below 1024
            ([(8192, 1, 0, 0)], [0], 8192),      # n above n_max
            ([(1024, 2, 0, 0)], [0], 2048),      # prime list too short
            ([(1024, 1, 0, 0)], [9], 1024),      # prime index outside the pool
            ([(1024, 1, 0, 2)], [0], 4096),      # misaligned offset
            ([(1024, 2, 0, 0)], [0, 1], 1500),   # rows outside the buffers
        ]
        for descs, idx, total in bad:
            with pytest.raises(pm.PolymulError) as ei:
                pm.polymul_ragged_prepare(ctx, descs, idx, total)
            assert ei.value.code == pm.POLYMUL_EINVAL
    finally:
        pm.polymul_ragged_destroy(ctx)
    with pytest.raises(pm.PolymulError):
        pm.polymul_ragged_create([3329], 1024)  # 3329 - 1 is not divisible by 2048


@pytest.mark.parametrize("choice", [0, 1, 2, 3])
def test_every_shape_set_is_exact(pm, choice):
    """Both shape sets of both launches (swizzled / padded exchanges, one or
    both operands in registers), on a list that has every degree class."""
    rag = wl.ragged_2000(count=25, seed=32)
    assert {p.n for p in rag.products} == {1024, 2048, 4096, 8192, 16384}
    c, offsets = _run(pm, rag, choice=choice)
    _check(rag, c, offsets, range(len(rag.products)))


def test_tuned_list_is_exact_direct_and_graph(pm):
    rag = wl.ragged_2000(count=25, seed=35)
    c, offsets = _run(pm, rag, tune=True)
    _check(rag, c, offsets, range(len(rag.products)))
    c, offsets = _run(pm, rag, tune=True, graph=True)
    _check(rag, c, offsets, range(len(rag.products)))


ALL_CLASSES = (10, 11, 12, 13, 14)


@pytest.mark.parametrize("logns,sets", [(ALL_CLASSES, 3), ((10, 12, 14), 1), ((11, 13), 2), ((14,), 0)])
def test_tensor_classes_are_exact(pm, logns, sets):
    """Degree classes on the tensor path, the rest on the NTT launches (with
    either shape set), direct and as a graph: every product against the
    oracle."""
    rag = wl.ragged_2000(count=25, seed=32)
    choice = sets | pm.ragged_tensor_bits(*logns)
    c, offsets = _run(pm, rag, choice=choice)
    _check(rag, c, offsets, range(len(rag.products)))
    c2, _ = _run(pm, rag, choice=choice, graph=True)
    assert np.array_equal(c, c2)


def test_tensor_classes_relaunch_and_switch(pm):
    """The same list launched repeatedly while its classes move between the
    paths (the tensor launches' counters reset, the NTT segment list is
    rewritten, a recorded graph is rebuilt): identical results each time."""
    import torch
    rag = wl.ragged_2000(count=30, seed=36, kmax=4)
    a, b = _pack(rag)
    outs = []
    with pm.Ragged(rag.pool, 16384, [(p.n, p.prime_idx) for p in rag.products]) as r:
        ta = torch.from_numpy(a.view(np.int32)).cuda()
        tb = torch.from_numpy(b.view(np.int32)).cuda()
        for choice, graph in ((1, True), (1 | pm.ragged_tensor_bits(*ALL_CLASSES), True),
                              (1 | pm.ragged_tensor_bits(*ALL_CLASSES), False), (3 | pm.ragged_tensor_bits(12), True),
                              (1, False)):
            r.select(choice)
            for _ in range(2):
                tc = torch.full_like(ta, -1)
                r.run(ta, tb, tc, graph=graph)
                pm.polymul_ragged_status(r.batch)
                outs.append(tc.cpu().numpy().view(np.uint32))
        off = list(r.offsets)
    for c in outs[1:]:
        assert np.array_equal(c, outs[0])
    _check(rag, outs[0], off, range(len(rag.products)))


def test_select_rejects_bad_choice(pm):
    import torch
    rag = wl.ragged_2000(count=3, seed=37, degrees=(1024,), kmax=2, pool_size=4)
    with pm.Ragged(rag.pool, 4096, [(p.n, p.prime_idx) for p in rag.products]) as r:
        with pytest.raises(pm.PolymulError) as ei:
            r.select(128)
        assert ei.value.code == pm.POLYMUL_EINVAL
        r.select(pm.ragged_tensor_bits(13, 14))  # classes the list does not hold: ignored
        a, b = _pack(rag)
        ta = torch.from_numpy(a.view(np.int32)).cuda()
        tb = torch.from_numpy(b.view(np.int32)).cuda()
        tc = torch.full_like(ta, -1)
        r.run(ta, tb, tc)
        pm.polymul_ragged_status(r.batch)
        c = tc.cpu().numpy().view(np.uint32)
        off = list(r.offsets)
    _check(rag, c, off, range(len(rag.products)))

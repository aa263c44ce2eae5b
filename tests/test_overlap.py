"""Back-to-back batches on one stream with POLYMUL_FLAG_OVERLAP: a batch may
start loading and multiplying before the previous batch launch on the stream
has finished, and only when neither writes what the other reads or writes.
Every result is compared with the CPU oracle, including chains where one
batch's result is the next one's operand (the library must then wait)."""
import numpy as np
import pytest

from oracle import native
from paper_2307_06554_gb300 import workloads as wl

from helpers import assert_equal_residues, from_dev, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pm():
    from paper_2307_06554_gb300 import polymul
    return polymul


def _operands(seed, batch, q_list, n, dtype):
    rng = np.random.default_rng(seed)
    return (wl.uniform_coeffs(rng, batch, q_list, n, dtype), wl.uniform_coeffs(rng, batch, q_list, n, dtype))


@pytest.mark.parametrize("n,bits,k,batch,dtype", [
    (1024, 14, 1, 2048, np.uint32),   # more units than teams: counter grabs after the early first unit
    (2048, 30, 3, 700, np.uint32),
    (256, 30, 2, 3000, np.uint32),
    (1024, 59, 2, 300, np.uint64),
])
def test_independent_batches(pm, n, bits, k, batch, dtype):
    import torch
    rng = np.random.default_rng(n + bits + k)
    if bits == 14:
        q_list = [12289]
    else:
        q_list = wl.draw_primes(rng, k, bits, bits, (2 * n).bit_length() - 1)
    sets = [_operands(10 * i + n, batch, q_list, n, dtype) for i in range(4)]
    stream = torch.cuda.Stream()
    with pm.Plan(n, q_list, flags=pm.FLAG_OVERLAP) as plan:
        assert plan.info["launch_flags"] & 4, plan.info
        dev = [(to_dev(a), to_dev(b)) for a, b in sets]
        outs = [torch.full_like(ta, -1) for ta, _ in dev]
        with torch.cuda.stream(stream):
            for rep in range(3):
                for i, (ta, tb) in enumerate(dev):
                    plan.batch(ta, tb, outs[i], stream=stream.cuda_stream)
        stream.synchronize()
        pm.polymul_plan_status(plan.handle, stream.cuda_stream)
    for i, (a, b) in enumerate(sets):
        assert_equal_residues(from_dev(outs[i], dtype), native.polymul_batch(a, b, q_list), "set %d" % i)


def test_chain_waits_for_its_operand(pm):
    """c_{i+1} = c_i * b_i: each batch reads the previous batch's result
    (read after write), so no batch may run ahead."""
    import torch
    n, q, batch = 1024, 12289, 2048
    a, _ = _operands(1, batch, [q], n, np.uint32)
    bs = [_operands(20 + i, batch, [q], n, np.uint32)[1] for i in range(5)]
    stream = torch.cuda.Stream()
    with pm.Plan(n, [q], flags=pm.FLAG_OVERLAP) as plan:
        cur = to_dev(a)
        tbs = [to_dev(b) for b in bs]
        bufs = [torch.empty_like(cur) for _ in bs]
        with torch.cuda.stream(stream):
            for i, tb in enumerate(tbs):
                plan.batch(cur, tb, bufs[i], stream=stream.cuda_stream)
                cur = bufs[i]
        stream.synchronize()
        got = from_dev(cur, np.uint32)
    want = a
    for b in bs:
        want = native.polymul_batch(want, b, [q]).astype(np.uint32)
    assert_equal_residues(got, want, "chain of 5")


def test_result_overwrites_previous_operand(pm):
    """The second batch writes its result over the first batch's operand a
    (write after read): it may not start before the first has read it."""
    import torch
    n, q, batch = 1024, 12289, 2048
    a1, b1 = _operands(3, batch, [q], n, np.uint32)
    a2, b2 = _operands(4, batch, [q], n, np.uint32)
    stream = torch.cuda.Stream()
    with pm.Plan(n, [q], flags=pm.FLAG_OVERLAP) as plan:
        ta1, tb1, ta2, tb2 = to_dev(a1), to_dev(b1), to_dev(a2), to_dev(b2)
        c1 = torch.empty_like(ta1)
        with torch.cuda.stream(stream):
            plan.batch(ta1, tb1, c1, stream=stream.cuda_stream)
            plan.batch(ta2, tb2, ta1, stream=stream.cuda_stream)  # result over a1
        stream.synchronize()
        got1, got2 = from_dev(c1, np.uint32), from_dev(ta1, np.uint32)
    assert_equal_residues(got1, native.polymul_batch(a1, b1, [q]), "first batch")
    assert_equal_residues(got2, native.polymul_batch(a2, b2, [q]), "second batch")


def test_plans_with_and_without_the_flag_share_a_stream(pm):
    """A batch of a plan without the flag, then batches of a plan with it
    that read its result and that do not: the record of the previous launch
    on the stream is kept across plans."""
    import torch
    n, q, batch = 1024, 12289, 1600
    a, b = _operands(5, batch, [q], n, np.uint32)
    x, y = _operands(6, batch, [q], n, np.uint32)
    stream = torch.cuda.Stream()
    with pm.Plan(n, [q]) as plain, pm.Plan(n, [q], flags=pm.FLAG_OVERLAP) as over:
        assert not plain.info["launch_flags"] & 4
        ta, tb, tx, ty = to_dev(a), to_dev(b), to_dev(x), to_dev(y)
        c0, c1, c2 = torch.empty_like(ta), torch.empty_like(ta), torch.empty_like(ta)
        with torch.cuda.stream(stream):
            plain.batch(ta, tb, c0, stream=stream.cuda_stream)
            over.batch(c0, tb, c1, stream=stream.cuda_stream)   # reads the plain plan's result
            over.batch(tx, ty, c2, stream=stream.cuda_stream)   # independent: may run ahead
        stream.synchronize()
        g0, g1, g2 = (from_dev(t, np.uint32) for t in (c0, c1, c2))
    w0 = native.polymul_batch(a, b, [q])
    assert_equal_residues(g0, w0, "plain")
    assert_equal_residues(g1, native.polymul_batch(w0.astype(np.uint32), b, [q]), "dependent")
    assert_equal_residues(g2, native.polymul_batch(x, y, [q]), "independent")


def test_default_stream_ignores_the_flag(pm):
    """On the legacy default stream the flag has no effect (results exact)."""
    import torch
    n, q, batch = 1024, 12289, 512
    a, b = _operands(7, batch, [q], n, np.uint32)
    with pm.Plan(n, [q], flags=pm.FLAG_OVERLAP) as plan:
        ta, tb = to_dev(a), to_dev(b)
        c1, c2 = torch.empty_like(ta), torch.empty_like(ta)
        pm.polymul_batch(plan.handle, ta, tb, c1, batch, 0)
        pm.polymul_batch(plan.handle, c1, tb, c2, batch, 0)
        torch.cuda.synchronize()
        got = from_dev(c2, np.uint32)
    w = native.polymul_batch(a, b, [q]).astype(np.uint32)
    assert_equal_residues(got, native.polymul_batch(w, b, [q]), "default stream chain")

"""Path (a), the batched negacyclic NTT, against the CPU oracle: bit-exact
on seeded inputs at sizes spanning several teams/CTAs with ragged tails, at
the full sizes of the standing workloads, and on the edge cases."""
import numpy as np
import pytest

from oracle import native
from oracle import schoolbook as sb
from paper_2307_06554_gb300 import workloads as wl

from helpers import assert_equal_residues, run_plan_batch, to_dev, from_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pm():
    from paper_2307_06554_gb300 import polymul
    return polymul


def _primes(seed, k, bits, n, exclude=()):
    rng = np.random.default_rng(seed)
    return wl.draw_primes(rng, k, bits, bits, max(n.bit_length(), 1), exclude)


def _case(seed, batch, q_list, n, dtype=None):
    rng = np.random.default_rng(seed)
    return wl.uniform_coeffs(rng, batch, q_list, n, dtype), wl.uniform_coeffs(rng, batch, q_list, n, dtype)


@pytest.mark.parametrize("logn", list(range(4, 15)))
@pytest.mark.parametrize("bits", [30, 31])
def test_u32_all_degrees(pm, logn, bits):
    n = 1 << logn
    k = 3 if n <= 4096 else 2
    batch = {16: 37, 32: 37, 64: 29, 128: 21, 256: 19, 512: 13, 1024: 11}.get(n, 3)
    q_list = _primes(100 + logn + bits, k, bits, 2 * n)
    a, b = _case(logn * 7 + bits, batch, q_list, n, np.uint32)
    with pm.Plan(n, q_list) as plan:
        assert plan.info["path"] == pm.PATH_NTT and plan.elem_bytes == 4
        got = run_plan_batch(plan, a, b)
    assert_equal_residues(got, native.polymul_batch(a, b, q_list), "n=%d bits=%d" % (n, bits))


@pytest.mark.parametrize("logn", list(range(4, 14)))
@pytest.mark.parametrize("bits", [59, 62])
def test_u64_all_degrees(pm, logn, bits):
    n = 1 << logn
    k = 2
    batch = {16: 37, 32: 33, 64: 19, 128: 17, 256: 9, 512: 7, 1024: 5}.get(n, 2)
    q_list = _primes(200 + logn + bits, k, bits, 2 * n)
    a, b = _case(logn * 11 + bits, batch, q_list, n, np.uint64)
    with pm.Plan(n, q_list) as plan:
        assert plan.info["path"] == pm.PATH_NTT and plan.elem_bytes == 8
        got = run_plan_batch(plan, a, b)
    assert_equal_residues(got, native.polymul_batch(a, b, q_list), "n=%d bits=%d" % (n, bits))


@pytest.mark.parametrize("logn", list(range(4, 15)))
def test_u32_small_moduli_all_degrees(pm, logn):
    """Small moduli (PQC sizes) run with no conditional subtractions; the
    bound tracking must hold at every degree, including all-(q-1) inputs."""
    n = 1 << logn
    q_list = [65537] + ([40961] if logn <= 12 else []) + ([12289] if logn <= 11 else []) \
        + ([8380417] if logn <= 8 else [])
    batch = 23 if n <= 1024 else 3
    a, b = _case(300 + logn, batch, q_list, n, np.uint32)
    for j, q in enumerate(q_list):
        a[-1, j, :] = q - 1
        b[-1, j, :] = q - 1
    with pm.Plan(n, q_list) as plan:
        got = run_plan_batch(plan, a, b)
    assert_equal_residues(got, native.polymul_batch(a, b, q_list), "small q n=%d" % n)


@pytest.mark.parametrize("logn", [4, 8, 10, 13])
def test_u64_small_moduli(pm, logn):
    n = 1 << logn
    q_list = _primes(400 + logn, 2, 40, 2 * n)
    a, b = _case(500 + logn, 5, q_list, n, np.uint64)
    q_list = [int(q) for q in q_list]
    a[-1] = np.array(q_list, np.uint64)[:, None] - 1
    b[-1] = np.array(q_list, np.uint64)[:, None] - 1
    with pm.Plan(n, q_list) as plan:
        got = run_plan_batch(plan, a, b)
    assert_equal_residues(got, native.polymul_batch(a, b, q_list), "u64 small q n=%d" % n)


def test_ring_1024_full_size(pm):
    """n=1024, q=12289, 4096 pairs: every output coefficient."""
    w = wl.ring_1024()
    with pm.Plan(w.n, w.q_list) as plan:
        got = run_plan_batch(plan, w.a, w.b)
    assert_equal_residues(got, native.polymul_batch(w.a, w.b, w.q_list), w.name)


def test_rns_4096_full_size(pm):
    """n=4096, 8 primes of 30 bits, 256 pairs, ternary b: every output."""
    w = wl.rns_4096()
    with pm.Plan(w.n, w.q_list) as plan:
        got = run_plan_batch(plan, w.a, w.b)
    assert_equal_residues(got, native.polymul_batch(w.a, w.b, w.q_list), w.name)


@pytest.mark.parametrize("n,q", [(1024, 12289), (4096, 786433), (2048, 2013265921)])
def test_edge_values(pm, n, q):
    assert (q - 1) % (2 * n) == 0 and wl.is_prime(q)
    zeros = np.zeros((1, 1, n), np.uint32)
    top = np.full((1, 1, n), q - 1, np.uint32)
    mono = np.zeros((1, 1, n), np.uint32)
    mono[0, 0, n - 1] = 1
    one = np.zeros((1, 1, n), np.uint32)
    one[0, 0, 0] = 1
    rng = np.random.default_rng(3)
    r = rng.integers(0, q, size=(1, 1, n), dtype=np.uint64).astype(np.uint32)
    a = np.concatenate([zeros, top, mono, one, r, top])
    b = np.concatenate([r, top, mono, r, zeros, r])
    with pm.Plan(n, [q]) as plan:
        got = run_plan_batch(plan, a, b).astype(np.uint64)
    want = native.polymul_batch(a, b, [q])
    assert_equal_residues(got, want, "edges")
    assert not got[0].any() and not got[4].any()
    # x^(n-1) * x^(n-1) = -x^(n-2)
    exp = np.zeros(n, np.uint64)
    exp[n - 2] = q - 1
    assert np.array_equal(got[2, 0], exp)
    assert np.array_equal(got[3, 0], r[0, 0].astype(np.uint64))
    # all (q-1) squared: coefficient j is 2j + 2 - n mod q
    assert np.array_equal(got[1, 0], np.array([(2 * j + 2 - n) % q for j in range(n)], np.uint64))


def test_batch_zero_and_one(pm):
    import torch
    n, q = 1024, 12289
    a, b = _case(5, 1, [q], n, np.uint32)
    with pm.Plan(n, [q]) as plan:
        ta, tb = to_dev(a), to_dev(b)
        tc = torch.full_like(ta, 7)
        pm.polymul_batch(plan.handle, ta, tb, tc, 0)  # no-op
        torch.cuda.synchronize()
        assert (tc == 7).all()
        got = run_plan_batch(plan, a, b)
    assert_equal_residues(got, native.polymul_batch(a, b, [q]), "batch 1")


def test_validate_flag_rejects_out_of_range(pm):
    n, q = 256, 7681
    a, b = _case(6, 4, [q], n, np.uint32)
    a[2, 0, 17] = q  # not canonical
    with pm.Plan(n, [q], flags=pm.FLAG_VALIDATE) as plan:
        with pytest.raises(pm.PolymulError) as ei:
            run_plan_batch(plan, a, b)
        assert ei.value.code == pm.POLYMUL_EDOMAIN
        a[2, 0, 17] = q - 1
        got = run_plan_batch(plan, a, b)
    assert_equal_residues(got, native.polymul_batch(a, b, [q]), "validated")


def test_host_buffer_entry_matches_device_entry(pm):
    w = wl.ring_1024(batch=3000, seed=12)
    with pm.Plan(w.n, w.q_list) as plan:
        dev = run_plan_batch(plan, w.a, w.b)
        c = np.zeros_like(w.a)
        plan.batch_host(w.a, w.b, c)
    assert np.array_equal(c, dev)
    # spot-check against the oracle
    idx = [0, 1499, 2999]
    want = native.polymul_batch(w.a[idx], w.b[idx], w.q_list)
    assert_equal_residues(c[idx], want, "host entry")


def test_other_stream_and_reuse(pm):
    import torch
    n = 2048
    q_list = _primes(77, 2, 30, 2 * n)
    a, b = _case(8, 9, q_list, n, np.uint32)
    with pm.Plan(n, q_list) as plan:
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            ta, tb = to_dev(a), to_dev(b)
            tc = torch.empty_like(ta)
            for _ in range(3):
                plan.batch(ta, tb, tc, stream=s)
        s.synchronize()
        got = from_dev(tc, np.uint32)
    assert_equal_residues(got, native.polymul_batch(a, b, q_list), "stream")


@pytest.mark.parametrize("n,batch", [(1024, 3000), (256, 64), (4096, 300)])
def test_chained_batches_on_one_stream(pm, n, batch):
    """Each launch reads the previous launch's results (the batch kernels take
    a programmatic dependent launch: a dependent kernel may start while the
    previous one drains, and must still see all of its results), with a
    foreign kernel interleaved, all on one stream without synchronisation."""
    import torch
    q_list = [12289] if n <= 1024 else _primes(77, 1, 30, 2 * n)
    a, b = _case(900 + n, batch, q_list, n, np.uint32)
    stream = torch.cuda.Stream()
    with pm.Plan(n, q_list) as plan, torch.cuda.stream(stream):
        assert plan.info["launch_flags"] & 2
        x, y = to_dev(a), to_dev(b)
        outs = []
        for i in range(4):
            z = torch.empty_like(x)
            plan.batch(x, y, z, stream=stream.cuda_stream)
            if i == 1:
                z = z.clone()  # a torch kernel between two dependent launches
            outs.append(z)
            x = z
        stream.synchronize()
        polymul_status = pm.polymul_plan_status(plan.handle, stream.cuda_stream)
    assert polymul_status is None
    want = a
    for i in range(4):
        want = native.polymul_batch(want.astype(np.uint32), b, q_list)
        assert_equal_residues(from_dev(outs[i], np.uint32), want, "link %d" % i)


@pytest.mark.parametrize("path", ["ntt", "tensor"])
def test_host_entry_more_chunks_than_slots(pm, path):
    """polymul_batch_host on 256 products of n = 4096 with 8 primes: 8 chunks
    of 32 products through the 6 staging slots of its three-stream pipeline
    (every slot reused), on both paths; equal to the device entry and to the
    oracle on a sample."""
    import torch
    w = wl.rns_4096()
    p_id = pm.PATH_NTT if path == "ntt" else pm.PATH_TENSOR
    with pm.Plan(w.n, w.q_list, path=p_id) as plan:
        c = np.zeros_like(w.a)
        plan.batch_host(w.a, w.b, c)
        ta = torch.from_numpy(w.a.view(np.int32)).cuda()
        tb = torch.from_numpy(w.b.view(np.int32)).cuda()
        tc = torch.empty_like(ta)
        plan.batch(ta, tb, tc)
        torch.cuda.synchronize()
        pm.polymul_plan_status(plan.handle)
        dev = tc.cpu().numpy().view(np.uint32)
    assert np.array_equal(c, dev)
    for p in (0, 131, 255):
        assert_equal_residues(c[p:p + 1], native.polymul_batch(w.a[p:p + 1], w.b[p:p + 1], w.q_list), "product %d" % p)

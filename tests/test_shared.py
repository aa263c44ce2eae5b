"""Shared-operand products (polymul_batch_shared): c_i = a * b_i for one a,
as the GEMM C = B * T(a) on the tensor cores and on the NTT path (a's
transform once), against the CPU oracle: ragged batch tails (not a multiple
of the 128-row tile), several moduli, both rings, both digit widths, every
NTT reduction mode, extreme operands, and the error cases."""
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


def _run(pm, plan, a, b):
    import torch
    ta, tb = to_dev(a), to_dev(b)
    tc = torch.full_like(tb, -1)
    pm.polymul_batch_shared(plan.handle, ta, tb, tc, b.shape[0])
    torch.cuda.synchronize()
    pm.polymul_plan_status(plan.handle)
    return from_dev(tc, b.dtype)


def _want(a, b, q_list, cyclic=False):
    return native.polymul_batch(np.broadcast_to(a[None], b.shape).copy(), b, q_list, cyclic=cyclic)


@pytest.mark.parametrize("n,q_list,batch", [(1024, [12289], 300), (1024, [12289, 7681], 129), (1024, [3329], 1),
                                            (2048, [12289], 200), (1024, [12289], 128)])
def test_shared_against_oracle(pm, n, q_list, batch):
    rng = np.random.default_rng(n + batch)
    a = wl.uniform_coeffs(rng, 1, q_list, n, np.uint32)[0]
    b = wl.uniform_coeffs(rng, batch, q_list, n, np.uint32)
    with pm.Plan(n, q_list, path=pm.PATH_TENSOR) as plan:
        assert plan.info["digits"] == 2
        got = _run(pm, plan, a, b)
    assert_equal_residues(got, _want(a, b, q_list), "n=%d k=%d batch=%d" % (n, len(q_list), batch))


@pytest.mark.parametrize("n", [1024, 2048])
def test_shared_cyclic(pm, n):
    rng = np.random.default_rng(n + 5)
    q_list = [12289]
    a = wl.uniform_coeffs(rng, 1, q_list, n, np.uint32)[0]
    b = wl.uniform_coeffs(rng, 70, q_list, n, np.uint32)
    with pm.Plan(n, q_list, path=pm.PATH_TENSOR, flags=pm.FLAG_CYCLIC) as plan:
        got = _run(pm, plan, a, b)
    assert_equal_residues(got, _want(a, b, q_list, cyclic=True), "cyclic n=%d" % n)


def test_shared_extremes(pm):
    """All q-1 and the most negative centred value: the largest digit sums."""
    n, q = 1024, 12289
    a = np.full((1, n), q - 1, np.uint32)
    b = np.empty((3, 1, n), np.uint32)
    b[0] = q - 1
    b[1] = q // 2 + 1
    b[2] = q // 2
    with pm.Plan(n, [q], path=pm.PATH_TENSOR) as plan:
        got = _run(pm, plan, a, b)
    assert_equal_residues(got, _want(a, b, [q]), "extremes")
    # (q-1)^2 * x-sum: coefficient j of (sum x^i)^2 mod x^n+1 is 2j+2-n
    assert np.array_equal(got[0, 0].astype(np.int64), np.array([(2 * j + 2 - n) % q for j in range(n)]))


def test_shared_large_batch_sampled(pm):
    """The headline's shape (4096 products): sampled products."""
    w = wl.ring_1024()
    a = w.a[0]
    with pm.Plan(w.n, w.q_list, path=pm.PATH_TENSOR) as plan:
        got = _run(pm, plan, a, w.b)
    idx = [0, 1, 2047, 4095]
    assert_equal_residues(got[idx], _want(a, w.b[idx], w.q_list), "sampled")


def test_shared_reuses_scratch_and_grows(pm):
    n, q = 1024, 12289
    rng = np.random.default_rng(9)
    a = wl.uniform_coeffs(rng, 1, [q], n, np.uint32)[0]
    with pm.Plan(n, [q], path=pm.PATH_TENSOR) as plan:
        for batch in (10, 300, 40):
            b = wl.uniform_coeffs(rng, batch, [q], n, np.uint32)
            assert_equal_residues(_run(pm, plan, a, b), _want(a, b, [q]), "batch %d" % batch)


@pytest.mark.parametrize("n,bits,k,cyclic", [(1024, 14, 1, False), (1024, 30, 2, False), (2048, 31, 1, False),
                                              (4096, 29, 2, True), (8192, 20, 1, False), (1024, 14, 1, True)])
def test_shared_ntt_path(pm, n, bits, k, cyclic):
    """The NTT path: a's transforms once per prime, two transforms per product."""
    rng = np.random.default_rng(n + bits + k)
    q_list = [12289] if bits == 14 else wl.draw_primes(rng, k, bits, bits, n.bit_length())
    a = wl.uniform_coeffs(rng, 1, q_list, n, np.uint32)[0]
    b = wl.uniform_coeffs(rng, 37, q_list, n, np.uint32)
    flags = pm.FLAG_CYCLIC if cyclic else 0
    with pm.Plan(n, q_list, path=pm.PATH_NTT, flags=flags) as plan:
        got = _run(pm, plan, a, b)
        got2 = _run(pm, plan, a, b[:5])  # the counter resets between launches
    want = _want(a, b, q_list, cyclic=cyclic)
    assert_equal_residues(got, want, "ntt n=%d bits=%d" % (n, bits))
    assert_equal_residues(got2, want[:5], "second launch")


def test_shared_unsupported(pm):
    import torch
    x = torch.zeros(1 << 16, dtype=torch.int32, device="cuda")
    for n, q in ((512, 12289), (16384, 65537)):  # NTT path outside 1024 .. 8192
        with pm.Plan(n, [q], path=pm.PATH_NTT) as plan:
            with pytest.raises(pm.PolymulError) as ei:
                pm.polymul_batch_shared(plan.handle, x, x, x, 1)
            assert ei.value.code == pm.POLYMUL_ENOTSUP
    q = wl.draw_primes(np.random.default_rng(1), 1, 30, 30, 1)[0]  # four digits
    with pm.Plan(1024, [q], path=pm.PATH_TENSOR) as plan:
        with pytest.raises(pm.PolymulError) as ei:
            pm.polymul_batch_shared(plan.handle, x, x, x, 1)
        assert ei.value.code == pm.POLYMUL_ENOTSUP

"""Shared-operand products (polymul_batch_shared): c_i = a * b_i for one a,
as the GEMM C = B * T(a) on the tensor cores, against the CPU oracle:
ragged batch tails (not a multiple of the 128-row tile), several moduli,
both rings, both digit widths, extreme operands, and the error cases."""
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


def test_shared_unsupported(pm):
    import torch
    x = torch.zeros(1024, dtype=torch.int32, device="cuda")
    with pm.Plan(1024, [12289], path=pm.PATH_NTT) as plan:
        with pytest.raises(pm.PolymulError) as ei:
            pm.polymul_batch_shared(plan.handle, x, x, x, 1)
        assert ei.value.code == pm.POLYMUL_ENOTSUP
    q = wl.draw_primes(np.random.default_rng(1), 1, 30, 30, 1)[0]  # four digits
    with pm.Plan(1024, [q], path=pm.PATH_TENSOR) as plan:
        with pytest.raises(pm.PolymulError) as ei:
            pm.polymul_batch_shared(plan.handle, x, x, x, 1)
        assert ei.value.code == pm.POLYMUL_ENOTSUP

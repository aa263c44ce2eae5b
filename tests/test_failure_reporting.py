"""A bounded device wait that expires is reported, never returned as a
result.  The expiry is made without any device fault: the diagnostics entry
polymul_selftest_inject_wait makes the next batch-kernel launches expect 16
bytes more than their copies deliver, so their waits give up after a few
polls.  Plans report it through polymul_plan_status, server requests come
back failed with POLYMUL_ETIMEOUT, and the launches after it are exact."""
import numpy as np
import pytest

from oracle import native
from paper_2307_06554_gb300 import workloads as wl

from helpers import assert_equal_residues, from_dev, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pm():
    from paper_2307_06554_gb300 import polymul
    yield polymul
    polymul.polymul_selftest_inject_wait(0, 1)  # nothing left pending for later tests


def _operands(seed, batch, q_list, n, dtype):
    rng = np.random.default_rng(seed)
    return wl.uniform_coeffs(rng, batch, q_list, n, dtype), wl.uniform_coeffs(rng, batch, q_list, n, dtype)


def test_inject_rejects_bad_arguments(pm):
    with pytest.raises(pm.PolymulError) as e:
        pm.polymul_selftest_inject_wait(1, 0)
    assert e.value.code == pm.POLYMUL_EINVAL
    with pytest.raises(pm.PolymulError) as e:
        pm.polymul_selftest_inject_wait(1, (1 << 22) + 1)
    assert e.value.code == pm.POLYMUL_EINVAL


@pytest.mark.parametrize("flags", [0, 16])
def test_plan_reports_expired_wait_and_recovers(pm, flags):
    """Batch 1 takes an expired wait; batch 2, queued right behind it on the
    same plan before anyone looks at the status, is exact (the work counter
    is consistent); the status then reports the expiry once."""
    import torch
    n, q, batch = 1024, 12289, 2048
    a1, b1 = _operands(1, batch, [q], n, np.uint32)
    a2, b2 = _operands(2, batch, [q], n, np.uint32)
    stream = torch.cuda.Stream()
    with pm.Plan(n, [q], flags=flags) as plan:
        ta1, tb1, ta2, tb2 = to_dev(a1), to_dev(b1), to_dev(a2), to_dev(b2)
        c1, c2 = torch.full_like(ta1, -1), torch.full_like(ta1, -1)
        pm.polymul_selftest_inject_wait(1, 64)
        pm.polymul_batch(plan.handle, ta1, tb1, c1, batch, stream.cuda_stream)
        pm.polymul_batch(plan.handle, ta2, tb2, c2, batch, stream.cuda_stream)
        with pytest.raises(pm.PolymulError) as e:
            pm.polymul_plan_status(plan.handle, stream.cuda_stream)
        assert e.value.code == pm.POLYMUL_ETIMEOUT
        pm.polymul_plan_status(plan.handle, stream.cuda_stream)  # reported once, then clear
        got2 = from_dev(c2, np.uint32)
        assert_equal_residues(got2, native.polymul_batch(a2, b2, [q]), "batch after the expired one")
        # and a fresh batch once the status was read
        c3 = torch.full_like(ta1, -1)
        pm.polymul_batch(plan.handle, ta1, tb1, c3, batch, stream.cuda_stream)
        pm.polymul_plan_status(plan.handle, stream.cuda_stream)
        assert_equal_residues(from_dev(c3, np.uint32), native.polymul_batch(a1, b1, [q]), "fresh batch")


def test_server_request_with_expired_wait_fails(pm):
    """The request whose kernel took an expired wait comes back failed with
    POLYMUL_ETIMEOUT and is counted in `failed`, not `completed`; requests
    after it, on every lane, are exact."""
    import torch
    rng = np.random.default_rng(11)
    pool = wl.draw_primes(rng, 4, 59, 59, 14)
    n, lanes = 4096, 4
    with pm.Server(pool, 8192, device_bytes=256 << 20, lanes=lanes) as srv:
        srv.set_route(pm.ROUTE_STAGED)  # the injected expiry needs the kernel's copy waits
        a, b = _operands(12, 1, [pool[0], pool[2]], n, np.uint64)
        a, b = a[0], b[0]
        ha = torch.from_numpy(a.view(np.int64).copy()).pin_memory()
        hb = torch.from_numpy(b.view(np.int64).copy()).pin_memory()
        hc = torch.zeros_like(ha).pin_memory()
        pm.polymul_selftest_inject_wait(1, 64)
        t = srv.submit(n, [0, 2], ha.numpy(), hb.numpy(), hc.numpy())
        with pytest.raises(pm.PolymulError) as e:
            srv.wait(t, timeout_s=30.0)
        assert e.value.code == pm.POLYMUL_ETIMEOUT
        st = srv.stats(reset=True)
        assert st["failed"] == 1 and st["completed"] == 0, st
        want = native.polymul_batch(a[None], b[None], [pool[0], pool[2]])[0]
        outs = []
        for i in range(2 * lanes):
            c = torch.zeros_like(ha).pin_memory()
            outs.append((srv.submit(n, [0, 2], ha.numpy(), hb.numpy(), c.numpy()), c))
        for tk, c in outs:
            srv.wait(tk, timeout_s=30.0)
            assert_equal_residues(c.numpy().view(np.uint64).reshape(2, n), want, "request after the failure")
        st = srv.stats(reset=True)
        assert st["failed"] == 0 and st["completed"] == 2 * lanes, st

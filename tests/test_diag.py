"""Failure detection without a fault: a device wait with nothing to wait
for gives up after its poll limit and is reported as POLYMUL_ETIMEOUT, and
the CUDA context stays usable afterwards."""
import time

import numpy as np
import pytest

from oracle import native
from paper_2307_06554_gb300 import workloads as wl

from helpers import assert_equal_residues, run_plan_batch


@pytest.fixture(scope="module")
def pm():
    from paper_2307_06554_gb300 import polymul
    return polymul


def test_selftest_rejects_bad_limits(pm):
    for polls in (0, (1 << 22) + 1):
        with pytest.raises(pm.PolymulError) as ei:
            pm.polymul_selftest_wait(polls)
        assert ei.value.code == pm.POLYMUL_EINVAL


@pytest.mark.gpu
def test_bounded_wait_gives_up_and_context_survives(pm):
    t0 = time.time()
    for _ in range(3):
        with pytest.raises(pm.PolymulError) as ei:
            pm.polymul_selftest_wait(1 << 12)
        assert ei.value.code == pm.POLYMUL_ETIMEOUT
    assert time.time() - t0 < 60
    # the context is still usable: an ordinary batch after the expired waits
    rng = np.random.default_rng(3)
    a = wl.uniform_coeffs(rng, 9, [12289], 1024, np.uint32)
    b = wl.uniform_coeffs(rng, 9, [12289], 1024, np.uint32)
    with pm.Plan(1024, [12289]) as plan:
        got = run_plan_batch(plan, a, b)
        pm.polymul_plan_status(plan.handle)
    assert_equal_residues(got, native.polymul_batch(a, b, [12289]), "after the self-test")

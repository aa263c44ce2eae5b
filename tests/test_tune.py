"""Autotuner: every candidate kernel of a plan (NTT with 16, 32 or 8
coefficients per thread per operand, swizzled or padded exchanges, one or
both operands in registers, one CTA or a cluster per product; the tensor
path where it applies) is bit-exact; tuning picks one of them and records it; the on-disk cache is
written and reused by a fresh process."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from oracle import native
from paper_2307_06554_gb300 import workloads as wl

from helpers import assert_equal_residues, run_plan_batch

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pm():
    from paper_2307_06554_gb300 import polymul
    return polymul


@pytest.mark.parametrize("n,bits,elem", [(512, 14, 4), (1024, 14, 4), (2048, 14, 4),
                                         (2048, 30, 4), (4096, 29, 4), (8192, 20, 4), (16384, 30, 4), (16384, 17, 4),
                                         (1024, 59, 8), (4096, 59, 8)])
def test_every_candidate_is_exact(pm, n, bits, elem):
    rng = np.random.default_rng(n + bits)
    if bits == 14:
        q_list = [12289]
    elif bits == 17:
        q_list = [65537]  # the small-q mode at n = 2^14
    else:
        q_list = wl.draw_primes(rng, 2, bits, bits, max(14, n.bit_length() + 1))
    dt = np.uint32 if elem == 4 else np.uint64
    a = wl.uniform_coeffs(rng, 7, q_list, n, dt)
    b = wl.uniform_coeffs(rng, 7, q_list, n, dt)
    want = native.polymul_batch(a, b, q_list)
    with pm.Plan(n, q_list) as plan:
        ncand = plan.info["candidates"]
        assert ncand >= 2
        labels = []
        for i in range(ncand):
            info = plan.select(i)
            labels.append((info["path"], info["radix_bits"], info["ntt_mode"], info["regs"], info["tensor_groups"],
                           info["rns_moduli"], info["exchange_pad"], info["one_operand"], info["block"],
                           info["tensor_kernel"], info["digits"]))
            assert_equal_residues(run_plan_batch(plan, a, b), want, "candidate %d %s" % (i, labels[-1]))
    assert len(set(labels)) == ncand


def test_tune_chooses_and_stays_exact(pm):
    w = wl.ring_1024(batch=64, seed=31)
    with pm.Plan(w.n, w.q_list, flags=pm.FLAG_TUNE, tune_batch=4096) as plan:
        assert plan.info["tuned"] == 1 and plan.info["tuned_batch"] == 4096
        got = run_plan_batch(plan, w.a, w.b)
    assert_equal_residues(got, native.polymul_batch(w.a, w.b, w.q_list), "tuned")


def test_tune_cache_file_is_written_and_reused(pm, tmp_path):
    cache = tmp_path / "tune.txt"
    script = (
        "import sys, json; sys.path.insert(0, %r)\n"
        "from paper_2307_06554_gb300 import polymul\n"
        "p = polymul.Plan(1024, [12289]); p.tune(2048); print(json.dumps(p.info)); p.close()\n" % ROOT)
    env = dict(os.environ, POLYMUL_TUNE_CACHE=str(cache))
    r1 = subprocess.run([sys.executable, "-c", script], env=env, capture_output=True, text=True, check=True)
    lines = cache.read_text().strip().splitlines()
    assert len(lines) == 1 and "|n1024|" in lines[0] and "\t" in lines[0]
    r2 = subprocess.run([sys.executable, "-c", script], env=env, capture_output=True, text=True, check=True)
    assert len(cache.read_text().strip().splitlines()) == 1  # the second process used the cache
    i1, i2 = json.loads(r1.stdout.strip()), json.loads(r2.stdout.strip())
    assert (i1["path"], i1["radix_bits"]) == (i2["path"], i2["radix_bits"])


def test_launch_flags(pm):
    """NTT batch kernels take a programmatic dependent launch; the tensor and
    cluster kernels take plain launches."""
    with pm.Plan(1024, [12289], path=pm.PATH_NTT) as plan:
        assert plan.info["launch_flags"] == 2
    with pm.Plan(1024, [12289], path=pm.PATH_TENSOR) as plan:
        assert plan.info["launch_flags"] == 0
    with pm.Plan(32768, wl.draw_primes(np.random.default_rng(3), 1, 30, 30, 16)) as plan:
        assert plan.info["launch_flags"] == 0  # the thread-block cluster kernel

"""Small, self-contained launches of each kernel family, for profilers.

    python -m paper_2307_06554_gb300.probes.cases <case> [--launches K]

Every case builds its plan through the public binding, fills the operands
with seeded uniform residues, runs K launches on one stream (operands
rotated over buffer sets larger than L2, so DRAM counters mean something)
and checks the plan's device status.  Device memory stays below 1 GB.

cases:
  ntt_ring1024     n = 1024, q = 12289, 4096 products (path a, default kernel)
  tensor_ring1024  the same batch through the Toeplitz tensor-core path
  tensor_rns4096   n = 4096, 8 primes of 30 bits, 64 products on the tiled
                   tensor kernel (5 digits, 4 output groups per product)
  tensor_u64_4096  n = 4096, 2 primes of 59 bits, 64 products on the tensor
                   path's residue-number-system kernel (21 small moduli)
  n16384           n = 16384, one 30-bit prime, 1024 products (one CTA per product)
  cluster_32768    n = 32768, one 30-bit prime, 256 products (thread-block clusters)
  u64_4096         n = 4096, one 59-bit prime, 1024 products (64-bit words)
  ragged_300       the first 300 products of the uneven 2000-product list
                   (n 1024..16384, 1..16 primes), one persistent launch
  shared_ring1024  one a times 4096 b's (n = 1024, q = 12289) as the
                   tensor-core GEMM of polymul_batch_shared
  shared_ntt1024   the same on the NTT path (a's transform once)
"""
from __future__ import annotations

import argparse
import math
import sys

import numpy as np

from .. import polymul
from .. import workloads as wl

L2_BYTES = 129 * 1024 * 1024


def _homogeneous(n, q_list, batch, path, launches, seed=7):
    import torch
    dev = torch.device("cuda", 0)
    rng = np.random.default_rng(seed)
    a = wl.uniform_coeffs(rng, batch, q_list, n)
    b = wl.uniform_coeffs(rng, batch, q_list, n)
    view = np.int32 if a.dtype == np.uint32 else np.int64
    ta = torch.from_numpy(a.view(view)).to(dev)
    tb = torch.from_numpy(b.view(view)).to(dev)
    nsets = max(1, math.ceil(1.5 * L2_BYTES / (3 * ta.numel() * ta.element_size())))
    sets = [(ta.clone(), tb.clone(), torch.empty_like(ta)) for _ in range(nsets)]
    stream = torch.cuda.Stream(dev)
    with polymul.Plan(n, q_list, path=path) as plan:
        for i in range(launches):
            x, y, z = sets[i % nsets]
            polymul.polymul_batch(plan.handle, x, y, z, batch, stream.cuda_stream)
        stream.synchronize()
        polymul.polymul_plan_status(plan.handle, stream.cuda_stream)
        info = plan.info
    return {"n": n, "k": len(q_list), "batch": batch, "launches": launches, "grid": info["grid"],
            "block": info["block"], "smem_bytes": info["smem_bytes"], "sets": nsets}


def _ragged(count, launches):
    import torch
    dev = torch.device("cuda", 0)
    rag = wl.ragged_2000(count=count)
    total = sum(p.n * len(p.prime_idx) for p in rag.products)
    ah = np.concatenate([p.a.reshape(-1) for p in rag.products]).astype(np.uint32)
    bh = np.concatenate([p.b.reshape(-1) for p in rag.products]).astype(np.uint32)
    assert ah.size == total
    stream = torch.cuda.Stream(dev)
    with polymul.Ragged(rag.pool, 16384, [(p.n, p.prime_idx) for p in rag.products]) as r:
        ta = torch.from_numpy(ah.view(np.int32)).to(dev)
        tb = torch.from_numpy(bh.view(np.int32)).to(dev)
        tc = torch.empty_like(ta)
        for _ in range(launches):
            r.run(ta, tb, tc, stream=stream.cuda_stream)
        stream.synchronize()
        polymul.polymul_ragged_status(r.batch, stream.cuda_stream)
        info = r.info
    return {"products": count, "words": total, "launches": launches, **info}


def _shared(n, q, batch, launches, seed=7, path=polymul.PATH_TENSOR):
    import torch
    dev = torch.device("cuda", 0)
    rng = np.random.default_rng(seed)
    a = wl.uniform_coeffs(rng, 1, [q], n)[0]
    b = wl.uniform_coeffs(rng, batch, [q], n)
    ta = torch.from_numpy(a.view(np.int32)).to(dev)
    tb = torch.from_numpy(b.view(np.int32)).to(dev)
    nsets = max(1, math.ceil(1.5 * L2_BYTES / (2 * tb.numel() * 4)))
    sets = [(tb.clone(), torch.empty_like(tb)) for _ in range(nsets)]
    stream = torch.cuda.Stream(dev)
    with polymul.Plan(n, [q], path=path) as plan:
        for i in range(launches):
            x, y = sets[i % nsets]
            polymul.polymul_batch_shared(plan.handle, ta, x, y, batch, stream.cuda_stream)
        stream.synchronize()
        polymul.polymul_plan_status(plan.handle, stream.cuda_stream)
    return {"n": n, "batch": batch, "launches": launches, "sets": nsets}


def main(argv=None):
    p = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    p.add_argument("case", choices=["ntt_ring1024", "tensor_ring1024", "tensor_rns4096", "tensor_u64_4096", "n16384",
                                    "cluster_32768", "u64_4096", "ragged_300", "shared_ring1024", "shared_ntt1024"])
    p.add_argument("--launches", type=int, default=4)
    args = p.parse_args(argv)
    rng = np.random.default_rng(8)
    if args.case == "ntt_ring1024":
        res = _homogeneous(1024, [12289], 4096, polymul.PATH_NTT, args.launches)
    elif args.case == "tensor_ring1024":
        res = _homogeneous(1024, [12289], 4096, polymul.PATH_TENSOR, args.launches)
    elif args.case == "tensor_rns4096":
        res = _homogeneous(4096, wl.draw_primes(rng, 8, 30, 30, 13), 64, polymul.PATH_TENSOR, args.launches)
    elif args.case == "tensor_u64_4096":
        res = _homogeneous(4096, wl.draw_primes(rng, 2, 59, 59, 13), 64, polymul.PATH_TENSOR, args.launches)
    elif args.case == "n16384":
        res = _homogeneous(16384, wl.draw_primes(rng, 1, 30, 30, 15), 1024, polymul.PATH_NTT, args.launches)
    elif args.case == "cluster_32768":
        res = _homogeneous(32768, wl.draw_primes(rng, 1, 30, 30, 16), 256, polymul.PATH_NTT, args.launches)
    elif args.case == "u64_4096":
        res = _homogeneous(4096, wl.draw_primes(rng, 1, 59, 59, 13), 1024, polymul.PATH_NTT, args.launches)
    elif args.case == "shared_ring1024":
        res = _shared(1024, 12289, 4096, args.launches)
    elif args.case == "shared_ntt1024":
        res = _shared(1024, 12289, 4096, args.launches, path=polymul.PATH_NTT)
    else:
        res = _ragged(300, args.launches)
    print(args.case, res)
    return 0


if __name__ == "__main__":
    sys.exit(main())

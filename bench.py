#!/usr/bin/env python3
"""Throughput benchmark: exact negacyclic products/s on one GB300.

Workload (one "step"): one batch of 4096 products in Z_q[x]/(x^n+1) with
n = 1024, q = 12289, coefficients uniform in [0, q) stored as 32-bit words
(seeded synthetic data), computed by the library's tuned path through the
C-ABI (polymul_batch on device buffers).

Printed: ONE JSON line with the device-timed throughput (``value``), the
end-to-end throughput through the host-buffer entry point (``e2e``), the
roofline of the dominant kernel, the CPU-oracle baseline and the SM clocks
sampled during the timed region.

``--impl reference`` times the CPU oracle (plain C schoolbook on the host
cores) on the same metric and workload instead; under torchrun only rank 0
runs it.

Multi-GPU: one process per GPU (torchrun); every rank runs an independent
replica of the workload (the products are independent, nothing is
exchanged), ``value`` counts the products of all ranks over the slowest
rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# The serving leg runs 8 lanes of three streams each (copies in, kernels,
# copies out); with the default 8 hardware queues, streams share queues and
# one lane's copies wait behind another lane's kernels.  Must be set before
# the CUDA context exists (measured: saturated 1.31 -> 1.21 s).
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

METRIC = "negacyclic polymul products/s per (n,q), tensor vs NTT, bit-exact; % roofline"
WORKLOAD = "ring_1024: n=1024, q=12289 (q = 1 mod 2n), batch 4096 pairs, coefficients uniform in [0,q) int32, seed 2"
L2_BYTES = 129 * 1024 * 1024
# Integer multiply-add lanes per SM per clock (IMAD issues on one FMA
# datapath: 16 lanes per SM sub-partition, 4 sub-partitions); the high-half
# multiply (IMAD.HI) runs at half that rate.
IMAD_LANES_PER_SM = 64
# IMAD-lane slots per 32-bit Shoup modular multiplication: high product (2),
# low product (1), multiply-subtract (1).  Peak = 16 mulmod/clk/SM, which a
# dependency-free microbenchmark of the same sequence reproduces (5.02e12/s
# at 2070 MHz on 152 SMs).
IMAD_SLOTS_PER_MULMOD = 4
# 64-bit Shoup modular multiplications per second on one GB300, measured by
# `python bench.py --case alu_peak` (profiles/alu_peak.md): the ALU ceiling of
# the kernels on 64-bit words (4.11x the cost of a 32-bit one), scaled by the
# SM clock at which it was taken (2070 MHz)
SHOUP64_PER_S = 1.2227e12
SHOUP64_MHZ = 2070.0
MODE_NAMES = {0: "[0,2q)", 1: "[0,4q)", 2: "small-q"}


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=50)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=10.0, help="CPU oracle sample budget")
    p.add_argument("--no-extras", action="store_true", help="skip the other standing workloads")
    p.add_argument("--case", choices=sorted(CASES), help="run one small profiling case (or the ALU-peak "
                   "microbenchmark) instead of the benchmark, and print what it ran")
    p.add_argument("--launches", type=int, default=4, help="launches of a --case")
    p.add_argument("--karatsuba-model", action="store_true",
                   help="print the tile cost model of one degree-level Karatsuba step on the tensor path (no GPU)")
    return p.parse_args()


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def aggregate_over_ranks(durations, device=None):
    """Per-rank durations -> their maximum over all ranks, element-wise.

    The job is done when its slowest rank is; with one process (or no
    initialised process group) the durations come back unchanged.  The
    all-reduce runs on ``device`` (a CUDA device under NCCL, the CPU under
    gloo)."""
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(x) for x in durations], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.cpu().tolist()]


def job_rate(units_per_rank: float, seconds: float, world_size: int) -> float:
    """Whole-job throughput of independent replicas: every rank processes
    ``units_per_rank`` units, the job takes the slowest rank's ``seconds``."""
    if seconds <= 0:
        raise ValueError("non-positive duration")
    return units_per_rank * world_size / seconds


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def _host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1



# ------------------------------------------------------------------ cases
# Small, self-contained launches of each kernel family for profilers
# (``python bench.py --case <name> [--launches K]``): the plan is built through
# the public binding, operands are seeded uniform residues, K launches run on
# one stream with operands rotated over buffer sets larger than L2 (so DRAM
# counters mean something), and the plan's device status is checked.  Device
# memory stays below 1 GB.
def _case_homogeneous(n, q_list, batch, path, launches, seed=7, flags=0, tensor_kernel=0):
    import torch
    from paper_2307_06554_gb300 import polymul, workloads as wl
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
    with polymul.Plan(n, q_list, path=path, flags=flags) as plan:
        if tensor_kernel:  # a given tensor kernel (polymul_tensor_shape_info.kernel code) instead of the default
            codes = [plan.select(i)["tensor_kernel"] for i in range(plan.info["candidates"])]
            plan.select(codes.index(tensor_kernel))
        for i in range(launches):
            x, y, z = sets[i % nsets]
            polymul.polymul_batch(plan.handle, x, y, z, batch, stream.cuda_stream)
        stream.synchronize()
        polymul.polymul_plan_status(plan.handle, stream.cuda_stream)
        info = plan.info
    return {"n": n, "k": len(q_list), "batch": batch, "launches": launches, "grid": info["grid"],
            "block": info["block"], "smem_bytes": info["smem_bytes"], "sets": nsets}


def _case_mapped(n, q_list, batch, launches, seed=7):
    """polymul_batch_mapped on page-locked host buffers (the direct form of
    the batch kernel), launches back to back on one stream over host sets
    rotated beyond L2."""
    import torch
    from paper_2307_06554_gb300 import polymul, workloads as wl
    rng = np.random.default_rng(seed)
    a = wl.uniform_coeffs(rng, batch, q_list, n)
    b = wl.uniform_coeffs(rng, batch, q_list, n)
    view = np.int32 if a.dtype == np.uint32 else np.int64
    nsets = max(1, math.ceil(1.5 * L2_BYTES / (3 * a.nbytes)))
    sets = [(torch.from_numpy(np.roll(a, s, axis=0).view(view)).pin_memory(),
             torch.from_numpy(np.roll(b, s, axis=0).view(view)).pin_memory(),
             torch.empty(a.shape, dtype=torch.int32 if view is np.int32 else torch.int64).pin_memory())
            for s in range(nsets)]
    stream = torch.cuda.Stream()
    with polymul.Plan(n, q_list, flags=polymul.FLAG_OVERLAP) as plan:
        for i in range(launches):
            x, y, z = sets[i % nsets]
            polymul.polymul_batch_mapped(plan.handle, x, y, z, batch, stream.cuda_stream)
        stream.synchronize()
        polymul.polymul_plan_status(plan.handle, stream.cuda_stream)
    return {"n": n, "k": len(q_list), "batch": batch, "launches": launches, "sets": nsets}


def _case_ragged(count, launches):
    import torch
    from paper_2307_06554_gb300 import polymul, workloads as wl
    dev = torch.device("cuda", 0)
    rag = wl.ragged_2000(count=count)
    total = sum(p.n * len(p.prime_idx) for p in rag.products)
    ah = np.concatenate([p.a.reshape(-1) for p in rag.products]).astype(np.uint32)
    bh = np.concatenate([p.b.reshape(-1) for p in rag.products]).astype(np.uint32)
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


def _case_shared(n, q, batch, launches, path, seed=7):
    import torch
    from paper_2307_06554_gb300 import polymul, workloads as wl
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


# Integer- and tensor-pipe ceilings the rooflines are reported against (the
# measured peaks cover HBM and cuBLAS bf16 only).  Each thread runs 8
# independent chains of one operation, no memory traffic inside the loop, the
# grid filling every SM; the MMA operations run 8 independent accumulator
# chains per warp.
ALU_PROBE_SRC = r"""
#include <cstdint>
#include <cstdio>
#include <cuda_runtime.h>
#define CHAINS 8
#define UNROLL 16
template <int OP>
__global__ void k_probe(uint64_t* out, uint64_t w, uint64_t wp, uint64_t q, int iters) {
  uint32_t x[CHAINS];
  uint64_t y[CHAINS];
  uint32_t acc[CHAINS][4];
  for (int j = 0; j < CHAINS; ++j) {
    x[j] = threadIdx.x * 131u + j;
    y[j] = threadIdx.x * 131ull + j;
    for (int r = 0; r < 4; ++r) acc[j][r] = j + r;
  }
  const uint32_t w32 = (uint32_t)w, wp32 = (uint32_t)wp, q32 = (uint32_t)q;
  const uint32_t fa0 = threadIdx.x * 0x01010101u, fa1 = fa0 ^ 0x5a5a5a5au, fa2 = fa0 + 7u, fa3 = fa0 ^ 0x33u;
  const uint32_t fb0 = threadIdx.x * 0x00ff00ffu, fb1 = fb0 ^ 0x12345678u;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < UNROLL; ++u)
#pragma unroll
      for (int j = 0; j < CHAINS; ++j) {
        if (OP == 0) x[j] = x[j] * w32 + wp32;                                       // IMAD
        if (OP == 1) x[j] = __umulhi(x[j], wp32) ^ x[j];                             // IMAD.HI (+LOP)
        if (OP == 2) x[j] = x[j] * w32 - __umulhi(x[j], wp32) * q32;                 // 32-bit Shoup
        if (OP == 3) y[j] = y[j] * w - __umul64hi(y[j], wp) * q;                     // 64-bit Shoup
        if (OP == 4) x[j] = x[j] * w32 - ((x[j] * wp32) >> 16) * q32;                // Shoup, 16-bit quotient
        if (OP == 5)                                                                 // mma.sync u8 -> s32
          asm volatile("mma.sync.aligned.m16n8k32.row.col.s32.u8.u8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                       "{%0,%1,%2,%3};"
                       : "+r"(acc[j][0]), "+r"(acc[j][1]), "+r"(acc[j][2]), "+r"(acc[j][3])
                       : "r"(fa0), "r"(fa1), "r"(fa2), "r"(fa3), "r"(fb0), "r"(fb1));
        if (OP == 6)                                                                 // mma.sync bf16 -> f32
          asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                       "{%0,%1,%2,%3};"
                       : "+r"(acc[j][0]), "+r"(acc[j][1]), "+r"(acc[j][2]), "+r"(acc[j][3])
                       : "r"(fa0 & 0x3f803f80u), "r"(fa1 & 0x3f803f80u), "r"(fa2 & 0x3f803f80u),
                         "r"(fa3 & 0x3f803f80u), "r"(fb0 & 0x3f803f80u), "r"(fb1 & 0x3f803f80u));
      }
  }
  uint64_t r = 0;
  for (int j = 0; j < CHAINS; ++j) r ^= x[j] ^ y[j] ^ acc[j][0] ^ acc[j][1] ^ acc[j][2] ^ acc[j][3];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = r;
}
int main() {
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int threads = 256, blocks = sms * 8, iters = 2048;
  uint64_t* out = nullptr;
  if (cudaMalloc(&out, sizeof(uint64_t) * threads * blocks) != cudaSuccess) return 1;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const double per_thread = (double)iters * UNROLL * CHAINS;
  const char* names[] = {"imad32", "imad32_hi", "shoup32_mulmod", "shoup64_mulmod", "shoup16q_mulmod",
                         "mma_sync_u8_s32_ops", "mma_sync_bf16_f32_flops"};
  const uint64_t W32 = 5000, WP32 = (uint64_t)((5000ull << 32) / 12289), Q32 = 12289;
  const uint64_t Q64 = 288230376151760897ull, W64 = (1ull << 40) + 7;
  const uint64_t WP64 = (uint64_t)(((unsigned __int128)W64 << 64) / Q64);
  const uint64_t WP16 = (5000ull << 16) / 12289;  // x stays below 2q < 2^16 along each chain
  printf("{\"sms\": %d, \"results\": [", sms);
  for (int op = 0; op < 7; ++op) {
    float best = 1e30f;
    const int it = op == 3 ? iters / 4 : (op >= 5 ? iters / 8 : iters);
    for (int rep = 0; rep < 3; ++rep) {
      cudaEventRecord(e0);
      if (op == 0) k_probe<0><<<blocks, threads>>>(out, W32, WP32, Q32, it);
      if (op == 1) k_probe<1><<<blocks, threads>>>(out, W32, WP32, Q32, it);
      if (op == 2) k_probe<2><<<blocks, threads>>>(out, W32, WP32, Q32, it);
      if (op == 3) k_probe<3><<<blocks, threads>>>(out, W64, WP64, Q64, it);
      if (op == 4) k_probe<4><<<blocks, threads>>>(out, W32, WP16, Q32, it);
      if (op == 5) k_probe<5><<<blocks, threads>>>(out, W32, WP32, Q32, it);
      if (op == 6) k_probe<6><<<blocks, threads>>>(out, W32, WP32, Q32, it);
      cudaEventRecord(e1);
      cudaEventSynchronize(e1);
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) best = ms;
    }
    double n = (double)threads * blocks * per_thread * it / iters;
    if (op == 5) n = n / 32 * (2.0 * 16 * 8 * 32);   // per warp-MMA: 16x8x32 MACs
    if (op == 6) n = n / 32 * (2.0 * 16 * 8 * 16);
    printf("%s{\"op\": \"%s\", \"per_s\": %.4e}", op ? ", " : "", names[op], n / (best * 1e-3));
  }
  printf("], \"error\": \"%s\"}\n", cudaGetErrorString(cudaGetLastError()));
  cudaFree(out);
  return 0;
}
"""


# Host-link microbenchmark (`python bench.py --case host_link`,
# profiles/host_link.md): page-locked host <-> device traffic by the copy
# engines (cudaMemcpyAsync, one direction and both at once) and by SM loads
# and stores on mapped page-locked memory (one direction, and the 2:1 mix of
# a polynomial product: two operand rows in, one result row out).  The
# second is the route of polymul_batch_host's direct form.  Buffers of
# 256 MB in and 128 MB out, beyond L2.
LINK_PROBE_SRC = r"""
#include <cstdio>
#include <cstdint>
#include <cuda_runtime.h>
#define CK(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) { printf("{\"error\": \"%s\"}\n", cudaGetErrorString(e_)); return 1; } } while (0)
__global__ void copy16(const uint4* __restrict__ src, uint4* __restrict__ dst, size_t n16) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += stride) dst[i] = src[i];
}
__global__ void mix16(const uint4* __restrict__ a, const uint4* __restrict__ b, uint4* __restrict__ c, size_t n16) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += stride) {
    const uint4 x = a[i], y = b[i];
    c[i] = make_uint4(x.x ^ y.x, x.y ^ y.y, x.z ^ y.z, x.w ^ y.w);
  }
}
struct Ctx { cudaStream_t s, s2; cudaEvent_t fork, join; char *hin, *hout, *din, *dout; size_t nin, nout; int grid; };
static void run(Ctx& c, int what) {
  switch (what) {
    case 0: cudaMemcpyAsync(c.din, c.hin, c.nin, cudaMemcpyHostToDevice, c.s); break;
    case 1: cudaMemcpyAsync(c.hout, c.dout, c.nout, cudaMemcpyDeviceToHost, c.s); break;
    case 2:
      cudaEventRecord(c.fork, c.s); cudaStreamWaitEvent(c.s2, c.fork, 0);
      cudaMemcpyAsync(c.din, c.hin, c.nin, cudaMemcpyHostToDevice, c.s);
      cudaMemcpyAsync(c.hout, c.dout, c.nout, cudaMemcpyDeviceToHost, c.s2);
      cudaEventRecord(c.join, c.s2); cudaStreamWaitEvent(c.s, c.join, 0);
      break;
    case 3: copy16<<<c.grid, 512, 0, c.s>>>((const uint4*)c.hin, (uint4*)c.din, c.nin / 16); break;
    case 4: copy16<<<c.grid, 512, 0, c.s>>>((const uint4*)c.dout, (uint4*)c.hout, c.nout / 16); break;
    default: mix16<<<c.grid, 512, 0, c.s>>>((const uint4*)c.hin, (const uint4*)(c.hin + c.nout), (uint4*)c.hout, c.nout / 16);
  }
}
int main() {
  Ctx c{};
  c.nin = 256u << 20; c.nout = 128u << 20;
  int sms = 0; CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0));
  c.grid = 4 * sms;
  CK(cudaHostAlloc((void**)&c.hin, c.nin, cudaHostAllocMapped));
  CK(cudaHostAlloc((void**)&c.hout, c.nout, cudaHostAllocMapped));
  CK(cudaMalloc((void**)&c.din, c.nin)); CK(cudaMalloc((void**)&c.dout, c.nout));
  for (size_t i = 0; i < c.nin; i += 4096) c.hin[i] = 1;
  CK(cudaMemset(c.dout, 2, c.nout));
  CK(cudaStreamCreateWithFlags(&c.s, cudaStreamNonBlocking)); CK(cudaStreamCreateWithFlags(&c.s2, cudaStreamNonBlocking));
  CK(cudaEventCreateWithFlags(&c.fork, cudaEventDisableTiming)); CK(cudaEventCreateWithFlags(&c.join, cudaEventDisableTiming));
  cudaEvent_t e0, e1; CK(cudaEventCreate(&e0)); CK(cudaEventCreate(&e1));
  const char* names[] = {"copy_engine_h2d", "copy_engine_d2h", "copy_engine_both", "sm_load_host", "sm_store_host", "sm_mix_2in_1out"};
  const double bytes[] = {(double)c.nin, (double)c.nout, (double)(c.nin + c.nout), (double)c.nin, (double)c.nout, 3.0 * c.nout};
  printf("{\"sms\": %d, \"results\": [", sms);
  for (int w = 0; w < 6; ++w) {
    for (int r = 0; r < 2; ++r) run(c, w);
    CK(cudaEventRecord(e0, c.s));
    for (int r = 0; r < 5; ++r) run(c, w);
    CK(cudaEventRecord(e1, c.s));
    CK(cudaEventSynchronize(e1));
    float ms = 0; CK(cudaEventElapsedTime(&ms, e0, e1));
    printf("%s{\"op\": \"%s\", \"GBs\": %.1f}", w ? ", " : "", names[w], bytes[w] * 5 / (ms * 1e-3) / 1e9);
  }
  printf("], \"error\": \"%s\"}\n", cudaGetErrorString(cudaGetLastError()));
  return 0;
}
"""


def _case_host_link():
    from paper_2307_06554_gb300 import build as _build
    work = tempfile.mkdtemp()
    src = os.path.join(work, "host_link.cu")
    exe = os.path.join(work, "host_link")
    with open(src, "w") as f:
        f.write(LINK_PROBE_SRC)
    subprocess.check_call([_build.nvcc()] + _build.ARCH + ["-O3", "-o", exe, src])
    return json.loads(subprocess.run([exe], capture_output=True, text=True, check=True).stdout)


def _case_alu_peak():
    from paper_2307_06554_gb300 import build as _build
    work = tempfile.mkdtemp()
    src = os.path.join(work, "alu_peak.cu")
    exe = os.path.join(work, "alu_peak")
    with open(src, "w") as f:
        f.write(ALU_PROBE_SRC)
    subprocess.check_call([_build.nvcc()] + _build.ARCH + ["-O3", "-o", exe, src])
    smi = subprocess.Popen(["nvidia-smi", "--query-gpu=clocks.sm,clocks.max.sm", "--format=csv,noheader,nounits",
                            "-lms", "50"], stdout=subprocess.PIPE, text=True)
    out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout
    smi.terminate()
    clocks = [l.split(",") for l in smi.communicate()[0].splitlines() if "," in l]
    res = json.loads(out)
    res["sm_mhz_max_seen"] = max(float(c[0]) for c in clocks) if clocks else None
    mhz = res["sm_mhz_max_seen"] or 2070.0
    for r in res["results"]:
        r["per_sm_per_clk"] = r["per_s"] / res["sms"] / (mhz * 1e6)
    return res


def _case(name, launches):
    from paper_2307_06554_gb300 import polymul, workloads as wl
    rng = np.random.default_rng(8)
    if name == "alu_peak":
        return _case_alu_peak()
    if name == "host_link":
        return _case_host_link()
    if name == "ntt_ring1024":
        return _case_homogeneous(1024, [12289], 4096, polymul.PATH_NTT, launches)
    if name == "mapped_ring1024":
        return _case_mapped(1024, [12289], 4096, launches)
    if name == "ntt_ring1024_overlap":
        return _case_homogeneous(1024, [12289], 4096, polymul.PATH_NTT, launches, flags=polymul.FLAG_OVERLAP)
    if name == "tensor_ring1024":
        return _case_homogeneous(1024, [12289], 4096, polymul.PATH_TENSOR, launches)
    if name == "tensor_rns4096":
        return _case_homogeneous(4096, wl.draw_primes(rng, 8, 30, 30, 13), 64, polymul.PATH_TENSOR, launches)
    if name == "tensor_rns4096_pipelined":
        return _case_homogeneous(4096, wl.draw_primes(rng, 8, 30, 30, 13), 64, polymul.PATH_TENSOR, launches,
                                 tensor_kernel=5)
    if name == "tensor_u64_16384":
        return _case_homogeneous(16384, wl.draw_primes(rng, 2, 59, 59, 15), 8, polymul.PATH_TENSOR, launches)
    if name == "tensor_u64_4096":
        return _case_homogeneous(4096, wl.draw_primes(rng, 2, 59, 59, 13), 64, polymul.PATH_TENSOR, launches)
    if name == "n16384":
        return _case_homogeneous(16384, wl.draw_primes(rng, 1, 30, 30, 15), 1024, polymul.PATH_NTT, launches)
    if name == "cluster_32768":
        return _case_homogeneous(32768, wl.draw_primes(rng, 1, 30, 30, 16), 256, polymul.PATH_NTT, launches)
    if name == "u64_4096":
        return _case_homogeneous(4096, wl.draw_primes(rng, 1, 59, 59, 13), 1024, polymul.PATH_NTT, launches)
    if name == "shared_ring1024":
        return _case_shared(1024, 12289, 4096, launches, polymul.PATH_TENSOR)
    if name == "shared_ntt1024":
        return _case_shared(1024, 12289, 4096, launches, polymul.PATH_NTT)
    return _case_ragged(300, launches)


CASES = {
    "alu_peak": "integer- and tensor-pipe microbenchmark (IMAD, Shoup 32/64-bit, mma.sync u8 and bf16)",
    "host_link": "host-link microbenchmark: copy engines and SM loads/stores on mapped page-locked memory",
    "ntt_ring1024": "n = 1024, q = 12289, 4096 products (path a, default kernel)",
    "ntt_ring1024_overlap": "the same with POLYMUL_FLAG_OVERLAP",
    "mapped_ring1024": "the same batch from page-locked host buffers through polymul_batch_mapped (direct form)",
    "tensor_ring1024": "the same batch through the Toeplitz tensor-core path",
    "tensor_rns4096": "n = 4096, 8 primes of 30 bits, 64 products on the tiled tensor kernel",
    "tensor_rns4096_pipelined": "the same on the warp-specialised pipeline form of the drained kernel",
    "tensor_u64_4096": "n = 4096, 2 primes of 59 bits, 64 products on the residue-number-system tensor kernel",
    "tensor_u64_16384": "n = 16384, 2 primes of 59 bits, 8 products on the 64-bit-word digit kernel",
    "n16384": "n = 16384, one 30-bit prime, 1024 products (one CTA per product)",
    "cluster_32768": "n = 32768, one 30-bit prime, 256 products (thread-block clusters)",
    "u64_4096": "n = 4096, one 59-bit prime, 1024 products (64-bit words)",
    "ragged_300": "the first 300 products of the uneven 2000-product list, one persistent launch",
    "shared_ring1024": "one a times 4096 b's (n = 1024, q = 12289), tensor-core GEMM",
    "shared_ntt1024": "the same on the NTT path (a's transform once)",
}

# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "100", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        try:
            with open(self.path) as f:
                for line in f:
                    parts = [x.strip() for x in line.split(",")]
                    if len(parts) >= 9:
                        rows.append(parts)
            os.unlink(self.path)
        except Exception:
            return None
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


def _tensor_digits(n: int, qmax: int):
    """Digit width and count of the tensor path (mirrors the plan's rule:
    n 2^(2w-2) <= 2^24, w <= 8, L balanced digits in [-2^(w-1), 2^(w-1))
    reach floor(q/2))."""
    logn = n.bit_length() - 1
    w = min(8, (24 - logn) // 2 + 1)
    L = next(l for l in range(1, 9)
             if ((1 << (w - 1)) - 1) * ((1 << (w * l)) - 1) // ((1 << w) - 1) >= qmax // 2)
    return w, L


# ------------------------------------------------------------------ traffic record
def _kernel_source_hash() -> str:
    h = hashlib.sha256()
    for fn in ("ntt.cuh", "arith.cuh", "async.cuh", "ntt_info.cuh", "polymul_types.h"):
        with open(os.path.join(ROOT, "paper_2307_06554_gb300", "csrc", fn), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def _recorded_traffic(kernel_tag: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "ntt_ring1024_traffic.txt")
    try:
        kv = {}
        with open(path) as f:
            for line in f:
                if "=" in line and not line.startswith("#"):
                    k, v = line.strip().split("=", 1)
                    kv[k.strip()] = v.strip()
        if kv.get("kernel") == kernel_tag and kv.get("source_sha") == _kernel_source_hash():
            return float(kv["dram_bytes_per_launch"])
    except Exception:
        pass
    return None


# ------------------------------------------------------------------ CPU oracle leg
class Samples:
    """GPU outputs of sampled products, kept for the CPU oracle leg to check
    (the GPU legs never call the oracle themselves)."""

    def __init__(self):
        self.rows = []    # (name, a [m][k][n], b [m][k][n], q_list, got [m][k][n])
        self.coeffs = []  # (name, a [n], b [n], q, coefficient indices, got)

    def add(self, name, a, b, q_list, got, cyclic=False):
        self.rows.append((name, np.asarray(a), np.asarray(b), list(q_list), np.asarray(got, dtype=np.uint64),
                          cyclic))

    def add_coeffs(self, name, a, b, q, js, got):
        self.coeffs.append((name, np.asarray(a), np.asarray(b), int(q), list(js), np.asarray(got, dtype=np.uint64)))

    def check(self):
        """name -> every sample of that name equals the oracle's result."""
        from oracle import native
        ok = {}
        for name, a, b, q_list, got, cyclic in self.rows:
            want = native.polymul_batch(a, b, q_list, cyclic=cyclic)
            ok[name] = ok.get(name, True) and bool(np.array_equal(got.reshape(want.shape), want))
        for name, a, b, q, js, got in self.coeffs:
            ok[name] = ok.get(name, True) and bool(np.array_equal(got, native.coeffs(a, b, q, js)))
        return ok


def cpu_oracle_rate(w, seconds: float, max_products: int = None):
    """The oracle as it stands (plain C schoolbook, one thread per host core)
    on whole batches of the workload, repeated until ``seconds`` elapsed."""
    from oracle import native
    threads = _host_cores()
    a, b = w.a, w.b
    if max_products:
        a, b = a[:max_products], b[:max_products]
    done = 0
    t0 = time.perf_counter()
    while True:
        native.polymul_batch(a, b, w.q_list, threads=threads)
        done += a.shape[0]
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    return done / el, threads, done, el


def _ntt_mulmods(n: int) -> int:
    """Algorithmic modular multiplications of one NTT unit, the scope table's
    count: two forward transforms, one inverse, the pointwise product."""
    return 3 * (n // 2) * int(math.log2(n)) + n


def _ntt_mulmods_kernel(n: int) -> int:
    """What the kernels execute: the above plus the last inverse stage's
    scaling by n^-1 of the half of the outputs that carries no twiddle."""
    return _ntt_mulmods(n) + n // 2


def _alu_peak_g(elem: int, sms: int, sm_mhz: float) -> float:
    """ALU ceiling in Gmulmod/s for the kernels on `elem`-byte words."""
    if elem == 8:
        return SHOUP64_PER_S * (sm_mhz / SHOUP64_MHZ) / 1e9
    return sms * IMAD_LANES_PER_SM * sm_mhz * 1e6 / IMAD_SLOTS_PER_MULMOD / 1e9


# Shared-memory bytes a tcgen05 MMA of the tensor path reads per instruction:
# the A slice (128 rows x 16 bf16) and the B slice (N rows x 16 bf16).  The
# A operand is the aliased Hankel view of a's digits, re-read by every MMA,
# so shared-memory bandwidth (128 B/clk/SM, nominal) bounds the path before
# the tensor pipe does.
SMEM_BYTES_PER_CLK_SM = 128


def _host_link(dev, h2d_bytes, d2h_bytes, reps=10):
    """Page-locked host <-> device copy bandwidth of this machine, measured now
    with plain copies of the e2e step's sizes: one direction at a time and
    both at once (separate streams); the ceiling for the e2e number."""
    import torch
    h_in = torch.empty(h2d_bytes, dtype=torch.uint8).pin_memory()
    d_in = torch.empty(h2d_bytes, dtype=torch.uint8, device=dev)
    h_out = torch.empty(d2h_bytes, dtype=torch.uint8).pin_memory()
    d_out = torch.empty(d2h_bytes, dtype=torch.uint8, device=dev)
    s1, s2 = torch.cuda.Stream(dev), torch.cuda.Stream(dev)

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            fn()
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) / reps

    def both():
        with torch.cuda.stream(s1):
            d_in.copy_(h_in, non_blocking=True)
        with torch.cuda.stream(s2):
            h_out.copy_(d_out, non_blocking=True)

    t_in = timed(lambda: d_in.copy_(h_in, non_blocking=True))
    t_out = timed(lambda: h_out.copy_(d_out, non_blocking=True))
    t_both = timed(both)
    return {"h2d_GBs": h2d_bytes / t_in / 1e9, "d2h_GBs": d2h_bytes / t_out / 1e9,
            "both_GBs": (h2d_bytes + d2h_bytes) / t_both / 1e9,
            "note": "plain page-locked copies of the step's sizes, measured in this run"}


def _tiled_shifts(n, info, same_digits=True):
    """Shifted copies of b per A slice of a tiled tensor kernel, from the
    plan's output groups: with as many digits on both sides each unit of
    work is one A slice against S shifted copies of b, so the n/1024 output
    blocks of a product split into n/1024/S groups."""
    if not info["tensor_groups"] or not same_digits:
        return 1
    return max(1, max(1, n // 1024) // info["tensor_groups"])


def _rns_shifts(n, r):
    """Shifted copies of b per A slice in the RNS tensor kernel (mirrors its
    tiling: r chains of N = 8 S columns within 512)."""
    s = 1
    while s * 2 <= max(1, n // 1024) and r * 8 * s * 2 <= 512:
        s *= 2
    return s


# ------------------------------------------------------------------ Karatsuba cost model
# Tile cost of the tensor path's matrix form (Sec. 2.2, 2.5), for deciding
# whether one degree-level Karatsuba step (Sec. 4: h0 = a0 b0, h2 = a1 b1,
# h1 = (a0 + a1)(b0 + b1) - h0 - h2, three half-size linear products) pays.
# An MMA covers 128 rows of A (8 outputs each: a block of 1024 outputs) by
# K = 16 by N = 8 x digits of b x shifts (padded to 16); it reads a 4 KB A
# tile and an N x 16 bf16 B tile from shared memory.  The direct negacyclic
# kernels run every (block group, K step) tile; a linear product of size m
# (2m outputs, K = m) can skip the tiles of its Toeplitz matrix that are all
# zero, at that granularity.  Optimistic for Karatsuba: the operand sums
# and the recombination of h0, h1, h2 are counted as free.

def _digit_reach(w, L):
    return ((1 << (w - 1)) - 1) * ((1 << (w * L)) - 1) // ((1 << w) - 1)


def _digits_for(w, bound):
    """Balanced w-bit digits that reach every |x| <= bound."""
    return next(L for L in range(1, 16) if _digit_reach(w, L) >= bound)


def _mma_n(lb, shifts):
    return (8 * lb * shifts + 15) // 16 * 16


def _mma_smem_bytes(nn):
    return 128 * 16 * 2 + nn * 16 * 2


def _linear_tile_needed(m, blocks, k0):
    """Whether the tile of output blocks `blocks` (1024 outputs each) and
    K step [k0, k0 + 16) of a linear product of size m holds a nonzero entry
    (c_j sums a_{j-k} b_k, 0 <= j - k < m, 0 <= k < m)."""
    return any(1024 * o + 1023 - k0 >= 0 and 1024 * o - (k0 + 15) <= m - 1 for o in blocks)


def _linear_tiles(m, shifts):
    nblk = max(1, 2 * m // 1024)
    return sum(_linear_tile_needed(m, range(g, min(nblk, g + shifts)), 16 * c)
               for g in range(0, nblk, shifts) for c in range(m // 16))


def _tile_cost(mmas, nn):
    return {"mmas": mmas, "mma_n": nn, "smem_bytes": mmas * _mma_smem_bytes(nn), "mac_slots": mmas * 128 * 16 * nn}


def karatsuba_model(n, q, la, lb, shifts, ternary_b=False):
    """Per (product, prime): the direct kernel's tiles against one
    Karatsuba step's, with 8-bit digits (the drained kernel's; exact per K
    chunk at any length).  h1's operands are sums of two centred residues
    (|x| <= 2 floor(q/2)): one digit more where that crosses a digit
    boundary; a ternary b's sums stay within one digit."""
    direct = _tile_cost(la * (max(1, n // 1024) // shifts) * (n // 16), _mma_n(lb, shifts))
    m = n // 2
    la1 = la if ternary_b else max(la, _digits_for(8, 2 * (q // 2)))
    lb1 = max(lb, _digits_for(8, 2 * (q // 2)))
    out = {"n": n, "q_bits": q.bit_length(), "digits": [la, lb], "h1_digits": [la1, lb1], "direct": direct}
    for s in sorted({1, shifts}):
        t = _linear_tiles(m, s)
        h02 = _tile_cost(2 * la * t, _mma_n(lb, s))
        h1 = _tile_cost(la1 * t, _mma_n(lb1, s))
        kara = {k: h02[k] + h1[k] for k in ("mmas", "smem_bytes", "mac_slots")}
        kara["tiles_per_linear_product"] = t
        kara["smem_ratio"] = kara["smem_bytes"] / direct["smem_bytes"]
        kara["mac_slot_ratio"] = kara["mac_slots"] / direct["mac_slots"]
        out["karatsuba_shifts_%d" % s] = kara
    return out


KARATSUBA_SHAPES = [
    ("ring_1024 (n = 1024, q = 12289)", 1024, 12289, 2, 2, 1, False),
    ("rns_4096 (n = 4096, 30-bit primes)", 4096, (1 << 30) - 35, 4, 4, 2, False),
    ("rns_4096, ternary b", 4096, (1 << 30) - 35, 1, 4, 1, True),
    ("n = 16384, 30-bit prime", 16384, (1 << 30) - 35, 4, 4, 2, False),
]


def _tensor_smem_roofline(n, digits, units, seconds, sms, sm_mhz, la=None, shifts=1):
    """`digits` of the operand on the MMA's B (Toeplitz) side, `la` (default
    the same) on its A (aliased) side; `shifts` copies of b share one A
    slice (N = 8 digits shifts)."""
    nb = (8 * digits * shifts + 15) // 16 * 16
    la = digits if la is None else la
    # per (product, prime): A-side digits x A slices (128 rows each; one
    # below n = 1024, its rows past n/8 discarded) x K steps of 16
    mmas = la * max(1, n // 1024 // shifts) * (n // 16)
    byts = units * mmas * (128 * 32 + nb * 32)
    peak = sms * SMEM_BYTES_PER_CLK_SM * sm_mhz * 1e6 / 1e9
    ach = byts / seconds / 1e9
    return {"bound": "smem", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
            "bytes_per_launch": byts,
            "peak_source": "derived: %d SMs x %d B/clk x %.0f MHz (shared-memory operand reads of the MMAs)" % (
                sms, SMEM_BYTES_PER_CLK_SM, sm_mhz)}


def _time_steps(step, stream, reps):
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for i in range(reps):
        step(i)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def other_workloads(dev, stream, peaks, alu_peak_g, samples):
    """Throughput of the other standing workloads (not the headline line):
    n=256 q=3329 (auxiliary-prime NTT, launch-latency bound), n=4096 with 8
    RNS primes and ternary b, each also on the tensor path, the headline's
    batch in the cyclic ring x^n - 1, and the 2000-product uneven list (two
    concurrent persistent launches replayed as a CUDA graph)."""
    import torch
    from paper_2307_06554_gb300 import polymul, workloads as wl
    out = {}
    sp = stream.cuda_stream
    hbm = peaks["hbm_gbs"]
    sms = torch.cuda.get_device_properties(dev).multi_processor_count

    def homogeneous(name, w, sets_needed, reps, cyclic=False, path=None, extra_flags=0):
        # tuned plans: back-to-back batches on rotating buffers may overlap
        # tensor plans are tuned over their own kernels (digit forms, RNS)
        flags = ((polymul.FLAG_TUNE | polymul.FLAG_OVERLAP) if path is None else polymul.FLAG_TUNE) | \
            (polymul.FLAG_CYCLIC if cyclic else 0) | extra_flags
        plan = polymul.Plan(w.n, w.q_list, path=polymul.PATH_AUTO if path is None else path, flags=flags,
                            tune_batch=w.batch)
        k = len(w.q_list)
        elem = plan.elem_bytes
        view = np.int32 if elem == 4 else np.int64
        a0 = torch.from_numpy(w.a.view(view)).to(dev)
        b0 = torch.from_numpy(w.b.view(view)).to(dev)
        sets = [(a0.clone(), b0.clone(), torch.empty_like(a0)) for _ in range(sets_needed)]

        def step(i):
            a, b, c = sets[i % len(sets)]
            polymul.polymul_batch(plan.handle, a, b, c, w.batch, sp)
        for i in range(3):
            step(i)
        ms = _time_steps(step, stream, reps)
        idx = [0, w.batch - 1]
        got = sets[(reps - 1) % len(sets)][2][idx].cpu().numpy().view(w.a.dtype)
        samples.add(name, w.a[idx], w.b[idx], w.q_list, got, cyclic=cyclic)
        units = w.batch * k
        mm = units * _ntt_mulmods(w.n)
        byts = 3 * units * w.n * elem
        path = {1: "ntt", 2: "tensor"}.get(plan.info["path"], "?")
        if plan.info["aux_primes"]:
            path += " (auxiliary prime)"
        elif plan.info["path"] == 1:
            path += " (radix %d register passes, autotuned over %d)" % (1 << plan.info["radix_bits"],
                                                                     plan.info["candidates"])
        info = plan.info
        if info["path"] == 2 and info["rns_moduli"]:
            desc = "tensor, residue number system of %d small moduli (%d output groups per product)" % (
                info["rns_moduli"], info["tensor_groups"])
        elif info["path"] == 2:
            desc = "tensor (%d digits of %d bits%s, %s)" % (
                info["digits"], info["digit_bits"], "; b ternary, one digit" if extra_flags & polymul.FLAG_TERNARY_B else "",
                "%d output groups per product" % info["tensor_groups"] if info["tensor_groups"] else "whole product per CTA")
        out[name] = {"products_per_s": w.batch / (ms / 1e3), "us_per_step": ms * 1e3, "batch": w.batch,
                     "n": w.n, "k": k, "path": desc if info["path"] == 2 else path,
                     "hbm_frac": byts / (ms / 1e3) / 1e9 / hbm,
                     "bit_exact_sample": None,
                     "l2": "inputs rotated over %d buffer sets" % len(sets) if len(sets) > 1 else "L2-resident"}
        if info["path"] == 2 and info["rns_moduli"]:
            # one chain per small modulus, N = 16 rows of which 8 carry residues
            flops = 2.0 * w.n * w.n * info["rns_moduli"] * units
            out[name]["tensor_frac_bf16"] = flops / (ms / 1e3) / 1e12 / peaks.get("bf16_tflops", 1911.7)
            out[name]["tensor_frac_smem"] = _tensor_smem_roofline(
                w.n, 1, units, ms / 1e3, sms, peaks.get("sm_max_mhz", 2070.0), la=info["rns_moduli"],
                shifts=_rns_shifts(w.n, info["rns_moduli"]))["frac"]
        elif info["path"] == 2:
            la, lb = (1, info["digits"]) if extra_flags & polymul.FLAG_TERNARY_B else (info["digits"], info["digits"])
            flops = 2.0 * w.n * w.n * la * lb * units
            out[name]["tensor_frac_bf16"] = flops / (ms / 1e3) / 1e12 / peaks.get("bf16_tflops", 1911.7)
            out[name]["tensor_frac_smem"] = _tensor_smem_roofline(
                w.n, info["digits"], units, ms / 1e3, sms, peaks.get("sm_max_mhz", 2070.0), la=la,
                shifts=_tiled_shifts(w.n, info, la == lb))["frac"]
        else:
            peak_g = _alu_peak_g(elem, sms, peaks.get("sm_max_mhz", 2070.0))
            out[name]["alu_frac"] = mm / (ms / 1e3) / 1e9 / peak_g
            out[name]["alu_peak"] = ("measured 64-bit Shoup rate (bench.py --case alu_peak), %.4g Gmulmod/s" % peak_g
                                     if elem == 8 else "derived 32-bit Shoup rate, %.4g Gmulmod/s" % peak_g)
        plan.close()

    homogeneous("ring_small", wl.ring_small(), 1, 200)
    out["ring_small"]["graph_1000"] = graph_replay(dev, wl.ring_small(), 1000)
    homogeneous("ring_small_tensor", wl.ring_small(), 1, 200, path=polymul.PATH_TENSOR)
    homogeneous("rns_4096", wl.rns_4096(), 6, 20)
    homogeneous("rns_4096_tensor", wl.rns_4096(), 6, 5, path=polymul.PATH_TENSOR)
    # its b is ternary: one digit of b, on the MMA's A side
    homogeneous("rns_4096_tensor_ternary_b", wl.rns_4096(), 6, 10, path=polymul.PATH_TENSOR,
                extra_flags=polymul.FLAG_TERNARY_B)
    # 59-bit moduli (the serving workload's prime size) at n = 4096: the NTT
    # path on 64-bit words beside the tensor path's residue-number-system
    # kernel (seed 12)
    rng = np.random.default_rng(12)
    q59 = wl.draw_primes(rng, 2, 59, 59, 13)
    w59 = wl.Batch("u64_4096 n=4096 k=2 59-bit batch=128", 4096, q59, wl.uniform_coeffs(rng, 128, q59, 4096),
                   wl.uniform_coeffs(rng, 128, q59, 4096))
    homogeneous("u64_4096", w59, 6, 20)
    homogeneous("u64_4096_tensor_rns", w59, 6, 5, path=polymul.PATH_TENSOR)
    # the cyclic ring x^n - 1 on the headline's shape and data
    homogeneous("ring_1024_cyclic", wl.ring_1024(), 9, 50, cyclic=True)

    rag = wl.ragged_2000()
    total = sum(p.n * len(p.prime_idx) for p in rag.products)
    ah = np.empty(total, np.uint32)
    bh = np.empty(total, np.uint32)
    off = 0
    for p in rag.products:
        m = p.n * len(p.prime_idx)
        ah[off:off + m] = p.a.reshape(-1)
        bh[off:off + m] = p.b.reshape(-1)
        off += m
    with polymul.Ragged(rag.pool, 16384, [(p.n, p.prime_idx) for p in rag.products]) as r:
        ta = torch.from_numpy(ah.view(np.int32)).to(dev)
        tb = torch.from_numpy(bh.view(np.int32)).to(dev)
        tc = torch.empty_like(ta)
        choice = r.tune(ta, tb, tc, stream=sp)  # each launch's shape set, by measurement
        for _ in range(2):
            r.run(ta, tb, tc, stream=sp, graph=True)
        ms = _time_steps(lambda i: r.run(ta, tb, tc, stream=sp, graph=True), stream, 10)
        polymul.polymul_ragged_status(r.batch, sp)
        p0 = rag.products[0]
        qs = [rag.pool[j] for j in p0.prime_idx]
        got = tc[:p0.n * len(qs)].cpu().numpy().view(np.uint32).reshape(1, len(qs), p0.n)
        samples.add("ragged_2000", p0.a[None], p0.b[None], qs, got)
        mm = sum(len(p.prime_idx) * _ntt_mulmods(p.n) for p in rag.products)
        out["ragged_2000"] = {"products_per_s": len(rag.products) / (ms / 1e3), "us_per_launch": ms * 1e3,
                              "units": r.info["units"], "work_items": r.info["items"], "grid": r.info["grid"],
                              "path": "ntt, two concurrent persistent launches (2^14; 2^10..2^13) replayed as a CUDA graph",
                              "shape_sets": {"2^10..2^13": choice & 1, "2^14": (choice >> 1) & 1,
                                             "legend": "0 swizzled, both operands (at 2^14 the homogeneous "
                                                       "one-CTA-per-product kernel over the segment's rows); 1 "
                                                       "padded, one operand at 2^10, 2^11, 2^14 (polymul_ragged_tune)"},
                              "alu_frac": mm / (ms / 1e3) / 1e9 / alu_peak_g,
                              "hbm_frac": 3 * total * 4 / (ms / 1e3) / 1e9 / hbm,
                              "bit_exact_sample": None, "l2": "inputs 1.3 GB (> L2)"}
        # the tensor route of the same list: each degree class as one launch
        # of the drained tiled digit kernel (four 8-bit digits per operand),
        # beside the tuner's per-class path choice
        ntt_out = tc.clone()
        out["ragged_2000"]["class_paths"] = {
            "2^%d" % l: ("tensor" if (choice >> (polymul.RAGGED_TENSOR_SHIFT + l - 10)) & 1 else "ntt")
            for l in range(10, 15)}
        r.select((choice & 3) | polymul.ragged_tensor_bits(10, 11, 12, 13, 14))
        r.run(ta, tb, tc, stream=sp, graph=True)
        tms = _time_steps(lambda i: r.run(ta, tb, tc, stream=sp, graph=True), stream, 2)
        polymul.polymul_ragged_status(r.batch, sp)
        flops = sum(2.0 * p.n * p.n * 16 * len(p.prime_idx) for p in rag.products)
        out["ragged_2000"]["tensor_route"] = {
            "us_per_launch": tms * 1e3, "products_per_s": len(rag.products) / (tms / 1e3),
            "kernel": "k_toeplitz_tiled drained, 4 x 4 digits of 8 bits, one launch per degree class (graph)",
            "tensor_frac_bf16": flops / (tms / 1e3) / 1e12 / peaks.get("bf16_tflops", 1911.7),
            "bit_exact_vs_ntt": bool(torch.equal(tc, ntt_out))}
        r.select(choice)
    return out


def graph_replay(dev, w, launches):
    """Launch-latency view of a small batch: `launches` calls of
    polymul_batch captured once in a CUDA graph and replayed (the kernels keep
    their programmatic dependent launches inside the graph)."""
    import torch
    from paper_2307_06554_gb300 import polymul
    try:
        plan = polymul.Plan(w.n, w.q_list)
        ta = torch.from_numpy(w.a.view(np.int32)).to(dev)
        tb = torch.from_numpy(w.b.view(np.int32)).to(dev)
        tc = torch.empty_like(ta)
        s = torch.cuda.Stream(dev)
        with torch.cuda.stream(s):
            polymul.polymul_batch(plan.handle, ta, tb, tc, w.batch, s.cuda_stream)  # first call outside capture
        s.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            cs = torch.cuda.current_stream().cuda_stream
            for _ in range(launches):
                polymul.polymul_batch(plan.handle, ta, tb, tc, w.batch, cs)
        g.replay()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        g.replay()
        e1.record()
        torch.cuda.synchronize()
        polymul.polymul_plan_status(plan.handle)
        us = e0.elapsed_time(e1) * 1e3 / launches
        plan.close()
        return {"launches": launches, "us_per_call": us, "products_per_s": w.batch / (us * 1e-6)}
    except Exception as exc:  # report, do not fail the bench
        return {"error": str(exc)[:200]}


def crossover(dev, stream, peaks, alu_peak_g, samples):
    """Tensor (Toeplitz) path against the NTT path on the same inputs, over
    n = 2^6 .. 2^14 at a fixed number of coefficients per batch (2^22), for
    two modulus families: the smallest NTT-friendly prime from 12289 up (12289
    itself to n = 2048; 40961, 65537 above: 2 or 3 digits) and a 30-bit prime
    (4 or 5 digits).  Inputs: seed 6, uniform residues, operands rotated over
    buffer sets larger than L2.  Both paths must agree on every coefficient
    of the batch."""
    import torch
    from paper_2307_06554_gb300 import polymul, workloads as wl
    rng = np.random.default_rng(6)

    def small_prime(n):
        q = 12289
        while (q - 1) % (2 * n) or not wl.is_prime(q):
            q += 1
        return q
    shapes = []
    for logn in range(6, 15):
        n = 1 << logn
        shapes.append((n, small_prime(n)))
        shapes.append((n, wl.draw_primes(rng, 1, 30, 30, logn + 1)[0]))
    sp = stream.cuda_stream
    rows = []
    for n, q in shapes:
        batch = (1 << 22) // n
        a = wl.uniform_coeffs(rng, batch, [q], n)
        b = wl.uniform_coeffs(rng, batch, [q], n)
        ta = torch.from_numpy(a.view(np.int32)).to(dev)
        tb = torch.from_numpy(b.view(np.int32)).to(dev)
        nsets = max(2, math.ceil(3 * L2_BYTES / (3 * batch * n * 4)))
        sets = [(ta.clone(), tb.clone(), torch.empty_like(ta)) for _ in range(nsets)]
        row = {"n": n, "q": q, "q_bits": q.bit_length(), "batch": batch}
        outs = {}
        for name, path, flags in (("ntt", polymul.PATH_NTT, polymul.FLAG_TUNE), ("tensor", polymul.PATH_TENSOR, 0)):
            plan = polymul.Plan(n, [q], path=path, flags=flags, tune_batch=batch)

            def step(i, h=plan.handle):
                x, y, z = sets[i % nsets]
                polymul.polymul_batch(h, x, y, z, batch, sp)
            for i in range(3):
                step(i)
            ms = _time_steps(step, stream, 20 if n * q.bit_length() < 4096 * 20 else 5)
            info = plan.info
            row[name + "_us"] = ms * 1e3
            row[name + "_products_per_s"] = batch / (ms / 1e3)
            if name == "tensor":
                row["tensor_groups"], row["rns_moduli"] = info["tensor_groups"], info["rns_moduli"]
                sms = torch.cuda.get_device_properties(dev).multi_processor_count
                if info["rns_moduli"]:  # more digits than the digit kernels take: the RNS kernel
                    row["digit_bits"], row["digits"] = 0, 0
                    flops = 2.0 * n * n * info["rns_moduli"] * batch
                    row["tensor_frac_smem"] = _tensor_smem_roofline(
                        n, 1, batch, ms / 1e3, sms, peaks.get("sm_max_mhz", 2070.0), la=info["rns_moduli"],
                        shifts=_rns_shifts(n, info["rns_moduli"]))["frac"]
                else:
                    row["digit_bits"], row["digits"] = info["digit_bits"], info["digits"]
                    flops = 2.0 * n * n * info["digits"] ** 2 * batch
                    row["tensor_frac_smem"] = _tensor_smem_roofline(
                        n, info["digits"], batch, ms / 1e3, sms, peaks.get("sm_max_mhz", 2070.0),
                        shifts=_tiled_shifts(n, info))["frac"]
                row["tensor_frac_bf16"] = flops / (ms / 1e3) / 1e12 / peaks.get("bf16_tflops", 1911.7)
            else:
                row["ntt_alu_frac"] = batch * _ntt_mulmods(n) / (ms / 1e3) / 1e9 / alu_peak_g
            c = torch.empty_like(ta)
            polymul.polymul_batch(plan.handle, ta, tb, c, batch, sp)
            stream.synchronize()
            outs[name] = c
            plan.close()
        row["tensor_over_ntt"] = row["ntt_us"] / row["tensor_us"]
        row["paths_agree"] = bool(torch.equal(outs["ntt"], outs["tensor"]))
        samples.add("crossover", a[[0, batch - 1]], b[[0, batch - 1]], [q],
                    outs["tensor"][[0, batch - 1]].cpu().numpy().view(np.uint32))
        rows.append(row)
        del sets, outs
    return {"rows": rows, "bit_exact_sample": None,
            "tensor_wins_at": [r["n"] for r in rows if r["tensor_over_ntt"] > 1.0]}


def shared_operand(dev, stream, peaks, samples):
    """One operand a shared by the whole batch (the paper's many-vector
    batching), polymul_batch_shared on both paths: the GEMM C = B * T(a) on
    the tensor cores, and the NTT with a's transform computed once (two
    transforms per product); beside them the ordinary NTT batch on the same
    products (a repeated per product).  ring_1024's b operands and its first
    a, and the same at n = 2048."""
    import torch
    from paper_2307_06554_gb300 import polymul, workloads as wl
    sp = stream.cuda_stream
    rows = []
    for n in (1024, 2048):
        w = wl.ring_1024(n=n, batch=4096 * 1024 // n)
        batch, q_list = w.batch, w.q_list
        a = w.a[0]
        ta = torch.from_numpy(a.view(np.int32)).to(dev)
        tb = torch.from_numpy(w.b.view(np.int32)).to(dev)
        nsets = max(2, math.ceil(3 * L2_BYTES / (2 * tb.numel() * 4)))
        sets = [(tb.clone(), torch.empty_like(tb)) for _ in range(nsets)]
        row = {"n": n, "batch": batch, "q": q_list}
        with polymul.Plan(n, q_list, path=polymul.PATH_TENSOR) as plan:
            def step(i, h=plan.handle):
                x, y = sets[i % nsets]
                polymul.polymul_batch_shared(h, ta, x, y, batch, sp)
            for i in range(3):
                step(i)
            ms = _time_steps(step, stream, 20)
            polymul.polymul_plan_status(plan.handle, sp)
            c_t = torch.empty_like(tb)
            polymul.polymul_batch_shared(plan.handle, ta, tb, c_t, batch, sp)
        flops = 2.0 * batch * n * n * 4  # two digits of each operand: four digit-pair GEMMs
        peak = peaks.get("bf16_tflops", 1911.7)
        row.update({"tensor_shared_us": ms * 1e3, "products_per_s": batch / (ms / 1e3),
                    "tflops": flops / (ms / 1e3) / 1e12, "bf16_frac": flops / (ms / 1e3) / 1e12 / peak})
        with polymul.Plan(n, q_list, path=polymul.PATH_NTT) as plan:
            def step3(i, h=plan.handle):
                x, y = sets[i % nsets]
                polymul.polymul_batch_shared(h, ta, x, y, batch, sp)
            for i in range(3):
                step3(i)
            ms3 = _time_steps(step3, stream, 20)
            c_s = torch.empty_like(tb)
            polymul.polymul_batch_shared(plan.handle, ta, tb, c_s, batch, sp)
        row["ntt_shared_us"] = ms3 * 1e3
        ab = ta.repeat(batch, 1).view(batch, len(q_list), n)
        with polymul.Plan(n, q_list) as plan:
            def step2(i, h=plan.handle):
                x, y = sets[i % nsets]
                polymul.polymul_batch(h, ab, x, y, batch, sp)
            for i in range(3):
                step2(i)
            ms2 = _time_steps(step2, stream, 20)
            c_n = torch.empty_like(tb)
            polymul.polymul_batch(plan.handle, ab, tb, c_n, batch, sp)
        stream.synchronize()
        row["ntt_us"] = ms2 * 1e3
        row["tensor_over_ntt"] = ms2 / ms
        row["tensor_over_ntt_shared"] = ms3 / ms
        row["paths_agree"] = bool(torch.equal(c_t, c_n)) and bool(torch.equal(c_s, c_n))
        idx = [0, batch - 1]
        samples.add("shared_operand", np.stack([w.a[0]] * 2), w.b[idx], q_list, c_t[idx].cpu().numpy().view(np.uint32))
        rows.append(row)
        del sets
    return {"rows": rows, "bit_exact_sample": None,
            "kernels": "k_shared_bdigits + k_shared_tdigits (digit planes, tiled) + k_shared_gemm "
                       "(tcgen05 kind::f16, M = N = 128, 4 digit-pair accumulators in tensor memory)"}


def serving(dev, peaks, samples, count=20000, lanes=8):
    """The 20k-request serving workload: Poisson arrivals, n uniform over
    4096..65536, 1..32 primes of 59 bits per request (seed 5), operands in
    page-locked host memory.  Operand data: 16 sets of 32 x 65536 words
    uniform below 2^58 -- canonical residues of every 59-bit pool prime -- so
    request i reads the first k*n words of set i mod 16 as its [k][n]
    operands without a copy.  Every buffer is page-locked, so requests take
    the server's direct route (kernels read a, b and write c in host
    memory); the saturated replay is repeated on the staged route (copies
    through the device arena) for comparison.  Throughput: all requests
    submitted at t = 0 (admitted as device memory frees up; the request
    array is marshalled before the timed replays).  Latency: Poisson
    schedules at 0.5 and 0.8 of that throughput.  Results: a seeded sample of 24 requests of
    the mix write to buffers of their own and are checked against the CPU
    oracle after each replay; the other requests share a pool of output
    buffers whose contents are not read (two of them may be in flight at
    once, which does not change the work or the timing)."""
    import torch
    from paper_2307_06554_gb300 import polymul, workloads as wl
    pool = wl.serve_pool()
    reqs = wl.serve_requests(count=count)
    nmax, kmax, nsets = 65536, 32, 16
    rng = np.random.default_rng(9)
    sets = [(torch.from_numpy(rng.integers(0, 1 << 58, size=kmax * nmax, dtype=np.uint64).view(np.int64)).pin_memory(),
             torch.from_numpy(rng.integers(0, 1 << 58, size=kmax * nmax, dtype=np.uint64).view(np.int64)).pin_memory())
            for _ in range(nsets)]
    shared_outs = [torch.empty(kmax * nmax, dtype=torch.int64).pin_memory() for _ in range(64)]
    checked = sorted(np.random.default_rng(15).choice(len(reqs), size=24, replace=False).tolist())
    own = {i: torch.zeros(len(reqs[i].prime_idx) * reqs[i].n, dtype=torch.int64).pin_memory() for i in checked}
    plist = []
    for i, r in enumerate(reqs):
        a, b = sets[i % nsets]
        out = own[i] if i in own else shared_outs[i % 64]
        plist.append((r.n, r.prime_idx, a.numpy(), b.numpy(), out.numpy()))
    units = sum(len(r.prime_idx) for r in reqs)
    byts = sum(3 * len(r.prime_idx) * r.n * 8 for r in reqs)

    def check_sample(tag):
        for i in checked:
            r = reqs[i]
            a, b = sets[i % nsets]
            k, n = len(r.prime_idx), r.n
            av = a.numpy().view(np.uint64)[:k * n].reshape(k, n)
            bv = b.numpy().view(np.uint64)[:k * n].reshape(k, n)
            cv = own[i].numpy().view(np.uint64).reshape(k, n)
            js = [0, 1 + i % (n - 2), n - 1]
            for j, p in enumerate(r.prime_idx):
                samples.add_coeffs("serve_20k", av[j].copy(), bv[j].copy(), pool[p], js, cv[j, js].copy())
            own[i].zero_()

    prep = polymul.Server.prepare(plist)  # marshalled once, outside the timed replays
    with polymul.Server(pool, nmax, device_bytes=8 << 30, lanes=lanes) as srv:
        srv.replay(plist[:256], [0.0] * 256)  # warm-up
        srv.stats(reset=True)
        t0 = time.perf_counter()
        srv.replay(prep, [0.0] * len(plist))
        el = time.perf_counter() - t0
        sat = srv.stats(reset=True)
        check_sample("saturated")
        # the same with every request copied through the device arena
        srv.set_route(polymul.ROUTE_STAGED)
        t0 = time.perf_counter()
        srv.replay(prep, [0.0] * len(plist))
        el_staged = time.perf_counter() - t0
        sat_staged = srv.stats(reset=True)
        srv.set_route(polymul.ROUTE_DIRECT)
        check_sample("saturated_staged")
        # latency under Poisson arrivals at fractions of the measured
        # saturated rate (the host link it depends on varies between hosts)
        poisson = {}
        for load in (0.5, 0.8):
            rate = load * len(plist) / el
            arrivals = np.cumsum(np.random.default_rng(5).exponential(1.0 / rate, size=len(plist))).tolist()
            t0 = time.perf_counter()
            lat = np.array(srv.replay(prep, arrivals))
            el2 = time.perf_counter() - t0
            st = srv.stats(reset=True)
            poisson["poisson_%.1f" % load] = {
                "offered_per_s": rate, "achieved_per_s": len(plist) / el2, "p50_us": float(np.percentile(lat, 50)),
                "p99_us": float(np.percentile(lat, 99)), "mean_us": float(lat.mean()),
                "queue_p50_us": st["queue_p50_us"], "queue_p99_us": st["queue_p99_us"],
                "service_p50_us": st["service_p50_us"], "service_p99_us": st["service_p99_us"],
                "server_issue_us": st["issue_us_mean"], "direct_requests": st["completed_direct"],
                "failed": st["failed"]}
            check_sample("poisson_%.1f" % load)
        # the tensor path (polymul_server_set_path): the first requests of the
        # mix, all submitted at t = 0, on the 64-bit-word digit kernel; a
        # sample of them checked against the oracle
        tcount = 200
        tcheck = [0, 37, 99, 150, tcount - 1]
        town = {i: torch.zeros(len(reqs[i].prime_idx) * reqs[i].n, dtype=torch.int64).pin_memory() for i in tcheck}
        tlist = [(p[0], p[1], p[2], p[3], town[i].numpy() if i in town else p[4]) for i, p in enumerate(plist[:tcount])]
        tprep = polymul.Server.prepare(tlist)
        srv.set_path(polymul.PATH_TENSOR)
        t0 = time.perf_counter()
        srv.replay(tprep, [0.0] * tcount)
        tel = time.perf_counter() - t0
        tst = srv.stats(reset=True)
        srv.set_path(polymul.PATH_NTT)
        for i in tcheck:
            r = reqs[i]
            a, b = sets[i % nsets]
            k, n = len(r.prime_idx), r.n
            av = a.numpy().view(np.uint64)[:k * n].reshape(k, n)
            bv = b.numpy().view(np.uint64)[:k * n].reshape(k, n)
            cv = town[i].numpy().view(np.uint64).reshape(k, n)
            js = [0, 1 + (7 * i) % (n - 2), n - 1]
            for j, pidx in enumerate(r.prime_idx):
                samples.add_coeffs("serve_20k_tensor", av[j].copy(), bv[j].copy(), pool[pidx], js, cv[j, js].copy())
        tunits = sum(len(r.prime_idx) for r in reqs[:tcount])
        tflops = sum(2.0 * r.n * r.n * 64 * len(r.prime_idx) for r in reqs[:tcount])
        tensor_path = {"requests": tcount, "units": tunits, "seconds": tel, "products_per_s": tcount / tel,
                       "units_per_s": tunits / tel, "failed": tst["failed"],
                       "kernel": "k_toeplitz_u64: 8 x 8 balanced 8-bit digits, K chunks drained into 64-bit "
                                 "modular sums, one launch per request",
                       "tensor_frac_bf16": tflops / tel / 1e12 / peaks.get("bf16_tflops", 1911.7),
                       "ntt_same_requests_per_s": len(plist) / el,
                       "checked": "%d requests, 3 coefficients per prime" % len(tcheck)}
    return {"requests": len(plist), "units": units, "lanes": lanes, "arena_bytes": 8 << 30,
            "bytes_moved": byts,
            "saturated": {"products_per_s": len(plist) / el, "units_per_s": units / el, "seconds": el,
                          "host_link_GBs": byts / el / 1e9, "p50_us": sat["p50_us"], "p99_us": sat["p99_us"],
                          "arena_peak_bytes": sat["arena_peak_bytes"], "failed": sat["failed"],
                          "direct_requests": sat["completed_direct"], "server_issue_us": sat["issue_us_mean"],
                          "route": "direct: each request's kernel reads a, b and writes c in page-locked host "
                                   "memory over the host link"},
            "saturated_staged": {"products_per_s": len(plist) / el_staged, "seconds": el_staged,
                                 "host_link_GBs": byts / el_staged / 1e9, "p50_us": sat_staged["p50_us"],
                                 "p99_us": sat_staged["p99_us"], "failed": sat_staged["failed"],
                                 "server_issue_us": sat_staged["issue_us_mean"],
                                 "route": "staged (polymul_server_set_route): copies in and out through the "
                                          "device arena on each lane's copy streams"},
            **poisson,
            "tensor_path": tensor_path,
            "bit_exact_sample": None,
            "checked": "%d requests of the mix (own output buffers), 3 coefficients per prime, after every replay"
                       % len(checked),
            "data": "16 page-locked operand sets (values < 2^58, canonical for every pool prime)"}


def run_reference(args, ws, rank):
    if rank != 0:
        return
    from paper_2307_06554_gb300 import workloads as wl
    w = wl.ring_1024()
    from oracle import native
    threads = _host_cores()
    per_step = 512  # products per step: a bounded sample of the 4096-product batch
    for i in range(args.warmup):
        s = (i * per_step) % w.batch
        native.polymul_batch(w.a[s:s + per_step], w.b[s:s + per_step], w.q_list, threads=threads)
    t0 = time.perf_counter()
    for i in range(args.steps):
        s = (i * per_step) % w.batch
        native.polymul_batch(w.a[s:s + per_step], w.b[s:s + per_step], w.q_list, threads=threads)
    el = time.perf_counter() - t0
    value = args.steps * per_step / el
    sample = "%d products of the 4096-product batch per step (rotating), plain C schoolbook oracle" % per_step
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "products/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64 (192-bit accumulators)",
        "data": "synthetic", "config": {"workload": WORKLOAD, "path": "cpu oracle", "parallelism": "host threads"},
        "e2e": {"value": value, "unit": "products/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "cpu_baseline": {"value": value, "unit": "products/s", "cores": threads, "kind": "oracle", "sample": sample},
        "gpu_launches": 0,
    }), flush=True)


# ------------------------------------------------------------------ GPU arm
def run_ours(args, ws, rank, local):
    import torch
    from paper_2307_06554_gb300 import polymul, workloads as wl

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    w = wl.ring_1024()
    n, batch, q_list = w.n, w.batch, w.q_list
    # the autotuned kernel for this shape (tuning runs before the timed
    # region); consecutive batches use different buffers, so each may start
    # while the previous one drains (POLYMUL_FLAG_OVERLAP)
    plan = polymul.Plan(n, q_list, flags=polymul.FLAG_TUNE | polymul.FLAG_OVERLAP, tune_batch=batch)
    info = plan.info
    assert info["path"] == polymul.PATH_NTT, "the roofline below describes the NTT kernel"
    elem = info["elem_bytes"]
    set_bytes = 3 * batch * len(q_list) * n * elem
    nsets = max(2, math.ceil(3 * L2_BYTES / set_bytes))
    a0 = torch.from_numpy(w.a.view(np.int32)).to(dev)
    b0 = torch.from_numpy(w.b.view(np.int32)).to(dev)
    sets = [(a0.clone(), b0.clone(), torch.empty_like(a0)) for _ in range(nsets)]
    stream = torch.cuda.Stream(dev)
    sp = stream.cuda_stream

    def step(i):
        a, b, c = sets[i % nsets]
        polymul.polymul_batch(plan.handle, a, b, c, batch, sp)

    with torch.cuda.stream(stream):
        for i in range(args.warmup):
            step(i)
    stream.synchronize()

    clocks = ClockSampler(local)
    clocks.start()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed")  # lets a profiler select the timed launches
    ev0.record(stream)
    for i in range(args.steps):
        step(args.warmup + i)
    ev1.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    elapsed_ms = ev0.elapsed_time(ev1)
    # the dominant kernel's average launch duration over the timed region
    # (one launch per step, back to back on the launching stream)
    launch_ms = elapsed_ms / args.steps
    # the same kernel without the overlap (each batch waits for the previous
    # one to complete before it starts), back to back, for reference
    seq_plan = polymul.Plan(n, q_list, flags=polymul.FLAG_TUNE, tune_batch=batch)
    with torch.cuda.stream(stream):
        for i in range(args.warmup):
            a, b, c = sets[i % nsets]
            polymul.polymul_batch(seq_plan.handle, a, b, c, batch, sp)
    stream.synchronize()
    s0 = torch.cuda.Event(enable_timing=True)
    s1 = torch.cuda.Event(enable_timing=True)
    s0.record(stream)
    for i in range(args.steps):
        a, b, c = sets[i % nsets]
        polymul.polymul_batch(seq_plan.handle, a, b, c, batch, sp)
    s1.record(stream)
    torch.cuda.synchronize()
    no_overlap_ms = s0.elapsed_time(s1) / args.steps
    seq_plan.close()
    # and launches timed one at a time (each bracketed by its own events and
    # a synchronisation, so each starts cold)
    per = []
    for i in range(min(args.steps, 20)):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step(i)
        e1.record(stream)
        e1.synchronize()
        per.append(e0.elapsed_time(e1))

    # the same workload through the tensor (Toeplitz) path, side by side
    tensor = None
    try:
        tplan = polymul.Plan(n, q_list, path=polymul.PATH_TENSOR)
    except polymul.PolymulError:
        tplan = None
    if tplan is not None:
        def tstep(i):
            a, b, c = sets[i % nsets]
            polymul.polymul_batch(tplan.handle, a, b, c, batch, sp)
        with torch.cuda.stream(stream):
            for i in range(args.warmup):
                tstep(i)
        torch.cuda.synchronize()
        t0e = torch.cuda.Event(enable_timing=True)
        t1e = torch.cuda.Event(enable_timing=True)
        t0e.record(stream)
        for i in range(args.steps):
            tstep(i)
        t1e.record(stream)
        torch.cuda.synchronize()
        t_ms = t0e.elapsed_time(t1e) / args.steps
        tc_last = sets[(args.steps - 1) % nsets][2]
        t_got = tc_last[[0, 4095]].cpu().numpy().view(np.uint32)
        tinfo = tplan.info
        tensor = {"ms_per_step": t_ms, "value": batch / (t_ms / 1e3), "unit": "products/s",
                  "kernel": "k_toeplitz_batch (tcgen05 kind::f16, bf16 digits, fp32 TMEM accumulators)",
                  "grid": tinfo["grid"], "block": tinfo["block"], "smem_bytes": tinfo["smem_bytes"],
                  "_check": t_got}
        tplan.close()

    # end to end through the host-buffer entry point, from page-locked host
    # buffers: its direct route (the kernel reads a, b and writes c in host
    # memory over the host link) and, for comparison, the staged route
    # (copy engines through device buffers).  Host sets rotate so that the
    # operands of a step were last read more than 2x L2 of traffic earlier.
    hsets = max(2, math.ceil(2 * L2_BYTES / set_bytes))
    host_np = [(np.roll(w.a, s, axis=0), np.roll(w.b, s, axis=0)) for s in range(hsets)]
    host = [(torch.from_numpy(x.view(np.int32)).pin_memory(), torch.from_numpy(y.view(np.int32)).pin_memory(),
             torch.empty(x.shape, dtype=torch.int32).pin_memory()) for x, y in host_np]
    staged_plan = polymul.Plan(n, q_list, flags=polymul.FLAG_OVERLAP | polymul.FLAG_HOST_STAGED)
    e2e_steps = max(10, args.steps)

    def e2e_run(p):
        """Synchronous host-buffer calls (polymul_batch_host), one per step."""
        for i in range(2):  # warm-up on the last two sets, the timed steps start at set 0
            polymul.polymul_batch_host(p.handle, *host[(hsets - 2 + i) % hsets], batch, None)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i in range(e2e_steps):
            polymul.polymul_batch_host(p.handle, *host[i % hsets], batch, None)
        return time.perf_counter() - t0

    def e2e_stream():
        """Streaming from host buffers (polymul_batch_mapped): step i is
        queued on the stream, then the host waits for step i - 1's event and
        reads that step's result, so one step is always queued behind the
        running one and every step's result is read by the host."""
        evs = [torch.cuda.Event() for _ in range(2)]
        seen = []
        with torch.cuda.stream(stream):
            for i in range(2):
                polymul.polymul_batch_mapped(plan.handle, *host[(hsets - 2 + i) % hsets], batch, sp)
        stream.synchronize()
        t0 = time.perf_counter()
        for i in range(e2e_steps):
            polymul.polymul_batch_mapped(plan.handle, *host[i % hsets], batch, sp)
            evs[i % 2].record(stream)
            if i >= 1:
                evs[(i - 1) % 2].synchronize()
                seen.append(int(host[(i - 1) % hsets][2][-1, 0, -1]))
        evs[(e2e_steps - 1) % 2].synchronize()
        seen.append(int(host[(e2e_steps - 1) % hsets][2][-1, 0, -1]))
        return time.perf_counter() - t0

    e2e_last = (e2e_steps - 1) % hsets
    idx = [0, 1, 2047, 4095]
    e2e_s = e2e_stream()
    e2e_got = host[e2e_last][2].numpy().view(np.uint32)[idx].copy()
    direct_before = polymul.polymul_plan_info_get(plan.handle)["host_direct"]
    sync_s = e2e_run(plan)
    sync_direct = polymul.polymul_plan_info_get(plan.handle)["host_direct"] - direct_before == e2e_steps + 2
    sync_got = host[e2e_last][2].numpy().view(np.uint32)[idx].copy()
    staged_s = e2e_run(staged_plan)
    assert polymul.polymul_plan_info_get(staged_plan.handle)["host_direct"] == 0
    staged_plan.close()
    clk = clocks.stop()
    link = _host_link(dev, 2 * batch * n * elem, batch * n * elem)  # a and b in, c out
    if ws == 1 and rank == 0:
        # the SM-driven ceiling of the direct routes, measured now: loads and
        # stores on mapped page-locked memory mixed 2:1 (the host-link probe)
        try:
            probe = {r["op"]: r["GBs"] for r in _case_host_link()["results"]}
            link["sm_mix_2in_1out_GBs"] = probe["sm_mix_2in_1out"]
            link["sm_probe"] = "bench.py --case host_link, run inside this bench"
        except Exception as exc:  # no compiler on the GPU machine: the copy-engine figures stand alone
            link["sm_probe_error"] = str(exc)[:200]

    # sampled products of the timed batch, checked by the CPU oracle leg
    samples = Samples()
    c_last = sets[(args.warmup + args.steps - 1) % nsets][2]
    samples.add("ring_1024", w.a[idx], w.b[idx], q_list, c_last[idx].cpu().numpy().view(np.uint32))
    hx, hy = host_np[e2e_last]
    samples.add("ring_1024", hx[idx], hy[idx], q_list, e2e_got)  # the streamed last step
    samples.add("ring_1024", hx[idx], hy[idx], q_list, sync_got)  # the synchronous direct call's
    samples.add("ring_1024", hx[idx], hy[idx], q_list,
                host[e2e_last][2].numpy().view(np.uint32)[idx])  # the staged route's
    if tensor is not None:
        samples.add("ring_1024_tensor", w.a[[0, 4095]], w.b[[0, 4095]], q_list, tensor.pop("_check"))

    elapsed_ms, e2e_s, sync_s, staged_s = aggregate_over_ranks([elapsed_ms, e2e_s, sync_s, staged_s], device=dev)
    if rank != 0:
        return
    value = job_rate(batch * args.steps, elapsed_ms / 1e3, ws)
    e2e_value = job_rate(batch * e2e_steps, e2e_s, ws)
    staged_value = job_rate(batch * e2e_steps, staged_s, ws)
    sync_value = job_rate(batch * e2e_steps, sync_s, ws)

    peaks, peak_src = _peaks()
    isolated_ms = statistics.mean(per)
    units = batch * len(q_list)
    mulmods = units * _ntt_mulmods(n)
    mulmods_kernel = units * _ntt_mulmods_kernel(n)
    bytes_alg = 3 * units * n * elem
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_mhz = peaks.get("sm_max_mhz", 2070.0)
    mode = info["ntt_mode"]
    slots = IMAD_SLOTS_PER_MULMOD
    alu_peak = sms * IMAD_LANES_PER_SM * sm_mhz * 1e6 / slots / 1e9  # Gmulmod/s
    alu_ach = mulmods / (launch_ms / 1e3) / 1e9
    hbm_ach = bytes_alg / (launch_ms / 1e3) / 1e9
    hbm_peak = peaks["hbm_gbs"]
    tag = "k_ntt_batch<u32,logn=10,%s,RB=%d,pad=%d,%s>" % (MODE_NAMES[mode], info["radix_bits"], info["exchange_pad"],
                                                            "one-operand" if info["one_operand"] else "two-operand")
    traffic = _recorded_traffic(tag)
    roof = {"bound": "alu", "achieved": alu_ach, "peak": alu_peak, "unit": "Gmulmod/s",
            "frac": alu_ach / alu_peak, "traffic": traffic,
            "work": "3 (n/2) log2 n + n modular multiplications per product (two forward transforms, inverse, "
                    "pointwise); the kernel also scales half of the outputs by n^-1: with those, frac %.3f" % (
                        mulmods_kernel / (launch_ms / 1e3) / 1e9 / alu_peak),
            "kernel": tag + " (forward x2, pointwise, inverse; one launch per step)",
            "peak_source": "derived: %d SMs x %d IMAD lanes x %.0f MHz / %d IMAD slots per Shoup mulmod" % (
                sms, IMAD_LANES_PER_SM, sm_mhz, slots),
            "mulmods_per_launch": mulmods, "launch_ms": launch_ms,
            "launch_ms_source": "CUDA events over the timed region / launches (one per step); consecutive "
                                "launches overlap (POLYMUL_FLAG_OVERLAP: a batch starts while the previous drains)",
            "no_overlap_launch_ms": no_overlap_ms,
            "isolated_launch_ms": isolated_ms,
            "hbm": {"achieved": hbm_ach, "peak": hbm_peak, "unit": "GB/s", "frac": hbm_ach / hbm_peak,
                    "bytes_per_launch": bytes_alg, "peak_source": "MEASURED_PEAKS.json hbm_gbs (%s)" % peak_src}}

    if tensor is not None:
        digits = _tensor_digits(n, max(q_list))
        flops = 2.0 * n * n * digits[1] * digits[1] * units  # every digit-pair product, as the method performs it
        peak_tf = peaks.get("bf16_tflops", 1911.7)
        ach_tf = flops / (tensor["ms_per_step"] / 1e3) / 1e12
        tensor["digit_bits"], tensor["digits"] = digits
        tensor["roofline"] = {"bound": "tensor", "achieved": ach_tf, "peak": peak_tf, "unit": "TFLOP/s",
                              "frac": ach_tf / peak_tf, "flops_per_launch": flops,
                              "peak_source": "MEASURED_PEAKS.json bf16_tflops burst (%s)" % peak_src}
        tensor["roofline_smem"] = _tensor_smem_roofline(n, digits[1], units, tensor["ms_per_step"] / 1e3, sms, sm_mhz)
        tensor["vs_ntt"] = tensor["value"] / value

    extras = None
    if not args.no_extras:
        extras = other_workloads(dev, stream, peaks, alu_peak, samples)
        extras["crossover"] = crossover(dev, stream, peaks, alu_peak, samples)
        extras["shared_operand"] = shared_operand(dev, stream, peaks, samples)
        extras["serve_20k"] = serving(dev, peaks, samples)
        if link.get("sm_mix_2in_1out_GBs"):
            sat = extras["serve_20k"]["saturated"]
            sat["host_link_frac_of_sm_mix"] = sat["host_link_GBs"] / link["sm_mix_2in_1out_GBs"]

    # CPU oracle leg: its throughput (the CPU baseline) and its verdict on
    # the sampled GPU outputs; skipped with --no-cpu-baseline (verdicts null)
    cpu, verdict = None, {}
    if not args.no_cpu_baseline:
        rate, cores, done, el = cpu_oracle_rate(w, args.cpu_seconds)
        cpu = {"value": rate, "unit": "products/s", "cores": cores, "kind": "oracle",
               "sample": "%d products (whole 4096-product batches, repeated) in %.1f s, plain C schoolbook" % (done, el)}
        verdict = samples.check()
    bit_exact = verdict.get("ring_1024")
    if tensor is not None:
        tensor["bit_exact_sample"] = verdict.get("ring_1024_tensor")
    if extras is not None:
        for name, x in extras.items():
            if isinstance(x, dict) and "bit_exact_sample" in x:
                x["bit_exact_sample"] = verdict.get(name)
        tp = (extras.get("serve_20k") or {}).get("tensor_path")
        if isinstance(tp, dict):
            tp["bit_exact_sample"] = verdict.get("serve_20k_tensor")

    out = {
        "metric": METRIC, "value": value, "unit": "products/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic (seeded uniform residues)",
        "config": {"workload": WORKLOAD, "path": {1: "ntt", 2: "tensor"}.get(info["path"], "?"),
                   "autotuned": {"candidates": info["candidates"], "radix_bits": info["radix_bits"],
                                 "ntt_mode": MODE_NAMES[info["ntt_mode"]], "launch_flags": info["launch_flags"],
                                 "exchange_pad": info["exchange_pad"], "one_operand": info["one_operand"],
                                 "regs": info["regs"]},
                   "overlap": "POLYMUL_FLAG_OVERLAP (each batch starts while the previous one drains)",
                   "n": n, "q": q_list, "batch": batch,
                   "l2": "inputs rotated over %d buffer sets (%.0f MB > 3x L2)" % (nsets, nsets * set_bytes / 2**20),
                   "parallelism": "replicas" if ws > 1 else "single"},
        "e2e": {"value": e2e_value, "unit": "products/s", "h2d_bytes_per_step": 2 * batch * n * elem,
                "roofline": ({"bound": "host link", "achieved": 3 * batch * n * elem / (e2e_s / e2e_steps) / 1e9,
                              "peak": link["sm_mix_2in_1out_GBs"], "unit": "GB/s",
                              "frac": 3 * batch * n * elem / (e2e_s / e2e_steps) / 1e9 / link["sm_mix_2in_1out_GBs"],
                              "peak_source": "SM loads and stores on mapped page-locked memory mixed 2:1, "
                                             "measured in this run"}
                             if link.get("sm_mix_2in_1out_GBs") else None),
                "d2h_bytes_per_step": batch * n * elem,
                "api": "polymul_batch_mapped on page-locked host buffers: the NTT batch kernel loads a, b "
                       "from and stores c to host memory over the host link, so every step moves a and b to "
                       "the GPU and c back inside the timed region; step i is queued, then the host waits "
                       "for step i-1's event and reads its result",
                "host_sets": "%d rotating sets of a, b, c (%.0f MB)" % (hsets, hsets * set_bytes / 2**20),
                "per_call_sync": {"value": sync_value, "unit": "products/s",
                                  "api": "polymul_batch_host, synchronous per call",
                                  "route": "direct" if sync_direct else "staged"},
                "staged": {"value": staged_value, "unit": "products/s",
                           "api": "polymul_batch_host on a POLYMUL_FLAG_HOST_STAGED plan: copy engines through "
                                  "device staging buffers, synchronous per call"},
                "host_link": dict(link, achieved_GBs=3 * batch * n * elem / (e2e_s / e2e_steps) / 1e9,
                                  frac_of_copy_engines_both=(3 * batch * n * elem / (e2e_s / e2e_steps) / 1e9)
                                  / link["both_GBs"])},
        "gpu_launches": args.steps,
        "roofline": roof,
        "cpu_baseline": cpu,
        "clocks": clk,
        "bit_exact_sample": bit_exact,
        "tensor_path": tensor,
        "other_workloads": extras,
    }
    print(json.dumps(out), flush=True)
    plan.close()


def main():
    args = _args()
    if args.karatsuba_model:
        for name, n, q, la, lb, s, tern in KARATSUBA_SHAPES:
            print(json.dumps({"shape": name, **karatsuba_model(n, q, la, lb, s, tern)}), flush=True)
        return
    if args.case:
        print(args.case, json.dumps(_case(args.case, args.launches)), flush=True)
        return
    ws, rank, local = _dist()
    if args.impl == "reference":
        run_reference(args, ws, rank)
    else:
        run_ours(args, ws, rank, local)


if __name__ == "__main__":
    main()

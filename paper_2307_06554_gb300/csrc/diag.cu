// polymul_selftest_wait: checks, on the device, that a bounded wait gives up.
//
// Every wait in the library's kernels (bulk-copy completion, MMA completion)
// polls an mbarrier a bounded number of times and, when the limit runs out,
// sets the plan's error word and leaves, so that a stuck copy surfaces as
// POLYMUL_ETIMEOUT instead of a hung GPU.  This kernel exercises exactly
// that path without any fault: it waits on an mbarrier that nothing will
// ever arrive on, with a caller-chosen poll limit, and reports the expiry.
#include <cuda_runtime.h>

#include <atomic>

#include "../../include/polymul.h"
#include "async.cuh"
#include "plan.h"
#include "trace.h"

namespace pm {

// Launches of the NTT batch kernel that still have to take an expired wait
// (polymul_selftest_inject_wait), and the poll limit they use.
static std::atomic<uint32_t> g_inject_launches{0};
static std::atomic<uint32_t> g_inject_polls{1};

bool take_injected_wait(uint32_t* tx_pad, uint32_t* polls) {
  uint32_t left = g_inject_launches.load();
  while (left > 0 && !g_inject_launches.compare_exchange_weak(left, left - 1)) {
  }
  if (left == 0) return false;
  *tx_pad = 16;  // one bulk-copy granule more than the copies deliver
  *polls = g_inject_polls.load();
  return true;
}

__global__ void k_wait_selftest(uint32_t polls, int* err) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) mbar_init(&bar, 1);
  fence_mbar_init();
  __syncthreads();
  // phase 0 of a fresh barrier with one expected arrival and none coming
  const bool ok = mbar_wait(&bar, 0, polls);
  if (__syncthreads_or(!ok) && threadIdx.x == 0) atomicExch(err, 1);
}

}  // namespace pm

using namespace pm;

extern "C" int polymul_selftest_wait(uint32_t polls, void* stream) {
  clear_error();
  TraceRange trace("polymul_selftest_wait");
  if (polls == 0 || polls > (1u << 22)) return fail(POLYMUL_EINVAL, "polls=%u must be in [1, 2^22]", polls);
  cudaStream_t st = (cudaStream_t)stream;
  int* d_err = nullptr;
  if (cudaMalloc(&d_err, sizeof(int)) != cudaSuccess) return fail(POLYMUL_ENOMEM, "error word");
  int h = 0;
  cudaError_t e = cudaMemsetAsync(d_err, 0, sizeof(int), st);
  if (e == cudaSuccess) {
    k_wait_selftest<<<1, 32, 0, st>>>(polls, d_err);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d_err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(d_err);
  if (e != cudaSuccess) return cuda_fail(e, "wait self-test");
  if (h) return fail(POLYMUL_ETIMEOUT, "the device wait gave up after %u polls, as it must", polls);
  return fail(POLYMUL_ECUDA, "a wait with nothing to wait for completed");
}

extern "C" int polymul_selftest_inject_wait(uint32_t launches, uint32_t polls) {
  clear_error();
  if (polls == 0 || polls > (1u << 22)) return fail(POLYMUL_EINVAL, "polls=%u must be in [1, 2^22]", polls);
  if (launches > (1u << 20)) return fail(POLYMUL_EINVAL, "launches=%u must be at most 2^20", launches);
  g_inject_polls.store(polls);
  g_inject_launches.store(launches);
  return POLYMUL_OK;
}

// polymul_batch_static: the NTT batch multiplication for callers that must
// not allocate device memory.
//
// Who cannot allocate: code that runs while some thread of the process is
// capturing a CUDA graph in the global capture mode (cudaMalloc and cudaFree
// are illegal then), latency-critical callers that cannot afford the
// implicit device synchronisation of cudaMalloc/cudaFree, and host
// frameworks whose caching allocator owns the device memory and forbids
// allocations behind its back.  polymul_create allocates its tables, so such
// callers cannot hold a plan; this entry point needs none.
//
// Everything the kernel needs besides the caller's operands lives in one
// fixed array in device memory, compiled into the library
// (g_static_scratch): the kernel's work counter and error word, the prime's
// constants and its forward and inverse twiddle tables.  Every GPU that loads
// the library holds the array until the process exits.  Consequences:
//  * one modulus per call, n <= kStaticMaxN;
//  * every call uses the same array, so calls whose kernels could overlap on
//    the GPU (different streams, no ordering between them) race and give
//    wrong results: order them (same stream, or events);
//  * the array keeps the last call's contents: the tables are re-uploaded
//    only when (n, q) changes on that device, and the work counter and error
//    word are cleared on every call;
//  * the first call on a device looks up the array's device address
//    (cudaGetSymbolAddress), so make that first call before any stream
//    capture begins.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "../../include/polymul.h"
#include "kernels.h"
#include "host_math.h"
#include "ntt_tables.h"
#include "trace.h"
#include "plan.h"
#include "polymul_types.h"
#include "stream_order.h"

using namespace pm;

namespace {

constexpr uint32_t kStaticMaxN = 4096;
// byte layout: [0, 16) work counter pair | [16, 20) error word |
// [32, 64) PrimeConst<uint32_t> | forward twiddle pairs (8 n bytes) |
// inverse twiddle pairs (8 n bytes)
constexpr size_t kStaticOffPc = 32;
constexpr size_t kStaticOffTw = 64;
constexpr size_t kStaticBytes = kStaticOffTw + 2 * (size_t)kStaticMaxN * 8;

static_assert(sizeof(PrimeConst<uint32_t>) == 32, "constants block");

}  // namespace

static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

namespace {

struct StaticDeviceState {
  bool ready = false;
  unsigned char* ptr = nullptr;  // device address of g_static_scratch on this device
  uint32_t n = 0;                // (n, q) whose tables the array holds
  uint64_t q = 0;
};

std::mutex g_static_mu;
StaticDeviceState g_static_dev[64];
// host-side staging of the tables (static: the entry point allocates nothing)
uint32_t g_host_tw[2][2 * kStaticMaxN];
PrimeConst<uint32_t> g_host_pc;

// psi^brv(i), psi^-brv(i) with Shoup companions, and the constants of q, n:
// the plan builder's tables, written into the static host staging arrays
void fill_tables(uint64_t q, uint32_t n) { build_ntt_tables_into<uint32_t>(q, n, g_host_tw[0], g_host_tw[1], g_host_pc); }

bool lookup_u32(int logn, int mode, KernelInfo* ki) {
  if (mode == 0) return lookup_ntt_u32_m0(logn, ki);
  if (mode == 1) return lookup_ntt_u32_m1(logn, ki);
  if (mode == 2) return lookup_ntt_u32_m2(logn, ki);
  return false;
}

}  // namespace

#define PM_CUDA(call)                                       \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return pm::cuda_fail(e_, #call); \
  } while (0)

extern "C" int polymul_batch_static(uint32_t n, uint64_t q, const void* a, const void* b, void* c,
                                    uint64_t batch, void* stream) {
  clear_error();
  TraceRange trace_("polymul_batch_static");
  if (n < 16 || n > kStaticMaxN || (n & (n - 1)))
    return fail(POLYMUL_EINVAL, "n=%u must be a power of two in [16, %u]", n, kStaticMaxN);
  if (q >= (1ull << 31) || !pm::host::is_prime(q) || (q - 1) % (2ull * n) != 0)
    return fail(POLYMUL_EINVAL, "q=%llu must be a prime below 2^31 with 2n | q - 1", (unsigned long long)q);
  if (batch == 0) return POLYMUL_OK;
  if (!a || !b || !c) return fail(POLYMUL_EINVAL, "null operand pointer");
  if (((uintptr_t)a | (uintptr_t)b | (uintptr_t)c) & 15u) return fail(POLYMUL_EINVAL, "operands must be 16-byte aligned");
  if (batch > (1ull << 40)) return fail(POLYMUL_EINVAL, "batch too large");
  const uint32_t logn = (uint32_t)__builtin_ctz(n);
  const int mode = ntt_mode(q, logn, 4);
  KernelInfo ki;
  if (!lookup_u32((int)logn, mode, &ki)) return fail(POLYMUL_ENOTSUP, "no kernel for n=%u", n);
  cudaStream_t st = (cudaStream_t)stream;

  int dev = 0;
  PM_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(POLYMUL_ENOTSUP, "device ordinal %d", dev);
  std::lock_guard<std::mutex> lock(g_static_mu);
  StaticDeviceState& s = g_static_dev[dev];
  if (!s.ready) {
    // the host-side name of the array is not a device address: look the
    // address up once per device, with that device current
    void* p = nullptr;
    PM_CUDA(cudaGetSymbolAddress(&p, g_static_scratch));
    s.ptr = static_cast<unsigned char*>(p);
    s.ready = true;
  }
  if (s.n != n || s.q != q) {
    fill_tables(q, n);
    // pageable sources: each copy has consumed its source when it returns
    s.n = 0;
    PM_CUDA(cudaMemcpyAsync(s.ptr + kStaticOffPc, &g_host_pc, sizeof g_host_pc, cudaMemcpyHostToDevice, st));
    PM_CUDA(cudaMemcpyAsync(s.ptr + kStaticOffTw, g_host_tw[0], (size_t)n * 8, cudaMemcpyHostToDevice, st));
    PM_CUDA(cudaMemcpyAsync(s.ptr + kStaticOffTw + (size_t)n * 8, g_host_tw[1], (size_t)n * 8,
                            cudaMemcpyHostToDevice, st));
    s.n = n;
    s.q = q;
  }
  PM_CUDA(cudaMemsetAsync(s.ptr, 0, 20, st));  // work counter pair and error word start at zero

  int per_sm = 0, sms = 0;
  PM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  PM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ki.fn, ki.block, ki.smem));
  if (per_sm < 1) return fail(POLYMUL_ENOTSUP, "kernel does not fit on an SM");
  const uint64_t need = (batch + ki.units_per_cta - 1) / ki.units_per_cta;
  const int grid = (int)std::min<uint64_t>(need, (uint64_t)per_sm * sms);
  uint32_t tx_pad = 0, polls = 0;
  take_injected_wait(&tx_pad, &polls);
  NttBatchArgs<uint32_t> args{(const uint32_t*)a,
                              (const uint32_t*)b,
                              (uint32_t*)c,
                              s.ptr + kStaticOffTw,
                              s.ptr + kStaticOffTw + (size_t)n * 8,
                              reinterpret_cast<const PrimeConst<uint32_t>*>(s.ptr + kStaticOffPc),
                              batch,
                              1u,
                              reinterpret_cast<unsigned long long*>(s.ptr),
                              reinterpret_cast<int*>(s.ptr + 16),
                              nullptr,
                              nullptr,
                              n,
                              1u,
                              0u,
                              0u,
                              tx_pad,
                              polls};
  void* argv[] = {&args};
  // the kernel lets the next one on the stream start once it is running:
  // record what it reads and writes (stream_order.h)
  const uintptr_t bytes = (uintptr_t)(batch * n * 4);
  LaunchFootprint fp;
  fp.a_lo = (uintptr_t)a, fp.a_hi = (uintptr_t)a + bytes;
  fp.b_lo = (uintptr_t)b, fp.b_hi = (uintptr_t)b + bytes;
  fp.c_lo = (uintptr_t)c, fp.c_hi = (uintptr_t)c + bytes;
  StreamOrderGuard order(dev, st);
  PM_CUDA(cudaLaunchKernel(ki.fn, grid, ki.block, argv, ki.smem, st));
  order.record(&fp);
  return POLYMUL_OK;
}

// The error word sits in the same fixed array and every call clears it, so
// it describes the most recent call on the device; reading it allocates
// nothing (a plain copy into a local word).
extern "C" int polymul_static_status(void* stream) {
  clear_error();
  int dev = 0;
  PM_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(POLYMUL_ENOTSUP, "device ordinal %d", dev);
  std::lock_guard<std::mutex> lock(g_static_mu);
  StaticDeviceState& s = g_static_dev[dev];
  if (!s.ready) return POLYMUL_OK;  // no call on this device yet
  PM_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  int h = 0;
  PM_CUDA(cudaMemcpy(&h, s.ptr + 16, sizeof(int), cudaMemcpyDeviceToHost));
  if (!h) return POLYMUL_OK;
  PM_CUDA(cudaMemset(s.ptr + 16, 0, sizeof(int)));
  return fail(POLYMUL_ETIMEOUT, "a bounded device wait of the last polymul_batch_static call expired; its results are invalid");
}

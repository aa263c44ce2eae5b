// Shared-operand products on the tensor cores: c_i = a * b_i for one
// operand a and many b_i (the paper's many-vector batching, Sec. 2.2: one
// matrix times many vectors is a single matrix product).
//
// With the roles of Eq. equ-genereal-mat swapped (c_i = b_i * T(a), T(a) the
// negacyclic matrix of a, or its circulant for x^n - 1) the whole batch is
//     C [batch x n] = B [batch x n] * T(a) [n x n],
// a real GEMM with M = batch, N = K = n.  Coefficients are split into L
// balanced w-bit digits as on the per-product path (Sec. 2.4), so that every
// fp32 partial sum over K = n terms is an exact integer:
//     C = sum_{s,t} 2^(w (s + t)) B_s T_t,
// and the L^2 digit-pair products are recombined mod q in the epilogue
// (Algorithm 1, ConvertMatrix).
//
// Operands are prepared once per call into bf16 digit planes stored already
// tiled in the tcgen05 canonical no-swizzle K-major layout: a 128-row x 64-K
// tile is 16 KB, core matrix (row group g, K group c) at (8 g + c) * 128
// bytes, rows 16 bytes apart.  One bulk copy moves a whole tile.  The GEMM
// kernel computes a 128-product x 128-output tile of every digit pair with
// its accumulators in tensor memory (L^2 x 128 columns), fed by a 3-stage
// pipeline: one thread issues the bulk copies, one thread issues the MMAs,
// and tcgen05.commit hands each stage back to the copier.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "../../include/polymul.h"
#include "kernels.h"
#include "trace.h"
#include "plan.h"
#include "stream_order.h"
#include "polymul_types.h"
#include "tcgen05.cuh"

namespace pm {

constexpr int kShRows = 128;                  // rows per tile (MMA M, and N of the B operand tiles)
constexpr int kShK = 64;                      // K elements per tile and pipeline stage
constexpr int kShTileBytes = kShRows * kShK * 2;  // 16 KB
constexpr int kShStages = 3;
constexpr int kShL = 2;                       // digits per coefficient
constexpr int kShThreads = 128;
constexpr int kShSmem = kShStages * 2 * kShL * kShTileBytes;  // 192 KB

struct SharedGemmArgs {
  const unsigned char* bd;  // [k][L][rblocks][kblocks] tiles of b's digits
  const unsigned char* td;  // [k][L][nblocks][kblocks] tiles of T(a)'s digits (rows = outputs)
  uint32_t* c;              // [batch][k][n]
  const TensorPrime* tp;    // [k]
  uint64_t batch;
  uint32_t k, n, rblocks, nblocks, kblocks;
  int* err;
};

// byte offset of the 16-byte row chunk (row r, K group kg) inside a tile
__device__ __forceinline__ uint32_t sh_chunk(uint32_t r, uint32_t kg) {
  return ((r >> 3) * 8 + kg) * 128 + (r & 7) * 16;
}

__device__ __forceinline__ uint32_t sh_bf16x2(int d0, int d1) {
  // exact bf16 of small integers (|d| <= 256): see k_toeplitz_batch
  const float f0 = __int_as_float(0x4B400000 + d0) - 12582912.0f;
  const float f1 = __int_as_float(0x4B400000 + d1) - 12582912.0f;
  return __byte_perm(__float_as_uint(f0), __float_as_uint(f1), 0x7632);
}

// b's digit planes.  One thread per (prime, row, K group of 8): 8 threads
// with consecutive ids write the 8 rows of one 128-byte core matrix.
// Rows at or beyond `batch` (padding to a whole tile) are zero.
template <int WB>
__global__ void k_shared_bdigits(const uint32_t* __restrict__ b, unsigned char* __restrict__ bd,
                                 const TensorPrime* __restrict__ tp, uint64_t batch, uint32_t k, uint32_t n,
                                 uint32_t rblocks) {
  constexpr int HALF = 1 << (WB - 1), MASK = (1 << WB) - 1;
  const uint32_t kgroups = n / 8;
  const uint64_t total = (uint64_t)k * rblocks * kShRows * kgroups;
  for (uint64_t id = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; id < total;
       id += (uint64_t)gridDim.x * blockDim.x) {
    // id = (((j * rblocks + rb) * kgroups + g) * 16 + rg) * 8 + r8: row = rb*128 + rg*8 + r8
    const uint32_t r8 = (uint32_t)(id & 7), rg = (uint32_t)((id >> 3) & 15);
    uint64_t rest = id >> 7;
    const uint32_t g = (uint32_t)(rest % kgroups);
    rest /= kgroups;
    const uint32_t rb = (uint32_t)(rest % rblocks);
    const uint32_t j = (uint32_t)(rest / rblocks);
    const uint32_t r = rg * 8 + r8;
    const uint64_t row = (uint64_t)rb * kShRows + r;
    int d[kShL][8];
    if (row < batch) {
      const uint32_t q = tp[j].q;
      const int32_t qh = (int32_t)(q >> 1);
      const uint4* src = reinterpret_cast<const uint4*>(b + (row * k + j) * n + 8 * g);
      const uint4 v0 = src[0], v1 = src[1];
      const uint32_t v[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        int32_t x = (int32_t)v[e] > qh ? (int32_t)(v[e] - q) : (int32_t)v[e];
#pragma unroll
        for (int s = 0; s < kShL; ++s) {
          const int32_t dd = ((x + HALF) & MASK) - HALF;
          x = (x - dd) >> WB;
          d[s][e] = dd;
        }
      }
    } else {
#pragma unroll
      for (int s = 0; s < kShL; ++s)
#pragma unroll
        for (int e = 0; e < 8; ++e) d[s][e] = 0;
    }
    const uint32_t kb = g / 8, kg = g % 8;
#pragma unroll
    for (int s = 0; s < kShL; ++s) {
      unsigned char* tile = bd + ((((uint64_t)j * kShL + s) * rblocks + rb) * (n / kShK) + kb) * kShTileBytes;
      *reinterpret_cast<uint4*>(tile + sh_chunk(r, kg)) =
          make_uint4(sh_bf16x2(d[s][0], d[s][1]), sh_bf16x2(d[s][2], d[s][3]), sh_bf16x2(d[s][4], d[s][5]),
                     sh_bf16x2(d[s][6], d[s][7]));
    }
  }
}

// T(a)'s digit planes as the GEMM's B operand (rows = output index jj, K =
// input index k): entry (jj, k) is the extended a~_{jj-k} (a~_{i-n} = -a_i
// for x^n + 1, +a_i for x^n - 1).  One thread per (prime, 16-byte chunk),
// spread over the whole GPU; 8 consecutive threads write one core matrix.
// a is small (n words per prime) and stays in L1/L2.
template <int WB>
__global__ void k_shared_tdigits(const uint32_t* __restrict__ a, unsigned char* __restrict__ td,
                                 const TensorPrime* __restrict__ tp, uint32_t k, uint32_t n, uint32_t wrap) {
  constexpr int HALF = 1 << (WB - 1), MASK = (1 << WB) - 1;
  const uint32_t nblocks = n / kShRows, kgroups = n / 8;
  const uint64_t total = (uint64_t)k * nblocks * kShRows * kgroups;
  for (uint64_t id = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; id < total;
       id += (uint64_t)gridDim.x * blockDim.x) {
    // id = (((j * nblocks + nb) * kgroups + g) * 16 + rg) * 8 + r8
    const uint32_t r8 = (uint32_t)(id & 7), rg = (uint32_t)((id >> 3) & 15);
    uint64_t rest = id >> 7;
    const uint32_t g = (uint32_t)(rest % kgroups);
    rest /= kgroups;
    const uint32_t nb = (uint32_t)(rest % nblocks);
    const uint32_t j = (uint32_t)(rest / nblocks);
    const uint32_t r = rg * 8 + r8, jj = nb * kShRows + r;
    const uint32_t q = tp[j].q;
    const int32_t qh = (int32_t)(q >> 1);
    const uint32_t* aj = a + (size_t)j * n;
    uint32_t h[kShL][8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int32_t idx = (int32_t)jj - (int32_t)(8 * g + e);
      const uint32_t v = __ldg(aj + (idx >= 0 ? idx : idx + (int32_t)n));
      int32_t x = (int32_t)v > qh ? (int32_t)(v - q) : (int32_t)v;
      const uint32_t flip = idx >= 0 ? 0u : (wrap & 0xFFFFu);
#pragma unroll
      for (int s = 0; s < kShL; ++s) {
        const int32_t dd = ((x + HALF) & MASK) - HALF;
        x = (x - dd) >> WB;
        h[s][e] = (sh_bf16x2(dd, 0) & 0xFFFFu) ^ flip;
      }
    }
    const uint32_t kb = g / 8, kg = g % 8;
#pragma unroll
    for (int s = 0; s < kShL; ++s) {
      unsigned char* tile = td + ((((uint64_t)j * kShL + s) * nblocks + nb) * (n / kShK) + kb) * kShTileBytes;
      *reinterpret_cast<uint4*>(tile + sh_chunk(r, kg)) =
          make_uint4(h[s][0] | (h[s][1] << 16), h[s][2] | (h[s][3] << 16), h[s][4] | (h[s][5] << 16),
                     h[s][6] | (h[s][7] << 16));
    }
  }
}

__device__ __forceinline__ uint32_t sh_barrett(uint64_t x, uint32_t q, uint64_t mu) {
  const uint64_t qh = __umul64hi(x, mu);
  const uint32_t r = (uint32_t)(x - qh * q);
  return r >= q ? r - q : r;
}

// One 128-product x 128-output tile of one prime, every digit pair.
__global__ void __launch_bounds__(kShThreads, 1) k_shared_gemm(SharedGemmArgs args) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ __align__(8) uint64_t full[kShStages], empty[kShStages], done;
  __shared__ uint32_t s_tmem;
  __shared__ int s_fail;
  __shared__ uint32_t s_issued, s_consumed;  // K blocks copied / read by the MMAs
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t tile = blockIdx.x;
  const uint32_t nb = tile % args.nblocks, rb = (tile / args.nblocks) % args.rblocks,
                 j = tile / (args.nblocks * args.rblocks);
  const uint32_t kblocks = args.kblocks;
  constexpr uint32_t NCOLS = kShL * kShL * kShRows;  // 512 accumulator columns
  constexpr uint32_t IDESC = idesc_bf16(kShRows, kShRows);
  constexpr uint32_t STAGE = 2 * kShL * kShTileBytes;

  if (warp == 0) {
    tmem_alloc(&s_tmem, NCOLS);
    tmem_relinquish();
  }
  if (tid == 0) {
    for (int i = 0; i < kShStages; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    mbar_init(&done, 1);
    s_fail = 0;
    s_issued = 0;
    s_consumed = 0;
  }
  fence_mbar_init();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  const size_t kb_stride = kShTileBytes;
  const unsigned char* a_src = args.bd + (((size_t)j * kShL) * args.rblocks + rb) * kblocks * kb_stride;
  const unsigned char* b_src = args.td + (((size_t)j * kShL) * args.nblocks + nb) * kblocks * kb_stride;
  const size_t a_digit = (size_t)args.rblocks * kblocks * kb_stride;  // between digit planes of b
  const size_t b_digit = (size_t)args.nblocks * kblocks * kb_stride;  // between digit planes of T(a)

  // the copier and the MMA issuer are lane 0 of warps 0 and 1; their other
  // lanes wait at the warp barrier, not on an mbarrier (a warp suspended in
  // an mbarrier poll would also hold back its issuing lane)
  if (tid == 0) {
    // copier: stage st holds A digit tiles then B digit tiles of K block kb
    for (uint32_t kb = 0; kb < kblocks; ++kb) {
      const uint32_t st = kb % kShStages;
      if (kb >= (uint32_t)kShStages && !mbar_wait(&empty[st], ((kb / kShStages) - 1) & 1u)) {
        atomicExch(&s_fail, 1);
        break;
      }
      if (*(volatile int*)&s_fail) break;
      unsigned char* dst = sm + st * STAGE;
      mbar_arrive_expect_tx(&full[st], STAGE);
      for (int s = 0; s < kShL; ++s)
        bulk_g2s(dst + s * kShTileBytes, a_src + s * a_digit + kb * kb_stride, kShTileBytes, &full[st]);
      for (int t = 0; t < kShL; ++t)
        bulk_g2s(dst + (kShL + t) * kShTileBytes, b_src + t * b_digit + kb * kb_stride, kShTileBytes, &full[st]);
      s_issued = kb + 1;
    }
  } else if (tid == 32) {
    // MMA issuer
    for (uint32_t kb = 0; kb < kblocks; ++kb) {
      const uint32_t st = kb % kShStages;
      if (!mbar_wait(&full[st], (kb / kShStages) & 1u)) {
        atomicExch(&s_fail, 1);
        break;
      }
      tc_fence_after();
      const uint32_t base = smem_u32(sm + st * STAGE);
#pragma unroll
      for (int kk = 0; kk < kShK / 16; ++kk) {
#pragma unroll
        for (int s = 0; s < kShL; ++s) {
          const uint64_t ad = smem_desc(base + s * kShTileBytes + kk * 256, 128, 1024);
#pragma unroll
          for (int t = 0; t < kShL; ++t) {
            const uint64_t bdsc = smem_desc(base + (kShL + t) * kShTileBytes + kk * 256, 128, 1024);
            tc_mma_f16(tmem + (uint32_t)((s * kShL + t) * kShRows), ad, bdsc, IDESC, (kb | kk) ? 1u : 0u);
          }
        }
      }
      tc_commit(&empty[st]);  // the stage is free once these MMAs have read it
      s_consumed = kb + 1;
    }
    tc_commit(&done);  // every MMA issued so far has completed
  }
  if (warp < 2) __syncwarp();
  // epilogue: thread = TMEM lane = row of the tile
  const bool ok_done = mbar_wait(&done, 0);
  if (!ok_done) atomicExch(&s_fail, 1);
  __syncthreads();
  const bool failed = s_fail != 0;
  tc_fence_after();
  const uint64_t row = (uint64_t)rb * kShRows + warp * 32 + lane;
  // tcgen05.ld is warp-collective (.sync.aligned): every lane loads, and only
  // the rows inside the batch are stored
  const bool store = row < args.batch;
  if (!failed) {
    const uint32_t q = args.tp[j].q;
    const uint64_t mu = args.tp[j].mu, bias = args.tp[j].bias;
    int64_t pw[2 * kShL - 1];
#pragma unroll
    for (int e = 0; e < 2 * kShL - 1; ++e) pw[e] = (int64_t)args.tp[j].pw[e];
    uint32_t* crow = args.c + ((store ? row : 0) * args.k + j) * args.n + nb * kShRows;
#pragma unroll 1
    for (int c16 = 0; c16 < kShRows / 16; ++c16) {
      int64_t acc[16];
#pragma unroll
      for (int x = 0; x < 16; ++x) acc[x] = 0;
#pragma unroll
      for (int s = 0; s < kShL; ++s) {
#pragma unroll
        for (int t = 0; t < kShL; ++t) {
          uint32_t r[16];
          tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)((s * kShL + t) * kShRows + 16 * c16), r);
          tmem_wait_ld();
#pragma unroll
          for (int x = 0; x < 16; ++x) acc[x] += (int64_t)__float2int_rn(__uint_as_float(r[x])) * pw[s + t];
        }
      }
      uint32_t o[16];
#pragma unroll
      for (int x = 0; x < 16; ++x) o[x] = sh_barrett((uint64_t)(acc[x] + (int64_t)bias), q, mu);
      if (store) {
        uint4* dst = reinterpret_cast<uint4*>(crow + 16 * c16);
        dst[0] = make_uint4(o[0], o[1], o[2], o[3]);
        dst[1] = make_uint4(o[4], o[5], o[6], o[7]);
        dst[2] = make_uint4(o[8], o[9], o[10], o[11]);
        dst[3] = make_uint4(o[12], o[13], o[14], o[15]);
      }
    }
  }
  if (failed && tid == 0) {
    atomicExch(args.err, 1);
    // let copies still in flight land before the shared memory is released
    // (stages copied but never read by the MMAs: their next phases)
    for (uint32_t kb = s_consumed; kb < s_issued; ++kb) mbar_wait(&full[kb % kShStages], (kb / kShStages) & 1u);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, NCOLS);
  }
}

}  // namespace pm

using namespace pm;

#define PM_CUDA(call)                                       \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return pm::cuda_fail(e_, #call); \
  } while (0)

static bool sh_misaligned(const void* x) { return ((uintptr_t)x & 15u) != 0; }

// scratch of the plan: at least `bytes`, of which the first 16 bytes are a
// zeroed work counter pair
static int sh_scratch(polymul_plan* p, size_t bytes) {
  if (p->sh_bytes >= bytes) return POLYMUL_OK;
  if (p->d_sh) PM_CUDA(cudaFree(p->d_sh));
  p->d_sh = nullptr;
  p->sh_bytes = 0;
  if (cudaMalloc(&p->d_sh, bytes) != cudaSuccess) return fail(POLYMUL_ENOMEM, "shared-operand scratch");
  PM_CUDA(cudaMemset(p->d_sh, 0, 256));
  p->sh_bytes = bytes;
  return POLYMUL_OK;
}

// a launch with programmatic stream serialisation: the kernel's CTAs may
// start while the previous kernel on the stream drains (the kernels wait for
// it with griddepcontrol before touching memory)
static int pdl_launch(const void* fn, int grid, int block, int smem, void** argv, cudaStream_t st) {
  cudaLaunchConfig_t cfg;
  memset(&cfg, 0, sizeof cfg);
  cudaLaunchAttribute attr;
  attr.id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr.val.programmaticStreamSerializationAllowed = 1;
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = &attr;
  cfg.numAttrs = 1;
  PM_CUDA(cudaLaunchKernelExC(&cfg, fn, argv));
  return POLYMUL_OK;
}

// NTT path: a's transforms (k units) then the batch
static int shared_ntt(polymul_plan* p, const void* a, const void* b, void* c, uint64_t batch, cudaStream_t st) {
  KernelInfo prep, kmain;
  if (p->elem != 4 || p->aux_prime || p->ki.cluster || !lookup_ntt_shared((int)p->logn, p->mode, &prep, &kmain))
    return fail(POLYMUL_ENOTSUP, "shared-operand NTT products need 32-bit words, n in [1024, 8192] and a direct NTT");
  const size_t ahat_bytes = (size_t)p->k * p->n * 4;
  int rc = sh_scratch(p, 256 + ahat_bytes);
  if (rc != POLYMUL_OK) return rc;
  unsigned long long* ctr = static_cast<unsigned long long*>(p->d_sh);
  uint32_t* ahat = reinterpret_cast<uint32_t*>(static_cast<unsigned char*>(p->d_sh) + 256);
  const PrimeConst<uint32_t>* pc = static_cast<const PrimeConst<uint32_t>*>(p->d_pc);
  NttSharedArgs<uint32_t> pa{(const uint32_t*)a, nullptr, ahat, p->d_twf, p->d_twi, pc, p->k, 0, p->k, p->n, nullptr,
                             p->d_err};
  void* argv_p[] = {&pa};
  // both kernels let the next one on the stream start once they run; their
  // footprint includes plan scratch, so record it as unknown: the next batch
  // launch on the stream then waits for them in full (stream_order.h)
  StreamOrderGuard order(p->device, st);
  order.record(nullptr);
  int rc2 = pdl_launch(prep.fn, (int)p->k, prep.block, prep.smem, argv_p, st);
  if (rc2 != POLYMUL_OK) return rc2;
  int per_sm = 0;
  if (kmain.smem > 48 * 1024)
    PM_CUDA(cudaFuncSetAttribute(kmain.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, kmain.smem));
  PM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kmain.fn, kmain.block, kmain.smem));
  if (per_sm < 1) return fail(POLYMUL_ENOTSUP, "shared-operand NTT kernel does not fit on an SM");
  const uint64_t pairs = (batch + 1) / 2 * p->k;
  const int grid = (int)std::min<uint64_t>(pairs, (uint64_t)per_sm * p->num_sms);
  NttSharedArgs<uint32_t> ma{ahat, (const uint32_t*)b, (uint32_t*)c, p->d_twf, p->d_twi, pc, pairs, batch, p->k, p->n,
                             ctr, p->d_err};
  void* argv_m[] = {&ma};
  return pdl_launch(kmain.fn, grid, kmain.block, kmain.smem, argv_m, st);
}

extern "C" int polymul_batch_shared(polymul_plan* p, const void* a, const void* b, void* c, uint64_t batch,
                                    void* stream) {
  clear_error();
  TraceRange trace_("polymul_batch_shared");
  if (!p) return fail(POLYMUL_EINVAL, "plan is NULL");
  if (batch == 0) return POLYMUL_OK;
  if (!a || !b || !c) return fail(POLYMUL_EINVAL, "null operand pointer");
  if (sh_misaligned(a) || sh_misaligned(b) || sh_misaligned(c)) return fail(POLYMUL_EINVAL, "operands must be 16-byte aligned");
  if (batch > (1ull << 32)) return fail(POLYMUL_EINVAL, "batch too large");
  cudaStream_t st = (cudaStream_t)stream;
  if (p->path == POLYMUL_PATH_NTT) return shared_ntt(p, a, b, c, batch, st);
  if (p->path != POLYMUL_PATH_TENSOR || p->digits != kShL || !p->d_tpc)
    return fail(POLYMUL_ENOTSUP, "shared-operand products need a tensor-path plan with %d digits per coefficient", kShL);
  if (p->n % kShRows != 0) return fail(POLYMUL_ENOTSUP, "n=%u is not a multiple of %d", p->n, kShRows);
  const uint32_t n = p->n, k = p->k;
  const uint32_t rblocks = (uint32_t)((batch + kShRows - 1) / kShRows), nblocks = n / kShRows, kblocks = n / kShK;
  const size_t bd_bytes = (size_t)k * kShL * rblocks * kblocks * kShTileBytes;
  const size_t td_bytes = (size_t)k * kShL * nblocks * kblocks * kShTileBytes;
  // scratch: digit planes of b and of T(a), kept with the plan and grown on demand
  int rc = sh_scratch(p, 256 + bd_bytes + td_bytes);
  if (rc != POLYMUL_OK) return rc;
  unsigned char* bd = static_cast<unsigned char*>(p->d_sh) + 256;
  unsigned char* td = bd + bd_bytes;
  const TensorPrime* tp = static_cast<const TensorPrime*>(p->d_tpc);
  const uint32_t wrap = p->cyclic ? 0u : 0x8000u;
  const int wb = p->digit_bits;
  // digit planes
  const uint64_t threads_b = (uint64_t)k * rblocks * kShRows * (n / 8);
  const uint64_t threads_t = (uint64_t)k * nblocks * kShRows * (n / 8);
  const int grid_b = (int)std::min<uint64_t>((threads_b + 255) / 256, (uint64_t)p->num_sms * 16);
  const int grid_t = (int)std::min<uint64_t>((threads_t + 255) / 256, (uint64_t)p->num_sms * 16);
  if (wb == 8) {
    k_shared_bdigits<8><<<grid_b, 256, 0, st>>>((const uint32_t*)b, bd, tp, batch, k, n, rblocks);
    k_shared_tdigits<8><<<grid_t, 256, 0, st>>>((const uint32_t*)a, td, tp, k, n, wrap);
  } else if (wb == 7) {
    k_shared_bdigits<7><<<grid_b, 256, 0, st>>>((const uint32_t*)b, bd, tp, batch, k, n, rblocks);
    k_shared_tdigits<7><<<grid_t, 256, 0, st>>>((const uint32_t*)a, td, tp, k, n, wrap);
  } else {
    return fail(POLYMUL_ENOTSUP, "digit width %d", wb);
  }
  PM_CUDA(cudaGetLastError());
  PM_CUDA(cudaFuncSetAttribute(k_shared_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, kShSmem));
  SharedGemmArgs args{bd, td, (uint32_t*)c, tp, batch, k, n, rblocks, nblocks, kblocks, p->d_err};
  k_shared_gemm<<<k * rblocks * nblocks, kShThreads, kShSmem, st>>>(args);
  PM_CUDA(cudaGetLastError());
  return POLYMUL_OK;
}

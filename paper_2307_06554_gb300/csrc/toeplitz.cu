// Path (b): the paper's matrix form on the tensor cores.
//
// What it computes: c = a * T(b) in Z_q[x]/(x^n+1), the row vector of a
// times the negacyclic (Toeplitz) matrix of b (Sec. 2.2, Eq.
// equ-genereal-mat), for many independent (a, b) pairs.
//
// Large coefficients (Sec. 2.4): each coefficient is taken as its centred
// representative in (-q/2, q/2] and split into L balanced digits of w bits
// (the "several basic units" representation of Sec. 2.4).  Every digit is an
// integer of magnitude <= 2^(w-1) <= 128, exact in bf16; every partial sum of
// digit products has magnitude <= n * 2^(2w-2) <= 2^24 (w is chosen so), so
// the fp32 tensor-core accumulation is exact.  The digit pairs are
// recombined and reduced mod q in the epilogue (Algorithm 1, ConvertMatrix).
//
// Matrix shape (Sec. 2.5 division, 8-coefficient blocks): with
// j = 8u + v (v < 8) and the summation index k = 8d' + r (r < 8),
//   c_j = sum_k  A[u][k] * B[(v)][k],
//   A[u][k] = a~_{8u + k - 8(n/8 - 1)}            (block-Hankel in a)
//   B[v][k] = b~_{8(n/8 - 1 - d') + v - r}         (block-Toeplitz in b)
// where a~, b~ are the antiperiodic extensions (x~_{i-n} = -x_i), so the n
// terms of every sum are exactly the negacyclic convolution; with periodic
// extensions (x~_{i-n} = x_i) the same sums are the cyclic convolution of
// Z_q[x]/(x^n-1), the other ring Sec. 2.1 names (args.wrap selects).  A's rows are
// its digit array shifted by 8 elements = 16 bytes per row, which is the row
// pitch of a tcgen05 core matrix: A is read straight from the 1-D digit
// array through a descriptor with 16-byte K stride and 128-byte row-group
// stride, so it is never materialised.  B (8 rows per digit of b) is
// materialised in the canonical K-major layout.  One MMA chain per digit of
// a and per 128-row block: M = 128, N = 8 L_b (padded to 16), K = n.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "kernels.h"
#include "polymul_types.h"
#include "tcgen05.cuh"
#include "toeplitz_common.cuh"

namespace pm {

template <int LOGN_, int WB_, int LA_, int LB_>
struct TShape {
  static constexpr int LOGN = LOGN_, WB = WB_, LA = LA_, LB = LB_;
  static constexpr int N = 1 << LOGN;
  static constexpr int D = N / 8 - 1;
  static constexpr int RBLK = N / 1024;             // 128-row blocks of A
  static constexpr int NB = (8 * LB + 15) / 16 * 16;  // MMA N
  static constexpr int NG = NB / 8;                 // 8-row groups of B
  static constexpr int TCOLS = RBLK * LA * NB;      // fp32 accumulator columns
  static constexpr int NCOLS = TCOLS <= 32 ? 32 : TCOLS <= 64 ? 64 : TCOLS <= 128 ? 128 : TCOLS <= 256 ? 256 : 512;
  static constexpr int THREADS = 128;
  static constexpr int CPT = N / THREADS;           // coefficients per thread
  static constexpr int GPT = CPT / 8;               // 8-coefficient groups per thread
  static constexpr int XA_LEN = 2 * N;              // a~ over [-n, n)
  static constexpr int XA_OFF = 0;
  // B: K-major core matrices; those adjacent along K are BT_PITCH bytes
  // apart (16 bytes more than the N-groups need, so that the 16-byte
  // stores of consecutive threads, one K-block each, fall in distinct banks)
  static constexpr int BT_PITCH = NG * 128 + 16;
  static constexpr int BT_OFF = (XA_OFF + LA * XA_LEN * 2 + 127) / 128 * 128;
  static constexpr int BT_BYTES = (N / 8) * BT_PITCH;
  static constexpr int SMEM = BT_OFF + BT_BYTES;
  static_assert(TCOLS <= 512, "accumulators exceed tensor memory");
  static_assert(N >= 1024 && CPT % 8 == 0 && THREADS == 128, "n >= 1024, four warps");
  static_assert(N * (1 << (2 * WB - 2)) <= (1 << 24), "digit width breaks fp32 exactness");
};

template <class TS>
__global__ void __launch_bounds__(128, 1) k_toeplitz_batch(TensorBatchArgs args) {
  extern __shared__ __align__(128) unsigned char sm[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t s_tmem;
  __shared__ unsigned long long s_next;
  uint16_t* Xa = reinterpret_cast<uint16_t*>(sm + TS::XA_OFF);
  unsigned char* Bt = sm + TS::BT_OFF;
  // each warp's last 8 digits of b (per digit slot), for the next warp's first lane
  __shared__ __align__(16) uint4 s_edge[4][TS::LB];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint64_t units = args.units;
  const uint32_t k = args.k;
  const uint32_t wrap = args.wrap;  // sign flip of the wrapped-around copies (x^n + 1), none for x^n - 1
  constexpr uint32_t IDESC = idesc_bf16(128, TS::NB);
  constexpr int HALF = 1 << (TS::WB - 1), MASK = (1 << TS::WB) - 1;

  if (warp == 0) {
    tmem_alloc(&s_tmem, TS::NCOLS);
    tmem_relinquish();
  }
  if (tid == 0) mbar_init(&mbar, 1);
  fence_mbar_init();
  // padded rows of B (digit slots >= LB) stay zero for the whole launch
  for (int ch = tid; ch < (TS::N / 8) * TS::NG * 8; ch += TS::THREADS) {
    const int dp = ch / (TS::NG * 8), g = (ch / 8) % TS::NG, v = ch % 8;
    if (g >= TS::LB) *reinterpret_cast<uint4*>(Bt + dp * TS::BT_PITCH + g * 128 + 16 * v) = make_uint4(0, 0, 0, 0);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;

  if (tid == 0) s_next = atomicAdd(args.ctr, 1ull);
  __syncthreads();
  unsigned long long cur = s_next;
  uint32_t parity = 0;
  bool failed = false;
  while (cur < units) {
    __syncthreads();  // every thread has read s_next
    if (tid == 0) s_next = atomicAdd(args.ctr, 1ull);
    const uint32_t j = (uint32_t)(cur % k);
    const uint32_t q = args.tp[j].q;
    const int32_t qh = (int32_t)(q >> 1);

    // ---- ConvertPoly: balanced digits of the centred coefficients, as bf16 ----
    // thread t holds coefficients [t CPT, (t+1) CPT): groups g = t GPT + gi
    const uint32_t* a = args.a + (size_t)cur * TS::N;
    const uint32_t* b = args.b + (size_t)cur * TS::N;
    uint4 bw[TS::GPT][TS::LB];  // b's digits of each own group, bf16 pairs
#pragma unroll
    for (int gi = 0; gi < TS::GPT; ++gi) {
      const int i0 = tid * TS::CPT + 8 * gi;
      const uint4 va0 = *reinterpret_cast<const uint4*>(a + i0);
      const uint4 va1 = *reinterpret_cast<const uint4*>(a + i0 + 4);
      const uint4 vb0 = *reinterpret_cast<const uint4*>(b + i0);
      const uint4 vb1 = *reinterpret_cast<const uint4*>(b + i0 + 4);
      const uint32_t av[8] = {va0.x, va0.y, va0.z, va0.w, va1.x, va1.y, va1.z, va1.w};
      const uint32_t bv[8] = {vb0.x, vb0.y, vb0.z, vb0.w, vb1.x, vb1.y, vb1.z, vb1.w};
      int da[TS::LA][8], db[TS::LB][8];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        int32_t x = (int32_t)av[e] > qh ? (int32_t)(av[e] - q) : (int32_t)av[e];
#pragma unroll
        for (int s = 0; s < TS::LA; ++s) {
          const int32_t d = ((x + HALF) & MASK) - HALF;
          x = (x - d) >> TS::WB;
          da[s][e] = d;
        }
        int32_t y = (int32_t)bv[e] > qh ? (int32_t)(bv[e] - q) : (int32_t)bv[e];
#pragma unroll
        for (int s = 0; s < TS::LB; ++s) {
          const int32_t d = ((y + HALF) & MASK) - HALF;
          y = (y - d) >> TS::WB;
          db[s][e] = d;
        }
      }
#pragma unroll
      for (int s = 0; s < TS::LA; ++s) {
        uint16_t* xs = Xa + s * TS::XA_LEN;
        const uint4 p = make_uint4(bf16x2_of(da[s][0], da[s][1]), bf16x2_of(da[s][2], da[s][3]),
                                   bf16x2_of(da[s][4], da[s][5]), bf16x2_of(da[s][6], da[s][7]));
        *reinterpret_cast<uint4*>(xs + TS::N + i0) = p;
        *reinterpret_cast<uint4*>(xs + i0) = make_uint4(p.x ^ wrap, p.y ^ wrap, p.z ^ wrap, p.w ^ wrap);
      }
#pragma unroll
      for (int s = 0; s < TS::LB; ++s)
        bw[gi][s] = make_uint4(bf16x2_of(db[s][0], db[s][1]), bf16x2_of(db[s][2], db[s][3]),
                               bf16x2_of(db[s][4], db[s][5]), bf16x2_of(db[s][6], db[s][7]));
    }
    if (lane == 31) {
#pragma unroll
      for (int s = 0; s < TS::LB; ++s) s_edge[warp][s] = bw[TS::GPT - 1][s];
    }
    __syncthreads();
    // ---- B tile: row (s', v), column k = 8 d' + r holds b~_{8(D - d') + v - r} ----
    // For the K-block d' = D - g of group g, E[i] = b~_{8g - 8 + i} (i < 16)
    // is the previous group followed by the own one (group -1 is minus the
    // last group, negated for x^n + 1: the extension); row v is E[v + 8 - r],
    // r = 0..7, a reversed window cut from E with byte permutes.
#pragma unroll
    for (int gi = 0; gi < TS::GPT; ++gi) {
      const int g = tid * TS::GPT + gi, dp = TS::D - g;
#pragma unroll
      for (int s2 = 0; s2 < TS::LB; ++s2) {
        uint4 pv;
        if (gi > 0) {
          pv = bw[gi - 1][s2];
        } else {
          const uint4 last = bw[TS::GPT - 1][s2];
          pv.x = __shfl_up_sync(0xffffffffu, last.x, 1);
          pv.y = __shfl_up_sync(0xffffffffu, last.y, 1);
          pv.z = __shfl_up_sync(0xffffffffu, last.z, 1);
          pv.w = __shfl_up_sync(0xffffffffu, last.w, 1);
          if (lane == 0) {
            pv = s_edge[(warp + 3) & 3][s2];
            if (warp == 0) pv = make_uint4(pv.x ^ wrap, pv.y ^ wrap, pv.z ^ wrap, pv.w ^ wrap);
          }
        }
        const uint4 ow = bw[gi][s2];
        const uint32_t E[8] = {pv.x, pv.y, pv.z, pv.w, ow.x, ow.y, ow.z, ow.w};
        b_block_rows(E, Bt + dp * TS::BT_PITCH + s2 * 128);
      }
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();

    // ---- TPUMul: one elected thread issues the MMA chains ----
    if (tid == 0) {
      tc_fence_after();
      const uint32_t xa0 = smem_u32(Xa), bt0 = smem_u32(Bt);
      // descriptors advance by (byte step >> 4) in their address field
      const uint64_t bd0 = smem_desc(bt0, TS::BT_PITCH, 128);
      constexpr uint64_t BSTEP = (2 * TS::BT_PITCH) >> 4;
#pragma unroll 1
      for (int blk = 0; blk < TS::RBLK; ++blk) {
#pragma unroll 1
        for (int s = 0; s < TS::LA; ++s) {
          const uint32_t dcol = tmem + (uint32_t)((blk * TS::LA + s) * TS::NB);
          const uint64_t ad0 = smem_desc(xa0 + (uint32_t)(s * TS::XA_LEN + 8 + 1024 * blk) * 2, 16, 128);
#pragma unroll 8
          for (int kk = 0; kk < TS::N / 16; ++kk)
            tc_mma_f16(dcol, ad0 + 2u * (uint64_t)kk, bd0 + BSTEP * (uint64_t)kk, IDESC, kk > 0 ? 1u : 0u);
        }
      }
      tc_commit(&mbar);
    }
    // warp 0's other lanes wait for the issuing lane at the warp barrier, not
    // in mbarrier polls that would suspend the warp it shares with them
    if (warp == 0) __syncwarp();

    // ---- ConvertMatrix: recombine digit pairs, reduce mod q, store ----
    const bool ok = mbar_wait(&mbar, parity);
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }
    parity ^= 1u;
    tc_fence_after();
    uint32_t* c = args.c + (size_t)cur * TS::N;
    const uint64_t mu = args.tp[j].mu, bias = args.tp[j].bias;
#pragma unroll 1
    for (int blk = 0; blk < TS::RBLK; ++blk) {
      int64_t acc[8];
#pragma unroll
      for (int v = 0; v < 8; ++v) acc[v] = 0;
#pragma unroll
      for (int s = 0; s < TS::LA; ++s) {
#pragma unroll
        for (int c16 = 0; c16 < TS::NB / 16; ++c16) {
          uint32_t r[16];
          tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)((blk * TS::LA + s) * TS::NB + 16 * c16), r);
          tmem_wait_ld();
#pragma unroll
          for (int cc = 0; cc < 16; ++cc) {
            const int col = 16 * c16 + cc, s2 = col / 8, v = col % 8;
            if (s2 < TS::LB)
              acc[v] += (int64_t)__float2int_rn(__uint_as_float(r[cc])) * (int64_t)(int32_t)args.tp[j].pw[s + s2];
          }
        }
      }
      uint32_t out[8];
#pragma unroll
      for (int v = 0; v < 8; ++v) out[v] = barrett64((uint64_t)(acc[v] + (int64_t)bias), q, mu);
      const int u = blk * 128 + tid;
      *reinterpret_cast<uint4*>(c + 8 * u) = make_uint4(out[0], out[1], out[2], out[3]);
      *reinterpret_cast<uint4*>(c + 8 * u + 4) = make_uint4(out[4], out[5], out[6], out[7]);
    }
    tc_fence_before();
    __syncthreads();
    cur = s_next;
  }
  if (failed) {
    if (tid == 0) atomicExch(args.err, 1);
    mbar_wait(&mbar, parity);  // let the MMAs in flight finish before freeing their memory
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, TS::NCOLS);
  }
  if (!failed && tid == 0) {
    __threadfence();
    if (atomicAdd(args.ctr + 1, 1ull) == (unsigned long long)gridDim.x - 1) {
      atomicExch(args.ctr, 0ull);
      atomicExch(args.ctr + 1, 0ull);
    }
  }
}

template <class TS>
static KernelInfo toeplitz_info() {
  KernelInfo ki;
  ki.fn = (const void*)k_toeplitz_batch<TS>;
  ki.block = TS::THREADS;
  ki.smem = TS::SMEM;
  ki.team = TS::THREADS;
  ki.units_per_cta = 1;
  ki.tmem_cols = TS::NCOLS;
  return ki;
}

bool lookup_toeplitz(int logn, int wb, int la, int lb, KernelInfo* ki) {
#define PM_T(LOGN, WB, L)                                                        \
  if (logn == LOGN && wb == WB && la == L && lb == L) {                          \
    *ki = toeplitz_info<TShape<LOGN, WB, L, L>>();                               \
    return true;                                                                 \
  }
  PM_T(10, 8, 2)
  PM_T(10, 8, 3)
  PM_T(10, 8, 4)
  PM_T(11, 7, 2)
  PM_T(11, 7, 3)
#undef PM_T
  return false;
}

}  // namespace pm

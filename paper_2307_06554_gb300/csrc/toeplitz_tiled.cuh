// Device helpers shared by the tiled Toeplitz kernels (toeplitz_tiled.cu,
// toeplitz_ws.cu): balanced digits of centred residues packed as bf16, the
// MMA N and B-operand layout of a tiling, and the drain of a chunk's
// accumulators into 64-bit integer sums.
#pragma once
#include <cuda_bf16.h>

#include <cstdint>
#include <type_traits>

#include "tcgen05.cuh"
#include "toeplitz_common.cuh"

namespace pm {

// balanced w-bit digits of the centred representative of v mod q (v < q <
// 2^31); returns what the L digits leave over (0 whenever L digits cover
// (-q/2, q/2], as the host chooses L; nonzero only for a single-digit
// operand that does not fit one digit)
template <int L>
__device__ __forceinline__ int32_t centred_digits(uint32_t v, uint32_t q, int wb, int (&d)[L]) {
  const int32_t half = 1 << (wb - 1), mask = (1 << wb) - 1;
  int32_t x = v > (q >> 1) ? (int32_t)(v - q) : (int32_t)v;
#pragma unroll
  for (int s = 0; s < L; ++s) {
    const int32_t t = ((x + half) & mask) - half;
    x = (x - t) >> wb;
    d[s] = t;
  }
  return x;
}

// 8 consecutive coefficients (16-byte aligned) -> per digit, 8 bf16 packed
// in a uint4; false if a coefficient does not fit the L digits
template <int L>
__device__ __forceinline__ bool digits8(const uint32_t* src, uint32_t q, int wb, uint4 (&out)[L]) {
  const uint4 v0 = *reinterpret_cast<const uint4*>(src);
  const uint4 v1 = *reinterpret_cast<const uint4*>(src + 4);
  const uint32_t xv[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
  int d[8][L];
  int32_t rest = 0;
#pragma unroll
  for (int e = 0; e < 8; ++e) rest |= centred_digits<L>(xv[e], q, wb, d[e]);
#pragma unroll
  for (int s = 0; s < L; ++s)
    out[s] = make_uint4(bf16x2_of(d[0][s], d[1][s]), bf16x2_of(d[2][s], d[3][s]), bf16x2_of(d[4][s], d[5][s]),
                        bf16x2_of(d[6][s], d[7][s]));
  return rest == 0;
}

// MMA N and the B layout for LB digits of b and S shifted copies of it
template <int LB, int S>
struct TTShape {
  static constexpr int NB = (8 * LB * S + 15) / 16 * 16;  // 8 rows per digit and shift, padded
  static constexpr int NG = NB / 8;                       // 8-row groups of B
  // core matrices adjacent along K are BT_PITCH bytes apart (16 bytes more
  // than the N-groups need: consecutive threads' 16-byte stores, one K-block
  // each, fall in distinct banks)
  static constexpr int BT_PITCH = NG * 128 + 16;
};

// 32 lanes x 8 consecutive 32-bit columns: thread i of the warp receives
// lane (taddr.lane + i); taddr.lane must be the warp's own 32-lane quarter
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr)
               : "memory");
}

// f(integral_constant<int, i>) for i = B .. E - 1
template <int B, int E, class F>
__device__ __forceinline__ void cfor(F&& f) {
  if constexpr (B < E) {
    f(std::integral_constant<int, B>{});
    cfor<B + 1, E>(f);
  }
}

// Adds to acc[v] (output v of this thread's row) the digit pairs (s, g),
// s in [S0, S1), of shift SH of the chains at tensor-memory address `base`
// (chain s at column s N): per e = s + g the exact fp32 sums, each at most
// 2^24 in magnitude, summed in 32-bit integers (at most four: < 2^26), then
// times 2^(8e) mod q in 64 bits -- one multiplication per e instead of one
// per pair.
template <int LA, int LB, int S, int SH, int S0, int S1>
__device__ __forceinline__ void drain_pairs(uint32_t base, const uint32_t* pw, int64_t (&acc)[8]) {
  using TS = TTShape<LB, S>;
  cfor<S0, S1 + LB - 1>([&](auto ec) {
    constexpr int e = decltype(ec)::value;
    constexpr int s_lo = e - (LB - 1) > S0 ? e - (LB - 1) : S0;
    constexpr int s_hi = e + 1 < S1 ? e + 1 : S1;  // s in [s_lo, s_hi): g = e - s in [0, LB)
    uint32_t r[s_hi - s_lo][8];
    cfor<s_lo, s_hi>([&](auto sc) {
      constexpr int s = decltype(sc)::value;
      tmem_ld8(base + (uint32_t)(s * TS::NB + 8 * (SH * LB + (e - s))), r[s - s_lo]);
    });
    tmem_wait_ld();
    const int64_t w = (int64_t)pw[e];
#pragma unroll
    for (int v = 0; v < 8; ++v) {
      int32_t x = 0;
#pragma unroll
      for (int i = 0; i < s_hi - s_lo; ++i) x += __float2int_rn(__uint_as_float(r[i][v]));
      acc[v] += (int64_t)x * w;
    }
  });
}

// one plain arrival on an mbarrier (no transaction bytes)
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

}  // namespace pm

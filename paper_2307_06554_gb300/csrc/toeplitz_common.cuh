// Device helpers shared by the Toeplitz (tensor-core) kernels: exact bf16
// digits, the Barrett reduction of the recombined sums, and the rows of the
// block-Toeplitz operand B cut from a 16-coefficient window.
#pragma once
#include <cstdint>

namespace pm {

// bf16 bit pattern of a small integer d (|d| <= 256, so exact in bf16):
// adding d to the pattern of 1.5 * 2^23 puts d in the units of the
// mantissa; subtracting 1.5 * 2^23 leaves d exactly as a float, whose top
// 16 bits are then its bf16 pattern.  Two digits, packed low/high.
__device__ __forceinline__ uint32_t bf16x2_of(int d0, int d1) {
  const float f0 = __int_as_float(0x4B400000 + d0) - 12582912.0f;
  const float f1 = __int_as_float(0x4B400000 + d1) - 12582912.0f;
  return __byte_perm(__float_as_uint(f0), __float_as_uint(f1), 0x7632);
}

// x mod q for 0 <= x < 2^64 (Barrett, mu = floor(2^64 / q)): the estimate
// is floor(x / q) or one less.
__device__ __forceinline__ uint32_t barrett64(uint64_t x, uint32_t q, uint64_t mu) {
  const uint64_t qh = __umul64hi(x, mu);
  const uint32_t r = (uint32_t)(x - qh * q);
  return r >= q ? r - q : r;
}

// The 8 rows (v = 0..7) of one K-block of B for one digit of b, as eight
// 16-byte core-matrix rows at dst + 16 v.  E holds the window
// b~_{8g - 8 + i}, i = 0..15, as bf16 pairs (E[w] = elements 2w, 2w + 1);
// row v, K-offset r = 0..7 is element 8 + v - r: a reversed window cut with
// byte permutes (low half: element 8 + v - 2jj, high half: 7 + v - 2jj).
__device__ __forceinline__ void b_block_rows(const uint32_t (&E)[8], unsigned char* dst) {
#pragma unroll
  for (int v = 0; v < 8; ++v) {
    uint32_t o[4];
    const int c = v >> 1;
#pragma unroll
    for (int jj = 0; jj < 4; ++jj)
      o[jj] = (v & 1) ? __byte_perm(E[c + 4 - jj], 0u, 0x1032) : __byte_perm(E[c + 4 - jj], E[c + 3 - jj], 0x7610);
    *reinterpret_cast<uint4*>(dst + 16 * v) = make_uint4(o[0], o[1], o[2], o[3]);
  }
}

}  // namespace pm

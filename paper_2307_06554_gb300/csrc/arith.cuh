// Word-size modular arithmetic used by the NTT kernels.
//
// Reduction methods (the paper leaves the choice open and names Montgomery
// and Barrett reduction as the natural next step, Sec. 2.6 "RNS base
// selection", last paragraph):
//   * Shoup multiplication by a precomputed constant w with companion
//     w' = floor(w * 2^bits / q): r = x*w - floor(x*w'/2^bits)*q lies in
//     [0, 2q) for every word x when q < 2^(bits-1).  Three multiplies.
//   * Montgomery multiplication of two variables: returns x*y*2^-bits mod q.
//
// Lazy ranges: for q < 2^(bits-2) values live in [0, 4q) through the forward
// transform and [0, 2q) through the inverse (Harvey's bounds); for
// 2^(bits-2) <= q < 2^(bits-1) ("Q31" mode, 32-bit words only) every sum is
// brought back to [0, q) before it can overflow.
#pragma once
#include <cstdint>

namespace pm {

// x in [0, 2m) -> [0, m): if x < m the subtraction wraps to a value > x.
template <typename W>
__device__ __forceinline__ W csub(W x, W m) {
  W y = x - m;
  return y < x ? y : x;
}

__device__ __forceinline__ uint32_t mulhi(uint32_t a, uint32_t b) { return __umulhi(a, b); }
__device__ __forceinline__ uint64_t mulhi(uint64_t a, uint64_t b) { return __umul64hi(a, b); }

// Shoup: x * w mod q, result in [0, 2q).  Needs q < 2^(bits-1).
template <typename W>
__device__ __forceinline__ W shoup(W x, W w, W wp, W q) {
  W qh = mulhi(x, wp);
  return x * w - qh * q;
}

// Montgomery: (x * y) / 2^bits mod q, result in (-q, x*y/2^bits) shifted by
// +q when negative, i.e. in [0, q + x*y/2^bits).  qinv = q^-1 mod 2^bits.
template <typename W>
__device__ __forceinline__ W montmul(W x, W y, W q, W qinv) {
  W lo = x * y;
  W hi = mulhi(x, y);
  W m = lo * qinv;
  W mh = mulhi(m, q);
  W u = hi - mh;
  return hi < mh ? u + q : u;
}

}  // namespace pm

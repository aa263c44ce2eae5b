// Launch description of one k_ntt_batch instantiation.
#pragma once
#include "kernels.h"
#include "ntt.cuh"

namespace pm {

constexpr int kNttWarps = 4;  // warps per CTA when a team fits in a warp

// Default shape of the batch kernel per word size and degree: stage bits per
// register pass (RB), exchange layout (PAD: 0 the XOR swizzle, else the
// padded layout with one word after every 2^PAD), register budget per thread
// and whether one operand at a time is held in registers (SEQ).  Measured on
// GB300 with 2^22 coefficients per batch (2^21 for 64-bit words), reduction
// modes 1 and 2, launches back to back:
//   32-bit words, n <= 2^9:      radix 16, padded, 96 registers, both operands;
//   32-bit words, n = 2^10,2^11: radix 16, padded, 96 registers, one operand
//                                 (n = 1024, q = 12289: 27.0 -> 25.7 us);
//   32-bit words, n >= 2^12:     radix 16, swizzled, 128 registers (the
//                                 padded kernels were 5-10 % slower there);
//   64-bit words, 2^6 .. 2^11:   radix 8, padded, 96 registers, one operand
//                                 (radix 16 spills: 1.35-1.47x faster);
//   64-bit words, 2^12, 2^13:    radix 16, padded, 128 registers.
template <typename W, int LOGN>
struct NttCfg {
  static constexpr bool u32 = sizeof(W) == 4;
  static constexpr int RB = u32 ? 4 : (LOGN >= 6 && LOGN <= 11 ? 3 : 4);
  static constexpr int PAD = u32 ? (LOGN >= 5 && LOGN <= 11 ? 4 : 0) : (LOGN >= 6 ? RB : 0);
  static constexpr int REGS = u32 ? (LOGN >= 5 && LOGN <= 11 ? 96 : 128) : (LOGN >= 6 && LOGN <= 11 ? 96 : 128);
  static constexpr bool SEQ = u32 ? (LOGN == 10 || LOGN == 11) : (LOGN >= 6 && LOGN <= 11);
};

// every parameter explicit
template <typename W, int LOGN, int MODE, bool AUX, int RB, int REGS, int PAD, bool SEQ, bool DIRECT = false>
KernelInfo ntt_info_x() {
  using S = Shape<W, LOGN, RB, PAD>;
  KernelInfo ki;
  ki.fn = (const void*)k_ntt_batch<S, MODE, kNttWarps, REGS, AUX, SEQ, DIRECT>;
  ki.rb = RB;
  ki.mode = MODE;
  ki.regs = REGS;
  ki.pad = PAD;
  ki.seq = SEQ ? 1 : 0;
  ki.team = S::T;
  if (S::T <= 32) {
    ki.block = 32 * kNttWarps;
    ki.units_per_cta = kNttWarps * (32 / S::T);
  } else {
    ki.block = S::T;
    ki.units_per_cta = 1;
  }
  ki.smem = ki.units_per_cta * S::SMEM_WORDS * (int)sizeof(W);
  return ki;
}

// the default shape for (W, LOGN)
template <typename W, int LOGN, int MODE, bool AUX = false>
KernelInfo ntt_info() {
  using C = NttCfg<W, LOGN>;
  return ntt_info_x<W, LOGN, MODE, AUX, C::RB, C::REGS, C::PAD, C::SEQ>();
}

// another register radix, swizzled layout, 128 registers, both operands
template <typename W, int LOGN, int MODE, bool AUX, int RB>
KernelInfo ntt_info_rb() {
  return ntt_info_x<W, LOGN, MODE, AUX, RB, 128, 0, false>();
}

}  // namespace pm

// Launch description of one k_ntt_batch instantiation.
#pragma once
#include "kernels.h"
#include "ntt.cuh"

namespace pm {

constexpr int kNttWarps = 4;  // warps per CTA when a team fits in a warp

// stage bits held in registers per phase (the radix of the register passes):
// 16 coefficients per operand per thread.  Measured on n = 1024 (32-bit):
// RB = 4 beats RB = 5 (more resident warps for the same work) and RB = 3
// (twice the exchanges).
template <typename W, int LOGN>
constexpr int ntt_rb() {
  return 4;
}

// register budget per thread (measured at n = 1024, 4096 products: 128
// registers 27.5 us; radix 16 at 96 registers (20 warps per SM, no spills)
// 28.0 us; radix 8 at 64 registers (32 warps per SM, no spills) 29.3 us)
template <typename W, int LOGN>
constexpr int ntt_regs() {
  return 128;
}

template <typename W, int LOGN, int MODE, bool AUX = false, int RB = ntt_rb<W, LOGN>(),
          int REGS = ntt_regs<W, LOGN>()>
KernelInfo ntt_info() {
  using S = Shape<W, LOGN, RB>;
  using W_ = W;
  KernelInfo ki;
  ki.fn = (const void*)k_ntt_batch<S, MODE, kNttWarps, REGS, AUX>;
  ki.rb = RB;
  ki.mode = MODE;
  ki.regs = REGS;
  ki.team = S::T;
  if (S::T <= 32) {
    ki.block = 32 * kNttWarps;
    ki.units_per_cta = kNttWarps * (32 / S::T);
  } else {
    ki.block = S::T;
    ki.units_per_cta = 1;
  }
  ki.smem = ki.units_per_cta * S::SMEM_WORDS * (int)sizeof(W_);
  return ki;
}

}  // namespace pm

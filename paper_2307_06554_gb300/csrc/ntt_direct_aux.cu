// k_ntt_batch with direct operand access (see ntt_direct_u32.cu) in
// auxiliary-prime mode: 32-bit words, one NTT prime in (2^30, 2^31), ring
// moduli without a 2n-th root of unity, n = 2^4 .. 2^14, both operands in
// registers.
#include "ntt_info.cuh"

namespace pm {
bool lookup_ntt_direct_aux(int logn, KernelInfo* ki) {
  switch (logn) {
#define PM_CASE(L)                                                                                  \
  case L:                                                                                           \
    *ki = ntt_info_x<uint32_t, L, 0, true, 4, NttCfg<uint32_t, L>::REGS, NttCfg<uint32_t, L>::PAD, \
                     false, true>();                                                                \
    return true;
    PM_CASE(4) PM_CASE(5) PM_CASE(6) PM_CASE(7) PM_CASE(8) PM_CASE(9) PM_CASE(10)
    PM_CASE(11) PM_CASE(12) PM_CASE(13)
#undef PM_CASE
    case 14:  // a 512-thread CTA per product (32 coefficients per operand per thread)
      *ki = ntt_info_x<uint32_t, 14, 0, true, 5, 128, 0, false, true>();
      return true;
    default:
      return false;
  }
}
}  // namespace pm

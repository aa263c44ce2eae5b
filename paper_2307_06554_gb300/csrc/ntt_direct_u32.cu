// k_ntt_batch with direct operand access (DIRECT = true): the kernel of the
// host-buffer entry when a, b and c are page-locked host memory that the
// device maps.  32-bit words, n = 2^4 .. 2^14, reduction mode 0 (values in
// [0, 2q), valid for every modulus below 2^31 and for the tables of every
// mode), both operands in registers so that a team's loads of a and b are
// in flight together.  The host link, not the arithmetic, bounds this
// kernel, so one shape per degree serves every plan.
#include "ntt_info.cuh"

namespace pm {
bool lookup_ntt_direct_u32(int logn, KernelInfo* ki) {
  switch (logn) {
#define PM_CASE(L)                                                                                   \
  case L:                                                                                            \
    *ki = ntt_info_x<uint32_t, L, 0, false, 4, NttCfg<uint32_t, L>::REGS, NttCfg<uint32_t, L>::PAD, \
                     false, true>();                                                                 \
    return true;
    PM_CASE(4) PM_CASE(5) PM_CASE(6) PM_CASE(7) PM_CASE(8) PM_CASE(9) PM_CASE(10)
    PM_CASE(11) PM_CASE(12) PM_CASE(13)
#undef PM_CASE
    case 14:  // a 512-thread CTA per product (32 coefficients per operand per thread)
      *ki = ntt_info_x<uint32_t, 14, 0, false, 5, 128, 0, false, true>();
      return true;
    default:
      return false;
  }
}
}  // namespace pm

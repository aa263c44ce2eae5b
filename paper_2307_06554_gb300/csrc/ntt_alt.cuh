// Alternative k_ntt_batch shapes per degree (see NttCfg in ntt_info.cuh):
// where the default is padded, the swizzled two-operand kernel at 128
// registers; where it is swizzled, the padded one-operand kernel at 96.
#pragma once
#include "ntt_info.cuh"

namespace pm {

template <int MODE>
bool ntt_alt_u32(int logn, KernelInfo* ki) {
  switch (logn) {
#define PM_OLD(L)                                        \
  case L:                                                \
    *ki = ntt_info_rb<uint32_t, L, MODE, false, 4>();    \
    return true;
#define PM_PAD(L)                                                  \
  case L:                                                          \
    *ki = ntt_info_x<uint32_t, L, MODE, false, 4, 96, 4, true>();  \
    return true;
    PM_OLD(5) PM_OLD(6) PM_OLD(7) PM_OLD(8) PM_OLD(9) PM_OLD(10) PM_OLD(11)
    PM_PAD(12) PM_PAD(13)
#undef PM_OLD
#undef PM_PAD
    default:
      return false;
  }
}

}  // namespace pm

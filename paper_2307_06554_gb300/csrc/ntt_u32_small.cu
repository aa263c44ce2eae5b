// k_ntt_batch instantiations: 32-bit words, n = 2^4 .. 2^10.
#include "ntt_info.cuh"

namespace pm {
bool lookup_ntt_u32_small(int logn, bool l4, KernelInfo* ki) {
  switch (logn) {
#define PM_CASE(L)                                                                         \
  case L:                                                                                  \
    *ki = l4 ? ntt_info<uint32_t, L, true>() : ntt_info<uint32_t, L, false>();             \
    return true;
    PM_CASE(4) PM_CASE(5) PM_CASE(6) PM_CASE(7) PM_CASE(8) PM_CASE(9) PM_CASE(10)
#undef PM_CASE
    default:
      return false;
  }
}
}  // namespace pm

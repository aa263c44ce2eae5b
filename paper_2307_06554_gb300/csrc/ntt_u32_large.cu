// k_ntt_batch instantiations: 32-bit words, n = 2^11 .. 2^14.
#include "ntt_info.cuh"

namespace pm {
bool lookup_ntt_u32_large(int logn, bool l4, KernelInfo* ki) {
  switch (logn) {
#define PM_CASE(L)                                                                         \
  case L:                                                                                  \
    *ki = l4 ? ntt_info<uint32_t, L, true>() : ntt_info<uint32_t, L, false>();             \
    return true;
    PM_CASE(11) PM_CASE(12) PM_CASE(13) PM_CASE(14)
#undef PM_CASE
    default:
      return false;
  }
}
}  // namespace pm

// k_ntt_batch instantiations: 64-bit words, reduction mode 1, n = 2^4 .. 2^13.
#include "ntt_info.cuh"

namespace pm {
bool lookup_ntt_u64_m1(int logn, KernelInfo* ki) {
  switch (logn) {
#define PM_CASE(L)                         \
  case L:                                  \
    *ki = ntt_info<uint64_t, L, 1>();      \
    return true;
    PM_CASE(4) PM_CASE(5) PM_CASE(6) PM_CASE(7) PM_CASE(8) PM_CASE(9) PM_CASE(10)
    PM_CASE(11) PM_CASE(12) PM_CASE(13)
#undef PM_CASE
    default:
      return false;
  }
}
}  // namespace pm

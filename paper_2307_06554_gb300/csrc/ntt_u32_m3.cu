// k_ntt_batch instantiations: 32-bit words, reduction mode 3 (q < 2^14,
// 16-bit Shoup quotients), n = 2^4 .. 2^12 (a prime q < 2^14 with
// q = 1 mod 2n needs n <= 2^12).
#include "ntt_info.cuh"

namespace pm {
bool lookup_ntt_u32_m3(int logn, KernelInfo* ki) {
  switch (logn) {
#define PM_CASE(L)                         \
  case L:                                  \
    *ki = ntt_info<uint32_t, L, 3>();      \
    return true;
    PM_CASE(4) PM_CASE(5) PM_CASE(6) PM_CASE(7) PM_CASE(8) PM_CASE(9) PM_CASE(10)
    PM_CASE(11) PM_CASE(12)
#undef PM_CASE
    default:
      return false;
  }
}
}  // namespace pm

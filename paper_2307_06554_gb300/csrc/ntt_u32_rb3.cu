// Radix-8 register passes (8 coefficients per operand per thread, more
// threads per product, more exchanges): autotuner candidates.
// 32-bit words, reduction modes 1 and 2, n = 2^9 .. 2^12.
#include "ntt_info.cuh"

namespace pm {
bool lookup_ntt_u32_rb3(int logn, int mode, KernelInfo* ki) {
#define PM_V(L, M)                                  \
  if (logn == L && mode == M) {                     \
    *ki = ntt_info_rb<uint32_t, L, M, false, 3>();     \
    return true;                                    \
  }
  PM_V(9, 1) PM_V(10, 1) PM_V(11, 1) PM_V(12, 1)
  PM_V(9, 2) PM_V(10, 2) PM_V(11, 2) PM_V(12, 2)
#undef PM_V
  return false;
}
}  // namespace pm

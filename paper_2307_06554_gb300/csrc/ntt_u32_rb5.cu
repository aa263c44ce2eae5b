// Radix-32 register passes (32 coefficients per operand per thread):
// candidates the autotuner weighs against the default radix-16 kernels
// (n <= 2^13) and against the thread-block-cluster kernel (n = 2^14, where
// a 512-thread CTA holds the whole product).
// 32-bit words, reduction modes 1 and 2, n = 2^9 .. 2^13; modes 0..2 at 2^14.
#include "ntt_info.cuh"

namespace pm {
bool lookup_ntt_u32_rb5(int logn, int mode, KernelInfo* ki) {
#define PM_V(L, M)                                  \
  if (logn == L && mode == M) {                     \
    *ki = ntt_info_rb<uint32_t, L, M, false, 5>();     \
    return true;                                    \
  }
  PM_V(9, 1) PM_V(10, 1) PM_V(11, 1) PM_V(12, 1) PM_V(13, 1)
  PM_V(9, 2) PM_V(10, 2) PM_V(11, 2) PM_V(12, 2) PM_V(13, 2)
  PM_V(14, 0) PM_V(14, 1) PM_V(14, 2)
#undef PM_V
  return false;
}
}  // namespace pm

// Radix-8 register passes for 64-bit words (half the registers of the
// default radix-16 kernels, which spill): autotuner candidates.
// Reduction mode 1, n = 2^9 .. 2^12.
#include "ntt_info.cuh"

namespace pm {
bool lookup_ntt_u64_rb3(int logn, int mode, KernelInfo* ki) {
#define PM_V(L, M)                                  \
  if (logn == L && mode == M) {                     \
    *ki = ntt_info<uint64_t, L, M, false, 3>();     \
    return true;                                    \
  }
  PM_V(9, 1) PM_V(10, 1) PM_V(11, 1) PM_V(12, 1)
#undef PM_V
  return false;
}
}  // namespace pm

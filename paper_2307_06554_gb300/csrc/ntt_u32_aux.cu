// k_ntt_batch instantiations in auxiliary-prime mode: 32-bit words, one NTT
// prime in (2^30, 2^31) (reduction mode 0), n = 2^4 .. 2^14.
#include "ntt_info.cuh"

namespace pm {
bool lookup_ntt_u32_aux(int logn, KernelInfo* ki) {
  switch (logn) {
#define PM_CASE(L)                           \
  case L:                                    \
    *ki = ntt_info<uint32_t, L, 0, true>();  \
    return true;
    PM_CASE(4) PM_CASE(5) PM_CASE(6) PM_CASE(7) PM_CASE(8) PM_CASE(9) PM_CASE(10)
    PM_CASE(11) PM_CASE(12) PM_CASE(13) PM_CASE(14)
#undef PM_CASE
    default:
      return false;
  }
}

// Radix-4 register passes (4 coefficients per operand per thread, four
// times the threads per product): shorter dependency chains per thread, for
// batches too small to fill the GPU, where one product's latency is the
// whole call (autotuner candidates; the exchange swizzle is conflict-free
// for these team sizes, n >= 2^7).
bool lookup_ntt_u32_aux_rb2(int logn, KernelInfo* ki) {
  switch (logn) {
#define PM_CASE(L)                              \
  case L:                                       \
    *ki = ntt_info_rb<uint32_t, L, 0, true, 2>();  \
    return true;
    PM_CASE(7) PM_CASE(8) PM_CASE(9) PM_CASE(10)
#undef PM_CASE
    default:
      return false;
  }
}
}  // namespace pm

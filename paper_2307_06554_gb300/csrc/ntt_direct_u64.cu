// k_ntt_batch with direct operand access (see ntt_direct_u32.cu): 64-bit
// words, n = 2^4 .. 2^13, reduction mode 1 (Harvey's bounds, valid for every
// modulus below 2^62 and for the tables of every mode), both operands in
// registers.
#include "ntt_info.cuh"

namespace pm {
bool lookup_ntt_direct_u64(int logn, KernelInfo* ki) {
  switch (logn) {
#define PM_CASE(L)                                                                                   \
  case L:                                                                                            \
    *ki = ntt_info_x<uint64_t, L, 1, false, NttCfg<uint64_t, L>::RB, NttCfg<uint64_t, L>::REGS,     \
                     NttCfg<uint64_t, L>::PAD, false, true>();                                       \
    return true;
    PM_CASE(4) PM_CASE(5) PM_CASE(6) PM_CASE(7) PM_CASE(8) PM_CASE(9) PM_CASE(10)
    PM_CASE(11) PM_CASE(12) PM_CASE(13)
#undef PM_CASE
    default:
      return false;
  }
}
}  // namespace pm

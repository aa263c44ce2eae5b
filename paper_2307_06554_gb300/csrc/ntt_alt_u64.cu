// k_ntt_batch alternative shapes, 64-bit words, reduction mode 1 (autotuner
// candidates): radix 16, padded, both operands, 128 registers where the
// default is the radix-8 one-operand kernel (2^6 .. 2^11), and that radix-8
// kernel where the default is radix 16 (2^12; at 2^13 its 1024-thread CTA
// leaves 64 registers per thread).
#include "ntt_alt.cuh"

namespace pm {

bool lookup_ntt_alt_u32_m1(int logn, KernelInfo* ki);
bool lookup_ntt_alt_u32_m2(int logn, KernelInfo* ki);

bool lookup_ntt_alt(uint32_t elem, int logn, int mode, KernelInfo* ki) {
  if (elem == 4) {
    if (mode == 1) return lookup_ntt_alt_u32_m1(logn, ki);
    if (mode == 2) return lookup_ntt_alt_u32_m2(logn, ki);
    return false;
  }
  if (mode != 1) return false;
  switch (logn) {
#define PM_R16(L)                                                   \
  case L:                                                           \
    *ki = ntt_info_x<uint64_t, L, 1, false, 4, 128, 4, false>();    \
    return true;
#define PM_R8(L)                                                    \
  case L:                                                           \
    *ki = ntt_info_x<uint64_t, L, 1, false, 3, 96, 3, true>();      \
    return true;
    PM_R16(6) PM_R16(7) PM_R16(8) PM_R16(9) PM_R16(10) PM_R16(11)
    PM_R8(12)
#undef PM_R16
#undef PM_R8
    default:
      return false;
  }
}

}  // namespace pm

// k_ntt_batch alternative shapes, 32-bit words, reduction mode 1: the shape
// the default was measured against at each degree (autotuner candidates).
#include "ntt_alt.cuh"

namespace pm {
bool lookup_ntt_alt_u32_m1(int logn, KernelInfo* ki) { return ntt_alt_u32<1>(logn, ki); }
}  // namespace pm

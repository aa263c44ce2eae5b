// Registry of compiled kernel instantiations (one translation unit per
// size range, so that they compile in parallel).
#pragma once
#include <cstdint>

namespace pm {

struct KernelInfo {
  const void* fn = nullptr;  // __global__ entry, launched with cudaLaunchKernel
  int block = 0;             // threads per CTA
  int smem = 0;              // dynamic shared memory bytes per CTA
  int team = 0;              // threads per unit
  int units_per_cta = 0;     // units a CTA processes per iteration
};

// batched negacyclic NTT, k_ntt_batch<W, LOGN, L4>
bool lookup_ntt_u32_small(int logn, bool l4, KernelInfo* ki);  // logn 4..10
bool lookup_ntt_u32_large(int logn, bool l4, KernelInfo* ki);  // logn 11..14
bool lookup_ntt_u64(int logn, bool l4, KernelInfo* ki);        // logn 4..13

}  // namespace pm

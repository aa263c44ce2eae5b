// Path (b) for moduli up to 2^62 in 64-bit words: launch arguments and the
// host-side tiling of the 64-bit digit kernel (see toeplitz_u64.cu).
#pragma once
#include <cstdint>

#include "kernels.h"
#include "toeplitz_tiled.h"

namespace pm {

// Per prime: digit-pair weights 2^(8e) mod q for e = s + g < 2L - 1 with
// their Shoup companions floor(w 2^64 / q), and a multiple of q at or above
// 2^28 that makes every per-weight integer sum of a chunk non-negative.
struct alignas(16) TensorPrime64 {
  uint64_t q;
  uint64_t bias;
  uint64_t pw[15];
  uint64_t pwp[15];
};

struct TensorU64Args {
  const uint64_t* a;
  const uint64_t* b;
  uint64_t* c;
  const TensorPrime64* tp;  // indexed by pmap[row % k] (or row % k without a map)
  const uint32_t* pmap;     // k table indices, or null
  uint64_t units;           // batch * k * ngrp
  uint32_t k;
  uint32_t wrap;            // bf16x2 sign mask of the operand extensions: 0x80008000 (x^n + 1) or 0 (x^n - 1)
  uint32_t logn;
  uint32_t ngrp, kc, a_win, bt_off, tmem_cols;
  unsigned long long* ctr;  // {next unit, finished CTAs}
  int* err;
};

// Tiling of degree 2^logn (2^10 .. 2^16) with L 8-bit digits per operand
// (5 .. 8): one A slice of 1024 outputs per unit of work, L chains of
// N = 8 L (padded to 16) in at most 512 tensor-memory columns, K chunks of
// at most 1024 (exact fp32 sums per chunk), one CTA per SM.
bool toeplitz_u64_config(int logn, int L, TiledCfg* cfg);
bool lookup_toeplitz_u64(int logn, int L, KernelInfo* ki);

// balanced 8-bit digits that cover the centred residues of moduli up to
// qmax (0 if more than 8 are needed)
int u64_digits(uint64_t qmax);

}  // namespace pm

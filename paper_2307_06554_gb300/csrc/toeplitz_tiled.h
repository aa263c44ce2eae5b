// Path (b) at every degree 2^6 .. 2^14: launch arguments and the host-side
// choice of output groups and K chunks (see toeplitz_tiled.cu).
#pragma once
#include <cstdint>

#include "kernels.h"
#include "polymul_types.h"

namespace pm {

// Tiling of one (product, prime) row: the outputs in blocks of 1024 (128
// rows of A, 8 outputs each); a unit of work (`ngrp` per row) covers
// `bpg` x `shifts` blocks: `bpg` consecutive A slices (one MMA chain per
// slice and digit of a), or, with `shifts` > 1, one A slice against that
// many copies of b shifted by 1024 coefficients in the B operand (N = nb
// columns, K-blocks `b_pitch` bytes apart); the summation dimension in
// chunks of `kc`.  Shared memory per CTA: the digit window of a~ (la x
// a_win bf16 values) at offset 0 and the chunk of B at `bt_off`.
struct TiledCfg {
  uint32_t bpg = 0, shifts = 0, nb = 0, b_pitch = 0, ngrp = 0, kc = 0, a_win = 0, bt_off = 0, tmem_cols = 0;
  int smem = 0;
  uint32_t stage_bytes = 0;  // warp-specialised kernel: bytes per shared-memory stage (two stages)
};

struct TensorTiledArgs {
  const uint32_t* a;
  const uint32_t* b;
  uint32_t* c;
  const TensorPrime* tp;  // [k]
  uint64_t units;         // batch * k * ngrp
  uint32_t k;
  uint32_t wrap;          // bf16x2 sign mask of the operand extensions: 0x80008000 (x^n + 1) or 0 (x^n - 1)
  uint32_t logn, wb;      // degree, digit width
  uint32_t bpg, ngrp, kc, a_win, bt_off, tmem_cols;
  unsigned long long* ctr;  // {next unit, finished CTAs}
  int* err;
  // NULL: row r (product r / k, prime r % k) at element offset r n of a, b,
  // c with tp[r % k]; else row r at rows[r].offset with tp[rows[r].prime]
  // (the rows of one degree class of an uneven list)
  const RaggedUnit* rows;
  uint32_t stage_bytes;  // warp-specialised kernel: shared-memory stage size (0 otherwise)
};

// The tiling for degree 2^logn with la digits of a and lb of b (false if
// the accumulators of one 128-row block do not fit in 256 tensor-memory
// columns).
bool toeplitz_tiled_config(int logn, int la, int lb, TiledCfg* cfg);

// k_toeplitz_tiled<LA, LB, S> for LA = LB = 1 .. 5 and for LA = 1, LB = 2
// .. 5 (a single-digit operand on the A side), S the shifts the tiling
// chose; ki->smem and ki->tmem_cols from the tiling of degree 2^logn.
bool lookup_toeplitz_tiled(int logn, int la, int lb, KernelInfo* ki);

// The drained variant: each K chunk's fp32 accumulators are drained into
// 64-bit integer sums, so 8-bit digits are exact at every degree (chunks of
// at most 1024); at most 4 digits (every q < 2^31); with la == lb one A
// slice per unit of work against shifted copies of b as tensor memory
// allows, with la == 1 up to 4 A slices.  ki->wb = 8, ki->digits = lb.
bool toeplitz_tiled_config_drain(int logn, int la, int lb, TiledCfg* cfg);
bool lookup_toeplitz_tiled_drain(int logn, int la, int lb, KernelInfo* ki);

// The drained kernel as a warp-specialised pipeline (k_toeplitz_ws, one CTA
// per SM): two shared-memory stages and two tensor-memory buffers, so that
// builder warps fill one stage and drainer warps empty one buffer while the
// MMAs of the other run.  Same digits, shifts and slices as the drained
// kernel; K chunks as large as two stages allow.  ki->ws = 1, ki->drain = 1.
bool toeplitz_ws_config(int logn, int la, int lb, TiledCfg* cfg);
bool lookup_toeplitz_ws(int logn, int la, int lb, KernelInfo* ki);

}  // namespace pm

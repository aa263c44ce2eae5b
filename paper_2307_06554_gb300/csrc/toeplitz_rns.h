// Path (b) with the paper's residue number system of small moduli
// (Sec. 2.4; the RNS base of the key-parameter section): launch arguments,
// device tables and the host-side choice of the base (toeplitz_rns.cu).
#pragma once
#include <cstdint>
#include <vector>

#include "kernels.h"

namespace pm {

constexpr int kRnsMax = 32;  // small moduli per base (16 tensor-memory columns each)

// The base, shared by every prime of a plan.
struct RnsBase {
  uint32_t r;                // number of moduli
  uint32_t m[kRnsMax];       // the moduli: odd, pairwise coprime, largest first
  uint32_t mu32[kRnsMax];    // floor(2^32 / m): residues of 32-bit values
  uint32_t t[kRnsMax];       // (M / m_i)^-1 mod m_i, M the product of the moduli
  uint32_t off[kRnsMax];     // the least multiple of m_i >= 2^24 (makes accumulator values non-negative)
  float inv_m[kRnsMax];      // 1 / m_i
  uint64_t mu64[kRnsMax];    // floor(2^64 / m): residues of 64-bit values
};

// Per prime q of the plan.
struct RnsPrime {
  uint64_t q;
  uint64_t mq;               // M mod q
  uint64_t Mq[kRnsMax];      // (M / m_i) mod q
  uint32_t qm[kRnsMax];      // q mod m_i
};

struct TensorRnsArgs {
  const int8_t* ra;          // [batch * k][r][n] centred residues of a's lift (k_rns_prep)
  const int8_t* rb;          // the same for b
  void* c;
  const RnsBase* base;
  const RnsPrime* tp;        // [k]
  uint64_t units;            // batch * k * ngrp
  uint32_t k;
  uint32_t wrap;             // bf16x2 sign mask of the operand extensions: 0x80008000 (x^n + 1) or 0 (x^n - 1)
  uint32_t logn;
  uint32_t shifts;           // S: 1024-output blocks per unit, one per shifted copy of b in the B operand
  uint32_t nb;               // MMA N = max(16, 8 S)
  uint32_t b_pitch;          // bytes between K-blocks of B
  uint32_t ngrp, kc, a_win, bt_off, buf_bytes, tmem_cols;
  unsigned long long* ctr;   // {next unit, finished CTAs}
  int* err;
};

struct RnsCfg {
  uint32_t shifts = 0, nb = 0, b_pitch = 0, ngrp = 0, kc = 0, a_win = 0, bt_off = 0, buf_bytes = 0, tmem_cols = 0;
  int smem = 0;
};

// Largest odd modulus whose centred residues keep every fp32 partial sum of
// a degree-n product exact: n ((m - 1) / 2)^2 <= 2^24, and m < 2^8.
uint32_t rns_modulus_cap(uint32_t n);

// The base for degree n and moduli up to qmax: odd moduli from the cap down,
// each kept if coprime to those already kept, until their product exceeds
// 16 n floor(qmax/2)^2 (the centred product's range, with the margin the
// reconstruction's rounded quotient needs).  False if kRnsMax moduli do not
// reach it.
bool rns_choose_base(uint32_t n, uint64_t qmax, std::vector<uint32_t>* moduli);

// Tables of the base and of each prime (host side).
void rns_tables(const std::vector<uint32_t>& moduli, const std::vector<uint64_t>& primes, RnsBase* base,
                std::vector<RnsPrime>* per_prime);

// Shifts per unit, K chunk and the shared-memory stages for degree 2^logn
// and r moduli.
bool rns_config(int logn, uint32_t r, RnsCfg* cfg);

// k_toeplitz_rns<W> for 4-byte (elem 4) or 8-byte words; smem and
// tensor-memory columns from rns_config.
bool lookup_toeplitz_rns(int logn, uint32_t r, uint32_t elem, KernelInfo* ki);

// Residue planes of a and b for `rows` (product, prime) rows of degree n:
// out[(x * rows + row) * r + i][n] (x = 0 for a, 1 for b), on `stream`.
// Returns the launch's cudaError_t.
int rns_prep_launch(uint32_t elem, const void* a, const void* b, int8_t* out, uint64_t rows, uint32_t n,
                    uint32_t k, const RnsBase* base, const RnsPrime* tp, uint32_t r, int num_sms, void* stream);

}  // namespace pm

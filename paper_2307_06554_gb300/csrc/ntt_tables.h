// Host-side NTT tables of one prime (plan creation): bit-reversed powers of
// psi and psi^-1 with Shoup companions, and the per-prime constants.
#pragma once
#include <cstdint>
#include <vector>

#include "host_math.h"
#include "polymul_types.h"

namespace pm {

template <typename W>
inline void build_ntt_tables(uint64_t q, uint32_t n, std::vector<W>& twf, std::vector<W>& twi, PrimeConst<W>& pc) {
  using namespace pm::host;
  using pm::host::u128;
  const int bits = 8 * (int)sizeof(W);
  const int logn = __builtin_ctz(n);
  const uint64_t psi = primitive_2n_root(q, n);
  const uint64_t psi_inv = powmod(psi, q - 2, q);
  twf.resize(2 * (size_t)n);
  twi.resize(2 * (size_t)n);
  for (uint32_t i = 0; i < n; ++i) {
    const uint32_t r = bitrev(i, logn);
    const uint64_t w = powmod(psi, r, q), v = powmod(psi_inv, r, q);
    twf[2 * i] = (W)w;
    twf[2 * i + 1] = (W)shoup_companion(w, q, bits);
    twi[2 * i] = (W)v;
    twi[2 * i + 1] = (W)shoup_companion(v, q, bits);
  }
  const uint64_t r_mod_q = bits == 64 ? (uint64_t)(((u128)1 << 64) % q) : (uint64_t)((1ull << 32) % q);
  const uint64_t ninv = powmod(n, q - 2, q);
  const uint64_t scale = mulmod(ninv, r_mod_q, q);
  const uint64_t scale_w = mulmod(powmod(psi_inv, bitrev(1, logn), q), scale, q);
  pc.q = (W)q;
  pc.q2 = (W)(2 * q);
  pc.qinv = (W)inv_pow2_64(q);  // low bits are the inverse mod 2^32 too
  pc.scale = (W)scale;
  pc.scale_p = (W)shoup_companion(scale, q, bits);
  pc.scale_w = (W)scale_w;
  pc.scale_wp = (W)shoup_companion(scale_w, q, bits);
  pc.pad = 0;
}

// Reduction mode for the largest modulus (see the mode notes in ntt.cuh):
// 2 = no conditional subtractions, 1 = Harvey [0, 4q), 0 = [0, 2q).
inline int ntt_mode(uint64_t qmax, uint32_t logn, uint32_t elem) {
  using pm::host::u128;
  const int bits = 8 * (int)elem;
  const u128 lim = (u128)1 << bits;
  const u128 g = 1 + 2 * (u128)logn;
  if (((u128)qmax << (logn + 1)) < lim && g * g * qmax < lim) return 2;
  if ((u128)qmax * 4 < lim) return 1;
  if ((u128)qmax * 2 < lim) return 0;
  return -1;
}

}  // namespace pm

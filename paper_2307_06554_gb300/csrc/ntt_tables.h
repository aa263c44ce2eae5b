// Host-side NTT tables of one prime (plan creation): bit-reversed powers of
// psi and psi^-1 with Shoup companions, and the per-prime constants.
//
// The kernels walk a fixed tree of butterflies; the ring is set by the
// table.  Entry k (heap order, level l = floor(log2 k), j = k - 2^l) is the
// root that splits node k's polynomial x^(2m) - z^2 into x^m - z and
// x^m + z:
//   x^n + 1 (negacyclic): psi^brv(k), psi of order 2n (q = 1 mod 2n);
//   x^n - 1 (cyclic, Sec. 2.1's other ring): w^(brv(j)/2), w of order n
//   (q = 1 mod n); the root node splits x^n - 1 by z = 1.
// brv is the bit reversal over log2 n bits.
#pragma once
#include <cstdint>
#include <vector>

#include "host_math.h"
#include "polymul_types.h"

namespace pm {

// Writes 2n words to each of twf and twi (caller-owned) and the constants.
template <typename W>
inline void build_ntt_tables_into(uint64_t q, uint32_t n, W* twf, W* twi, PrimeConst<W>& pc, bool cyclic = false) {
  using namespace pm::host;
  using pm::host::u128;
  const int bits = 8 * (int)sizeof(W);
  const int logn = __builtin_ctz(n);
  // negacyclic: root psi, exponent brv(k); cyclic: root w, exponent brv(j)/2
  const uint64_t psi = cyclic ? primitive_n_root(q, n) : primitive_2n_root(q, n);
  const uint64_t psi_inv = powmod(psi, q - 2, q);
  for (uint32_t i = 0; i < n; ++i) {
    uint32_t r = bitrev(i, logn);
    if (cyclic) r = i == 0 ? 0u : bitrev(i - (1u << (31 - __builtin_clz(i))), logn) / 2;
    const uint64_t w = powmod(psi, r, q), v = powmod(psi_inv, r, q);
    twf[2 * i] = (W)w;
    twf[2 * i + 1] = (W)shoup_companion(w, q, bits);
    twi[2 * i] = (W)v;
    twi[2 * i + 1] = (W)shoup_companion(v, q, bits);
  }
  const uint64_t r_mod_q = bits == 64 ? (uint64_t)(((u128)1 << 64) % q) : (uint64_t)((1ull << 32) % q);
  const uint64_t ninv = powmod(n, q - 2, q);
  const uint64_t scale = mulmod(ninv, r_mod_q, q);
  // the last inverse stage's twiddle (table entry 1) folded into its scale
  const uint64_t v1 = cyclic ? 1 : powmod(psi_inv, bitrev(1, logn), q);
  const uint64_t scale_w = mulmod(v1, scale, q);
  pc.q = (W)q;
  pc.q2 = (W)(2 * q);
  pc.qinv = (W)inv_pow2_64(q);  // low bits are the inverse mod 2^32 too
  pc.scale = (W)scale;
  pc.scale_p = (W)shoup_companion(scale, q, bits);
  pc.scale_w = (W)scale_w;
  pc.scale_wp = (W)shoup_companion(scale_w, q, bits);
  pc.pad = 0;
}

template <typename W>
inline void build_ntt_tables(uint64_t q, uint32_t n, std::vector<W>& twf, std::vector<W>& twi, PrimeConst<W>& pc,
                             bool cyclic = false) {
  twf.resize(2 * (size_t)n);
  twi.resize(2 * (size_t)n);
  build_ntt_tables_into<W>(q, n, twf.data(), twi.data(), pc, cyclic);
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

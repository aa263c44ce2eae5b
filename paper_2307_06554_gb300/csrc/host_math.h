// Host-side number theory for plan construction (roots of unity, twiddle
// tables, constants).  Runs once per plan; nothing here is on the batch path.
#pragma once
#include <cstdint>
#include <vector>

namespace pm {
namespace host {

typedef unsigned __int128 u128;

inline uint64_t mulmod(uint64_t a, uint64_t b, uint64_t m) { return (uint64_t)((u128)a * b % m); }

inline uint64_t powmod(uint64_t b, uint64_t e, uint64_t m) {
  uint64_t r = 1 % m;
  b %= m;
  while (e) {
    if (e & 1) r = mulmod(r, b, m);
    b = mulmod(b, b, m);
    e >>= 1;
  }
  return r;
}

// Deterministic Miller-Rabin for 64-bit integers (first twelve prime bases).
inline bool is_prime(uint64_t m) {
  static const uint64_t bases[] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
  if (m < 2) return false;
  for (uint64_t p : bases) {
    if (m % p == 0) return m == p;
  }
  uint64_t d = m - 1;
  int s = 0;
  while ((d & 1) == 0) {
    d >>= 1;
    ++s;
  }
  for (uint64_t a : bases) {
    uint64_t x = powmod(a, d, m);
    if (x == 1 || x == m - 1) continue;
    bool comp = true;
    for (int r = 1; r < s; ++r) {
      x = mulmod(x, x, m);
      if (x == m - 1) {
        comp = false;
        break;
      }
    }
    if (comp) return false;
  }
  return true;
}

// psi with psi^n = -1 (mod prime q), i.e. of multiplicative order exactly 2n
// (n a power of two).  Requires 2n | q-1.  Deterministic: smallest base.
inline uint64_t primitive_2n_root(uint64_t q, uint64_t n) {
  uint64_t e = (q - 1) / (2 * n);
  for (uint64_t g = 2; g < q; ++g) {
    uint64_t psi = powmod(g, e, q);
    if (powmod(psi, n, q) == q - 1) return psi;
  }
  return 0;
}

// w of multiplicative order exactly n (mod prime q; n a power of two >= 2),
// i.e. w^(n/2) = -1.  Requires n | q-1.  Deterministic: smallest base.
inline uint64_t primitive_n_root(uint64_t q, uint64_t n) {
  uint64_t e = (q - 1) / n;
  for (uint64_t g = 2; g < q; ++g) {
    uint64_t w = powmod(g, e, q);
    if (powmod(w, n / 2, q) == q - 1) return w;
  }
  return 0;
}

inline uint32_t bitrev(uint32_t x, int bits) {
  uint32_t r = 0;
  for (int i = 0; i < bits; ++i) r |= ((x >> i) & 1u) << (bits - 1 - i);
  return r;
}

// x^-1 mod 2^64 for odd x (Newton: each step doubles the correct low bits)
inline uint64_t inv_pow2_64(uint64_t x) {
  uint64_t y = x;  // correct to 3 bits for odd x
  for (int i = 0; i < 6; ++i) y *= 2 - x * y;
  return y;
}

// floor(w * 2^bits / q)
inline uint64_t shoup_companion(uint64_t w, uint64_t q, int bits) {
  return (uint64_t)(((u128)w << bits) / q);
}

}  // namespace host
}  // namespace pm

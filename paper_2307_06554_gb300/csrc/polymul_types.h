// Structures shared by the host code and the kernels of libpolymul.
#pragma once
#include <cstdint>

namespace pm {

// Per-prime constants of one NTT plan (device resident, one per prime).
template <typename W>
struct alignas(16) PrimeConst {
  W q;         // the prime
  W q2;        // 2q
  W qinv;      // q^-1 mod 2^bits (Montgomery)
  W scale;     // n^-1 * 2^bits mod q   (undoes the Montgomery factor and 1/n)
  W scale_p;   // Shoup companion of scale
  W scale_w;   // psi^-brv(1) * scale mod q (last inverse stage twiddle)
  W scale_wp;  // Shoup companion of scale_w
  W pad;
};

// One (product, prime) row of an uneven list: its element offset in a, b, c
// and its prime's index in the pool.
struct alignas(16) RaggedUnit {
  uint64_t offset;  // element offset of the row in a, b, c
  uint32_t prime;   // index into the prime pool
  uint32_t pad;
};

template <typename W>
struct NttBatchArgs {
  const W* a;
  const W* b;
  W* c;
  const void* tw_fwd;  // [k][n] TwPair<W>, psi^brv(i)
  const void* tw_inv;  // [k][n] TwPair<W>, psi^-brv(i)
  const PrimeConst<W>* pc;  // [k]
  uint64_t units;      // batch * k
  uint32_t k;
  unsigned long long* ctr;  // {next unit, finished teams}, zero between launches
  int* err;                 // set to 1 when a bounded device wait expires
  const W* outer_q;         // auxiliary-prime mode: the ring moduli [k]
  // Table selection: unit prime j uses tables of prime pj = pmap ? pmap[j] : j,
  // twiddles at tw_fwd/tw_inv + pj * tw_stride pairs and constants
  // pc[pj * pc_stride + pc_off].  A plan passes (null, n, 1, 0); a server whose
  // tables cover a prime pool at the largest degree passes the request's pool
  // indices, that degree and the per-degree constant slot.
  const uint32_t* pmap;
  uint32_t tw_stride;
  uint32_t pc_stride;
  uint32_t pc_off;
  // 1: the previous kernel on the stream is a batch launch of this library
  // that writes none of a, b and touches none of c (checked by the host), so
  // each team may load and multiply its first unit before waiting for it
  uint32_t early;
  // diagnostics (0 in normal use): extra bytes each unit's completion
  // barrier expects beyond what its copies deliver, and the poll limit of
  // its bounded waits (0: the default).  A nonzero tx_pad makes every wait
  // expire after wait_polls polls, the path of a copy that never completes.
  uint32_t tx_pad;
  uint32_t wait_polls;
  // unit prime j's table index as 8-bit fields (index j in byte j & 3 of word
  // j >> 2) when pmap_inline is set: up to 32 primes of a pool of at most
  // 256, carried by the launch itself instead of a device array
  uint32_t pmap_inline;
  uint32_t pmap_pack[8];
  // kernels with one team per CTA only: when set, unit u is the row at
  // rows[u].offset with tables of pool prime rows[u].prime (the rows of one
  // degree class of an uneven list); k and the prime map are then unused
  const RaggedUnit* rows;
};

// table index of unit prime j (see NttBatchArgs::pmap, pmap_pack)
template <typename W>
__device__ __forceinline__ uint32_t table_index(const NttBatchArgs<W>& args, uint32_t j) {
  if (args.pmap_inline) {
    uint32_t w = args.pmap_pack[0];
#pragma unroll
    for (uint32_t i = 1; i < 8; ++i) w = (j >> 2) == i ? args.pmap_pack[i] : w;  // no dynamic parameter index
    return (w >> (8 * (j & 3))) & 255u;
  }
  return args.pmap ? args.pmap[j] : j;
}

// Ragged (uneven) batches: one unit = one (product, prime) row of n words.
// Degree segments per list: at most one per degree; the work counters of a
// list are kRaggedMaxSegs segment counters and one finished-CTA count.
constexpr int kRaggedMaxSegs = 15;

// One degree segment: `count` consecutive units of degree 2^logn.
struct alignas(16) RaggedItem {
  uint32_t logn;
  uint32_t first;
  uint32_t count;
  uint32_t pad;
};

struct RaggedArgs {
  const uint32_t* a;
  const uint32_t* b;
  uint32_t* c;
  const RaggedUnit* units;
  const RaggedItem* items;
  uint64_t n_items;
  const void* tw_fwd;              // [pool][nmax] TwPair<uint32_t>
  const void* tw_inv;
  const PrimeConst<uint32_t>* pc;  // [pool][16]: constants for degree 2^logn at [p * 16 + logn]
  uint32_t nmax;
  unsigned long long* ctr;
  int* err;
};

// Shared-operand products on the NTT path (k_ntt_prep / k_ntt_shared).
template <typename W>
struct NttSharedArgs {
  const W* a;      // prep: [k][n] operand; product kernel: a^ in register layout [k][T][R]
  const W* b;      // [batch][k][n]
  W* c;            // prep: a^ out; product kernel: [batch][k][n]
  const void* tw_fwd;
  const void* tw_inv;
  const PrimeConst<W>* pc;
  uint64_t units;  // prep: k; product kernel: pairs of products, ceil(batch / 2) * k
  uint64_t batch;  // product kernel: products per prime
  uint32_t k;
  uint32_t tw_stride;
  unsigned long long* ctr;  // {next, finished}, zero between launches
  int* err;
};

// Per-prime constants of the Toeplitz (tensor) path.
struct alignas(16) TensorPrime {
  uint32_t q;
  uint32_t pw[15];  // pw[e] = 2^(w e) mod q: weight of digit pair (s, s') with s + s' = e
  uint64_t mu;      // floor(2^64 / q), Barrett reduction of the recombined sums
  uint64_t bias;    // the multiple of q at or just above 2^60 (makes every recombined sum positive)
};

struct TensorBatchArgs {
  const uint32_t* a;
  const uint32_t* b;
  uint32_t* c;
  const TensorPrime* tp;  // [k]
  uint64_t units;         // batch * k
  uint32_t k;
  uint32_t wrap;          // sign of the operand extensions, as a bf16x2 XOR mask: 0x80008000 for x^n + 1, 0 for x^n - 1
  unsigned long long* ctr;  // {next unit, finished CTAs}
  int* err;
};

}  // namespace pm

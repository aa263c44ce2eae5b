// Uneven batches in one persistent launch: products of different degrees n
// (2^10 .. 2^14) and different numbers of RNS primes (each prime a separate
// ring, Sec. 2.4), all through the negacyclic NTT unit of ntt.cuh.
//
// The host flattens the products into units (product, prime) and packs units
// of the same degree into work items of up to 512 / T units (T = threads per
// unit), largest degree first; CTAs of 512 threads take items from a device
// counter.  Inside an item each team of T threads owns one unit: its leader
// bulk-copies the unit's operand rows into the team's shared buffers
// (tracked by the team's own mbarrier), the team synchronises on its own
// named barrier, and the result goes straight back to HBM.  Twiddle tables
// are built once per pool prime at the largest degree: the table for n is
// the length-n prefix of the table for n_max (psi_n = psi_nmax^(nmax/n) and
// bit reversal of a log n-bit index into log nmax bits multiplies it by
// nmax/n).
#include <cuda_runtime.h>

#include "kernels.h"
#include "ntt.cuh"
#include "polymul_types.h"

namespace pm {

constexpr int kRaggedThreads = 512;
constexpr int kRaggedMaxTeams = 8;

// team barrier: named barrier `id` (1..15) over `n` threads
struct TeamSync {
  uint32_t id, n;
  __device__ __forceinline__ void operator()() const {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
  }
};

// degree class -> register radix (16 coefficients per thread up to 2^13,
// 32 for 2^14 so that a unit fits in 512 threads)
template <int LOGN>
using RaggedShape = Shape<uint32_t, LOGN, (LOGN <= 13 ? 4 : 5)>;

struct NoHook {
  __device__ __forceinline__ void operator()() const {}
};

// `phases`: one parity bit per team barrier (an item completes one phase on
// the barriers of the teams it uses, and only on those)
template <class S, int MODE>
__device__ __forceinline__ bool ragged_item(const RaggedArgs& args, const RaggedItem& item, uint32_t* smem,
                                            uint64_t* mbar, uint32_t& phases) {
  static_assert(S::T <= kRaggedThreads && S::T >= 32, "team size");
  constexpr int TEAMS = kRaggedThreads / S::T;
  static_assert(TEAMS <= kRaggedMaxTeams, "too many teams");
  constexpr uint32_t ROW = S::N * 4u;
  const uint32_t team = threadIdx.x / S::T, t = threadIdx.x % S::T;
  uint32_t* sa = smem + (size_t)team * S::SMEM_WORDS;
  uint32_t* sb = sa + S::SLICE;
  const bool act = team < item.count;
  const RaggedUnit unit = args.units[item.first + (act ? team : 0u)];
  if (t == 0) {
    // inactive teams copy the item's first unit again so that every team's
    // barrier completes exactly one phase per item
    fence_proxy_async();
    mbar_arrive_expect_tx(&mbar[team], 2 * ROW);
    bulk_g2s(sa, args.a + unit.offset, ROW, &mbar[team]);
    bulk_g2s(sb, args.b + unit.offset, ROW, &mbar[team]);
  }
  // a bounded wait; the team agrees on its outcome (barrier reduction) so
  // that its barriers stay uniform
  uint32_t fail = mbar_wait(&mbar[team], (phases >> team) & 1u) ? 0u : 1u;
  phases ^= (1u << TEAMS) - 1u;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 q, %1, 0;\n\t"
      "bar.red.or.pred p, %2, %3, q;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(fail)
      : "r"(fail), "r"(1u + team), "r"((uint32_t)S::T)
      : "memory");
  const bool ok = fail == 0;
  const PrimeConst<uint32_t> pc = args.pc[(size_t)unit.prime * 16 + S::LOGN];
  const TwPair<uint32_t>* twf = reinterpret_cast<const TwPair<uint32_t>*>(args.tw_fwd) + (size_t)unit.prime * args.nmax;
  const TwPair<uint32_t>* twi = reinterpret_cast<const TwPair<uint32_t>*>(args.tw_inv) + (size_t)unit.prime * args.nmax;
  polymul_unit<S, MODE, false>(args.c + unit.offset, twf, twi, pc, sa, sb, t, act && ok, TeamSync{1 + team, S::T},
                               NoHook{});
  return ok;
}

template <int MODE>
__global__ void __launch_bounds__(kRaggedThreads, 1) k_ntt_ragged(RaggedArgs args) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t mbar[kRaggedMaxTeams];
  __shared__ RaggedItem s_item;
  uint32_t* smem = reinterpret_cast<uint32_t*>(smem_raw);
  if (threadIdx.x < kRaggedMaxTeams) mbar_init(&mbar[threadIdx.x], 1);
  fence_mbar_init();
  __syncthreads();
  uint32_t phases = 0;
  bool failed = false;
  for (;;) {
    if (threadIdx.x == 0) {
      const unsigned long long w = atomicAdd(args.ctr, 1ull);
      if (w < args.n_items) {
        s_item = args.items[w];
      } else {
        s_item.count = 0;
      }
    }
    __syncthreads();
    const RaggedItem item = s_item;
    __syncthreads();
    if (item.count == 0) break;
    bool ok = true;
    switch (item.logn) {
      case 10: ok = ragged_item<RaggedShape<10>, MODE>(args, item, smem, mbar, phases); break;
      case 11: ok = ragged_item<RaggedShape<11>, MODE>(args, item, smem, mbar, phases); break;
      case 12: ok = ragged_item<RaggedShape<12>, MODE>(args, item, smem, mbar, phases); break;
      case 13: ok = ragged_item<RaggedShape<13>, MODE>(args, item, smem, mbar, phases); break;
      case 14: ok = ragged_item<RaggedShape<14>, MODE>(args, item, smem, mbar, phases); break;
      default: break;
    }
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }
  }
  if (failed) {
    if (threadIdx.x == 0) atomicExch(args.err, 1);
    // let copies in flight land: a barrier whose current phase is pending
    // completes it (parity bit = the phase being waited for)
    if (threadIdx.x < kRaggedMaxTeams) mbar_wait(&mbar[threadIdx.x], ((phases >> threadIdx.x) & 1u) ^ 1u);
    return;
  }
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(args.ctr + 1, 1ull) == (unsigned long long)gridDim.x - 1) {
      atomicExch(args.ctr, 0ull);
      atomicExch(args.ctr + 1, 0ull);
    }
  }
}

// dynamic shared memory: the largest class's team buffers
int ragged_smem_bytes() {
  int m = 0;
  m = m > (kRaggedThreads / RaggedShape<10>::T) * RaggedShape<10>::SMEM_WORDS * 4 ? m : (kRaggedThreads / RaggedShape<10>::T) * RaggedShape<10>::SMEM_WORDS * 4;
  m = m > (kRaggedThreads / RaggedShape<11>::T) * RaggedShape<11>::SMEM_WORDS * 4 ? m : (kRaggedThreads / RaggedShape<11>::T) * RaggedShape<11>::SMEM_WORDS * 4;
  m = m > (kRaggedThreads / RaggedShape<12>::T) * RaggedShape<12>::SMEM_WORDS * 4 ? m : (kRaggedThreads / RaggedShape<12>::T) * RaggedShape<12>::SMEM_WORDS * 4;
  m = m > (kRaggedThreads / RaggedShape<13>::T) * RaggedShape<13>::SMEM_WORDS * 4 ? m : (kRaggedThreads / RaggedShape<13>::T) * RaggedShape<13>::SMEM_WORDS * 4;
  m = m > (kRaggedThreads / RaggedShape<14>::T) * RaggedShape<14>::SMEM_WORDS * 4 ? m : (kRaggedThreads / RaggedShape<14>::T) * RaggedShape<14>::SMEM_WORDS * 4;
  return m;
}

int ragged_teams(int logn) {
  switch (logn) {
    case 10: return kRaggedThreads / RaggedShape<10>::T;
    case 11: return kRaggedThreads / RaggedShape<11>::T;
    case 12: return kRaggedThreads / RaggedShape<12>::T;
    case 13: return kRaggedThreads / RaggedShape<13>::T;
    case 14: return kRaggedThreads / RaggedShape<14>::T;
    default: return 0;
  }
}

bool lookup_ntt_ragged(int mode, KernelInfo* ki) {
  if (mode != 0 && mode != 1) return false;
  ki->fn = mode == 0 ? (const void*)k_ntt_ragged<0> : (const void*)k_ntt_ragged<1>;
  ki->block = kRaggedThreads;
  ki->smem = ragged_smem_bytes();
  ki->team = 0;
  ki->units_per_cta = 1;
  ki->tmem_cols = 0;
  return true;
}

}  // namespace pm

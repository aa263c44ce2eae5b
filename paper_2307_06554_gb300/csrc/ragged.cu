// Uneven batches in one persistent launch: products of different degrees n
// (2^10 .. 2^14) and different numbers of RNS primes (each prime a separate
// ring, Sec. 2.4), all through the negacyclic NTT unit of ntt.cuh.
//
// The host flattens the products into units (product, prime) and sorts them
// into degree segments, largest degree first.  CTAs of 512 threads walk the
// segments in order; inside a segment the CTA is cut into teams of T threads
// (T = threads per unit), and each team takes units from the segment's
// device counter on its own, synchronising on its own named barrier, so that
// teams drift apart as independent CTAs would and their exchange and
// arithmetic phases overlap.  A CTA waits for all its teams only when it
// moves to the next segment (a new team layout).  Twiddle tables
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
static_assert(kRaggedMaxSegs >= 5, "one segment per degree 2^10 .. 2^14");

// team barrier: named barrier `id` (1..15) over `n` threads
struct TeamSync {
  uint32_t id, n;
  __device__ __forceinline__ void operator()() const {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
  }
};

// degree class -> register radix (16 coefficients per thread up to 2^13,
// 32 for 2^14 so that a unit fits in 512 threads).  Two shape sets, chosen
// per list by measurement (polymul_ragged_tune):
//   set 0: the XOR-swizzled exchange layout, both operands in registers;
//   set 1: the padded layout (one word after every 2^RB, a base register
//          plus constant offsets per layout), one operand in registers at a
//          time for 2^10, 2^11 (as the homogeneous kernels measured) and for
//          2^14, whose 32 coefficients per operand and thread otherwise spill.
constexpr int ragged_rb(int logn) { return logn <= 13 ? 4 : 5; }
template <int LOGN, int SET>
using RaggedShape = Shape<uint32_t, LOGN, ragged_rb(LOGN), SET == 1 ? ragged_rb(LOGN) : 0>;
template <int LOGN, int SET>
constexpr bool ragged_seq() {
  return SET == 1 && (LOGN == 10 || LOGN == 11 || LOGN == 14);
}

// One degree segment: the units of degree 2^LOGN, taken one at a time by
// the teams of the CTA (T threads each, 512 / T teams) from the segment's
// own counter, every team on its own: its leader bulk-copies the unit's
// rows into the team's buffers (tracked by the team's mbarrier), and as soon
// as the unit's last exchange is done it takes the next unit and issues that
// copy, which then overlaps the last inverse pass.  `phases`: one parity bit
// per team barrier, exact for the thread's own team (teams complete
// different numbers of phases); at the end the leader publishes its team's
// bit in s_bits[team] so that the CTA can agree on all of them.  Returns
// false when a bounded wait expired (the team stops; the copy it waited for
// is the only one it has in flight).
template <class S, int MODE, bool SEQ>
__device__ __forceinline__ bool ragged_segment(const RaggedArgs& args, const RaggedItem& seg,
                                               unsigned long long* ctr, uint32_t* smem, uint64_t* mbar,
                                               uint32_t& phases, unsigned long long* s_next, uint32_t* s_bits) {
  static_assert(S::T <= kRaggedThreads && S::T >= 32, "team size");
  static_assert(kRaggedThreads / S::T <= kRaggedMaxTeams, "too many teams");
  constexpr uint32_t ROW = S::N * 4u;
  const uint32_t team = threadIdx.x / S::T, t = threadIdx.x % S::T;
  uint32_t* sa = smem + (size_t)team * S::SMEM_WORDS;
  uint32_t* sb = sa + S::SLICE;
  const TeamSync sync{1 + team, S::T};
  auto take = [&]() {  // team leader: next unit index of the segment, and its copy
    const unsigned long long u = atomicAdd(ctr, 1ull);
    s_next[team] = u;
    if (u < seg.count) {
      const RaggedUnit un = args.units[seg.first + u];
      fence_proxy_async();
      mbar_arrive_expect_tx(&mbar[team], 2 * ROW);
      bulk_g2s(sa, args.a + un.offset, ROW, &mbar[team]);
      bulk_g2s(sb, args.b + un.offset, ROW, &mbar[team]);
    }
  };
  if (t == 0) take();
  sync();
  unsigned long long cur = s_next[team];
  while (cur < seg.count) {
    // a bounded wait; the team agrees on its outcome (barrier reduction)
    uint32_t fail = mbar_wait(&mbar[team], (phases >> team) & 1u) ? 0u : 1u;
    phases ^= 1u << team;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 q, %1, 0;\n\t"
        "bar.red.or.pred p, %2, %3, q;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(fail)
        : "r"(fail), "r"(1u + team), "r"((uint32_t)S::T)
        : "memory");
    if (fail) break;
    const RaggedUnit unit = args.units[seg.first + cur];
    const PrimeConst<uint32_t> pc = args.pc[(size_t)unit.prime * 16 + S::LOGN];
    const TwPair<uint32_t>* twf = reinterpret_cast<const TwPair<uint32_t>*>(args.tw_fwd) + (size_t)unit.prime * args.nmax;
    const TwPair<uint32_t>* twi = reinterpret_cast<const TwPair<uint32_t>*>(args.tw_inv) + (size_t)unit.prime * args.nmax;
    auto hook = [&]() {  // the whole team, once sa/sb are free
      if (t == 0) take();
    };
    polymul_unit_any<S, MODE, false, SEQ>(args.c + unit.offset, twf, twi, pc, sa, sb, sa, sb, t, true, sync, hook);
    sync();  // the leader's s_next[team] is visible
    cur = s_next[team];
  }
  if (t == 0) s_bits[team] = (phases >> team) & 1u;
  return cur >= seg.count;
}

// `items`: the degree segments, largest degree first; ctr[i] is segment i's
// unit counter, ctr[kRaggedMaxSegs] the count of finished CTAs (the last one
// resets them all).  A CTA changes team layout only between segments.
// One instantiation serves the degrees 2^LO .. 2^HI: the 2^14 body (32
// coefficients per thread) has a kernel of its own, so that its register
// pressure (and the spills it causes) does not reach the other degrees.
template <int MODE, int LO, int HI, int SET>
__global__ void __launch_bounds__(kRaggedThreads, 1) k_ntt_ragged(RaggedArgs args) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t mbar[kRaggedMaxTeams];
  __shared__ unsigned long long s_next[kRaggedMaxTeams];
  __shared__ uint32_t s_bits[2][kRaggedMaxTeams];  // per segment parity: published barrier phase bits
  uint32_t* smem = reinterpret_cast<uint32_t*>(smem_raw);
  if (threadIdx.x < kRaggedMaxTeams) mbar_init(&mbar[threadIdx.x], 1);
  fence_mbar_init();
  __syncthreads();
  uint32_t phases = 0;
  bool failed = false;
  for (uint64_t i = 0; i < args.n_items; ++i) {
    const RaggedItem seg = args.items[i];
    unsigned long long* ctr = args.ctr + i;
    uint32_t* bits = s_bits[i & 1];
    bool ok = true;
    int teams = 0;
    switch (seg.logn) {
#define PM_SEG(L)                                                                                      \
  case L:                                                                                              \
    if constexpr (L >= LO && L <= HI) {                                                                 \
      ok = ragged_segment<RaggedShape<L, SET>, MODE, ragged_seq<L, SET>()>(args, seg, ctr, smem, mbar,  \
                                                                           phases, s_next, bits);       \
      teams = kRaggedThreads / RaggedShape<L, SET>::T;                                                  \
    }                                                                                                   \
    break;
      PM_SEG(10) PM_SEG(11) PM_SEG(12) PM_SEG(13) PM_SEG(14)
#undef PM_SEG
      default: break;
    }
    // every team is done with the segment's layout before the next one
    const bool any_fail = __syncthreads_or(!ok);
    // agree on the phase bits of the barriers this segment used (the next
    // segment may put this thread in another team)
    for (int tm = 0; tm < teams; ++tm) phases = (phases & ~(1u << tm)) | (bits[tm] << tm);
    if (any_fail) {
      failed = true;
      break;
    }
  }
  if (failed) {
    if (threadIdx.x == 0) atomicExch(args.err, 1);
    // let the copy in flight land: a barrier whose current phase is pending
    // completes it (parity bit = the phase being waited for); the others
    // return at once
    if (threadIdx.x < kRaggedMaxTeams) mbar_wait(&mbar[threadIdx.x], ((phases >> threadIdx.x) & 1u) ^ 1u);
    return;
  }
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(args.ctr + kRaggedMaxSegs, 1ull) == (unsigned long long)gridDim.x - 1) {
      for (uint64_t i = 0; i < args.n_items; ++i) atomicExch(args.ctr + i, 0ull);
      atomicExch(args.ctr + kRaggedMaxSegs, 0ull);
    }
  }
}

// dynamic shared memory of one degree class's team buffers
template <int L, int SET>
constexpr int ragged_class_smem() {
  return (kRaggedThreads / RaggedShape<L, SET>::T) * RaggedShape<L, SET>::SMEM_WORDS * 4;
}

template <int MODE, int LO, int HI, int SET>
static void ragged_info(KernelInfo* ki) {
  ki->fn = (const void*)k_ntt_ragged<MODE, LO, HI, SET>;
  ki->block = kRaggedThreads;
  int m = 0;
  if (LO <= 10 && 10 <= HI) m = m > ragged_class_smem<10, SET>() ? m : ragged_class_smem<10, SET>();
  if (LO <= 11 && 11 <= HI) m = m > ragged_class_smem<11, SET>() ? m : ragged_class_smem<11, SET>();
  if (LO <= 12 && 12 <= HI) m = m > ragged_class_smem<12, SET>() ? m : ragged_class_smem<12, SET>();
  if (LO <= 13 && 13 <= HI) m = m > ragged_class_smem<13, SET>() ? m : ragged_class_smem<13, SET>();
  if (LO <= 14 && 14 <= HI) m = m > ragged_class_smem<14, SET>() ? m : ragged_class_smem<14, SET>();
  ki->smem = m;
  ki->team = 0;
  ki->units_per_cta = 1;
  ki->tmem_cols = 0;
}

// small: degrees 2^10 .. 2^13; big: 2^14; `set` as for RaggedShape
bool lookup_ntt_ragged(int mode, int set, KernelInfo* small, KernelInfo* big) {
#define PM_R(M, S)                    \
  if (mode == M && set == S) {        \
    ragged_info<M, 10, 13, S>(small); \
    ragged_info<M, 14, 14, S>(big);   \
    return true;                      \
  }
  PM_R(0, 0) PM_R(0, 1) PM_R(1, 0) PM_R(1, 1)
#undef PM_R
  return false;
}

}  // namespace pm

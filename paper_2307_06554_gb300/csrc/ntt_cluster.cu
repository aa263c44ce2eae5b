// Negacyclic NTT products whose degree exceeds one CTA: a thread-block
// cluster of C = n / 8192 CTAs (512 threads each) is one team, every thread
// holding 16 coefficients of each operand.  The exchanges between register
// passes go through distributed shared memory: coefficient j lives in the
// shared buffer of cluster rank j / 8192, at the same XOR-swizzled position
// as in a single-CTA team; stores and loads reach the other CTAs' shared
// memory through generic addresses of the cluster window (mapa), and the
// team barrier is the cluster barrier.  Operands are loaded and results
// stored directly (the top-phase layout makes both fully coalesced); units
// are assigned to clusters statically.
#include <cuda_runtime.h>

#include "kernels.h"
#include "ntt.cuh"
#include "polymul_types.h"

namespace pm {

constexpr int kClusterThreads = 512;
constexpr int kClusterLocalLog = 13;  // 8192 coefficients per CTA and operand

template <typename W, int RB, int LOCAL_LOG>
struct ClusterBuf {
  static constexpr bool kCluster = true;
  W* base;  // generic address of this buffer in the executing CTA
  __device__ __forceinline__ W* ptr(uint32_t j) const {
    const uint32_t rank = j >> LOCAL_LOG;
    W* loc = base + spos<RB>(j & ((1u << LOCAL_LOG) - 1u));
    W* r;
    // the same shared-memory offset in cluster rank `rank`, as a generic address
    asm("mapa.u64 %0, %1, %2;" : "=l"(r) : "l"(loc), "r"(rank));
    return r;
  }
  __device__ __forceinline__ void store(uint32_t j, W v) const { *ptr(j) = v; }
  __device__ __forceinline__ W load(uint32_t j) const { return *ptr(j); }
};

struct ClusterSync {
  __device__ __forceinline__ void operator()() const {
    asm volatile(
        "barrier.cluster.arrive.release.aligned;\n\t"
        "barrier.cluster.wait.acquire.aligned;" ::
            : "memory");
  }
};

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cluster_id() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cluster_count() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(r));
  return r;
}

struct NoHookC {
  __device__ __forceinline__ void operator()() const {}
};

// Double-buffered exchanges (32-bit words: four buffers fit in shared
// memory).  Exchange e of a unit (forward exchanges first, e = 0, 1, ...)
// uses buffer set e & 1, so a set is written again only two exchanges after
// it was last read, with a whole exchange's barrier in between: no team
// barrier is needed before the stores, only the one that publishes them.
// Across units the same holds (the last exchange of a unit uses set 1, the
// first of the next set 0).
template <class S, int MODE, int P, class Buf, typename W = typename S::W>
__device__ __forceinline__ void fwd_db(W (&xa)[S::R], W (&xb)[S::R], const Buf (&a)[2], const Buf (&b)[2],
                                       const TwPair<W>* __restrict__ tw, const PrimeConst<W>& pc, uint32_t t) {
  fwd_phase2<S, MODE, P>(xa, xb, tw, pc, t);
  if constexpr (P > 0) {
    constexpr int SET = (S::NPH - 1 - P) & 1;
    store_layout<S, P>(xa, a[SET], t);
    store_layout<S, P>(xb, b[SET], t);
    ClusterSync{}();
    load_layout<S, P - 1>(xa, a[SET], t);
    load_layout<S, P - 1>(xb, b[SET], t);
    fwd_db<S, MODE, P - 1>(xa, xb, a, b, tw, pc, t);
  }
}

template <class S, int MODE, int P, class Buf, typename W = typename S::W>
__device__ __forceinline__ void inv_db(W (&x)[S::R], const Buf (&a)[2], const TwPair<W>* __restrict__ tw,
                                       const PrimeConst<W>& pc, uint32_t t) {
  inv_phase<S, MODE, P>(x, tw, pc, t);
  if constexpr (P + 1 < S::NPH) {
    constexpr int SET = (S::NPH - 1 + P) & 1;
    store_layout<S, P>(x, a[SET], t);
    ClusterSync{}();
    load_layout<S, P + 1>(x, a[SET], t);
    inv_db<S, MODE, P + 1>(x, a, tw, pc, t);
  }
}

// DB: double-buffered exchanges (four buffers of 8192 words per CTA)
template <class S, int MODE, bool DB>
__global__ void __launch_bounds__(kClusterThreads, 1) k_ntt_cluster(NttBatchArgs<typename S::W> args) {
  using W = typename S::W;
  using Buf = ClusterBuf<W, S::RB, kClusterLocalLog>;
  static_assert(S::T % kClusterThreads == 0 && S::N == (S::T / kClusterThreads) << kClusterLocalLog,
                "one CTA per 8192 coefficients");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  W* buf = reinterpret_cast<W*>(smem_raw);
  constexpr uint32_t L = 1u << kClusterLocalLog;
  const Buf sa{buf};
  const Buf sb{buf + L};
  const Buf da[2] = {Buf{buf}, Buf{buf + 2 * L}};
  const Buf db[2] = {Buf{buf + L}, Buf{buf + 3 * L}};
  const uint32_t t = cluster_rank() * kClusterThreads + threadIdx.x;
  constexpr int TOP = S::NPH - 1;
  const TwPair<W>* twf = reinterpret_cast<const TwPair<W>*>(args.tw_fwd);
  const TwPair<W>* twi = reinterpret_cast<const TwPair<W>*>(args.tw_inv);
  for (uint64_t u = cluster_id(); u < args.units; u += cluster_count()) {
    const uint32_t j = (uint32_t)(u % args.k);
    const uint32_t pj = table_index(args, j);
    const PrimeConst<W> pc = args.pc[(size_t)pj * args.pc_stride + args.pc_off];
    const W* a = args.a + (size_t)u * S::N;
    const W* b = args.b + (size_t)u * S::N;
    W xa[S::R], xb[S::R];
    sfor<0, S::R>([&](auto ec) {
      constexpr int e = decltype(ec)::value;
      const uint32_t i = elem_index<S, TOP>(e, t);
      xa[e] = a[i];
      xb[e] = b[i];
    });
    if constexpr (DB) {
      fwd_db<S, MODE, TOP>(xa, xb, da, db, twf + (size_t)pj * args.tw_stride, pc, t);
    } else {
      fwd_from<S, MODE, TOP>(xa, xb, sa, sb, twf + (size_t)pj * args.tw_stride, pc, t, ClusterSync{});
    }
    sfor<0, S::R>([&](auto ec) {
      constexpr int e = decltype(ec)::value;
      if constexpr (MODE == kSmall) {
        xa[e] = montmul(xa[e], xb[e], pc.q, pc.qinv);
      } else if constexpr (MODE == kL4) {
        xa[e] = csub(montmul(xa[e], xb[e], pc.q, pc.qinv), pc.q2);
      } else {
        xa[e] = montmul(csub(xa[e], pc.q), csub(xb[e], pc.q), pc.q, pc.qinv);
      }
    });
    if constexpr (DB) {
      inv_db<S, MODE, 0>(xa, da, twi + (size_t)pj * args.tw_stride, pc, t);
    } else {
      inv_from<S, MODE, 0>(xa, sa, twi + (size_t)pj * args.tw_stride, pc, t, ClusterSync{}, NoHookC{});
    }
    W* c = args.c + (size_t)u * S::N;
    sfor<0, S::R>([&](auto ec) {
      constexpr int e = decltype(ec)::value;
      c[elem_index<S, TOP>(e, t)] = csub(xa[e], pc.q);
    });
    if constexpr (!DB) ClusterSync{}();  // no CTA reuses its buffers while another still reads them
  }
  ClusterSync{}();  // no CTA leaves while another may still address its shared memory
}

// ---------------------------------------------------------------- local exchanges
// Second form of the cluster kernel.  Coefficient j's home is cluster rank
// j >> 13 (8192 per CTA and operand), local index j & 8191.  In every layout
// but the top phase's, the team-thread bits that select the CTA (bits 9 and
// up of t = rank * 512 + thread) sit at coefficient bits 13 and up: each
// thread's coefficients live in its own CTA, and an exchange between two such
// layouts runs through the CTA's own shared memory with a CTA barrier (a warp
// barrier when the warps keep their coefficients).  Only the exchange into
// or out of the top phase reaches the other CTAs (distributed shared memory)
// and takes the cluster barrier.  Buffers use the padded layout on the local
// index (word jl at jl + (jl >> PAD)).
template <class S, int P>
constexpr bool cta_local() {
  for (int b = 9; (1 << b) < S::T; ++b)
    if (tbit_pos<S, P>(b) != b + (kClusterLocalLog - 9)) return false;
  return true;
}

template <class S>
__host__ __device__ constexpr uint32_t lpos(uint32_t jl) {
  return jl + (jl >> S::PAD);
}

// elem_index(e, 0) as a constant expression: the slot part of a coefficient
// index in layout P
template <class S, int P>
__host__ __device__ constexpr uint32_t elem_index_c(int e) {
  using PB = PhaseBits<S, P>;
  const uint32_t u = (uint32_t)e & (PB::GS - 1);
  const uint32_t g = (uint32_t)S::T * (uint32_t)(e >> PB::B);
  return (g & ((1u << PB::LO) - 1)) | (u << PB::LO) | ((g >> PB::LO) << PB::HI);
}

// This thread's base address in the buffer of every cluster rank, computed
// in place at each exchange (one mapa per rank; volatile, so that the
// compiler does not keep 64-bit remote addresses alive across the unit).
template <class S, typename W>
__device__ __forceinline__ void rank_bases(W* local, W* (&rb)[S::T / kClusterThreads]) {
  sfor<0, S::T / kClusterThreads>([&](auto rc) {
    constexpr int r = decltype(rc)::value;
    asm volatile("mapa.u64 %0, %1, %2;" : "=l"(rb[r]) : "l"(local), "r"(r));
  });
}

// stores of register slots in layout P: local layouts into this CTA's buffer,
// the top layout into each coefficient's home CTA; both as a base plus
// constant offsets (the local index is the OR of the thread part and the
// slot part, and the padded position is additive over it)
template <class S, int P, typename W = typename S::W>
__device__ __forceinline__ void cstore(const W (&x)[S::R], W* buf, uint32_t t) {
  constexpr uint32_t M = (1u << kClusterLocalLog) - 1u;
  W* base = buf + lpos<S>(elem_index<S, P>(0, t) & M);
  if constexpr (cta_local<S, P>()) {
    sfor<0, S::R>([&](auto ec) {
      constexpr int e = decltype(ec)::value;
      base[lpos<S>(elem_index<S, P>(e, 0) & M)] = x[e];
    });
  } else {
    W* rb[S::T / kClusterThreads];
    rank_bases<S>(base, rb);
    sfor<0, S::R>([&](auto ec) {
      constexpr int e = decltype(ec)::value;
      constexpr uint32_t je = elem_index_c<S, P>(e);  // the home rank comes from the slot bits
      rb[je >> kClusterLocalLog][lpos<S>(je & M)] = x[e];
    });
  }
}

template <class S, int P, typename W = typename S::W>
__device__ __forceinline__ void cload(W (&x)[S::R], W* buf, uint32_t t) {
  constexpr uint32_t M = (1u << kClusterLocalLog) - 1u;
  W* base = buf + lpos<S>(elem_index<S, P>(0, t) & M);
  if constexpr (cta_local<S, P>()) {
    sfor<0, S::R>([&](auto ec) {
      constexpr int e = decltype(ec)::value;
      x[e] = base[lpos<S>(elem_index<S, P>(e, 0) & M)];
    });
  } else {
    W* rb[S::T / kClusterThreads];
    rank_bases<S>(base, rb);
    sfor<0, S::R>([&](auto ec) {
      constexpr int e = decltype(ec)::value;
      constexpr uint32_t je = elem_index_c<S, P>(e);
      x[e] = rb[je >> kClusterLocalLog][lpos<S>(je & M)];
    });
  }
}

// barrier between the stores in layout P and the loads in layout Q
template <class S, int P, int Q>
__device__ __forceinline__ void cmid() {
  if constexpr (!(cta_local<S, P>() && cta_local<S, Q>()))
    ClusterSync{}();
  else if constexpr (warp_local<S, P, Q>())
    __syncwarp();
  else
    __syncthreads();
}

// Before the stores of an exchange nothing is needed: a local layout is
// stored at the positions this thread loaded, and the top layout's remote
// stores follow a cluster barrier that every CTA passed after its last
// access to the buffer (see k_ntt_cluster2).
template <class S, int MODE, int P, bool TWO, typename W = typename S::W>
__device__ __forceinline__ void cfwd(W (&xa)[S::R], W (&xb)[S::R], W* sa, W* sb, const TwPair<W>* __restrict__ tw,
                                     const PrimeConst<W>& pc, uint32_t t) {
  fwd_phase<S, MODE, P, TWO>(xa, xb, tw, pc, t);
  if constexpr (P > 0) {
    cstore<S, P>(xa, sa, t);
    if constexpr (TWO) cstore<S, P>(xb, sb, t);
    cmid<S, P, P - 1>();
    cload<S, P - 1>(xa, sa, t);
    if constexpr (TWO) cload<S, P - 1>(xb, sb, t);
    cfwd<S, MODE, P - 1, TWO>(xa, xb, sa, sb, tw, pc, t);
  }
}

template <class S, int MODE, int P, typename W = typename S::W>
__device__ __forceinline__ void cinv(W (&x)[S::R], W* s, const TwPair<W>* __restrict__ tw, const PrimeConst<W>& pc,
                                     uint32_t t) {
  inv_phase<S, MODE, P>(x, tw, pc, t);
  if constexpr (P + 1 < S::NPH) {
    cstore<S, P>(x, s, t);
    cmid<S, P, P + 1>();
    cload<S, P + 1>(x, s, t);
    cinv<S, MODE, P + 1>(x, s, tw, pc, t);
  }
}

template <class S, int MODE, typename W = typename S::W>
__device__ __forceinline__ W pointwise1(W x, W y, const PrimeConst<W>& pc) {
  if constexpr (MODE == kSmall) {
    return montmul(x, y, pc.q, pc.qinv);
  } else if constexpr (MODE == kL4) {
    return csub(montmul(x, y, pc.q, pc.qinv), pc.q2);
  } else {
    return montmul(csub(x, pc.q), csub(y, pc.q), pc.q, pc.qinv);
  }
}

// One unit per cluster at a time.  SEQ: one operand in registers at a time
// (a's transform parked in its buffer at this thread's own words); the
// inverse's top exchange then separates every CTA's last access to the
// buffers from the next unit's remote stores, so units need no barrier of
// their own.  Both operands at once (SEQ false): the inverse runs on a's
// buffer, whose last remote reads the next unit's remote stores would race,
// so each unit ends with a cluster barrier.
template <class S, int MODE, bool SEQ>
__global__ void __launch_bounds__(kClusterThreads, 1) k_ntt_cluster2(NttBatchArgs<typename S::W> args) {
  using W = typename S::W;
  static_assert(S::T % kClusterThreads == 0 && S::N == (S::T / kClusterThreads) << kClusterLocalLog,
                "one CTA per 8192 coefficients");
  static_assert(S::PAD > 0, "padded local layout");
  static_assert(!cta_local<S, S::NPH - 1>(), "the top layout spans the cluster");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr uint32_t L = (1u << kClusterLocalLog) + ((1u << kClusterLocalLog) >> S::PAD);
  W* sa = reinterpret_cast<W*>(smem_raw);
  W* sb = sa + L;
  const uint32_t t = cluster_rank() * kClusterThreads + threadIdx.x;
  constexpr int TOP = S::NPH - 1;
  const TwPair<W>* twf = reinterpret_cast<const TwPair<W>*>(args.tw_fwd);
  const TwPair<W>* twi = reinterpret_cast<const TwPair<W>*>(args.tw_inv);
  const W* g0 = nullptr;
  for (uint64_t u = cluster_id(); u < args.units; u += cluster_count()) {
    const uint32_t j = (uint32_t)(u % args.k);
    const uint32_t pj = table_index(args, j);
    const PrimeConst<W> pc = args.pc[(size_t)pj * args.pc_stride + args.pc_off];
    const TwPair<W>* tf = twf + (size_t)pj * args.tw_stride;
    const TwPair<W>* ti = twi + (size_t)pj * args.tw_stride;
    const W* a = args.a + (size_t)u * S::N;
    const W* b = args.b + (size_t)u * S::N;
    W xa[S::R];
    (void)g0;
    if constexpr (SEQ) {
      sfor<0, S::R>([&](auto ec) {
        constexpr int e = decltype(ec)::value;
        xa[e] = a[elem_index<S, TOP>(e, t)];
      });
      cfwd<S, MODE, TOP, false>(xa, xa, sa, sa, tf, pc, t);
      __syncthreads();  // this CTA's layout-0 reads of sa are done
      sfor<0, S::R>([&](auto ec) {
        constexpr int e = decltype(ec)::value;
        sa[e * kClusterThreads + threadIdx.x] = xa[e];
      });
      sfor<0, S::R>([&](auto ec) {
        constexpr int e = decltype(ec)::value;
        xa[e] = b[elem_index<S, TOP>(e, t)];
      });
      // the same table through an opaque copy of its address: b's transform
      // loads its twiddles again instead of keeping a's alive across the park
      const TwPair<W>* tf_b;
      asm volatile("mov.b64 %0, %1;" : "=l"(tf_b) : "l"(tf));
      cfwd<S, MODE, TOP, false>(xa, xa, sb, sb, tf_b, pc, t);
      sfor<0, S::R>([&](auto ec) {
        constexpr int e = decltype(ec)::value;
        xa[e] = pointwise1<S, MODE>(sa[e * kClusterThreads + threadIdx.x], xa[e], pc);
      });
      cinv<S, MODE, 0>(xa, sb, ti, pc, t);
    } else {
      W xb[S::R];
      sfor<0, S::R>([&](auto ec) {
        constexpr int e = decltype(ec)::value;
        const uint32_t i = elem_index<S, TOP>(e, t);
        xa[e] = a[i];
        xb[e] = b[i];
      });
      cfwd<S, MODE, TOP, true>(xa, xb, sa, sb, tf, pc, t);
      sfor<0, S::R>([&](auto ec) {
        constexpr int e = decltype(ec)::value;
        xa[e] = pointwise1<S, MODE>(xa[e], xb[e], pc);
      });
      cinv<S, MODE, 0>(xa, sa, ti, pc, t);
    }
    W* c = args.c + (size_t)u * S::N;
    sfor<0, S::R>([&](auto ec) {
      constexpr int e = decltype(ec)::value;
      c[elem_index<S, TOP>(e, t)] = csub(xa[e], pc.q);
    });
    if constexpr (!SEQ) ClusterSync{}();
  }
  ClusterSync{}();  // no CTA leaves while another may still address its shared memory
}

template <typename W, int LOGN, int MODE, bool SEQ>
static KernelInfo cluster2_info() {
  using S = Shape<W, LOGN, 4, 4>;
  KernelInfo ki;
  ki.fn = (const void*)k_ntt_cluster2<S, MODE, SEQ>;
  ki.block = kClusterThreads;
  ki.smem = 2 * ((1 << kClusterLocalLog) + ((1 << kClusterLocalLog) >> 4)) * (int)sizeof(W);
  ki.team = S::T;
  ki.units_per_cta = 1;
  ki.cluster = S::T / kClusterThreads;
  ki.rb = 4;
  ki.mode = MODE;
  ki.regs = 65536 / kClusterThreads;
  ki.pad = 4;
  ki.seq = SEQ ? 1 : 0;
  return ki;
}

template <typename W, int LOGN, int MODE>
static KernelInfo cluster_info() {
  using S = Shape<W, LOGN, 4>;
  constexpr bool DB = sizeof(W) == 4;  // four 32 KB buffers; 64-bit words keep two
  KernelInfo ki;
  ki.fn = (const void*)k_ntt_cluster<S, MODE, DB>;
  ki.block = kClusterThreads;
  ki.smem = (DB ? 4 : 2) * (1 << kClusterLocalLog) * (int)sizeof(W);
  ki.team = S::T;
  ki.units_per_cta = 1;
  ki.cluster = S::T / kClusterThreads;
  ki.rb = 4;
  ki.mode = MODE;
  ki.regs = 65536 / kClusterThreads;
  return ki;
}

// the second form (CTA-local exchanges, padded layout); seq: one operand at a time
bool lookup_ntt_cluster2(uint32_t elem, int logn, int mode, bool seq, KernelInfo* ki) {
#define PM_C2(W, L, M)                                                           \
  if (logn == L && mode == M) {                                                  \
    *ki = seq ? cluster2_info<W, L, M, true>() : cluster2_info<W, L, M, false>(); \
    return true;                                                                 \
  }
  if (elem == 8) {
    PM_C2(uint64_t, 14, 1)
    PM_C2(uint64_t, 15, 1)
    PM_C2(uint64_t, 16, 1)
  } else {
    PM_C2(uint32_t, 14, 0)
    PM_C2(uint32_t, 15, 0)
    PM_C2(uint32_t, 16, 0)
    PM_C2(uint32_t, 14, 1)
    PM_C2(uint32_t, 15, 1)
    PM_C2(uint32_t, 16, 1)
  }
#undef PM_C2
  return false;
}

bool lookup_ntt_cluster(uint32_t elem, int logn, int mode, KernelInfo* ki) {
#define PM_C(W, L, M)                      \
  if (logn == L && mode == M) {            \
    *ki = cluster_info<W, L, M>();         \
    return true;                           \
  }
  if (elem == 8) {
    PM_C(uint64_t, 14, 1)
    PM_C(uint64_t, 15, 1)
    PM_C(uint64_t, 16, 1)
    PM_C(uint64_t, 14, 2)
    PM_C(uint64_t, 15, 2)
    PM_C(uint64_t, 16, 2)
  } else {
    PM_C(uint32_t, 14, 0)
    PM_C(uint32_t, 15, 0)
    PM_C(uint32_t, 16, 0)
    PM_C(uint32_t, 14, 1)
    PM_C(uint32_t, 15, 1)
    PM_C(uint32_t, 16, 1)
    PM_C(uint32_t, 14, 2)
    PM_C(uint32_t, 15, 2)
  }
#undef PM_C
  return false;
}

}  // namespace pm

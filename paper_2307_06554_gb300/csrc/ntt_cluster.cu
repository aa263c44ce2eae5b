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
    const uint32_t pj = args.pmap ? args.pmap[j] : j;
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

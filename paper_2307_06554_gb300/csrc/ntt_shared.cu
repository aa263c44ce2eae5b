// Shared-operand products on the NTT path: c_i = a * b_i for one a.
//
// The transform of a is computed once per prime (k_ntt_prep) and kept in
// the register layout a team holds after its forward transform (word e of
// team thread t at t * R + e), so that the product kernel (k_ntt_shared)
// reads it back with R consecutive words per thread.  Each product then
// costs one forward transform (b), the pointwise product with the stored
// a^, and one inverse transform: two transforms instead of three.  Same
// arithmetic, tables, reduction modes and staging as k_ntt_batch.
#include <cuda_runtime.h>

#include "kernels.h"
#include "ntt.cuh"
#include "polymul_types.h"

namespace pm {

template <class S, int MODE>
__device__ __forceinline__ void pointwise(typename S::W (&x)[S::R], const typename S::W* __restrict__ ah,
                                          const PrimeConst<typename S::W>& pc) {
  using W = typename S::W;
  static_assert((S::R * sizeof(W)) % 16 == 0, "vector loads of a^");
  W y[S::R];
  const uint4* src = reinterpret_cast<const uint4*>(ah);
  sfor<0, (int)(S::R * sizeof(W) / 16)>([&](auto ic) {
    constexpr int i = decltype(ic)::value;
    *reinterpret_cast<uint4*>(&y[i * 16 / sizeof(W)]) = __ldg(src + i);
  });
  sfor<0, S::R>([&](auto ec) {
    constexpr int e = decltype(ec)::value;
    if constexpr (MODE == kSmall) {
      x[e] = montmul(x[e], y[e], pc.q, pc.qinv);
    } else if constexpr (MODE == kL4) {
      x[e] = csub(montmul(x[e], y[e], pc.q, pc.qinv), pc.q2);
    } else {
      x[e] = montmul(csub(x[e], pc.q), csub(y[e], pc.q), pc.q, pc.qinv);
    }
  });
}

// one CTA per prime: a_j through the forward transform, stored in the
// register layout
template <class S, int MODE>
__global__ void __launch_bounds__(S::T) k_ntt_prep(NttSharedArgs<typename S::W> args) {
  using W = typename S::W;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  W* s = reinterpret_cast<W*>(smem_raw);
  constexpr int TOP = S::NPH - 1;
  const uint32_t j = blockIdx.x, t = threadIdx.x;
  if (j >= args.units) return;
  const W* a = args.a + (size_t)j * S::N;
  W x[S::R];
  sfor<0, S::R>([&](auto ec) {
    constexpr int e = decltype(ec)::value;
    x[e] = a[elem_index<S, TOP>(e, t)];
  });
  const TwPair<W>* twf = reinterpret_cast<const TwPair<W>*>(args.tw_fwd) + (size_t)j * args.tw_stride;
  fwd_from1<S, MODE, TOP>(x, s, twf, args.pc[j], t, BlockSync{});
  W* out = args.c + ((size_t)j * S::T + t) * S::R;
  sfor<0, S::R>([&](auto ec) {
    constexpr int e = decltype(ec)::value;
    out[e] = x[e];
  });
}

// one product (unit) per CTA at a time, persistent over the batch; b's row
// arrives by bulk copy, the next one is issued after the last exchange
template <class S, int MODE>
__global__ void __launch_bounds__(S::T, 65536 / (S::T * 128)) k_ntt_shared(NttSharedArgs<typename S::W> args) {
  using W = typename S::W;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ unsigned long long s_next;
  W* s = reinterpret_cast<W*>(smem_raw);
  constexpr int TOP = S::NPH - 1;
  constexpr uint32_t ROW = S::N * (uint32_t)sizeof(W);
  const uint32_t t = threadIdx.x;
  const uint64_t units = args.units;
  griddep_launch_dependents();
  if (t == 0) mbar_init(&mbar, 1);
  fence_mbar_init();
  griddep_wait();  // the counter, operands and results of the previous kernel
  auto issue = [&](unsigned long long u) {  // thread 0 only
    fence_proxy_async();
    mbar_arrive_expect_tx(&mbar, ROW);
    bulk_g2s(s, args.b + (size_t)u * S::N, ROW, &mbar);
  };
  if (t == 0) {
    s_next = atomicAdd(args.ctr, 1ull);
    if (s_next < units) issue(s_next);
  }
  __syncthreads();
  unsigned long long cur = s_next;
  uint32_t parity = 0;
  while (cur < units) {
    const bool ok = mbar_wait(&mbar, parity);
    if (__syncthreads_or(!ok)) {
      if (t == 0) atomicExch(args.err, 1);
      mbar_wait(&mbar, parity);  // let the copy in flight land before leaving
      return;
    }
    parity ^= 1u;
    const uint32_t j = (uint32_t)(cur % args.k);
    const PrimeConst<W> pc = args.pc[j];
    W x[S::R];
    sfor<0, S::R>([&](auto ec) {
      constexpr int e = decltype(ec)::value;
      x[e] = s[elem_index<S, TOP>(e, t)];
    });
    const TwPair<W>* twf = reinterpret_cast<const TwPair<W>*>(args.tw_fwd) + (size_t)j * args.tw_stride;
    const TwPair<W>* twi = reinterpret_cast<const TwPair<W>*>(args.tw_inv) + (size_t)j * args.tw_stride;
    fwd_from1<S, MODE, TOP>(x, s, twf, pc, t, BlockSync{});
    pointwise<S, MODE>(x, args.a + ((size_t)j * S::T + t) * S::R, pc);
    auto hook = [&]() {  // after a barrier: every thread is done with s
      if (t == 0) {
        s_next = atomicAdd(args.ctr, 1ull);
        if (s_next < units) issue(s_next);
      }
    };
    inv_from<S, MODE, 0>(x, s, twi, pc, t, BlockSync{}, hook);
    W* c = args.c + (size_t)cur * S::N;
    sfor<0, S::R>([&](auto ec) {
      constexpr int e = decltype(ec)::value;
      c[elem_index<S, TOP>(e, t)] = csub(x[e], pc.q);
    });
    __syncthreads();
    cur = s_next;
  }
  if (t == 0) {
    __threadfence();
    if (atomicAdd(args.ctr + 1, 1ull) == (unsigned long long)gridDim.x - 1) {
      atomicExch(args.ctr, 0ull);
      atomicExch(args.ctr + 1, 0ull);
    }
  }
}

template <int LOGN, int MODE>
static void shared_info(KernelInfo* prep, KernelInfo* main) {
  using S = Shape<uint32_t, LOGN, 4>;
  static_assert(S::NPH >= 2, "at least one exchange (the hook point)");
  prep->fn = (const void*)k_ntt_prep<S, MODE>;
  main->fn = (const void*)k_ntt_shared<S, MODE>;
  prep->block = main->block = S::T;
  prep->smem = main->smem = S::N * 4;
  prep->team = main->team = S::T;
  prep->units_per_cta = main->units_per_cta = 1;
  prep->rb = main->rb = 4;
  prep->mode = main->mode = MODE;
  prep->regs = main->regs = 128;
}

bool lookup_ntt_shared(int logn, int mode, KernelInfo* prep, KernelInfo* main) {
#define PM_S(L, M)                   \
  if (logn == L && mode == M) {      \
    shared_info<L, M>(prep, main);   \
    return true;                     \
  }
  PM_S(10, 0) PM_S(11, 0) PM_S(12, 0) PM_S(13, 0)
  PM_S(10, 1) PM_S(11, 1) PM_S(12, 1) PM_S(13, 1)
  PM_S(10, 2) PM_S(11, 2) PM_S(12, 2) PM_S(13, 2)
#undef PM_S
  return false;
}

}  // namespace pm

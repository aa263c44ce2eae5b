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

// this thread's R words of a^ (R consecutive words, vector loads)
template <class S>
__device__ __forceinline__ void load_ahat(typename S::W (&y)[S::R], const typename S::W* __restrict__ ah) {
  using W = typename S::W;
  static_assert((S::R * sizeof(W)) % 16 == 0, "vector loads of a^");
  const uint4* src = reinterpret_cast<const uint4*>(ah);
  sfor<0, (int)(S::R * sizeof(W) / 16)>([&](auto ic) {
    constexpr int i = decltype(ic)::value;
    *reinterpret_cast<uint4*>(&y[i * 16 / sizeof(W)]) = __ldg(src + i);
  });
}

template <class S, int MODE>
__device__ __forceinline__ void pointwise(typename S::W (&x)[S::R], const typename S::W (&y)[S::R],
                                          const PrimeConst<typename S::W>& pc) {
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
  griddep_wait();               // a and the previous kernel's results
  // only now may the next kernel start: when it does, everything before this
  // one is complete
  griddep_launch_dependents();
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

// Two products of the same prime per CTA at a time (a pair: products p, p+1
// of prime j), persistent over the batch: both b rows arrive by bulk copy
// into the CTA's two buffers, go through the forward transform together
// (shared twiddles), meet the stored a^_j in the pointwise product, and go
// through the inverse transform together; the next pair's copies are issued
// after the last exchange.  Two operands per thread keep the same
// instruction-level parallelism as the plain batch kernel with a third less
// work per product.  args.units = pairs = ceil(batch / 2) * k; pair v is
// prime v mod k, products 2 (v / k) and 2 (v / k) + 1 (the second absent
// when the batch is odd: its slot copies and computes the first again and
// stores nothing).
template <class S, int MODE>
__global__ void __launch_bounds__(S::T, 65536 / (S::T * 128)) k_ntt_shared(NttSharedArgs<typename S::W> args) {
  using W = typename S::W;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ unsigned long long s_next;
  W* sx = reinterpret_cast<W*>(smem_raw);
  W* sy = sx + S::N;
  constexpr int TOP = S::NPH - 1;
  constexpr uint32_t ROW = S::N * (uint32_t)sizeof(W);
  const uint32_t t = threadIdx.x;
  const uint64_t pairs = args.units, k = args.k, batch = args.batch;
  if (t == 0) mbar_init(&mbar, 1);
  fence_mbar_init();
  griddep_wait();  // the counter, operands and results of the previous kernel
  griddep_launch_dependents();  // after the wait (see k_ntt_prep)
  auto rows = [&](unsigned long long v, uint64_t& r0, uint64_t& r1, bool& second) {
    const uint64_t j = v % k, p0 = 2 * (v / k);
    second = p0 + 1 < batch;
    r0 = p0 * k + j;
    r1 = (second ? p0 + 1 : p0) * k + j;
  };
  auto issue = [&](unsigned long long v) {  // thread 0 only
    uint64_t r0, r1;
    bool second;
    rows(v, r0, r1, second);
    fence_proxy_async();
    mbar_arrive_expect_tx(&mbar, 2 * ROW);
    bulk_g2s(sx, args.b + r0 * S::N, ROW, &mbar);
    bulk_g2s(sy, args.b + r1 * S::N, ROW, &mbar);
  };
  if (t == 0) {
    s_next = atomicAdd(args.ctr, 1ull);
    if (s_next < pairs) issue(s_next);
  }
  __syncthreads();
  unsigned long long cur = s_next;
  uint32_t parity = 0;
  while (cur < pairs) {
    const bool ok = mbar_wait(&mbar, parity);
    if (__syncthreads_or(!ok)) {
      if (t == 0) atomicExch(args.err, 1);
      mbar_wait(&mbar, parity);  // let the copies in flight land before leaving
      return;
    }
    parity ^= 1u;
    uint64_t r0, r1;
    bool second;
    rows(cur, r0, r1, second);
    const uint32_t j = (uint32_t)(cur % k);
    const PrimeConst<W> pc = args.pc[j];
    W x[S::R], y[S::R];
    sfor<0, S::R>([&](auto ec) {
      constexpr int e = decltype(ec)::value;
      const uint32_t i = elem_index<S, TOP>(e, t);
      x[e] = sx[i];
      y[e] = sy[i];
    });
    const TwPair<W>* twf = reinterpret_cast<const TwPair<W>*>(args.tw_fwd) + (size_t)j * args.tw_stride;
    const TwPair<W>* twi = reinterpret_cast<const TwPair<W>*>(args.tw_inv) + (size_t)j * args.tw_stride;
    W ah[S::R];  // loaded now, used after the forward transform: the loads hide behind it
    load_ahat<S>(ah, args.a + ((size_t)j * S::T + t) * S::R);
    fwd_from<S, MODE, TOP>(x, y, sx, sy, twf, pc, t, BlockSync{});
    pointwise<S, MODE>(x, ah, pc);
    pointwise<S, MODE>(y, ah, pc);
    auto hook = [&]() {  // after a barrier: every thread is done with sx and sy
      if (t == 0) {
        s_next = atomicAdd(args.ctr, 1ull);
        if (s_next < pairs) issue(s_next);
      }
    };
    inv_from2<S, MODE, 0>(x, y, sx, sy, twi, pc, t, BlockSync{}, hook);
    W* c0 = args.c + r0 * S::N;
    W* c1 = args.c + r1 * S::N;
    sfor<0, S::R>([&](auto ec) {
      constexpr int e = decltype(ec)::value;
      const uint32_t i = elem_index<S, TOP>(e, t);
      c0[i] = csub(x[e], pc.q);
      if (second) c1[i] = csub(y[e], pc.q);
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
  prep->smem = S::N * 4;
  main->smem = 2 * S::N * 4;
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

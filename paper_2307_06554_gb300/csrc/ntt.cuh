// Batched negacyclic NTT polynomial multiplication, one (product, prime)
// unit per team of threads.
//
// What it computes: c = a*b in Z_q[x]/(x^n+1) for prime q = 1 mod 2n
// (the "value representation" route of Sec. 2.1 (ii) of the paper, with the
// NTT the paper names as the O(n log n) transform; it requires the root of
// unity that Sec. 2.1 lists among NTT's restrictions).  The negacyclic twist
// by psi (a primitive 2n-th root) is merged into the twiddles:
//   forward  Cooley-Tukey, natural order in, bit-reversed out, table
//            W[k] = psi^brv(k);
//   pointwise Montgomery product (gives a^ b^ 2^-w);
//   inverse  Gentleman-Sande, bit-reversed in, natural out, table
//            V[k] = psi^-brv(k); the last stage also multiplies by
//            n^-1 * 2^w, which undoes the Montgomery factor and the 1/n.
//
// Register/shared-memory layout.  A thread holds R = 2^RB coefficients of
// each operand (RB = 5 for 32-bit words, 4 for 64-bit).  The log2(n) stage
// bits are cut into phases at multiples of RB: phase P owns bits
// [P*RB, min((P+1)*RB, log2 n)).  Inside a phase a thread's R values are
// whole butterfly groups (indices differing only in the phase's bits), so
// every stage of the phase runs in registers with no communication; between
// phases the team exchanges through shared memory, word j stored at
// j + (j >> RB) (one pad word per 2^RB), which makes every exchange pattern
// used here free of bank conflicts.  For n = 1024 and 32-bit words this is
// one exchange per transform with a team of one warp (32 lanes x 32 values).
// The top phase's layout puts consecutive lanes on consecutive coefficients,
// so global loads and stores are fully coalesced.
#pragma once
#include <cstdint>
#include <type_traits>
#include "arith.cuh"
#include "polymul_types.h"

namespace pm {

// Compile-time loop: calls f(std::integral_constant<int, i>) for i = B, B+S,
// ... while i != E.  Keeps every register-array index a constant.
template <int B, int E, int S = 1, class F>
__device__ __forceinline__ void sfor(F&& f) {
  if constexpr (B != E) {
    f(std::integral_constant<int, B>{});
    sfor<B + S, E, S>(f);
  }
}

template <typename W>
struct alignas(2 * sizeof(W)) TwPair {
  W w, wp;  // root power and its Shoup companion floor(w * 2^bits / q)
};

template <typename W>
__device__ __forceinline__ TwPair<W> ldtw(const TwPair<W>* p) {
  if constexpr (sizeof(W) == 4) {
    uint2 v = __ldg(reinterpret_cast<const uint2*>(p));
    return TwPair<W>{v.x, v.y};
  } else {
    ulonglong2 v = __ldg(reinterpret_cast<const ulonglong2*>(p));
    return TwPair<W>{v.x, v.y};
  }
}

// Operand traffic is streamed (read once, written once): keep it out of L1 so
// that the twiddle tables stay resident there.
__device__ __forceinline__ uint32_t ld_stream(const uint32_t* p) { return __ldcs(p); }
__device__ __forceinline__ uint64_t ld_stream(const uint64_t* p) {
  return (uint64_t)__ldcs(reinterpret_cast<const unsigned long long*>(p));
}
__device__ __forceinline__ void st_stream(uint32_t* p, uint32_t v) { __stcs(p, v); }
__device__ __forceinline__ void st_stream(uint64_t* p, uint64_t v) {
  __stcs(reinterpret_cast<unsigned long long*>(p), (unsigned long long)v);
}

// Bulk prefetch of `bytes` (multiple of 16, 16-byte aligned) into L2.
__device__ __forceinline__ void prefetch_l2(const void* p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

template <typename W, int LOGN>
struct Shape {
  static constexpr int RB = sizeof(W) == 4 ? 5 : 4;
  static constexpr int RLOG = LOGN < RB ? LOGN : RB;
  static constexpr int R = 1 << RLOG;           // values per thread per operand
  static constexpr int N = 1 << LOGN;
  static constexpr int T = N / R;               // threads per unit (team size)
  static constexpr int NPH = (LOGN + RB - 1) / RB;
  static constexpr int SLICE = N + (N >> RB);   // padded words per operand in smem
  // keep both operands' exchange buffers when they fit comfortably
  static constexpr bool DUAL = 2 * SLICE * (int)sizeof(W) <= 100 * 1024;
  static constexpr int SMEM_WORDS = DUAL ? 2 * SLICE : SLICE;
};

template <typename W, int LOGN, int P>
struct PhaseBits {
  using S = Shape<W, LOGN>;
  static constexpr int LO = P * S::RB;
  static constexpr int HI = (P + 1) * S::RB < LOGN ? (P + 1) * S::RB : LOGN;
  static constexpr int B = HI - LO;
  static constexpr int GS = 1 << B;   // butterfly group size
  static constexpr int NG = S::R / GS;  // groups per thread
};

// coefficient index held in register slot e by team thread t during phase P
template <typename W, int LOGN, int P>
__device__ __forceinline__ uint32_t elem_index(int e, uint32_t t) {
  using PB = PhaseBits<W, LOGN, P>;
  using S = Shape<W, LOGN>;
  const uint32_t u = (uint32_t)e & (PB::GS - 1);
  const uint32_t g = t + (uint32_t)S::T * (uint32_t)(e >> PB::B);
  return (g & ((1u << PB::LO) - 1)) | (u << PB::LO) | ((g >> PB::LO) << PB::HI);
}

template <int RB>
__device__ __forceinline__ uint32_t spos(uint32_t j) { return j + (j >> RB); }

// ---------------------------------------------------------------- butterflies
// Reduction modes (chosen per plan from the largest modulus, see
// ntt_mode()):
//   kQ31   q < 2^(bits-1): every value kept in [0, 2q);
//   kL4    q < 2^(bits-2): Harvey's bounds, [0, 4q) forward, [0, 2q) inverse;
//   kSmall q < 2^(bits-1-log2 n) and (1+2 log2 n)^2 q < 2^bits: no
//          conditional subtraction anywhere.  Forward values grow by at most
//          2q per stage ((1+2s)q after s stages); inverse values at most
//          double per stage (2^(s+1) q after s stages), the subtraction
//          offset of stage s being that bound.
enum { kQ31 = 0, kL4 = 1, kSmall = 2 };

template <typename W, int MODE>
__device__ __forceinline__ void ct_bfly(W& x, W& y, const TwPair<W>& w, const PrimeConst<W>& pc) {
  if constexpr (MODE == kSmall) {
    W t = shoup(y, w.w, w.wp, pc.q);
    y = x - t + pc.q2;
    x = x + t;
  } else if constexpr (MODE == kL4) {
    W xr = csub(x, pc.q2);
    W t = shoup(y, w.w, w.wp, pc.q);
    x = xr + t;
    y = xr - t + pc.q2;
  } else {
    W xr = csub(x, pc.q);
    W t = csub(shoup(y, w.w, w.wp, pc.q), pc.q);
    x = xr + t;
    y = xr - t + pc.q;
  }
}

// inverse butterfly of stage h (h = number of inverse stages already done)
template <typename W, int MODE, int H>
__device__ __forceinline__ void gs_bfly(W& x, W& y, W w, W wp, const PrimeConst<W>& pc) {
  if constexpr (MODE == kSmall) {
    W d = x - y + (pc.q << (H + 1));
    x = x + y;
    y = shoup(d, w, wp, pc.q);
  } else if constexpr (MODE == kL4) {
    W s = x + y;
    W d = x - y + pc.q2;
    x = csub(s, pc.q2);
    y = shoup(d, w, wp, pc.q);
  } else {
    W xr = csub(x, pc.q), yr = csub(y, pc.q);
    W d = xr - yr + pc.q;
    x = xr + yr;
    y = shoup(d, w, wp, pc.q);
  }
}

// last inverse stage: both outputs also multiplied by n^-1 * 2^bits
template <typename W, int MODE, int H>
__device__ __forceinline__ void gs_last(W& x, W& y, const PrimeConst<W>& pc) {
  W s, d;
  if constexpr (MODE == kSmall) {
    s = x + y;
    d = x - y + (pc.q << (H + 1));
  } else if constexpr (MODE == kL4) {
    s = x + y;
    d = x - y + pc.q2;
  } else {
    W xr = csub(x, pc.q), yr = csub(y, pc.q);
    s = xr + yr;
    d = xr - yr + pc.q;
  }
  x = shoup(s, pc.scale, pc.scale_p, pc.q);
  y = shoup(d, pc.scale_w, pc.scale_wp, pc.q);
}

// Two consecutive twiddle pairs in one 16-byte load (32-bit words), else
// one pair per load.  `p` is 16-byte aligned whenever a run has >= 2 pairs.
template <typename W>
__device__ __forceinline__ void ldtw2(const TwPair<W>* p, TwPair<W>& w0, TwPair<W>& w1) {
  if constexpr (sizeof(W) == 4) {
    uint4 v = __ldg(reinterpret_cast<const uint4*>(p));
    w0 = TwPair<W>{v.x, v.y};
    w1 = TwPair<W>{v.z, v.w};
  } else {
    w0 = ldtw(p);
    w1 = ldtw(p + 1);
  }
}

// ---------------------------------------------------------------- phases
// forward Cooley-Tukey stages of phase P on two operands sharing twiddles
template <typename W, int LOGN, int MODE, int P>
__device__ __forceinline__ void fwd_phase2(W (&xa)[Shape<W, LOGN>::R], W (&xb)[Shape<W, LOGN>::R],
                                           const TwPair<W>* __restrict__ tw, const PrimeConst<W>& pc,
                                           uint32_t t) {
  using PB = PhaseBits<W, LOGN, P>;
  using S = Shape<W, LOGN>;
  sfor<PB::HI - 1, PB::LO - 1, -1>([&](auto hc) {
    constexpr int h = decltype(hc)::value;
    constexpr int hb = h - PB::LO;
    constexpr int NUP = PB::GS >> (hb + 1);  // distinct twiddles per group
    sfor<0, PB::NG>([&](auto glc) {
      constexpr int gl = decltype(glc)::value;
      const uint32_t g = t + (uint32_t)S::T * gl;
      const uint32_t tb = (1u << (LOGN - 1 - h)) + ((g >> PB::LO) << (PB::HI - 1 - h));
      auto apply = [&](auto upc, const TwPair<W>& w) {
        constexpr int up = decltype(upc)::value;
        sfor<0, (1 << hb)>([&](auto lwc) {
          constexpr int lw = decltype(lwc)::value;
          constexpr int u0 = gl * PB::GS + ((up << (hb + 1)) | lw);
          constexpr int u1 = u0 + (1 << hb);
          ct_bfly<W, MODE>(xa[u0], xa[u1], w, pc);
          ct_bfly<W, MODE>(xb[u0], xb[u1], w, pc);
        });
      };
      if constexpr (NUP == 1) {
        apply(std::integral_constant<int, 0>{}, ldtw(tw + tb));
      } else {
        sfor<0, NUP, 2>([&](auto upc) {
          constexpr int up = decltype(upc)::value;
          TwPair<W> w0, w1;
          ldtw2(tw + tb + up, w0, w1);
          apply(std::integral_constant<int, up>{}, w0);
          apply(std::integral_constant<int, up + 1>{}, w1);
        });
      }
    });
  });
}

// inverse Gentleman-Sande stages of phase P
template <typename W, int LOGN, int MODE, int P>
__device__ __forceinline__ void inv_phase(W (&x)[Shape<W, LOGN>::R], const TwPair<W>* __restrict__ tw,
                                          const PrimeConst<W>& pc, uint32_t t) {
  using PB = PhaseBits<W, LOGN, P>;
  using S = Shape<W, LOGN>;
  sfor<PB::LO, PB::HI>([&](auto hc) {
    constexpr int h = decltype(hc)::value;
    constexpr int hb = h - PB::LO;
    constexpr int NUP = PB::GS >> (hb + 1);
    sfor<0, PB::NG>([&](auto glc) {
      constexpr int gl = decltype(glc)::value;
      const uint32_t g = t + (uint32_t)S::T * gl;
      const uint32_t tb = (1u << (LOGN - 1 - h)) + ((g >> PB::LO) << (PB::HI - 1 - h));
      auto apply = [&](auto upc, const TwPair<W>& w) {
        constexpr int up = decltype(upc)::value;
        sfor<0, (1 << hb)>([&](auto lwc) {
          constexpr int lw = decltype(lwc)::value;
          constexpr int u0 = gl * PB::GS + ((up << (hb + 1)) | lw);
          gs_bfly<W, MODE, h>(x[u0], x[u0 + (1 << hb)], w.w, w.wp, pc);
        });
      };
      if constexpr (h == LOGN - 1) {
        sfor<0, NUP>([&](auto upc) {
          constexpr int up = decltype(upc)::value;
          sfor<0, (1 << hb)>([&](auto lwc) {
            constexpr int lw = decltype(lwc)::value;
            constexpr int u0 = gl * PB::GS + ((up << (hb + 1)) | lw);
            gs_last<W, MODE, h>(x[u0], x[u0 + (1 << hb)], pc);
          });
        });
      } else if constexpr (NUP == 1) {
        apply(std::integral_constant<int, 0>{}, ldtw(tw + tb));
      } else {
        sfor<0, NUP, 2>([&](auto upc) {
          constexpr int up = decltype(upc)::value;
          TwPair<W> w0, w1;
          ldtw2(tw + tb + up, w0, w1);
          apply(std::integral_constant<int, up>{}, w0);
          apply(std::integral_constant<int, up + 1>{}, w1);
        });
      }
    });
  });
}

template <typename W, int LOGN, int P>
__device__ __forceinline__ void store_layout(const W (&x)[Shape<W, LOGN>::R], W* s, uint32_t t) {
  using S = Shape<W, LOGN>;
  sfor<0, S::R>([&](auto ec) {
    constexpr int e = decltype(ec)::value;
    s[spos<S::RB>(elem_index<W, LOGN, P>(e, t))] = x[e];
  });
}

template <typename W, int LOGN, int P>
__device__ __forceinline__ void load_layout(W (&x)[Shape<W, LOGN>::R], const W* s, uint32_t t) {
  using S = Shape<W, LOGN>;
  sfor<0, S::R>([&](auto ec) {
    constexpr int e = decltype(ec)::value;
    x[e] = s[spos<S::RB>(elem_index<W, LOGN, P>(e, t))];
  });
}

template <typename W, int LOGN, int MODE, int P, class Sync>
__device__ __forceinline__ void fwd_from(W (&xa)[Shape<W, LOGN>::R], W (&xb)[Shape<W, LOGN>::R], W* sa,
                                         W* sb, const TwPair<W>* __restrict__ tw, const PrimeConst<W>& pc,
                                         uint32_t t, Sync sync) {
  using S = Shape<W, LOGN>;
  fwd_phase2<W, LOGN, MODE, P>(xa, xb, tw, pc, t);
  if constexpr (P > 0) {
    if constexpr (S::DUAL) {
      sync();
      store_layout<W, LOGN, P>(xa, sa, t);
      store_layout<W, LOGN, P>(xb, sb, t);
      sync();
      load_layout<W, LOGN, P - 1>(xa, sa, t);
      load_layout<W, LOGN, P - 1>(xb, sb, t);
    } else {
      sync();
      store_layout<W, LOGN, P>(xa, sa, t);
      sync();
      load_layout<W, LOGN, P - 1>(xa, sa, t);
      sync();
      store_layout<W, LOGN, P>(xb, sa, t);
      sync();
      load_layout<W, LOGN, P - 1>(xb, sa, t);
    }
    fwd_from<W, LOGN, MODE, P - 1>(xa, xb, sa, sb, tw, pc, t, sync);
  }
}

template <typename W, int LOGN, int MODE, int P, class Sync>
__device__ __forceinline__ void inv_from(W (&x)[Shape<W, LOGN>::R], W* s, const TwPair<W>* __restrict__ tw,
                                         const PrimeConst<W>& pc, uint32_t t, Sync sync) {
  using S = Shape<W, LOGN>;
  inv_phase<W, LOGN, MODE, P>(x, tw, pc, t);
  if constexpr (P + 1 < S::NPH) {
    sync();
    store_layout<W, LOGN, P>(x, s, t);
    sync();
    load_layout<W, LOGN, P + 1>(x, s, t);
    inv_from<W, LOGN, MODE, P + 1>(x, s, tw, pc, t, sync);
  }
}

// One unit: c = a*b mod (x^n+1, q) for one prime.  Every thread of the team
// calls it (inactive threads with act = false compute on zeros and store
// nothing, so that team barriers stay uniform).
template <typename W, int LOGN, int MODE, class Sync>
__device__ __forceinline__ void polymul_unit(const W* __restrict__ a, const W* __restrict__ b, W* __restrict__ c,
                                             const TwPair<W>* __restrict__ twf,
                                             const TwPair<W>* __restrict__ twi, const PrimeConst<W>& pc,
                                             W* sa, W* sb, uint32_t t, bool act, Sync sync) {
  using S = Shape<W, LOGN>;
  constexpr int TOP = S::NPH - 1;
  W xa[S::R], xb[S::R];
  sfor<0, S::R>([&](auto ec) {
    constexpr int e = decltype(ec)::value;
    const uint32_t j = elem_index<W, LOGN, TOP>(e, t);
    xa[e] = act ? ld_stream(a + j) : W(0);
    xb[e] = act ? ld_stream(b + j) : W(0);
  });
  fwd_from<W, LOGN, MODE, TOP>(xa, xb, sa, sb, twf, pc, t, sync);
  // pointwise product in the bit-reversed domain (same layout for both)
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
  inv_from<W, LOGN, MODE, 0>(xa, sa, twi, pc, t, sync);
  if (act) {
    sfor<0, S::R>([&](auto ec) {
      constexpr int e = decltype(ec)::value;
      st_stream(c + elem_index<W, LOGN, TOP>(e, t), csub(xa[e], pc.q));
    });
  }
}

struct WarpSync {
  __device__ __forceinline__ void operator()() const { __syncwarp(); }
};
struct BlockSync {
  __device__ __forceinline__ void operator()() const { __syncthreads(); }
};

// Homogeneous batch: `units` = batch * k units, unit u uses prime u % k and
// the operand rows a + u*n, b + u*n, c + u*n.  Persistent grid (sized to the
// resident capacity); teams take units from a device counter, so the work
// balances across SMs whatever the unit count.  The counter pair
// ctr = {next, finished} is zero between launches: the last team to finish
// resets it.  Launches that share a counter must therefore not overlap.
template <typename W, int LOGN, int MODE, int WARPS>
__global__ void __launch_bounds__(Shape<W, LOGN>::T <= 32 ? 32 * WARPS : Shape<W, LOGN>::T)
    k_ntt_batch(NttBatchArgs<W> args) {
  using S = Shape<W, LOGN>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  W* smem = reinterpret_cast<W*>(smem_raw);
  const TwPair<W>* twf = reinterpret_cast<const TwPair<W>*>(args.tw_fwd);
  const TwPair<W>* twi = reinterpret_cast<const TwPair<W>*>(args.tw_inv);
  const uint64_t units = args.units;
  const uint32_t k = args.k;
  unsigned long long* ctr = args.ctr;
  if constexpr (S::T <= 32) {
    constexpr int TPW = 32 / S::T;  // teams per warp
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t team = lane / S::T, t = lane % S::T;
    W* sa = smem + (size_t)(warp * TPW + team) * S::SMEM_WORDS;
    W* sb = S::DUAL ? sa + S::SLICE : sa;
    // one ticket ahead: while a unit computes, its successor's rows are
    // prefetched into L2
    auto grab = [&]() {
      unsigned long long v = 0;
      if (lane == 0) v = atomicAdd(ctr, (unsigned long long)TPW);
      return __shfl_sync(0xffffffffu, v, 0);
    };
    unsigned long long cur = grab();
    while (cur < units) {
      const unsigned long long nxt = grab();
      if (lane == 0 && nxt < units) {
        const uint32_t cnt = (uint32_t)(units - nxt < (unsigned long long)TPW ? units - nxt : TPW);
        prefetch_l2(args.a + (size_t)nxt * S::N, cnt * S::N * (uint32_t)sizeof(W));
        prefetch_l2(args.b + (size_t)nxt * S::N, cnt * S::N * (uint32_t)sizeof(W));
      }
      const uint64_t u = cur + team;
      const bool act = u < units;
      const uint32_t j = act ? (uint32_t)(u % k) : 0u;
      const size_t off = act ? (size_t)u * S::N : 0;
      const PrimeConst<W> pc = args.pc[j];
      polymul_unit<W, LOGN, MODE>(args.a + off, args.b + off, args.c + off, twf + (size_t)j * S::N,
                                  twi + (size_t)j * S::N, pc, sa, sb, t, act, WarpSync{});
      cur = nxt;
    }
    if (lane == 0) {
      __threadfence();
      const unsigned long long teams = (unsigned long long)gridDim.x * WARPS;
      if (atomicAdd(ctr + 1, 1ull) == teams - 1) {
        atomicExch(ctr, 0ull);
        atomicExch(ctr + 1, 0ull);
      }
    }
  } else {
    __shared__ unsigned long long s_base;
    W* sa = smem;
    W* sb = S::DUAL ? smem + S::SLICE : smem;
    if (threadIdx.x == 0) s_base = atomicAdd(ctr, 1ull);
    __syncthreads();
    unsigned long long cur = s_base;
    while (cur < units) {
      __syncthreads();  // everyone has read s_base
      if (threadIdx.x == 0) {
        const unsigned long long nxt = atomicAdd(ctr, 1ull);
        s_base = nxt;
        if (nxt < units) {
          prefetch_l2(args.a + (size_t)nxt * S::N, S::N * (uint32_t)sizeof(W));
          prefetch_l2(args.b + (size_t)nxt * S::N, S::N * (uint32_t)sizeof(W));
        }
      }
      const uint32_t j = (uint32_t)(cur % k);
      const size_t off = (size_t)cur * S::N;
      const PrimeConst<W> pc = args.pc[j];
      polymul_unit<W, LOGN, MODE>(args.a + off, args.b + off, args.c + off, twf + (size_t)j * S::N,
                                  twi + (size_t)j * S::N, pc, sa, sb, threadIdx.x, true, BlockSync{});
      __syncthreads();  // s_base written before the unit's barriers; read it now
      cur = s_base;
    }
    if (threadIdx.x == 0) {
      __threadfence();
      if (atomicAdd(ctr + 1, 1ull) == (unsigned long long)gridDim.x - 1) {
        atomicExch(ctr, 0ull);
        atomicExch(ctr + 1, 0ull);
      }
    }
  }
}

}  // namespace pm

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
// each operand (RB is a template parameter, chosen per word size and n).  The log2(n) stage
// bits are cut into phases at multiples of RB: phase P owns bits
// [P*RB, min((P+1)*RB, log2 n)).  Inside a phase a thread's R values are
// whole butterfly groups (indices differing only in the phase's bits), so
// every stage of the phase runs in registers with no communication; between
// phases the team exchanges through shared memory, word j stored at an
// XOR-swizzled position (spos) that makes every exchange pattern used here
// free of bank conflicts.  For n = 1024 and 32-bit words this is
// one exchange per transform with a team of one warp (32 lanes x 32 values).
// The top phase's layout puts consecutive lanes on consecutive coefficients,
// so global loads and stores are fully coalesced.
#pragma once
#include <cstdint>
#include <type_traits>
#include "arith.cuh"
#include "async.cuh"
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

// PAD_ selects the exchange layout: 0 = the XOR swizzle spos (a bijection
// of [0, n)), s > 0 = word j at j + (j >> s), one padding word after every
// 2^s.  The padded position is additive over any split of j's bits, so a
// thread's exchange addresses are one base register per layout plus
// immediate offsets; the swizzle needs one register (or one XOR) per
// coefficient.
template <typename W_, int LOGN_, int RB_, int PAD_ = 0>
struct Shape {
  using W = W_;
  static constexpr int LOGN = LOGN_;
  static constexpr int RB = RB_;                // stage bits per phase
  static constexpr int PAD = PAD_;
  static constexpr int RLOG = LOGN < RB ? LOGN : RB;
  static constexpr int R = 1 << RLOG;           // values per thread per operand
  static constexpr int N = 1 << LOGN;
  static constexpr int T = N / R;               // threads per unit (team size)
  static constexpr int NPH = (LOGN + RB - 1) / RB;
  static constexpr int ALIGN_WORDS = 16 / (int)sizeof(W);
  // words per operand buffer
  static constexpr int SLICE =
      PAD == 0 ? N : (N + (N >> PAD) + ALIGN_WORDS - 1) / ALIGN_WORDS * ALIGN_WORDS;
  // two buffers per team (a and b): they receive the staged operands, then
  // serve the exchanges.  Teams that share a warp are offset by T words
  // (rounded up to 16 bytes, the bulk-copy alignment) so that their lanes
  // fall in different banks.
  static constexpr int TEAM_PAD = T < 32 ? (T + ALIGN_WORDS - 1) / ALIGN_WORDS * ALIGN_WORDS : 0;
  static constexpr int SMEM_WORDS = 2 * SLICE + TEAM_PAD;
  static_assert((SMEM_WORDS * sizeof(W)) % 16 == 0, "team buffers must stay 16-byte aligned");
};

template <class S, int P>
struct PhaseBits {
  static constexpr int LO = P * S::RB;
  static constexpr int HI = (P + 1) * S::RB < S::LOGN ? (P + 1) * S::RB : S::LOGN;
  static constexpr int B = HI - LO;
  static constexpr int GS = 1 << B;   // butterfly group size
  static constexpr int NG = S::R / GS;  // groups per thread
};

// coefficient index held in register slot e by team thread t during phase P
template <class S, int P>
__device__ __forceinline__ uint32_t elem_index(int e, uint32_t t) {
  using PB = PhaseBits<S, P>;
  const uint32_t u = (uint32_t)e & (PB::GS - 1);
  const uint32_t g = t + (uint32_t)S::T * (uint32_t)(e >> PB::B);
  return (g & ((1u << PB::LO) - 1)) | (u << PB::LO) | ((g >> PB::LO) << PB::HI);
}

// Shared-memory position of coefficient j during an exchange: an XOR swizzle
// of the low five bits by bits 1..5 and RB..RB+4 (a bijection inside every
// 32-word block).  Checked exhaustively for RB in {3,4,5}, n = 2^4..2^16 and
// 4- and 8-byte words: every warp access of every exchange is free of bank
// conflicts.
template <int RB>
__device__ __forceinline__ uint32_t spos(uint32_t j) { return j ^ ((j >> 1) & 31u) ^ ((j >> RB) & 31u); }

// exchange position of coefficient j in a team buffer of shape S
template <class S>
__device__ __forceinline__ uint32_t xpos(uint32_t j) {
  if constexpr (S::PAD > 0)
    return j + (j >> S::PAD);
  else
    return spos<S::RB>(j);
}

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
// forward Cooley-Tukey stages of phase P on one operand, or on two operands
// sharing twiddles (TWO)
template <class S, int MODE, int P, bool TWO, typename W = typename S::W>
__device__ __forceinline__ void fwd_phase(W (&xa)[S::R], W (&xb)[S::R], const TwPair<W>* __restrict__ tw,
                                          const PrimeConst<W>& pc, uint32_t t) {
  using PB = PhaseBits<S, P>;
  constexpr int LOGN = S::LOGN;
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
          if constexpr (TWO) ct_bfly<W, MODE>(xb[u0], xb[u1], w, pc);
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

template <class S, int MODE, int P, typename W = typename S::W>
__device__ __forceinline__ void fwd_phase2(W (&xa)[S::R], W (&xb)[S::R], const TwPair<W>* __restrict__ tw,
                                           const PrimeConst<W>& pc, uint32_t t) {
  fwd_phase<S, MODE, P, true>(xa, xb, tw, pc, t);
}

// inverse Gentleman-Sande stages of phase P on one operand, or on two
// operands sharing twiddles (TWO)
template <class S, int MODE, int P, bool TWO, typename W = typename S::W>
__device__ __forceinline__ void inv_phase_n(W (&x)[S::R], W (&y)[S::R], const TwPair<W>* __restrict__ tw,
                                            const PrimeConst<W>& pc, uint32_t t) {
  using PB = PhaseBits<S, P>;
  constexpr int LOGN = S::LOGN;
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
          if constexpr (TWO) gs_bfly<W, MODE, h>(y[u0], y[u0 + (1 << hb)], w.w, w.wp, pc);
        });
      };
      if constexpr (h == LOGN - 1) {
        sfor<0, NUP>([&](auto upc) {
          constexpr int up = decltype(upc)::value;
          sfor<0, (1 << hb)>([&](auto lwc) {
            constexpr int lw = decltype(lwc)::value;
            constexpr int u0 = gl * PB::GS + ((up << (hb + 1)) | lw);
            gs_last<W, MODE, h>(x[u0], x[u0 + (1 << hb)], pc);
            if constexpr (TWO) gs_last<W, MODE, h>(y[u0], y[u0 + (1 << hb)], pc);
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

template <class S, int MODE, int P, typename W = typename S::W>
__device__ __forceinline__ void inv_phase(W (&x)[S::R], const TwPair<W>* __restrict__ tw,
                                          const PrimeConst<W>& pc, uint32_t t) {
  inv_phase_n<S, MODE, P, false>(x, x, tw, pc, t);
}

// elem_index(e, t) is the bitwise OR of elem_index(e, 0) and elem_index(0, t)
// (disjoint bits: t < T), so with the padded layout a position is a
// per-thread base plus a compile-time offset.
template <class S, int P, typename W = typename S::W>
__device__ __forceinline__ void store_layout(const W (&x)[S::R], W* s, uint32_t t) {
  if constexpr (S::PAD > 0) {
    W* sb = s + xpos<S>(elem_index<S, P>(0, t));
    sfor<0, S::R>([&](auto ec) {
      constexpr int e = decltype(ec)::value;
      sb[xpos<S>(elem_index<S, P>(e, 0))] = x[e];
    });
  } else {
    sfor<0, S::R>([&](auto ec) {
      constexpr int e = decltype(ec)::value;
      s[xpos<S>(elem_index<S, P>(e, t))] = x[e];
    });
  }
}

template <class S, int P, typename W = typename S::W>
__device__ __forceinline__ void load_layout(W (&x)[S::R], const W* s, uint32_t t) {
  if constexpr (S::PAD > 0) {
    const W* sb = s + xpos<S>(elem_index<S, P>(0, t));
    sfor<0, S::R>([&](auto ec) {
      constexpr int e = decltype(ec)::value;
      x[e] = sb[xpos<S>(elem_index<S, P>(e, 0))];
    });
  } else {
    sfor<0, S::R>([&](auto ec) {
      constexpr int e = decltype(ec)::value;
      x[e] = s[xpos<S>(elem_index<S, P>(e, t))];
    });
  }
}

// Exchange buffers may also be spread over the CTAs of a cluster: any type
// with store(j, v) / load(j) and kCluster = true (see ntt_cluster.cu).
template <class S, int P, class CB, typename W = typename S::W, bool = CB::kCluster>
__device__ __forceinline__ void store_layout(const W (&x)[S::R], const CB& s, uint32_t t) {
  sfor<0, S::R>([&](auto ec) {
    constexpr int e = decltype(ec)::value;
    s.store(elem_index<S, P>(e, t), x[e]);
  });
}

template <class S, int P, class CB, typename W = typename S::W, bool = CB::kCluster>
__device__ __forceinline__ void load_layout(W (&x)[S::R], const CB& s, uint32_t t) {
  sfor<0, S::R>([&](auto ec) {
    constexpr int e = decltype(ec)::value;
    x[e] = s.load(elem_index<S, P>(e, t));
  });
}

// ---------------------------------------------------------------- exchanges
// Barriers of an exchange (stores in layout P, then loads in layout Q).
//  * Before the stores: a thread stores exactly at the positions it loaded
//    in layout P, so nothing is overwritten that another thread has still to
//    read -- except in the first exchange of a transform, whose buffer held
//    the staged operand at unswizzled positions.  Only that one needs the
//    team barrier first.
//  * Between stores and loads: when every warp holds the same coefficients
//    in layouts P and Q (the team-thread bits that select the warp land on
//    the same coefficient bits in both), each warp reads only what it wrote,
//    and a warp barrier orders the exchange.  Otherwise the team barrier.
// Exchange buffers spread over a cluster keep the cluster barrier at both
// points.
template <class B, class = void>
struct is_cluster_buf : std::false_type {};
template <class B>
struct is_cluster_buf<B, std::void_t<decltype(B::kCluster)>> : std::bool_constant<B::kCluster> {};

// coefficient-index bit that team-thread bit b occupies in layout P
template <class S, int P>
constexpr int tbit_pos(int b) {
  return b < PhaseBits<S, P>::LO ? b : b - PhaseBits<S, P>::LO + PhaseBits<S, P>::HI;
}

template <class S, int P, int Q>
constexpr bool warp_local() {
  for (int b = 5; (1 << b) < S::T; ++b)
    if (tbit_pos<S, P>(b) != tbit_pos<S, Q>(b)) return false;
  return true;
}

template <bool FIRST, class B, class Sync>
__device__ __forceinline__ void xsync_pre(Sync sync) {
  if constexpr (FIRST || is_cluster_buf<B>::value) sync();
}

template <class S, int P, int Q, class B, class Sync>
__device__ __forceinline__ void xsync_mid(Sync sync) {
  if constexpr (!is_cluster_buf<B>::value && warp_local<S, P, Q>())
    __syncwarp();
  else
    sync();
}

template <class S, int MODE, int P, class Sync, class B, typename W = typename S::W>
__device__ __forceinline__ void fwd_from(W (&xa)[S::R], W (&xb)[S::R], B sa, B sb,
                                         const TwPair<W>* __restrict__ tw, const PrimeConst<W>& pc,
                                         uint32_t t, Sync sync) {
  fwd_phase2<S, MODE, P>(xa, xb, tw, pc, t);
  if constexpr (P > 0) {
    xsync_pre<P == S::NPH - 1, B>(sync);
    store_layout<S, P>(xa, sa, t);
    store_layout<S, P>(xb, sb, t);
    xsync_mid<S, P, P - 1, B>(sync);
    load_layout<S, P - 1>(xa, sa, t);
    load_layout<S, P - 1>(xb, sb, t);
    fwd_from<S, MODE, P - 1>(xa, xb, sa, sb, tw, pc, t, sync);
  }
}

// one operand through the forward transform (phases P .. 0)
template <class S, int MODE, int P, class Sync, class B, typename W = typename S::W>
__device__ __forceinline__ void fwd_from1(W (&x)[S::R], B s, const TwPair<W>* __restrict__ tw,
                                          const PrimeConst<W>& pc, uint32_t t, Sync sync) {
  fwd_phase<S, MODE, P, false>(x, x, tw, pc, t);
  if constexpr (P > 0) {
    xsync_pre<P == S::NPH - 1, B>(sync);
    store_layout<S, P>(x, s, t);
    xsync_mid<S, P, P - 1, B>(sync);
    load_layout<S, P - 1>(x, s, t);
    fwd_from1<S, MODE, P - 1>(x, s, tw, pc, t, sync);
  }
}

// `hook` runs once the team has finished reading the exchange buffers for
// the last time in this unit (after the last exchange, behind a team
// barrier), so that the buffers can receive the next unit's operands.  The
// buffer was last read in layout 0 by the forward transform (same positions
// as the first stores here).
template <class S, int MODE, int P, class Sync, class Hook, class B, typename W = typename S::W>
__device__ __forceinline__ void inv_from(W (&x)[S::R], B s, const TwPair<W>* __restrict__ tw,
                                         const PrimeConst<W>& pc, uint32_t t, Sync sync, Hook&& hook) {
  inv_phase<S, MODE, P>(x, tw, pc, t);
  if constexpr (P + 1 < S::NPH) {
    xsync_pre<false, B>(sync);
    store_layout<S, P>(x, s, t);
    xsync_mid<S, P, P + 1, B>(sync);
    load_layout<S, P + 1>(x, s, t);
    if constexpr (P + 2 == S::NPH) {
      sync();
      hook();
    }
    inv_from<S, MODE, P + 1>(x, s, tw, pc, t, sync, hook);
  }
}

// two operands of the same prime through the inverse transform together
// (shared twiddle loads); `hook` as for inv_from, once both buffers are free
template <class S, int MODE, int P, class Sync, class Hook, class B, typename W = typename S::W>
__device__ __forceinline__ void inv_from2(W (&x)[S::R], W (&y)[S::R], B sx, B sy, const TwPair<W>* __restrict__ tw,
                                          const PrimeConst<W>& pc, uint32_t t, Sync sync, Hook&& hook) {
  inv_phase_n<S, MODE, P, true>(x, y, tw, pc, t);
  if constexpr (P + 1 < S::NPH) {
    xsync_pre<false, B>(sync);
    store_layout<S, P>(x, sx, t);
    store_layout<S, P>(y, sy, t);
    xsync_mid<S, P, P + 1, B>(sync);
    load_layout<S, P + 1>(x, sx, t);
    load_layout<S, P + 1>(y, sy, t);
    if constexpr (P + 2 == S::NPH) {
      sync();
      hook();
    }
    inv_from2<S, MODE, P + 1>(x, y, sx, sy, tw, pc, t, sync, hook);
  }
}

// One unit: c = a*b mod (x^n+1, q) for one prime, operands already staged
// (unswizzled, contiguous) in sa and sb.  Every thread of the team calls it;
// inactive threads (act = false) compute on stale data and store nothing, so
// that team barriers stay uniform.  `hook` is called once sa/sb are free.
// The operands are read from ia and ib: the staged rows in sa and sb, or the
// rows themselves in global memory (host memory the device maps included),
// in the same coalesced order.
// Auxiliary-prime mode (AUX = true): the ring modulus qo has no 2n-th root
// of unity, so the product is formed over the integers instead.  Operands
// are lifted to their centred representatives (|x| <= qo/2), which the NTT
// prime p (> 2 n (qo/2)^2) holds as residues; the result mod p, centred,
// is the exact integer negacyclic product, reduced mod qo on the way out.
template <class S, int MODE, bool AUX, class Sync, class Hook, typename W = typename S::W>
__device__ __forceinline__ void polymul_unit(W* __restrict__ c, const TwPair<W>* __restrict__ twf,
                                             const TwPair<W>* __restrict__ twi, const PrimeConst<W>& pc,
                                             W* sa, W* sb, const W* ia, const W* ib, uint32_t t, bool act,
                                             Sync sync, Hook&& hook, W qo = 0) {
  constexpr int TOP = S::NPH - 1;
  W xa[S::R], xb[S::R];
  const W lift = pc.q - qo, half = qo >> 1;
  sfor<0, S::R>([&](auto ec) {
    constexpr int e = decltype(ec)::value;
    const uint32_t j = elem_index<S, TOP>(e, t);
    xa[e] = ia[j];
    xb[e] = ib[j];
    if constexpr (AUX) {
      xa[e] = xa[e] > half ? xa[e] + lift : xa[e];
      xb[e] = xb[e] > half ? xb[e] + lift : xb[e];
    }
  });
  if constexpr (S::NPH == 1) {
    sync();
    hook();
  }
  fwd_from<S, MODE, TOP>(xa, xb, sa, sb, twf, pc, t, sync);
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
  inv_from<S, MODE, 0>(xa, sa, twi, pc, t, sync, hook);
  if (act) {
    sfor<0, S::R>([&](auto ec) {
      constexpr int e = decltype(ec)::value;
      W y = csub(xa[e], pc.q);
      if constexpr (AUX) {
        // centre mod p, then reduce mod qo
        if (y > (pc.q >> 1)) {
          const W r = (pc.q - y) % qo;
          y = r ? qo - r : W(0);
        } else {
          y = y % qo;
        }
      }
      c[elem_index<S, TOP>(e, t)] = y;
    });
  }
}

// The same unit with one operand in registers at a time: a's forward
// transform, its result parked in a's staging buffer in a thread-private
// order (word e*T + t, conflict-free), then b's forward transform, the
// pointwise product against the parked values, and the inverse.  Half the
// live coefficient registers of polymul_unit, so twice the units fit on an
// SM at the same register budget; costs one store and one load per
// coefficient of a and separate twiddle loads for the two forward
// transforms.
template <class S, int MODE, bool AUX, class Sync, class Hook, typename W = typename S::W>
__device__ __forceinline__ void polymul_unit_seq(W* __restrict__ c, const TwPair<W>* __restrict__ twf,
                                                 const TwPair<W>* __restrict__ twi, const PrimeConst<W>& pc,
                                                 W* sa, W* sb, const W* ia, const W* ib, uint32_t t, bool act,
                                                 Sync sync, Hook&& hook, W qo = 0) {
  constexpr int TOP = S::NPH - 1;
  W x[S::R];
  const W lift = pc.q - qo, half = qo >> 1;
  auto load_top = [&](const W* s) {
    sfor<0, S::R>([&](auto ec) {
      constexpr int e = decltype(ec)::value;
      x[e] = s[elem_index<S, TOP>(e, t)];
      if constexpr (AUX) x[e] = x[e] > half ? x[e] + lift : x[e];
    });
  };
  load_top(ia);
  fwd_from1<S, MODE, TOP>(x, sa, twf, pc, t, sync);
  if constexpr (S::NPH > 1) sync();  // every exchange read of sa is done
  sfor<0, S::R>([&](auto ec) {
    constexpr int e = decltype(ec)::value;
    sa[e * S::T + t] = x[e];
  });
  load_top(ib);
  fwd_from1<S, MODE, TOP>(x, sb, twf, pc, t, sync);
  sfor<0, S::R>([&](auto ec) {
    constexpr int e = decltype(ec)::value;
    const W y = sa[e * S::T + t];
    if constexpr (MODE == kSmall) {
      x[e] = montmul(y, x[e], pc.q, pc.qinv);
    } else if constexpr (MODE == kL4) {
      x[e] = csub(montmul(y, x[e], pc.q, pc.qinv), pc.q2);
    } else {
      x[e] = montmul(csub(y, pc.q), csub(x[e], pc.q), pc.q, pc.qinv);
    }
  });
  if constexpr (S::NPH == 1) {
    sync();
    hook();
  }
  inv_from<S, MODE, 0>(x, sb, twi, pc, t, sync, hook);
  if (act) {
    sfor<0, S::R>([&](auto ec) {
      constexpr int e = decltype(ec)::value;
      W y = csub(x[e], pc.q);
      if constexpr (AUX) {
        if (y > (pc.q >> 1)) {
          const W r = (pc.q - y) % qo;
          y = r ? qo - r : W(0);
        } else {
          y = y % qo;
        }
      }
      c[elem_index<S, TOP>(e, t)] = y;
    });
  }
}

template <class S, int MODE, bool AUX, bool SEQ, class Sync, class Hook, typename W = typename S::W>
__device__ __forceinline__ void polymul_unit_any(W* __restrict__ c, const TwPair<W>* __restrict__ twf,
                                                 const TwPair<W>* __restrict__ twi, const PrimeConst<W>& pc,
                                                 W* sa, W* sb, const W* ia, const W* ib, uint32_t t, bool act,
                                                 Sync sync, Hook&& hook, W qo = 0) {
  if constexpr (SEQ)
    polymul_unit_seq<S, MODE, AUX>(c, twf, twi, pc, sa, sb, ia, ib, t, act, sync, hook, qo);
  else
    polymul_unit<S, MODE, AUX>(c, twf, twi, pc, sa, sb, ia, ib, t, act, sync, hook, qo);
}

struct WarpSync {
  __device__ __forceinline__ void operator()() const { __syncwarp(); }
};
struct BlockSync {
  __device__ __forceinline__ void operator()() const { __syncthreads(); }
};

// Homogeneous batch: `units` = batch * k units, unit u uses prime u % k and
// the operand rows a + u*n, b + u*n, c + u*n.
//
// Persistent grid (sized to the resident capacity).  Teams take units from a
// device counter, so the work balances across SMs whatever the unit count.
// Operands arrive by bulk asynchronous copy (one elected thread per warp or
// CTA issues two row copies per unit into the team's two shared buffers,
// completion tracked by an mbarrier); the next unit's copy is issued as soon
// as the current unit has finished its last exchange, so DRAM latency hides
// behind the last inverse phase.
//
// The counter pair ctr = {next, finished} is zero between launches: the last
// team to finish resets it, so launches that share a counter must not
// overlap.  A bounded wait that expires sets *err = 1 and the team leaves
// its loop through the finish protocol (the counter stays consistent).
template <class S, int WARPS>
constexpr int ntt_block() {
  return S::T <= 32 ? 32 * WARPS : S::T;
}

// REGS: register budget per thread (sets the resident-CTA floor the
// compiler must honour).
// AUX: auxiliary-prime mode (see polymul_unit); every unit then uses the
// single NTT prime pc[0] and the ring modulus outer_q[u % k].
// SEQ: one operand in registers at a time (polymul_unit_seq).
// DIRECT: no staging copies; each team reads its unit's rows of a and b
// with plain coalesced loads where they lie and writes c the same way.  For
// operands in page-locked host memory that the device maps: over a coherent
// host link the loads and stores of many resident teams keep the link busy
// in both directions at once, with no copy engine and no device buffer
// (Sec. 4, overlapping computation with I/O, taken to the word level).
// No bounded waits are made (nothing is asynchronous).
template <class S, int MODE, int WARPS, int REGS, bool AUX = false, bool SEQ = false, bool DIRECT = false>
__global__ void __launch_bounds__(ntt_block<S, WARPS>(), 65536 / (ntt_block<S, WARPS>() * REGS))
    k_ntt_batch(NttBatchArgs<typename S::W> args) {
  using W = typename S::W;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t mbar[WARPS];
  W* smem = reinterpret_cast<W*>(smem_raw);
  const TwPair<W>* twf = reinterpret_cast<const TwPair<W>*>(args.tw_fwd);
  const TwPair<W>* twi = reinterpret_cast<const TwPair<W>*>(args.tw_inv);
  const uint64_t units = args.units;
  const uint32_t k = args.k;
  unsigned long long* ctr = args.ctr;
  constexpr uint32_t ROW = S::N * (uint32_t)sizeof(W);
  // Ordering against the previous kernel on the stream (programmatic
  // dependent launch).  The wait blocks until that kernel has completed and
  // its writes are visible; only then does this grid let the next kernel
  // start (so that, when the next kernel starts, everything before this one
  // is complete).  With args.early the host has checked that the previous
  // kernel is one of this library's batch launches that writes no operand
  // of this launch and touches none of its results: every team then loads
  // and multiplies its first unit before the wait, and waits only before
  // its first use of the work counter.
  const bool early = args.early != 0;
  const uint32_t polls = args.wait_polls ? args.wait_polls : kWaitPolls;
  bool waited = false;
  auto order = [&]() {  // every thread of the CTA, at the same point
    if (!waited) {
      griddep_wait();
      griddep_launch_dependents();
      waited = true;
    }
  };
  if (!early) order();
  if constexpr (S::T <= 32) {
    constexpr int TPW = 32 / S::T;  // teams per warp
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t team = lane / S::T, t = lane % S::T;
    W* wbase = smem + (size_t)warp * TPW * S::SMEM_WORDS;
    W* sa = wbase + (size_t)team * S::SMEM_WORDS;
    W* sb = sa + S::SLICE;
    uint64_t* bar = &mbar[warp];
    if (lane == 0) mbar_init(bar, 1);
    fence_mbar_init();
    __syncwarp();
    const unsigned long long first_round = (unsigned long long)gridDim.x * WARPS * TPW;
    auto grab = [&]() {  // every lane of the warp
      order();
      unsigned long long v = 0;
      if (lane == 0) v = first_round + atomicAdd(ctr, (unsigned long long)TPW);
      return __shfl_sync(0xffffffffu, v, 0);
    };
    auto issue = [&](unsigned long long base) {  // lane 0 only
      const uint32_t cnt = (uint32_t)(units - base < (unsigned long long)TPW ? units - base : TPW);
      fence_proxy_async();
      mbar_arrive_expect_tx(bar, 2 * cnt * ROW + args.tx_pad);
      for (uint32_t m = 0; m < cnt; ++m) {
        W* da = wbase + (size_t)m * S::SMEM_WORDS;
        bulk_g2s(da, args.a + (size_t)(base + m) * S::N, ROW, bar);
        bulk_g2s(da + S::SLICE, args.b + (size_t)(base + m) * S::N, ROW, bar);
      }
    };
    uint32_t parity = 0;
    // first units by position (no atomic on the critical path at start-up),
    // later ones from the counter, offset by the units handed out that way
    unsigned long long cur = ((unsigned long long)blockIdx.x * WARPS + warp) * TPW;
    if (!DIRECT && lane == 0 && cur < units) issue(cur);
    while (cur < units) {
      if constexpr (!DIRECT) {
        const bool ok = mbar_wait(bar, parity, polls);
        if (__any_sync(0xffffffffu, !ok)) {
          // record the failure, let the copy in flight land, and leave
          // through the finish protocol so that the work counter is reset as
          // usual
          if (lane == 0) atomicExch_system(args.err, 1);
          mbar_wait(bar, parity, polls);
          break;
        }
        parity ^= 1u;
      }
      const uint64_t u = cur + team;
      const bool act = u < units;
      const uint32_t j = act ? (uint32_t)(u % k) : 0u;
      const uint32_t pj = AUX ? 0u : table_index(args, j);
      const PrimeConst<W> pc = args.pc[(size_t)pj * args.pc_stride + args.pc_off];
      const W qo = AUX ? args.outer_q[j] : W(0);
      unsigned long long nxt = units;
      auto hook = [&]() {
        nxt = grab();
        if (!DIRECT && lane == 0 && nxt < units) issue(nxt);
      };
      // an inactive team (past the last unit) reads row 0 and stores nothing
      const size_t row = act ? (size_t)u * S::N : 0;
      polymul_unit_any<S, MODE, AUX, SEQ>(args.c + row, twf + (size_t)pj * args.tw_stride,
                                          twi + (size_t)pj * args.tw_stride, pc, sa, sb,
                                          DIRECT ? args.a + row : sa, DIRECT ? args.b + row : sb, t, act,
                                          WarpSync{}, hook, qo);
      cur = nxt;
    }
    order();
    // no fence: the next launch that uses the counter is ordered after this
    // kernel's completion, and every grab above returned before its team
    // got here
    if (lane == 0) {
      const unsigned long long teams = (unsigned long long)gridDim.x * WARPS;
      if (atomicAdd(ctr + 1, 1ull) == teams - 1) {
        atomicExch(ctr, 0ull);
        atomicExch(ctr + 1, 0ull);
      }
    }
  } else {
    __shared__ unsigned long long s_next;
    W* sa = smem;
    W* sb = smem + S::SLICE;
    uint64_t* bar = &mbar[0];
    if (threadIdx.x == 0) mbar_init(bar, 1);
    fence_mbar_init();
    // element offset of unit u's row (a row table, or u n)
    auto row_off = [&](unsigned long long u) -> size_t { return args.rows ? args.rows[u].offset : (size_t)u * S::N; };
    auto issue = [&](unsigned long long u) {  // thread 0 only
      fence_proxy_async();
      mbar_arrive_expect_tx(bar, 2 * ROW + args.tx_pad);
      const size_t off = row_off(u);
      bulk_g2s(sa, args.a + off, ROW, bar);
      bulk_g2s(sb, args.b + off, ROW, bar);
    };
    // first unit by position, later ones from the counter (see above)
    const unsigned long long first_round = gridDim.x;
    if (threadIdx.x == 0) {
      s_next = blockIdx.x;
      if (!DIRECT && s_next < units) issue(s_next);
    }
    __syncthreads();
    unsigned long long cur = s_next;
    uint32_t parity = 0;
    while (cur < units) {
      if constexpr (!DIRECT) {
        const bool ok = mbar_wait(bar, parity, polls);
        if (__syncthreads_or(!ok)) {  // as in the warp-team path
          if (threadIdx.x == 0) atomicExch_system(args.err, 1);
          mbar_wait(bar, parity, polls);
          break;
        }
        parity ^= 1u;
      }
      const uint32_t j = (uint32_t)(cur % k);
      const uint32_t pj = AUX ? 0u : args.rows ? args.rows[cur].prime : table_index(args, j);
      const PrimeConst<W> pc = args.pc[(size_t)pj * args.pc_stride + args.pc_off];
      const W qo = AUX ? args.outer_q[j] : W(0);
      auto hook = [&]() {  // every thread, after a barrier: all are done with sa/sb
        order();
        if (threadIdx.x == 0) {
          s_next = first_round + atomicAdd(ctr, 1ull);
          if (!DIRECT && s_next < units) issue(s_next);
        }
      };
      const size_t row = row_off(cur);
      polymul_unit_any<S, MODE, AUX, SEQ>(args.c + row, twf + (size_t)pj * args.tw_stride,
                                          twi + (size_t)pj * args.tw_stride, pc, sa, sb,
                                          DIRECT ? args.a + row : sa, DIRECT ? args.b + row : sb, threadIdx.x,
                                          true, BlockSync{}, hook, qo);
      __syncthreads();
      cur = s_next;
    }
    order();
    if (threadIdx.x == 0) {
      if (atomicAdd(ctr + 1, 1ull) == (unsigned long long)gridDim.x - 1) {
        atomicExch(ctr, 0ull);
        atomicExch(ctr + 1, 0ull);
      }
    }
  }
}

}  // namespace pm

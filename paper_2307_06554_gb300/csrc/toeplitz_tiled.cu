// Path (b) at every degree 2^6 .. 2^14: the matrix form of toeplitz.cu with
// the summation dimension in chunks and the outputs in groups.
//
// What it computes: c = a * T(b) in Z_q[x]/(x^n+1) (or x^n - 1), the row
// vector of a times the negacyclic (cyclic) Toeplitz matrix of b (Sec. 2.2),
// for many independent (a, b) pairs, with balanced w-bit digits of the
// centred coefficients (Sec. 2.4) recombined mod q in the epilogue
// (Algorithm 1, ConvertMatrix).  The algebra is that of toeplitz.cu
// (Sec. 2.5 division into 8-coefficient blocks):
//   c_j = sum_k A[u][k] B[v][k],  j = 8u + v,  k = 8d' + r,  D = n/8 - 1,
//   A[u][k] = a~_{8u + k - 8D},   B[v][k] = b~_{8(D - d') + v - r},
// a~, b~ the antiperiodic (periodic) extensions.
//
// Sec. 2.6 (high degrees): the product is cut into pieces that fit the
// matrix unit.  A unit of work is one (product, prime, output group) of
// blocks of 1024 outputs (128 rows of A each; for n < 1024 one block whose
// rows past n/8 compute outputs that are discarded): either BPG
// consecutive A slices (one chain per slice and digit of a), or, when b has
// no more digits than a, one A slice against S copies of b shifted by 1024
// coefficients in the B operand (template parameter S; the same A yields S
// blocks), accumulated in tensor memory over the K chunks
// [KC c, KC (c + 1)).  For each chunk the CTA builds in shared memory
//   * the window of a~'s digits that the chunk's rows read: row u of slice
//     bl starts 8 (128 bl + u) elements into it, so A is read through a
//     descriptor with a 16-byte row stride, never materialised, and
//   * the chunk's KC/8 K-blocks of B in the canonical K-major layout,
// one thread issues the MMA chains, and the CTA waits for them before it
// rebuilds the buffers.  Two CTAs share an SM (at most 256 tensor-memory
// columns and about 110 KB of shared memory each), so that one builds while
// the other's MMAs run.
//
// Exactness: every digit has magnitude <= 2^(w-1) <= 128 (exact in bf16) and
// n 2^(2w-2) <= 2^24 (the host chooses w so), so every fp32 partial sum over
// the whole of K is an exact integer.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "kernels.h"
#include "polymul_types.h"
#include "tcgen05.cuh"
#include "toeplitz_common.cuh"
#include "toeplitz_tiled.h"
#include "toeplitz_tiled.cuh"

namespace pm {

namespace {
constexpr int kTiledThreads = 128;
constexpr int kTiledSmemCap = 110 * 1024;  // two CTAs per SM
constexpr int kTiledTmemCap = 256;         // tensor-memory columns per CTA
}  // namespace


// DRAIN: each K chunk's accumulators are drained into 64-bit integer sums in
// registers after the chunk (and restart at zero), so only a chunk's partial
// sums must stay exact in fp32: kc * 2^(2w-2) <= 2^24, which 8-bit digits
// meet at kc = 1024 whatever n.  The running sums are reduced mod q after
// every chunk: a chunk adds at most LA LB 2^24 q < 2^59 in magnitude (at
// most 4 x 4 digit pairs), below the 2^60 bias.  BD: the A slices per unit
// of work of a drained kernel (its registers hold BD x S rows of sums; the
// host passes bpg == BD), 1 otherwise.
template <int LA, int LB, int S, bool DRAIN, int BD>
__global__ void __launch_bounds__(kTiledThreads, 2) k_toeplitz_tiled(TensorTiledArgs args) {
  using TS = TTShape<LB, S>;
  extern __shared__ __align__(128) unsigned char sm[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t s_tmem;
  __shared__ unsigned long long s_next;
  __shared__ int s_domain;  // a single-digit A-side coefficient did not fit its digit
  const int tid = threadIdx.x, warp = tid >> 5;
  const uint32_t n = 1u << args.logn, D = n / 8 - 1;
  const uint32_t kc = args.kc, nch = n / kc, bpg = args.bpg, ngrp = args.ngrp, awin = args.a_win;
  const int wb = (int)args.wb;
  const uint32_t wrap = args.wrap;
  const uint64_t units = args.units;
  uint16_t* Xw = reinterpret_cast<uint16_t*>(sm);  // [LA][awin] digits of a~ over the chunk's window
  unsigned char* Bt = sm + args.bt_off;             // [kc/8][BT_PITCH] the chunk of B
  constexpr uint32_t IDESC = idesc_bf16(128, TS::NB);

  if (warp == 0) {
    tmem_alloc(&s_tmem, args.tmem_cols);
    tmem_relinquish();
  }
  if (tid == 0) {
    mbar_init(&mbar, 1);
    s_domain = 0;
  }
  fence_mbar_init();
  // padded rows of B (8-row groups past the S x LB digit rows) stay zero
  // for the whole launch
  if (TS::NG > S * LB) {
    for (uint32_t ch = tid; ch < (kc / 8) * TS::NG * 8; ch += kTiledThreads) {
      const uint32_t dp = ch / (TS::NG * 8), g = (ch / 8) % TS::NG, v = ch % 8;
      if (g >= (uint32_t)(S * LB)) *reinterpret_cast<uint4*>(Bt + dp * TS::BT_PITCH + g * 128 + 16 * v) = make_uint4(0, 0, 0, 0);
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;

  if (tid == 0) s_next = atomicAdd(args.ctr, 1ull);
  __syncthreads();
  unsigned long long cur = s_next;
  uint32_t parity = 0;
  bool failed = false;
  // DRAIN: this thread's row, per A slice and shift and output, recombined
  // over the chunks drained so far
  int64_t dacc[BD * S][8];
  while (cur < units) {
    __syncthreads();  // every thread has read s_next
    if (tid == 0) s_next = atomicAdd(args.ctr, 1ull);
    const uint64_t row = cur / ngrp;
    const uint32_t grp = (uint32_t)(cur % ngrp);
    uint64_t off;
    uint32_t j;
    if (args.rows) {
      const RaggedUnit u = args.rows[row];
      off = u.offset;
      j = u.prime;
    } else {
      off = row * n;
      j = (uint32_t)(row % args.k);
    }
    const uint32_t q = args.tp[j].q;
    const uint32_t* a = args.a + off;
    const uint32_t* b = args.b + off;
    const uint32_t b0 = grp * bpg * S;  // the unit's first 1024-output block
    if constexpr (DRAIN) {
#pragma unroll
      for (int g = 0; g < BD * S; ++g)
#pragma unroll
        for (int v = 0; v < 8; ++v) dacc[g][v] = 0;
    }

    for (uint32_t ch = 0; ch < nch; ++ch) {
      // ---- ConvertPoly (a): digits of a~_{base + e}, e < awin ----
      // base and every group of 8 are multiples of 8, so a group lies wholly
      // in [0, n) (a itself), in [-n, 0) (the extension: a_{i+n}, sign per
      // `wrap`) or outside both (zero: rows past n/8 when n < 1024)
      const int32_t base = (int32_t)(1024 * b0) - (int32_t)n + 8 + (int32_t)(kc * ch);
      for (uint32_t gi = tid; gi < awin / 8; gi += kTiledThreads) {
        const int32_t i0 = base + 8 * (int32_t)gi;
        uint4 p[LA];
        uint32_t flip = 0;
        if (i0 >= (int32_t)n || i0 < -(int32_t)n) {
#pragma unroll
          for (int s = 0; s < LA; ++s) p[s] = make_uint4(0, 0, 0, 0);
        } else {
          flip = i0 < 0 ? wrap : 0u;
          const bool fits = digits8<LA>(a + (i0 < 0 ? i0 + (int32_t)n : i0), q, wb, p);
          if (!fits) s_domain = 1;
        }
#pragma unroll
        for (int s = 0; s < LA; ++s)
          *reinterpret_cast<uint4*>(Xw + (size_t)s * awin + 8 * gi) =
              make_uint4(p[s].x ^ flip, p[s].y ^ flip, p[s].z ^ flip, p[s].w ^ flip);
      }
      // ---- ConvertPoly (b): the chunk's K-blocks d' = kc/8 ch + dl of B ----
      // For shift sh, K-block d' is b~'s group G = D - d' + 128 sh after group
      // G - 1, b~ extended over [-n, 2n) (groups outside [0, n/8) are b's
      // groups n/8 away, negated for x^n + 1).  Shift sh gives, from the same
      // A, the outputs 1024 sh further on (a~ b~ is periodic in the
      // summation index); one 8-row group per digit of b.
      const int32_t ng = (int32_t)(n / 8);
      for (uint32_t dl = tid; dl < kc / 8; dl += kTiledThreads) {
        const int32_t g0 = (int32_t)(D - (kc / 8 * ch + dl));
#pragma unroll
        for (int sh = 0; sh < S; ++sh) {
          const int32_t G = g0 + 128 * sh, H = G - 1;
          const uint32_t gg = (uint32_t)(G >= ng ? G - ng : G);
          const uint32_t hh = (uint32_t)(H < 0 ? H + ng : H >= ng ? H - ng : H);
          const uint32_t fg = G >= ng ? wrap : 0u;
          const uint32_t fh = (H < 0 || H >= ng) ? wrap : 0u;
          uint4 pv[LB], ow[LB];
          digits8<LB>(b + 8 * hh, q, wb, pv);
          digits8<LB>(b + 8 * gg, q, wb, ow);
#pragma unroll
          for (int s2 = 0; s2 < LB; ++s2) {
            const uint32_t E[8] = {pv[s2].x ^ fh, pv[s2].y ^ fh, pv[s2].z ^ fh, pv[s2].w ^ fh,
                                   ow[s2].x ^ fg, ow[s2].y ^ fg, ow[s2].z ^ fg, ow[s2].w ^ fg};
            b_block_rows(E, Bt + dl * TS::BT_PITCH + (sh * LB + s2) * 128);
          }
        }
      }
      fence_proxy_async();
      tc_fence_before();
      __syncthreads();

      // ---- TPUMul: one thread issues the chains of this chunk ----
      if (tid == 0) {
        tc_fence_after();
        const uint32_t xa0 = smem_u32(Xw), bt0 = smem_u32(Bt);
        const uint64_t bd0 = smem_desc(bt0, TS::BT_PITCH, 128);
        constexpr uint64_t BSTEP = (2 * TS::BT_PITCH) >> 4;  // two K-blocks per MMA (K = 16)
        // one chain at a time (measured faster here than K steps outermost,
        // with two CTAs of an SM interleaving their chains)
#pragma unroll 1
        for (uint32_t bl = 0; bl < bpg; ++bl) {
#pragma unroll 1
          for (int s = 0; s < LA; ++s) {
            const uint32_t dcol = tmem + (bl * LA + s) * TS::NB;
            const uint64_t ad0 = smem_desc(xa0 + (uint32_t)(s * awin + 1024 * bl) * 2, 16, 128);
#pragma unroll 4
            for (uint32_t kk = 0; kk < kc / 16; ++kk)
              tc_mma_f16(dcol, ad0 + 2u * (uint64_t)kk, bd0 + BSTEP * (uint64_t)kk, IDESC,
                         ((!DRAIN && ch > 0) || kk > 0) ? 1u : 0u);
          }
        }
        tc_commit(&mbar);
      }
      // warp 0's other lanes wait for the issuing lane at the warp barrier
      if (warp == 0) __syncwarp();
      const bool ok = mbar_wait(&mbar, parity);
      if (__syncthreads_or(!ok)) {
        failed = true;
        break;
      }
      parity ^= 1u;
      tc_fence_after();
      if constexpr (DRAIN) {
        // the chunk's exact fp32 sums into the rows' integer recombination;
        // the next chunk's first MMA overwrites the accumulators only after
        // the barrier that precedes its issue
        // (digit pairs of one weight summed in 32-bit integers first)
        cfor<0, BD * S>([&](auto gc) {
          constexpr int g = decltype(gc)::value;
          int64_t (&acc)[8] = dacc[g];
          drain_pairs<LA, LB, S, g % S, 0, LA>(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)((g / S) * LA * TS::NB),
                                               args.tp[j].pw, acc);
#pragma unroll
          for (int v = 0; v < 8; ++v)
            acc[v] = barrett64((uint64_t)(acc[v] + (int64_t)args.tp[j].bias), q, args.tp[j].mu);
        });
      }
    }
    if (failed) break;

    // ---- ConvertMatrix: recombine digit pairs, reduce mod q, store ----
    uint32_t* c = args.c + off;
    const uint64_t mu = args.tp[j].mu, bias = args.tp[j].bias;
    if constexpr (DRAIN) {
#pragma unroll
      for (int g = 0; g < BD * S; ++g) {
        // accumulator group g = (slice bl, shift sh) holds block b0 + bl + sh
        // (one of the two is 0)
        const uint32_t j0 = 8 * (128 * (b0 + (uint32_t)(g / S) + (uint32_t)(g % S)) + (uint32_t)tid);
        if (j0 < n) {
          uint32_t out[8];
#pragma unroll
          for (int v = 0; v < 8; ++v) out[v] = (uint32_t)dacc[g][v];  // reduced after the last chunk
          *reinterpret_cast<uint4*>(c + j0) = make_uint4(out[0], out[1], out[2], out[3]);
          *reinterpret_cast<uint4*>(c + j0 + 4) = make_uint4(out[4], out[5], out[6], out[7]);
        }
      }
    }
#pragma unroll 1
    for (uint32_t bl = 0; bl < (DRAIN ? 0u : bpg); ++bl) {
#pragma unroll
      for (int sh = 0; sh < S; ++sh) {
        int64_t acc[8];
#pragma unroll
        for (int v = 0; v < 8; ++v) acc[v] = 0;
#pragma unroll
        for (int s = 0; s < LA; ++s) {
#pragma unroll
          for (int c16 = 0; c16 < TS::NB / 16; ++c16) {
            // only the 16-column loads that hold this shift's rows
            if (16 * c16 + 16 <= 8 * sh * LB || 16 * c16 >= 8 * (sh + 1) * LB) continue;
            uint32_t r[16];
            // warp-collective: every lane loads, only the stores below are predicated
            tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (bl * LA + s) * TS::NB + 16 * c16, r);
            tmem_wait_ld();
#pragma unroll
            for (int cc = 0; cc < 16; ++cc) {
              const int col = 16 * c16 + cc, g = col / 8, v = col % 8;
              if (g >= sh * LB && g < (sh + 1) * LB)
                acc[v] += (int64_t)__float2int_rn(__uint_as_float(r[cc])) * (int64_t)args.tp[j].pw[s + g - sh * LB];
            }
          }
        }
        const uint32_t j0 = 8 * (128 * (b0 + bl + sh) + (uint32_t)tid);
        if (j0 < n) {
          uint32_t out[8];
#pragma unroll
          for (int v = 0; v < 8; ++v) out[v] = barrett64((uint64_t)(acc[v] + (int64_t)bias), q, mu);
          *reinterpret_cast<uint4*>(c + j0) = make_uint4(out[0], out[1], out[2], out[3]);
          *reinterpret_cast<uint4*>(c + j0 + 4) = make_uint4(out[4], out[5], out[6], out[7]);
        }
      }
    }
    tc_fence_before();
    __syncthreads();
    cur = s_next;
  }
  if (failed) {
    if (tid == 0) atomicExch(args.err, 1);
    mbar_wait(&mbar, parity);  // let the MMAs in flight finish before freeing their memory
  }
  tc_fence_before();
  __syncthreads();
  if (tid == 0 && s_domain) atomicOr(args.err, 2);  // reported as POLYMUL_EDOMAIN
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, args.tmem_cols);
  }
  if (!failed && tid == 0) {
    __threadfence();
    if (atomicAdd(args.ctr + 1, 1ull) == (unsigned long long)gridDim.x - 1) {
      atomicExch(args.ctr, 0ull);
      atomicExch(args.ctr + 1, 0ull);
    }
  }
}

// the largest shift count instantiated for (la, lb): copies of b pay when
// b's digits are no more than a's (the B operand grows with the shifts)
static uint32_t max_shifts(int la, int lb) {
  if (la != lb) return 1;
  return la <= 2 ? 4 : la <= 4 ? 2 : 1;
}

bool toeplitz_tiled_config(int logn, int la, int lb, TiledCfg* cfg) {
  if (logn < 6 || logn > 14 || la < 1 || lb < 1 || la > 5 || lb > 5) return false;
  const uint32_t n = 1u << logn;
  auto nb_of = [&](uint32_t S) { return (8 * (uint32_t)lb * S + 15) / 16 * 16; };
  if ((uint32_t)la * nb_of(1) > (uint32_t)kTiledTmemCap) return false;
  const uint32_t rblk = n >= 1024 ? n / 1024 : 1;
  // shifted copies of b (one A slice), else consecutive A slices, as many as
  // the CTA's tensor memory holds
  uint32_t S = 1, bpg = 1;
  while (S * 2 <= rblk && S * 2 <= max_shifts(la, lb) && (uint32_t)la * nb_of(S * 2) <= (uint32_t)kTiledTmemCap) S *= 2;
  if (S == 1)
    while (bpg * 2 <= rblk && bpg * 2 * (uint32_t)la * nb_of(1) <= (uint32_t)kTiledTmemCap) bpg *= 2;
  const uint32_t nb = nb_of(S), pitch = nb / 8 * 128 + 16;
  uint32_t kc = n < 1024 ? n : 1024;
  for (;;) {
    const uint32_t a_win = 1024 * bpg + kc;
    const uint32_t bt_off = ((uint32_t)la * a_win * 2 + 127) / 128 * 128;
    const uint32_t smem = bt_off + kc / 8 * pitch;
    if (smem <= (uint32_t)kTiledSmemCap || kc <= 64) {
      if (smem > (uint32_t)kTiledSmemCap) return false;
      cfg->bpg = bpg;
      cfg->shifts = S;
      cfg->nb = nb;
      cfg->b_pitch = pitch;
      cfg->ngrp = rblk / (bpg * S);
      cfg->kc = kc;
      cfg->a_win = a_win;
      cfg->bt_off = bt_off;
      cfg->smem = (int)smem;
      uint32_t cols = 32;
      while (cols < bpg * (uint32_t)la * nb) cols *= 2;
      cfg->tmem_cols = cols;
      return true;
    }
    kc /= 2;
  }
}

template <int LA, int LB, int S, bool DRAIN = false, int BD = 1>
static void tiled_info(const TiledCfg& cfg, KernelInfo* ki) {
  ki->fn = (const void*)k_toeplitz_tiled<LA, LB, S, DRAIN, BD>;
  ki->drain = DRAIN ? 1 : 0;
  ki->block = kTiledThreads;
  ki->smem = cfg.smem;
  ki->team = kTiledThreads;
  ki->units_per_cta = 1;
  ki->tmem_cols = (int)cfg.tmem_cols;
  ki->tiled = 1;
}

bool lookup_toeplitz_tiled(int logn, int la, int lb, KernelInfo* ki) {
  TiledCfg cfg;
  if (!toeplitz_tiled_config(logn, la, lb, &cfg)) return false;
  const int S = (int)cfg.shifts;
#define PM_TT(A, B, SH)                    \
  if (la == A && lb == B && S == SH) {     \
    tiled_info<A, B, SH>(cfg, ki);         \
    return true;                           \
  }
  PM_TT(1, 1, 1) PM_TT(1, 1, 2) PM_TT(1, 1, 4)
  PM_TT(2, 2, 1) PM_TT(2, 2, 2) PM_TT(2, 2, 4)
  PM_TT(3, 3, 1) PM_TT(3, 3, 2)
  PM_TT(4, 4, 1) PM_TT(4, 4, 2)
  PM_TT(5, 5, 1)
  PM_TT(1, 2, 1) PM_TT(1, 3, 1) PM_TT(1, 4, 1) PM_TT(1, 5, 1)  // a single-digit operand on the A side (ternary b)
#undef PM_TT
  return false;
}

}  // namespace pm

namespace pm {

// Drained tiling: 8-bit digits (exact per chunk of at most 1024 K); with as
// many digits on both sides one A slice per unit of work against as many
// shifted copies of b as tensor memory holds, with a single-digit A side up
// to 4 A slices against one B (the undrained kernel's choice there too).

bool toeplitz_tiled_config_drain(int logn, int la, int lb, TiledCfg* cfg) {
  if (logn < 6 || logn > 14 || la < 1 || lb < 1 || la > 4 || lb > 4) return false;
  const uint32_t n = 1u << logn;
  auto nb_of = [&](uint32_t S) { return (8 * (uint32_t)lb * S + 15) / 16 * 16; };
  if ((uint32_t)la * nb_of(1) > (uint32_t)kTiledTmemCap) return false;
  const uint32_t rblk = n >= 1024 ? n / 1024 : 1;
  uint32_t S = 1, bpg = 1;
  if (la == lb) {
    while (S * 2 <= rblk && S * 2 <= max_shifts(la, lb) && (uint32_t)la * nb_of(S * 2) <= (uint32_t)kTiledTmemCap)
      S *= 2;
  } else {
    while (bpg * 2 <= rblk && bpg * 2 <= 4 && bpg * 2 * (uint32_t)la * nb_of(1) <= (uint32_t)kTiledTmemCap) bpg *= 2;
  }
  const uint32_t nb = nb_of(S), pitch = nb / 8 * 128 + 16;
  for (uint32_t kc = n < 1024 ? n : 1024; kc >= 64; kc /= 2) {
    const uint32_t a_win = 1024 * bpg + kc;
    const uint32_t bt_off = ((uint32_t)la * a_win * 2 + 127) / 128 * 128;
    const uint32_t smem = bt_off + kc / 8 * pitch;
    if (smem > (uint32_t)kTiledSmemCap) continue;
    cfg->bpg = bpg;
    cfg->shifts = S;
    cfg->nb = nb;
    cfg->b_pitch = pitch;
    cfg->ngrp = rblk / (bpg * S);
    cfg->kc = kc;
    cfg->a_win = a_win;
    cfg->bt_off = bt_off;
    cfg->smem = (int)smem;
    uint32_t cols = 32;
    while (cols < bpg * (uint32_t)la * nb) cols *= 2;
    cfg->tmem_cols = cols;
    return true;
  }
  return false;
}

bool lookup_toeplitz_tiled_drain(int logn, int la, int lb, KernelInfo* ki) {
  TiledCfg cfg;
  if (!toeplitz_tiled_config_drain(logn, la, lb, &cfg)) return false;
  const int S = (int)cfg.shifts, bd = (int)cfg.bpg;
#define PM_TD(A, B, SH, BPG)                       \
  if (la == A && lb == B && S == SH && bd == BPG) { \
    tiled_info<A, B, SH, true, BPG>(cfg, ki);      \
    ki->wb = 8;                                    \
    ki->digits = B;                                \
    return true;                                   \
  }
  PM_TD(1, 1, 1, 1) PM_TD(1, 1, 2, 1) PM_TD(1, 1, 4, 1)
  PM_TD(2, 2, 1, 1) PM_TD(2, 2, 2, 1) PM_TD(2, 2, 4, 1)
  PM_TD(3, 3, 1, 1) PM_TD(3, 3, 2, 1)
  PM_TD(4, 4, 1, 1) PM_TD(4, 4, 2, 1)
  // a single-digit operand on the A side (ternary b)
  PM_TD(1, 2, 1, 1) PM_TD(1, 2, 1, 2) PM_TD(1, 2, 1, 4)
  PM_TD(1, 3, 1, 1) PM_TD(1, 3, 1, 2) PM_TD(1, 3, 1, 4)
  PM_TD(1, 4, 1, 1) PM_TD(1, 4, 1, 2) PM_TD(1, 4, 1, 4)
#undef PM_TD
  return false;
}

}  // namespace pm

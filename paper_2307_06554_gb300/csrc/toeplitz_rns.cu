// Path (b) with the paper's residue number system (Sec. 2.4): the integer
// coefficients are carried as residues modulo a base of small pairwise
// coprime moduli, the matrix product runs once per modulus on small
// operands, and the Chinese remainder theorem brings the integer result
// back, reduced mod q.  The key-parameter section fixes the base: moduli of
// the matrix unit's word length, the largest first, whose product exceeds
// the range of the sums (l q^2 for l additions).
//
// What it computes: c = a * T(b) in Z_q[x]/(x^n+1) (or x^n - 1) for many
// independent (a, b) pairs, any q < 2^62 (4- or 8-byte words).  With the
// centred lifts a', b' of a and b (|a'|, |b'| <= q/2) the integer
// x_j = sum_i a'_i b'_{j-i} (signs of the wrap-around per the ring) has
// |x_j| <= n floor(q/2)^2 =: X; the base's product M exceeds 16 X.
//
// ConvertPoly: k_rns_prep writes the centred residues of a' and b' modulo
// every m_i once per row, as int8 planes (|r| <= (m-1)/2 <= 127).
//
// Per modulus m: the residues (as bf16, exact) form the same block-Hankel A
// and block-Toeplitz B as toeplitz.cu (Sec. 2.5 division, 8-coefficient
// blocks; A aliased onto a's residue window with a 16-byte row stride); B
// holds S copies of b's residues shifted by 1024 coefficients, so one A
// slice yields S blocks of 1024 outputs (N = max(16, 8 S)); one MMA chain
// per modulus; n ((m-1)/2)^2 <= 2^24 keeps every fp32 partial sum an exact
// integer.  A unit is one (product, prime, group of S blocks), K runs in
// chunks, a step is one modulus over one chunk.  Two pipelines, for the
// moduli of even and of odd index, each with its own group of four builder
// warps, its own two shared-memory stages and its own MMA-issuing warp
// (mbarrier hand-offs both ways), so the tensor cores run one step's chains
// while the next steps' operands are built (one CTA per SM, up to 512
// accumulator columns: N per modulus).
//
// Epilogue (ConvertMatrix, by the CRT): for each output, the accumulator of
// modulus i gives x mod m_i; with y_i = (x mod m_i) (M/m_i)^-1 mod m_i,
//   sum_i y_i (M/m_i) = x + k M,  k = round(sum_i y_i / m_i)
// (|x| < M/16, so the rounded quotient is exact even with the fp32 sum's
// error), and c_j = (sum_i y_i (M/m_i mod q) - k (M mod q)) mod q, summed in
// 128-bit integers.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "host_math.h"
#include "kernels.h"
#include "tcgen05.cuh"
#include "toeplitz_common.cuh"
#include "toeplitz_rns.h"

namespace pm {

namespace {
constexpr int kRnsGroup = 128;                        // threads of one builder group (4 warps)
constexpr int kRnsPipes = 2;                          // pipelines: builder group g + issuing warp g
constexpr int kRnsBuilders = kRnsGroup * kRnsPipes;   // warps 0-7: operand builds; warps 0-3 the epilogue
constexpr int kRnsThreads = kRnsBuilders + 32 * kRnsPipes;  // + warps 8, 9: MMA issue
constexpr int kRnsPipeStages = 2;                     // shared-memory stages of one pipeline
constexpr int kRnsStages = kRnsPipes * kRnsPipeStages;
constexpr int kRnsSmemCap = 200 * 1024;  // all stages
}  // namespace

// centred residue of the centred lift of v (v < q) modulo m
template <typename W>
__device__ __forceinline__ int centred_residue(W v, uint64_t q, uint32_t qm, uint32_t m, uint32_t mu32,
                                               uint64_t mu64) {
  uint32_t r;
  if constexpr (sizeof(W) == 4) {
    const uint32_t t = __umulhi((uint32_t)v, mu32);
    r = (uint32_t)v - t * m;
  } else {
    const uint64_t t = __umul64hi((uint64_t)v, mu64);
    r = (uint32_t)((uint64_t)v - t * m);
  }
  if (r >= m) r -= m;
  if ((uint64_t)v > (q >> 1)) r = r >= qm ? r - qm : r + m - qm;  // residue of v - q
  return r > (m >> 1) ? (int)r - (int)m : (int)r;
}

// Residue planes (ConvertPoly for the RNS form): one thread per 8
// coefficients of one row of a or b, all r moduli; each plane is written
// with 8-byte stores, consecutive threads on consecutive coefficients.
template <typename W>
__global__ void __launch_bounds__(256) k_rns_prep(const W* __restrict__ a, const W* __restrict__ b,
                                                 int8_t* __restrict__ out, uint64_t rows, uint32_t n, uint32_t k,
                                                 const RnsBase* __restrict__ base, const RnsPrime* __restrict__ tp,
                                                 uint32_t r) {
  const uint32_t groups = n / 8;
  const uint64_t total = 2 * rows * groups;
  for (uint64_t id = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; id < total;
       id += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t xr = id / groups;  // operand x (0: a, 1: b) and row
    const uint32_t g = (uint32_t)(id % groups);
    const uint64_t row = xr % rows;
    const W* src = (xr < rows ? a : b) + row * n + 8 * g;
    const RnsPrime& P = tp[row % k];
    W v[8];
    if constexpr (sizeof(W) == 4) {
      const uint4 x0 = *reinterpret_cast<const uint4*>(src);
      const uint4 x1 = *reinterpret_cast<const uint4*>(src + 4);
      v[0] = x0.x; v[1] = x0.y; v[2] = x0.z; v[3] = x0.w;
      v[4] = x1.x; v[5] = x1.y; v[6] = x1.z; v[7] = x1.w;
    } else {
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        const ulonglong2 x = *reinterpret_cast<const ulonglong2*>(src + 2 * h);
        v[2 * h] = x.x;
        v[2 * h + 1] = x.y;
      }
    }
    int8_t* dst = out + xr * r * n + 8 * g;
#pragma unroll 1
    for (uint32_t i = 0; i < r; ++i) {
      const uint32_t m = base->m[i], mu32 = base->mu32[i], qm = P.qm[i];
      const uint64_t mu64 = base->mu64[i];
      uint32_t lo = 0, hi = 0;
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const uint32_t byte = (uint32_t)(centred_residue<W>(v[e], P.q, qm, m, mu32, mu64) & 0xFF);
        if (e < 4)
          lo |= byte << (8 * e);
        else
          hi |= byte << (8 * (e - 4));
      }
      *reinterpret_cast<uint2*>(dst + (uint64_t)i * n) = make_uint2(lo, hi);
    }
  }
}

// 8 residues (int8, 8-byte aligned) -> 8 bf16 packed in a uint4
__device__ __forceinline__ uint4 bf16x8_of_i8(const int8_t* src) {
  const uint2 v = *reinterpret_cast<const uint2*>(src);
  auto sx = [](uint32_t w, int byte) { return (int)(w << (24 - 8 * byte)) >> 24; };
  return make_uint4(bf16x2_of(sx(v.x, 0), sx(v.x, 1)), bf16x2_of(sx(v.x, 2), sx(v.x, 3)),
                    bf16x2_of(sx(v.y, 0), sx(v.y, 1)), bf16x2_of(sx(v.y, 2), sx(v.y, 3)));
}

// plain arrival on an mbarrier (no transaction bytes)
__device__ __forceinline__ void mbar_arrive_plain(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Two independent pipelines, one for the moduli of even and one for those of
// odd index: pipeline g is a group of four builder warps (warps 4g .. 4g+3)
// that build its steps (one modulus over one K chunk each, in order) into
// its own two shared-memory stages, and one issuing warp (8 + g) that issues
// their MMA chains (one thread issuing alone measured about 100 cycles per
// small MMA; two issue in parallel).  full[s] (the group's 128 arrivals)
// hands a built stage to the issuer, empty[s] (tcgen05.commit) hands it back
// once its chains have read it.  Each barrier has one producer sequence and
// one consumer sequence, each waiting every phase in order, so an awaited
// phase is never more than one ahead and the parity test cannot alias (a
// shared ring whose stages two issuers took in turn could: an issuer could
// wait on a stage whose previous use, another issuer's, was not built yet).
// Warps 0-3 also run the epilogue.  Every wait is bounded; after the first
// expired wait the CTA stops waiting, finishes the unit (results invalid)
// and reports it.
template <typename W>
__global__ void __launch_bounds__(kRnsThreads, 1) k_toeplitz_rns(TensorRnsArgs args) {
  extern __shared__ __align__(128) unsigned char sm[];
  __shared__ __align__(8) uint64_t full[kRnsStages], empty[kRnsStages];
  __shared__ uint32_t s_tmem;
  __shared__ unsigned long long s_next;
  __shared__ int s_fail;
  __shared__ RnsBase s_base;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool builder = tid < kRnsBuilders;
  const uint32_t grp_id = (uint32_t)tid / kRnsGroup, gt = (uint32_t)tid % kRnsGroup;  // builder group, thread in it
  const uint32_t n = 1u << args.logn, D = n / 8 - 1;
  const uint32_t kc = args.kc, nch = n / kc, S = args.shifts, ngrp = args.ngrp, awin = args.a_win;
  const uint32_t NB = args.nb, pitch = args.b_pitch;
  const uint32_t wrap = args.wrap;
  const uint64_t units = args.units;
  W* C = static_cast<W*>(args.c);
  const uint32_t IDESC = idesc_bf16(128, (int)NB);

  for (uint32_t i = tid; i < sizeof(RnsBase) / 4; i += kRnsThreads)
    reinterpret_cast<uint32_t*>(&s_base)[i] = reinterpret_cast<const uint32_t*>(args.base)[i];
  if (warp == 0) {
    tmem_alloc(&s_tmem, args.tmem_cols);
    tmem_relinquish();
  }
  if (tid == 0) {
    for (int x = 0; x < kRnsStages; ++x) {
      mbar_init(&full[x], kRnsGroup);
      mbar_init(&empty[x], 1);
    }
    s_fail = 0;
  }
  fence_mbar_init();
  // padding rows of B (8-row groups past the S shifted copies: only when
  // S = 1) stay zero for the whole launch
  if (NB / 8 > S) {
    for (uint32_t ch = tid; ch < kRnsStages * (kc / 8) * 8; ch += kRnsThreads) {
      const uint32_t st = ch / ((kc / 8) * 8), dp = (ch / 8) % (kc / 8), v = ch % 8;
      *reinterpret_cast<uint4*>(sm + st * args.buf_bytes + args.bt_off + dp * pitch + 128 * S + 16 * v) =
          make_uint4(0, 0, 0, 0);
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  const uint32_t r = s_base.r;
  // steps of pipeline g per unit: every chunk times the moduli i = g mod 2
  const uint32_t cnt[kRnsPipes] = {(r + 1) / 2, r / 2};
  volatile int* fail = &s_fail;
  // a bounded wait, skipped once any wait of the CTA has expired
  auto wait = [&](uint64_t* bar, uint32_t parity) {
    if (*fail) return;
    if (!mbar_wait(bar, parity)) *fail = 1;
  };

  if (tid == 0) s_next = atomicAdd(args.ctr, 1ull);
  __syncthreads();
  unsigned long long cur = s_next;
  uint32_t done[kRnsPipes] = {0, 0};  // steps of each pipeline so far (the same counts in every thread)
  bool failed = false;
  while (cur < units) {
    __syncthreads();  // every thread has read s_next
    if (tid == 0) s_next = atomicAdd(args.ctr, 1ull);
    const uint64_t row = cur / ngrp;
    const uint32_t grp = (uint32_t)(cur % ngrp);
    const uint32_t j = (uint32_t)(row % args.k);
    const RnsPrime* tp = args.tp + j;
    const uint32_t b0 = grp * S;  // the unit's first 1024-output block

    if (builder) {
      const uint32_t g = grp_id;
      for (uint32_t t = 0; t < nch * cnt[g]; ++t) {
        const uint32_t lc = done[g] + t, x = g * kRnsPipeStages + lc % kRnsPipeStages;
        const uint32_t ch = t / cnt[g], i = g + 2 * (t % cnt[g]);
        if (lc >= (uint32_t)kRnsPipeStages) wait(&empty[x], ((lc / kRnsPipeStages) - 1) & 1u);
        unsigned char* buf = sm + x * args.buf_bytes;
        uint16_t* Xw = reinterpret_cast<uint16_t*>(buf);
        unsigned char* Bt = buf + args.bt_off;
        const int8_t* pa = args.ra + (row * r + i) * n;  // residue planes of modulus i
        const int8_t* pb = args.rb + (row * r + i) * n;
        // residues of a~_{base + e}, e < awin, as bf16 (zero outside [-n, n))
        const int32_t base = (int32_t)(1024 * b0) - (int32_t)n + 8 + (int32_t)(kc * ch);
        for (uint32_t gi = gt; gi < awin / 8; gi += kRnsGroup) {
          const int32_t i0 = base + 8 * (int32_t)gi;
          uint4 p = make_uint4(0, 0, 0, 0);
          if (i0 < (int32_t)n && i0 >= -(int32_t)n) {
            const uint32_t flip = i0 < 0 ? wrap : 0u;
            p = bf16x8_of_i8(pa + (i0 < 0 ? i0 + (int32_t)n : i0));
            p = make_uint4(p.x ^ flip, p.y ^ flip, p.z ^ flip, p.w ^ flip);
          }
          *reinterpret_cast<uint4*>(Xw + 8 * gi) = p;
        }
        // the chunk's K-blocks of B, one 8-row group per shift s: K-block d'
        // of shift s is b~'s group G = D - d' + 128 s after group G - 1, with
        // b~ the extension of b over [-n, 2n) (groups outside [0, n/8) are
        // b's groups n/8 away, negated for x^n + 1); shift s gives the
        // outputs 1024 s further on from the same A
        const uint32_t ng = n / 8;
        for (uint32_t dl = gt; dl < kc / 8; dl += kRnsGroup) {
          const int32_t g0 = (int32_t)(D - (kc / 8 * ch + dl));
          for (uint32_t sh = 0; sh < S; ++sh) {
            const int32_t G = g0 + 128 * (int32_t)sh, H = G - 1;
            const uint32_t gg = (uint32_t)(G >= (int32_t)ng ? G - (int32_t)ng : G);
            const uint32_t hh = (uint32_t)(H < 0 ? H + (int32_t)ng : H >= (int32_t)ng ? H - (int32_t)ng : H);
            const uint32_t fg = G >= (int32_t)ng ? wrap : 0u;
            const uint32_t fh = (H < 0 || H >= (int32_t)ng) ? wrap : 0u;
            const uint4 pv = bf16x8_of_i8(pb + 8 * hh);
            const uint4 ow = bf16x8_of_i8(pb + 8 * gg);
            const uint32_t E[8] = {pv.x ^ fh, pv.y ^ fh, pv.z ^ fh, pv.w ^ fh, ow.x ^ fg, ow.y ^ fg, ow.z ^ fg, ow.w ^ fg};
            b_block_rows(E, Bt + dl * pitch + 128 * sh);
          }
        }
        fence_proxy_async();  // this thread's stores, visible to the tensor cores
        mbar_arrive_plain(&full[x]);
      }
    } else if (lane == 0) {
      // ---- TPUMul: pipeline g's chains, as its stages fill ----
      const uint32_t g = (uint32_t)warp - kRnsBuilders / 32;
      const uint64_t BSTEP = (2 * pitch) >> 4;
      for (uint32_t t = 0; t < nch * cnt[g]; ++t) {
        const uint32_t lc = done[g] + t, x = g * kRnsPipeStages + lc % kRnsPipeStages;
        const uint32_t ch = t / cnt[g], i = g + 2 * (t % cnt[g]);
        wait(&full[x], (lc / kRnsPipeStages) & 1u);
        tc_fence_after();
        const uint32_t xa0 = smem_u32(sm + x * args.buf_bytes);
        const uint64_t ad0 = smem_desc(xa0, 16, 128), bd0 = smem_desc(xa0 + args.bt_off, pitch, 128);
        const uint32_t dcol = tmem + i * NB;
#pragma unroll 4
        for (uint32_t kk = 0; kk < kc / 16; ++kk)
          tc_mma_f16(dcol, ad0 + 2u * (uint64_t)kk, bd0 + BSTEP * (uint64_t)kk, IDESC, (ch > 0 || kk > 0) ? 1u : 0u);
        tc_commit(&empty[x]);
      }
    }
    if (warp >= kRnsBuilders / 32) __syncwarp();
    for (int g = 0; g < kRnsPipes; ++g) done[g] += nch * cnt[g];

    // ---- ConvertMatrix: the CRT per output, reduced mod q (warps 0-3) ----
    if (tid < kRnsGroup) {
      // every chain of the unit has completed: each pipeline's last commits,
      // in its order (each stage's previous commit was awaited by its
      // builders before they refilled it, so no awaited phase is more than
      // one ahead of its barrier)
      for (int g = 0; g < kRnsPipes; ++g)
        for (uint32_t lc = done[g] > (uint32_t)kRnsPipeStages ? done[g] - kRnsPipeStages : 0; lc < done[g]; ++lc)
          wait(&empty[g * kRnsPipeStages + lc % kRnsPipeStages], (lc / kRnsPipeStages) & 1u);
      tc_fence_after();
      const uint64_t q = tp->q;
      W* c = C + row * n;
#pragma unroll 1
      for (uint32_t sh = 0; sh < S; ++sh) {
        uint64_t slo[8], shi[8];
        float f[8];
#pragma unroll
        for (int v = 0; v < 8; ++v) {
          slo[v] = 0;
          shi[v] = 0;
          f[v] = 0.f;
        }
#pragma unroll 1
        for (uint32_t i = 0; i < r; ++i) {
          uint32_t acc[16];
          // warp-collective: every lane loads, only the stores below are predicated
          // columns i N + 8 sh .. + 7: the 16-column load that holds them
          tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + i * NB + 16 * (sh / 2), acc);
          tmem_wait_ld();
          const uint32_t o8 = 8 * (sh & 1u);
          const uint32_t m = s_base.m[i], mu32 = s_base.mu32[i], t = s_base.t[i], off = s_base.off[i];
          const float im = s_base.inv_m[i];
          const uint64_t Mq = tp->Mq[i];
#pragma unroll
          for (int v = 0; v < 8; ++v) {
            // x mod m from the exact integer accumulator (|value| <= 2^24)
            const uint32_t bits = o8 ? acc[8 + v] : acc[v];
            uint32_t u = (uint32_t)(__float2int_rn(__uint_as_float(bits)) + (int)off);
            u -= __umulhi(u, mu32) * m;
            if (u >= m) u -= m;
            uint32_t y = u * t;  // < 2^16
            y -= __umulhi(y, mu32) * m;
            if (y >= m) y -= m;
            const uint64_t plo = (uint64_t)y * Mq, phi = __umul64hi((uint64_t)y, Mq);
            slo[v] += plo;
            shi[v] += phi + (slo[v] < plo ? 1u : 0u);
            f[v] = fmaf((float)y, im, f[v]);
          }
        }
        const uint32_t j0 = 8 * (128 * (b0 + sh) + (uint32_t)tid);
        W out[8];
#pragma unroll
        for (int v = 0; v < 8; ++v) {
          const uint64_t kq = (uint64_t)rintf(f[v]);  // the quotient k of the reconstruction
          unsigned __int128 s = ((unsigned __int128)shi[v] << 64) | slo[v];
          s += (unsigned __int128)kq * (q - tp->mq);  // - k M  (mod q)
          out[v] = (W)(uint64_t)(s % q);
        }
        if (j0 < n) {
#pragma unroll
          for (int v = 0; v < 8; ++v) c[j0 + v] = out[v];
        }
      }
    }
    tc_fence_before();
    if (__syncthreads_or(*fail != 0)) {
      failed = true;
      break;
    }
    cur = s_next;
  }
  if (failed && tid == 0) {
    atomicExch(args.err, 1);
    // let the chains in flight finish before the memory they read is freed
    for (int g = 0; g < kRnsPipes; ++g)
      for (uint32_t lc = done[g] > (uint32_t)kRnsPipeStages ? done[g] - kRnsPipeStages : 0; lc < done[g]; ++lc)
        mbar_wait(&empty[g * kRnsPipeStages + lc % kRnsPipeStages], (lc / kRnsPipeStages) & 1u);
  }
  tc_fence_before();
  __syncthreads();
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

// ------------------------------------------------------------------ host

uint32_t rns_modulus_cap(uint32_t n) {
  uint32_t h = 0;
  while ((uint64_t)(h + 1) * (h + 1) * n <= (1ull << 24)) ++h;  // n h^2 <= 2^24
  uint32_t m = 2 * h + 1;
  return m > 255 ? 255 : m;
}

static uint32_t gcd32(uint32_t x, uint32_t y) {
  while (y) {
    const uint32_t t = x % y;
    x = y;
    y = t;
  }
  return x;
}

bool rns_choose_base(uint32_t n, uint64_t qmax, std::vector<uint32_t>* moduli) {
  moduli->clear();
  // log2 of the bound 16 n floor(qmax/2)^2
  const double hq = (double)(qmax / 2);
  const double need = 4.0 + std::log2((double)n) + 2.0 * std::log2(hq > 1.0 ? hq : 1.0);
  double have = 0.0;
  for (uint32_t m = rns_modulus_cap(n); m >= 3 && have <= need + 1e-6; m -= 2) {
    bool coprime = true;
    for (uint32_t x : *moduli) coprime = coprime && gcd32(m, x) == 1;
    if (!coprime) continue;
    if (moduli->size() == (size_t)kRnsMax) return false;
    moduli->push_back(m);
    have += std::log2((double)m);
  }
  return have > need + 1e-6;
}

void rns_tables(const std::vector<uint32_t>& moduli, const std::vector<uint64_t>& primes, RnsBase* base,
                std::vector<RnsPrime>* per_prime) {
  using host::u128;
  memset(base, 0, sizeof *base);
  const uint32_t r = (uint32_t)moduli.size();
  base->r = r;
  for (uint32_t i = 0; i < r; ++i) {
    const uint32_t m = moduli[i];
    base->m[i] = m;
    base->mu32[i] = (uint32_t)((1ull << 32) / m);
    base->mu64[i] = (uint64_t)(((u128)1 << 64) / m);
    base->off[i] = ((1u << 24) + m - 1) / m * m;
    base->inv_m[i] = 1.0f / (float)m;
    uint64_t Mi = 1;  // (M / m_i) mod m_i
    for (uint32_t l = 0; l < r; ++l)
      if (l != i) Mi = Mi * moduli[l] % m;
    base->t[i] = 0;
    for (uint32_t t = 1; t < m; ++t)  // its inverse mod m_i, by search (m_i < 256)
      if (Mi * t % m == 1) {
        base->t[i] = t;
        break;
      }
  }
  per_prime->assign(primes.size(), RnsPrime{});
  for (size_t j = 0; j < primes.size(); ++j) {
    RnsPrime& P = (*per_prime)[j];
    memset(&P, 0, sizeof P);
    const uint64_t q = primes[j];
    P.q = q;
    uint64_t M = 1 % q;
    for (uint32_t i = 0; i < r; ++i) M = (uint64_t)((u128)M * moduli[i] % q);
    P.mq = M;
    for (uint32_t i = 0; i < r; ++i) {
      uint64_t Mi = 1 % q;
      for (uint32_t l = 0; l < r; ++l)
        if (l != i) Mi = (uint64_t)((u128)Mi * moduli[l] % q);
      P.Mq[i] = Mi;
      P.qm[i] = (uint32_t)(q % moduli[i]);
    }
  }
}

bool rns_config(int logn, uint32_t r, RnsCfg* cfg) {
  if (logn < 6 || logn > 14 || r < 1 || r > (uint32_t)kRnsMax) return false;
  const uint32_t n = 1u << logn;
  const uint32_t rblk = n >= 1024 ? n / 1024 : 1;
  // shifted copies of b per chain: as many blocks as the accumulators of r
  // chains of N = 8 S columns allow
  uint32_t S = 1;
  while (S * 2 <= rblk && r * 8 * (S * 2) <= 512) S *= 2;
  const uint32_t nb = S * 8 < 16 ? 16 : S * 8;
  const uint32_t pitch = nb / 8 * 128 + 16;
  if (r * nb > 512) return false;
  uint32_t kc = n < 1024 ? n : 1024;
  for (;;) {
    const uint32_t a_win = 1024 + kc;  // one A slice (the unit's first block)
    const uint32_t bt_off = (a_win * 2 + 127) / 128 * 128;
    const uint32_t buf = (bt_off + kc / 8 * pitch + 127) / 128 * 128;
    if (kRnsStages * buf <= (uint32_t)kRnsSmemCap || kc <= 128) {
      if (kRnsStages * buf > (uint32_t)kRnsSmemCap) return false;
      cfg->shifts = S;
      cfg->nb = nb;
      cfg->b_pitch = pitch;
      cfg->ngrp = rblk / S;
      cfg->kc = kc;
      cfg->a_win = a_win;
      cfg->bt_off = bt_off;
      cfg->buf_bytes = buf;
      cfg->smem = (int)(kRnsStages * buf);
      uint32_t cols = 32;
      while (cols < r * nb) cols *= 2;
      cfg->tmem_cols = cols;
      return true;
    }
    kc /= 2;
  }
}

int rns_prep_launch(uint32_t elem, const void* a, const void* b, int8_t* out, uint64_t rows, uint32_t n,
                    uint32_t k, const RnsBase* base, const RnsPrime* tp, uint32_t r, int num_sms, void* stream) {
  const uint64_t threads = 2 * rows * (n / 8);
  const int grid = (int)std::min<uint64_t>((threads + 255) / 256, (uint64_t)num_sms * 16);
  cudaStream_t st = (cudaStream_t)stream;
  if (elem == 4)
    k_rns_prep<uint32_t><<<grid, 256, 0, st>>>((const uint32_t*)a, (const uint32_t*)b, out, rows, n, k, base, tp, r);
  else
    k_rns_prep<uint64_t><<<grid, 256, 0, st>>>((const uint64_t*)a, (const uint64_t*)b, out, rows, n, k, base, tp, r);
  return (int)cudaGetLastError();
}

bool lookup_toeplitz_rns(int logn, uint32_t r, uint32_t elem, KernelInfo* ki) {
  RnsCfg cfg;
  if (!rns_config(logn, r, &cfg)) return false;
  if (elem == 4)
    ki->fn = (const void*)k_toeplitz_rns<uint32_t>;
  else if (elem == 8)
    ki->fn = (const void*)k_toeplitz_rns<uint64_t>;
  else
    return false;
  ki->block = kRnsThreads;
  ki->smem = cfg.smem;
  ki->team = kRnsThreads;
  ki->units_per_cta = 1;
  ki->tmem_cols = (int)cfg.tmem_cols;
  ki->rns = 1;
  return true;
}

}  // namespace pm

// Path (b) for moduli up to 2^62 in 64-bit words: the drained tiled kernel's
// algebra (toeplitz_tiled.cu: Sec. 2.2 matrix form, Sec. 2.5 division into
// 8-coefficient blocks, Sec. 2.6 pieces for high degrees) with L = 5 .. 8
// balanced 8-bit digits of each centred residue (Sec. 2.4: eight cover
// |x| < 2^62), at every degree 2^10 .. 2^16.
//
// A unit of work is one (product, prime, 1024-output block): L chains (one
// per digit of a, N = 8 L columns: b's digits) accumulate a K chunk of at
// most 1024 in tensor memory (each fp32 partial sum is an exact integer of
// magnitude at most 1024 x 128^2 = 2^24), the CTA waits for them, and each
// thread (one output row of the block, 8 outputs) drains the chunk: per
// weight 2^(8e), e = s + g, the sums of the digit pairs with s + g = e are
// added in 32-bit integers (at most 8 of them: below 2^27), made
// non-negative with a multiple of q, and multiplied by 2^(8e) mod q with a
// 64-bit Shoup multiplication; the row's 8 outputs accumulate mod q over
// the chunks (ConvertMatrix, Algorithm 1).  One 128-thread CTA per SM
// (L chains of up to 64 columns fill the 512 tensor-memory columns).
// Every wait is bounded: an expired wait records the error and the CTA
// leaves through its finish protocol after its MMAs in flight complete.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "kernels.h"
#include "polymul_types.h"
#include "tcgen05.cuh"
#include "toeplitz_common.cuh"
#include "toeplitz_tiled.cuh"
#include "toeplitz_u64.h"

namespace pm {

namespace {
constexpr int kU64Threads = 128;
constexpr int kU64SmemCap = 224 * 1024;
constexpr int kU64TmemCap = 512;
}  // namespace

// balanced 8-bit digits of the centred representatives of 8 consecutive
// coefficients v < q < 2^62 (16-byte aligned); per digit 8 bf16 packed in
// a uint4
template <int L>
__device__ __forceinline__ void digits8_u64(const uint64_t* src, uint64_t q, uint4 (&out)[L]) {
  int d[8][L];
#pragma unroll
  for (int h = 0; h < 4; ++h) {
    const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(src + 2 * h);
    const uint64_t xv[2] = {v.x, v.y};
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      int64_t x = xv[i] > (q >> 1) ? (int64_t)(xv[i] - q) : (int64_t)xv[i];
#pragma unroll
      for (int s = 0; s < L; ++s) {
        const int32_t t = (((int32_t)x + 128) & 255) - 128;  // depends on the low byte only
        x = (x - t) >> 8;
        d[2 * h + i][s] = t;
      }
    }
  }
#pragma unroll
  for (int s = 0; s < L; ++s)
    out[s] = make_uint4(bf16x2_of(d[0][s], d[1][s]), bf16x2_of(d[2][s], d[3][s]), bf16x2_of(d[4][s], d[5][s]),
                        bf16x2_of(d[6][s], d[7][s]));
}

// x w mod q for x < 2^64, w < q < 2^62, wp = floor(w 2^64 / q) (Shoup)
__device__ __forceinline__ uint64_t mulmod_shoup64(uint64_t x, uint64_t w, uint64_t wp, uint64_t q) {
  const uint64_t qh = __umul64hi(x, wp);
  const uint64_t r = x * w - qh * q;
  return r >= q ? r - q : r;
}

// Adds chain sums of digit pairs with s + g = E (chains s at column s N of
// `base`, b's digit g at columns 8 g .. 8 g + 7) times 2^(8E) mod q to acc.
template <int L, int E>
__device__ __forceinline__ void drain_weight(uint32_t base, const TensorPrime64& tp, uint64_t (&acc)[8]) {
  using TS = TTShape<L, 1>;
  constexpr int s_lo = E - (L - 1) > 0 ? E - (L - 1) : 0;
  constexpr int s_hi = E + 1 < L ? E + 1 : L;  // s in [s_lo, s_hi), g = E - s
  int32_t x[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  // at most four 8-column loads in flight per wait
  cfor<0, (s_hi - s_lo + 3) / 4>([&](auto bc) {
    constexpr int b0 = s_lo + 4 * decltype(bc)::value;
    constexpr int b1 = b0 + 4 < s_hi ? b0 + 4 : s_hi;
    uint32_t r[b1 - b0][8];
    cfor<b0, b1>([&](auto sc) {
      constexpr int s = decltype(sc)::value;
      tmem_ld8(base + (uint32_t)(s * TS::NB + 8 * (E - s)), r[s - b0]);
    });
    tmem_wait_ld();
#pragma unroll
    for (int i = 0; i < b1 - b0; ++i)
#pragma unroll
      for (int v = 0; v < 8; ++v) x[v] += __float2int_rn(__uint_as_float(r[i][v]));
  });
#pragma unroll
  for (int v = 0; v < 8; ++v) {
    const uint64_t t = mulmod_shoup64((uint64_t)((int64_t)x[v] + (int64_t)tp.bias), tp.pw[E], tp.pwp[E], tp.q);
    const uint64_t y = acc[v] + t;
    acc[v] = y >= tp.q ? y - tp.q : y;
  }
}

template <int L>
__global__ void __launch_bounds__(kU64Threads, 1) k_toeplitz_u64(TensorU64Args args) {
  using TS = TTShape<L, 1>;
  extern __shared__ __align__(128) unsigned char sm[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t s_tmem;
  __shared__ unsigned long long s_next;
  const int tid = threadIdx.x, warp = tid >> 5;
  const uint32_t n = 1u << args.logn, D = n / 8 - 1;
  const uint32_t kc = args.kc, nch = n / kc, ngrp = args.ngrp, awin = args.a_win;
  const uint32_t wrap = args.wrap;
  const uint64_t units = args.units;
  uint16_t* Xw = reinterpret_cast<uint16_t*>(sm);  // [L][awin] digits of a~ over the chunk's window
  unsigned char* Bt = sm + args.bt_off;             // [kc/8][BT_PITCH] the chunk of B
  constexpr uint32_t IDESC = idesc_bf16(128, TS::NB);

  if (warp == 0) {
    tmem_alloc(&s_tmem, args.tmem_cols);
    tmem_relinquish();
  }
  if (tid == 0) mbar_init(&mbar, 1);
  fence_mbar_init();
  if (TS::NG > L) {  // padded rows of B stay zero for the whole launch
    for (uint32_t x = tid; x < (kc / 8) * TS::NG * 8; x += kU64Threads) {
      const uint32_t dp = x / (TS::NG * 8), g = (x / 8) % TS::NG, v = x % 8;
      if (g >= (uint32_t)L) *reinterpret_cast<uint4*>(Bt + dp * TS::BT_PITCH + g * 128 + 16 * v) = make_uint4(0, 0, 0, 0);
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  const uint32_t lane_base = tmem + ((uint32_t)(32 * warp) << 16);

  if (tid == 0) s_next = atomicAdd(args.ctr, 1ull);
  __syncthreads();
  unsigned long long cur = s_next;
  uint32_t parity = 0;
  bool failed = false;
  const int32_t ng = (int32_t)(n / 8);
  while (cur < units) {
    __syncthreads();  // every thread has read s_next
    if (tid == 0) s_next = atomicAdd(args.ctr, 1ull);
    const uint64_t row = cur / ngrp;
    const uint32_t grp = (uint32_t)(cur % ngrp);
    const uint32_t jr = (uint32_t)(row % args.k);
    const TensorPrime64& tp = args.tp[args.pmap ? args.pmap[jr] : jr];
    const uint64_t q = tp.q;
    const uint64_t* a = args.a + row * n;
    const uint64_t* b = args.b + row * n;
    uint64_t acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (uint32_t ch = 0; ch < nch; ++ch) {
      // ConvertPoly (a): digits of a~_{base + e}, e < awin (groups of 8 lie
      // wholly in a or in its extension: base and group sizes are multiples of 8)
      const int32_t base = (int32_t)(1024 * grp) - (int32_t)n + 8 + (int32_t)(kc * ch);
      for (uint32_t gi = tid; gi < awin / 8; gi += kU64Threads) {
        const int32_t i0 = base + 8 * (int32_t)gi;
        uint4 p[L];
        uint32_t flip = 0;
        if (i0 >= (int32_t)n || i0 < -(int32_t)n) {
#pragma unroll
          for (int s = 0; s < L; ++s) p[s] = make_uint4(0, 0, 0, 0);
        } else {
          flip = i0 < 0 ? wrap : 0u;
          digits8_u64<L>(a + (i0 < 0 ? i0 + (int32_t)n : i0), q, p);
        }
#pragma unroll
        for (int s = 0; s < L; ++s)
          *reinterpret_cast<uint4*>(Xw + (size_t)s * awin + 8 * gi) =
              make_uint4(p[s].x ^ flip, p[s].y ^ flip, p[s].z ^ flip, p[s].w ^ flip);
      }
      // ConvertPoly (b): K-block d' = kc/8 ch + dl is b~'s group G = D - d'
      // after group G - 1 (b~ over [-n, 2n))
      for (uint32_t dl = tid; dl < kc / 8; dl += kU64Threads) {
        const int32_t G = (int32_t)(D - (kc / 8 * ch + dl)), H = G - 1;
        const uint32_t gg = (uint32_t)G;
        const uint32_t hh = (uint32_t)(H < 0 ? H + ng : H);
        const uint32_t fh = H < 0 ? wrap : 0u;
        uint4 pv[L], ow[L];
        digits8_u64<L>(b + 8 * hh, q, pv);
        digits8_u64<L>(b + 8 * gg, q, ow);
#pragma unroll
        for (int s2 = 0; s2 < L; ++s2) {
          const uint32_t E[8] = {pv[s2].x ^ fh, pv[s2].y ^ fh, pv[s2].z ^ fh, pv[s2].w ^ fh,
                                 ow[s2].x,      ow[s2].y,      ow[s2].z,      ow[s2].w};
          b_block_rows(E, Bt + dl * TS::BT_PITCH + s2 * 128);
        }
      }
      fence_proxy_async();
      tc_fence_before();
      __syncthreads();
      // TPUMul: one thread issues the chunk's L chains, one at a time
      if (tid == 0) {
        tc_fence_after();
        const uint32_t xa0 = smem_u32(Xw), bt0 = smem_u32(Bt);
        const uint64_t bd0 = smem_desc(bt0, TS::BT_PITCH, 128);
        constexpr uint64_t BSTEP = (2 * TS::BT_PITCH) >> 4;  // two K-blocks per MMA (K = 16)
#pragma unroll 1
        for (int s = 0; s < L; ++s) {
          const uint64_t ad0 = smem_desc(xa0 + (uint32_t)(s * awin) * 2, 16, 128);
#pragma unroll 4
          for (uint32_t kk = 0; kk < kc / 16; ++kk)
            tc_mma_f16(tmem + (uint32_t)(s * TS::NB), ad0 + 2u * (uint64_t)kk, bd0 + BSTEP * (uint64_t)kk, IDESC,
                       kk > 0 ? 1u : 0u);
        }
        tc_commit(&mbar);
      }
      if (warp == 0) __syncwarp();
      const bool ok = mbar_wait(&mbar, parity);
      if (__syncthreads_or(!ok)) {
        failed = true;
        break;
      }
      parity ^= 1u;
      tc_fence_after();
      // drain: every weight 2^(8e) of the chunk's digit pairs
      cfor<0, 2 * L - 1>([&](auto ec) { drain_weight<L, decltype(ec)::value>(lane_base, tp, acc); });
      tc_fence_before();  // these loads before the next chunk's MMAs overwrite the accumulators
    }
    if (failed) break;
    // ConvertMatrix: the row's 8 outputs, reduced mod q over the chunks
    const uint32_t j0 = 8 * (128 * grp + (uint32_t)tid);
    if (j0 < n) {
      uint64_t* c = args.c + row * n + j0;
#pragma unroll
      for (int h = 0; h < 4; ++h) *reinterpret_cast<ulonglong2*>(c + 2 * h) = make_ulonglong2(acc[2 * h], acc[2 * h + 1]);
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

// ---------------------------------------------------------------- host side

int u64_digits(uint64_t qmax) {
  for (int l = 1; l <= 8; ++l) {
    // (2^7 - 1)(2^(8l) - 1)/(2^8 - 1) in 128 bits
    const unsigned __int128 reach = ((unsigned __int128)127 * (((unsigned __int128)1 << (8 * l)) - 1)) / 255;
    if (reach >= qmax / 2) return l;
  }
  return 0;
}

bool toeplitz_u64_config(int logn, int L, TiledCfg* cfg) {
  if (logn < 10 || logn > 16 || L < 5 || L > 8) return false;
  const uint32_t n = 1u << logn;
  const uint32_t nb = (8 * (uint32_t)L + 15) / 16 * 16, pitch = nb / 8 * 128 + 16;
  if ((uint32_t)L * nb > (uint32_t)kU64TmemCap) return false;
  for (uint32_t kc = 1024; kc >= 64; kc /= 2) {
    const uint32_t a_win = 1024 + kc;
    const uint32_t bt_off = ((uint32_t)L * a_win * 2 + 127) / 128 * 128;
    const uint32_t smem = bt_off + kc / 8 * pitch;
    if (smem > (uint32_t)kU64SmemCap) continue;
    cfg->bpg = 1;
    cfg->shifts = 1;
    cfg->nb = nb;
    cfg->b_pitch = pitch;
    cfg->ngrp = n / 1024;
    cfg->kc = kc;
    cfg->a_win = a_win;
    cfg->bt_off = bt_off;
    cfg->smem = (int)smem;
    uint32_t cols = 32;
    while (cols < (uint32_t)L * nb) cols *= 2;
    cfg->tmem_cols = cols;
    return true;
  }
  return false;
}

template <int L>
static void u64_info(const TiledCfg& cfg, KernelInfo* ki) {
  ki->fn = (const void*)k_toeplitz_u64<L>;
  ki->block = kU64Threads;
  ki->smem = cfg.smem;
  ki->team = kU64Threads;
  ki->units_per_cta = 1;
  ki->tmem_cols = (int)cfg.tmem_cols;
  ki->tiled = 1;
  ki->drain = 1;
  ki->u64 = 1;
  ki->wb = 8;
  ki->digits = L;
}

bool lookup_toeplitz_u64(int logn, int L, KernelInfo* ki) {
  TiledCfg cfg;
  if (!toeplitz_u64_config(logn, L, &cfg)) return false;
  switch (L) {
    case 5: u64_info<5>(cfg, ki); return true;
    case 6: u64_info<6>(cfg, ki); return true;
    case 7: u64_info<7>(cfg, ki); return true;
    case 8: u64_info<8>(cfg, ki); return true;
    default: return false;
  }
}

}  // namespace pm

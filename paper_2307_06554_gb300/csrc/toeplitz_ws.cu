// Path (b), drained K chunks, as a warp-specialised pipeline.  The algebra,
// digits and tiling are those of the drained tiled kernel (toeplitz_tiled.cu:
// Sec. 2.2 matrix form, Sec. 2.5 division into 8-coefficient blocks, Sec. 2.6
// pieces for high degrees, 8-bit balanced digits of the centred residues,
// each K chunk's exact fp32 sums drained into 64-bit integer sums).  There
// one CTA builds a chunk's operands, waits for its MMAs and drains them in
// turn, and only the second CTA of the SM fills the gaps.  Here one CTA per
// SM runs the three phases concurrently on different chunks:
//   * builder warps 0..10 build chunk i's digit window of a~ and its K-blocks
//     of B into shared-memory stage i % 2, once the MMAs of chunk i - 2 have
//     read that stage (`mma_done`), then arrive on `built`;
//   * lane 0 of warp 11 issues chunk i's MMA chains into tensor-memory buffer
//     i % 2, once `built` and once the drain of chunk i - 2 has emptied that
//     buffer (`drained`), and commits them to `mma_done`;
//   * drainer warps 12..15 (warp w reads tensor-memory lanes 32 (w % 4) ..
//     32 (w % 4) + 31, so each thread owns one output row of the 128-row
//     block) wait for `mma_done`, add the chunk's digit-pair sums times
//     2^(8(s+g)) mod q into registers, reduce them mod q, arrive on
//     `drained`, and store a unit's outputs after its last chunk.
// The build of chunk i + 1 and the drain of chunk i - 1 thus overlap the
// MMAs of chunk i.  The builds are bound by load latency and instruction
// issue, so they get most of the warps.  Units of work are assigned statically (the CTA's r-th
// unit is blockIdx.x + r gridDim.x), so every role walks the same sequence
// of (unit, chunk) steps without exchanging indices.  Every wait is bounded:
// a role whose wait expires records it and stops, the others' waits then
// expire in turn, and before tensor memory is released the issuing lane
// waits for the chains it committed.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "kernels.h"
#include "polymul_types.h"
#include "tcgen05.cuh"
#include "toeplitz_common.cuh"
#include "toeplitz_tiled.cuh"
#include "toeplitz_tiled.h"

namespace pm {

namespace {
// warps 0..6 build, warp 7 issues the MMAs, warps 8..15 drain (two sets of
// four, one warp per 32-lane quarter of tensor memory in each): 16 warps
// (registers are allocated to a CTA in groups of four warps, so 128 per
// thread; a 17th warp would cut that to 96)
constexpr int kWsBuildWarps = 7;
constexpr int kWsDrainWarps = 8;
constexpr int kWsBuilders = 32 * kWsBuildWarps;
constexpr int kWsDrainers = 32 * kWsDrainWarps;
constexpr int kWsMmaWarp = kWsBuildWarps;
constexpr int kWsDrainWarp0 = kWsMmaWarp + 1;
constexpr int kWsThreads = 32 * (kWsDrainWarp0 + kWsDrainWarps);
constexpr int kWsSmemCap = 224 * 1024;  // two stages in one CTA per SM
constexpr int kWsTmemCap = 512;         // two accumulator buffers
static_assert(kWsDrainWarps == 8 && kWsDrainWarp0 % 4 == 0,
              "drainer warp w reads the 32-lane quarter w % 4 of tensor memory");

// Drainer set H (warps kWsDrainWarp0 + 4H .. + 3) of the step's chunk in
// tensor-memory buffer `tb`: with several digits of a, set H takes digits
// [H LA/2, (H+1) LA/2) of a for every output group (the two sets' sums are
// added at the unit's end); with one digit of a, the output groups g with
// g % 2 == H.  Group g is A slice g / S, shift g % S.
template <int LA, int LB, int S, int BD, int H>
struct WsDrainSet {
  static constexpr bool kSplitDigits = LA >= 2;
  static constexpr int kS0 = kSplitDigits ? H * (LA / 2) : 0;
  static constexpr int kS1 = kSplitDigits ? (H == 0 ? LA / 2 : LA) : LA;
  static constexpr int kGroups = kSplitDigits ? BD * S : (BD * S + 1 - H) / 2;
  static constexpr int group(int li) { return kSplitDigits ? li : 2 * li + H; }
};

template <int LA, int LB, int S, int BD, int H, int NG>
__device__ __forceinline__ void ws_drain_chunk(uint32_t tb, const TensorPrime& tp, int64_t (&acc)[NG][8]) {
  using DS = WsDrainSet<LA, LB, S, BD, H>;
  using TS = TTShape<LB, S>;
  cfor<0, DS::kGroups>([&](auto lc) {
    constexpr int li = decltype(lc)::value, g = DS::group(li);
    drain_pairs<LA, LB, S, g % S, DS::kS0, DS::kS1>(tb + (uint32_t)((g / S) * LA * TS::NB), tp.pw, acc[li]);
#pragma unroll
    for (int v = 0; v < 8; ++v) acc[li][v] = barrett64((uint64_t)(acc[li][v] + (int64_t)tp.bias), tp.q, tp.mu);
  });
}
}  // namespace

// the unit's (product, prime) row: element offset and prime index
struct WsRow {
  uint64_t off;
  uint32_t j;
};
__device__ __forceinline__ WsRow ws_row(const TensorTiledArgs& args, uint64_t row, uint32_t n) {
  if (args.rows) {
    const RaggedUnit u = args.rows[row];
    return WsRow{u.offset, u.prime};
  }
  return WsRow{row * n, (uint32_t)(row % args.k)};
}

// One drainer set's walk over the CTA's steps: wait for the chunk's MMAs,
// drain its part of the buffer into 64-bit sums reduced mod q, release the
// buffer, and after a unit's last chunk store its outputs.  With the digits
// of a split between the sets, set 1 hands its reduced sums to set 0
// through shared memory (`comb`, guarded by two mbarriers), and set 0 adds
// them and stores.  Every wait is bounded; on expiry the set records it and
// returns.
template <int LA, int LB, int S, int BD, int H>
__device__ __forceinline__ void ws_drain_role(const TensorTiledArgs& args, uint64_t steps, uint32_t nch, uint32_t ngrp,
                                              uint32_t n, uint32_t r, uint32_t lane_base, uint32_t buf_cols,
                                              uint64_t* mma_done, uint64_t* drained, uint64_t* comb_full,
                                              uint64_t* comb_free, uint32_t* comb, int& s_fail) {
  using DS = WsDrainSet<LA, LB, S, BD, H>;
  constexpr int NG = DS::kGroups > 0 ? DS::kGroups : 1;
  int64_t acc[NG][8];
#pragma unroll
  for (int g = 0; g < NG; ++g)
#pragma unroll
    for (int v = 0; v < 8; ++v) acc[g][v] = 0;
  uint32_t units_done = 0;
  for (uint64_t st = 0; st < steps; ++st) {
    const uint32_t k = (uint32_t)(st & 1), use = (uint32_t)(st >> 1);
    if (!mbar_wait(&mma_done[k], use & 1u)) {
      s_fail = 1;
      return;
    }
    tc_fence_after();
    const uint64_t unit = blockIdx.x + (st / nch) * gridDim.x;
    const uint32_t ch = (uint32_t)(st % nch);
    const WsRow wr = ws_row(args, unit / ngrp, n);
    const TensorPrime& tp = args.tp[wr.j];
    if constexpr (DS::kGroups > 0) ws_drain_chunk<LA, LB, S, BD, H, NG>(lane_base + k * buf_cols, tp, acc);
    tc_fence_before();
    mbar_arrive(&drained[k]);  // the buffer may be overwritten by chunk i + 2
    if (ch != nch - 1) continue;
    // ConvertMatrix: the unit's outputs, reduced after its last chunk
    const uint32_t b0 = (uint32_t)(unit % ngrp) * BD * S;
    if constexpr (DS::kSplitDigits && H == 1) {
      if (units_done > 0 && !mbar_wait(comb_free, (units_done - 1) & 1u)) {
        s_fail = 1;
        return;
      }
#pragma unroll
      for (int g = 0; g < NG; ++g)
#pragma unroll
        for (int v = 0; v < 8; ++v) comb[((uint32_t)g * 128 + r) * 8 + v] = (uint32_t)acc[g][v];
      mbar_arrive(comb_full);
    } else {
      if constexpr (DS::kSplitDigits) {
        if (!mbar_wait(comb_full, units_done & 1u)) {
          s_fail = 1;
          return;
        }
#pragma unroll
        for (int g = 0; g < NG; ++g)
#pragma unroll
          for (int v = 0; v < 8; ++v) {
            const uint64_t x = (uint64_t)acc[g][v] + comb[((uint32_t)g * 128 + r) * 8 + v];  // < 2q
            acc[g][v] = (int64_t)(x >= tp.q ? x - tp.q : x);
          }
        mbar_arrive(comb_free);
      }
      uint32_t* c = args.c + wr.off;
#pragma unroll
      for (int li = 0; li < DS::kGroups; ++li) {
        const int g = DS::group(li);
        const uint32_t j0 = 8 * (128 * (b0 + (uint32_t)(g / S) + (uint32_t)(g % S)) + r);
        if (j0 < n) {
          *reinterpret_cast<uint4*>(c + j0) =
              make_uint4((uint32_t)acc[li][0], (uint32_t)acc[li][1], (uint32_t)acc[li][2], (uint32_t)acc[li][3]);
          *reinterpret_cast<uint4*>(c + j0 + 4) =
              make_uint4((uint32_t)acc[li][4], (uint32_t)acc[li][5], (uint32_t)acc[li][6], (uint32_t)acc[li][7]);
        }
      }
    }
#pragma unroll
    for (int g = 0; g < NG; ++g)
#pragma unroll
      for (int v = 0; v < 8; ++v) acc[g][v] = 0;
    ++units_done;
  }
}

template <int LA, int LB, int S, int BD>
__global__ void __launch_bounds__(kWsThreads, 1) k_toeplitz_ws(TensorTiledArgs args) {
  using TS = TTShape<LB, S>;
  static_assert(BD == 1 || S == 1, "A slices or shifted copies of b, not both");
  extern __shared__ __align__(128) unsigned char sm[];
  __shared__ __align__(8) uint64_t built[2], mma_done[2], drained[2], comb_full, comb_free;
  __shared__ uint32_t s_tmem;
  __shared__ int s_domain, s_fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t n = 1u << args.logn, D = n / 8 - 1;
  const uint32_t kc = args.kc, nch = n / kc, ngrp = args.ngrp, awin = args.a_win;
  const uint32_t wrap = args.wrap, stage_bytes = args.stage_bytes, tcols = args.tmem_cols;
  const uint64_t units = args.units;
  constexpr uint32_t IDESC = idesc_bf16(128, TS::NB);
  // the CTA's steps: chunk c of its r-th unit is step r nch + c
  const uint64_t my_units = blockIdx.x < units ? (units - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const uint64_t steps = my_units * nch;

  if (warp == kWsMmaWarp) {
    tmem_alloc(&s_tmem, tcols);
    tmem_relinquish();
  }
  if (tid == 0) {
    for (int k = 0; k < 2; ++k) {
      mbar_init(&built[k], kWsBuilders);
      mbar_init(&mma_done[k], 1);
      mbar_init(&drained[k], kWsDrainers);
    }
    mbar_init(&comb_full, kWsDrainers / 2);
    mbar_init(&comb_free, kWsDrainers / 2);
    s_domain = 0;
    s_fail = 0;
  }
  fence_mbar_init();
  // padded rows of B (8-row groups past the S x LB digit rows) stay zero in
  // both stages; the builders' fence before their first arrival publishes
  // these stores to the MMAs
  if (TS::NG > S * LB && tid < kWsBuilders) {
    for (uint32_t x = tid; x < 2 * (kc / 8) * TS::NG * 8; x += kWsBuilders) {
      const uint32_t stg = x / ((kc / 8) * TS::NG * 8), ch = x % ((kc / 8) * TS::NG * 8);
      const uint32_t dp = ch / (TS::NG * 8), g = (ch / 8) % TS::NG, v = ch % 8;
      if (g >= (uint32_t)(S * LB))
        *reinterpret_cast<uint4*>(sm + stg * stage_bytes + args.bt_off + dp * TS::BT_PITCH + g * 128 + 16 * v) =
            make_uint4(0, 0, 0, 0);
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  const uint32_t buf_cols = tcols / 2;  // accumulator buffer k at column k buf_cols

  if (warp < kWsBuildWarps) {
    // ---------------------------------------------------------------- builders
    const int32_t ng = (int32_t)(n / 8);
    for (uint64_t st = 0; st < steps; ++st) {
      const uint32_t k = (uint32_t)(st & 1), use = (uint32_t)(st >> 1);
      if (st >= 2 && !mbar_wait(&mma_done[k], (use - 1) & 1u)) {
        s_fail = 1;
        break;
      }
      const uint64_t unit = blockIdx.x + (st / nch) * gridDim.x;
      const uint32_t ch = (uint32_t)(st % nch);
      const uint64_t row = unit / ngrp;
      const uint32_t grp = (uint32_t)(unit % ngrp);
      const WsRow wr = ws_row(args, row, n);
      const uint32_t q = args.tp[wr.j].q;
      const uint32_t* a = args.a + wr.off;
      const uint32_t* b = args.b + wr.off;
      const uint32_t b0 = grp * BD * S;  // the unit's first 1024-output block
      uint16_t* Xw = reinterpret_cast<uint16_t*>(sm + k * stage_bytes);
      unsigned char* Bt = sm + k * stage_bytes + args.bt_off;
      // ConvertPoly (a): digits of a~_{base + e}, e < awin, as in the tiled
      // kernel (groups of 8 lie wholly in a, in its extension, or outside)
      const int32_t base = (int32_t)(1024 * b0) - (int32_t)n + 8 + (int32_t)(kc * ch);
      for (uint32_t gi = tid; gi < awin / 8; gi += kWsBuilders) {
        const int32_t i0 = base + 8 * (int32_t)gi;
        uint4 p[LA];
        uint32_t flip = 0;
        if (i0 >= (int32_t)n || i0 < -(int32_t)n) {
#pragma unroll
          for (int s = 0; s < LA; ++s) p[s] = make_uint4(0, 0, 0, 0);
        } else {
          flip = i0 < 0 ? wrap : 0u;
          if (!digits8<LA>(a + (i0 < 0 ? i0 + (int32_t)n : i0), q, 8, p)) s_domain = 1;
        }
#pragma unroll
        for (int s = 0; s < LA; ++s)
          *reinterpret_cast<uint4*>(Xw + (size_t)s * awin + 8 * gi) =
              make_uint4(p[s].x ^ flip, p[s].y ^ flip, p[s].z ^ flip, p[s].w ^ flip);
      }
      // ConvertPoly (b): K-block d' = kc/8 ch + dl of shift sh is b~'s group
      // G = D - d' + 128 sh after group G - 1 (b~ over [-n, 2n))
      for (uint32_t it = tid; it < (kc / 8) * S; it += kWsBuilders) {
        const uint32_t dl = it / S, sh = it % S;
        const int32_t G = (int32_t)(D - (kc / 8 * ch + dl)) + 128 * (int32_t)sh, H = G - 1;
        const uint32_t gg = (uint32_t)(G >= ng ? G - ng : G);
        const uint32_t hh = (uint32_t)(H < 0 ? H + ng : H >= ng ? H - ng : H);
        const uint32_t fg = G >= ng ? wrap : 0u;
        const uint32_t fh = (H < 0 || H >= ng) ? wrap : 0u;
        uint4 pv[LB], ow[LB];
        digits8<LB>(b + 8 * hh, q, 8, pv);
        digits8<LB>(b + 8 * gg, q, 8, ow);
#pragma unroll
        for (int s2 = 0; s2 < LB; ++s2) {
          const uint32_t E[8] = {pv[s2].x ^ fh, pv[s2].y ^ fh, pv[s2].z ^ fh, pv[s2].w ^ fh,
                                 ow[s2].x ^ fg, ow[s2].y ^ fg, ow[s2].z ^ fg, ow[s2].w ^ fg};
          b_block_rows(E, Bt + dl * TS::BT_PITCH + (sh * LB + s2) * 128);
        }
      }
      fence_proxy_async();  // these generic stores before the MMAs' async-proxy reads
      mbar_arrive(&built[k]);
    }
  } else if (warp >= kWsDrainWarp0) {
    // ---------------------------------------------------------------- drainers
    const uint32_t r = (uint32_t)(tid - 32 * kWsDrainWarp0) & 127u;  // output row of the block = tensor-memory lane
    const uint32_t lane_base = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
    uint32_t* comb = reinterpret_cast<uint32_t*>(sm + 2 * stage_bytes);  // [BD S][128][8], set 1 -> set 0
    if (warp < kWsDrainWarp0 + 4)
      ws_drain_role<LA, LB, S, BD, 0>(args, steps, nch, ngrp, n, r, lane_base, buf_cols, mma_done, drained, &comb_full,
                                      &comb_free, comb, s_fail);
    else
      ws_drain_role<LA, LB, S, BD, 1>(args, steps, nch, ngrp, n, r, lane_base, buf_cols, mma_done, drained, &comb_full,
                                      &comb_free, comb, s_fail);
  } else {
    // ---------------------------------------------------------------- MMA issue
    if (lane == 0) {
    uint64_t issued = 0;
    constexpr uint64_t BSTEP = (2 * TS::BT_PITCH) >> 4;  // two K-blocks per MMA (K = 16)
    for (uint64_t st = 0; st < steps; ++st) {
      const uint32_t k = (uint32_t)(st & 1), use = (uint32_t)(st >> 1);
      if (!mbar_wait(&built[k], use & 1u) || (st >= 2 && !mbar_wait(&drained[k], (use - 1) & 1u))) {
        s_fail = 1;
        break;
      }
      tc_fence_after();
      const uint32_t xa0 = smem_u32(sm + k * stage_bytes);
      const uint64_t bd0 = smem_desc(xa0 + args.bt_off, TS::BT_PITCH, 128);
      // K steps outermost: consecutive MMAs go to different accumulators
      // (one chain per A slice and digit of a), so none waits for the one
      // before it
      uint64_t ad[BD * LA];
#pragma unroll
      for (int x = 0; x < BD * LA; ++x)
        ad[x] = smem_desc(xa0 + (uint32_t)((x % LA) * awin + 1024 * (x / LA)) * 2, 16, 128);
#pragma unroll 1
      for (uint32_t kk = 0; kk < kc / 16; ++kk) {
#pragma unroll
        for (int x = 0; x < BD * LA; ++x)
          tc_mma_f16(tmem + k * buf_cols + (uint32_t)(x * TS::NB), ad[x] + 2u * (uint64_t)kk, bd0 + BSTEP * (uint64_t)kk,
                     IDESC, kk > 0 ? 1u : 0u);
      }
      tc_commit(&mma_done[k]);
      issued = st + 1;
    }
    // every committed chain completes before tensor memory is released: the
    // last use of each buffer (already awaited by the drainers when all went well)
    for (uint32_t k = 0; k < 2; ++k) {
      const uint64_t uses = issued > k ? (issued - k + 1) / 2 : 0;
      if (uses && !mbar_wait(&mma_done[k], (uint32_t)((uses - 1) & 1u))) s_fail = 1;
    }
    }
    __syncwarp();  // the other lanes wait here for the issuing one
  }
  tc_fence_before();
  __syncthreads();
  if (tid == 0 && s_fail) atomicExch(args.err, 1);
  if (tid == 0 && s_domain) atomicOr(args.err, 2);  // reported as POLYMUL_EDOMAIN
  if (warp == kWsMmaWarp) {
    tc_fence_after();
    tmem_dealloc(tmem, tcols);
  }
}

// ---------------------------------------------------------------- host side

// shifted copies of b per A slice (as many digits on both sides), as the
// tiled kernels take them
static uint32_t ws_max_shifts(int la, int lb) {
  if (la != lb) return 1;
  return la <= 2 ? 4 : 2;
}

bool toeplitz_ws_config(int logn, int la, int lb, TiledCfg* cfg) {
  if (logn < 6 || logn > 14 || la < 1 || lb < 1 || la > 4 || lb > 4) return false;
  const uint32_t n = 1u << logn;
  auto nb_of = [&](uint32_t S) { return (8 * (uint32_t)lb * S + 15) / 16 * 16; };
  const uint32_t buf_cap = kWsTmemCap / 2;
  if ((uint32_t)la * nb_of(1) > buf_cap) return false;
  const uint32_t rblk = n >= 1024 ? n / 1024 : 1;
  uint32_t S = 1, bpg = 1;
  if (la == lb) {
    while (S * 2 <= rblk && S * 2 <= ws_max_shifts(la, lb) && (uint32_t)la * nb_of(S * 2) <= buf_cap) S *= 2;
  } else {
    while (bpg * 2 <= rblk && bpg * 2 <= 4 && bpg * 2 * (uint32_t)la * nb_of(1) <= buf_cap) bpg *= 2;
  }
  const uint32_t nb = nb_of(S), pitch = nb / 8 * 128 + 16;
  for (uint32_t kc = n < 1024 ? n : 1024; kc >= 64 && kc <= n; kc /= 2) {
    const uint32_t a_win = 1024 * bpg + kc;
    const uint32_t bt_off = ((uint32_t)la * a_win * 2 + 127) / 128 * 128;
    const uint32_t stage = (bt_off + kc / 8 * pitch + 127) / 128 * 128;
    // the drainer sets' hand-off of reduced sums when they split a's digits
    const uint32_t comb = la >= 2 ? bpg * S * 128 * 8 * 4 : 0;
    if (2 * stage + comb > (uint32_t)kWsSmemCap) continue;
    cfg->bpg = bpg;
    cfg->shifts = S;
    cfg->nb = nb;
    cfg->b_pitch = pitch;
    cfg->ngrp = rblk / (bpg * S);
    cfg->kc = kc;
    cfg->a_win = a_win;
    cfg->bt_off = bt_off;
    cfg->stage_bytes = stage;
    cfg->smem = (int)(2 * stage + comb);
    uint32_t cols = 32;
    while (cols < bpg * (uint32_t)la * nb) cols *= 2;
    cfg->tmem_cols = 2 * cols;
    return true;
  }
  return false;
}

template <int LA, int LB, int S, int BD>
static void ws_info(const TiledCfg& cfg, KernelInfo* ki) {
  ki->fn = (const void*)k_toeplitz_ws<LA, LB, S, BD>;
  ki->block = kWsThreads;
  ki->smem = cfg.smem;
  ki->team = kWsThreads;
  ki->units_per_cta = 1;
  ki->tmem_cols = (int)cfg.tmem_cols;
  ki->tiled = 1;
  ki->drain = 1;
  ki->ws = 1;
  ki->wb = 8;
  ki->digits = LB;
}

bool lookup_toeplitz_ws(int logn, int la, int lb, KernelInfo* ki) {
  TiledCfg cfg;
  if (!toeplitz_ws_config(logn, la, lb, &cfg)) return false;
  const int S = (int)cfg.shifts, bd = (int)cfg.bpg;
#define PM_WS(A, B, SH, BPG)                        \
  if (la == A && lb == B && S == SH && bd == BPG) { \
    ws_info<A, B, SH, BPG>(cfg, ki);                \
    return true;                                    \
  }
  PM_WS(1, 1, 1, 1) PM_WS(1, 1, 2, 1) PM_WS(1, 1, 4, 1)
  PM_WS(2, 2, 1, 1) PM_WS(2, 2, 2, 1) PM_WS(2, 2, 4, 1)
  PM_WS(3, 3, 1, 1) PM_WS(3, 3, 2, 1)
  PM_WS(4, 4, 1, 1) PM_WS(4, 4, 2, 1)
  // a single-digit operand on the A side (ternary b)
  PM_WS(1, 2, 1, 1) PM_WS(1, 2, 1, 2) PM_WS(1, 2, 1, 4)
  PM_WS(1, 3, 1, 1) PM_WS(1, 3, 1, 2) PM_WS(1, 3, 1, 4)
  PM_WS(1, 4, 1, 1) PM_WS(1, 4, 1, 2) PM_WS(1, 4, 1, 4)
#undef PM_WS
  return false;
}

}  // namespace pm

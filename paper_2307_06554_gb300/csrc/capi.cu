// C-ABI entry points of libpolymul (declared in include/polymul.h).
//
// polymul_create plays the role of GenConfig/ExtractModuli/ExtractDimensions
// of the paper's Algorithm 1: it fixes the path, computes every per-prime
// constant and table once and uploads them; polymul_batch then only launches
// kernels (ConvertPoly/TPUMul/ConvertMatrix happen inside them).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/polymul.h"
#include "host_math.h"
#include "ntt_tables.h"
#include "kernels.h"
#include "trace.h"
#include "plan.h"
#include "stream_order.h"
#include "polymul_types.h"
#include "toeplitz_rns.h"
#include "toeplitz_tiled.h"
#include "toeplitz_u64.h"

using namespace pm;

// ---------------------------------------------------------------- errors
namespace pm {
static thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(POLYMUL_ECUDA, "%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
}

void clear_error() { g_err.clear(); }
}  // namespace pm

#define PM_CUDA(call)                                   \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return pm::cuda_fail(e_, #call); \
  } while (0)

extern "C" const char* polymul_last_error(void) { return g_err.c_str(); }

// ---------------------------------------------------------------- tables
namespace {

// Tables for the NTT primes: the plan's moduli, or (auxiliary-prime mode)
// the single auxiliary prime.
template <typename W>
int upload_ntt_tables(polymul_plan* p) {
  const std::vector<uint64_t> primes = p->aux_prime ? std::vector<uint64_t>{p->aux_prime} : p->q;
  const uint32_t np = (uint32_t)primes.size();
  std::vector<W> all_f, all_i, f, i;
  std::vector<PrimeConst<W>> pcs(np);
  all_f.reserve(2 * (size_t)p->n * np);
  all_i.reserve(2 * (size_t)p->n * np);
  for (uint32_t j = 0; j < np; ++j) {
    build_ntt_tables<W>(primes[j], p->n, f, i, pcs[j], p->cyclic);
    all_f.insert(all_f.end(), f.begin(), f.end());
    all_i.insert(all_i.end(), i.begin(), i.end());
  }
  const size_t tb = all_f.size() * sizeof(W);
  PM_CUDA(cudaMalloc(&p->d_twf, tb));
  PM_CUDA(cudaMalloc(&p->d_twi, tb));
  PM_CUDA(cudaMalloc(&p->d_pc, pcs.size() * sizeof(PrimeConst<W>)));
  PM_CUDA(cudaMemcpy(p->d_twf, all_f.data(), tb, cudaMemcpyHostToDevice));
  PM_CUDA(cudaMemcpy(p->d_twi, all_i.data(), tb, cudaMemcpyHostToDevice));
  PM_CUDA(cudaMemcpy(p->d_pc, pcs.data(), pcs.size() * sizeof(PrimeConst<W>), cudaMemcpyHostToDevice));
  if (p->aux_prime) {
    std::vector<W> qs(p->q.begin(), p->q.end());
    PM_CUDA(cudaMalloc(&p->d_outer, qs.size() * sizeof(W)));
    PM_CUDA(cudaMemcpy(p->d_outer, qs.data(), qs.size() * sizeof(W), cudaMemcpyHostToDevice));
  }
  return POLYMUL_OK;
}

// Auxiliary NTT prime for moduli without a 2n-th root of unity: the largest
// prime p < 2^31 with 2n | p - 1; usable when p > 2 n floor(qmax/2)^2 (the
// centred integer product then fits in (-p/2, p/2)).  0 if none.
uint64_t find_aux_prime(uint32_t n, uint64_t qmax) {
  const pm::host::u128 half = qmax / 2;
  const pm::host::u128 bound = 2 * (pm::host::u128)n * half * half;
  const uint64_t step = 2ull * n;
  for (uint64_t kk = ((1ull << 31) - 2) / step; kk > 0; --kk) {
    const uint64_t cand = kk * step + 1;
    if ((pm::host::u128)cand <= bound) return 0;
    if (pm::host::is_prime(cand)) return cand;
  }
  return 0;
}

// Tensor path shape: digit width w with n 2^(2w-2) <= 2^24 (exact fp32
// partial sums), w <= 8 (exact bf16 digits); L balanced digits cover the
// centred range |x| <= q/2.
bool tensor_shape(uint32_t n, uint64_t qmax, int* wb, int* L) {
  const int logn = __builtin_ctz(n);
  int w = (24 - logn) / 2 + 1;
  if (w > 8) w = 8;
  if (w < 2) return false;
  for (int l = 1; l <= 8; ++l) {
    // digits lie in [-2^(w-1), 2^(w-1) - 1], so l of them reach
    // (2^(w-1) - 1) (2^(wl) - 1) / (2^w - 1) on the positive side; the
    // centred residues reach floor(q/2) there (and less below zero)
    const pm::host::u128 cap = ((((pm::host::u128)1 << (w - 1)) - 1) * (((pm::host::u128)1 << (w * l)) - 1)) /
                               (((pm::host::u128)1 << w) - 1);
    if (cap >= qmax / 2) {
      *wb = w;
      *L = l;
      return true;
    }
  }
  return false;
}

// digits of the operand on the MMA's A side: one for a ternary b (which
// takes that side), else L
int tensor_la(const polymul_plan* p) { return p->ternary_b ? 1 : p->digits; }

// Balanced 8-bit digits covering the centred residues of moduli up to qmax:
// the drained tiled kernel's shape at any degree (its fp32 sums run over
// chunks of at most 1024 K, 1024 2^14 = 2^24)
int drain_digits(uint64_t qmax) {
  for (int l = 1; l <= 4; ++l)
    if ((uint64_t)127 * ((1ull << (8 * l)) - 1) / 255 >= qmax / 2) return l;
  return 0;
}

// digit width and the two operands' digit counts of the tensor digit kernel
// k in plan p (a drained kernel fixes its own)
struct DigitShape {
  int wb, la, lb;
};
DigitShape digit_shape(const polymul_plan* p, const KernelInfo& k) {
  if (k.wb) return DigitShape{k.wb, p->ternary_b ? 1 : k.digits, k.digits};
  return DigitShape{p->digit_bits, tensor_la(p), p->digits};
}

bool tiled_config_of(const KernelInfo& k, int logn, int la, int lb, TiledCfg* cfg) {
  if (k.u64) return toeplitz_u64_config(logn, lb, cfg);
  if (k.ws) return toeplitz_ws_config(logn, la, lb, cfg);
  return k.drain ? toeplitz_tiled_config_drain(logn, la, lb, cfg) : toeplitz_tiled_config(logn, la, lb, cfg);
}

// tensor kernel code reported by polymul_plan_info and polymul_tensor_shape
uint32_t tensor_kernel_code(const KernelInfo& k) {
  return k.rns ? 3u : k.u64 ? 6u : k.ws ? 5u : k.drain ? 4u : k.tiled ? 2u : 1u;
}

// The tensor path's kernels for degree n and moduli up to qmax, the default
// first: the digit kernels for moduli below 2^31 (the whole-product kernel
// at n = 1024, 2048 and the tiled one, the tiled first where it serves two
// blocks from one A slice: measured 101 vs 165 us for two digits at
// n = 2048, 174 vs 330 us for three), then the residue-number-system kernel
// (any q < 2^62 with a base of at most 32 moduli).  Host only.
struct TensorChoice {
  int wb = 0, L = 0;                  // digit width and count of the digit kernels
  std::vector<uint32_t> rns_moduli;   // the RNS base, when that kernel is a candidate
  std::vector<KernelInfo> kernels;    // [0] the default
};
bool choose_tensor(uint32_t n, uint64_t qmax, uint32_t elem, bool ternary_b, TensorChoice* tc) {
  const int logn = __builtin_ctz(n);
  tc->kernels.clear();
  tc->rns_moduli.clear();
  tc->wb = tc->L = 0;
  KernelInfo kwhole, ktiled, krns;
  bool whole = false, tiled = false;
  if (elem == 4 && qmax < (1ull << 31) && tensor_shape(n, qmax, &tc->wb, &tc->L)) {
    tiled = lookup_toeplitz_tiled(logn, ternary_b ? 1 : tc->L, tc->L, &ktiled);
    whole = !ternary_b && lookup_toeplitz(logn, tc->wb, tc->L, tc->L, &kwhole);
  }
  if (whole && tiled) {
    TiledCfg cfg;
    const bool shifted = toeplitz_tiled_config(logn, tc->L, tc->L, &cfg) && cfg.shifts > 1;
    tc->kernels.push_back(shifted ? ktiled : kwhole);
    tc->kernels.push_back(shifted ? kwhole : ktiled);
  } else if (whole) {
    tc->kernels.push_back(kwhole);
  } else if (tiled) {
    tc->kernels.push_back(ktiled);
  }
  // where exact fp32 sums over the whole of K force digits narrower than 8
  // bits (n >= 2048), the drained tiled kernel keeps 8-bit digits; first
  // where that saves digits (measured with 30-bit primes: 4 x 4 digits
  // 1318 us vs 5 x 5 2079 us at n = 4096, 335 vs 539 us at n = 2048; ternary
  // b, 1 x 4 vs 1 x 5: 439 vs 445 us at n = 4096, 109 vs 129 us at 2048)
  KernelInfo kdrain;
  const int l8 = elem == 4 && qmax < (1ull << 31) ? drain_digits(qmax) : 0;  // 0: no drained kernel
  if (l8 && tc->wb > 0 && tc->wb < 8 && lookup_toeplitz_tiled_drain(logn, ternary_b ? 1 : l8, l8, &kdrain)) {
    if (l8 < tc->L || tc->kernels.empty())
      tc->kernels.insert(tc->kernels.begin(), kdrain);
    else
      tc->kernels.push_back(kdrain);
  }
  // the drained kernel as a warp-specialised pipeline (one CTA per SM: the
  // operand builds and the drains overlap the MMAs), at every degree
  KernelInfo kws;
  if (l8 && lookup_toeplitz_ws(logn, ternary_b ? 1 : l8, l8, &kws)) tc->kernels.push_back(kws);
  std::vector<uint32_t> mods;
  if (rns_choose_base(n, qmax, &mods) && lookup_toeplitz_rns(logn, (uint32_t)mods.size(), elem, &krns)) {
    tc->kernels.push_back(krns);
    tc->rns_moduli = mods;
  }
  // 64-bit words: 5 .. 8 drained 8-bit digits per operand at n = 2^10 ..
  // 2^16; first up to n = 2048 and where the RNS kernel has no base (above
  // n = 4096 for 59-bit moduli), after it otherwise (measured with two
  // 59-bit primes: 41 vs 94 us for 64 products at n = 1024, 405 vs 357 us
  // at 4096)
  KernelInfo ku64;
  const int l64 = elem == 8 && !ternary_b ? std::max(5, u64_digits(qmax)) : 0;
  if (l64 && l64 <= 8 && lookup_toeplitz_u64(logn, l64, &ku64)) {
    if (logn <= 11 || tc->kernels.empty())
      tc->kernels.insert(tc->kernels.begin(), ku64);
    else
      tc->kernels.push_back(ku64);
  }
  return !tc->kernels.empty();
}

// the small-moduli base of the RNS tensor kernel and its per-prime constants
int upload_rns_tables(polymul_plan* p, const std::vector<uint32_t>& moduli) {
  if (p->d_rns_base) return POLYMUL_OK;
  RnsBase base;
  std::vector<RnsPrime> per;
  rns_tables(moduli, p->q, &base, &per);
  p->rns_r = base.r;
  PM_CUDA(cudaMalloc(&p->d_rns_base, sizeof base));
  PM_CUDA(cudaMemcpy(p->d_rns_base, &base, sizeof base, cudaMemcpyHostToDevice));
  PM_CUDA(cudaMalloc(&p->d_rns_primes, per.size() * sizeof(RnsPrime)));
  PM_CUDA(cudaMemcpy(p->d_rns_primes, per.data(), per.size() * sizeof(RnsPrime), cudaMemcpyHostToDevice));
  return POLYMUL_OK;
}

// per-prime constants of the 64-bit-word digit kernel
int upload_tensor_tables64(polymul_plan* p) {
  if (p->elem != 8 || p->d_tp64) return POLYMUL_OK;
  std::vector<TensorPrime64> tp(p->k);
  for (uint32_t j = 0; j < p->k; ++j) {
    memset(&tp[j], 0, sizeof tp[j]);
    const uint64_t q = p->q[j];
    tp[j].q = q;
    tp[j].bias = ((1ull << 28) + q - 1) / q * q;
    for (int e = 0; e < 15; ++e) {
      tp[j].pw[e] = pm::host::powmod(2, 8ull * e, q);
      tp[j].pwp[e] = (uint64_t)(((pm::host::u128)tp[j].pw[e] << 64) / q);
    }
  }
  PM_CUDA(cudaMalloc(&p->d_tp64, tp.size() * sizeof(TensorPrime64)));
  PM_CUDA(cudaMemcpy(p->d_tp64, tp.data(), tp.size() * sizeof(TensorPrime64), cudaMemcpyHostToDevice));
  return POLYMUL_OK;
}

int upload_tensor_tables(polymul_plan* p) {
  if (p->elem == 8) return upload_tensor_tables64(p);
  if (p->elem != 4 || p->d_tpc) return POLYMUL_OK;  // digit kernels only (32-bit words); once
  auto upload = [&](int wb, void** dst) -> int {
    std::vector<TensorPrime> tp(p->k);
    for (uint32_t j = 0; j < p->k; ++j) {
      memset(&tp[j], 0, sizeof tp[j]);
      const uint64_t q = p->q[j];
      tp[j].q = (uint32_t)q;
      for (int e = 0; e < 15; ++e) tp[j].pw[e] = (uint32_t)pm::host::powmod(2, (uint64_t)wb * e, q);
      tp[j].mu = (uint64_t)(((pm::host::u128)1 << 64) / q);
      tp[j].bias = ((1ull << 60) + q - 1) / q * q;
    }
    PM_CUDA(cudaMalloc(dst, tp.size() * sizeof(TensorPrime)));
    PM_CUDA(cudaMemcpy(*dst, tp.data(), tp.size() * sizeof(TensorPrime), cudaMemcpyHostToDevice));
    return POLYMUL_OK;
  };
  int r = upload(p->digit_bits, &p->d_tpc);
  if (r == POLYMUL_OK && p->digit_bits > 0 && p->digit_bits < 8) r = upload(8, &p->d_tpc8);
  return r;
}

bool lookup_ntt(uint32_t elem, int logn, int mode, KernelInfo* ki) {
  // n = 2^14, 32-bit words: one 512-thread CTA per product (32 coefficients
  // per thread) beats the two-CTA cluster (measured 101.9 vs 160.8 us for
  // 512 products); the cluster kernel stays an autotuner candidate
  if (elem == 4 && logn == 14 && lookup_ntt_u32_rb5(logn, mode, ki)) return true;
  if (logn >= 14) {
    // beyond one CTA: one product per thread-block cluster, the form with
    // CTA-local exchanges (measured on GB300 against the first form: 64-bit
    // words with both operands in registers 1.38-1.49x faster at 2^14 ..
    // 2^16; 32-bit words one operand at a time 1.2x at 2^15, 2^16); the
    // unreduced mode takes the Harvey-bound kernels, whose bounds hold for
    // its moduli too
    if (lookup_ntt_cluster2(elem, logn, mode == 2 ? 1 : mode, elem == 4, ki)) return true;
    return lookup_ntt_cluster(elem, logn, mode, ki) || (mode == 2 && lookup_ntt_cluster(elem, logn, 1, ki));
  }
  if (elem == 4) {
    if (mode == 0) return lookup_ntt_u32_m0(logn, ki);
    if (mode == 1) return lookup_ntt_u32_m1(logn, ki);
    return lookup_ntt_u32_m2(logn, ki);
  }
  if (mode == 1) return lookup_ntt_u64_m1(logn, ki);
  if (mode == 2) return lookup_ntt_u64_m2(logn, ki);
  return false;
}

}  // namespace

// The occupancy query reports one CTA per SM for kernels that allocate
// tensor memory; co-residency is in fact limited by shared memory,
// registers, threads and the 512 tensor-memory columns, so count those.
int pm::tmem_kernel_per_sm(const KernelInfo& ki, int device, int* per_sm) {
  cudaFuncAttributes fa;
  PM_CUDA(cudaFuncGetAttributes(&fa, ki.fn));
  int smem_sm = 0, resv = 0;
  PM_CUDA(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, device));
  PM_CUDA(cudaDeviceGetAttribute(&resv, cudaDevAttrReservedSharedMemoryPerBlock, device));
  const int regs = (fa.numRegs + 7) / 8 * 8;
  int n = smem_sm / (ki.smem + (int)fa.sharedSizeBytes + resv);
  n = std::min(n, 65536 / std::max(1, regs * ki.block));
  n = std::min(n, 2048 / ki.block);
  n = std::min(n, 512 / ki.tmem_cols);  // never wait for tensor memory
  *per_sm = n;
  return POLYMUL_OK;
}

namespace {

int configure_launch(polymul_plan* p) {
  PM_CUDA(cudaGetDevice(&p->device));
  PM_CUDA(cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device));
  if (p->ki.smem > 48 * 1024)
    PM_CUDA(cudaFuncSetAttribute(p->ki.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, p->ki.smem));
  PM_CUDA(cudaFuncSetAttribute(p->ki.fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
  int per_sm = 0;
  if (p->ki.cluster > 0) {
    // resident clusters: the persistent grid is that many clusters
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof cfg);
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = p->ki.cluster;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.gridDim = dim3(p->ki.cluster * p->num_sms);
    cfg.blockDim = dim3(p->ki.block);
    cfg.dynamicSmemBytes = p->ki.smem;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    PM_CUDA(cudaOccupancyMaxActiveClusters(&clusters, p->ki.fn, &cfg));
    if (clusters < 1) return fail(POLYMUL_ENOTSUP, "no %d-CTA cluster fits on the device", p->ki.cluster);
    p->grid_cap = clusters * p->ki.cluster;
    return POLYMUL_OK;
  }
  if (p->ki.tmem_cols > 0) {
    const int r = tmem_kernel_per_sm(p->ki, p->device, &per_sm);
    if (r != POLYMUL_OK) return r;
  } else {
    PM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, p->ki.fn, p->ki.block, p->ki.smem));
  }
  if (per_sm < 1) return fail(POLYMUL_ENOTSUP, "kernel does not fit on an SM (block %d, smem %d)", p->ki.block, p->ki.smem);
  p->grid_cap = per_sm * p->num_sms;
  return POLYMUL_OK;
}

}  // namespace

// ---------------------------------------------------------------- create
extern "C" int polymul_create(uint32_t n, const uint64_t* q_list, uint32_t k, const polymul_opts* opts,
                              polymul_plan** out) {
  clear_error();
  TraceRange trace_("polymul_create");
  if (!out) return fail(POLYMUL_EINVAL, "out is NULL");
  if (n < 16 || n > 65536 || (n & (n - 1))) return fail(POLYMUL_EINVAL, "n=%u must be a power of two in [16, 65536]", n);
  if (k == 0 || !q_list) return fail(POLYMUL_EINVAL, "need k >= 1 moduli");
  for (uint32_t j = 0; j < k; ++j) {
    if (q_list[j] < 2 || q_list[j] >= (1ull << 62))
      return fail(POLYMUL_EINVAL, "q[%u]=%llu outside [2, 2^62)", j, (unsigned long long)q_list[j]);
    for (uint32_t i = 0; i < j; ++i)
      if (q_list[i] == q_list[j]) return fail(POLYMUL_EINVAL, "duplicate modulus %llu", (unsigned long long)q_list[j]);
  }
  const uint32_t path = opts ? opts->path : POLYMUL_PATH_AUTO;
  if (path > POLYMUL_PATH_TENSOR) return fail(POLYMUL_EINVAL, "unknown path %u", path);

  polymul_plan* p = new polymul_plan();
  p->n = n;
  p->logn = __builtin_ctz(n);
  p->k = k;
  p->q.assign(q_list, q_list + k);
  p->flags = opts ? opts->flags : 0;
  p->cyclic = (p->flags & POLYMUL_FLAG_CYCLIC) != 0;
  p->ternary_b = (p->flags & POLYMUL_FLAG_TERNARY_B) != 0;
  uint64_t qmax = *std::max_element(p->q.begin(), p->q.end());
  p->elem = qmax < (1ull << 32) ? 4 : 8;

  // direct NTT: every modulus prime with 2n | q-1 (n | q-1 for the cyclic
  // ring) and within the word bounds
  const uint64_t root_order = p->cyclic ? n : 2ull * n;
  bool ntt_ok = true;
  for (uint64_t q : p->q) {
    if (!pm::host::is_prime(q) || (q - 1) % root_order != 0) ntt_ok = false;
    if (p->elem == 4 && q >= (1ull << 31)) ntt_ok = false;
  }
  p->mode = ntt_mode(qmax, p->logn, p->elem);
  if (p->mode < 0) ntt_ok = false;
  if (ntt_ok && !lookup_ntt(p->elem, (int)p->logn, p->mode, &p->ki)) ntt_ok = false;

  // auxiliary-prime NTT: one 31-bit prime carries the exact integer product
  bool aux_ok = false;
  if (!ntt_ok && p->elem == 4 && qmax < (1ull << 31)) {
    const uint64_t ap = find_aux_prime(n, qmax);
    KernelInfo aki;
    if (ap && ap > (1ull << 30) && lookup_ntt_u32_aux((int)p->logn, &aki)) {
      aux_ok = true;
      p->aux_candidate = ap;
      p->aki = aki;
    }
  }

  // tensor path: moduli below 2^31, n = 2^6 .. 2^14.  The whole-product
  // kernel where it is instantiated (n = 1024, 2048), the tiled kernel
  // otherwise, and as a second candidate beside the whole-product one
  TensorChoice tch;
  const bool tensor_ok = choose_tensor(n, qmax, p->elem, p->ternary_b, &tch);
  p->digit_bits = tch.wb;
  p->digits = tch.L;
  if (tensor_ok) p->tki = tch.kernels[0];
  auto add_tensor_candidates = [&](auto&& add) -> int {
    int r = upload_tensor_tables(p);
    for (const KernelInfo& k : tch.kernels) {
      if (r == POLYMUL_OK && k.rns) r = upload_rns_tables(p, tch.rns_moduli);
      if (r == POLYMUL_OK) r = add(POLYMUL_PATH_TENSOR, k);
    }
    return r;
  };

  int rc = POLYMUL_OK;
  // NTT batch kernels take a programmatic dependent launch (measured on
  // back-to-back batches: n = 1024, 4096 products 29.9 -> 27.6 us; n = 256,
  // 64 products 8.3 -> 5.7 us); cluster and tensor kernels take plain launches
  auto add_candidate = [&](uint32_t cpath, const KernelInfo& ki) -> int {
    p->ki = ki;
    p->path = cpath;
    int r = configure_launch(p);
    const uint32_t lf = cpath == POLYMUL_PATH_NTT && ki.cluster == 0 ? kLaunchPdl : 0u;
    if (r == POLYMUL_OK) p->cands.push_back(PlanCandidate{cpath, ki, p->grid_cap, lf});
    return r;
  };
  if ((path == POLYMUL_PATH_NTT || path == POLYMUL_PATH_AUTO) && !ntt_ok && aux_ok) {
    p->aux_prime = p->aux_candidate;
    p->mode = 0;
    rc = upload_ntt_tables<uint32_t>(p);
    if (rc == POLYMUL_OK) rc = add_candidate(POLYMUL_PATH_NTT, p->aki);
    KernelInfo v;
    if (rc == POLYMUL_OK && lookup_ntt_u32_aux_rb2((int)p->logn, &v)) rc = add_candidate(POLYMUL_PATH_NTT, v);
  } else if (path == POLYMUL_PATH_TENSOR || (path == POLYMUL_PATH_AUTO && !ntt_ok && tensor_ok)) {
    if (!tensor_ok) {
      rc = fail(POLYMUL_ENOTSUP, "tensor path not available for n=%u and these moduli", n);
    } else {
      rc = add_tensor_candidates(add_candidate);
    }
  } else if (!ntt_ok) {
    rc = fail(POLYMUL_ENOTSUP, "no NTT route for these moduli at n=%u (need prime q = 1 mod %s, q < 2^31 for 32-bit words)",
              n, p->cyclic ? "n" : "2n");
  } else {
    // the default kernel first, then the candidates the autotuner may prefer
    rc = p->elem == 4 ? upload_ntt_tables<uint32_t>(p) : upload_ntt_tables<uint64_t>(p);
    KernelInfo v;
    if (rc == POLYMUL_OK) rc = add_candidate(POLYMUL_PATH_NTT, p->ki);
    if (rc == POLYMUL_OK && p->elem == 4 && lookup_ntt_u32_rb5((int)p->logn, p->mode, &v) && v.fn != p->cands[0].ki.fn)
      rc = add_candidate(POLYMUL_PATH_NTT, v);
    if (rc == POLYMUL_OK && p->elem == 4 && p->logn == 14 &&
        (lookup_ntt_cluster(4, 14, p->mode, &v) || lookup_ntt_cluster(4, 14, 1, &v)))
      rc = add_candidate(POLYMUL_PATH_NTT, v);
    // the cluster kernels not already the default: the second form's other
    // operand scheme, and the first form
    if (p->logn >= 14) {
      const int cm = p->mode == 2 ? 1 : p->mode;
      for (int seq = 0; seq < 2; ++seq)
        if (rc == POLYMUL_OK && lookup_ntt_cluster2(p->elem, (int)p->logn, cm, seq != 0, &v) &&
            v.fn != p->cands[0].ki.fn)
          rc = add_candidate(POLYMUL_PATH_NTT, v);
      if (rc == POLYMUL_OK && p->logn >= 15 &&
          (lookup_ntt_cluster(p->elem, (int)p->logn, p->mode, &v) || lookup_ntt_cluster(p->elem, (int)p->logn, 1, &v)))
        rc = add_candidate(POLYMUL_PATH_NTT, v);
    }
    if (rc == POLYMUL_OK && p->elem == 4 && lookup_ntt_u32_rb3((int)p->logn, p->mode, &v)) rc = add_candidate(POLYMUL_PATH_NTT, v);
    if (rc == POLYMUL_OK && p->logn < 14 && lookup_ntt_alt(p->elem, (int)p->logn, p->mode, &v)) rc = add_candidate(POLYMUL_PATH_NTT, v);
    if (rc == POLYMUL_OK && path == POLYMUL_PATH_AUTO && tensor_ok) rc = add_tensor_candidates(add_candidate);
  }
  if (rc == POLYMUL_OK) apply_candidate(p, 0);
  if (rc == POLYMUL_OK) {
    // work counters for the three launch slots (device entry, two host-entry streams)
    if (cudaMalloc(&p->d_ctr, 2 * kCounterSlots * sizeof(unsigned long long)) != cudaSuccess ||
        cudaMemset(p->d_ctr, 0, 2 * kCounterSlots * sizeof(unsigned long long)) != cudaSuccess ||
        cudaMalloc(&p->d_err, sizeof(int)) != cudaSuccess || cudaMemset(p->d_err, 0, sizeof(int)) != cudaSuccess)
      rc = fail(POLYMUL_ENOMEM, "counter allocation failed");
  }
  if (rc != POLYMUL_OK) {
    std::string keep = g_err;
    polymul_destroy(p);
    g_err = keep;
    return rc;
  }
  if (p->flags & POLYMUL_FLAG_TUNE) {
    const uint64_t tb = opts && opts->tune_batch ? opts->tune_batch : 1024;
    rc = polymul_tune(p, tb, nullptr);
    if (rc != POLYMUL_OK) {
      std::string keep = g_err;
      polymul_destroy(p);
      g_err = keep;
      return rc;
    }
  }
  *out = p;
  return POLYMUL_OK;
}

extern "C" void polymul_destroy(polymul_plan* p) {
  if (!p) return;
  cudaFree(p->d_twf);
  cudaFree(p->d_twi);
  cudaFree(p->d_pc);
  cudaFree(p->d_tpc);
  cudaFree(p->d_tpc8);
  cudaFree(p->d_tp64);
  cudaFree(p->d_rns_base);
  cudaFree(p->d_rns_primes);
  for (int s = 0; s < kCounterSlots; ++s) cudaFree(p->d_rns_scr[s]);
  cudaFree(p->d_sh);
  cudaFree(p->d_flag);
  cudaFree(p->d_ctr);
  cudaFree(p->d_err);
  cudaFree(p->d_q);
  cudaFree(p->d_outer);
  for (int s = 0; s < kHostSlots; ++s) {
    cudaFree(p->d_hslot[s]);
    for (int g = 0; g < 3; ++g)
      if (p->hev[g][s]) cudaEventDestroy(p->hev[g][s]);
  }
  for (int g = 0; g < 3; ++g) {
    if (p->hs[g]) cudaStreamDestroy(p->hs[g]);
  }
  if (p->ev_entry) cudaEventDestroy(p->ev_entry);
  delete p;
}

extern "C" int polymul_plan_info_get(const polymul_plan* p, polymul_plan_info* info) {
  clear_error();
  if (!p || !info) return fail(POLYMUL_EINVAL, "null argument");
  memset(info, 0, sizeof *info);
  info->n = p->n;
  info->k = p->k;
  info->elem_bytes = p->elem;
  info->path = p->path;
  info->aux_primes = p->aux_prime ? 1u : 0u;
  info->block = (uint32_t)p->ki.block;
  info->grid = (uint32_t)p->grid_cap;
  info->smem_bytes = (uint32_t)p->ki.smem;
  info->ctas_per_sm = (uint32_t)(p->num_sms ? p->grid_cap / p->num_sms : 0);
  const DigitShape ds = digit_shape(p, p->ki);
  info->digit_bits = p->path == POLYMUL_PATH_TENSOR ? (uint32_t)ds.wb : 0;
  info->digits = p->path == POLYMUL_PATH_TENSOR ? (uint32_t)ds.lb : 0;
  info->radix_bits = p->path == POLYMUL_PATH_NTT ? (uint32_t)p->ki.rb : 0;
  info->candidates = (uint32_t)p->cands.size();
  info->tuned = p->tuned ? 1u : 0u;
  info->tuned_batch = (uint32_t)p->tuned_batch;
  info->launch_flags = p->launch_flags;
  if ((p->launch_flags & kLaunchPdl) && (p->flags & POLYMUL_FLAG_OVERLAP)) info->launch_flags |= 4u;
  info->ntt_mode = p->path == POLYMUL_PATH_NTT ? (uint32_t)p->ki.mode : 0u;
  info->regs = p->path == POLYMUL_PATH_NTT ? (uint32_t)p->ki.regs : 0u;
  info->cyclic = p->cyclic ? 1u : 0u;
  info->tensor_groups = 0;
  info->rns_moduli = p->path == POLYMUL_PATH_TENSOR && p->ki.rns ? p->rns_r : 0;
  info->exchange_pad = p->path == POLYMUL_PATH_NTT ? (uint32_t)p->ki.pad : 0u;
  info->one_operand = p->path == POLYMUL_PATH_NTT ? (uint32_t)p->ki.seq : 0u;
  info->tensor_kernel = p->path != POLYMUL_PATH_TENSOR ? 0u : tensor_kernel_code(p->ki);
  info->host_direct = (uint32_t)std::min<uint64_t>(p->host_direct, 0xffffffffu);
  cudaFuncAttributes fa;
  if (p->ki.fn && cudaFuncGetAttributes(&fa, p->ki.fn) == cudaSuccess) {
    info->kernel_regs = (uint32_t)fa.numRegs;
    info->kernel_max_block = (uint32_t)fa.maxThreadsPerBlock;
  }
  if (p->path == POLYMUL_PATH_TENSOR && p->ki.rns) {
    RnsCfg rc;
    if (rns_config((int)p->logn, p->rns_r, &rc)) info->tensor_groups = rc.ngrp;
  }
  if (p->path == POLYMUL_PATH_TENSOR && p->ki.tiled) {
    TiledCfg tc;
    if (tiled_config_of(p->ki, (int)p->logn, ds.la, ds.lb, &tc)) info->tensor_groups = tc.ngrp;
  }
  return POLYMUL_OK;
}

extern "C" int polymul_tensor_shape(uint32_t n, uint64_t qmax, uint32_t flags, polymul_tensor_shape_info* info) {
  clear_error();
  if (!info) return fail(POLYMUL_EINVAL, "info is NULL");
  if (n < 16 || n > 65536 || (n & (n - 1))) return fail(POLYMUL_EINVAL, "n=%u must be a power of two in [16, 65536]", n);
  if (qmax < 2 || qmax >= (1ull << 62)) return fail(POLYMUL_EINVAL, "qmax outside [2, 2^62)");
  const bool ternary = (flags & POLYMUL_FLAG_TERNARY_B) != 0;
  const uint32_t elem = qmax < (1ull << 32) ? 4 : 8;
  TensorChoice tch;
  if (!choose_tensor(n, qmax, elem, ternary, &tch))
    return fail(POLYMUL_ENOTSUP, "tensor path not available for n=%u and moduli up to %llu", n, (unsigned long long)qmax);
  memset(info, 0, sizeof *info);
  const KernelInfo& k = tch.kernels[0];
  const int logn = __builtin_ctz(n);
  info->candidates = (uint32_t)tch.kernels.size();
  info->smem_bytes = (uint32_t)k.smem;
  info->tmem_cols = (uint32_t)k.tmem_cols;
  if (k.rns) {
    RnsCfg rc;
    rns_config(logn, (uint32_t)tch.rns_moduli.size(), &rc);
    info->kernel = 3;
    info->rns_moduli = (uint32_t)tch.rns_moduli.size();
    info->digits_a = info->digits_b = 1;
    info->shifts = rc.shifts;
    info->slices = 1;
    info->groups = rc.ngrp;
  } else {
    const int wb = k.wb ? k.wb : tch.wb, L = k.digits ? k.digits : tch.L;
    info->digit_bits = (uint32_t)wb;
    info->digits_a = ternary ? 1u : (uint32_t)L;
    info->digits_b = (uint32_t)L;
    if (k.tiled) {
      TiledCfg tc;
      tiled_config_of(k, logn, (int)info->digits_a, L, &tc);
      info->kernel = tensor_kernel_code(k);
      info->shifts = tc.shifts;
      info->slices = tc.bpg;
      info->groups = tc.ngrp;
    } else {
      info->kernel = 1;
      info->shifts = 1;
      info->slices = n / 1024;
      info->groups = 0;
    }
  }
  return POLYMUL_OK;
}

extern "C" int polymul_tensor_rns_base(uint32_t n, uint64_t qmax, uint32_t* moduli, uint32_t cap, uint32_t* count) {
  clear_error();
  if (!count) return fail(POLYMUL_EINVAL, "count is NULL");
  if (n < 64 || n > 16384 || (n & (n - 1))) return fail(POLYMUL_EINVAL, "n=%u must be a power of two in [64, 16384]", n);
  if (qmax < 2) return fail(POLYMUL_EINVAL, "qmax must be at least 2");
  std::vector<uint32_t> m;
  if (!rns_choose_base(n, qmax, &m)) return fail(POLYMUL_ENOTSUP, "no base of at most %d moduli for n=%u", kRnsMax, n);
  *count = (uint32_t)m.size();
  for (uint32_t i = 0; i < cap && i < m.size(); ++i) moduli[i] = m[i];
  return POLYMUL_OK;
}

// ---------------------------------------------------------------- batch
namespace pm {

template <typename W>
__global__ void k_validate(const W* __restrict__ a, const W* __restrict__ b, uint64_t units, uint32_t n,
                           uint32_t k, const uint64_t* __restrict__ qs, int* flag) {
  const uint64_t total = units * n;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const W q = (W)qs[(i / n) % k];
    if (a[i] >= q || b[i] >= q) *flag = 1;
  }
}

// POLYMUL_FLAG_VALIDATE: every coefficient of a and b below its modulus
// (one kernel over both operands, then a synchronous read of its flag).
static int validate_operands(polymul_plan* p, const void* a, const void* b, uint64_t units, cudaStream_t st) {
  {
    if (!p->d_flag) PM_CUDA(cudaMalloc(&p->d_flag, sizeof(int)));
    if (!p->d_q) {
      PM_CUDA(cudaMalloc(&p->d_q, p->k * sizeof(uint64_t)));
      PM_CUDA(cudaMemcpy(p->d_q, p->q.data(), p->k * sizeof(uint64_t), cudaMemcpyHostToDevice));
    }
    PM_CUDA(cudaMemsetAsync(p->d_flag, 0, sizeof(int), st));
    const int grid = p->num_sms * 4;
    if (p->elem == 4)
      k_validate<uint32_t><<<grid, 256, 0, st>>>((const uint32_t*)a, (const uint32_t*)b, units, p->n, p->k,
                                                 p->d_q, p->d_flag);
    else
      k_validate<uint64_t><<<grid, 256, 0, st>>>((const uint64_t*)a, (const uint64_t*)b, units, p->n, p->k,
                                                 p->d_q, p->d_flag);
    PM_CUDA(cudaGetLastError());
    int h = 0;
    PM_CUDA(cudaMemcpyAsync(&h, p->d_flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    PM_CUDA(cudaStreamSynchronize(st));
    if (h) return fail(POLYMUL_EDOMAIN, "an input coefficient is not below its modulus");
  }
  return POLYMUL_OK;
}

int launch_batch(polymul_plan* p, const void* a, const void* b, void* c, uint64_t batch, cudaStream_t st, int slot) {
  const uint64_t units = batch * p->k;
  unsigned long long* ctr = p->d_ctr + 2 * slot;
  if (p->flags & POLYMUL_FLAG_VALIDATE) {
    const int r = validate_operands(p, a, b, units, st);
    if (r != POLYMUL_OK) return r;
  }
  const uint64_t need = (units + p->ki.units_per_cta - 1) / p->ki.units_per_cta;
  int grid = (int)std::min<uint64_t>(need, (uint64_t)p->grid_cap);
  if (p->ki.cluster > 0) {
    const uint64_t clusters = std::min<uint64_t>(units, (uint64_t)(p->grid_cap / p->ki.cluster));
    grid = (int)(clusters * p->ki.cluster);
  }
  auto launch = [&](void** argv) -> int {
    if (p->ki.cluster > 0) {
      cudaLaunchConfig_t cfg;
      memset(&cfg, 0, sizeof cfg);
      cudaLaunchAttribute attr;
      attr.id = cudaLaunchAttributeClusterDimension;
      attr.val.clusterDim.x = p->ki.cluster;
      attr.val.clusterDim.y = 1;
      attr.val.clusterDim.z = 1;
      cfg.gridDim = dim3(grid);
      cfg.blockDim = dim3(p->ki.block);
      cfg.dynamicSmemBytes = p->ki.smem;
      cfg.stream = st;
      cfg.attrs = &attr;
      cfg.numAttrs = 1;
      PM_CUDA(cudaLaunchKernelExC(&cfg, p->ki.fn, argv));
    } else if (p->launch_flags & kLaunchPdl) {
      cudaLaunchConfig_t cfg;
      memset(&cfg, 0, sizeof cfg);
      cudaLaunchAttribute attr;
      attr.id = cudaLaunchAttributeProgrammaticStreamSerialization;
      attr.val.programmaticStreamSerializationAllowed = 1;
      cfg.gridDim = dim3(grid);
      cfg.blockDim = dim3(p->ki.block);
      cfg.dynamicSmemBytes = p->ki.smem;
      cfg.stream = st;
      cfg.attrs = &attr;
      cfg.numAttrs = 1;
      PM_CUDA(cudaLaunchKernelExC(&cfg, p->ki.fn, argv));
    } else {
      PM_CUDA(cudaLaunchKernel(p->ki.fn, grid, p->ki.block, argv, p->ki.smem, st));
    }
    return POLYMUL_OK;
  };
  if (p->path == POLYMUL_PATH_TENSOR && p->ki.rns) {
    RnsCfg rc;
    if (!rns_config((int)p->logn, p->rns_r, &rc)) return fail(POLYMUL_ENOTSUP, "tensor RNS tiling");
    // residue planes of a and b (slot-private scratch), then the MMA kernel
    const size_t plane = (size_t)units * p->rns_r * p->n;
    if (p->rns_scr_bytes[slot] < 2 * plane) {
      if (p->d_rns_scr[slot]) PM_CUDA(cudaFree(p->d_rns_scr[slot]));
      p->d_rns_scr[slot] = nullptr;
      p->rns_scr_bytes[slot] = 0;
      if (cudaMalloc(&p->d_rns_scr[slot], 2 * plane) != cudaSuccess) return fail(POLYMUL_ENOMEM, "residue planes");
      p->rns_scr_bytes[slot] = 2 * plane;
    }
    int8_t* planes = static_cast<int8_t*>(p->d_rns_scr[slot]);
    PM_CUDA((cudaError_t)rns_prep_launch(p->elem, a, b, planes, units, p->n, p->k, (const RnsBase*)p->d_rns_base,
                                         (const RnsPrime*)p->d_rns_primes, p->rns_r, p->num_sms, st));
    const uint64_t tunits = units * rc.ngrp;
    TensorRnsArgs args{planes, planes + plane, c, (const RnsBase*)p->d_rns_base, (const RnsPrime*)p->d_rns_primes, tunits, p->k,
                       p->cyclic ? 0u : 0x80008000u, p->logn, rc.shifts, rc.nb, rc.b_pitch, rc.ngrp, rc.kc, rc.a_win,
                       rc.bt_off, rc.buf_bytes, rc.tmem_cols, ctr, p->d_err};
    void* argv[] = {&args};
    const int tgrid = (int)std::min<uint64_t>(tunits, (uint64_t)p->grid_cap);
    PM_CUDA(cudaLaunchKernel(p->ki.fn, tgrid, p->ki.block, argv, p->ki.smem, st));
  } else if (p->path == POLYMUL_PATH_TENSOR && p->ki.u64) {
    TiledCfg tc;
    if (!toeplitz_u64_config((int)p->logn, p->ki.digits, &tc)) return fail(POLYMUL_ENOTSUP, "tensor tiling (64-bit)");
    const uint64_t tunits = units * tc.ngrp;
    TensorU64Args args{(const uint64_t*)a, (const uint64_t*)b, (uint64_t*)c, (const TensorPrime64*)p->d_tp64, nullptr,
                       tunits, p->k, p->cyclic ? 0u : 0x80008000u, p->logn, tc.ngrp, tc.kc, tc.a_win, tc.bt_off,
                       tc.tmem_cols, ctr, p->d_err};
    void* argv[] = {&args};
    const int tgrid = (int)std::min<uint64_t>(tunits, (uint64_t)p->grid_cap);
    PM_CUDA(cudaLaunchKernel(p->ki.fn, tgrid, p->ki.block, argv, p->ki.smem, st));
  } else if (p->path == POLYMUL_PATH_TENSOR && p->ki.tiled) {
    TiledCfg tc;
    const DigitShape ds = digit_shape(p, p->ki);
    if (!tiled_config_of(p->ki, (int)p->logn, ds.la, ds.lb, &tc)) return fail(POLYMUL_ENOTSUP, "tensor tiling");
    const uint64_t tunits = units * tc.ngrp;
    // ternary b: c = b * T(a) (the ring is commutative), b's single digit on the A side
    const void* xa = p->ternary_b ? b : a;
    const void* xb = p->ternary_b ? a : b;
    const void* tpc = p->ki.drain && p->d_tpc8 ? p->d_tpc8 : p->d_tpc;
    TensorTiledArgs args{(const uint32_t*)xa, (const uint32_t*)xb, (uint32_t*)c, (const TensorPrime*)tpc,
                         tunits, p->k, p->cyclic ? 0u : 0x80008000u, p->logn, (uint32_t)ds.wb,
                         tc.bpg, tc.ngrp, tc.kc, tc.a_win, tc.bt_off, tc.tmem_cols, ctr, p->d_err, nullptr,
                         tc.stage_bytes};
    void* argv[] = {&args};
    const int tgrid = (int)std::min<uint64_t>(tunits, (uint64_t)p->grid_cap);
    PM_CUDA(cudaLaunchKernel(p->ki.fn, tgrid, p->ki.block, argv, p->ki.smem, st));
  } else if (p->path == POLYMUL_PATH_TENSOR) {
    TensorBatchArgs args{(const uint32_t*)a, (const uint32_t*)b, (uint32_t*)c, (const TensorPrime*)p->d_tpc,
                         units, p->k, p->cyclic ? 0u : 0x80008000u, ctr, p->d_err};
    void* argv[] = {&args};
    PM_CUDA(cudaLaunchKernel(p->ki.fn, grid, p->ki.block, argv, p->ki.smem, st));
  } else {
    // the batch kernel: record its footprint for the next launch on this
    // stream, and let it run ahead of the previous one where that is safe
    // (stream_order.h); the cluster kernel takes no dependent launch
    const uintptr_t bytes = (uintptr_t)(units * p->n * p->elem);
    LaunchFootprint fp;
    fp.a_lo = (uintptr_t)a, fp.a_hi = (uintptr_t)a + bytes;
    fp.b_lo = (uintptr_t)b, fp.b_hi = (uintptr_t)b + bytes;
    fp.c_lo = (uintptr_t)c, fp.c_hi = (uintptr_t)c + bytes;
    StreamOrderGuard order(p->device, st);
    const bool pdl = p->ki.cluster == 0 && (p->launch_flags & kLaunchPdl);
    const uint32_t early = pdl && (p->flags & POLYMUL_FLAG_OVERLAP) && order.may_run_ahead(fp) ? 1u : 0u;
    int r;
    uint32_t tx_pad = 0, polls = 0;
    if (p->ki.cluster == 0) take_injected_wait(&tx_pad, &polls);  // the cluster kernel has no copy waits
    if (p->elem == 4) {
      NttBatchArgs<uint32_t> args{(const uint32_t*)a, (const uint32_t*)b, (uint32_t*)c, p->d_twf, p->d_twi,
                                  (const PrimeConst<uint32_t>*)p->d_pc, units, p->k, ctr, p->d_err,
                                  (const uint32_t*)p->d_outer, nullptr, p->n, 1, 0, early, tx_pad, polls};
      void* argv[] = {&args};
      r = launch(argv);
    } else {
      NttBatchArgs<uint64_t> args{(const uint64_t*)a, (const uint64_t*)b, (uint64_t*)c, p->d_twf, p->d_twi,
                                  (const PrimeConst<uint64_t>*)p->d_pc, units, p->k, ctr, p->d_err,
                                  (const uint64_t*)p->d_outer, nullptr, p->n, 1, 0, early, tx_pad, polls};
      void* argv[] = {&args};
      r = launch(argv);
    }
    // a failed launch enqueued nothing; a cluster launch lets its successor
    // start only at completion, but recording it is harmless
    if (r == POLYMUL_OK) order.record(&fp);
    return r;
  }
  return POLYMUL_OK;
}

}  // namespace pm

static bool misaligned(const void* x) { return ((uintptr_t)x & 15u) != 0; }

extern "C" int polymul_batch(polymul_plan* p, const void* a, const void* b, void* c, uint64_t batch, void* stream) {
  clear_error();
  TraceRange trace_("polymul_batch");
  if (!p) return fail(POLYMUL_EINVAL, "plan is NULL");
  if (batch == 0) return POLYMUL_OK;
  if (!a || !b || !c) return fail(POLYMUL_EINVAL, "null operand pointer");
  if (misaligned(a) || misaligned(b) || misaligned(c)) return fail(POLYMUL_EINVAL, "operands must be 16-byte aligned");
  if (batch > (1ull << 40)) return fail(POLYMUL_EINVAL, "batch too large");
  return launch_batch(p, a, b, c, batch, (cudaStream_t)stream, 0);
}

// Waits for `stream`, then reports whether any kernel of the plan gave up on
// a bounded device wait since the last call; if so the plan's device state
// (work counters, error word) is reset so that the plan can be used again.
extern "C" int polymul_plan_status(polymul_plan* p, void* stream) {
  clear_error();
  if (!p) return fail(POLYMUL_EINVAL, "plan is NULL");
  PM_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  if (!p->d_err) return POLYMUL_OK;
  int h = 0;
  PM_CUDA(cudaMemcpy(&h, p->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (!h) return POLYMUL_OK;
  PM_CUDA(cudaMemset(p->d_err, 0, sizeof(int)));
  if (!(h & 1)) return fail(POLYMUL_EDOMAIN, "b has a coefficient outside {0, 1, q - 1} (ternary-b plan); results invalid");
  PM_CUDA(cudaMemset(p->d_ctr, 0, 2 * kCounterSlots * sizeof(unsigned long long)));
  return fail(POLYMUL_ETIMEOUT, "a device wait expired; results of the affected launches are invalid");
}

void* pm::mapped_host_range(const void* x, size_t bytes) {
  cudaPointerAttributes lo, hi;
  if (cudaPointerGetAttributes(&lo, x) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (lo.type != cudaMemoryTypeHost || !lo.devicePointer) return nullptr;
  if (cudaPointerGetAttributes(&hi, (const char*)x + (bytes - 1)) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (hi.type != cudaMemoryTypeHost || (char*)hi.devicePointer != (char*)lo.devicePointer + (bytes - 1)) return nullptr;
  return lo.devicePointer;
}

namespace {

// The kernel of the direct route for the plan's word size and degree
// (looked up and sized once per plan): the plan's own thread-block-cluster
// kernel where it has one (it loads and stores with plain accesses
// already), else the batch kernel in its direct form; false when neither
// applies.
bool direct_kernel(polymul_plan* p) {
  if (p->dki.fn) return true;
  if (p->ki.cluster > 0) {
    p->dki = p->ki;
    p->dgrid_cap = p->grid_cap;
    return true;
  }
  KernelInfo ki;
  const int logn = (int)p->logn;
  if (!(p->aux_prime        ? lookup_ntt_direct_aux(logn, &ki)
        : p->elem == 4 ? lookup_ntt_direct_u32(logn, &ki)
                       : lookup_ntt_direct_u64(logn, &ki)))
    return false;
  if (ki.smem > 48 * 1024 &&
      cudaFuncSetAttribute(ki.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, ki.smem) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ki.fn, ki.block, ki.smem) != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    return false;
  }
  // one CTA per SM: the link, not the SMs, bounds this kernel, and a shallow
  // queue of loads (one unit per CTA, 8 KB and more per SM in flight) ends
  // each launch sooner than a full one (n = 1024, 4096 products, back to
  // back: 174 us per batch at 1 CTA per SM, 179 / 182 / 189 at 2 / 3 / 4,
  // 188 at the occupancy limit of 10)
  p->dgrid_cap = p->num_sms;
  p->dki = ki;
  return true;
}

}  // namespace

// The direct route on host memory the device maps: one launch of the batch
// kernel's direct form (or of the plan's thread-block-cluster kernel) reads
// a and b and writes c in place over the coherent host link, so the link
// carries operands in and results out at the same time with no staging
// buffer, copy engine or chunk boundary.  a, b, c are the device addresses
// of the ranges.  Counter slot 2 (its own: a host-buffer
// call may follow device-pointer batches still running on other streams).
// Like a device-pointer batch the launch is recorded for the stream-order
// guard and, with POLYMUL_FLAG_OVERLAP, may run ahead of its predecessor.
static int launch_direct(polymul_plan* p, const void* a, const void* b, void* c, uint64_t batch, cudaStream_t st) {
  const uint64_t units = batch * p->k;
  if (p->flags & POLYMUL_FLAG_VALIDATE) {
    const int r = validate_operands(p, a, b, units, st);
    if (r != POLYMUL_OK) return r;
  }
  const uint64_t need = (units + p->dki.units_per_cta - 1) / p->dki.units_per_cta;
  const int grid = (int)std::min<uint64_t>(need, (uint64_t)p->dgrid_cap);
  unsigned long long* ctr = p->d_ctr + 2 * kDirectSlot;
  const uintptr_t bytes = (uintptr_t)(units * p->n * p->elem);
  LaunchFootprint fp;
  fp.a_lo = (uintptr_t)a, fp.a_hi = (uintptr_t)a + bytes;
  fp.b_lo = (uintptr_t)b, fp.b_hi = (uintptr_t)b + bytes;
  fp.c_lo = (uintptr_t)c, fp.c_hi = (uintptr_t)c + bytes;
  StreamOrderGuard order(p->device, st);
  // the cluster kernels take no dependent launch (their successor starts at
  // their completion; recording them is harmless)
  const bool cluster = p->dki.cluster > 0;
  const uint32_t early = !cluster && (p->flags & POLYMUL_FLAG_OVERLAP) && order.may_run_ahead(fp) ? 1u : 0u;
  cudaLaunchConfig_t cfg;
  memset(&cfg, 0, sizeof cfg);
  cudaLaunchAttribute attr;
  if (cluster) {
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = p->dki.cluster;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
  } else {
    attr.id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr.val.programmaticStreamSerializationAllowed = 1;
  }
  cfg.gridDim = dim3(cluster ? (unsigned)(std::min<uint64_t>(units, (uint64_t)(p->dgrid_cap / p->dki.cluster)) *
                                          p->dki.cluster)
                             : (unsigned)grid);
  cfg.blockDim = dim3(p->dki.block);
  cfg.dynamicSmemBytes = p->dki.smem;
  cfg.stream = st;
  cfg.attrs = &attr;
  cfg.numAttrs = 1;
  if (p->elem == 4) {
    NttBatchArgs<uint32_t> args{(const uint32_t*)a, (const uint32_t*)b, (uint32_t*)c, p->d_twf, p->d_twi,
                                (const PrimeConst<uint32_t>*)p->d_pc, units, p->k, ctr, p->d_err,
                                (const uint32_t*)p->d_outer, nullptr, p->n, 1, 0, early, 0, 0};
    void* argv[] = {&args};
    PM_CUDA(cudaLaunchKernelExC(&cfg, p->dki.fn, argv));
  } else {
    NttBatchArgs<uint64_t> args{(const uint64_t*)a, (const uint64_t*)b, (uint64_t*)c, p->d_twf, p->d_twi,
                                (const PrimeConst<uint64_t>*)p->d_pc, units, p->k, ctr, p->d_err,
                                nullptr, nullptr, p->n, 1, 0, early, 0, 0};
    void* argv[] = {&args};
    PM_CUDA(cudaLaunchKernelExC(&cfg, p->dki.fn, argv));
  }
  order.record(&fp);
  return POLYMUL_OK;
}

// The device addresses of a, b, c for the direct form, or a POLYMUL code:
// ENOTSUP when the plan has no direct kernel, EINVAL when a range is not
// mapped page-locked host memory or is misaligned.
static int direct_ranges(polymul_plan* p, const void* a, const void* b, void* c, uint64_t batch, void** da,
                         void** db, void** dc) {
  if (p->path != POLYMUL_PATH_NTT || !direct_kernel(p))
    return fail(POLYMUL_ENOTSUP, "no direct-access kernel for this plan (NTT path only)");
  if (((uintptr_t)a | (uintptr_t)b | (uintptr_t)c) % p->elem != 0)
    return fail(POLYMUL_EINVAL, "operands must be aligned to the %u-byte word", p->elem);
  const size_t bytes = (size_t)batch * p->k * p->n * p->elem;
  *da = mapped_host_range(a, bytes);
  *db = mapped_host_range(b, bytes);
  *dc = mapped_host_range(c, bytes);
  if (!*da || !*db || !*dc) return fail(POLYMUL_EINVAL, "a, b and c must lie in page-locked host memory the device maps");
  return POLYMUL_OK;
}

extern "C" int polymul_batch_mapped(polymul_plan* p, const void* a, const void* b, void* c, uint64_t batch,
                                    void* stream) {
  clear_error();
  TraceRange trace_("polymul_batch_mapped");
  if (!p) return fail(POLYMUL_EINVAL, "plan is NULL");
  if (batch == 0) return POLYMUL_OK;
  if (!a || !b || !c) return fail(POLYMUL_EINVAL, "null operand pointer");
  if (batch > (1ull << 40)) return fail(POLYMUL_EINVAL, "batch too large");
  void *da, *db, *dc;
  const int r = direct_ranges(p, a, b, c, batch, &da, &db, &dc);
  return r != POLYMUL_OK ? r : launch_direct(p, da, db, dc, batch, (cudaStream_t)stream);
}

// Host buffers: chunks of products flow through a three-stage pipeline --
// copies in, kernel, copy out, each stage on a stream of its own -- over
// kHostSlots plan-owned device staging slots, with one event per stage and
// slot: a chunk's kernel waits for its copies in, its copy out for its
// kernel, and the copies in of the chunk that next takes the slot for that
// copy out.  So copies in of later chunks, kernels and copies out of
// earlier ones overlap without one stream's order holding back another.
extern "C" int polymul_batch_host(polymul_plan* p, const void* a, const void* b, void* c, uint64_t batch,
                                  void* stream) {
  clear_error();
  TraceRange trace_("polymul_batch_host");
  if (!p) return fail(POLYMUL_EINVAL, "plan is NULL");
  if (batch == 0) return POLYMUL_OK;
  if (!a || !b || !c) return fail(POLYMUL_EINVAL, "null operand pointer");
  const size_t prod_bytes = (size_t)p->k * p->n * p->elem;
  void *da, *db, *dc;
  if (!(p->flags & POLYMUL_FLAG_HOST_STAGED) && batch <= (1ull << 40) &&
      direct_ranges(p, a, b, c, batch, &da, &db, &dc) == POLYMUL_OK) {
    const int rc = launch_direct(p, da, db, dc, batch, (cudaStream_t)stream);
    if (rc != POLYMUL_OK) return rc;
    ++p->host_direct;
    PM_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    return POLYMUL_OK;
  }
  clear_error();  // the staged route serves what the direct one cannot
  // about 4 MB of each operand per chunk by default (POLYMUL_HOST_CHUNK_BYTES
  // overrides)
  static const size_t chunk_target = [] {
    const char* e = getenv("POLYMUL_HOST_CHUNK_BYTES");
    const long long v = e ? atoll(e) : 0;
    return v > 0 ? (size_t)v : (size_t)(4u << 20);
  }();
  const uint64_t chunk = std::max<uint64_t>(1, chunk_target / prod_bytes);
  const size_t slot_bytes = 3 * chunk * prod_bytes;
  for (int g = 0; g < 3; ++g)
    if (!p->hs[g]) PM_CUDA(cudaStreamCreateWithFlags(&p->hs[g], cudaStreamNonBlocking));
  for (int s = 0; s < kHostSlots; ++s) {
    for (int g = 0; g < 3; ++g)
      if (!p->hev[g][s]) PM_CUDA(cudaEventCreateWithFlags(&p->hev[g][s], cudaEventDisableTiming));
    if (p->hslot_bytes < slot_bytes) {
      cudaFree(p->d_hslot[s]);
      p->d_hslot[s] = nullptr;
      if (cudaMalloc(&p->d_hslot[s], slot_bytes) != cudaSuccess)
        return fail(POLYMUL_ENOMEM, "staging allocation of %zu bytes failed", slot_bytes);
    }
  }
  p->hslot_bytes = std::max(p->hslot_bytes, slot_bytes);
  if (!p->ev_entry) PM_CUDA(cudaEventCreateWithFlags(&p->ev_entry, cudaEventDisableTiming));
  PM_CUDA(cudaEventRecord(p->ev_entry, (cudaStream_t)stream));
  for (int g = 0; g < 3; ++g) PM_CUDA(cudaStreamWaitEvent(p->hs[g], p->ev_entry, 0));
  cudaStream_t s_in = p->hs[0], s_k = p->hs[1], s_out = p->hs[2];
  const char* ha = (const char*)a;
  const char* hb = (const char*)b;
  char* hc = (char*)c;
  int rc = POLYMUL_OK;
  for (uint64_t first = 0, it = 0; first < batch; first += chunk, ++it) {
    const uint64_t cnt = std::min<uint64_t>(chunk, batch - first);
    const int s = (int)(it % kHostSlots);
    char* da = (char*)p->d_hslot[s];
    char* db = da + chunk * prod_bytes;
    char* dc = db + chunk * prod_bytes;
    const size_t off = first * prod_bytes, bytes = cnt * prod_bytes;
    // the slot's previous chunk has been copied out
    if (it >= (uint64_t)kHostSlots) PM_CUDA(cudaStreamWaitEvent(s_in, p->hev[2][s], 0));
    PM_CUDA(cudaMemcpyAsync(da, ha + off, bytes, cudaMemcpyHostToDevice, s_in));
    PM_CUDA(cudaMemcpyAsync(db, hb + off, bytes, cudaMemcpyHostToDevice, s_in));
    PM_CUDA(cudaEventRecord(p->hev[0][s], s_in));
    PM_CUDA(cudaStreamWaitEvent(s_k, p->hev[0][s], 0));
    rc = launch_batch(p, da, db, dc, cnt, s_k, 1);
    if (rc != POLYMUL_OK) break;
    PM_CUDA(cudaEventRecord(p->hev[1][s], s_k));
    PM_CUDA(cudaStreamWaitEvent(s_out, p->hev[1][s], 0));
    PM_CUDA(cudaMemcpyAsync(hc + off, dc, bytes, cudaMemcpyDeviceToHost, s_out));
    PM_CUDA(cudaEventRecord(p->hev[2][s], s_out));
  }
  for (int g = 0; g < 3; ++g) {
    cudaError_t e = cudaStreamSynchronize(p->hs[g]);
    if (e != cudaSuccess && rc == POLYMUL_OK) rc = cuda_fail(e, "cudaStreamSynchronize");
  }
  return rc;
}

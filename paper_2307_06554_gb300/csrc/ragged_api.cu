// C-ABI entry points for uneven batches (polymul_ragged_*), see
// include/polymul.h.  Host-side planning: tables per pool prime, units
// sorted into degree segments, two concurrent persistent launches (2^14;
// 2^10 .. 2^13), optional CUDA-graph replay; a degree class may instead run
// on the tensor path (Sec. 2.2 matrix form, the drained tiled kernel over
// that class's rows), chosen per class by measurement.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/polymul.h"
#include "host_math.h"
#include "kernels.h"
#include "trace.h"
#include "plan.h"
#include "polymul_types.h"
#include "toeplitz_tiled.h"

using namespace pm;

#define PM_CUDA(call)                                       \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return pm::cuda_fail(e_, #call); \
  } while (0)

struct polymul_ragged {
  uint32_t nmax = 0, lognmax = 0;
  std::vector<uint64_t> pool;
  int mode = 0;
  void* d_twf = nullptr;
  void* d_twi = nullptr;
  void* d_pc = nullptr;
  KernelInfo ki[kRaggedSets][2];    // [shape set][0: degrees 2^10 .. 2^13, 1: 2^14]
  // set 0 of the 2^14 launch is the homogeneous batch kernel (radix 32, both
  // operands in registers) over the segment's row table, not k_ntt_ragged
  bool batch14 = false;
  int grid_cap[kRaggedSets][2] = {};
  int device = 0, num_sms = 0;
  // the tensor route of degree class 2^(10 + i): the drained tiled kernel
  // with `tdigits` 8-bit digits per operand (enough for every pool prime),
  // its tiling and resident grid, and the pool's constants for it
  bool tensor_ok[kRaggedClasses] = {};
  KernelInfo tki[kRaggedClasses];
  TiledCfg tcfg[kRaggedClasses];
  int tgrid_cap[kRaggedClasses] = {};
  int tdigits = 0;
  void* d_tpc = nullptr;  // [pool] TensorPrime (8-bit digit weights)
};

// A prepared list runs as up to two persistent launches (the 2^14 segment
// and the smaller degrees), concurrent on two streams (or as two
// independent nodes of one CUDA graph).
struct polymul_ragged_batch {
  polymul_ragged* ctx = nullptr;
  uint64_t n_units = 0, n_items = 0, total_elems = 0;
  uint64_t part_units[2] = {0, 0};  // units of each launch ([0] small degrees, [1] 2^14)
  RaggedUnit* d_units = nullptr;
  RaggedItem* d_items = nullptr;
  unsigned long long* d_ctr = nullptr;  // 2 x (kRaggedMaxSegs + 1): one counter set per launch
  int* d_err = nullptr;
  RaggedArgs args[2]{};
  NttBatchArgs<uint32_t> bargs{};  // the 2^14 launch when it runs the batch kernel
  cudaStream_t side = nullptr;  // the second launch's stream (fork/join with the caller's)
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraphNode_t node[2] = {nullptr, nullptr};
  // shape set of each launch: the padded one-operand set by default (fewer
  // registers, no spills at 2^14); polymul_ragged_tune measures both
  int set[2] = {1, 1};
  // degree segments of the whole list (host copy; d_items holds those the
  // NTT launches take), and the classes on the tensor path (bit logn - 10)
  std::vector<RaggedItem> items_h;
  uint32_t present = 0;      // classes with units (bit logn - 10)
  uint32_t tensor_mask = 0;  // a subset of `present`
  unsigned long long* d_tctr = nullptr;  // 2 counters per tensor class launch
  TensorTiledArgs targs[kRaggedClasses]{};
  cudaGraphNode_t tnode[kRaggedClasses] = {};
  RaggedItem* d_item1 = nullptr;  // one segment, for timing a class alone
};

namespace {

// tables of one prime at nmax, plus the constants of every degree 2^logn
// <= nmax derived from the same root (so that each degree's tables are
// prefixes of these)
void build_ragged_prime(uint64_t q, uint32_t nmax, std::vector<uint32_t>& twf, std::vector<uint32_t>& twi,
                        PrimeConst<uint32_t>* pc16) {
  using namespace pm::host;
  const int lognmax = __builtin_ctz(nmax);
  const uint64_t psi = primitive_2n_root(q, nmax);
  const uint64_t psi_inv = powmod(psi, q - 2, q);
  for (uint32_t i = 0; i < nmax; ++i) {
    const uint32_t r = bitrev(i, lognmax);
    const uint64_t w = powmod(psi, r, q), v = powmod(psi_inv, r, q);
    twf.push_back((uint32_t)w);
    twf.push_back((uint32_t)shoup_companion(w, q, 32));
    twi.push_back((uint32_t)v);
    twi.push_back((uint32_t)shoup_companion(v, q, 32));
  }
  const uint64_t v1 = powmod(psi_inv, bitrev(1, lognmax), q);  // = psi_n^-brv_n(1) for every n <= nmax
  const uint64_t r_mod_q = (1ull << 32) % q;
  for (int logn = 0; logn < 16; ++logn) {
    PrimeConst<uint32_t>& c = pc16[logn];
    memset(&c, 0, sizeof c);
    if (logn > lognmax) continue;
    const uint64_t ninv = powmod(1ull << logn, q - 2, q);
    const uint64_t scale = mulmod(ninv, r_mod_q, q);
    const uint64_t scale_w = mulmod(v1, scale, q);
    c.q = (uint32_t)q;
    c.q2 = (uint32_t)(2 * q);
    c.qinv = (uint32_t)inv_pow2_64(q);
    c.scale = (uint32_t)scale;
    c.scale_p = (uint32_t)shoup_companion(scale, q, 32);
    c.scale_w = (uint32_t)scale_w;
    c.scale_wp = (uint32_t)shoup_companion(scale_w, q, 32);
  }
}

// 8-bit balanced digits covering the centred residues of every prime up to
// qmax (at most 4: q < 2^31); 0 if more are needed
int ragged_tensor_digits(uint64_t qmax) {
  for (int l = 1; l <= 4; ++l)
    if ((uint64_t)127 * ((1ull << (8 * l)) - 1) / 255 >= qmax / 2) return l;
  return 0;
}

// The tensor route of every degree class up to n_max: kernels, their
// resident grids, and the pool's digit-weight constants.  A class whose
// kernel does not fit keeps the NTT route only.
int ragged_tensor_setup(polymul_ragged* r) {
  const uint64_t qmax = *std::max_element(r->pool.begin(), r->pool.end());
  r->tdigits = ragged_tensor_digits(qmax);
  if (!r->tdigits) return POLYMUL_OK;
  for (int i = 0; i < kRaggedClasses; ++i) {
    const int logn = 10 + i;
    if (logn > (int)r->lognmax) break;
    KernelInfo ki;
    if (!lookup_toeplitz_tiled_drain(logn, r->tdigits, r->tdigits, &ki) ||
        !toeplitz_tiled_config_drain(logn, r->tdigits, r->tdigits, &r->tcfg[i]))
      continue;
    PM_CUDA(cudaFuncSetAttribute(ki.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, ki.smem));
    int per_sm = 0;
    const int rc = tmem_kernel_per_sm(ki, r->device, &per_sm);
    if (rc != POLYMUL_OK) return rc;
    if (per_sm < 1) continue;
    r->tki[i] = ki;
    r->tgrid_cap[i] = per_sm * r->num_sms;
    r->tensor_ok[i] = true;
  }
  std::vector<TensorPrime> tp(r->pool.size());
  for (size_t j = 0; j < r->pool.size(); ++j) {
    const uint64_t q = r->pool[j];
    memset(&tp[j], 0, sizeof tp[j]);
    tp[j].q = (uint32_t)q;
    for (int e = 0; e < 15; ++e) tp[j].pw[e] = (uint32_t)pm::host::powmod(2, 8ull * e, q);
    tp[j].mu = (uint64_t)(((pm::host::u128)1 << 64) / q);
    tp[j].bias = ((1ull << 60) + q - 1) / q * q;
  }
  if (cudaMalloc(&r->d_tpc, tp.size() * sizeof(TensorPrime)) != cudaSuccess)
    return fail(POLYMUL_ENOMEM, "tensor constants");
  PM_CUDA(cudaMemcpy(r->d_tpc, tp.data(), tp.size() * sizeof(TensorPrime), cudaMemcpyHostToDevice));
  return POLYMUL_OK;
}

}  // namespace

extern "C" void polymul_ragged_destroy(polymul_ragged* r) {
  if (!r) return;
  cudaFree(r->d_twf);
  cudaFree(r->d_twi);
  cudaFree(r->d_pc);
  cudaFree(r->d_tpc);
  delete r;
}

extern "C" int polymul_ragged_create(const uint64_t* pool, uint32_t pool_size, uint32_t n_max, polymul_ragged** out) {
  clear_error();
  if (!out || !pool || pool_size == 0) return fail(POLYMUL_EINVAL, "need a non-empty prime pool and an out pointer");
  if (n_max < 1024 || n_max > 16384 || (n_max & (n_max - 1)))
    return fail(POLYMUL_EINVAL, "n_max=%u must be a power of two in [1024, 16384]", n_max);
  for (uint32_t j = 0; j < pool_size; ++j) {
    const uint64_t q = pool[j];
    if (q >= (1ull << 31) || !pm::host::is_prime(q) || (q - 1) % (2ull * n_max) != 0)
      return fail(POLYMUL_EINVAL, "pool[%u]=%llu must be a prime < 2^31 with 2 n_max | q - 1", j,
                  (unsigned long long)q);
    for (uint32_t i = 0; i < j; ++i)
      if (pool[i] == q) return fail(POLYMUL_EINVAL, "duplicate pool prime %llu", (unsigned long long)q);
  }
  polymul_ragged* r = new polymul_ragged();
  r->nmax = n_max;
  r->lognmax = __builtin_ctz(n_max);
  r->pool.assign(pool, pool + pool_size);
  const uint64_t qmax = *std::max_element(r->pool.begin(), r->pool.end());
  r->mode = qmax < (1ull << 30) ? 1 : 0;  // Harvey bounds when every prime allows them
  int rc = POLYMUL_OK;
  std::vector<uint32_t> twf, twi;
  std::vector<PrimeConst<uint32_t>> pcs((size_t)pool_size * 16);
  for (uint32_t j = 0; j < pool_size; ++j) build_ragged_prime(r->pool[j], n_max, twf, twi, &pcs[(size_t)j * 16]);
  auto up = [&](void** dst, const void* src, size_t bytes) -> int {
    if (cudaMalloc(dst, bytes) != cudaSuccess) return fail(POLYMUL_ENOMEM, "table allocation failed");
    PM_CUDA(cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice));
    return POLYMUL_OK;
  };
  if (rc == POLYMUL_OK) rc = up(&r->d_twf, twf.data(), twf.size() * 4);
  if (rc == POLYMUL_OK) rc = up(&r->d_twi, twi.data(), twi.size() * 4);
  if (rc == POLYMUL_OK) rc = up(&r->d_pc, pcs.data(), pcs.size() * sizeof(PrimeConst<uint32_t>));
  for (int set = 0; set < kRaggedSets && rc == POLYMUL_OK; ++set)
    if (!lookup_ntt_ragged(r->mode, set, &r->ki[set][0], &r->ki[set][1])) rc = fail(POLYMUL_ENOTSUP, "no ragged kernel");
  // the 2^14 segment's set 0: the homogeneous one-CTA-per-product kernel
  // with a row table (measured 504 vs 555 us for the 2000-product list's
  // 2^14 rows; it spills less at the 128 registers a 512-thread CTA allows)
  if (rc == POLYMUL_OK && r->lognmax >= 14 && lookup_ntt_u32_rb5(14, r->mode, &r->ki[0][1])) r->batch14 = true;
  if (rc == POLYMUL_OK) {
    cudaError_t e = cudaGetDevice(&r->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&r->num_sms, cudaDevAttrMultiProcessorCount, r->device);
    for (int k = 0; k < 2 * kRaggedSets && e == cudaSuccess && rc == POLYMUL_OK; ++k) {
      const int set = k / 2, i = k % 2;
      const KernelInfo& ki = r->ki[set][i];
      int per_sm = 0;
      e = cudaFuncSetAttribute(ki.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, ki.smem);
      if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ki.fn, ki.block, ki.smem);
      if (e == cudaSuccess && per_sm < 1) rc = fail(POLYMUL_ENOTSUP, "ragged kernel does not fit on an SM");
      r->grid_cap[set][i] = per_sm * r->num_sms;
    }
    if (e != cudaSuccess) rc = cuda_fail(e, "ragged kernel configuration");
  }
  if (rc == POLYMUL_OK) rc = ragged_tensor_setup(r);
  if (rc != POLYMUL_OK) {
    std::string keep = polymul_last_error();
    polymul_ragged_destroy(r);
    fail(rc, "%s", keep.c_str());
    return rc;
  }
  *out = r;
  return POLYMUL_OK;
}

extern "C" void polymul_ragged_batch_destroy(polymul_ragged_batch* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->side) cudaStreamDestroy(b->side);
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  if (b->ev_join) cudaEventDestroy(b->ev_join);
  cudaFree(b->d_units);
  cudaFree(b->d_items);
  cudaFree(b->d_ctr);
  cudaFree(b->d_err);
  cudaFree(b->d_tctr);
  cudaFree(b->d_item1);
  delete b;
}

namespace {

// The launches of the list under its path choice: the NTT segments (d_items,
// rewritten here; the 2^14 one, if present and on the NTT path, goes to the
// second kernel) and one tiled tensor launch per class on the tensor path.
// The caller makes sure that no launch of the list is in flight.
void apply_paths(polymul_ragged_batch* b) {
  polymul_ragged* r = b->ctx;
  std::vector<RaggedItem> ntt;
  uint64_t ntt_units = 0;
  for (const RaggedItem& it : b->items_h) {
    const int cls = (int)it.logn - 10;
    if (r->tensor_ok[cls]) {
      const TiledCfg& tc = r->tcfg[cls];
      const TensorTiledArgs keep = b->targs[cls];  // operands, if set
      b->targs[cls] = TensorTiledArgs{keep.a, keep.b, keep.c, (const TensorPrime*)r->d_tpc,
                                      (uint64_t)it.count * tc.ngrp, 1, 0x80008000u, it.logn, 8u, tc.bpg, tc.ngrp,
                                      tc.kc, tc.a_win, tc.bt_off, tc.tmem_cols, b->d_tctr + 2 * cls, b->d_err,
                                      b->d_units + it.first};
    }
    if (!((b->tensor_mask >> cls) & 1u)) {
      ntt.push_back(it);
      ntt_units += it.count;
    }
  }
  if (!ntt.empty()) cudaMemcpy(b->d_items, ntt.data(), ntt.size() * sizeof(RaggedItem), cudaMemcpyHostToDevice);
  const uint64_t n_big = (!ntt.empty() && ntt[0].logn == 14) ? 1 : 0;
  b->part_units[1] = n_big ? ntt[0].count : 0;
  b->part_units[0] = ntt_units - b->part_units[1];
  b->args[1] = RaggedArgs{nullptr, nullptr, nullptr, b->d_units, b->d_items, n_big, r->d_twf, r->d_twi,
                          (const PrimeConst<uint32_t>*)r->d_pc, r->nmax, b->d_ctr, b->d_err};
  b->args[0] = RaggedArgs{nullptr, nullptr, nullptr, b->d_units, b->d_items + n_big, ntt.size() - n_big,
                          r->d_twf, r->d_twi, (const PrimeConst<uint32_t>*)r->d_pc, r->nmax,
                          b->d_ctr + (kRaggedMaxSegs + 1), b->d_err};
  // the batch kernel's form of the 2^14 launch: unit u is row u of the
  // segment, tables of its pool prime at degree 2^14 (tw_stride = n_max,
  // constants at [prime][14])
  const NttBatchArgs<uint32_t> keep = b->bargs;
  b->bargs = NttBatchArgs<uint32_t>{};
  b->bargs.a = keep.a;
  b->bargs.b = keep.b;
  b->bargs.c = keep.c;
  b->bargs.tw_fwd = r->d_twf;
  b->bargs.tw_inv = r->d_twi;
  b->bargs.pc = (const PrimeConst<uint32_t>*)r->d_pc;
  b->bargs.units = b->part_units[1];
  b->bargs.k = 1;
  b->bargs.ctr = b->d_ctr;
  b->bargs.err = b->d_err;
  b->bargs.tw_stride = r->nmax;
  b->bargs.pc_stride = 16;
  b->bargs.pc_off = 14;
  b->bargs.rows = n_big ? b->d_units + ntt[0].first : nullptr;
}

}  // namespace

extern "C" int polymul_ragged_prepare(polymul_ragged* r, const polymul_desc* descs, uint32_t count,
                                      const uint32_t* prime_idx, uint64_t prime_idx_len, uint64_t total_elems,
                                      polymul_ragged_batch** out) {
  clear_error();
  TraceRange trace_("polymul_ragged_prepare");
  if (!r || !out || (count && (!descs || !prime_idx))) return fail(POLYMUL_EINVAL, "null argument");
  // units grouped by degree class
  std::vector<std::vector<RaggedUnit>> cls(16);
  for (uint32_t p = 0; p < count; ++p) {
    const polymul_desc& d = descs[p];
    if (d.n < 1024 || d.n > r->nmax || (d.n & (d.n - 1)))
      return fail(POLYMUL_EINVAL, "product %u: n=%u must be a power of two in [1024, %u]", p, d.n, r->nmax);
    if (d.k == 0 || (uint64_t)d.prime_offset + d.k > prime_idx_len)
      return fail(POLYMUL_EINVAL, "product %u: primes [%u, %u) outside the index array", p, d.prime_offset,
                  d.prime_offset + d.k);
    if (d.offset % 4 != 0 || d.offset + (uint64_t)d.k * d.n > total_elems)
      return fail(POLYMUL_EINVAL, "product %u: rows must be 16-byte aligned and inside the buffers", p);
    const int logn = __builtin_ctz(d.n);
    for (uint32_t i = 0; i < d.k; ++i) {
      const uint32_t pi = prime_idx[d.prime_offset + i];
      if (pi >= r->pool.size()) return fail(POLYMUL_EINVAL, "product %u: prime index %u outside the pool", p, pi);
      cls[logn].push_back(RaggedUnit{d.offset + (uint64_t)i * d.n, pi, 0});
    }
  }
  // degree segments, largest degree first (the longest units start first)
  std::vector<RaggedUnit> units;
  std::vector<RaggedItem> items;
  for (int logn = 15; logn >= 0; --logn) {
    if (cls[logn].empty()) continue;
    if (cls[logn].size() > 0xFFFFFFFFull || units.size() + cls[logn].size() > 0xFFFFFFFFull)
      return fail(POLYMUL_EINVAL, "too many units in one list");
    items.push_back(RaggedItem{(uint32_t)logn, (uint32_t)units.size(), (uint32_t)cls[logn].size(), 0});
    units.insert(units.end(), cls[logn].begin(), cls[logn].end());
  }
  polymul_ragged_batch* b = new polymul_ragged_batch();
  b->ctx = r;
  b->n_units = units.size();
  b->n_items = items.size();
  b->total_elems = total_elems;
  int rc = POLYMUL_OK;
  auto up = [&](void** dst, const void* src, size_t bytes) -> int {
    if (cudaMalloc(dst, bytes ? bytes : 16) != cudaSuccess) return fail(POLYMUL_ENOMEM, "batch allocation failed");
    if (bytes) PM_CUDA(cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice));
    return POLYMUL_OK;
  };
  rc = up((void**)&b->d_units, units.data(), units.size() * sizeof(RaggedUnit));
  if (rc == POLYMUL_OK) rc = up((void**)&b->d_items, items.data(), items.size() * sizeof(RaggedItem));
  if (rc == POLYMUL_OK) {
    const unsigned long long zero[2 * (kRaggedMaxSegs + 1)] = {};
    const int z = 0;
    rc = up((void**)&b->d_ctr, zero, sizeof zero);
    if (rc == POLYMUL_OK) rc = up((void**)&b->d_err, &z, sizeof z);
    if (rc == POLYMUL_OK) rc = up((void**)&b->d_tctr, zero, 2 * kRaggedClasses * sizeof(unsigned long long));
    if (rc == POLYMUL_OK) rc = up((void**)&b->d_item1, nullptr, 0);
  }
  if (rc == POLYMUL_OK && (cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking) != cudaSuccess ||
                           cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
                           cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming) != cudaSuccess))
    rc = fail(POLYMUL_ECUDA, "stream or event creation failed");
  if (rc != POLYMUL_OK) {
    std::string keep = polymul_last_error();
    polymul_ragged_batch_destroy(b);
    fail(rc, "%s", keep.c_str());
    return rc;
  }
  b->items_h = items;
  for (const RaggedItem& it : items) b->present |= 1u << (it.logn - 10);
  apply_paths(b);
  *out = b;
  return POLYMUL_OK;
}

namespace {
int ragged_check(polymul_ragged_batch* b, const void* a, const void* bb, void* c) {
  if (!b) return fail(POLYMUL_EINVAL, "batch is NULL");
  if (b->n_items && (!a || !bb || !c)) return fail(POLYMUL_EINVAL, "null operand pointer");
  if (((uintptr_t)a | (uintptr_t)bb | (uintptr_t)c) & 15u) return fail(POLYMUL_EINVAL, "operands must be 16-byte aligned");
  return POLYMUL_OK;
}
const KernelInfo& ragged_kernel(const polymul_ragged_batch* b, int part) { return b->ctx->ki[b->set[part]][part]; }
// the recorded graph holds the kernels of the previous shape sets
void drop_graph(polymul_ragged_batch* b) {
  if (!b->exec) return;
  cudaGraphExecDestroy(b->exec);
  cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  b->node[0] = b->node[1] = nullptr;
  for (int i = 0; i < kRaggedClasses; ++i) b->tnode[i] = nullptr;
}
int ragged_grid(const polymul_ragged_batch* b, int part) {
  return (int)std::min<uint64_t>((uint64_t)b->ctx->grid_cap[b->set[part]][part],
                                 std::max<uint64_t>(1, b->part_units[part]));
}
void set_operands(polymul_ragged_batch* b, const void* a, const void* bb, void* c) {
  for (int i = 0; i < 2; ++i) {
    b->args[i].a = (const uint32_t*)a;
    b->args[i].b = (const uint32_t*)bb;
    b->args[i].c = (uint32_t*)c;
  }
  for (int i = 0; i < kRaggedClasses; ++i) {
    b->targs[i].a = (const uint32_t*)a;
    b->targs[i].b = (const uint32_t*)bb;
    b->targs[i].c = (uint32_t*)c;
  }
  b->bargs.a = (const uint32_t*)a;
  b->bargs.b = (const uint32_t*)bb;
  b->bargs.c = (uint32_t*)c;
}
// the argument block of launch `part` under its shape set
void* part_args(polymul_ragged_batch* b, int part) {
  return (part == 1 && b->set[1] == 0 && b->ctx->batch14) ? (void*)&b->bargs : (void*)&b->args[part];
}
cudaError_t launch_part(polymul_ragged_batch* b, int part, cudaStream_t s) {
  const KernelInfo& ki = ragged_kernel(b, part);
  void* argv[] = {part_args(b, part)};
  return cudaLaunchKernel(ki.fn, ragged_grid(b, part), ki.block, argv, ki.smem, s);
}
int tensor_grid(const polymul_ragged_batch* b, int cls) {
  return (int)std::min<uint64_t>((uint64_t)b->ctx->tgrid_cap[cls], std::max<uint64_t>(1, b->targs[cls].units));
}
bool tensor_class(const polymul_ragged_batch* b, int cls) { return (b->tensor_mask >> cls) & 1u; }
cudaError_t launch_tensor(polymul_ragged_batch* b, int cls, cudaStream_t s) {
  const KernelInfo& ki = b->ctx->tki[cls];
  void* argv[] = {&b->targs[cls]};
  return cudaLaunchKernel(ki.fn, tensor_grid(b, cls), ki.block, argv, ki.smem, s);
}
}  // namespace

// Up to two persistent launches: the 2^14 segment on the caller's stream and
// the smaller degrees on a side stream that forks from and joins back into
// it, so that either launch's tail can fill with the other's CTAs.
extern "C" int polymul_ragged_run(polymul_ragged_batch* b, const void* a, const void* bb, void* c, void* stream) {
  clear_error();
  TraceRange trace_("polymul_ragged_run");
  int rc = ragged_check(b, a, bb, c);
  if (rc != POLYMUL_OK || b->n_items == 0) return rc;
  set_operands(b, a, bb, c);
  cudaStream_t st = (cudaStream_t)stream;
  const bool both = b->part_units[0] && b->part_units[1];
  if (both) {
    PM_CUDA(cudaEventRecord(b->ev_fork, st));
    PM_CUDA(cudaStreamWaitEvent(b->side, b->ev_fork, 0));
  }
  for (int i = 1; i >= 0; --i) {
    if (!b->part_units[i]) continue;
    cudaStream_t s = (both && i == 0) ? b->side : st;
    PM_CUDA(launch_part(b, i, s));
  }
  if (both) {
    PM_CUDA(cudaEventRecord(b->ev_join, b->side));
    PM_CUDA(cudaStreamWaitEvent(st, b->ev_join, 0));
  }
  // classes on the tensor path: one tiled launch each, behind the NTT ones
  for (int cls = kRaggedClasses - 1; cls >= 0; --cls)
    if (tensor_class(b, cls)) PM_CUDA(launch_tensor(b, cls, st));
  return POLYMUL_OK;
}

// The same launches, recorded once as a CUDA graph of one or two independent
// kernel nodes and replayed; a change of operand pointers updates the nodes
// in place.
extern "C" int polymul_ragged_run_graph(polymul_ragged_batch* b, const void* a, const void* bb, void* c,
                                        void* stream) {
  clear_error();
  TraceRange trace_("polymul_ragged_run_graph");
  int rc = ragged_check(b, a, bb, c);
  if (rc != POLYMUL_OK || b->n_items == 0) return rc;
  set_operands(b, a, bb, c);
  cudaKernelNodeParams kp[2];
  void* argv[2][1] = {{part_args(b, 0)}, {part_args(b, 1)}};
  for (int i = 0; i < 2; ++i) {
    memset(&kp[i], 0, sizeof kp[i]);
    const KernelInfo& ki = ragged_kernel(b, i);
    kp[i].func = const_cast<void*>(ki.fn);
    kp[i].gridDim = dim3(ragged_grid(b, i));
    kp[i].blockDim = dim3(ki.block);
    kp[i].sharedMemBytes = ki.smem;
    kp[i].kernelParams = argv[i];
  }
  // the tensor classes' launches: independent nodes as well
  cudaKernelNodeParams tp[kRaggedClasses];
  void* targv[kRaggedClasses][1];
  for (int i = 0; i < kRaggedClasses; ++i) {
    memset(&tp[i], 0, sizeof tp[i]);
    if (!tensor_class(b, i)) continue;
    const KernelInfo& ki = b->ctx->tki[i];
    targv[i][0] = &b->targs[i];
    tp[i].func = const_cast<void*>(ki.fn);
    tp[i].gridDim = dim3(tensor_grid(b, i));
    tp[i].blockDim = dim3(ki.block);
    tp[i].sharedMemBytes = ki.smem;
    tp[i].kernelParams = targv[i];
  }
  if (!b->exec) {
    PM_CUDA(cudaGraphCreate(&b->graph, 0));
    for (int i = 1; i >= 0; --i)
      if (b->part_units[i]) PM_CUDA(cudaGraphAddKernelNode(&b->node[i], b->graph, nullptr, 0, &kp[i]));
    for (int i = kRaggedClasses - 1; i >= 0; --i)
      if (tensor_class(b, i)) PM_CUDA(cudaGraphAddKernelNode(&b->tnode[i], b->graph, nullptr, 0, &tp[i]));
    PM_CUDA(cudaGraphInstantiate(&b->exec, b->graph, 0));
  } else {
    for (int i = 0; i < 2; ++i)
      if (b->node[i]) PM_CUDA(cudaGraphExecKernelNodeSetParams(b->exec, b->node[i], &kp[i]));
    for (int i = 0; i < kRaggedClasses; ++i)
      if (b->tnode[i]) PM_CUDA(cudaGraphExecKernelNodeSetParams(b->exec, b->tnode[i], &tp[i]));
  }
  PM_CUDA(cudaGraphLaunch(b->exec, (cudaStream_t)stream));
  return POLYMUL_OK;
}

extern "C" int polymul_ragged_status(polymul_ragged_batch* b, void* stream) {
  clear_error();
  if (!b) return fail(POLYMUL_EINVAL, "batch is NULL");
  PM_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  int h = 0;
  PM_CUDA(cudaMemcpy(&h, b->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (!h) return POLYMUL_OK;
  PM_CUDA(cudaMemset(b->d_err, 0, sizeof(int)));
  PM_CUDA(cudaMemset(b->d_ctr, 0, 2 * (kRaggedMaxSegs + 1) * sizeof(unsigned long long)));
  PM_CUDA(cudaMemset(b->d_tctr, 0, 2 * kRaggedClasses * sizeof(unsigned long long)));
  return fail(POLYMUL_ETIMEOUT, "a device wait expired; results of the affected launches are invalid");
}

extern "C" int polymul_ragged_batch_info(const polymul_ragged_batch* b, uint64_t* units, uint64_t* items,
                                         uint32_t* grid) {
  clear_error();
  if (!b) return fail(POLYMUL_EINVAL, "batch is NULL");
  if (units) *units = b->n_units;
  if (items) *items = b->n_items;
  if (grid) *grid = (uint32_t)std::max(b->part_units[0] ? ragged_grid(b, 0) : 0, b->part_units[1] ? ragged_grid(b, 1) : 0);
  return POLYMUL_OK;
}

// The shape set of each of the list's launches, by measurement on the
// caller's operands (Sec. 2.6 leaves the shapes to experiment): each launch
// alone, with each set, three timed rounds after a warm-up, the minimum per
// set.  The graph, if any, is rebuilt on its next replay.  Synchronous.
extern "C" int polymul_ragged_tune(polymul_ragged_batch* b, const void* a, const void* bb, void* c, void* stream,
                                   uint32_t* choice) {
  clear_error();
  TraceRange trace_("polymul_ragged_tune");
  int rc = ragged_check(b, a, bb, c);
  if (rc != POLYMUL_OK) return rc;
  PM_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  b->tensor_mask = 0;  // shape sets first, on every class's NTT segment
  apply_paths(b);
  set_operands(b, a, bb, c);
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  PM_CUDA(cudaEventCreate(&e0));
  PM_CUDA(cudaEventCreate(&e1));
  for (int part = 0; part < 2 && rc == POLYMUL_OK; ++part) {
    if (!b->part_units[part]) continue;
    float best[kRaggedSets];
    for (int set = 0; set < kRaggedSets; ++set) best[set] = 1e30f;
    for (int round = 0; round < 4 && rc == POLYMUL_OK; ++round) {
      for (int set = 0; set < kRaggedSets && rc == POLYMUL_OK; ++set) {
        b->set[part] = set;
        cudaError_t e = cudaEventRecord(e0, st);
        if (e == cudaSuccess) e = launch_part(b, part, st);
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) rc = cuda_fail(e, "ragged tuning launch");
        if (round > 0 && ms < best[set]) best[set] = ms;  // round 0 warms up
      }
    }
    int pick = 0;
    for (int set = 1; set < kRaggedSets; ++set)
      if (best[set] < best[pick]) pick = set;
    b->set[part] = pick;
  }
  // then the path of each degree class: its NTT segment alone (a one-segment
  // launch of its kernel, shape set as chosen) against its tensor launch
  auto time_launch = [&](auto&& launch_one) -> float {
    float best = 1e30f;
    for (int round = 0; round < 4 && rc == POLYMUL_OK; ++round) {
      cudaError_t e = cudaEventRecord(e0, st);
      if (e == cudaSuccess) e = launch_one();
      if (e == cudaSuccess) e = cudaEventRecord(e1, st);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e != cudaSuccess) rc = cuda_fail(e, "ragged tuning launch");
      if (round > 0 && ms < best) best = ms;
    }
    return best;
  };
  uint32_t mask = 0;
  for (const RaggedItem& it : b->items_h) {
    const int cls = (int)it.logn - 10;
    if (rc != POLYMUL_OK || !b->ctx->tensor_ok[cls]) continue;
    const int part = it.logn == 14 ? 1 : 0;
    if (cudaMemcpy(b->d_item1, &it, sizeof it, cudaMemcpyHostToDevice) != cudaSuccess) {
      rc = fail(POLYMUL_ECUDA, "ragged tuning segment");
      break;
    }
    RaggedArgs one = b->args[part];
    one.items = b->d_item1;
    one.n_items = 1;
    const KernelInfo& ki = ragged_kernel(b, part);
    const int grid = (int)std::min<uint64_t>((uint64_t)b->ctx->grid_cap[b->set[part]][part],
                                             std::max<uint32_t>(1u, it.count));
    // the 2^14 launch holds the 2^14 class alone: time it as it runs
    const float t_ntt = time_launch([&]() {
      if (part == 1) return launch_part(b, 1, st);
      void* argv[] = {&one};
      return cudaLaunchKernel(ki.fn, grid, ki.block, argv, ki.smem, st);
    });
    const float t_tc = time_launch([&]() { return launch_tensor(b, cls, st); });
    if (t_tc < t_ntt) mask |= 1u << cls;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != POLYMUL_OK) return rc;
  b->tensor_mask = mask;
  apply_paths(b);
  drop_graph(b);
  if (choice) *choice = (uint32_t)b->set[0] | ((uint32_t)b->set[1] << 1) | (mask << 2);
  return polymul_ragged_status(b, stream);
}

extern "C" int polymul_ragged_select(polymul_ragged_batch* b, uint32_t choice) {
  clear_error();
  if (!b) return fail(POLYMUL_EINVAL, "batch is NULL");
  if (choice >= (4u << kRaggedClasses)) return fail(POLYMUL_EINVAL, "choice=%u must be below %u", choice, 4u << kRaggedClasses);
  const uint32_t mask = (choice >> 2) & b->present;
  for (int cls = 0; cls < kRaggedClasses; ++cls)
    if (((mask >> cls) & 1u) && !b->ctx->tensor_ok[cls])
      return fail(POLYMUL_EINVAL, "degree 2^%d has no tensor kernel for this pool", 10 + cls);
  // the NTT launches' segment list is rewritten: let every launch finish
  PM_CUDA(cudaDeviceSynchronize());
  b->set[0] = (int)(choice & 1u);
  b->set[1] = (int)((choice >> 1) & 1u);
  b->tensor_mask = mask;
  apply_paths(b);
  drop_graph(b);
  return POLYMUL_OK;
}

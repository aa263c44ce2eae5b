// Autotuner: choose a plan's kernel by measurement (polymul_tune).
//
// The paper picks its matrix dimensions by experiment (Sec. 2.6, "matrix
// dimension selection"); here the experiment is automated: each candidate
// kernel of a plan (the NTT with 16, 32 or 8 coefficients per thread per
// operand, and the tensor path where the shape allows it) runs on a batch
// of the requested size, and the fastest is kept.  Results are cached per
// (GPU, word, n, k, mode, modulus bits, batch bucket) in the process and,
// if POLYMUL_TUNE_CACHE names a file, on disk as "key<TAB>label" lines.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/polymul.h"
#include "kernels.h"
#include "trace.h"
#include "plan.h"

using namespace pm;

namespace {

std::mutex g_tune_mu;
std::map<std::string, std::string> g_tune_cache;
bool g_tune_loaded = false;

std::string cache_path() {
  const char* p = getenv("POLYMUL_TUNE_CACHE");
  return p ? std::string(p) : std::string();
}

void load_cache() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  const std::string path = cache_path();
  if (path.empty()) return;
  std::ifstream f(path);
  std::string line;
  while (std::getline(f, line)) {
    const size_t tab = line.find('\t');
    if (tab != std::string::npos) g_tune_cache[line.substr(0, tab)] = line.substr(tab + 1);
  }
}

void store_cache(const std::string& key, const std::string& label) {
  g_tune_cache[key] = label;
  const std::string path = cache_path();
  if (path.empty()) return;
  std::ofstream f(path, std::ios::app);
  f << key << '\t' << label << '\n';
}

std::string label_of(const PlanCandidate& c) {
  if (c.path == POLYMUL_PATH_TENSOR) return c.ki.rns ? "tensor-rns" : c.ki.tiled ? "tensor-tiled" : "tensor";
  return "ntt-rb" + std::to_string(c.ki.rb) + (c.ki.cluster ? "-cluster" : "");
}

uint64_t bucket_of(uint64_t batch) {
  uint64_t b = 1;
  while (b < batch && b < (1ull << 16)) b <<= 1;
  return b;
}

}  // namespace

extern "C" int polymul_tune(polymul_plan* p, uint64_t batch, void* stream) {
  clear_error();
  TraceRange trace_("polymul_tune");
  if (!p) return fail(POLYMUL_EINVAL, "plan is NULL");
  if (batch == 0) return fail(POLYMUL_EINVAL, "batch must be positive");
  if (p->cands.size() <= 1) {
    p->tuned = true;
    p->tuned_batch = batch;
    return POLYMUL_OK;
  }
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, p->device) != cudaSuccess) return fail(POLYMUL_ECUDA, "device query failed");
  const uint64_t qmax = *std::max_element(p->q.begin(), p->q.end());
  const int qbits = 64 - __builtin_clzll(qmax);
  uint64_t bucket = bucket_of(batch);
  const size_t prod_bytes = (size_t)p->k * p->n * p->elem;
  while (bucket > 1 && 3 * bucket * prod_bytes > (1ull << 30)) bucket >>= 1;  // at most 1 GiB of scratch
  char keybuf[256];
  snprintf(keybuf, sizeof keybuf, "%s|w%u|n%u|k%u|m%d|q%d|b%llu", prop.name, p->elem, p->n, p->k, p->mode, qbits,
           (unsigned long long)bucket);
  const std::string key(keybuf);
  std::lock_guard<std::mutex> lock(g_tune_mu);
  load_cache();
  auto hit = g_tune_cache.find(key);
  if (hit != g_tune_cache.end()) {
    for (size_t i = 0; i < p->cands.size(); ++i)
      if (label_of(p->cands[i]) == hit->second) {
        apply_candidate(p, i);
        p->tuned = true;
        p->tuned_batch = bucket;
        return POLYMUL_OK;
      }
  }
  // measure every candidate on zero operands (timing does not depend on the
  // data), rotating over enough buffer sets that the operands come from
  // HBM, not L2, as they do in a stream of real batches
  cudaStream_t st = (cudaStream_t)stream;
  const size_t bytes = bucket * prod_bytes;
  int l2 = 0;
  cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, p->device);
  int nsets = (int)std::min<uint64_t>(8, (3ull * (uint64_t)l2 + 3 * bytes - 1) / (3 * bytes));
  while (nsets > 1 && (uint64_t)nsets * 3 * bytes > (1ull << 30)) --nsets;
  if (nsets < 1) nsets = 1;
  void* buf = nullptr;
  if (cudaMalloc(&buf, (size_t)nsets * 3 * bytes) != cudaSuccess)
    return fail(POLYMUL_ENOMEM, "tuning buffers (%zu bytes)", (size_t)nsets * 3 * bytes);
  auto set_ptr = [&](int i, int which) { return (char*)buf + ((size_t)(i % nsets) * 3 + which) * bytes; };
  int rc = POLYMUL_OK;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaMemsetAsync(buf, 0, (size_t)nsets * 3 * bytes, st) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess)
    rc = fail(POLYMUL_ECUDA, "tuning setup failed");
  const size_t saved_chosen = p->chosen;
  const uint32_t saved_flags = p->flags;
  p->flags &= ~POLYMUL_FLAG_VALIDATE;
  std::vector<float> best_ms(p->cands.size(), 1e30f);
  int launch_no = 0;
  auto run = [&](int times) {
    bool ok = true;
    for (int r = 0; r < times && ok; ++r, ++launch_no)
      ok = launch_batch(p, set_ptr(launch_no, 0), set_ptr(launch_no, 1), set_ptr(launch_no, 2), bucket, st, 0) ==
           POLYMUL_OK;
    return ok;
  };
  // warm-up: bring the clocks up before anything is timed (about 50 ms)
  if (rc == POLYMUL_OK) {
    apply_candidate(p, 0);
    float ms = 0;
    for (int w = 0; w < 64 && rc == POLYMUL_OK && ms < 50.f; ++w) {
      bool ok = cudaEventRecord(e0, st) == cudaSuccess && run(4) && cudaEventRecord(e1, st) == cudaSuccess &&
                cudaEventSynchronize(e1) == cudaSuccess;
      float m = 0;
      if (ok) ok = cudaEventElapsedTime(&m, e0, e1) == cudaSuccess;
      if (!ok) rc = fail(POLYMUL_ECUDA, "warm-up failed: %s", cudaGetErrorString(cudaGetLastError()));
      ms += m;
    }
  }
  // three round-robin rounds; each candidate keeps its fastest round
  for (int round = 0; round < 3 && rc == POLYMUL_OK; ++round) {
    for (size_t i = 0; rc == POLYMUL_OK && i < p->cands.size(); ++i) {
      apply_candidate(p, i);
      constexpr int kTimed = 10;
      bool ok = run(2) && cudaEventRecord(e0, st) == cudaSuccess && run(kTimed) &&
                cudaEventRecord(e1, st) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess;
      float ms = 0;
      if (ok) ok = cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
      if (!ok) {
        rc = fail(POLYMUL_ECUDA, "candidate %s failed while tuning: %s", label_of(p->cands[i]).c_str(),
                  cudaGetErrorString(cudaGetLastError()));
        break;
      }
      best_ms[i] = std::min(best_ms[i], ms);
    }
  }
  size_t best = saved_chosen;
  for (size_t i = 0; i < p->cands.size(); ++i)
    if (best_ms[i] < best_ms[best]) best = i;
  p->flags = saved_flags;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(buf);
  apply_candidate(p, rc == POLYMUL_OK ? best : saved_chosen);
  if (rc != POLYMUL_OK) return rc;
  p->tuned = true;
  p->tuned_batch = bucket;
  store_cache(key, label_of(p->cands[best]));
  return POLYMUL_OK;
}

extern "C" int polymul_plan_select(polymul_plan* p, uint32_t candidate) {
  clear_error();
  if (!p) return fail(POLYMUL_EINVAL, "plan is NULL");
  if (candidate >= p->cands.size())
    return fail(POLYMUL_EINVAL, "candidate %u of %zu", candidate, p->cands.size());
  apply_candidate(p, candidate);
  return POLYMUL_OK;
}

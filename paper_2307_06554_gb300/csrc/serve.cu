// Serving: a continuously batching request loop for mixed-size negacyclic
// products (polymul_server_*, see include/polymul.h).
//
// State kept resident for the server's lifetime (the paper's advice to keep
// prepared operands loaded rather than rebuild them per product, Sec. 4,
// "fine-tuning the design" (i)): forward and inverse twiddle tables of every
// pool prime at the largest degree (a product of degree n reads the length-n
// prefix), and the per-degree constants.
//
// Requests carry host operands.  A server thread owns the device: it admits
// queued requests in arrival order as soon as device memory (a first-fit
// arena) and an in-flight slot are free, issues each one on the stream lane
// with the least work in flight -- copy in, one kernel over the request's
// (prime) units, copy
// out, completion event -- and retires requests whose event has fired,
// releasing their memory to the next admissions.  Work of different requests
// overlaps on the device (lanes are independent streams), and copies of one
// request overlap kernels of others (Sec. 4, "optimizing computation and
// I/O" (ii)).  A request whose a, b and c lie in page-locked host memory the
// device maps takes the direct route instead: its kernel loads a and b and
// stores c in host memory itself over the coherent host link, with no arena
// memory, copy or copy stream (the batch kernel's direct form below 2^14;
// the cluster kernels load and store with plain accesses already).  Latency
// is taken from submission to the moment the server observes completion.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/polymul.h"
#include "host_math.h"
#include "toeplitz_u64.h"
#include "kernels.h"
#include "trace.h"
#include "plan.h"
#include "polymul_types.h"

using namespace pm;

namespace {

using Clock = std::chrono::steady_clock;

double now_s() { return std::chrono::duration<double>(Clock::now().time_since_epoch()).count(); }

constexpr int kServeMaxLog = 16;
constexpr size_t kArenaAlign = 256;

struct ServeReq {
  uint64_t ticket = 0;
  uint32_t n = 0, k = 0, logn = 0;
  std::vector<uint32_t> primes;
  const void* ha = nullptr;
  const void* hb = nullptr;
  void* hc = nullptr;
  double t_submit = 0, t_admit = 0, t_done = 0;
  int state = 0;  // 0 queued, 1 in flight, 2 done, 3 failed (CUDA error), 4 failed (device wait expired)
  int outcome = 0;  // the state it will take, decided by the server thread before it publishes it
  size_t off = 0, bytes = 0;
  int lane = 0;
  int slot = -1;  // page-locked word that receives the lane's error word after the kernel
  bool tensor = false;  // runs on the tensor path (decided at submission)
  // direct route (decided at submission): a, b, c are mapped page-locked
  // host memory, read and written in place at these device addresses
  bool direct = false;
  const void* da = nullptr;
  const void* db = nullptr;
  void* dc = nullptr;
  size_t weight = 0;  // bytes the request moves (lane balancing)
  cudaEvent_t ev = nullptr;     // the result is in host memory (end of the copy-out stage)
  cudaEvent_t ev_in = nullptr;  // operands are on the device (end of the copy-in stage)
  cudaEvent_t ev_k = nullptr;   // the kernel is done
};

}  // namespace

struct polymul_server {
  uint32_t nmax = 0, lognmax = 0;
  std::vector<uint64_t> pool;
  void* d_twf = nullptr;
  void* d_twi = nullptr;
  void* d_pc = nullptr;  // PrimeConst<uint64_t>[pool][17]
  KernelInfo ki[kServeMaxLog + 1];
  int grid_cap[kServeMaxLog + 1] = {};
  // the direct route's kernel per degree: the batch kernel's direct form
  // below 2^14, the cluster kernel (ki) from there
  KernelInfo dki[kServeMaxLog + 1];
  int dgrid_cap[kServeMaxLog + 1] = {};
  std::atomic<int> staged{0};  // polymul_server_set_route: 1 keeps every request on copies
  // the tensor path (polymul_server_set_path): the 64-bit-word digit kernel
  // per degree 2^10 .. n_max and the pool's digit-weight constants, set up
  // once by the first switch; `tensor` is read by the server thread at issue
  std::atomic<int> tensor{0};
  std::mutex tensor_mu;  // serialises the set-up
  bool tensor_ready = false;
  KernelInfo tki[kServeMaxLog + 1];
  TiledCfg tcfg[kServeMaxLog + 1];
  int tgrid_cap[kServeMaxLog + 1] = {};
  void* d_tp64 = nullptr;
  int device = 0, num_sms = 0;
  int nlanes = 0;
  // each lane is a three-stage pipeline: copies in, kernels, copies out, on
  // streams of their own joined by events, so that a request's copies in do
  // not wait for the previous request's kernel and copy out on the lane
  std::vector<cudaStream_t> lanes, lanes_in, lanes_out;
  unsigned long long* d_ctr = nullptr;  // 2 per lane
  int* d_err = nullptr;                 // one error word per lane
  int* h_err = nullptr;                 // page-locked, one per in-flight slot
  // where the device supports native atomics on host memory, h_err is also
  // mapped into the device's address space (d_err_mapped): each request's
  // kernel reports into its slot's word directly, with no copy or reset on
  // the lane; otherwise the lane's device word is copied back and cleared
  int* d_err_mapped = nullptr;
  // page-locked staging of each in-flight slot's prime-index map (pool size
  // words per slot): a copy from pageable memory would first wait for the
  // lane's stream to drain, stalling the server thread behind large requests
  uint32_t* h_map = nullptr;
  std::vector<int> free_slots;
  char* d_arena = nullptr;
  size_t arena_bytes = 0, arena_used = 0, arena_peak = 0;
  std::map<size_t, size_t> free_list;  // offset -> size
  size_t max_inflight = 64;
  // shared with submitting and waiting threads, under `mu`: the submission
  // queue, the tickets, the published states and statistics
  std::mutex mu;
  std::condition_variable cv;
  std::deque<ServeReq*> queue;
  std::unordered_map<uint64_t, ServeReq*> reqs;
  std::vector<double> latencies_us, queue_us, service_us;
  double issue_s = 0, loop_busy_s = 0;  // server-thread time issuing requests, and in passes that did work
  uint64_t issued = 0;
  uint64_t next_ticket = 1, submitted = 0, completed = 0, failed = 0, completed_direct = 0;
  size_t published_inflight = 0, published_pending = 0;
  // owned by the server thread alone (no lock): requests taken from the
  // queue and not yet admitted, the requests in flight on each lane in issue
  // order (a lane is one stream, so they complete in that order), the
  // arena, slots, events and lane loads
  std::deque<ServeReq*> pending;
  std::vector<std::deque<ServeReq*>> lane_fifo;
  size_t inflight = 0;
  std::vector<cudaEvent_t> event_pool;
  std::vector<uint64_t> lane_bytes;  // bytes of the requests in flight on each lane
  std::atomic<bool> stop{false};
  std::thread loop;
  int cuda_error = 0;
  std::string cuda_error_msg;
};

namespace {

size_t arena_alloc(polymul_server* s, size_t bytes) {
  bytes = (bytes + kArenaAlign - 1) / kArenaAlign * kArenaAlign;
  for (auto it = s->free_list.begin(); it != s->free_list.end(); ++it) {
    if (it->second >= bytes) {
      const size_t off = it->first, rest = it->second - bytes;
      s->free_list.erase(it);
      if (rest) s->free_list[off + bytes] = rest;
      s->arena_used += bytes;
      s->arena_peak = std::max(s->arena_peak, s->arena_used);
      return off;
    }
  }
  return (size_t)-1;
}

void arena_free(polymul_server* s, size_t off, size_t bytes) {
  bytes = (bytes + kArenaAlign - 1) / kArenaAlign * kArenaAlign;
  s->arena_used -= bytes;
  auto it = s->free_list.emplace(off, bytes).first;
  auto next = std::next(it);
  if (next != s->free_list.end() && it->first + it->second == next->first) {
    it->second += next->second;
    s->free_list.erase(next);
  }
  if (it != s->free_list.begin()) {
    auto prev = std::prev(it);
    if (prev->first + prev->second == it->first) {
      prev->second += it->second;
      s->free_list.erase(it);
    }
  }
}

size_t request_bytes(uint32_t n, uint32_t k) {
  const size_t row = (size_t)k * n * 8;
  const size_t map = ((size_t)k * 4 + kArenaAlign - 1) / kArenaAlign * kArenaAlign;
  return 3 * ((row + kArenaAlign - 1) / kArenaAlign * kArenaAlign) + map;
}

// after a request's kernel: its error word, the copy out and the
// completion event (server thread)
cudaError_t finish_issue(polymul_server* s, ServeReq* r, uint64_t* dc, size_t row, int* lane_err) {
  cudaStream_t st = s->lanes[r->lane], st_out = s->lanes_out[r->lane];
  cudaError_t e;
  if (!s->d_err_mapped) {
    // the lane's error word belongs to this request until the lane's next
    // kernel: bring it back, then clear it, in the kernel stage
    if ((e = cudaMemcpyAsync(s->h_err + r->slot, lane_err, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
      return e;
    if ((e = cudaMemsetAsync(lane_err, 0, sizeof(int), st)) != cudaSuccess) return e;
  }
  if ((e = cudaEventRecord(r->ev_k, st)) != cudaSuccess) return e;
  if ((e = cudaStreamWaitEvent(st_out, r->ev_k, 0)) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(r->hc, dc, row, cudaMemcpyDeviceToHost, st_out)) != cudaSuccess) return e;
  return cudaEventRecord(r->ev, st_out);
}

// one launch of an NTT kernel over `units` units on stream st: a cluster
// launch for the cluster kernels, else a persistent grid of at most `cap`
cudaError_t launch_ntt(const KernelInfo& ki, int cap, uint32_t units, void** argv, cudaStream_t st) {
  if (ki.cluster > 0) {
    const int clusters = std::min<int>((int)units, cap / ki.cluster);
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof cfg);
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = ki.cluster;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.gridDim = dim3(clusters * ki.cluster);
    cfg.blockDim = dim3(ki.block);
    cfg.dynamicSmemBytes = ki.smem;
    cfg.stream = st;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, ki.fn, argv);
  }
  const int grid = std::min<int>((int)((units + ki.units_per_cta - 1) / ki.units_per_cta), cap);
  return cudaLaunchKernel(ki.fn, grid, ki.block, argv, ki.smem, st);
}

// The prime map rides in the launch's arguments when it fits (up to 32
// primes of a pool of at most 256), else it is copied to the arena.
bool inline_map(const polymul_server* s, uint32_t k) { return k <= 32 && s->pool.size() <= 256; }

// direct route: the kernel on the lane's kernel stream reads a and b and
// writes c in host memory; then its error word and the completion event
// (server thread)
cudaError_t issue_direct(polymul_server* s, ServeReq* r) {
  cudaStream_t st = s->lanes[r->lane];
  cudaError_t e;
  uint32_t* dmap = nullptr;
  if (!inline_map(s, r->k)) {
    dmap = reinterpret_cast<uint32_t*>(s->d_arena + r->off);
    uint32_t* hmap = s->h_map + (size_t)r->slot * s->pool.size();
    std::copy(r->primes.begin(), r->primes.end(), hmap);
    if ((e = cudaMemcpyAsync(dmap, hmap, r->k * 4, cudaMemcpyHostToDevice, st)) != cudaSuccess) return e;
  }
  int* lane_err = s->d_err + r->lane;
  int* err = s->d_err_mapped ? s->d_err_mapped + r->slot : lane_err;
  NttBatchArgs<uint64_t> args{(const uint64_t*)r->da, (const uint64_t*)r->db, (uint64_t*)r->dc, s->d_twf, s->d_twi,
                              (const PrimeConst<uint64_t>*)s->d_pc, r->k, r->k, s->d_ctr + 2 * r->lane, err,
                              nullptr, dmap, s->nmax, (uint32_t)(kServeMaxLog + 1), r->logn, 0u, 0u, 0u};
  if (!dmap) {
    args.pmap_inline = 1;
    for (uint32_t i = 0; i < r->k; ++i) args.pmap_pack[i >> 2] |= r->primes[i] << (8 * (i & 3));
  }
  void* argv[] = {&args};
  if ((e = launch_ntt(s->dki[r->logn], s->dgrid_cap[r->logn], r->k, argv, st)) != cudaSuccess) return e;
  if (!s->d_err_mapped) {
    if ((e = cudaMemcpyAsync(s->h_err + r->slot, lane_err, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
      return e;
    if ((e = cudaMemsetAsync(lane_err, 0, sizeof(int), st)) != cudaSuccess) return e;
  }
  return cudaEventRecord(r->ev, st);
}

// issue copy-in, kernel, copy-out and the completion event (server thread)
cudaError_t issue(polymul_server* s, ServeReq* r) {
  if (r->direct) return issue_direct(s, r);
  const size_t row = (size_t)r->k * r->n * 8;
  const size_t rowa = (row + kArenaAlign - 1) / kArenaAlign * kArenaAlign;
  char* base = s->d_arena + r->off;
  uint64_t* da = reinterpret_cast<uint64_t*>(base);
  uint64_t* db = reinterpret_cast<uint64_t*>(base + rowa);
  uint64_t* dc = reinterpret_cast<uint64_t*>(base + 2 * rowa);
  uint32_t* dmap = reinterpret_cast<uint32_t*>(base + 3 * rowa);
  cudaStream_t st = s->lanes[r->lane], st_in = s->lanes_in[r->lane], st_out = s->lanes_out[r->lane];
  cudaError_t e;
  const bool inline_map = ::inline_map(s, r->k);
  if (!inline_map) {
    uint32_t* hmap = s->h_map + (size_t)r->slot * s->pool.size();
    std::copy(r->primes.begin(), r->primes.end(), hmap);
    if ((e = cudaMemcpyAsync(dmap, hmap, r->k * 4, cudaMemcpyHostToDevice, st_in)) != cudaSuccess) return e;
  }
  if ((e = cudaMemcpyAsync(da, r->ha, row, cudaMemcpyHostToDevice, st_in)) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(db, r->hb, row, cudaMemcpyHostToDevice, st_in)) != cudaSuccess) return e;
  if ((e = cudaEventRecord(r->ev_in, st_in)) != cudaSuccess) return e;
  if ((e = cudaStreamWaitEvent(st, r->ev_in, 0)) != cudaSuccess) return e;
  int* lane_err = s->d_err + r->lane;
  int* err = s->d_err_mapped ? s->d_err_mapped + r->slot : lane_err;
  if (r->tensor) {
    // the tensor path: the 64-bit-word digit kernel over the request's k
    // rows, its prime map in the arena
    if (inline_map) {
      uint32_t* hmap = s->h_map + (size_t)r->slot * s->pool.size();
      std::copy(r->primes.begin(), r->primes.end(), hmap);
      if ((e = cudaMemcpyAsync(dmap, hmap, r->k * 4, cudaMemcpyHostToDevice, st)) != cudaSuccess) return e;
    }
    const TiledCfg& tc = s->tcfg[r->logn];
    const KernelInfo& tk = s->tki[r->logn];
    const uint64_t tunits = (uint64_t)r->k * tc.ngrp;
    TensorU64Args targs{da, db, dc, (const TensorPrime64*)s->d_tp64, dmap, tunits, r->k, 0x80008000u, r->logn,
                        tc.ngrp, tc.kc, tc.a_win, tc.bt_off, tc.tmem_cols, s->d_ctr + 2 * r->lane, err};
    void* targv[] = {&targs};
    const int tgrid = (int)std::min<uint64_t>(tunits, (uint64_t)s->tgrid_cap[r->logn]);
    if ((e = cudaLaunchKernel(tk.fn, tgrid, tk.block, targv, tk.smem, st)) != cudaSuccess) return e;
    return finish_issue(s, r, dc, row, lane_err);
  }
  const KernelInfo& ki = s->ki[r->logn];
  uint32_t tx_pad = 0, polls = 0;
  if (ki.cluster == 0) take_injected_wait(&tx_pad, &polls);
  NttBatchArgs<uint64_t> args{da,      db,       dc,      s->d_twf, s->d_twi, (const PrimeConst<uint64_t>*)s->d_pc,
                              r->k,    r->k,     s->d_ctr + 2 * r->lane, err, nullptr, inline_map ? nullptr : dmap,
                              s->nmax, (uint32_t)(kServeMaxLog + 1), r->logn, 0u, tx_pad, polls};
  if (inline_map) {
    args.pmap_inline = 1;
    for (uint32_t i = 0; i < r->k; ++i) args.pmap_pack[i >> 2] |= r->primes[i] << (8 * (i & 3));
  }
  void* argv[] = {&args};
  if ((e = launch_ntt(ki, s->grid_cap[r->logn], r->k, argv, st)) != cudaSuccess) return e;
  return finish_issue(s, r, dc, row, lane_err);
}

void take_events(polymul_server* s, ServeReq* r) {
  cudaEvent_t* evs[3] = {&r->ev, &r->ev_in, &r->ev_k};
  for (cudaEvent_t* ev : evs) {
    if (s->event_pool.empty()) {
      cudaEvent_t e;
      cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
      s->event_pool.push_back(e);
    }
    *ev = s->event_pool.back();
    s->event_pool.pop_back();
  }
}

void release_events(polymul_server* s, ServeReq* r) {
  cudaEvent_t* evs[3] = {&r->ev, &r->ev_in, &r->ev_k};
  for (cudaEvent_t* ev : evs) {
    if (*ev) s->event_pool.push_back(*ev);
    *ev = nullptr;
  }
}

// The server thread.  Each pass: take the new submissions (under the lock),
// retire what has completed, admit what fits (CUDA calls without the lock,
// so that submitters never wait behind them), then publish the outcomes
// (under the lock).  While work is in flight it polls with a yield; with
// nothing in flight and nothing queued it sleeps on the condition variable
// until a submission arrives.
void server_loop(polymul_server* s) {
  cudaSetDevice(s->device);
  std::vector<ServeReq*> done;
  std::string err_msg;
  while (!s->stop.load()) {
    bool progress = false;
    const double t_pass = now_s();
    double issue_time = 0;
    uint64_t issued = 0;
    {
      std::lock_guard<std::mutex> lock(s->mu);
      while (!s->queue.empty()) {
        s->pending.push_back(s->queue.front());
        s->queue.pop_front();
      }
    }
    // retire: only the oldest request of each lane can be the next to finish
    for (int l = 0; l < s->nlanes; ++l) {
      std::deque<ServeReq*>& f = s->lane_fifo[l];
      while (!f.empty()) {
        ServeReq* r = f.front();
        const cudaError_t q = cudaEventQuery(r->ev);
        if (q == cudaErrorNotReady) break;
        r->t_done = now_s();
        if (q != cudaSuccess) {
          r->outcome = 3;
          err_msg = cudaGetErrorString(q);
        } else {
          // a nonzero error word: a bounded device wait of the request's
          // kernel expired and its result is invalid
          r->outcome = s->h_err[r->slot] != 0 ? 4 : 2;
        }
        s->free_slots.push_back(r->slot);
        r->slot = -1;
        if (r->bytes) arena_free(s, r->off, r->bytes);
        s->lane_bytes[r->lane] -= r->weight;
        release_events(s, r);
        f.pop_front();
        --s->inflight;
        done.push_back(r);
      }
    }
    // admit in arrival order while memory and slots allow
    while (!s->pending.empty() && s->inflight < s->max_inflight) {
      ServeReq* r = s->pending.front();
      const size_t off = r->bytes ? arena_alloc(s, r->bytes) : 0;  // a direct request may need none
      if (off == (size_t)-1) break;
      r->off = off;
      // the lane with the least work in flight: a small request does not
      // queue behind a large one while another lane is idle
      int lane = 0;
      for (int l = 1; l < s->nlanes; ++l)
        if (s->lane_bytes[l] < s->lane_bytes[lane]) lane = l;
      r->lane = lane;
      s->lane_bytes[lane] += r->weight;
      take_events(s, r);
      r->slot = s->free_slots.back();  // fewer than max_inflight requests are in flight
      s->free_slots.pop_back();
      s->h_err[r->slot] = 0;
      std::atomic_thread_fence(std::memory_order_release);  // cleared before the launch that may report into it
      r->t_admit = now_s();
      const cudaError_t e = issue(s, r);
      issue_time += now_s() - r->t_admit;
      ++issued;
      s->pending.pop_front();
      if (e != cudaSuccess) {
        err_msg = cudaGetErrorString(e);
        r->outcome = 3;
        r->t_done = now_s();
        s->free_slots.push_back(r->slot);
        r->slot = -1;
        if (r->bytes) arena_free(s, r->off, r->bytes);
        s->lane_bytes[r->lane] -= r->weight;
        release_events(s, r);
        done.push_back(r);
      } else {
        s->lane_fifo[lane].push_back(r);
        ++s->inflight;
      }
      progress = true;
    }
    if (!done.empty() || progress) {
      std::lock_guard<std::mutex> lock(s->mu);
      s->issue_s += issue_time;
      s->issued += issued;
      s->loop_busy_s += now_s() - t_pass;
      for (ServeReq* r : done) {
        r->state = r->outcome;
        if (r->outcome == 2) {
          if (r->direct) ++s->completed_direct;
          s->latencies_us.push_back((r->t_done - r->t_submit) * 1e6);
          s->queue_us.push_back((r->t_admit - r->t_submit) * 1e6);
          s->service_us.push_back((r->t_done - r->t_admit) * 1e6);
          ++s->completed;
        } else {
          ++s->failed;
          if (r->outcome == 3) {
            s->cuda_error = 1;
            s->cuda_error_msg = err_msg;
          }
        }
      }
      s->published_inflight = s->inflight;
      s->published_pending = s->pending.size();
      if (!done.empty()) s->cv.notify_all();
      progress = progress || !done.empty();
      done.clear();
    }
    if (progress) continue;
    if (s->inflight == 0 && s->pending.empty()) {
      std::unique_lock<std::mutex> lock(s->mu);
      s->cv.wait_for(lock, std::chrono::milliseconds(1), [&] { return !s->queue.empty() || s->stop.load(); });
    } else {
      std::this_thread::yield();
    }
  }
}

void build_serve_prime(uint64_t q, uint32_t nmax, std::vector<uint64_t>& twf, std::vector<uint64_t>& twi,
                       PrimeConst<uint64_t>* pc17) {
  using namespace pm::host;
  const int lognmax = __builtin_ctz(nmax);
  const uint64_t psi = primitive_2n_root(q, nmax);
  const uint64_t psi_inv = powmod(psi, q - 2, q);
  for (uint32_t i = 0; i < nmax; ++i) {
    const uint32_t r = bitrev(i, lognmax);
    const uint64_t w = powmod(psi, r, q), v = powmod(psi_inv, r, q);
    twf.push_back(w);
    twf.push_back(shoup_companion(w, q, 64));
    twi.push_back(v);
    twi.push_back(shoup_companion(v, q, 64));
  }
  const uint64_t v1 = powmod(psi_inv, bitrev(1, lognmax), q);
  const uint64_t r_mod_q = (uint64_t)(((u128)1 << 64) % q);
  for (int logn = 0; logn <= kServeMaxLog; ++logn) {
    PrimeConst<uint64_t>& c = pc17[logn];
    memset(&c, 0, sizeof c);
    if (logn > lognmax) continue;
    const uint64_t scale = mulmod(powmod(1ull << logn, q - 2, q), r_mod_q, q);
    const uint64_t scale_w = mulmod(v1, scale, q);
    c.q = q;
    c.q2 = 2 * q;
    c.qinv = inv_pow2_64(q);
    c.scale = scale;
    c.scale_p = shoup_companion(scale, q, 64);
    c.scale_w = scale_w;
    c.scale_wp = shoup_companion(scale_w, q, 64);
  }
}

}  // namespace

#define PM_CUDA(call)                                       \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return pm::cuda_fail(e_, #call); \
  } while (0)

extern "C" void polymul_server_destroy(polymul_server* s) {
  if (!s) return;
  s->stop.store(true);
  s->cv.notify_all();
  if (s->loop.joinable()) s->loop.join();
  for (auto* v : {&s->lanes_in, &s->lanes, &s->lanes_out})
    for (cudaStream_t st : *v) {
      cudaStreamSynchronize(st);
      cudaStreamDestroy(st);
    }
  for (auto& kv : s->reqs) {
    for (cudaEvent_t ev : {kv.second->ev, kv.second->ev_in, kv.second->ev_k})
      if (ev) cudaEventDestroy(ev);
    delete kv.second;
  }
  for (cudaEvent_t ev : s->event_pool) cudaEventDestroy(ev);
  cudaFree(s->d_twf);
  cudaFree(s->d_twi);
  cudaFree(s->d_pc);
  cudaFree(s->d_ctr);
  cudaFree(s->d_err);
  cudaFree(s->d_arena);
  cudaFree(s->d_tp64);
  if (s->h_err) cudaFreeHost(s->h_err);
  if (s->h_map) cudaFreeHost(s->h_map);
  delete s;
}

extern "C" int polymul_server_create(const uint64_t* pool, uint32_t pool_size, uint32_t n_max,
                                     uint64_t device_bytes, uint32_t lanes, polymul_server** out) {
  clear_error();
  if (!out || !pool || pool_size == 0) return fail(POLYMUL_EINVAL, "need a prime pool and an out pointer");
  if (n_max < 16 || n_max > 65536 || (n_max & (n_max - 1)))
    return fail(POLYMUL_EINVAL, "n_max=%u must be a power of two in [16, 65536]", n_max);
  if (lanes == 0 || lanes > 32) return fail(POLYMUL_EINVAL, "lanes must be in [1, 32]");
  for (uint32_t j = 0; j < pool_size; ++j) {
    const uint64_t q = pool[j];
    if (q >= (1ull << 62) || !pm::host::is_prime(q) || (q - 1) % (2ull * n_max) != 0)
      return fail(POLYMUL_EINVAL, "pool[%u]=%llu must be a prime < 2^62 with 2 n_max | q - 1", j,
                  (unsigned long long)q);
    for (uint32_t i = 0; i < j; ++i)
      if (pool[i] == q) return fail(POLYMUL_EINVAL, "duplicate pool prime");
  }
  if (device_bytes < request_bytes(n_max, 1))
    return fail(POLYMUL_EINVAL, "device_bytes too small for one product of degree n_max");
  polymul_server* s = new polymul_server();
  s->nmax = n_max;
  s->lognmax = __builtin_ctz(n_max);
  s->pool.assign(pool, pool + pool_size);
  s->nlanes = (int)lanes;
  s->lane_bytes.assign(lanes, 0);
  s->lane_fifo.resize(lanes);
  s->max_inflight = std::max<size_t>(64, 8 * (size_t)lanes);  // enough requests to keep every lane busy
  int rc = POLYMUL_OK;
  auto bail = [&](int code) {
    std::string keep = polymul_last_error();
    polymul_server_destroy(s);
    fail(code, "%s", keep.c_str());
    return code;
  };
  std::vector<uint64_t> twf, twi;
  std::vector<PrimeConst<uint64_t>> pcs((size_t)pool_size * (kServeMaxLog + 1));
  for (uint32_t j = 0; j < pool_size; ++j)
    build_serve_prime(s->pool[j], n_max, twf, twi, &pcs[(size_t)j * (kServeMaxLog + 1)]);
  if (cudaGetDevice(&s->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, s->device) != cudaSuccess)
    return bail(cuda_fail(cudaGetLastError(), "device query"));
  if (cudaMalloc(&s->d_twf, twf.size() * 8) != cudaSuccess || cudaMalloc(&s->d_twi, twi.size() * 8) != cudaSuccess ||
      cudaMalloc(&s->d_pc, pcs.size() * sizeof(PrimeConst<uint64_t>)) != cudaSuccess ||
      cudaMalloc(&s->d_ctr, 2 * lanes * sizeof(unsigned long long)) != cudaSuccess ||
      cudaMalloc(&s->d_err, lanes * sizeof(int)) != cudaSuccess ||
      cudaMalloc(&s->d_arena, device_bytes) != cudaSuccess ||
      cudaHostAlloc(&s->h_err, s->max_inflight * sizeof(int), cudaHostAllocMapped) != cudaSuccess ||
      cudaHostAlloc(&s->h_map, s->max_inflight * pool_size * sizeof(uint32_t), cudaHostAllocDefault) != cudaSuccess)
    return bail(fail(POLYMUL_ENOMEM, "device allocation failed"));
  for (int i = (int)s->max_inflight - 1; i >= 0; --i) s->free_slots.push_back(i);
  {
    int native_atomics = 0, can_map = 0;
    cudaDeviceGetAttribute(&native_atomics, cudaDevAttrHostNativeAtomicSupported, s->device);
    cudaDeviceGetAttribute(&can_map, cudaDevAttrCanMapHostMemory, s->device);
    void* dp = nullptr;
    if (native_atomics && can_map && cudaHostGetDevicePointer(&dp, s->h_err, 0) == cudaSuccess)
      s->d_err_mapped = static_cast<int*>(dp);
    cudaGetLastError();  // a refused mapping only selects the copied error words
  }
  if (cudaMemcpy(s->d_twf, twf.data(), twf.size() * 8, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(s->d_twi, twi.data(), twi.size() * 8, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(s->d_pc, pcs.data(), pcs.size() * sizeof(PrimeConst<uint64_t>), cudaMemcpyHostToDevice) !=
          cudaSuccess ||
      cudaMemset(s->d_ctr, 0, 2 * lanes * sizeof(unsigned long long)) != cudaSuccess ||
      cudaMemset(s->d_err, 0, lanes * sizeof(int)) != cudaSuccess)
    return bail(cuda_fail(cudaGetLastError(), "table upload"));
  s->arena_bytes = device_bytes;
  s->free_list[0] = device_bytes;
  // kernels per degree (64-bit words, Harvey bounds: every pool prime < 2^62)
  for (int logn = 4; logn <= (int)s->lognmax; ++logn) {
    KernelInfo ki;
    const bool ok = logn >= 14 ? lookup_ntt_cluster2(8, logn, 1, false, &ki) : lookup_ntt_u64_m1(logn, &ki);
    if (!ok) return bail(fail(POLYMUL_ENOTSUP, "no kernel for n=2^%d", logn));
    if (ki.smem > 48 * 1024 &&
        cudaFuncSetAttribute(ki.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, ki.smem) != cudaSuccess)
      return bail(cuda_fail(cudaGetLastError(), "smem attribute"));
    int cap = 0;
    if (ki.cluster > 0) {
      cudaLaunchConfig_t cfg;
      memset(&cfg, 0, sizeof cfg);
      cudaLaunchAttribute attr;
      attr.id = cudaLaunchAttributeClusterDimension;
      attr.val.clusterDim.x = ki.cluster;
      attr.val.clusterDim.y = 1;
      attr.val.clusterDim.z = 1;
      cfg.gridDim = dim3(ki.cluster * s->num_sms);
      cfg.blockDim = dim3(ki.block);
      cfg.dynamicSmemBytes = ki.smem;
      cfg.attrs = &attr;
      cfg.numAttrs = 1;
      int clusters = 0;
      if (cudaOccupancyMaxActiveClusters(&clusters, ki.fn, &cfg) != cudaSuccess || clusters < 1)
        return bail(fail(POLYMUL_ENOTSUP, "no cluster fits for n=2^%d", logn));
      cap = clusters * ki.cluster;
    } else {
      int per_sm = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ki.fn, ki.block, ki.smem) != cudaSuccess ||
          per_sm < 1)
        return bail(fail(POLYMUL_ENOTSUP, "kernel for n=2^%d does not fit", logn));
      cap = per_sm * s->num_sms;
    }
    s->ki[logn] = ki;
    s->grid_cap[logn] = cap;
    s->dki[logn] = ki;  // the cluster kernels read and write with plain accesses
    s->dgrid_cap[logn] = cap;
    KernelInfo dk;
    if (ki.cluster == 0 && lookup_ntt_direct_u64(logn, &dk)) {
      if (dk.smem > 48 * 1024 &&
          cudaFuncSetAttribute(dk.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, dk.smem) != cudaSuccess)
        return bail(cuda_fail(cudaGetLastError(), "smem attribute"));
      int per_sm = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dk.fn, dk.block, dk.smem) != cudaSuccess || per_sm < 1)
        return bail(fail(POLYMUL_ENOTSUP, "direct kernel for n=2^%d does not fit", logn));
      s->dki[logn] = dk;
      s->dgrid_cap[logn] = s->num_sms;  // one CTA per SM, as for polymul_batch_mapped
    }
  }
  for (auto* v : {&s->lanes_in, &s->lanes, &s->lanes_out})
    for (uint32_t l = 0; l < lanes; ++l) {
      cudaStream_t st;
      if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess)
        return bail(cuda_fail(cudaGetLastError(), "stream creation"));
      v->push_back(st);
    }
  s->loop = std::thread(server_loop, s);
  *out = s;
  return rc;
}

extern "C" int polymul_server_submit(polymul_server* s, const polymul_request* q, uint64_t* ticket) {
  clear_error();
  TraceRange trace_("polymul_server_submit");
  if (!s || !q || !ticket) return fail(POLYMUL_EINVAL, "null argument");
  if (q->n < 16 || q->n > s->nmax || (q->n & (q->n - 1)))
    return fail(POLYMUL_EINVAL, "n=%u must be a power of two in [16, %u]", q->n, s->nmax);
  if (q->k == 0 || q->k > s->pool.size() || !q->prime_idx) return fail(POLYMUL_EINVAL, "bad prime list");
  if (!q->a || !q->b || !q->c) return fail(POLYMUL_EINVAL, "null operand pointer");
  for (uint32_t i = 0; i < q->k; ++i)
    if (q->prime_idx[i] >= s->pool.size()) return fail(POLYMUL_EINVAL, "prime index outside the pool");
  // the route: in place when a, b and c are mapped page-locked memory (no
  // arena but for a prime map that does not fit the launch arguments), else
  // copies through the arena
  const bool tensor = s->tensor.load(std::memory_order_acquire) != 0 && q->n >= 1024 &&
                      s->tgrid_cap[__builtin_ctz(q->n)] > 0;
  const size_t row = (size_t)q->k * q->n * 8;
  void *da = nullptr, *db = nullptr, *dc = nullptr;
  if (!tensor && s->staged.load(std::memory_order_acquire) == 0 &&
      (((uintptr_t)q->a | (uintptr_t)q->b | (uintptr_t)q->c) & 7) == 0) {
    da = mapped_host_range(q->a, row);
    db = da ? mapped_host_range(q->b, row) : nullptr;
    dc = db ? mapped_host_range(q->c, row) : nullptr;
  }
  const bool direct = dc != nullptr;
  const size_t bytes = !direct ? request_bytes(q->n, q->k)
                       : inline_map(s, q->k) ? 0
                                             : ((size_t)q->k * 4 + kArenaAlign - 1) / kArenaAlign * kArenaAlign;
  if (bytes > s->arena_bytes) return fail(POLYMUL_EINVAL, "request larger than the server's device memory");
  ServeReq* r = new ServeReq();
  r->n = q->n;
  r->k = q->k;
  r->logn = (uint32_t)__builtin_ctz(q->n);
  r->tensor = tensor;
  r->primes.assign(q->prime_idx, q->prime_idx + q->k);
  r->ha = q->a;
  r->hb = q->b;
  r->hc = q->c;
  r->direct = direct;
  r->da = da;
  r->db = db;
  r->dc = dc;
  r->bytes = bytes;
  r->weight = direct ? 3 * row : bytes;
  r->t_submit = now_s();
  {
    std::lock_guard<std::mutex> lock(s->mu);
    r->ticket = s->next_ticket++;
    s->reqs[r->ticket] = r;
    s->queue.push_back(r);
    ++s->submitted;
  }
  s->cv.notify_all();
  *ticket = r->ticket;
  return POLYMUL_OK;
}

// 1: done (and forgotten), 0: pending, <0 failure code
static int take_if_done(polymul_server* s, uint64_t ticket) {
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return -POLYMUL_EINVAL;
  ServeReq* r = it->second;
  if (r->state < 2) return 0;
  const int st = r->state;
  delete r;
  s->reqs.erase(it);
  return st == 2 ? 1 : st == 4 ? -POLYMUL_ETIMEOUT : -POLYMUL_ECUDA;
}

static int request_failure(polymul_server* s, int code, uint64_t ticket) {
  if (code == POLYMUL_EINVAL) return fail(code, "unknown ticket %llu", (unsigned long long)ticket);
  if (code == POLYMUL_ETIMEOUT)
    return fail(code, "request %llu: a bounded device wait of its kernel expired; its result is invalid",
                (unsigned long long)ticket);
  return fail(code, "request %llu failed: %s", (unsigned long long)ticket, s->cuda_error_msg.c_str());
}

// Requests submitted after this call run on `path`: POLYMUL_PATH_NTT (the
// default) or POLYMUL_PATH_TENSOR (the 64-bit-word digit kernel, Sec. 2.2
// matrix form, for degrees 2^10 .. n_max; smaller degrees stay on the NTT
// path).  The first switch to the tensor path sets up its kernels and the
// pool's constants (synchronous).
extern "C" int polymul_server_set_path(polymul_server* s, uint32_t path) {
  clear_error();
  if (!s) return fail(POLYMUL_EINVAL, "server is NULL");
  if (path != POLYMUL_PATH_NTT && path != POLYMUL_PATH_TENSOR)
    return fail(POLYMUL_EINVAL, "path=%u must be POLYMUL_PATH_NTT or POLYMUL_PATH_TENSOR", path);
  if (path == POLYMUL_PATH_NTT) {
    s->tensor.store(0, std::memory_order_release);
    return POLYMUL_OK;
  }
  std::lock_guard<std::mutex> lk(s->tensor_mu);
  if (!s->tensor_ready) {
    if (s->lognmax < 10) return fail(POLYMUL_ENOTSUP, "the tensor path needs n_max >= 1024");
    const uint64_t qmax = *std::max_element(s->pool.begin(), s->pool.end());
    const int L = std::max(5, u64_digits(qmax));  // at least the smallest instantiated digit count
    std::vector<TensorPrime64> tp(s->pool.size());
    for (size_t j = 0; j < s->pool.size(); ++j) {
      const uint64_t q = s->pool[j];
      memset(&tp[j], 0, sizeof tp[j]);
      tp[j].q = q;
      tp[j].bias = ((1ull << 28) + q - 1) / q * q;
      for (int e = 0; e < 15; ++e) {
        tp[j].pw[e] = pm::host::powmod(2, 8ull * e, q);
        tp[j].pwp[e] = (uint64_t)(((pm::host::u128)tp[j].pw[e] << 64) / q);
      }
    }
    if (cudaMalloc(&s->d_tp64, tp.size() * sizeof(TensorPrime64)) != cudaSuccess)
      return fail(POLYMUL_ENOMEM, "tensor constants");
    if (cudaMemcpy(s->d_tp64, tp.data(), tp.size() * sizeof(TensorPrime64), cudaMemcpyHostToDevice) != cudaSuccess)
      return cuda_fail(cudaGetLastError(), "tensor constants");
    for (int logn = 10; logn <= (int)s->lognmax; ++logn) {
      KernelInfo ki;
      if (!lookup_toeplitz_u64(logn, L, &ki) || !toeplitz_u64_config(logn, L, &s->tcfg[logn])) continue;
      if (cudaFuncSetAttribute(ki.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, ki.smem) != cudaSuccess)
        return cuda_fail(cudaGetLastError(), "smem attribute");
      int per_sm = 0;
      const int rc = tmem_kernel_per_sm(ki, s->device, &per_sm);
      if (rc != POLYMUL_OK) return rc;
      if (per_sm < 1) continue;
      s->tki[logn] = ki;
      s->tgrid_cap[logn] = per_sm * s->num_sms;
    }
    s->tensor_ready = true;
  }
  s->tensor.store(1, std::memory_order_release);
  return POLYMUL_OK;
}

// Requests submitted after this call: POLYMUL_ROUTE_DIRECT (the default:
// operands in mapped page-locked host memory are read and written in place)
// or POLYMUL_ROUTE_STAGED (always copies through the arena).
extern "C" int polymul_server_set_route(polymul_server* s, uint32_t route) {
  clear_error();
  if (!s) return fail(POLYMUL_EINVAL, "server is NULL");
  if (route != POLYMUL_ROUTE_DIRECT && route != POLYMUL_ROUTE_STAGED)
    return fail(POLYMUL_EINVAL, "route=%u must be POLYMUL_ROUTE_DIRECT or POLYMUL_ROUTE_STAGED", route);
  s->staged.store(route == POLYMUL_ROUTE_STAGED ? 1 : 0, std::memory_order_release);
  return POLYMUL_OK;
}

extern "C" int polymul_server_poll(polymul_server* s, uint64_t ticket, int* done) {
  clear_error();
  if (!s || !done) return fail(POLYMUL_EINVAL, "null argument");
  std::lock_guard<std::mutex> lock(s->mu);
  const int r = take_if_done(s, ticket);
  if (r < 0) return request_failure(s, -r, ticket);
  *done = r;
  return POLYMUL_OK;
}

extern "C" int polymul_server_wait(polymul_server* s, uint64_t ticket, double timeout_s) {
  clear_error();
  if (!s) return fail(POLYMUL_EINVAL, "server is NULL");
  const auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(timeout_s));
  std::unique_lock<std::mutex> lock(s->mu);
  for (;;) {
    const int r = take_if_done(s, ticket);
    if (r < 0) return request_failure(s, -r, ticket);
    if (r == 1) return POLYMUL_OK;
    if (s->cv.wait_until(lock, deadline) == std::cv_status::timeout && Clock::now() >= deadline)
      return fail(POLYMUL_ETIMEOUT, "request %llu not finished within %.3f s", (unsigned long long)ticket, timeout_s);
  }
}

extern "C" int polymul_server_replay(polymul_server* s, const polymul_request* reqs, uint32_t count,
                                     const double* arrival_s, double* latency_us) {
  clear_error();
  TraceRange trace_("polymul_server_replay");
  if (!s || (count && (!reqs || !arrival_s))) return fail(POLYMUL_EINVAL, "null argument");
  std::vector<uint64_t> tickets(count);
  const auto t0 = Clock::now();
  for (uint32_t i = 0; i < count; ++i) {
    const auto at = t0 + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(arrival_s[i]));
    while (Clock::now() < at) {
      const auto left = at - Clock::now();
      if (left > std::chrono::microseconds(200)) std::this_thread::sleep_for(left - std::chrono::microseconds(100));
    }
    const int rc = polymul_server_submit(s, &reqs[i], &tickets[i]);
    if (rc != POLYMUL_OK) return rc;
  }
  std::unique_lock<std::mutex> lock(s->mu);
  for (uint32_t i = 0; i < count; ++i) {
    for (;;) {
      auto it = s->reqs.find(tickets[i]);
      if (it == s->reqs.end()) return fail(POLYMUL_EINVAL, "ticket vanished");
      ServeReq* r = it->second;
      if (r->state >= 2) {
        if (latency_us) latency_us[i] = (r->t_done - r->t_submit) * 1e6;
        const int st = r->state;
        delete r;
        s->reqs.erase(it);
        if (st != 2) return request_failure(s, st == 4 ? POLYMUL_ETIMEOUT : POLYMUL_ECUDA, tickets[i]);
        break;
      }
      s->cv.wait_for(lock, std::chrono::milliseconds(50));
    }
  }
  return POLYMUL_OK;
}

extern "C" int polymul_server_stats_get(polymul_server* s, polymul_server_stats* out, int reset) {
  clear_error();
  if (!s || !out) return fail(POLYMUL_EINVAL, "null argument");
  std::lock_guard<std::mutex> lock(s->mu);
  memset(out, 0, sizeof *out);
  out->submitted = s->submitted;
  out->completed = s->completed;
  out->failed = s->failed;
  out->queued = s->queue.size() + s->published_pending;
  out->in_flight = s->published_inflight;
  out->arena_bytes = s->arena_bytes;
  out->arena_peak_bytes = s->arena_peak;
  auto pct = [](std::vector<double> l, double p) {
    if (l.empty()) return 0.0;
    std::sort(l.begin(), l.end());
    return l[std::min(l.size() - 1, (size_t)(p * (l.size() - 1) + 0.5))];
  };
  const std::vector<double>& l = s->latencies_us;
  if (!l.empty()) {
    out->p50_us = pct(l, 0.50);
    out->p99_us = pct(l, 0.99);
    out->max_us = pct(l, 1.0);
    double sum = 0;
    for (double x : l) sum += x;
    out->mean_us = sum / l.size();
    out->queue_p50_us = pct(s->queue_us, 0.50);
    out->queue_p99_us = pct(s->queue_us, 0.99);
    out->service_p50_us = pct(s->service_us, 0.50);
    out->service_p99_us = pct(s->service_us, 0.99);
  }
  out->completed_direct = s->completed_direct;
  out->issue_us_mean = s->issued ? s->issue_s / s->issued * 1e6 : 0.0;
  out->server_busy_s = s->loop_busy_s;
  if (reset) {
    s->latencies_us.clear();
    s->queue_us.clear();
    s->service_us.clear();
    s->issue_s = s->loop_busy_s = 0;
    s->issued = 0;
    s->completed = s->submitted = s->failed = s->completed_direct = 0;
    s->arena_peak = s->arena_used;
  }
  return POLYMUL_OK;
}

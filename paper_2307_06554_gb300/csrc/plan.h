// The opaque plan behind polymul_plan* (library-internal).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "kernels.h"

constexpr int kHostSlots = 6;  // staging slots of the host-buffer entry's pipeline
// work-counter slots: 0 the device entry point, 1 the kernels of the staged
// host-buffer pipeline, 2 the direct form on mapped host memory
constexpr int kCounterSlots = 3;
constexpr int kDirectSlot = 2;

// One launchable way of computing a plan's products (the autotuner's choices).
struct PlanCandidate {
  uint32_t path;     // POLYMUL_PATH_NTT or POLYMUL_PATH_TENSOR
  pm::KernelInfo ki;
  int grid_cap;
  uint32_t launch_flags = 0;  // kLaunchPdl for the NTT batch kernels
};

constexpr uint32_t kLaunchPdl = 2u;  // programmatic dependent launch

struct polymul_plan {
  uint32_t n = 0, logn = 0, k = 0;
  uint32_t elem = 4;   // bytes per coefficient word (4 or 8)
  uint32_t path = 0;   // POLYMUL_PATH_NTT or POLYMUL_PATH_TENSOR
  uint32_t flags = 0;
  bool cyclic = false;  // ring x^n - 1 (POLYMUL_FLAG_CYCLIC) instead of x^n + 1
  bool ternary_b = false;  // POLYMUL_FLAG_TERNARY_B: b one digit, on the MMA's A side (operands swapped)
  std::vector<uint64_t> q;
  int mode = -1;       // NTT reduction mode (0 = [0,2q), 1 = [0,4q), 2 = unreduced)
  int digit_bits = 0;  // tensor path: digit width w and digits per coefficient L
  int digits = 0;
  int device = 0, num_sms = 0;
  // NTT tables: [k][n] (w, w') pairs, forward and inverse; [k] constants
  void* d_twf = nullptr;
  void* d_twi = nullptr;
  void* d_pc = nullptr;
  pm::KernelInfo ki;   // the main kernel of the chosen path
  pm::KernelInfo tki;  // tensor-path kernel, when one exists for the shape
  std::vector<PlanCandidate> cands;  // [0] is the default
  size_t chosen = 0;
  bool tuned = false;
  uint64_t tuned_batch = 0;  // batch bucket of the tuned choice
  void* d_tpc = nullptr;  // tensor-path constants
  void* d_tpc8 = nullptr;  // the same for 8-bit digits (drained tiled kernel), when the plan's width is less
  void* d_tp64 = nullptr;  // TensorPrime64 per prime (64-bit-word digit kernel)
  // tensor path, residue number system of small moduli: the base and its
  // per-prime constants (when the RNS kernel is a candidate)
  uint32_t rns_r = 0;
  void* d_rns_base = nullptr;
  void* d_rns_primes = nullptr;
  // residue planes of a and b, one buffer per launch slot (the host-buffer
  // entry's streams run concurrently), grown on demand
  void* d_rns_scr[kCounterSlots] = {};
  size_t rns_scr_bytes[kCounterSlots] = {};
  uint64_t* d_q = nullptr;  // moduli on the device (input validation)
  // auxiliary-prime NTT (moduli without a 2n-th root of unity)
  uint64_t aux_prime = 0, aux_candidate = 0;
  pm::KernelInfo aki;
  void* d_outer = nullptr;  // the ring moduli as words [k]
  int grid_cap = 0;    // resident CTAs of ki (persistent grid)
  uint32_t launch_flags = 0;
  int* d_flag = nullptr;
  unsigned long long* d_ctr = nullptr;  // kCounterSlots x {next, finished}: device entry, host streams
  int* d_err = nullptr;                 // set by kernels whose bounded waits expired
  // polymul_batch_shared scratch (digit planes of b and of T(a))
  void* d_sh = nullptr;
  size_t sh_bytes = 0;
  // polymul_batch_host: staging slots (a, b, c of one chunk each) and the
  // three streams of its pipeline with one event per stage and slot
  void* d_hslot[kHostSlots] = {};
  size_t hslot_bytes = 0;
  cudaStream_t hs[3] = {};                // copies in, kernels, copies out
  cudaEvent_t hev[3][kHostSlots] = {};    // after the copies in, the kernel, the copy out (slot free)
  cudaEvent_t ev_entry = nullptr;
  // polymul_batch_host, direct route: the batch kernel that reads a and b
  // and writes c where they lie (mapped page-locked host memory), its
  // persistent grid, and the calls that took the route
  pm::KernelInfo dki;
  int dgrid_cap = 0;
  uint64_t host_direct = 0;
};

inline void apply_candidate(polymul_plan* p, size_t i) {
  p->chosen = i;
  p->path = p->cands[i].path;
  p->ki = p->cands[i].ki;
  p->grid_cap = p->cands[i].grid_cap;
  p->launch_flags = p->cands[i].launch_flags;
}

extern "C" int polymul_tune(polymul_plan* plan, uint64_t batch, void* stream);

namespace pm {
int launch_batch(polymul_plan* p, const void* a, const void* b, void* c, uint64_t batch, cudaStream_t st, int slot);
// The device address of [x, x + bytes) when the whole range is page-locked
// host memory that the device maps (both ends checked), else null.
void* mapped_host_range(const void* x, size_t bytes);
int fail(int code, const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what);
void clear_error();
// diagnostics: true (and the kernel arguments that make its waits expire)
// when this NTT batch launch is one that polymul_selftest_inject_wait asked for
bool take_injected_wait(uint32_t* tx_pad, uint32_t* polls);
}  // namespace pm

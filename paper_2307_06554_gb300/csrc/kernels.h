// Registry of compiled kernel instantiations (one translation unit per
// size range, so that they compile in parallel).
#pragma once
#include <cstdint>

namespace pm {

struct KernelInfo {
  const void* fn = nullptr;  // __global__ entry, launched with cudaLaunchKernel
  int block = 0;             // threads per CTA
  int smem = 0;              // dynamic shared memory bytes per CTA
  int team = 0;              // threads per unit
  int units_per_cta = 0;     // units a CTA processes per iteration
  int tmem_cols = 0;         // tensor-memory columns allocated per CTA (0: none)
  int cluster = 0;           // CTAs per thread-block cluster (0: no cluster launch)
  int rb = 0;                // NTT: stage bits per register pass
  int mode = 0;              // NTT: reduction mode (0..2, see ntt.cuh)
  int regs = 0;              // NTT: register budget per thread
  int pad = 0;               // NTT: exchange layout (0 XOR swizzle, s > 0 one padding word per 2^s)
  int seq = 0;               // NTT: 1 = one operand in registers at a time
  int tiled = 0;             // tensor path: 1 for k_toeplitz_tiled (output groups, K chunks)
  int drain = 0;             // tensor path: tiled kernel draining each K chunk (8-bit digits at any n)
  int ws = 0;                // tensor path: the drained kernel's warp-specialised pipeline (k_toeplitz_ws)
  int u64 = 0;               // tensor path: the 64-bit-word digit kernel (k_toeplitz_u64)
  int wb = 0, digits = 0;    // tensor path: the digit width and count a kernel fixes itself (0: the plan's)
  int rns = 0;               // tensor path: 1 for k_toeplitz_rns (residues of small moduli)
};

// batched negacyclic NTT, k_ntt_batch<W, LOGN, MODE> (MODE: 0 = kQ31,
// 1 = kL4, 2 = kSmall; see ntt.cuh)
bool lookup_ntt_u32_m0(int logn, KernelInfo* ki);  // logn 4..14
bool lookup_ntt_u32_m1(int logn, KernelInfo* ki);
bool lookup_ntt_u32_m2(int logn, KernelInfo* ki);
bool lookup_ntt_u64_m1(int logn, KernelInfo* ki);  // logn 4..13
bool lookup_ntt_u64_m2(int logn, KernelInfo* ki);
bool lookup_ntt_u32_aux(int logn, KernelInfo* ki);  // auxiliary-prime mode, logn 4..14
bool lookup_ntt_u32_aux_rb2(int logn, KernelInfo* ki);  // the same with radix-4 passes, logn 7..10
// autotuner candidates: other register radices (RB = stage bits per pass)
bool lookup_ntt_u32_rb5(int logn, int mode, KernelInfo* ki);  // logn 9..13, modes 1, 2; logn 14, modes 0..2
bool lookup_ntt_u32_rb3(int logn, int mode, KernelInfo* ki);  // logn 9..12, modes 1, 2
// the alternative shape of the default kernel's measurements (the other
// layout / operand scheme): 32-bit words, modes 1, 2, logn 5..13; 64-bit
// words, mode 1, logn 6..12
bool lookup_ntt_alt(uint32_t elem, int logn, int mode, KernelInfo* ki);

// the batch kernel reading a and b and writing c where they lie (host
// memory the device maps): 32-bit words logn 4..14, 64-bit words logn 4..13
bool lookup_ntt_direct_u32(int logn, KernelInfo* ki);
bool lookup_ntt_direct_u64(int logn, KernelInfo* ki);
bool lookup_ntt_direct_aux(int logn, KernelInfo* ki);  // auxiliary-prime mode, logn 4..14

// shared-operand products on the NTT path: a's transform once per prime
// (prep), then forward(b), pointwise, inverse per product (32-bit words,
// logn 10..13, modes 0..2)
bool lookup_ntt_shared(int logn, int mode, KernelInfo* prep, KernelInfo* main);

// one product per thread-block cluster (n = 2^14 .. 2^16)
bool lookup_ntt_cluster(uint32_t elem, int logn, int mode, KernelInfo* ki);
// its second form: CTA-local exchanges except the top phase's, padded
// layout; one operand in registers at a time (seq) or both (mode 1 only)
bool lookup_ntt_cluster2(uint32_t elem, int logn, int mode, bool seq, KernelInfo* ki);

// uneven batches (32-bit words): one persistent kernel for the degrees
// 2^10..2^13 and one for 2^14, in two shape sets (0: swizzled exchanges,
// both operands; 1: padded exchanges, one operand at 2^10, 2^11 and 2^14)
constexpr int kRaggedSets = 2;
constexpr int kRaggedClasses = 5;  // degree classes 2^10 .. 2^14 of an uneven list
bool lookup_ntt_ragged(int mode, int set, KernelInfo* small, KernelInfo* big);

// Toeplitz path on the tensor cores, k_toeplitz_batch<TShape<LOGN, WB, LA, LB>>
bool lookup_toeplitz(int logn, int wb, int la, int lb, KernelInfo* ki);

// Resident CTAs per SM of a kernel that allocates tensor memory (shared
// memory, registers, threads and the 512 columns; the occupancy query does
// not count them).  The kernel's dynamic shared-memory attribute must be set.
// Returns a POLYMUL_* code.
int tmem_kernel_per_sm(const KernelInfo& ki, int device, int* per_sm);

}  // namespace pm

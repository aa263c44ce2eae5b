// Overlap of consecutive batch launches on one stream.
//
// The NTT batch kernel takes a programmatic dependent launch: its CTAs come
// up while the previous kernel on the stream drains, and wait for that
// kernel to complete before they touch memory.  Every kernel of this library
// that lets its successor start early does so only after its own wait, so
// when a kernel starts, everything before its predecessor is complete.
//
// A batch launch may go further and load and multiply its first products
// before that wait (NttBatchArgs::early) when its predecessor on the stream
// is a launch of this library whose footprint is known and disjoint from
// this launch's: the predecessor writes none of this launch's operands and
// reads or writes none of its results.  The record below holds, per device
// and stream, the last such launch.  Launches of kernels that let their
// successor start only at completion need no record: whatever follows them
// starts after they are done.
//
// The caller opts in per plan (POLYMUL_FLAG_OVERLAP): a kernel of the
// caller's own that lets its dependents start early, launched right before a
// batch and producing its operands, would otherwise be read before it
// completes.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

namespace pm {

// Byte ranges [lo, hi) of a launch's operands (read) and results (written).
struct LaunchFootprint {
  uintptr_t a_lo = 0, a_hi = 0;
  uintptr_t b_lo = 0, b_hi = 0;
  uintptr_t c_lo = 0, c_hi = 0;
};

inline bool ranges_meet(uintptr_t lo0, uintptr_t hi0, uintptr_t lo1, uintptr_t hi1) {
  return lo0 < hi1 && lo1 < hi0;
}

// true when `next` may run ahead of `prev`: no read-after-write, write-after-
// read or write-after-write between them
inline bool footprints_independent(const LaunchFootprint& prev, const LaunchFootprint& next) {
  return !ranges_meet(prev.c_lo, prev.c_hi, next.a_lo, next.a_hi) &&
         !ranges_meet(prev.c_lo, prev.c_hi, next.b_lo, next.b_hi) &&
         !ranges_meet(next.c_lo, next.c_hi, prev.a_lo, prev.a_hi) &&
         !ranges_meet(next.c_lo, next.c_hi, prev.b_lo, prev.b_hi) &&
         !ranges_meet(next.c_lo, next.c_hi, prev.c_lo, prev.c_hi);
}

// Holds the record's lock from the decision until the launch has been
// enqueued and recorded, so that launches from several host threads onto
// one stream are recorded in their stream order.
class StreamOrderGuard {
 public:
  StreamOrderGuard(int device, cudaStream_t st);
  ~StreamOrderGuard();
  // may a launch with footprint `next` start before the previous kernel on
  // the stream has completed?  (false for the legacy and per-thread default
  // streams, and when the last recorded launch's footprint is unknown)
  bool may_run_ahead(const LaunchFootprint& next) const;
  // the launch just enqueued: its footprint, or nullptr when unknown (the
  // next launch on the stream then waits in full)
  void record(const LaunchFootprint* fp);

 private:
  std::unique_lock<std::mutex> lock_;
  int device_;
  cudaStream_t st_;
};

}  // namespace pm

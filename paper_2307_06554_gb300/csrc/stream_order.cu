// Per-stream record of the last batch launch (see stream_order.h).
#include "stream_order.h"

#include <map>
#include <utility>

namespace pm {

namespace {

struct Entry {
  bool known = false;
  LaunchFootprint fp;
};

std::mutex g_mu;
// keyed by (device, stream); bounded: when it grows past kMaxStreams every
// entry is dropped, which only makes the next launch on each stream wait
std::map<std::pair<int, uintptr_t>, Entry> g_last;
constexpr size_t kMaxStreams = 4096;

bool default_stream(cudaStream_t st) {
  return st == nullptr || st == cudaStreamLegacy || st == cudaStreamPerThread;
}

}  // namespace

StreamOrderGuard::StreamOrderGuard(int device, cudaStream_t st) : lock_(g_mu), device_(device), st_(st) {}

StreamOrderGuard::~StreamOrderGuard() = default;

bool StreamOrderGuard::may_run_ahead(const LaunchFootprint& next) const {
  if (default_stream(st_)) return false;
  auto it = g_last.find({device_, (uintptr_t)st_});
  if (it == g_last.end() || !it->second.known) return false;
  return footprints_independent(it->second.fp, next);
}

void StreamOrderGuard::record(const LaunchFootprint* fp) {
  if (g_last.size() >= kMaxStreams) g_last.clear();
  Entry& e = g_last[{device_, (uintptr_t)st_}];
  e.known = fp != nullptr;
  if (fp) e.fp = *fp;
}

}  // namespace pm

// Observability: a process-wide count of the kernels this library launched,
// and CUDA-event bracketing of one kernel class for live per-launch timing.
#include "bmg_internal.h"

#include <atomic>
#include <mutex>
#include <vector>

namespace bmg {

namespace {

std::atomic<long long> g_launches{0};

struct Prof {
  std::mutex mu;
  int which = BMG_PROF_NONE;
  std::vector<cudaEvent_t> ev;   // pairs (start, stop)
  size_t used = 0;               // events used
  cudaEvent_t pending = nullptr; // start event awaiting its stop
};

Prof& prof() {
  static Prof p;
  return p;
}

constexpr size_t kMaxPairs = 65536;

}  // namespace

void count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

void prof_begin(int which, cudaStream_t s) {
  Prof& p = prof();
  if (p.which == BMG_PROF_NONE || p.which != which) return;
  std::lock_guard<std::mutex> g(p.mu);
  if (p.used + 2 > 2 * kMaxPairs) return;
  if (p.ev.size() < p.used + 2) {
    for (int k = 0; k < 2; ++k) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return;
      p.ev.push_back(e);
    }
  }
  cudaEventRecord(p.ev[p.used], s);
  p.pending = p.ev[p.used];
}

void prof_end(int which, cudaStream_t s) {
  Prof& p = prof();
  if (p.which == BMG_PROF_NONE || p.which != which) return;
  std::lock_guard<std::mutex> g(p.mu);
  if (!p.pending || p.pending != p.ev[p.used]) return;
  cudaEventRecord(p.ev[p.used + 1], s);
  p.used += 2;
  p.pending = nullptr;
}

}  // namespace bmg

extern "C" {

long long bmg_kernel_launches(void) { return bmg::g_launches.load(); }

int bmg_profile_set(int which) {
  if (which < BMG_PROF_NONE || which > BMG_PROF_COARSE) return BMG_EINVAL;
  bmg::Prof& p = bmg::prof();
  std::lock_guard<std::mutex> g(p.mu);
  p.which = which;
  p.used = 0;
  p.pending = nullptr;
  return BMG_OK;
}

int bmg_profile_read(int* launches, double* total_ms) {
  if (!launches || !total_ms) return BMG_EINVAL;
  bmg::Prof& p = bmg::prof();
  std::lock_guard<std::mutex> g(p.mu);
  double tot = 0.0;
  for (size_t k = 0; k + 1 < p.used; k += 2) {
    if (cudaEventSynchronize(p.ev[k + 1]) != cudaSuccess) return BMG_ECUDA;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p.ev[k], p.ev[k + 1]) != cudaSuccess) return BMG_ECUDA;
    tot += ms;
  }
  *launches = int(p.used / 2);
  *total_ms = tot;
  return BMG_OK;
}

}  // extern "C"

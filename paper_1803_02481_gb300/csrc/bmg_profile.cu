// Observability: a process-wide count of the kernels this library launched,
// and CUDA-event bracketing of one kernel class for live per-launch timing.
#include "bmg_internal.h"

#include <nvtx3/nvToolsExt.h>

#include <atomic>
#include <mutex>
#include <vector>

namespace bmg {

namespace {

std::atomic<long long> g_launches{0};

constexpr int kClasses = 9;
constexpr size_t kMaxPairs = 65536;

struct ClassRec {
  std::vector<cudaEvent_t> ev;   // pairs (start, stop)
  size_t used = 0;               // events used
  bool open = false;             // a start awaits its stop
};

struct Prof {
  std::mutex mu;
  unsigned mask = 0;             // bit c: class c is recorded
  ClassRec cls[kClasses];
};

Prof& prof() {
  static Prof p;
  return p;
}

}  // namespace

void count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

NvtxRange::NvtxRange(const char* op, int level) {
  nvtxEventAttributes_t a = {};
  a.version = NVTX_VERSION;
  a.size = NVTX_EVENT_ATTRIB_STRUCT_SIZE;
  a.messageType = NVTX_MESSAGE_TYPE_ASCII;
  a.message.ascii = op;
  a.payloadType = NVTX_PAYLOAD_TYPE_INT32;
  a.payload.iValue = level;
  nvtxRangePushEx(&a);
}

NvtxRange::~NvtxRange() { nvtxRangePop(); }

bool prof_active() { return prof().mask != 0; }

void prof_begin(int which, cudaStream_t s) {
  Prof& p = prof();
  if (!(p.mask & (1u << which))) return;
  std::lock_guard<std::mutex> g(p.mu);
  ClassRec& c = p.cls[which];
  if (c.open || c.used + 2 > 2 * kMaxPairs) return;
  while (c.ev.size() < c.used + 2) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return;
    c.ev.push_back(e);
  }
  cudaEventRecord(c.ev[c.used], s);
  c.open = true;
}

void prof_end(int which, cudaStream_t s) {
  Prof& p = prof();
  if (!(p.mask & (1u << which))) return;
  std::lock_guard<std::mutex> g(p.mu);
  ClassRec& c = p.cls[which];
  if (!c.open) return;
  cudaEventRecord(c.ev[c.used + 1], s);
  c.used += 2;
  c.open = false;
}

}  // namespace bmg

extern "C" {

long long bmg_kernel_launches(void) { return bmg::g_launches.load(); }

int bmg_profile_set(int mask) {
  if (mask < 0 || mask >= (1 << bmg::kClasses)) return BMG_EINVAL;
  bmg::Prof& p = bmg::prof();
  std::lock_guard<std::mutex> g(p.mu);
  p.mask = unsigned(mask);
  for (auto& c : p.cls) {
    c.used = 0;
    c.open = false;
  }
  return BMG_OK;
}

int bmg_profile_read(int which, int* launches, double* total_ms) {
  if (!launches || !total_ms || which < 0 || which >= bmg::kClasses) return BMG_EINVAL;
  bmg::Prof& p = bmg::prof();
  std::lock_guard<std::mutex> g(p.mu);
  bmg::ClassRec& c = p.cls[which];
  double tot = 0.0;
  for (size_t k = 0; k + 1 < c.used; k += 2) {
    if (cudaEventSynchronize(c.ev[k + 1]) != cudaSuccess) return BMG_ECUDA;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, c.ev[k], c.ev[k + 1]) != cudaSuccess) return BMG_ECUDA;
    tot += ms;
  }
  *launches = int(c.used / 2);
  *total_ms = tot;
  return BMG_OK;
}

}  // extern "C"

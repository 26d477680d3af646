// Kernel-level tracing: when enabled, every launch region records a CUDA event pair on the
// stream it is launched on and counts the library's own kernels launched inside it;
// mtp_profiler_read() synchronises, accumulates device time and kernel launches per region name,
// and clears the record.
#include <cuda_runtime.h>

#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "mtp_internal.h"
#include "profiler.h"

namespace mtp {
namespace {

struct Rec {
  const char* name;
  cudaEvent_t a, b;
  int kernels;
};
thread_local ProfRegion* t_open = nullptr;   // innermost open region of this thread
std::mutex g_mu;
bool g_on = false;
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_pool;

cudaEvent_t take() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

}  // namespace

ProfRegion::ProfRegion(const char* name, cudaStream_t s) : name_(name), s_(s), outer_(t_open) {
  t_open = this;
  nvtxRangePushA(name);   // host-side range for timeline tools (a no-op without one attached)
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_on) return;
  a_ = take();
  b_ = take();
  if (a_ && b_) cudaEventRecord(a_, s_);
}

ProfRegion::~ProfRegion() {
  t_open = outer_;
  nvtxRangePop();
  std::lock_guard<std::mutex> lk(g_mu);
  if (!a_ || !b_) return;
  cudaEventRecord(b_, s_);
  g_recs.push_back({name_, a_, b_, kernels_});
}

void ProfRegion::launched() {
  if (t_open) ++t_open->kernels_;
}

}  // namespace mtp

using namespace mtp;

extern "C" {

mtp_status mtp_profiler_enable(int on) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_on = on != 0;
  return MTP_OK;
}

mtp_status mtp_profiler_read(int32_t capacity, char* names, double* ms, int64_t* launches, int32_t* count) {
  std::vector<Rec> recs;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    recs.swap(g_recs);
  }
  std::map<std::string, std::pair<double, int64_t>> acc;
  std::vector<std::string> order;
  mtp_status st = MTP_OK;
  for (auto& r : recs) {
    float t = 0.f;
    if (cudaEventSynchronize(r.b) != cudaSuccess || cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess) {
      set_error("profiler: event query failed");
      st = MTP_ERR_CUDA;
    }
    auto it = acc.find(r.name);
    if (it == acc.end()) { order.push_back(r.name); acc[r.name] = {0.0, 0}; }
    acc[r.name].first += t;
    acc[r.name].second += r.kernels;
  }
  {
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto& r : recs) { g_pool.push_back(r.a); g_pool.push_back(r.b); }
  }
  int32_t n = 0;
  for (auto& nm : order) {
    if (n >= capacity) break;
    if (names) {
      std::memset(names + 48 * n, 0, 48);
      std::strncpy(names + 48 * n, nm.c_str(), 47);
    }
    if (ms) ms[n] = acc[nm].first;
    if (launches) launches[n] = acc[nm].second;
    ++n;
  }
  if (count) *count = n;
  return st;
}

}  // extern "C"

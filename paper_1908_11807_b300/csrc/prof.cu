// Per-launch CUDA-event timing; see prof.cuh.
#include <atomic>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/arborx_b300.h"
#include "prof.cuh"

namespace abx {
namespace prof {

namespace {
struct Pending {
  std::string name;
  cudaEvent_t a, b;
};
struct Acc {
  long long count = 0;
  double ms = 0.0;
};
std::atomic<bool> g_on{false};
std::mutex g_mu;
std::vector<Pending> g_pending;
std::vector<cudaEvent_t> g_pool;
std::map<std::string, Acc> g_acc;

cudaEvent_t take_event() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}
}  // namespace

bool enabled() { return g_on.load(std::memory_order_relaxed); }

int begin(cudaStream_t s, const char *name) {
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return -1;  // no event pairs inside a graph being captured
  }
  std::lock_guard<std::mutex> lk(g_mu);
  Pending p;
  p.name = name;
  p.a = take_event();
  p.b = take_event();
  cudaEventRecord(p.a, s);
  g_pending.push_back(p);
  return (int)g_pending.size() - 1;
}

void end(cudaStream_t s, int slot) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (slot >= 0 && slot < (int)g_pending.size()) cudaEventRecord(g_pending[slot].b, s);
}

}  // namespace prof
}  // namespace abx

using namespace abx::prof;

extern "C" {

int arborx_profile_enable(int on) {
  g_on.store(on != 0);
  return ARBORX_OK;
}

int arborx_profile_report(char *buf, size_t cap) {
  std::lock_guard<std::mutex> lk(g_mu);
  for (auto &p : g_pending) {
    if (cudaEventSynchronize(p.b) != cudaSuccess) return ARBORX_ECUDA;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, p.a, p.b);
    Acc &a = g_acc[p.name];
    a.count += 1;
    a.ms += ms;
    g_pool.push_back(p.a);
    g_pool.push_back(p.b);
  }
  g_pending.clear();
  std::string out;
  char line[256];
  for (auto &kv : g_acc) {
    std::snprintf(line, sizeof line, "%s %lld %.6f\n", kv.first.c_str(), kv.second.count, kv.second.ms);
    out += line;
  }
  g_acc.clear();
  if (!buf || cap == 0) return ARBORX_EINVAL;
  std::strncpy(buf, out.c_str(), cap - 1);
  buf[cap - 1] = '\0';
  return out.size() < cap ? ARBORX_OK : ARBORX_EOVERFLOW;
}

}  // extern "C"

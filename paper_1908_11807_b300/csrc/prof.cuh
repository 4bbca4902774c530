// Per-launch CUDA-event timing of the library's kernels (process-wide switch).
//
// When enabled, every launcher records an event pair around its kernel on the
// launching stream; arborx_profile_report resolves the pairs and reports, per
// kernel name, the launch count and the summed device time.
#pragma once

#include <cuda_runtime.h>

namespace abx {
namespace prof {

bool enabled();
int begin(cudaStream_t s, const char *name);  // returns a slot id, or -1 when disabled
void end(cudaStream_t s, int slot);

struct Scope {
  cudaStream_t s;
  int slot;
  Scope(cudaStream_t s_, const char *name) : s(s_), slot(enabled() ? begin(s_, name) : -1) {}
  ~Scope() {
    if (slot >= 0) end(s, slot);
  }
};

}  // namespace prof
}  // namespace abx

// Radix sort of (key, index) pairs that allocates nothing.
//
// For callers that may not allocate device memory during a call: code running
// inside another framework's memory budget, a pre-planned real-time loop, or a
// host process whose allocator must stay untouched.  The temporaries of the
// sort (the second key / index buffers, the digit histograms, the tile
// counters and the look-back status words) live in one file-scope device
// array of fixed size instead of coming from cudaMalloc or a pool.
#include <cstdint>
#include <mutex>

#include "../../include/arborx_b300.h"
#include "radix_sort.cuh"
#include "status.cuh"

namespace abx {
namespace {

constexpr size_t kScratchBytes = (size_t)16 << 20;  // 16 MiB: ARBORX_SORT_NOALLOC_MAX_KEYS 64-bit keys fit
static_assert(ARBORX_SORT_NOALLOC_MAX_KEYS <= (1 << 20), "scratch sized for at most 2^20 keys");

// Shared by every call on a device; kept for the life of the process.
static __device__ __align__(256) unsigned char g_sort_scratch[kScratchBytes];

constexpr int kMaxDev = 64;
std::mutex g_mu;
void *g_scratch_addr[kMaxDev] = {};

constexpr size_t kAlign = 256;
size_t up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

// Device address of the scratch array on the current device.  Host code only
// holds a stand-in symbol for it; the real address is looked up once per device
// and kept for the life of the process (like the library's per-device memory
// pool, it does not survive a cudaDeviceReset of that device).
int scratch_address(void **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) {
    cudaGetLastError();
    return ARBORX_ECUDA;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_sort_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return ARBORX_ECUDA;
    }
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return ARBORX_OK;
}

template <typename K>
int sort_in_scratch(K *keys, uint32_t *perm, uint32_t n, int key_bits, char *scratch, cudaStream_t s) {
  const size_t ws_words = sort_ws_words<K>(n, key_bits);
  K *kB = reinterpret_cast<K *>(scratch);
  uint32_t *vB = reinterpret_cast<uint32_t *>(scratch + up((size_t)n * sizeof(K)));
  uint32_t *wsb = reinterpret_cast<uint32_t *>(reinterpret_cast<char *>(vB) + up((size_t)n * 4));
  uint32_t *err = reinterpret_cast<uint32_t *>(reinterpret_cast<char *>(wsb) + up(ws_words * 4));
  if (reinterpret_cast<char *>(err) + kAlign > scratch + kScratchBytes) return ARBORX_EINVAL;
  // the array keeps the previous call's contents: clear what must start at zero
  if (cudaMemsetAsync(wsb, 0, up(ws_words * 4) + kAlign, s) != cudaSuccess) return launch_status();
  const SortWs ws = sort_ws_carve<K>(wsb, n, key_bits);
  launch_histogram<K>(keys, n, ws.passes, ws.hist, s);
  const bool inA = launch_onesweep<K>(keys, kB, perm, vB, n, ws, err, s);
  if (!inA) {  // an odd number of passes leaves the result in the scratch buffers
    if (cudaMemcpyAsync(keys, kB, (size_t)n * sizeof(K), cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(perm, vB, (size_t)n * 4, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
      return launch_status();
  }
  uint32_t bits = 0;
  if (cudaMemcpyAsync(&bits, err, sizeof bits, cudaMemcpyDeviceToHost, s) != cudaSuccess) return launch_status();
  // the same status mapping as arborx_sort_pairs
  if (cudaStreamSynchronize(s) != cudaSuccess) return ARBORX_ECUDA;
  const int st = launch_status();
  if (st) return st;
  return err_bits_to_status(bits);
}

}  // namespace
}  // namespace abx

extern "C" int arborx_sort_pairs_noalloc(void *d_keys, uint32_t *d_perm, int64_t n, int32_t key_bits,
                                         void *stream) {
  if (n < 0 || key_bits < 1 || key_bits > 64 || (n > 0 && (!d_keys || !d_perm))) return ARBORX_EINVAL;
  if (n > ARBORX_SORT_NOALLOC_MAX_KEYS) return ARBORX_EINVAL;  // beyond the fixed scratch array
  if (n == 0) return ARBORX_OK;
  void *scratch = nullptr;
  const int st = abx::scratch_address(&scratch);
  if (st) return st;
  const cudaStream_t s = (cudaStream_t)stream;
  if (key_bits > 32)
    return abx::sort_in_scratch<uint64_t>((uint64_t *)d_keys, d_perm, (uint32_t)n, key_bits, (char *)scratch, s);
  return abx::sort_in_scratch<uint32_t>((uint32_t *)d_keys, d_perm, (uint32_t)n, key_bits, (char *)scratch, s);
}

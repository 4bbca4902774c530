// Rows of a spatial result in ascending primitive index (the opts.sorted_rows option).
//
// Two stable radix sorts over the result entries: by primitive index, then by
// row.  The second sort keeps the order of the first within each row, and the
// rows come out in row order, which is the CSR layout, so every row lands in
// its own place, sorted.  Positions at or past the total (offsets[m], read on
// the device) take keys above every real one and stay at the end.
#include <algorithm>

#include "kernels.cuh"
#include "prof.cuh"
#include "radix_sort.cuh"

namespace abx {

namespace {

// pass-1 keys: the primitive index, or `pad` (above every index) past the total
__global__ void k_rows_keys(const int32_t *__restrict__ indices, const int64_t *__restrict__ offsets, uint32_t m,
                            uint32_t cap, uint32_t pad, uint32_t *__restrict__ keys) {
  const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= cap) return;
  keys[j] = (int64_t)j < offsets[m] ? (uint32_t)indices[j] : pad;
}

// pass-2 keys: the row of the entry now at sorted position j (its position p = p1[j] lies in
// [offsets[r], offsets[r + 1]); the last such r by binary search), or m past the total
__global__ void k_rows_rowkeys(const uint32_t *__restrict__ p1, const int64_t *__restrict__ offsets, uint32_t m,
                               uint32_t cap, uint32_t *__restrict__ keys) {
  const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= cap) return;
  const int64_t p = p1[j];
  if (p >= offsets[m]) {
    keys[j] = m;
    return;
  }
  uint32_t lo = 0, hi = m;  // offsets[lo] <= p < offsets[hi]
  while (hi - lo > 1) {
    const uint32_t mid = lo + (hi - lo) / 2;
    if (offsets[mid] <= p) lo = mid;
    else hi = mid;
  }
  keys[j] = lo;
}

__global__ void k_rows_out(const uint32_t *__restrict__ sorted_idx, const uint32_t *__restrict__ p2,
                           const int64_t *__restrict__ offsets, uint32_t m, uint32_t cap,
                           int32_t *__restrict__ indices) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= cap || (int64_t)i >= offsets[m]) return;
  indices[i] = (int32_t)sorted_idx[p2[i]];
}

int bits_for(uint64_t v) {  // bits that hold every value up to v
  int b = 1;
  while (b < 32 && (v >> b) != 0) ++b;
  return b;
}

constexpr size_t kRowsAlign = 256;
size_t round_up(size_t x) { return (x + kRowsAlign - 1) & ~(kRowsAlign - 1); }

}  // namespace

size_t sort_rows_bytes(uint32_t cap, uint32_t m, uint32_t n_prims) {
  const size_t words = std::max(sort_ws_words<uint32_t>(cap, bits_for(n_prims)),
                                sort_ws_words<uint32_t>(cap, bits_for(m)));
  return 5 * round_up((size_t)cap * 4) + round_up(words * 4);
}

void launch_sort_rows(const int64_t *offsets, int32_t *indices, uint32_t m, uint32_t cap, uint32_t n_prims,
                      void *ws, uint32_t *err, cudaStream_t s) {
  if (cap == 0 || m == 0) return;
  prof::Scope ps(s, "sort_rows");
  unsigned char *base = static_cast<unsigned char *>(ws);
  uint32_t *buf[5];
  for (int i = 0; i < 5; ++i) buf[i] = reinterpret_cast<uint32_t *>(base + i * round_up((size_t)cap * 4));
  uint32_t *sws = reinterpret_cast<uint32_t *>(base + 5 * round_up((size_t)cap * 4));
  const unsigned blocks = (unsigned)ceil_div<uint32_t>(cap, 256u);

  // pass 1: by primitive index; the pad n_prims sorts after every real index
  const int b1 = bits_for(n_prims);
  const SortWs w1 = sort_ws_carve<uint32_t>(sws, cap, b1);
  cudaMemsetAsync(sws, 0, sort_ws_words<uint32_t>(cap, b1) * 4, s);
  k_rows_keys<<<blocks, 256, 0, s>>>(indices, offsets, m, cap, n_prims, buf[0]);
  launch_histogram<uint32_t>(buf[0], cap, w1.passes, w1.hist, s);
  const bool in1 = launch_onesweep<uint32_t>(buf[0], buf[1], buf[2], buf[3], cap, w1, err, s);
  uint32_t *sk = in1 ? buf[0] : buf[1];   // primitive indices, ascending
  uint32_t *p1 = in1 ? buf[2] : buf[3];   // where each came from
  uint32_t *kfree = in1 ? buf[1] : buf[0];
  uint32_t *vfree = in1 ? buf[3] : buf[2];

  // pass 2: by row, stable; its keys come from p1, whose buffer is then free for the sort
  k_rows_rowkeys<<<blocks, 256, 0, s>>>(p1, offsets, m, cap, kfree);
  const int b2 = bits_for(m);
  const SortWs w2 = sort_ws_carve<uint32_t>(sws, cap, b2);
  cudaMemsetAsync(sws, 0, sort_ws_words<uint32_t>(cap, b2) * 4, s);
  launch_histogram<uint32_t>(kfree, cap, w2.passes, w2.hist, s);
  const bool in2 = launch_onesweep<uint32_t>(kfree, p1, vfree, buf[4], cap, w2, err, s);
  const uint32_t *p2 = in2 ? vfree : buf[4];

  k_rows_out<<<blocks, 256, 0, s>>>(sk, p2, offsets, m, cap, indices);
}

}  // namespace abx

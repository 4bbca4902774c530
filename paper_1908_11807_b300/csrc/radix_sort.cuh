// Onesweep LSD radix sort of (key, index) pairs -- the sort step of the LBVH
// build (ArborX Sec. 2.1, the sort by Morton code).
//
// Design (B300): 8-bit digits; the digit histograms of all passes come from
// one read of the keys (fused into the Morton-code kernel, or the standalone
// histogram kernel); each pass is one kernel in which a block takes the next
// tile id from an atomic counter, ranks its keys per warp with digit-bit ballots,
// publishes its per-digit counts, obtains the counts of all earlier tiles by
// decoupled look-back over 30-bit status words (bounded spin, error flag on
// give-up), stages the tile in shared memory in digit order and writes it out
// in runs.  Stable: ties keep input order, so equal codes end up ordered by
// index, the paper's tie rule for equal codes.
#pragma once

#include "common.cuh"

namespace abx {

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;

template <typename K>
struct SortTile {
  static constexpr int items = sizeof(K) == 4 ? 16 : 12;
  static constexpr int tile = kSortThreads * items;
};

inline int sort_passes(int key_bits) { return (key_bits + kRadixBits - 1) / kRadixBits; }

// Workspace for one sort of n keys: [passes*256] histogram, [passes] tile
// counters, [passes * tiles * 256] look-back status; all must start at zero.
struct SortWs {
  uint32_t *hist;
  uint32_t *tile_ctr;
  uint32_t *status;
  int passes;
  uint32_t tiles;
};

template <typename K>
size_t sort_ws_words(int64_t n, int key_bits) {
  int p = sort_passes(key_bits);
  uint64_t tiles = n > 0 ? ceil_div<uint64_t>((uint64_t)n, (uint64_t)SortTile<K>::tile) : 1;
  return (size_t)p * kRadix + (size_t)p + 32 + (size_t)p * tiles * kRadix;
}

template <typename K>
SortWs sort_ws_carve(uint32_t *base, int64_t n, int key_bits) {
  SortWs w;
  w.passes = sort_passes(key_bits);
  w.tiles = n > 0 ? (uint32_t)ceil_div<uint64_t>((uint64_t)n, (uint64_t)SortTile<K>::tile) : 1;
  w.hist = base;
  w.tile_ctr = base + (size_t)w.passes * kRadix;
  w.status = w.tile_ctr + w.passes + 32;
  return w;
}

// Histogram of every pass's digit (standalone; the build fuses it into the
// Morton kernel).  hist must be zero.
template <typename K>
void launch_histogram(const K *keys, uint32_t n, int passes, uint32_t *hist, cudaStream_t s);

// One thread waiting on *flag with the look-back's iteration cap and backoff; sets ERR_TIMEOUT in
// *err when it gives up (self-test of the bounded wait).
void launch_spin_probe(const uint32_t *flag, uint32_t *err, cudaStream_t s);

// Run all passes.  keys/vals: A buffers hold the input keys (vals unused: the
// first pass generates the identity); B buffers are scratch of the same size.
// Result lands in (keysA, valsA) when passes is even, else in (keysB, valsB);
// the function returns true when the result is in the A buffers.
template <typename K>
bool launch_onesweep(K *keysA, K *keysB, uint32_t *valsA, uint32_t *valsB, uint32_t n, const SortWs &ws,
                     uint32_t *err, cudaStream_t s);

}  // namespace abx

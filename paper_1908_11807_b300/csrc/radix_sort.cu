// Onesweep LSD radix sort of (key, index) pairs; see radix_sort.cuh.
#include <algorithm>

#include "prof.cuh"
#include "radix_sort.cuh"

namespace abx {

namespace {

constexpr uint32_t kFlagAgg = 1u << 30;   // tile's own digit count published
constexpr uint32_t kFlagPre = 2u << 30;   // inclusive prefix over tiles 0..t published
constexpr uint32_t kValMask = (1u << 30) - 1u;
constexpr uint32_t kSpinCap = 1u << 20;   // look-back give-up bound (about a second with the sleeps)
// a blocked look-back round sleeps this long, so that waiting tiles leave the issue slots to the
// working ones (measured 82.2 -> 79.7 us per 1e7-key pass against sleeping only after 256 rounds)
constexpr uint32_t kSpinSleepNs = 512;
constexpr int kWin = 4;                   // predecessors loaded per look-back round trip

// Exclusive scans over the 256 threads of a block, two values at once.
__device__ __forceinline__ void block_excl_scan2(uint32_t a, uint32_t b, uint32_t &a_ex, uint32_t &b_ex,
                                                 uint32_t (*s_scan)[kSortWarps]) {
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = a, y = b;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t xo = __shfl_up_sync(0xffffffffu, x, o);
    uint32_t yo = __shfl_up_sync(0xffffffffu, y, o);
    if (lane >= (uint32_t)o) {
      x += xo;
      y += yo;
    }
  }
  if (lane == 31) {
    s_scan[0][warp] = x;
    s_scan[1][warp] = y;
  }
  __syncthreads();
  uint32_t wa = 0, wb = 0;
#pragma unroll
  for (int w = 0; w < kSortWarps; ++w) {
    if ((uint32_t)w < warp) {
      wa += s_scan[0][w];
      wb += s_scan[1][w];
    }
  }
  a_ex = wa + x - a;
  b_ex = wb + y - b;
}

// Four resident 256-thread blocks per SM (64 registers): the values are read only when the tile
// is staged, so they hold no registers while the keys are ranked (measured 85.4 -> 82.4 us per
// pass of 1e7 keys against three blocks of 80 registers; five blocks spill heavily).
template <typename K, bool FIRST>
__global__ void __launch_bounds__(kSortThreads, 4) k_onesweep(const K *__restrict__ kin, const uint32_t *__restrict__ vin,
                                                          K *__restrict__ kout, uint32_t *__restrict__ vout,
                                                          uint32_t n, int shift, const uint32_t *__restrict__ hist,
                                                          uint32_t *__restrict__ status,
                                                          uint32_t *__restrict__ tile_ctr, uint32_t *__restrict__ err) {
  constexpr int ITEMS = SortTile<K>::items;
  constexpr int TILE = SortTile<K>::tile;
  // 32-bit keys find the lanes sharing a digit through one shared-memory OR per key (73.3 against
  // 77.9 us per 1e7-key pass with eight ballots); 64-bit keys keep the ballots (99 against 94 us)
  constexpr bool kMaskRank = sizeof(K) == 4;
  __shared__ uint32_t s_whist[kSortWarps][kRadix];  // per-warp digit counts, then per-warp offsets
  __shared__ uint32_t s_match[kMaskRank ? kSortWarps : 1][kRadix + 1];  // lane masks of one item's digits
  __shared__ uint32_t s_dstart[kRadix];             // tile-local start of each digit run
  __shared__ uint32_t s_gofs[kRadix];               // global destination of run start minus s_dstart
  __shared__ uint32_t s_scan[2][kSortWarps];
  __shared__ uint32_t s_tile;
  __shared__ K s_k[TILE];
  __shared__ uint32_t s_v[TILE];

  const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) s_tile = atomicAdd(tile_ctr, 1u);  // dynamic tile order: predecessors already run
  for (int i = tid; i < kSortWarps * kRadix; i += kSortThreads) (&s_whist[0][0])[i] = 0;
  if (kMaskRank)
    for (int i = tid; i < kSortWarps * (kRadix + 1); i += kSortThreads) (&s_match[0][0])[i] = 0;
  __syncthreads();
  const uint32_t tile = s_tile;
  const uint32_t tbase = tile * (uint32_t)TILE;
  const uint32_t wbase = tbase + warp * (uint32_t)(ITEMS * 32);

  K k[ITEMS];
  uint32_t rk[ITEMS];
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) {
    const uint32_t pos = wbase + i * 32 + lane;
    k[i] = pos < n ? __ldcs(kin + pos) : (K)0;  // read once per pass: evict first (measured 7% faster)
  }

  // warp-level ranking in input order (item-major, lane-minor): the lanes
  // holding the same digit are found through a shared-memory lane mask per
  // digit (32-bit keys) or one ballot per digit bit (64-bit keys; both cheaper
  // than match.any when most of the 32 digits differ); the lowest lane of
  // each group adds the group size to the warp's counter and hands the
  // previous count to its peers; items are counted in order
  const uint32_t lt = lanemask_lt();
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) {
    const uint32_t pos = wbase + i * 32 + lane;
    const bool valid = pos < n;
    const uint32_t d = valid ? (uint32_t)(k[i] >> shift) & (kRadix - 1) : (uint32_t)kRadix;
    uint32_t peers;
    if constexpr (kMaskRank) {
      atomicOr(&s_match[warp][d], 1u << lane);  // lanes holding the same digit meet in one word
      __syncwarp();
      peers = s_match[warp][d];
    } else {
      peers = __ballot_sync(0xffffffffu, valid);
      if (!valid) peers = ~peers;
#pragma unroll
      for (int b = 0; b < kRadixBits; ++b) {
        const bool bit = (d >> b) & 1u;
        const uint32_t bal = __ballot_sync(0xffffffffu, bit);
        peers &= bit ? bal : ~bal;
      }
    }
    const int leader = __ffs(peers) - 1;
    uint32_t old = 0;
    if constexpr (kMaskRank) {
      __syncwarp();  // every lane has read its mask before the leaders clear them
      if ((int)lane == leader) s_match[warp][d] = 0;
    }
    if (valid && (int)lane == leader) {  // the warp's own counters, one leader per digit: no atomic needed
      old = s_whist[warp][d];
      s_whist[warp][d] = old + (uint32_t)__popc(peers);
    }
    __syncwarp();  // item i's counter update is visible to every lane before item i + 1 reads
    old = __shfl_sync(0xffffffffu, old, leader);
    rk[i] = old + __popc(peers & lt);
  }
  __syncthreads();

  // one thread per digit: warp offsets, tile count, publish, look back
  const uint32_t d = tid;
  uint32_t cnt = 0;
#pragma unroll
  for (int w = 0; w < kSortWarps; ++w) {
    const uint32_t c = s_whist[w][d];
    s_whist[w][d] = cnt;
    cnt += c;
  }
  uint32_t *my_status = status + (size_t)tile * kRadix + d;
  st_relaxed_gpu(my_status, (tile == 0 ? kFlagPre : kFlagAgg) | cnt);

  uint32_t cnt_ex, h_ex;
  block_excl_scan2(cnt, hist[d], cnt_ex, h_ex, s_scan);
  s_dstart[d] = cnt_ex;

  __syncthreads();  // s_dstart and the warp offsets are complete

  // stage in digit order (needs only tile-local offsets, so it runs before the
  // look-back and gives the predecessors time to publish); the values are read only
  // here, so they hold no registers during the ranking
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) {
    const uint32_t pos = wbase + i * 32 + lane;
    if (pos < n) {
      const uint32_t dd = (uint32_t)(k[i] >> shift) & (kRadix - 1);
      const uint32_t p = s_dstart[dd] + s_whist[warp][dd] + rk[i];
      s_k[p] = k[i];
      s_v[p] = FIRST ? pos : __ldcs(vin + pos);
    }
  }

  // decoupled look-back over a window of kWin predecessors at a time (independent
  // loads, one round trip per window); stops at the first inclusive prefix
  uint32_t excl = 0;
  if (tile > 0) {
    int j = (int)tile - 1;  // nearest predecessor not yet accounted for
    uint32_t spins = 0;
    bool done = false;
    while (!done) {
      uint32_t st[kWin];
#pragma unroll
      for (int w = 0; w < kWin; ++w)
        st[w] = (j - w >= 0) ? ld_relaxed_gpu(status + (size_t)(j - w) * kRadix + d) : kFlagPre;
      bool blocked = false;
#pragma unroll
      for (int w = 0; w < kWin; ++w) {
        if (done || blocked) continue;
        if ((st[w] & (kFlagAgg | kFlagPre)) == 0) {
          blocked = true;  // predecessor j not published yet: wait for it
        } else {
          excl += st[w] & kValMask;
          if (st[w] & kFlagPre) done = true;
          --j;
        }
      }
      if (blocked) {
        if (++spins >= kSpinCap) {  // give up: flag the error, unblock successors
          set_err(err, ERR_TIMEOUT);
          done = true;
        } else {
          __nanosleep(kSpinSleepNs);
        }
      }
    }
    st_relaxed_gpu(my_status, kFlagPre | ((excl + cnt) & kValMask));
  }
  s_gofs[d] = h_ex + excl - cnt_ex;
  __syncthreads();

  // write runs (unrolled: the shared-memory loads of all items are independent)
  const uint32_t tn = min((uint32_t)TILE, n - tbase);
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) {
    const uint32_t j = tid + i * kSortThreads;
    if (j < tn) {
      const K key = s_k[j];
      const uint32_t dd = (uint32_t)(key >> shift) & (kRadix - 1);
      const uint32_t dst = s_gofs[dd] + j;
      kout[dst] = key;
      vout[dst] = s_v[j];
    }
  }
}

template <typename K>
__global__ void __launch_bounds__(256) k_histogram(const K *__restrict__ keys, uint32_t n, int passes,
                                                  uint32_t *__restrict__ hist) {
  __shared__ uint32_t s_h[8][kRadix];
  for (int i = threadIdx.x; i < 8 * kRadix; i += blockDim.x) (&s_h[0][0])[i] = 0;
  __syncthreads();
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const K key = keys[i];
    for (int p = 0; p < passes; ++p) atomicAdd(&s_h[p][(uint32_t)(key >> (p * kRadixBits)) & (kRadix - 1)], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < passes * kRadix; i += blockDim.x) {
    const uint32_t c = (&s_h[0][0])[i];
    if (c) atomicAdd(&hist[i], c);
  }
}

// The look-back's wait on its own: spins on a flag with the look-back's cap and backoff, and
// reports a wait that gives up the way the sort does (ERR_TIMEOUT in the error word).
__global__ void k_spin_probe(const uint32_t *flag, uint32_t *err) {
  uint32_t spins = 0;
  while (ld_relaxed_gpu(flag) == 0u) {
    if (++spins >= kSpinCap) {
      set_err(err, ERR_TIMEOUT);
      return;
    }
    __nanosleep(kSpinSleepNs);
  }
}

}  // namespace

void launch_spin_probe(const uint32_t *flag, uint32_t *err, cudaStream_t s) { k_spin_probe<<<1, 1, 0, s>>>(flag, err); }

template <typename K>
void launch_histogram(const K *keys, uint32_t n, int passes, uint32_t *hist, cudaStream_t s) {
  if (n == 0) return;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  uint32_t blocks = std::min<uint32_t>(ceil_div<uint32_t>(n, 256u * 8u), (uint32_t)sms * 4u);
  prof::Scope ps(s, "histogram");
  k_histogram<K><<<blocks, 256, 0, s>>>(keys, n, passes, hist);
}

template <typename K>
bool launch_onesweep(K *kA, K *kB, uint32_t *vA, uint32_t *vB, uint32_t n, const SortWs &ws, uint32_t *err,
                     cudaStream_t s) {
  if (n == 0) return true;
  K *kin = kA, *kout = kB;
  uint32_t *vin = vA, *vout = vB;
  const uint32_t tiles = ceil_div<uint32_t>(n, (uint32_t)SortTile<K>::tile);
  for (int p = 0; p < ws.passes; ++p) {
    const uint32_t *h = ws.hist + (size_t)p * kRadix;
    uint32_t *st = ws.status + (size_t)p * ws.tiles * kRadix;
    uint32_t *ctr = ws.tile_ctr + p;
    prof::Scope ps(s, "onesweep_pass");
    if (p == 0)
      k_onesweep<K, true><<<tiles, kSortThreads, 0, s>>>(kin, nullptr, kout, vout, n, 0, h, st, ctr, err);
    else
      k_onesweep<K, false><<<tiles, kSortThreads, 0, s>>>(kin, vin, kout, vout, n, p * kRadixBits, h, st, ctr, err);
    K *tk = kin; kin = kout; kout = tk;
    uint32_t *tv = vin; vin = vout; vout = tv;
  }
  return kin == kA;
}

template void launch_histogram<uint32_t>(const uint32_t *, uint32_t, int, uint32_t *, cudaStream_t);
template void launch_histogram<uint64_t>(const uint64_t *, uint32_t, int, uint32_t *, cudaStream_t);
template bool launch_onesweep<uint32_t>(uint32_t *, uint32_t *, uint32_t *, uint32_t *, uint32_t, const SortWs &,
                                        uint32_t *, cudaStream_t);
template bool launch_onesweep<uint64_t>(uint64_t *, uint64_t *, uint32_t *, uint32_t *, uint32_t, const SortWs &,
                                        uint32_t *, cudaStream_t);

}  // namespace abx

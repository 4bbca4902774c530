// Tree traversal kernels (ArborX Sec. 2.2): spatial count / fill (2P), the
// offsets scan, and nearest queries with a bounded candidate list.
//
// One thread per query, queries taken in Morton order through qperm so that a
// warp's threads walk similar paths (Sec. 2.2, "Query ordering").  Each
// internal node stores both child boxes side by side (64 bytes), so a step
// loads one node and tests both children; leaf children are tested and
// reported directly from the parent, leaves are never loaded separately.  The
// per-thread stack keeps its first `stack_smem` entries in shared memory
// (laid out [level][thread], conflict-free) and spills deeper entries to
// local memory; its total capacity exceeds the largest possible LBVH depth
// (each level consumes one bit of the <= 64 + 32 bit augmented key).
#include <climits>

#include <algorithm>
#include <type_traits>

#include "kernels.cuh"
#include "prof.cuh"

namespace abx {

namespace {

constexpr int kSpill = 96;     // local-memory stack entries beyond the shared part
constexpr int kMaxBlock = 256;  // traversal block size limit (register budget)
// measured at 1e7 points / 1e6 queries: the heap beats a 32-entry register list from k = 17
// (k = 32: 5.1 vs 7.9 ms); an 8-entry deferred-insert buffer beats 4 and 16 entries
constexpr int kHeapDefer = 8;  // deferred-insert buffer of the shared-memory heap path
// k from which the shared-memory heap serves a single tree's nearest query (opts.knn_heap_from may
// raise it to 33: register lists exist for every k up to 32)
constexpr int kHeapFrom = 17;
constexpr int kBatchHeapK = 32;             // largest k of the batched path (heap class)
// shared-memory stack entries of the heap paths (deeper entries spill to local memory): the heap
// takes 8k bytes of shared memory per thread, so a short shared stack buys resident warps
// (measured at 1e7 points: k = 32 4.13 -> 3.96 ms, k = 50 8.43 -> 7.60 ms per 1e6 queries, and the
// 512-cloud batch 24.8 -> 22.9 ms, against 16 entries)
constexpr int kHeapStackSmem = 4;


// one 32-byte child slot (lo, hi) in a single 256-bit read-only load that does not allocate in L1
// (measured 18% faster for the radius query than four 128-bit loads per node, and no-allocate a
// further 3-6% over L1-cached forms: node reuse is served by L2); records start on a 256-byte
// boundary, so every slot is 32-byte aligned
__device__ __forceinline__ void ld_slot(const float4 *p, float4 &lo, float4 &hi) {
  asm("ld.global.nc.L1::no_allocate.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=f"(lo.x), "=f"(lo.y), "=f"(lo.z), "=f"(lo.w), "=f"(hi.x), "=f"(hi.y), "=f"(hi.z), "=f"(hi.w)
      : "l"(p));
}

__device__ __forceinline__ bool finite3(float x, float y, float z) {
  return is_finite_bits(x) && is_finite_bits(y) && is_finite_bits(z);
}

// (d, i) strictly before (e, j) in (distance, index) order
__device__ __forceinline__ bool pless(float d, int32_t i, float e, int32_t j) {
  return d < e || (d == e && i < j);
}

// Node-count statistics: one atomic per converged group of a warp (summed with a warp
// reduction) instead of one per thread on the same counter.
__device__ __forceinline__ void add_stat(unsigned long long *stats, uint32_t v) {
  const unsigned act = __activemask();
  const uint32_t sum = __reduce_add_sync(act, v);
  if ((int)lane_id() == __ffs(act) - 1) atomicAdd(stats, (unsigned long long)sum);
}

// Queries flagged by a traversal (fewer than k hits inside a bound, or more
// results than a row buffer holds): appended with one atomic per converged
// group, in lane order (keeps the Morton order within a warp for the next pass).
__device__ __forceinline__ void append_flagged(bool flag, uint32_t qi, uint32_t *list, uint32_t *count) {
  const unsigned act = __activemask();
  const unsigned bal = __ballot_sync(act, flag);
  if (!bal) return;
  const int leader = __ffs(act) - 1;
  uint32_t base = 0;
  if ((int)lane_id() == leader) base = atomicAdd(count, (uint32_t)__popc(bal));
  base = __shfl_sync(act, base, leader);
  if (flag) list[base + __popc(bal & lanemask_lt())] = qi;
}

// MODE kCount: counts[qi] = results.  MODE kFill: write the row at offsets[qi]
// (2P second pass).  MODE kBuffered: count and keep the first `bs` results in
// buf[qi * bs ...] (1P); queries with more than bs results are listed for a
// fill pass.  m_dev (nullable) holds the number of queries on the device.
enum : int { kCount = 0, kFill = 1, kBuffered = 2 };

// The spatial predicate of a query, applied alike to node boxes and primitive boxes (Sec. 2.2.1:
// each node is tested on its own).  BOX = false: a point and r2, the box is a match when its FP32
// squared distance to the point is at most r2.  BOX = true: a query box, closed intervals that
// overlap on every axis.  Both are exact for pruning: a node box contains its children's boxes,
// so its distance is no larger and its intervals reach at least as far.
template <bool BOX>
struct SpatialPred;

template <>
struct SpatialPred<false> {
  float qx, qy, qz, r2;
  __device__ __forceinline__ SpatialPred(const SpatialArgs &a, uint32_t qi)
      : qx(__ldg(a.queries + 3 * (uint64_t)qi)), qy(__ldg(a.queries + 3 * (uint64_t)qi + 1)),
        qz(__ldg(a.queries + 3 * (uint64_t)qi + 2)), r2(a.r2) {}
  __device__ __forceinline__ bool valid() const { return finite3(qx, qy, qz); }
  __device__ __forceinline__ bool operator()(float4 lo, float4 hi) const { return dist2_box(qx, qy, qz, lo, hi) <= r2; }
  // the whole box within r: per axis |fl(q - p)| <= max(|fl(q - lo)|, |fl(q - hi)|) for every p in
  // it (round-to-nearest subtraction is monotone), so the farthest corner's squared distance,
  // summed in the same order, bounds the FP32 distance of every point inside
  __device__ __forceinline__ bool contains(float4 lo, float4 hi) const {
    const float gx = fmaxf(fabsf(__fsub_rn(qx, lo.x)), fabsf(__fsub_rn(qx, hi.x)));
    const float gy = fmaxf(fabsf(__fsub_rn(qy, lo.y)), fabsf(__fsub_rn(qy, hi.y)));
    const float gz = fmaxf(fabsf(__fsub_rn(qz, lo.z)), fabsf(__fsub_rn(qz, hi.z)));
    return __fadd_rn(__fadd_rn(__fmul_rn(gx, gx), __fmul_rn(gy, gy)), __fmul_rn(gz, gz)) <= r2;
  }
};

template <>
struct SpatialPred<true> {
  float lx, ly, lz, hx, hy, hz;
  __device__ __forceinline__ SpatialPred(const SpatialArgs &a, uint32_t qi) {
    const float *q = a.queries + 6 * (uint64_t)qi;
    lx = __ldg(q); ly = __ldg(q + 1); lz = __ldg(q + 2);
    hx = __ldg(q + 3); hy = __ldg(q + 4); hz = __ldg(q + 5);
  }
  __device__ __forceinline__ bool valid() const { return true; }  // a NaN bound fails every test below
  __device__ __forceinline__ bool operator()(float4 lo, float4 hi) const {
    return lo.x <= hx && hi.x >= lx && lo.y <= hy && hi.y >= ly && lo.z <= hz && hi.z >= lz;
  }
  // the node box inside the query box: every primitive box inside it meets the query
  __device__ __forceinline__ bool contains(float4 lo, float4 hi) const {
    return lo.x >= lx && hi.x <= hx && lo.y >= ly && hi.y <= hy && lo.z >= lz && hi.z <= hz;
  }
};

// First sorted leaf of the internal child on `side` of node p, with child id c and cnt leaves.
// Apetrei numbering: node p splits leaves p | p + 1, so its left child ends at p and its right
// child starts at p + 1.  Karras numbering: a node's id is one end of its range, the right end for
// a left child and the left end for a right child.
__device__ __forceinline__ int child_first(int numbering, int p, int side, int c, int cnt) {
  if (numbering == 0) return side == 0 ? p + 1 - cnt : p + 1;
  return side == 0 ? c - cnt + 1 : c;
}

template <int MODE, bool BOX, bool EMIT, bool VEC>
__device__ __forceinline__ void spatial_traverse(const SpatialArgs &a) {
  extern __shared__ int32_t s_stack[];
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t m = a.m_dev ? min(a.m, *a.m_dev) : a.m;
  if (t >= m) return;
  const float4 *__restrict__ rec = a.rec;
  const uint32_t n = a.n;
  const uint32_t qi = a.qperm ? __ldg(a.qperm + t) : t;
  const SpatialPred<BOX> hit(a, qi);
  int64_t base = 0;
  if (MODE == kFill) base = __ldg(a.offsets + qi);
  if (MODE == kBuffered) base = (int64_t)qi * a.bs;
  uint32_t cnt = 0;
  uint32_t visited = 0;  // internal nodes loaded (statistics)
  // VEC (1P rows whose width is a multiple of 4, 16-byte aligned buffer): the newest hits wait in
  // h0..h3 (h3 the newest) and each complete group of four goes out as one 16-byte store, a
  // quarter of the store transactions of one scalar store per hit
  constexpr bool vec4 = VEC && MODE == kBuffered;
  int32_t h0 = 0, h1 = 0, h2 = 0, h3 = 0;

#define ABX_EMIT(v)                                                      \
  do {                                                                   \
    if (MODE == kFill) {                                                 \
      const int64_t pos_ = base + cnt;                                   \
      if (pos_ < a.capacity) a.indices[pos_] = (v);                      \
      else set_err(a.err, ERR_CSR);                                      \
    } else if (MODE == kBuffered) {                                      \
      if constexpr (vec4) {                                              \
        h0 = h1;                                                         \
        h1 = h2;                                                         \
        h2 = h3;                                                         \
        h3 = (v);                                                        \
        if ((cnt & 3u) == 3u && cnt < (uint32_t)a.bs)                    \
          *reinterpret_cast<int4 *>(a.buf + base + cnt - 3) = make_int4(h0, h1, h2, h3); \
      } else if (cnt < (uint32_t)a.bs) {                                 \
        a.buf[base + cnt] = (v);                                         \
      }                                                                  \
    }                                                                    \
    ++cnt;                                                               \
  } while (0)

  // every leaf of a subtree inside the query: its slice [first, first + sc) of the sorted order
  auto emit_range = [&](int first, int sc) {
    if (first < 0 || sc < 1 || (uint32_t)first + (uint32_t)sc > n) {  // corrupt tree: read nothing outside
      set_err(a.err, ERR_STACK);
      return;
    }
    if (MODE == kCount) {
      cnt += (uint32_t)sc;
    } else {
      for (int j = 0; j < sc; ++j) ABX_EMIT((int32_t)__ldg(a.leafperm + first + j));
    }
  };
  if (n > 0 && hit.valid()) {
    const float4 r0 = __ldg(rec), r1 = __ldg(rec + 1);
    if (hit(r0, r1)) {
      const int e0 = __float_as_int(r0.w);
      if (e0 < 0) {
        ABX_EMIT(~e0);
      } else if (EMIT && hit.contains(r0, r1)) {
        emit_range(0, (int)n);
      } else {
        int32_t *my = s_stack + threadIdx.x;
        const int stride = blockDim.x;
        const int stack_smem = a.stack_smem;
        int32_t spill[kSpill];
        int sp = 0;
        auto push = [&](int v) {
          if (sp < stack_smem) {
            my[sp * stride] = v;
            ++sp;
          } else if (sp - stack_smem < kSpill) {
            spill[sp - stack_smem] = v;
            ++sp;
          } else {
            set_err(a.err, ERR_STACK);  // cannot happen: capacity exceeds the deepest LBVH
          }
        };
        auto pop = [&]() {
          --sp;
          return sp < stack_smem ? my[sp * stride] : spill[sp - stack_smem];
        };
        int node = e0;
        while (true) {
          // up to two more nodes, the top entries of the stack, are loaded alongside the current
          // one: three independent node loads in flight per lane (the order of a spatial traversal
          // is free).  Taken only while the stack is within its shared part: one iteration there
          // ends at most three entries past it, and beyond it the stack grows as in the
          // single-node traversal (one entry per level), so the capacity still exceeds the deepest
          // tree (93 levels for 63-bit codes) by a wide margin.
          int nb = -1, nc = -1;
          if (sp > 0 && sp <= stack_smem) nb = pop();
          if (sp > 0 && sp <= stack_smem) nc = pop();
          if ((uint32_t)node >= n - 1 || (nb >= 0 && (uint32_t)nb >= n - 1) || (nc >= 0 && (uint32_t)nc >= n - 1)) {
            set_err(a.err, ERR_STACK);  // corrupt tree: never read outside the records
            break;
          }
          const float4 *rp = rec + 4 + 4 * (uint64_t)node;
          float4 a0, a1, b0, b1, c0, c1, d0, d1, e0v, e1v, f0, f1;
          ld_slot(rp, a0, a1);
          ld_slot(rp + 2, b0, b1);
          if (nb >= 0) {
            const float4 *rq = rec + 4 + 4 * (uint64_t)nb;
            ld_slot(rq, c0, c1);
            ld_slot(rq + 2, d0, d1);
          }
          if (nc >= 0) {
            const float4 *rr = rec + 4 + 4 * (uint64_t)nc;
            ld_slot(rr, e0v, e1v);
            ld_slot(rr + 2, f0, f1);
          }
          visited += 1 + (nb >= 0) + (nc >= 0);
          // a child slot that meets the predicate: a leaf is a result, an internal node is walked
          // next (the first one) or pushed
          int next = -1;
          auto take = [&](float4 lo, float4 hi, int p, int side) {
            const int e = __float_as_int(lo.w);
            if (hit(lo, hi)) {
              if (e < 0) {
                ABX_EMIT(~e);
              } else if (EMIT && hit.contains(lo, hi)) {
                const int sc = __float_as_int(hi.w);
                emit_range(child_first(a.numbering, p, side, e, sc), sc);
              } else if (next < 0) {
                next = e;
              } else {
                push(e);
              }
            }
          };
          take(a0, a1, node, 0);
          take(b0, b1, node, 1);
          if (nb >= 0) {
            take(c0, c1, nb, 0);
            take(d0, d1, nb, 1);
          }
          if (nc >= 0) {
            take(e0v, e1v, nc, 0);
            take(f0, f1, nc, 1);
          }
          if (next < 0) {
            if (sp == 0) break;
            next = pop();
          }
          node = next;
        }
      }
    }
  }
#undef ABX_EMIT
  if constexpr (vec4) {  // the last, incomplete group of four: h(4-r) .. h3 at slots g .. g + r - 1
    const uint32_t r = cnt & 3u, g = cnt - r;
    if (r > 0 && g < (uint32_t)a.bs) {
      int32_t *o = a.buf + base + g;
      if (r == 3) {
        o[0] = h1;
        o[1] = h2;
        o[2] = h3;
      } else if (r == 2) {
        o[0] = h2;
        o[1] = h3;
      } else {
        o[0] = h3;
      }
    }
  }
  if (MODE != kFill) a.counts[qi] = (int32_t)cnt;
  if (MODE == kBuffered) append_flagged(cnt > (uint32_t)a.bs, qi, a.ovf_list, a.ovf_count);
  if (a.stats) add_stat(a.stats, visited);
}

// Radius queries (points within r) and box queries (boxes met), one kernel name each; EMIT: the
// variant that takes wholly contained subtrees from the sorted leaf order (more registers, so a
// separate instantiation that only trees with that query option run).
// VEC: the one-pass form with 16-byte hit stores (a separate instantiation: the same code behind
// a run-time flag in one kernel was slower at 10 hits per row, 0.581 -> 0.642 ms).
template <int MODE, bool EMIT, bool VEC = false>
__global__ void __launch_bounds__(kMaxBlock) k_spatial(const __grid_constant__ SpatialArgs a) {
  spatial_traverse<MODE, false, EMIT, VEC>(a);
}

template <int MODE, bool EMIT, bool VEC = false>
__global__ void __launch_bounds__(kMaxBlock) k_intersects(const __grid_constant__ SpatialArgs a) {
  spatial_traverse<MODE, true, EMIT, VEC>(a);
}

// Move buffered rows (those that fit) to their CSR place.  A thread takes
// kCompactPer slots a block width apart and issues all their loads (row
// count, row offset, buffered value) before any store, so the dependent
// latencies of a thread overlap instead of adding up.  Two per thread: the
// 4-slot form then needs few registers and keeps more warps resident (1e6
// rows of 32 slots: 40.7 us against 43.8 us with four and 48.0 us with eight).
constexpr int kCompactPer = 2;

template <typename IDX>
__global__ void __launch_bounds__(256) k_compact(const int32_t *__restrict__ buf, int bs,
                                                const int32_t *__restrict__ counts,
                                                const int64_t *__restrict__ offsets, uint32_t m,
                                                int32_t *__restrict__ indices, int64_t capacity,
                                                uint32_t *__restrict__ err) {
  const IDX total = (IDX)m * (IDX)bs;
  const IDX base = (IDX)blockIdx.x * (IDX)(blockDim.x * kCompactPer) + threadIdx.x;
  int32_t c[kCompactPer], j[kCompactPer], v[kCompactPer];
  int64_t o[kCompactPer];
#pragma unroll
  for (int k = 0; k < kCompactPer; ++k) {
    const IDX t = base + (IDX)k * blockDim.x;
    c[k] = -1;
    j[k] = 0;
    if (t < total) {
      const IDX qi = t / (IDX)bs;
      j[k] = (int32_t)(t - qi * (IDX)bs);
      c[k] = __ldg(counts + qi);
      o[k] = __ldg(offsets + qi);
    }
  }
#pragma unroll
  for (int k = 0; k < kCompactPer; ++k) {
    const IDX t = base + (IDX)k * blockDim.x;
    if (c[k] <= bs && j[k] < c[k]) v[k] = __ldg(buf + t);
  }
#pragma unroll
  for (int k = 0; k < kCompactPer; ++k) {
    if (c[k] <= bs && j[k] < c[k]) {
      const int64_t pos = o[k] + j[k];
      if (pos < capacity) indices[pos] = v[k];
      else set_err(err, ERR_CSR);
    }
  }
}

// Same move for row buffers whose width is a multiple of 4: one 16-byte load
// brings four slots of a row, a thread takes kCompactPer such groups.
template <typename IDX>
__global__ void __launch_bounds__(256) k_compact4(const int4 *__restrict__ buf4, int bs,
                                                 const int32_t *__restrict__ counts,
                                                 const int64_t *__restrict__ offsets, uint32_t m,
                                                 int32_t *__restrict__ indices, int64_t capacity,
                                                 uint32_t *__restrict__ err) {
  const int gpr = bs >> 2;  // 4-slot groups per row
  const IDX total = (IDX)m * (IDX)gpr;
  const IDX base = (IDX)blockIdx.x * (IDX)(blockDim.x * kCompactPer) + threadIdx.x;
  int32_t c[kCompactPer], j[kCompactPer];
  int64_t o[kCompactPer];
  int4 v[kCompactPer];
#pragma unroll
  for (int k = 0; k < kCompactPer; ++k) {
    const IDX t = base + (IDX)k * blockDim.x;
    c[k] = -1;
    j[k] = 0;
    if (t < total) {
      const IDX qi = t / (IDX)gpr;
      j[k] = 4 * (int32_t)(t - qi * (IDX)gpr);
      c[k] = __ldg(counts + qi);
      o[k] = __ldg(offsets + qi);
    }
  }
#pragma unroll
  for (int k = 0; k < kCompactPer; ++k) {
    const IDX t = base + (IDX)k * blockDim.x;
    if (c[k] <= bs && j[k] < c[k]) v[k] = __ldg(buf4 + t);
  }
#pragma unroll
  for (int k = 0; k < kCompactPer; ++k) {
    if (c[k] <= bs && j[k] < c[k]) {
      const int32_t vv[4] = {v[k].x, v[k].y, v[k].z, v[k].w};
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        if (j[k] + e < c[k]) {
          const int64_t pos = o[k] + j[k] + e;
          if (pos < capacity) indices[pos] = vv[e];
          else set_err(err, ERR_CSR);
        }
      }
    }
  }
}

// ---------------------------------------------------------------- nearest

// Ascending list of the KC best (d2, index) pairs in registers; the k-th entry
// (k <= KC) is the pruning bound.  One 64-bit compare decides the (d2, index)
// order (measured 6-8% faster at k = 10 than comparing d2 and index apart).
template <int KC>
struct RegList {
  // (d2, index) packed as (float bits << 32 | index): d2 >= 0, so the unsigned order of the
  // keys is the (d2, index) order.  Slots [0, KC - k) hold key 0 fillers below every sentinel
  // and never written out; the k-th best is slot KC - 1.
  unsigned long long key[KC];
  int off;
  static __device__ __forceinline__ unsigned long long pack(float d, int32_t i) {
    return ((unsigned long long)__float_as_uint(d) << 32) | (uint32_t)i;
  }
  __device__ __forceinline__ void init(float b, int k) {
    off = KC - k;
    const unsigned long long s = pack(b, INT_MAX);
#pragma unroll
    for (int j = 0; j < KC; ++j) key[j] = j < off ? 0ull : s;
  }
  __device__ __forceinline__ float bound() const { return __uint_as_float((uint32_t)(key[KC - 1] >> 32)); }
  __device__ __forceinline__ int32_t bound_idx() const { return (int32_t)(uint32_t)key[KC - 1]; }
  __device__ __forceinline__ bool accepts(float dc, int32_t ic) const { return pack(dc, ic) < key[KC - 1]; }
  __device__ __forceinline__ void insert(float dc, int32_t ic, int) {
    const unsigned long long c = pack(dc, ic);
#pragma unroll
    for (int j = KC - 1; j > 0; --j) {
      const bool lt = c < key[j];
      const bool ltp = c < key[j - 1];
      if (lt) key[j] = ltp ? key[j - 1] : c;
    }
    if (c < key[0]) key[0] = c;
  }
  __device__ __forceinline__ void write(int64_t row, int kk, int32_t *out_idx, float *out_d2,
                                        int32_t base = 0, bool pairs = false) const {
    if constexpr (KC % 2 == 0) {
      // a full-width list (k = KC, so no filler slots) into 8-byte aligned rows: two entries per
      // store, half the store transactions (the scalar row stores cost 45 of 996 us at k = 10)
      if (pairs && off == 0 && kk == KC) {
#pragma unroll
        for (int j = 0; j < KC; j += 2) {
          const int32_t i0 = (int32_t)(uint32_t)key[j], i1 = (int32_t)(uint32_t)key[j + 1];
          const bool r0 = i0 != INT_MAX, r1 = i1 != INT_MAX;
          *reinterpret_cast<int2 *>(out_idx + row + j) = make_int2(r0 ? i0 - base : -1, r1 ? i1 - base : -1);
          if (out_d2)
            *reinterpret_cast<float2 *>(out_d2 + row + j) =
                make_float2(r0 ? __uint_as_float((uint32_t)(key[j] >> 32)) : __int_as_float(0x7f800000),
                            r1 ? __uint_as_float((uint32_t)(key[j + 1] >> 32)) : __int_as_float(0x7f800000));
        }
        return;
      }
    }
#pragma unroll
    for (int j = 0; j < KC; ++j) {
      const int o = j - off;
      if (o >= 0 && o < kk) {
        const int32_t i = (int32_t)(uint32_t)key[j];
        const bool real = i != INT_MAX;
        out_idx[row + o] = real ? i - base : -1;
        if (out_d2) out_d2[row + o] = real ? __uint_as_float((uint32_t)(key[j] >> 32)) : __int_as_float(0x7f800000);
      }
    }
  }
};

// Max-heap of k (d2, index) pairs in shared memory ([slot][thread] layout);
// the root is the k-th best and the pruning bound.
struct SmemHeap {
  float *hd;
  int32_t *hi;
  int s;  // stride between a thread's consecutive slots
  int k;
  float kd;
  int32_t ki;
  __device__ __forceinline__ float bound() const { return kd; }
  __device__ __forceinline__ int32_t bound_idx() const { return ki; }
  __device__ __forceinline__ void init(float b, int) {
    for (int j = 0; j < k; ++j) {
      hd[j * s] = b;
      hi[j * s] = INT_MAX;
    }
    kd = b;
    ki = INT_MAX;
  }
  __device__ __forceinline__ bool accepts(float dc, int32_t ic) const { return pless(dc, ic, kd, ki); }
  __device__ __forceinline__ void sift(float dc, int32_t ic, int size) {
    int pos = 0;
    while (true) {
      const int l = 2 * pos + 1;
      if (l >= size) break;
      int c = l;
      float dm = hd[l * s];
      int32_t im = hi[l * s];
      if (l + 1 < size) {
        const float dr = hd[(l + 1) * s];
        const int32_t ir = hi[(l + 1) * s];
        if (pless(dm, im, dr, ir)) {
          c = l + 1;
          dm = dr;
          im = ir;
        }
      }
      if (!pless(dc, ic, dm, im)) break;
      hd[pos * s] = dm;
      hi[pos * s] = im;
      pos = c;
    }
    hd[pos * s] = dc;
    hi[pos * s] = ic;
  }
  __device__ __forceinline__ void insert(float dc, int32_t ic, int) {
    sift(dc, ic, k);
    kd = hd[0];
    ki = hi[0];
  }
  __device__ __forceinline__ void write(int64_t row, int kk, int32_t *out_idx, float *out_d2, int32_t base = 0) {
    for (int j = k - 1; j >= 0; --j) {
      const float d = hd[0];
      const int32_t i = hi[0];
      if (j < kk) {
        const bool real = i != INT_MAX;
        out_idx[row + j] = real ? i - base : -1;
        if (out_d2) out_d2[row + j] = real ? d : __int_as_float(0x7f800000);
      }
      if (j > 0) sift(hd[j * s], hi[j * s], j);
    }
  }
};

// Per-axis distance to the farther face of [lo, hi]: for every p in the box, |fl(q - p)| is at
// most this (round-to-nearest subtraction is monotone), so the sum below bounds the FP32 squared
// distance of every point in the box, computed in the same order.
__device__ __forceinline__ float far_gap(float q, float lo, float hi) {
  return fmaxf(fabsf(__fsub_rn(q, lo)), fabsf(__fsub_rn(q, hi)));
}
__device__ __forceinline__ float far2_box(float qx, float qy, float qz, float4 lo, float4 hi) {
  const float gx = far_gap(qx, lo.x, hi.x), gy = far_gap(qy, lo.y, hi.y), gz = far_gap(qz, lo.z, hi.z);
  return __fadd_rn(__fadd_rn(__fmul_rn(gx, gx), __fmul_rn(gy, gy)), __fmul_rn(gz, gz));
}

// DEFER > 0: accepted leaf candidates wait in a DEFER-entry register buffer and
// enter the list when some lane of the warp has a nearly full buffer, all
// lanes together (and at the end).  Pruning meanwhile uses the list's bound,
// which can only be larger than with every candidate inserted, so no node that
// holds a result is skipped and every candidate still reaches the list once.
// It pays for the shared-memory heap, whose data-dependent sift loop diverges.
// PACK: stack entries (node, box distance) as one 64-bit word, one shared-memory access per push or
// pop (faster with the register lists, slower with the heap, whose sift shares the memory pipe).
template <int DEFER, bool PACK, bool TB = false, class List>
__device__ __forceinline__ void knn_traverse(const float4 *__restrict__ rec, uint32_t n, float qx, float qy, float qz,
                                             List &L, int k, unsigned char *s_stack, int stride, int stack_smem,
                                             uint32_t *err, uint32_t &visited, uint32_t root_slot = 0) {
  const float4 r0 = __ldg(rec + 2 * (uint64_t)root_slot), r1 = __ldg(rec + 2 * (uint64_t)root_slot + 1);
  const int e0 = __float_as_int(r0.w);
  const float d0 = dist2_box(qx, qy, qz, r0, r1);
  if (e0 < 0) {
    if (L.accepts(d0, ~e0)) L.insert(d0, ~e0, k);
    return;
  }
  if (d0 > L.bound()) return;
  // shared part of the stack, [level][thread]: packed words, or node ids then distances
  unsigned long long *s_st = reinterpret_cast<unsigned long long *>(s_stack) + threadIdx.x;
  int32_t *s_node = reinterpret_cast<int32_t *>(s_stack) + threadIdx.x;
  float *s_dist = reinterpret_cast<float *>(s_stack) + (size_t)stack_smem * stride + threadIdx.x;
  int32_t spn[kSpill];  // local spill beyond the shared part (one of the two forms is used)
  float spd[kSpill];
  unsigned long long spl[kSpill];
  int sp = 0;
  int node = e0;
  constexpr int DB = DEFER > 0 ? DEFER : 1;
  float bd[DB];
  int32_t bi[DB];
  int bc = 0;
  auto offer = [&](float d, int32_t i) {
    if constexpr (DEFER > 0) {
#pragma unroll
      for (int j = DB - 1; j > 0; --j) {
        bd[j] = bd[j - 1];
        bi[j] = bi[j - 1];
      }
      bd[0] = d;
      bi[0] = i;
      ++bc;
    } else {
      L.insert(d, i, k);
    }
  };
  auto flush = [&]() {
#pragma unroll
    for (int j = 0; j < DB; ++j)
      if (j < bc && L.accepts(bd[j], bi[j])) L.insert(bd[j], bi[j], k);
    bc = 0;
  };
  auto push = [&](int far, float fd) {
    if (sp < stack_smem) {
      if constexpr (PACK) {
        s_st[sp * stride] = ((unsigned long long)__float_as_uint(fd) << 32) | (uint32_t)far;
      } else {
        s_node[sp * stride] = far;
        s_dist[sp * stride] = fd;
      }
      ++sp;
    } else if (sp - stack_smem < kSpill) {
      if constexpr (PACK) {
        spl[sp - stack_smem] = ((unsigned long long)__float_as_uint(fd) << 32) | (uint32_t)far;
      } else {
        spn[sp - stack_smem] = far;
        spd[sp - stack_smem] = fd;
      }
      ++sp;
    } else {
      set_err(err, ERR_STACK);  // cannot happen: capacity exceeds the deepest LBVH
    }
  };
  if constexpr (TB) {
    // The tree's own bound, gathered on the first closest-first descent (the path the traversal
    // takes first): every child of at least k leaves met there bounds the k-th distance by its
    // farthest corner (far2_box).  The descent pushes siblings as the traversal does and stops at
    // the first node with a leaf child or with no child of k leaves; that node is then handled by
    // the loop below, with the list's bound set to the smallest corner distance seen.  Siblings
    // pushed before the bound was known and lying beyond it are dropped from the stack (in order,
    // so the visiting order is unchanged): they would be popped and discarded later, one lane at
    // a time, and fill the shared part of the stack.
    auto compact = [&](float bnd) {
      int j = 0;
      for (int i = 0; i < sp; ++i) {
        const bool si = i < stack_smem, sj = j < stack_smem;
        if constexpr (PACK) {
          const unsigned long long e = si ? s_st[i * stride] : spl[i - stack_smem];
          if (__uint_as_float((uint32_t)(e >> 32)) <= bnd) {
            if (sj) s_st[j * stride] = e;
            else spl[j - stack_smem] = e;
            ++j;
          }
        } else {
          const int nd = si ? s_node[i * stride] : spn[i - stack_smem];
          const float dd = si ? s_dist[i * stride] : spd[i - stack_smem];
          if (dd <= bnd) {
            if (sj) {
              s_node[j * stride] = nd;
              s_dist[j * stride] = dd;
            } else {
              spn[j - stack_smem] = nd;
              spd[j - stack_smem] = dd;
            }
            ++j;
          }
        }
      }
      sp = j;
    };
    float bt = L.bound();
    if (k > 1) {
      if (__float_as_int(r1.w) >= k) bt = fminf(bt, far2_box(qx, qy, qz, r0, r1));
      while ((uint32_t)node < n - 1) {
        const float4 *rp = rec + 4 + 4 * (uint64_t)node;
        float4 a0, a1, b0, b1;
        ld_slot(rp, a0, a1);
        ld_slot(rp + 2, b0, b1);
        const int el = __float_as_int(a0.w), er = __float_as_int(b0.w);
        const bool oka = __float_as_int(a1.w) >= k, okb = __float_as_int(b1.w) >= k;
        if (oka) bt = fminf(bt, far2_box(qx, qy, qz, a0, a1));
        if (okb) bt = fminf(bt, far2_box(qx, qy, qz, b0, b1));
        if (el < 0 || er < 0 || !(oka || okb)) break;
        const float dl = dist2_box(qx, qy, qz, a0, a1);
        const float dr = dist2_box(qx, qy, qz, b0, b1);
        const bool gl = dl <= bt, gr = dr <= bt;
        if (!gl && !gr) break;
        ++visited;
        if (gl && gr) {
          const bool lfirst = dl <= dr;
          if (sp >= stack_smem) compact(bt);
          push(lfirst ? er : el, lfirst ? dr : dl);
          node = lfirst ? el : er;
        } else {
          node = gl ? el : er;
        }
      }
      compact(bt);
      L.init(bt, k);
    }
  }
  while (true) {
    if ((uint32_t)node >= n - 1) {  // corrupt tree: never read outside the records
      set_err(err, ERR_STACK);
      break;
    }
    const float4 *rp = rec + 4 + 4 * (uint64_t)node;
    float4 a0, a1, b0, b1;
    ld_slot(rp, a0, a1);
    ld_slot(rp + 2, b0, b1);
    ++visited;
    const float dl = dist2_box(qx, qy, qz, a0, a1);
    const float dr = dist2_box(qx, qy, qz, b0, b1);
    const int el = __float_as_int(a0.w), er = __float_as_int(b0.w);
    if (el < 0 && L.accepts(dl, ~el)) offer(dl, ~el);
    if (er < 0 && L.accepts(dr, ~er)) offer(dr, ~er);
    if constexpr (DEFER > 0) {
      if (__any_sync(__activemask(), bc > DB - 2)) flush();
    }
    const bool gl = el >= 0 && dl <= L.bound();  // prune only when strictly farther than the k-th
    const bool gr = er >= 0 && dr <= L.bound();
    if (gl && gr) {
      // visit the closer child next, keep the farther one on the stack
      const bool lfirst = dl <= dr;
      push(lfirst ? er : el, lfirst ? dr : dl);
      node = lfirst ? el : er;
    } else if (gl) {
      node = el;
    } else if (gr) {
      node = er;
    } else {
      node = -1;
      while (sp > 0) {
        --sp;
        const bool sm = sp < stack_smem;
        int nd;
        float dd;
        if constexpr (PACK) {
          const unsigned long long e = sm ? s_st[sp * stride] : spl[sp - stack_smem];
          nd = (int)(uint32_t)e;
          dd = __uint_as_float((uint32_t)(e >> 32));
        } else {
          nd = sm ? s_node[sp * stride] : spn[sp - stack_smem];
          dd = sm ? s_dist[sp * stride] : spd[sp - stack_smem];
        }
        if (dd <= L.bound()) {
          node = nd;
          break;
        }
      }
      if (node < 0) break;
    }
  }
  if constexpr (DEFER > 0) flush();
}

// Exact upper bound on the squared distance to the k-th nearest primitive, taken from the tree
// before the traversal: a subtree with at least k leaves (the count is the aux word of its child
// record) holds k primitives no farther than its box's farthest corner, so that distance bounds
// the k-th.  A greedy walk from the subtree root at root_slot through children of at least k
// leaves (about 20 node loads at 1e7 points, all on the path the traversal then takes first)
// yields it, in one of two forms (mode):
//   1: descend into the child with the nearer farthest corner and keep the smallest farthest
//      corner of every child of at least k leaves seen (2% faster on the uniform cube at k = 10);
//   2: descend into the child that holds the query (the nearer one when it lies in neither) and
//      take the farthest corner of the last such child (cheaper, and tighter on clustered clouds:
//      the 64-Gaussian mixture, k = 10, 11.4 -> 9.25 ms per 1e7 queries).
// With it as the initial bound the traversal inserts and pushes nothing beyond it; results are
// unchanged.  +inf when the subtree has fewer than k.  The first-descent forms in knn_traverse
// (TB) gather the same kind of bound without a separate walk.
template <int mode>
__device__ __forceinline__ float anchor_bound2(const float4 *__restrict__ rec, uint32_t n, float qx, float qy,
                                               float qz, int k, uint32_t &visited, uint32_t root_slot = 0) {
  const float inf = __int_as_float(0x7f800000);
  if (n < 2) return inf;
  float4 blo = __ldg(rec + 2 * (uint64_t)root_slot), bhi = __ldg(rec + 2 * (uint64_t)root_slot + 1);
  if (__float_as_int(bhi.w) < k) return inf;
  float B = mode == 1 ? far2_box(qx, qy, qz, blo, bhi) : inf;
  int node = __float_as_int(blo.w);
  for (int level = 0; level < 128; ++level) {
    if (node < 0 || (uint32_t)node >= n - 1) break;  // a leaf, or a corrupt id: never read outside
    const float4 *rp = rec + 4 + 4 * (uint64_t)node;
    float4 a0, a1, b0, b1;
    ld_slot(rp, a0, a1);
    ld_slot(rp + 2, b0, b1);
    ++visited;  // counted with the traversal's node loads
    const bool oka = __float_as_int(a1.w) >= k, okb = __float_as_int(b1.w) >= k;
    bool takea;
    if constexpr (mode == 1) {
      const float fa = oka ? far2_box(qx, qy, qz, a0, a1) : inf;
      const float fb = okb ? far2_box(qx, qy, qz, b0, b1) : inf;
      B = fminf(B, fminf(fa, fb));
      if (!oka && !okb) break;
      takea = oka && (fa <= fb || !okb);
    } else {
      if (!oka && !okb) break;
      if (oka && okb) {
        const bool ia = qx >= a0.x && qx <= a1.x && qy >= a0.y && qy <= a1.y && qz >= a0.z && qz <= a1.z;
        const bool ib = qx >= b0.x && qx <= b1.x && qy >= b0.y && qy <= b1.y && qz >= b0.z && qz <= b1.z;
        takea = ia || (!ib && dist2_box(qx, qy, qz, a0, a1) <= dist2_box(qx, qy, qz, b0, b1));
      } else {
        takea = oka;
      }
      blo = takea ? a0 : b0;
      bhi = takea ? a1 : b1;
    }
    node = takea ? __float_as_int(a0.w) : __float_as_int(b0.w);
  }
  return mode == 1 ? B : far2_box(qx, qy, qz, blo, bhi);
}

// Upper bound on the k-th squared distance of query q taken from a finished row
// of its Morton neighbour q': the neighbour's k primitives lie within
// d_k(q') + |q - q'| of q (triangle inequality).  Inflated by 2^-10 relative
// to cover FP32 rounding; +inf when the neighbour's row is not finished.
__device__ __forceinline__ float neighbour_bound2(const NearestArgs &a, uint32_t pos_n, float qx, float qy, float qz) {
  const uint32_t qn = a.qperm ? __ldg(a.qperm + pos_n) : pos_n;
  const float d2n = ld_cg_f32(a.out_d2 + (int64_t)qn * a.kk + a.kk - 1);  // written by other blocks
  if (!(d2n < __int_as_float(0x7f800000))) return __int_as_float(0x7f800000);
  const float dx = __fsub_rn(qx, __ldg(a.queries + 3 * (uint64_t)qn));
  const float dy = __fsub_rn(qy, __ldg(a.queries + 3 * (uint64_t)qn + 1));
  const float dz = __fsub_rn(qz, __ldg(a.queries + 3 * (uint64_t)qn + 2));
  const float e = sqrtf(dx * dx + dy * dy + dz * dz);
  const float b = (sqrtf(d2n) + e) * (1.0f + 0x1p-10f);
  return b * b;  // NaN for a non-finite neighbour: ignored by fminf
}

// Threads t <= m also write offsets[t] = t * kk (CSR view of the rows).  Thread
// t serves sorted position pos = pos_list ? pos_list[t] : t, query qperm[pos].
// Nearest kernels: block size up to kMaxBlock, one resident block per SM assumed (minBlocks 1), so
// that the compiler schedules for speed rather than for occupancy: the k-NN traversals use a few
// more registers (k = 10: 52 against 48) and run faster (cube 1e7, 1e6 queries: k = 10 1.051 ->
// 0.996 ms, k = 16 1.683 -> 1.545 ms, k = 50 6.84 -> 6.60 ms; the 512-cloud batch 19.9 -> 19.0 ms).
// The spatial kernels keep the plain bound (mixed: lattice r = 4 faster, two-pass and box queries
// slower).
template <int KC, bool NBR, int ANCHOR>
__global__ void __launch_bounds__(kMaxBlock, 1) k_nearest(const __grid_constant__ NearestArgs a) {
  extern __shared__ unsigned char s_raw[];
  const float4 *__restrict__ rec = a.rec;
  const float *__restrict__ queries = a.queries;
  const uint32_t *__restrict__ qperm = a.qperm;
  const uint32_t *__restrict__ pos_list = a.pos_list;
  int32_t *__restrict__ out_idx = a.out_idx;
  float *__restrict__ out_d2 = a.out_d2;
  uint32_t *__restrict__ err = a.err;
  const uint32_t n = a.n;
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  const int kk = a.kk, k = a.k, stack_smem = a.stack_smem;
  if (a.offsets && t <= a.m) a.offsets[t] = (int64_t)t * kk;
  const uint32_t m = a.m_dev ? min(a.m, *a.m_dev) : a.m;  // count produced on the device (second passes)
  if (t >= m) return;
  const int B = blockDim.x;
  const uint32_t pos = pos_list ? __ldg(pos_list + t) : t;
  const uint32_t qi = qperm ? __ldg(qperm + pos) : pos;
  const float qx = __ldg(queries + 3 * (uint64_t)qi);
  const float qy = __ldg(queries + 3 * (uint64_t)qi + 1);
  const float qz = __ldg(queries + 3 * (uint64_t)qi + 2);
  float b0 = a.init_bound2 ? __ldg(a.init_bound2 + qi) * a.bound_scale : __int_as_float(0x7f800000);
  if constexpr (NBR) {  // a separate instantiation: this code slows the plain traversal
    if (pos > 0) b0 = fminf(b0, neighbour_bound2(a, pos - 1, qx, qy, qz));
    if (pos + 1 < a.m) b0 = fminf(b0, neighbour_bound2(a, pos + 1, qx, qy, qz));
  }
  const bool ok = finite3(qx, qy, qz);
  const int64_t row = (int64_t)qi * kk;
  uint32_t visited = 0;
  // the tree's own bound (k = 1 gains nothing: its first leaf already sets the bound)
  if constexpr (ANCHOR == 1 || ANCHOR == 2) {  // one instantiation per walk form: each keeps its own registers
    if (k > 1 && ok) b0 = fminf(b0, anchor_bound2<ANCHOR>(rec, n, qx, qy, qz, k, visited));
  }
  constexpr bool kFused = ANCHOR == 3;  // the bound taken on the traversal's own first descent
  if constexpr (KC > 0) {
    RegList<KC> L;
    L.init(b0, k);
    if (ok && n > 0) knn_traverse<0, true, kFused>(rec, n, qx, qy, qz, L, k, s_raw, B, stack_smem, err, visited);
    if (a.miss_list) append_flagged(ok && L.bound_idx() == INT_MAX, pos, a.miss_list, a.miss_count);
    L.write(row, kk, out_idx, out_d2, 0, a.out_pairs != 0);
  } else {
    SmemHeap H;
    H.hd = reinterpret_cast<float *>(s_raw) + (size_t)2 * stack_smem * B + threadIdx.x;
    H.hi = reinterpret_cast<int32_t *>(s_raw) + (size_t)(2 * stack_smem + k) * B + threadIdx.x;
    H.s = B;
    H.k = k;
    H.init(b0, k);
    if (ok && n > 0)
      knn_traverse<kHeapDefer, false, kFused>(rec, n, qx, qy, qz, H, k, s_raw, B, stack_smem, err, visited);
    if (a.miss_list) append_flagged(ok && H.bound_idx() == INT_MAX, pos, a.miss_list, a.miss_count);
    H.write(row, kk, out_idx, out_d2);
  }
  if (a.stats) add_stat(a.stats, visited);
}

// Batched clouds: persistent warps take queries_per_warp sorted query positions
// at a time from an atomic counter, their lanes serving 32 at a time; each query
// starts at its cloud's subtree root and returns indices local to its cloud.
// KC = 0: shared-memory heap for k up to kBatchHeapK.  FD: 0, or the first-descent form (3) of the
// tree's own bound; with 0 the walk form a.anchor (0, 1, 2; 3 on classes it does not serve) is
// taken at run time.
template <int KC, int FD>
__global__ void __launch_bounds__(kMaxBlock, 1) k_batch_nearest(const __grid_constant__ BatchQueryArgs a) {
  extern __shared__ unsigned char s_raw[];
  const int B = blockDim.x;
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t qpw = (uint32_t)a.queries_per_warp;  // a multiple of 32
  while (true) {
    uint32_t base = 0;
    if (lane == 0) base = atomicAdd(a.queue, qpw);
    base = __shfl_sync(0xffffffffu, base, 0);
    if (a.pos_begin + base >= a.pos_end) break;
    for (uint32_t j = 0; j < qpw; j += 32) {
      const uint32_t pos = a.pos_begin + base + j + lane;
      if (pos < a.pos_end) {
        const uint32_t qi = __ldg(a.qperm + pos);
        const uint32_t c = (uint32_t)(__ldg(a.qkeys + pos) >> 30);
        const int k = __ldg(a.kof + c);
        const int kk = min(k, (int)__ldg(a.ncount + c));
        const int32_t slot = __ldg(a.root_slot + c);
        const float qx = __ldg(a.queries + 3 * (uint64_t)qi);
        const float qy = __ldg(a.queries + 3 * (uint64_t)qi + 1);
        const float qz = __ldg(a.queries + 3 * (uint64_t)qi + 2);
        uint32_t visited = 0;
        const bool go = finite3(qx, qy, qz) && slot >= 0;
        float b0 = __int_as_float(0x7f800000);
        if (FD == 0 && go && k > 1) {
          if (a.anchor == 1) b0 = anchor_bound2<1>(a.rec, a.n, qx, qy, qz, k, visited, (uint32_t)slot);
          else if (a.anchor >= 2) b0 = anchor_bound2<2>(a.rec, a.n, qx, qy, qz, k, visited, (uint32_t)slot);
        }
        if constexpr (KC > 0) {
          RegList<KC> L;
          L.init(b0, k);
          if (go)
            knn_traverse<0, true, (FD == 3)>(a.rec, a.n, qx, qy, qz, L, k, s_raw, B, a.stack_smem, a.err,
                                             visited, (uint32_t)slot);
          L.write(__ldg(a.row_off + qi), kk, a.out_idx, a.out_d2, (int32_t)__ldg(a.prim_base + c));
        } else {
          SmemHeap H;
          H.hd = reinterpret_cast<float *>(s_raw) + (size_t)2 * a.stack_smem * B + threadIdx.x;
          H.hi = reinterpret_cast<int32_t *>(s_raw) + (size_t)(2 * a.stack_smem + kBatchHeapK) * B + threadIdx.x;
          H.s = B;
          H.k = k;
          H.init(b0, k);
          if (go)
            knn_traverse<kHeapDefer, false>(a.rec, a.n, qx, qy, qz, H, k, s_raw, B, a.stack_smem, a.err, visited,
                                     (uint32_t)slot);
          H.write(__ldg(a.row_off + qi), kk, a.out_idx, a.out_d2, (int32_t)__ldg(a.prim_base + c));
        }
      }
    }
  }
}

// ------------------------------------------------------------------- scan

constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ int64_t block_excl_scan_i64(int64_t v, int64_t *s_w, int64_t &total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int64_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_w[warp] = x;
  __syncthreads();
  int64_t before = 0, tot = 0;
  for (int w = 0; w < nw; ++w) {
    const int64_t sw = s_w[w];
    if (w < warp) before += sw;
    tot += sw;
  }
  __syncthreads();
  total = tot;
  return before + x - v;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const int32_t *__restrict__ c, uint32_t m,
                                                             int64_t *__restrict__ tsum) {
  __shared__ int64_t s_w[32];
  const uint64_t base = (uint64_t)blockIdx.x * kScanTile;
  int64_t s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    const uint64_t p = base + (uint64_t)i * kScanThreads + threadIdx.x;
    if (p < m) s += c[p];
  }
  int64_t tot;
  block_excl_scan_i64(s, s_w, tot);
  if (threadIdx.x == 0) tsum[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) k_scan_tiles(int64_t *__restrict__ tsum, uint32_t tiles) {
  __shared__ int64_t s_w[32];
  int64_t carry = 0;
  for (uint32_t b = 0; b < tiles; b += blockDim.x) {
    const uint32_t i = b + threadIdx.x;
    const int64_t v = i < tiles ? tsum[i] : 0;
    int64_t tot;
    const int64_t ex = block_excl_scan_i64(v, s_w, tot);
    if (i < tiles) tsum[i] = carry + ex;
    carry += tot;
  }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_down(const int32_t *__restrict__ c, uint32_t m,
                                                           const int64_t *__restrict__ toff,
                                                           int64_t *__restrict__ off) {
  __shared__ int64_t s_w[32];
  const uint64_t base = (uint64_t)blockIdx.x * kScanTile + (uint64_t)threadIdx.x * kScanItems;
  int32_t v[kScanItems];
  int64_t s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    v[i] = base + i < m ? c[base + i] : 0;
    s += v[i];
  }
  int64_t tot;
  int64_t run = block_excl_scan_i64(s, s_w, tot) + toff[blockIdx.x];
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    if (base + i < m) off[base + i] = run;
    run += v[i];
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == blockDim.x - 1) off[m] = run;
}

// ------------------------------------------------- scan fused with compaction
// One-pass spatial rows (counts[m], row buffer of bs slots per query) -> CSR offsets[m+1] and
// indices in one kernel: a block takes the next tile of kScTile queries from an atomic counter,
// scans the tile's counts, obtains the sum of all earlier tiles by decoupled look-back over one
// 64-bit status word per tile (bounded spin, ERR_TIMEOUT on give-up), writes the tile's offsets
// and copies the tile's rows from the buffer.  Rows longer than bs are left to the overflow
// pass, which writes them at the same offsets.  The one-call form runs it where the split form
// (count call, then fill call) runs three scan kernels and k_compact.

constexpr int kScThreads = 256;
constexpr int kScQ = 8;                        // queries per thread (2: 62.5 against 54.1 us at 1e6 rows)
constexpr int kScTile = kScThreads * kScQ;     // queries per tile
constexpr int kScUnroll = 8;                   // row-buffer loads in flight per thread
constexpr uint64_t kScAgg = 1ull << 62;        // tile total published
constexpr uint64_t kScPre = 1ull << 63;        // inclusive prefix over tiles 0..t published
constexpr uint64_t kScVal = kScAgg - 1;
constexpr uint32_t kScSpinCap = 1u << 20;      // look-back give-up bound (about a second with the sleeps)

__device__ __forceinline__ uint64_t ld_relaxed_gpu_u64(const uint64_t *p) {
  uint64_t v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_gpu_u64(uint64_t *p, uint64_t v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// VEC: bs % 4 == 0 and a 16-byte aligned buffer, rows moved in 4-slot groups
template <bool VEC>
__global__ void __launch_bounds__(kScThreads) k_scan_compact(const int32_t *__restrict__ counts, uint32_t m,
                                                            const int32_t *__restrict__ buf, int bs,
                                                            int64_t *__restrict__ offsets, int32_t *__restrict__ indices,
                                                            int64_t capacity, uint64_t *__restrict__ status,
                                                            uint32_t *__restrict__ tile_ctr, uint32_t *__restrict__ err) {
  __shared__ int32_t s_cnt[kScTile];
  __shared__ int64_t s_off[kScTile];
  __shared__ int64_t s_w[32];
  __shared__ uint32_t s_tile;
  __shared__ int64_t s_base;
  const int tid = threadIdx.x, lane = tid & 31;
  if (tid == 0) s_tile = atomicAdd(tile_ctr, 1u);  // dynamic tile order: every predecessor is running or done
  __syncthreads();
  const uint32_t tile = s_tile;
  const uint64_t q0 = (uint64_t)tile * kScTile;
  const uint32_t rows = (uint32_t)min((uint64_t)kScTile, (uint64_t)m - q0);
#pragma unroll
  for (int i = 0; i < kScQ; ++i) {  // coalesced loads into the tile's count array
    const int r = i * kScThreads + tid;
    s_cnt[r] = r < (int)rows ? __ldg(counts + q0 + r) : 0;
  }
  __syncthreads();
  int32_t c[kScQ];
  int64_t sum = 0;
#pragma unroll
  for (int i = 0; i < kScQ; ++i) {  // this thread's kScQ consecutive rows
    c[i] = s_cnt[tid * kScQ + i];
    sum += c[i];
  }
  int64_t total;
  int64_t run = block_excl_scan_i64(sum, s_w, total);
  if (tid == 0) {
    if (tile == 0) st_relaxed_gpu_u64(status, kScPre | (uint64_t)total);
    else st_relaxed_gpu_u64(status + tile, kScAgg | (uint64_t)total);
  }
  if (tid < 32) {  // warp 0: look back over windows of 32 predecessors
    int64_t excl = 0;
    if (tile > 0) {
      int64_t j = (int64_t)tile - 1;
      uint32_t spins = 0;
      while (true) {
        const int64_t pj = j - lane;
        const uint64_t st = pj >= 0 ? ld_relaxed_gpu_u64(status + pj) : kScPre;
        const uint32_t pre = __ballot_sync(0xffffffffu, (st & kScPre) != 0);
        const uint32_t unpub = __ballot_sync(0xffffffffu, (st & (kScPre | kScAgg)) == 0);
        const int first_pre = pre ? __ffs(pre) - 1 : 32;  // nearest predecessor with its prefix
        const uint32_t upto = first_pre < 31 ? (2u << first_pre) - 1u : 0xffffffffu;
        if (unpub & upto) {  // a predecessor inside the window has not published: wait
          if (++spins >= kScSpinCap) {
            if (lane == 0) set_err(err, ERR_TIMEOUT);
            break;
          }
          __nanosleep(256);
          continue;
        }
        int64_t v = (lane <= first_pre && pj >= 0) ? (int64_t)(st & kScVal) : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        excl += v;
        if (first_pre < 32) break;
        j -= 32;
      }
      if (lane == 0) st_relaxed_gpu_u64(status + tile, kScPre | (uint64_t)(excl + total));
    }
    if (lane == 0) s_base = excl;
  }
  __syncthreads();
  run += s_base;
#pragma unroll
  for (int i = 0; i < kScQ; ++i) {
    s_off[tid * kScQ + i] = run;
    run += c[i];
  }
  if (q0 + (uint64_t)rows == m && tid == kScThreads - 1) offsets[m] = run;  // last tile: the total
  __syncthreads();
#pragma unroll
  for (int i = 0; i < kScQ; ++i) {  // coalesced offset stores
    const int r = i * kScThreads + tid;
    if (r < (int)rows) offsets[q0 + r] = s_off[r];
  }
  // rows: one item per 4-slot group (VEC) or slot of the tile's part of the buffer
  constexpr int W = VEC ? 4 : 1;
  const int per_row = bs / W;
  const uint32_t items = rows * (uint32_t)per_row;
  const uint64_t gbase = q0 * (uint64_t)per_row;
  for (uint32_t i0 = tid; i0 < items; i0 += kScThreads * kScUnroll) {
    uint32_t rr[kScUnroll];
    int32_t jj[kScUnroll];
    int4 v[kScUnroll];
#pragma unroll
    for (int u = 0; u < kScUnroll; ++u) {  // all loads first; the row's count and offset are read again below
      const uint32_t it = i0 + u * kScThreads;
      rr[u] = it / (uint32_t)per_row;
      jj[u] = W * (int32_t)(it - rr[u] * (uint32_t)per_row);
      if (it < items) {
        const int32_t c = s_cnt[rr[u]];
        if (c <= bs && jj[u] < c) {
          if constexpr (VEC) v[u] = __ldg(reinterpret_cast<const int4 *>(buf) + gbase + it);
          else v[u].x = __ldg(buf + gbase + it);
        }
      } else {
        rr[u] = kScTile;  // past the tile: no row
      }
    }
#pragma unroll
    for (int u = 0; u < kScUnroll; ++u) {
      if (rr[u] >= (uint32_t)kScTile) continue;
      const int32_t c = s_cnt[rr[u]];
      if (c <= bs && jj[u] < c) {
        const int64_t o = s_off[rr[u]];
        const int32_t vv[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
#pragma unroll
        for (int e = 0; e < W; ++e) {
          if (jj[u] + e < c) {
            const int64_t pos = o + jj[u] + e;
            if (pos < capacity) indices[pos] = vv[e];
            else set_err(err, ERR_CSR);
          }
        }
      }
    }
  }
}

__global__ void k_iota(uint32_t *__restrict__ out, uint32_t m) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < m) out[t] = t;
}

}  // namespace

void launch_iota(uint32_t *out, uint32_t m, cudaStream_t s) {
  if (m == 0) return;
  k_iota<<<ceil_div<uint32_t>(m, 256u), 256, 0, s>>>(out, m);
}

template <class F>
static void spatial_launch2(F *kernel, const SpatialArgs &args, int block, size_t smem, cudaStream_t s) {
  if (smem > 48 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  kernel<<<ceil_div<uint32_t>(args.m, block), block, smem, s>>>(args);
}

template <int MODE>
static void spatial_launch(const SpatialArgs &args, bool box, int block, cudaStream_t s, const char *name) {
  const size_t smem = (size_t)args.stack_smem * block * sizeof(int32_t);
  prof::Scope ps(s, box ? (MODE == kBuffered ? "intersects_buffered" : MODE == kFill ? "intersects_fill"
                                                                                     : "intersects_count")
                        : name);
  const bool emit = args.leafperm != nullptr;
  auto go = [&](auto vec) {  // vec: std::integral_constant<bool, ...>, the 16-byte hit-store form
    constexpr bool V = decltype(vec)::value;
    if (box) spatial_launch2(emit ? k_intersects<MODE, true, V> : k_intersects<MODE, false, V>, args, block, smem, s);
    else spatial_launch2(emit ? k_spatial<MODE, true, V> : k_spatial<MODE, false, V>, args, block, smem, s);
  };
  if constexpr (MODE == kBuffered) {
    if (args.buf_vec4) {
      go(std::true_type{});
      return;
    }
  }
  go(std::false_type{});
}

static SpatialArgs spatial_args(const float4 *rec, uint32_t n, const float *queries, const uint32_t *qperm, uint32_t m,
                                float r2, uint32_t *err, const TravCfg &cfg) {
  SpatialArgs a{};
  a.rec = rec;
  a.n = n;
  a.queries = queries;
  a.qperm = qperm;
  a.m = m;
  a.r2 = r2;
  a.err = err;
  a.stack_smem = cfg.stack_smem;
  a.stats = cfg.stats_nodes;
  a.leafperm = cfg.leafperm;
  a.numbering = cfg.numbering;
  return a;
}

void launch_spatial_count(const float4 *rec, uint32_t n, const float *queries, const uint32_t *qperm, uint32_t m,
                          float r2, int32_t *counts, uint32_t *err, const TravCfg &cfg, cudaStream_t s, bool box) {
  if (m == 0) return;
  SpatialArgs a = spatial_args(rec, n, queries, qperm, m, r2, err, cfg);
  a.counts = counts;
  spatial_launch<kCount>(a, box, cfg.block, s, "spatial_count");
}

void launch_spatial_fill(const float4 *rec, uint32_t n, const float *queries, const uint32_t *qperm, uint32_t m,
                         float r2, const int64_t *offsets, int32_t *indices, int64_t capacity, uint32_t *err,
                         const TravCfg &cfg, cudaStream_t s, const uint32_t *m_dev, bool box) {
  if (m == 0) return;
  SpatialArgs a = spatial_args(rec, n, queries, qperm, m, r2, err, cfg);
  a.offsets = offsets;
  a.indices = indices;
  a.capacity = capacity;
  a.m_dev = m_dev;
  spatial_launch<kFill>(a, box, cfg.block, s, "spatial_fill");
}

void launch_spatial_buffered(const float4 *rec, uint32_t n, const float *queries, const uint32_t *qperm, uint32_t m,
                             float r2, int32_t *counts, int32_t *buf, int bs, uint32_t *ovf_list, uint32_t *ovf_count,
                             uint32_t *err, const TravCfg &cfg, cudaStream_t s, bool box) {
  if (m == 0) return;
  SpatialArgs a = spatial_args(rec, n, queries, qperm, m, r2, err, cfg);
  a.counts = counts;
  a.buf = buf;
  a.bs = bs;
  // 16-byte hit stores (cube 1e7, 1e6 queries: mean 10 hits with 32 slots 0.579 -> 0.577 ms, 20
  // with 40 0.875 -> 0.853, 40 with 72 1.266 -> 1.195, 80 with 136 2.141 -> 1.79; the lattice
  // r = 4 with 260 slots 6.54 -> 4.53 ms)
  a.buf_vec4 = bs % 4 == 0 && (reinterpret_cast<uintptr_t>(buf) & 15u) == 0;
  a.ovf_list = ovf_list;
  a.ovf_count = ovf_count;
  spatial_launch<kBuffered>(a, box, cfg.block, s, "spatial_buffered");
}

void launch_compact(const int32_t *buf, int bs, const int32_t *counts, const int64_t *offsets, uint32_t m,
                    int32_t *indices, int64_t capacity, uint32_t *err, cudaStream_t s) {
  const uint64_t slots = (uint64_t)m * bs;
  if (slots == 0) return;
  prof::Scope ps(s, "compact");
  if (bs % 4 == 0 && (reinterpret_cast<uintptr_t>(buf) & 15u) == 0) {
    const uint64_t groups = slots / 4;
    const uint64_t gblocks = (groups + 256 * kCompactPer - 1) / (256 * kCompactPer);
    const int4 *buf4 = reinterpret_cast<const int4 *>(buf);
    if (groups + 256 * kCompactPer < (1ull << 32))
      k_compact4<uint32_t><<<(unsigned)gblocks, 256, 0, s>>>(buf4, bs, counts, offsets, m, indices, capacity, err);
    else
      k_compact4<uint64_t><<<(unsigned)gblocks, 256, 0, s>>>(buf4, bs, counts, offsets, m, indices, capacity, err);
    return;
  }
  const uint64_t blocks = (slots + 256 * kCompactPer - 1) / (256 * kCompactPer);
  if (slots + 256 * kCompactPer < (1ull << 32))  // 32-bit slot arithmetic cannot wrap
    k_compact<uint32_t><<<(unsigned)blocks, 256, 0, s>>>(buf, bs, counts, offsets, m, indices, capacity, err);
  else
    k_compact<uint64_t><<<(unsigned)blocks, 256, 0, s>>>(buf, bs, counts, offsets, m, indices, capacity, err);
}

size_t scan_compact_ws_words(uint32_t m) { return (size_t)ceil_div<uint32_t>(m > 0 ? m : 1, (uint32_t)kScTile) + 2; }

void launch_scan_compact(const int32_t *counts, uint32_t m, const int32_t *buf, int bs, int64_t *offsets,
                         int32_t *indices, int64_t capacity, uint64_t *ws, uint32_t *err, cudaStream_t s) {
  if (m == 0) {
    cudaMemsetAsync(offsets, 0, sizeof(int64_t), s);
    return;
  }
  const uint32_t tiles = ceil_div<uint32_t>(m, (uint32_t)kScTile);
  uint32_t *ctr = reinterpret_cast<uint32_t *>(ws + tiles);
  prof::Scope ps(s, "scan_compact");
  if (bs % 4 == 0 && (reinterpret_cast<uintptr_t>(buf) & 15u) == 0)
    k_scan_compact<true><<<tiles, kScThreads, 0, s>>>(counts, m, buf, bs, offsets, indices, capacity, ws, ctr, err);
  else
    k_scan_compact<false><<<tiles, kScThreads, 0, s>>>(counts, m, buf, bs, offsets, indices, capacity, ws, ctr, err);
}

uint32_t scan_compact_probe_queries() { return 2 * kScTile; }

void launch_scan_compact_wait_probe(int32_t *counts, int64_t *offsets, uint64_t *ws, uint32_t *err, cudaStream_t s) {
  // two tiles of empty rows; the tile counter starts at 1, so the single block takes tile 1 and
  // looks back at tile 0, whose status word nobody publishes
  const uint32_t m = scan_compact_probe_queries();
  cudaMemsetAsync(counts, 0, (size_t)m * sizeof(int32_t), s);
  cudaMemsetAsync(ws, 0, scan_compact_ws_words(m) * sizeof(uint64_t), s);
  cudaMemsetAsync(reinterpret_cast<uint32_t *>(ws + 2), 1, 1, s);  // the tile counter (after the 2 status words): 1
  k_scan_compact<false><<<1, kScThreads, 0, s>>>(counts, m, counts, 1, offsets, nullptr, 0, ws,
                                                reinterpret_cast<uint32_t *>(ws + 2), err);
}

size_t scan_tmp_words(uint32_t m) { return (size_t)ceil_div<uint32_t>(m > 0 ? m : 1, (uint32_t)kScanTile) + 1; }

void launch_scan(const int32_t *counts, uint32_t m, int64_t *offsets, int64_t *tmp, cudaStream_t s) {
  if (m == 0) {
    cudaMemsetAsync(offsets, 0, sizeof(int64_t), s);
    return;
  }
  const uint32_t tiles = ceil_div<uint32_t>(m, (uint32_t)kScanTile);
  prof::Scope ps(s, "scan");
  k_scan_reduce<<<tiles, kScanThreads, 0, s>>>(counts, m, tmp);
  k_scan_tiles<<<1, 1024, 0, s>>>(tmp, tiles);
  k_scan_down<<<tiles, kScanThreads, 0, s>>>(counts, m, tmp, offsets);
}

template <int KC, bool NBR, int ANCHOR>
static void nearest_kc2(dim3 grid, int block, size_t smem, cudaStream_t s, const NearestArgs &a) {
  if (smem > 48 * 1024) {
    cudaFuncSetAttribute(k_nearest<KC, NBR, ANCHOR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(k_nearest<KC, NBR, ANCHOR>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  }
  k_nearest<KC, NBR, ANCHOR><<<grid, block, smem, s>>>(a);
}

// The first-descent form (3) serves register lists of 2 to 10; wider lists and the heap take the
// query-path walk (form 2) in its place, measured as fast or faster there (cube 1e7, 1e6 queries:
// k = 16 1.546 against 1.557 ms, the 64-Gaussian mixture 1.618 against 1.637 ms).
template <int KC>
constexpr bool kFirstDescent = KC >= 2 && KC <= 10;

template <int KC>
static void nearest_kc(dim3 grid, int block, size_t smem, cudaStream_t s, const NearestArgs &a) {
  prof::Scope ps(s, "nearest");
  if (a.nbr_bound) {
    nearest_kc2<KC, true, 0>(grid, block, smem, s, a);  // bounded by finished neighbours
  } else if (KC == 1 || a.anchor == 0) {
    nearest_kc2<KC, false, 0>(grid, block, smem, s, a);  // k = 1: its first leaf already sets the bound
  } else if (a.anchor == 1) {
    nearest_kc2<KC, false, 1>(grid, block, smem, s, a);
  } else {
    if constexpr (kFirstDescent<KC>) {
      if (a.anchor == 3) nearest_kc2<KC, false, 3>(grid, block, smem, s, a);
      else nearest_kc2<KC, false, 2>(grid, block, smem, s, a);
    } else {
      nearest_kc2<KC, false, 2>(grid, block, smem, s, a);
    }
  }
}

int launch_batch_nearest(const BatchQueryArgs &args, int kc, const TravCfg &cfg, cudaStream_t s) {
  if (args.pos_end <= args.pos_begin) return 0;
  BatchQueryArgs a = args;
  if (kc == 0) a.stack_smem = std::min(a.stack_smem, kHeapStackSmem);
  // the heap class runs 64-thread blocks at most (its shared heap limits the resident blocks)
  const int block = kc == 0 ? std::min(cfg.block, 64) : cfg.block;
  size_t smem = (size_t)2 * a.stack_smem * block * sizeof(int32_t);
  if (kc == 0) {
    smem += (size_t)2 * kBatchHeapK * block * sizeof(int32_t);
    if (smem > 227 * 1024) return -1;
    if (smem > 48 * 1024) {
      cudaFuncSetAttribute(k_batch_nearest<0, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      cudaFuncSetAttribute(k_batch_nearest<0, 0>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    }
  }
  int dev = 0, sms = 148, per_sm = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // one profiler name per query class, so that the report splits the batch's time by list width
  const char *name = kc == 0 ? "batch_nearest_heap" : kc == 1 ? "batch_nearest_k1" : kc == 2 ? "batch_nearest_k2"
                     : kc == 4 ? "batch_nearest_k4" : kc == 8 ? "batch_nearest_k8" : kc == 10 ? "batch_nearest_k10"
                     : kc == 16 ? "batch_nearest_k16" : "batch_nearest_k32";
  prof::Scope ps(s, name);
  const uint32_t need = ceil_div<uint32_t>(a.pos_end - a.pos_begin, (uint32_t)block);
  auto go = [&](auto kern) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, block, smem);
    const uint32_t grid = std::max<uint32_t>(1u, std::min<uint32_t>(need, (uint32_t)(sms * std::max(per_sm, 1))));
    kern<<<grid, block, smem, s>>>(a);
  };
  switch (kc) {
    case 0: go(k_batch_nearest<0, 0>); break;
    case 1: go(k_batch_nearest<1, 0>); break;
    case 2: a.anchor == 3 ? go(k_batch_nearest<2, 3>) : go(k_batch_nearest<2, 0>); break;
    case 4: a.anchor == 3 ? go(k_batch_nearest<4, 3>) : go(k_batch_nearest<4, 0>); break;
    case 8: a.anchor == 3 ? go(k_batch_nearest<8, 3>) : go(k_batch_nearest<8, 0>); break;
    case 10: a.anchor == 3 ? go(k_batch_nearest<10, 3>) : go(k_batch_nearest<10, 0>); break;
    case 16: go(k_batch_nearest<16, 0>); break;  // the first-descent form runs as the query-path walk here
    case 32: go(k_batch_nearest<32, 0>); break;
    default: return -1;
  }
  return 0;
}

int launch_nearest(NearestArgs a, const TravCfg &cfg, cudaStream_t s) {
  a.kk = (int)std::min<int64_t>(a.k, a.n);
  a.stats = cfg.stats_nodes;
  a.out_pairs = (reinterpret_cast<uintptr_t>(a.out_idx) & 7u) == 0 &&
                (a.out_d2 == nullptr || (reinterpret_cast<uintptr_t>(a.out_d2) & 7u) == 0);
  const int k = a.k;
  const uint32_t threads = a.m + 1;
  int block = cfg.block;
  // large k: candidates in a shared-memory heap (a 64-entry register list measured 2x slower at k = 50)
  const bool use_heap = k >= (cfg.heap_from > 0 ? cfg.heap_from : kHeapFrom);
  a.stack_smem = use_heap ? std::min(cfg.stack_smem, kHeapStackSmem) : cfg.stack_smem;
  size_t smem = (size_t)2 * a.stack_smem * block * sizeof(int32_t);
  if (use_heap) {
    // heap of k pairs per thread in shared memory: shrink the block to fit
    while (block > 32 && smem + (size_t)2 * k * block * sizeof(int32_t) > 200 * 1024) {
      block >>= 1;
      smem = (size_t)2 * a.stack_smem * block * sizeof(int32_t);
    }
    smem += (size_t)2 * k * block * sizeof(int32_t);
    if (smem > 227 * 1024) return -1;
  }
  const dim3 grid(ceil_div<uint32_t>(threads, (uint32_t)block));
  if (use_heap) nearest_kc<0>(grid, block, smem, s, a);
  else if (k <= 1) nearest_kc<1>(grid, block, smem, s, a);
  else if (k <= 2) nearest_kc<2>(grid, block, smem, s, a);
  else if (k <= 4) nearest_kc<4>(grid, block, smem, s, a);
  else if (k <= 8) nearest_kc<8>(grid, block, smem, s, a);
  else if (k <= 10) nearest_kc<10>(grid, block, smem, s, a);
  else if (k <= 16) nearest_kc<16>(grid, block, smem, s, a);
  else nearest_kc<32>(grid, block, smem, s, a);  // k <= 32 < heap_from
  return 0;
}

}  // namespace abx

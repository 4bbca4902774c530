// LBVH construction kernels (ArborX Sec. 2.1): scene box, Morton codes with
// fused radix histograms, binary radix-tree hierarchy, bottom-up box fit.
#include <algorithm>

#include "kernels.cuh"
#include "prof.cuh"
#include "radix_sort.cuh"

namespace abx {

namespace {

__device__ __forceinline__ void acc_axis(float v, float &mn, float &mx, uint32_t &bad) {
  const bool ok = is_finite_bits(v);
  bad += ok ? 0u : 1u;
  mn = fminf(mn, ok ? v : __int_as_float(0x7f800000));
  mx = fmaxf(mx, ok ? v : __int_as_float(0xff800000));
}

// Scene box: per-axis min / max over every coordinate of every box corner.
// The coordinate array is nf floats, coordinate i belonging to axis i % 3 for
// both points (3 per row) and boxes (6 per row).
__global__ void __launch_bounds__(256) k_bounds(const float *__restrict__ f, uint64_t nf, bool vec,
                                                  DevMeta *__restrict__ meta) {
  float mn[3], mx[3];
  uint32_t bad = 0;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    mn[a] = __int_as_float(0x7f800000);
    mx[a] = __int_as_float(0xff800000);
  }
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t groups = vec ? nf / 12 : 0;  // 12 floats = 3 float4 = axes x y z x | y z x y | z x y z
  const float4 *f4 = reinterpret_cast<const float4 *>(f);
  for (uint64_t g = tid; g < groups; g += stride) {
    const float4 a = __ldg(f4 + 3 * g), b = __ldg(f4 + 3 * g + 1), c = __ldg(f4 + 3 * g + 2);
    acc_axis(a.x, mn[0], mx[0], bad); acc_axis(a.y, mn[1], mx[1], bad); acc_axis(a.z, mn[2], mx[2], bad);
    acc_axis(a.w, mn[0], mx[0], bad); acc_axis(b.x, mn[1], mx[1], bad); acc_axis(b.y, mn[2], mx[2], bad);
    acc_axis(b.z, mn[0], mx[0], bad); acc_axis(b.w, mn[1], mx[1], bad); acc_axis(c.x, mn[2], mx[2], bad);
    acc_axis(c.y, mn[0], mx[0], bad); acc_axis(c.z, mn[1], mx[1], bad); acc_axis(c.w, mn[2], mx[2], bad);
  }
  for (uint64_t i = groups * 12 + tid; i < nf; i += stride) {
    const int a = (int)(i % 3);
    acc_axis(f[i], mn[a], mx[a], bad);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      mn[a] = fminf(mn[a], __shfl_xor_sync(0xffffffffu, mn[a], o));
      mx[a] = fmaxf(mx[a], __shfl_xor_sync(0xffffffffu, mx[a], o));
    }
    bad += __shfl_xor_sync(0xffffffffu, bad, o);
  }
  __shared__ float s_v[8][6];
  __shared__ uint32_t s_bad[8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      s_v[warp][a] = mn[a];
      s_v[warp][3 + a] = mx[a];
    }
    s_bad[warp] = bad;
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    const int a = threadIdx.x;
    float v = s_v[0][a];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) v = a < 3 ? fminf(v, s_v[w][a]) : fmaxf(v, s_v[w][a]);
    if (a < 3) atomicMin(&meta->bounds_ord[a], f2ord(v));
    else atomicMax(&meta->bounds_ord[a], f2ord(v));
  } else if (threadIdx.x == 32) {
    uint32_t b = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b += s_bad[w];
    if (b) {
      atomicAdd(&meta->nonfinite, b);
      atomicOr(&meta->err, ERR_NONFINITE);
    }
  }
}

__global__ void k_init_meta(DevMeta *meta) {
  const int t = threadIdx.x;
  if (t < 3) meta->bounds_ord[t] = 0xffffffffu;
  else if (t < 6) meta->bounds_ord[t] = 0u;
  else if (t == 6) meta->nonfinite = 0;
  else if (t == 7) meta->err = 0;
  else if (t >= 8 && t < 11) meta->scene[t - 8] = __int_as_float(0x7f800000);   // empty box: +inf
  else if (t >= 11 && t < 14) meta->scene[t - 8] = __int_as_float(0xff800000);  // -inf
  else if (t >= 14 && t < 16) meta->nodes[t - 14] = 0ull;
  else if (t >= 16 && t < 18) meta->queries[t - 16] = 0ull;
}

// k_init_meta over block 0 and, over the whole grid, zero `words` 16-byte words at `zero` (the
// build's counters and sort workspace), in one launch
__global__ void __launch_bounds__(256) k_init_meta_zero(DevMeta *meta, uint4 *__restrict__ zero, uint64_t words) {
  if (blockIdx.x == 0 && threadIdx.x < 32) {
    const int t = threadIdx.x;
    if (t < 3) meta->bounds_ord[t] = 0xffffffffu;
    else if (t < 6) meta->bounds_ord[t] = 0u;
    else if (t == 6) meta->nonfinite = 0;
    else if (t == 7) meta->err = 0;
    else if (t >= 8 && t < 11) meta->scene[t - 8] = __int_as_float(0x7f800000);
    else if (t >= 11 && t < 14) meta->scene[t - 8] = __int_as_float(0xff800000);
    else if (t >= 14 && t < 16) meta->nodes[t - 14] = 0ull;
    else if (t >= 16 && t < 18) meta->queries[t - 16] = 0ull;
  }
  const uint4 z = make_uint4(0u, 0u, 0u, 0u);
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < words; i += (uint64_t)gridDim.x * blockDim.x)
    zero[i] = z;
}

// ------------------------------------------------------------ Morton codes

template <int BITS>
__device__ __forceinline__ uint32_t quantise(float c, float L, float H) {
  const float ext = __fsub_rn(H, L);
  float u = 0.0f;
  if (ext > 0.0f) u = __fdiv_rn(__fsub_rn(c, L), ext);
  if (!(u >= 0.0f)) u = 0.0f;  // also NaN
  if (u > 1.0f) u = 1.0f;
  const uint32_t q = (uint32_t)floorf(__fmul_rn(u, (float)(1u << BITS)));
  return min(q, (1u << BITS) - 1u);
}

__device__ __forceinline__ uint32_t spread10(uint32_t x) {
  x &= 0x3ffu;
  x = (x | (x << 16)) & 0x030000FFu;
  x = (x | (x << 8)) & 0x0300F00Fu;
  x = (x | (x << 4)) & 0x030C30C3u;
  x = (x | (x << 2)) & 0x09249249u;
  return x;
}

__device__ __forceinline__ uint64_t spread21(uint64_t x) {
  x &= 0x1fffffull;
  x = (x | (x << 32)) & 0x1f00000000ffffull;
  x = (x | (x << 16)) & 0x1f0000ff0000ffull;
  x = (x | (x << 8)) & 0x100f00f00f00f00full;
  x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
  x = (x | (x << 2)) & 0x1249249249249249ull;
  return x;
}

template <typename K>
__device__ __forceinline__ K morton(float cx, float cy, float cz, const float *sc);

template <>
__device__ __forceinline__ uint32_t morton<uint32_t>(float cx, float cy, float cz, const float *sc) {
  return (spread10(quantise<10>(cx, sc[0], sc[3])) << 2) | (spread10(quantise<10>(cy, sc[1], sc[4])) << 1) |
         spread10(quantise<10>(cz, sc[2], sc[5]));
}
template <>
__device__ __forceinline__ uint64_t morton<uint64_t>(float cx, float cy, float cz, const float *sc) {
  return (spread21(quantise<21>(cx, sc[0], sc[3])) << 2) | (spread21(quantise<21>(cy, sc[1], sc[4])) << 1) |
         spread21(quantise<21>(cz, sc[2], sc[5]));
}

// 10-bit quantisation without the division in the common case.  rs = fl(2^10 * fl(1 / ext)) for a
// normal extent ext well inside the float range (NaN otherwise, which sends every call to the
// exact form).  Then f = fl(x * rs) = 2^10 * fl(x * fl(1 / ext)), and against the exact
// u = fl(x / ext) two roundings of relative size 2^-24 each separate them from x / ext on one side
// and one on the other: |f - 2^10 u| <= 2^10 (x / ext) 1.5 * 2^-23 <= 1.9e-4 for f <= 2^10.  When
// f lies at least kQuantEps (2^-11, 2.6 times that bound) inside an open cell (c, c + 1) with
// 0 <= c <= 1023, 2^10 u lies in the same cell, u is inside (0, 1) so neither clamp applies, and
// floor(2^10 u) = c: the exact result.  Anything else (a cell edge within the margin, outside
// the box, a flat axis, NaN) takes quantise<10>.
constexpr float kQuantEps = 0x1p-11f;

__device__ __forceinline__ float quant_scale10(float L, float H) {
  const float ext = __fsub_rn(H, L);
  return (ext >= 0x1p-116f && ext <= 0x1p116f) ? __fmul_rn(__frcp_rn(ext), 1024.0f) : __int_as_float(0x7fffffff);
}

__device__ __forceinline__ uint32_t quantise10_fast(float c, float L, float H, float rs) {
  const float f = __fmul_rn(__fsub_rn(c, L), rs);
  const float cell = floorf(f);
  const float fr = __fsub_rn(f, cell);
  if (fr >= kQuantEps && fr <= 1.0f - kQuantEps && cell >= 0.0f && cell <= 1023.0f) return (uint32_t)cell;
  return quantise<10>(c, L, H);
}

__device__ __forceinline__ uint32_t morton_fast10(float cx, float cy, float cz, const float *sc, const float *rs) {
  return (spread10(quantise10_fast(cx, sc[0], sc[3], rs[0])) << 2) |
         (spread10(quantise10_fast(cy, sc[1], sc[4], rs[1])) << 1) | spread10(quantise10_fast(cz, sc[2], sc[5], rs[2]));
}

// 30-bit codes take the division-free form; 63-bit codes (21 bits per axis, where the margin
// would exceed the cell) the exact one
template <typename K>
__device__ __forceinline__ K morton_block(float cx, float cy, float cz, const float *sc, const float *rs) {
  if constexpr (sizeof(K) == 4) return morton_fast10(cx, cy, cz, sc, rs);
  else return morton<K>(cx, cy, cz, sc);
}

template <typename K>
__device__ __forceinline__ void hist_add(uint32_t (*s_h)[kRadix], int passes, K code) {
  for (int p = 0; p < passes; ++p) atomicAdd(&s_h[p][(uint32_t)(code >> (p * kRadixBits)) & (kRadix - 1)], 1u);
}

// Morton code of each primitive's centroid (points: the point; boxes: the box
// centre), scaled by the scene box in `meta`, without its `drop` lowest bits;
// histograms of every radix pass.
template <typename K, int KIND>
__global__ void __launch_bounds__(256) k_morton(const float *__restrict__ prims, uint32_t n, bool vec,
                                               DevMeta *__restrict__ meta, K *__restrict__ codes,
                                               uint32_t *__restrict__ hist, int passes, bool write_scene,
                                               int drop) {
  __shared__ uint32_t s_h[8][kRadix];
  __shared__ float s_sc[6];
  for (int i = threadIdx.x; i < passes * kRadix; i += blockDim.x) (&s_h[0][0])[i] = 0;
  if (threadIdx.x < 6) s_sc[threadIdx.x] = ord2f(meta->bounds_ord[threadIdx.x]);
  __syncthreads();
  if (write_scene && blockIdx.x == 0 && threadIdx.x < 6) meta->scene[threadIdx.x] = s_sc[threadIdx.x];
  float sc[6], rs[3];
#pragma unroll
  for (int a = 0; a < 6; ++a) sc[a] = s_sc[a];
#pragma unroll
  for (int a = 0; a < 3; ++a) rs[a] = quant_scale10(sc[a], sc[3 + a]);

  constexpr int PER = KIND == 0 ? 3 : 6;  // floats per primitive
  constexpr int GP = 12 / PER;            // primitives per 3-float4 group
  const uint32_t stride = gridDim.x * blockDim.x;
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t groups = vec ? n / GP : 0;
  const float4 *f4 = reinterpret_cast<const float4 *>(prims);
  for (uint32_t g = tid; g < groups; g += stride) {
    const float4 a = __ldg(f4 + 3 * (uint64_t)g), b = __ldg(f4 + 3 * (uint64_t)g + 1),
                 c = __ldg(f4 + 3 * (uint64_t)g + 2);
    const float v[12] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, c.x, c.y, c.z, c.w};
    K out[GP];
#pragma unroll
    for (int j = 0; j < GP; ++j) {
      float cx, cy, cz;
      if (KIND == 0) {
        cx = v[3 * j]; cy = v[3 * j + 1]; cz = v[3 * j + 2];
      } else {
        cx = __fmul_rn(__fadd_rn(v[6 * j], v[6 * j + 3]), 0.5f);
        cy = __fmul_rn(__fadd_rn(v[6 * j + 1], v[6 * j + 4]), 0.5f);
        cz = __fmul_rn(__fadd_rn(v[6 * j + 2], v[6 * j + 5]), 0.5f);
      }
      out[j] = morton_block<K>(cx, cy, cz, sc, rs) >> drop;
      hist_add<K>(s_h, passes, out[j]);
    }
#pragma unroll
    for (int j = 0; j < GP; ++j) codes[(uint64_t)g * GP + j] = out[j];
  }
  for (uint32_t i = groups * GP + tid; i < n; i += stride) {
    const float *p = prims + (uint64_t)i * PER;
    float cx, cy, cz;
    if (KIND == 0) {
      cx = p[0]; cy = p[1]; cz = p[2];
    } else {
      cx = __fmul_rn(__fadd_rn(p[0], p[3]), 0.5f);
      cy = __fmul_rn(__fadd_rn(p[1], p[4]), 0.5f);
      cz = __fmul_rn(__fadd_rn(p[2], p[5]), 0.5f);
    }
    const K code = morton_block<K>(cx, cy, cz, sc, rs) >> drop;
    codes[i] = code;
    hist_add<K>(s_h, passes, code);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < passes * kRadix; i += blockDim.x) {
    const uint32_t c = (&s_h[0][0])[i];
    if (c) atomicAdd(&hist[i], c);
  }
}

// ------------------------------------------------------------ hierarchy

template <typename K>
__device__ __forceinline__ int clz_key(K x);
template <>
__device__ __forceinline__ int clz_key<uint32_t>(uint32_t x) { return __clz(x); }
template <>
__device__ __forceinline__ int clz_key<uint64_t>(uint64_t x) { return __clzll(x); }

// Length of the common prefix of the index-augmented keys (code_i, i) and
// (code_j, j); -1 outside [0, n).
template <typename K>
__device__ __forceinline__ int delta(const K *__restrict__ codes, K ci, int i, int j, int n) {
  if (j < 0 || j >= n) return -1;
  const K cj = codes[j];
  if (cj != ci) return clz_key<K>(ci ^ cj);
  return (int)(8 * sizeof(K)) + __clz((uint32_t)(i ^ j));
}

// Internal node i (of n - 1) finds the range of sorted leaves it covers and the
// split inside it where the highest differing bit of the augmented keys flips
// (binary radix tree, Karras 2012); records parent links (p << 1 | side) of its
// two children.  Node ids: internal 0 .. n-2 (root 0), leaf t is n - 1 + t.
template <typename K>
__global__ void __launch_bounds__(256) k_hierarchy(const K *__restrict__ codes, uint32_t n,
                                                  int32_t *__restrict__ parent) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int N = (int)n;
  if (i >= N - 1) return;
  const K ci = codes[i];
  const int dl = delta<K>(codes, ci, i, i - 1, N);
  const int dr = delta<K>(codes, ci, i, i + 1, N);
  const int d = dr > dl ? 1 : -1;
  const int dmin = min(dl, dr);
  int lmax = 2;
  while (delta<K>(codes, ci, i, i + lmax * d, N) > dmin) lmax <<= 1;
  int l = 0;
  for (int t = lmax >> 1; t >= 1; t >>= 1)
    if (delta<K>(codes, ci, i, i + (l + t) * d, N) > dmin) l += t;
  const int j = i + l * d;
  const int dnode = delta<K>(codes, ci, i, j, N);
  int s = 0, t = l;
  do {
    t = (t + 1) >> 1;
    if (delta<K>(codes, ci, i, i + (s + t) * d, N) > dnode) s += t;
  } while (t > 1);
  const int gamma = i + s * d + min(d, 0);
  const int left = (min(i, j) == gamma) ? (N - 1 + gamma) : gamma;
  const int right = (max(i, j) == gamma + 1) ? (N - 1 + gamma + 1) : gamma + 1;
  parent[left] = (i << 1);
  parent[right] = (i << 1) | 1;
}

// Bottom-up fit: one thread per sorted leaf writes its primitive's box into its
// parent's child slot, then climbs; at each internal node the first arriving
// thread stops and the second merges both child boxes and continues.
template <int KIND>
__global__ void __launch_bounds__(256) k_fit(const float *__restrict__ prims, uint32_t n,
                                            const uint32_t *__restrict__ perm, const int32_t *__restrict__ parent,
                                            uint32_t *__restrict__ arrival, float4 *__restrict__ rec,
                                            uint32_t *__restrict__ err) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const uint32_t prim = perm[t];
  float lx, ly, lz, hx, hy, hz;
  if (KIND == 0) {
    const float *p = prims + 3 * (uint64_t)prim;
    lx = hx = p[0]; ly = hy = p[1]; lz = hz = p[2];
  } else {
    const float *p = prims + 6 * (uint64_t)prim;
    lx = p[0]; ly = p[1]; lz = p[2]; hx = p[3]; hy = p[4]; hz = p[5];
  }
  int enc = ~(int)prim;
  int cnt = 1;  // leaves under the current node (the record's aux word)
  if (n == 1) {
    rec[0] = make_float4(lx, ly, lz, __int_as_float(enc));
    rec[1] = make_float4(hx, hy, hz, __int_as_float(1));
    return;
  }
  int c = (int)n - 1 + (int)t;
  for (int level = 0;; ++level) {
    const int pp = __ldg(parent + c);
    const int p = pp >> 1, side = pp & 1;
    if (pp < 0 || p >= (int)n - 1 || level > 128) {  // broken hierarchy: report, never write outside
      set_err(err, ERR_STACK);
      return;
    }
    float4 *slot = rec + 4 + 4 * (uint64_t)p + 2 * side;
    slot[0] = make_float4(lx, ly, lz, __int_as_float(enc));
    slot[1] = make_float4(hx, hy, hz, __int_as_float(cnt));
    if (atom_add_acq_rel_gpu(arrival + p, 1u) == 0u) return;  // sibling not done yet
    const float4 *sib = rec + 4 + 4 * (uint64_t)p + 2 * (1 - side);
    const float4 slo = ld_cg_f4(sib), shi = ld_cg_f4(sib + 1);
    lx = fminf(lx, slo.x); ly = fminf(ly, slo.y); lz = fminf(lz, slo.z);
    hx = fmaxf(hx, shi.x); hy = fmaxf(hy, shi.y); hz = fmaxf(hz, shi.z);
    cnt += __float_as_int(shi.w);
    enc = p;
    c = p;
    if (p == 0) {
      rec[0] = make_float4(lx, ly, lz, __int_as_float(0));
      rec[1] = make_float4(hx, hy, hz, __int_as_float(cnt));
      return;
    }
  }
}

// Single bottom-up pass (Apetrei 2014): hierarchy and boxes together.  Internal
// node p is the node whose split lies between sorted leaves p and p + 1.  A
// climb starts at leaf t with range [t, t]: the parent of a node covering
// [l, r] splits at r (node is its left child) when the augmented keys share a
// longer prefix across r | r+1 than across l-1 | l, else at l - 1 (node is its
// right child).  Each child writes its box record into the parent's slot and
// exchanges its outer range end; the first arriver stops, the second learns
// the parent's full range, merges the two boxes and continues.  Same binary
// radix tree as the top-down split rule.
//
// Two kernels.  k_apetrei_local: block b owns the sorted leaves [c0, c0 + C)
// and the inner splits c0 .. c0 + C - 2.  With d_i the common-prefix length of
// the augmented keys at i | i+1, the node split at p covers [l, r] where l - 1
// and r are the nearest positions on either side with d < d_p (the binary
// radix tree is the Cartesian tree of d); its box is the union of the leaf
// boxes l..r; its parent splits at r if d_r > d_(l-1), else at l - 1 (the
// same rule the climb uses).  The block finds these nearest smaller values in
// a shared-memory minimum table of d and the unions in shared-memory prefix /
// suffix / segment tables, one leaf and one split per thread, with no climb,
// atomic or fence.  A split whose nearest smaller value lies outside the chunk
// on some side is a crossing node: it records in other[p] the outer end of
// its local child if it has one (a completed first arrival), else -1.  A node
// or leaf whose parent is a boundary split (c0 - 1 or c0 + C - 1) goes to the
// block's frontier list (at most one per side).  k_apetrei_top then climbs
// from every frontier node with the GPU-scope exchange on other[]; crossing
// nodes are few (about ten per chunk).  Each node sees exactly two arrivals.

// one 32-byte record (lo, hi) in a single 256-bit store; records are 32-byte aligned
__device__ __forceinline__ void st_rec(float4 *p, const float4 lo, const float4 hi) {
  asm volatile("st.global.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "f"(lo.x), "f"(lo.y), "f"(lo.z),
               "f"(lo.w), "f"(hi.x), "f"(hi.y), "f"(hi.z), "f"(hi.w)
               : "memory");
}

struct Frontier {
  float4 lo;  // w: enc
  float4 hi;
  int32_t l, r, pad0, pad1;  // l < 0: empty
};

template <typename K>
__device__ __forceinline__ void apetrei_climb_global(const K *__restrict__ codes, int N, int32_t *__restrict__ other,
                                                     float4 *__restrict__ rec, uint32_t *__restrict__ err, int l,
                                                     int r, float4 lo, float4 hi) {
  for (int level = 0;; ++level) {
    bool left_child;
    if (l == 0) {
      left_child = true;
    } else if (r == N - 1) {
      left_child = false;
    } else {
      const K cl = __ldg(codes + l), cr = __ldg(codes + r);
      left_child = delta<K>(codes, cr, r, r + 1, N) > delta<K>(codes, cl, l, l - 1, N);
    }
    const int p = left_child ? r : l - 1;
    if (p < 0 || p >= N - 1 || level > 128) {  // cannot happen for sorted keys; never write outside
      set_err(err, ERR_STACK);
      return;
    }
    float4 *slot = rec + 4 + 4 * (uint64_t)p + (left_child ? 0 : 2);
    st_rec(slot, lo, hi);
    const int got = atom_exch_acq_rel_gpu(other + p, left_child ? l : r);
    if (got < 0) return;  // sibling not done yet
    if (left_child) r = got;
    else l = got;
    const float4 *sib = rec + 4 + 4 * (uint64_t)p + (left_child ? 2 : 0);
    const float4 slo = ld_cg_f4(sib), shi = ld_cg_f4(sib + 1);
    lo = make_float4(fminf(lo.x, slo.x), fminf(lo.y, slo.y), fminf(lo.z, slo.z), __int_as_float(p));
    hi = make_float4(fmaxf(hi.x, shi.x), fmaxf(hi.y, shi.y), fmaxf(hi.z, shi.z), __int_as_float(r - l + 1));
    if (l == 0 && r == N - 1) {
      rec[0] = lo;
      rec[1] = hi;
      return;
    }
  }
}

constexpr int kApBlock = 256;
constexpr int kApChunk = kApBlock;  // sorted leaves (and threads) per block of k_apetrei_local
constexpr int kApLevels = 9;        // minimum table levels: 2^8 <= kApChunk + 1 entries
constexpr int kApSeg = 16;          // leaves per union segment
constexpr int kApSegs = kApChunk / kApSeg;
constexpr int kApSegLevels = 5;     // 2^4 = kApSegs

__device__ __forceinline__ void box_union(float4 &lo, float4 &hi, const float4 a, const float4 b) {
  lo.x = fminf(lo.x, a.x); lo.y = fminf(lo.y, a.y); lo.z = fminf(lo.z, a.z);
  hi.x = fmaxf(hi.x, b.x); hi.y = fmaxf(hi.y, b.y); hi.z = fmaxf(hi.z, b.z);
}

template <typename K, int KIND>
__global__ void __launch_bounds__(kApBlock) k_apetrei_local(const float *__restrict__ prims, uint32_t n,
                                                           const K *__restrict__ codes,
                                                           const uint32_t *__restrict__ perm,
                                                           int32_t *__restrict__ other, float4 *__restrict__ rec,
                                                           Frontier *__restrict__ front, uint32_t *__restrict__ err) {
  constexpr int C = kApChunk;
  __shared__ int32_t s_dmin[kApLevels][C + 1];         // [j][x]: min d over positions c0-1+x .. +2^j-1
  __shared__ float4 s_leaf[2][C];                      // leaf boxes (lo, hi)
  __shared__ float4 s_pre[2][C], s_suf[2][C];          // unions from segment start to t / t to segment end
  __shared__ float4 s_seg[kApSegLevels][2][kApSegs];   // [j][.][s]: union of segments s .. s + 2^j - 1
  __shared__ Frontier s_front[2];                      // children of the boundary splits c0 - 1, c0 + C - 1
  const int N = (int)n;
  const int c0 = (int)blockIdx.x * C;
  const int cend = min(c0 + C, N) - 1;  // last leaf of the chunk
  const int last = cend - c0 + 1;       // largest valid index into s_dmin[0]
  const int tid = (int)threadIdx.x;
  if (N == 1) {
    if (tid == 0) {
      const uint32_t prim = perm[0];
      const float *q = prims + (KIND == 0 ? 3 : 6) * (uint64_t)prim;
      rec[0] = make_float4(q[0], q[1], q[2], __int_as_float(~(int)prim));
      rec[1] = KIND == 0 ? make_float4(q[0], q[1], q[2], __int_as_float(1))
                         : make_float4(q[3], q[4], q[5], __int_as_float(1));
      front[0].l = front[1].l = -1;
    }
    return;
  }
  // the leaf gather is issued first; the d values, which need only the codes, are computed
  // while it is in flight
  const int t = c0 + tid;  // this thread's leaf, and split t (between t and t + 1)
  const bool has_leaf = t <= cend;
  uint32_t prim = 0;
  float4 lo = make_float4(0.f, 0.f, 0.f, 0.f), hi = lo;
  if (has_leaf) {
    prim = perm[t];
    if (KIND == 0) {
      const float *q = prims + 3 * (uint64_t)prim;
      lo = make_float4(q[0], q[1], q[2], 0.0f);
      hi = lo;
    } else {
      const float *q = prims + 6 * (uint64_t)prim;
      lo = make_float4(q[0], q[1], q[2], 0.0f);
      hi = make_float4(q[3], q[4], q[5], 0.0f);
    }
  }
  if (tid < 2) s_front[tid].l = -1;  // read after the barrier below
  // d at positions c0 - 1 + x (-1 outside [0, N - 2]), straight from the codes in global memory
  // (each code is read by two neighbouring threads, the second time from L1), so no barrier
  // stands between the code loads and the table
  auto dl = [&](int pos) -> int {
    if (pos < 0 || pos >= N - 1) return -1;
    const K ci = __ldg(codes + pos), cj = __ldg(codes + pos + 1);
    if (ci != cj) return clz_key<K>(ci ^ cj);
    return (int)(8 * sizeof(K)) + __clz((uint32_t)(pos ^ (pos + 1)));
  };
  for (int x = tid; x <= last; x += kApBlock) s_dmin[0][x] = dl(c0 - 1 + x);
  // unions within 16-leaf segments (lanes of one half-warp), before and after each leaf
  {
    float4 plo = lo, phi = hi, slo = lo, shi = hi;
    const int sl = tid & (kApSeg - 1);
    const int valid_to = has_leaf ? kApSeg - 1 : -1;  // beyond the last leaf: contribute nothing
    const int seg_last = min(kApSeg - 1, cend - (c0 + (tid & ~(kApSeg - 1))));
#pragma unroll
    for (int o = 1; o < kApSeg; o <<= 1) {
      float4 a, b;
      a.x = __shfl_up_sync(0xffffffffu, plo.x, o, kApSeg); a.y = __shfl_up_sync(0xffffffffu, plo.y, o, kApSeg);
      a.z = __shfl_up_sync(0xffffffffu, plo.z, o, kApSeg); b.x = __shfl_up_sync(0xffffffffu, phi.x, o, kApSeg);
      b.y = __shfl_up_sync(0xffffffffu, phi.y, o, kApSeg); b.z = __shfl_up_sync(0xffffffffu, phi.z, o, kApSeg);
      if (sl >= o) box_union(plo, phi, a, b);
      a.x = __shfl_down_sync(0xffffffffu, slo.x, o, kApSeg); a.y = __shfl_down_sync(0xffffffffu, slo.y, o, kApSeg);
      a.z = __shfl_down_sync(0xffffffffu, slo.z, o, kApSeg); b.x = __shfl_down_sync(0xffffffffu, shi.x, o, kApSeg);
      b.y = __shfl_down_sync(0xffffffffu, shi.y, o, kApSeg); b.z = __shfl_down_sync(0xffffffffu, shi.z, o, kApSeg);
      if (sl + o <= seg_last) box_union(slo, shi, a, b);
    }
    (void)valid_to;
    s_leaf[0][tid] = lo;
    s_leaf[1][tid] = hi;
    s_pre[0][tid] = plo;
    s_pre[1][tid] = phi;
    s_suf[0][tid] = slo;
    s_suf[1][tid] = shi;
    if (sl == 0) {
      s_seg[0][0][tid / kApSeg] = slo;
      s_seg[0][1][tid / kApSeg] = shi;
    }
  }
  __syncthreads();
#pragma unroll 1
  // two table levels per barrier: levels j and j + 1 both from level j - 1 (the same loads as one
  // level at a time, half the barriers)
  static_assert(kApLevels % 2 == 1 && kApSegLevels % 2 == 1, "levels are built in pairs");
  for (int j = 1; j < kApLevels; j += 2) {
    const int h = 1 << (j - 1);
    if (tid + 2 * h - 1 <= last) {
      const int m01 = min(s_dmin[j - 1][tid], s_dmin[j - 1][tid + h]);
      s_dmin[j][tid] = m01;
      if (tid + 4 * h - 1 <= last) s_dmin[j + 1][tid] = min(m01, min(s_dmin[j - 1][tid + 2 * h], s_dmin[j - 1][tid + 3 * h]));
    }
    if (j < kApSegLevels && tid + 2 * h <= kApSegs) {
      float4 a = s_seg[j - 1][0][tid], b = s_seg[j - 1][1][tid];
      box_union(a, b, s_seg[j - 1][0][tid + h], s_seg[j - 1][1][tid + h]);
      s_seg[j][0][tid] = a;
      s_seg[j][1][tid] = b;
      if (tid + 4 * h <= kApSegs) {
        box_union(a, b, s_seg[j - 1][0][tid + 2 * h], s_seg[j - 1][1][tid + 2 * h]);
        box_union(a, b, s_seg[j - 1][0][tid + 3 * h], s_seg[j - 1][1][tid + 3 * h]);
        s_seg[j + 1][0][tid] = a;
        s_seg[j + 1][1][tid] = b;
      }
    }
    __syncthreads();
  }
  auto D = [&](int pos) -> int { return s_dmin[0][pos - c0 + 1]; };
  // write node [l, r] (box lo/hi, enc in lo.w) into its parent's slot, or as the root
  auto emit = [&](int l, int r, float4 blo, float4 bhi) {
    if (l == 0 && r == N - 1) {
      st_rec(rec, blo, bhi);
      return;
    }
    const bool left_child = D(r) > D(l - 1);
    const int p = left_child ? r : l - 1;
    float4 *slot = rec + 4 + 4 * (uint64_t)p + (left_child ? 0 : 2);
    st_rec(slot, blo, bhi);
    if (p < c0 || p >= cend) {  // boundary split: continued by the top kernel
      Frontier &f = s_front[p < c0 ? 0 : 1];
      f.lo = blo;
      f.hi = bhi;
      f.r = r;
      f.l = l;
    }
  };
  if (has_leaf) {
    lo.w = __int_as_float(~(int)prim);
    hi.w = __int_as_float(1);
    emit(t, t, lo, hi);
  }
  if (t < cend) {
    const int xp = tid + 1;  // index of d_t
    const int dp = s_dmin[0][xp];
    int y = xp;  // smallest y with d >= dp on [y, xp - 1]
#pragma unroll
    for (int j = kApLevels - 1; j >= 0; --j)
      if (y >= (1 << j) && s_dmin[j][y - (1 << j)] >= dp) y -= 1 << j;
    const bool found_l = y > 0;
    const int l = c0 - 1 + y;  // valid when found_l
    int z = xp + 1;  // largest z - 1 with d >= dp on [xp + 1, z - 1]
#pragma unroll
    for (int j = kApLevels - 1; j >= 0; --j)
      if (z + (1 << j) - 1 <= last && s_dmin[j][z] >= dp) z += 1 << j;
    const bool found_r = z <= last;
    const int r = c0 - 1 + z;  // valid when found_r
    if (found_l && found_r) {
      const int a = l - c0, b = r - c0;
      const int sa = a / kApSeg, sb = b / kApSeg;
      float4 blo, bhi;
      if (sa == sb) {
        blo = s_leaf[0][a];
        bhi = s_leaf[1][a];
        for (int i = a + 1; i <= b; ++i) box_union(blo, bhi, s_leaf[0][i], s_leaf[1][i]);
      } else {
        blo = s_suf[0][a];
        bhi = s_suf[1][a];
        box_union(blo, bhi, s_pre[0][b], s_pre[1][b]);
        if (sb - sa >= 2) {
          const int s0 = sa + 1, s1 = sb - 1;
          const int j = 31 - __clz(s1 - s0 + 1);
          box_union(blo, bhi, s_seg[j][0][s0], s_seg[j][1][s0]);
          box_union(blo, bhi, s_seg[j][0][s1 - (1 << j) + 1], s_seg[j][1][s1 - (1 << j) + 1]);
        }
      }
      blo.w = __int_as_float(t);
      bhi.w = __int_as_float(r - l + 1);  // leaves under the node
      emit(l, r, blo, bhi);
    } else {
      other[t] = found_l ? l : (found_r ? r : -1);  // local child's outer end: a completed first arrival
    }
  }
  __syncthreads();
  if (tid == 0 && c0 > 0) other[c0 - 1] = -1;
  if (tid < 2) front[2 * blockIdx.x + tid] = s_front[tid];
  (void)err;
}

// One thread per frontier entry: continue the climb with the GPU-scope protocol.
template <typename K>
__global__ void __launch_bounds__(256) k_apetrei_top(const K *__restrict__ codes, uint32_t n,
                                                    int32_t *__restrict__ other, float4 *__restrict__ rec,
                                                    const Frontier *__restrict__ front, uint32_t n_front,
                                                    uint32_t *__restrict__ err) {
  const uint32_t f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= n_front) return;
  const Frontier e = front[f];
  if (e.l < 0) return;
  apetrei_climb_global<K>(codes, (int)n, other, rec, err, e.l, e.r, e.lo, e.hi);
}

// Identity order when a sort of the order's keys gave up its bounded wait (ERR_TIMEOUT in *err):
// every permutation is a correct traversal order, the identity included.
__global__ void k_iota_on_timeout(uint32_t *__restrict__ out, uint32_t m, const uint32_t *__restrict__ err) {
  if (!(*err & ERR_TIMEOUT)) return;
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) out[i] = i;
}

// ------------------------------------------------------ batched clouds
// Cloud c of a batch owns points [off[c], off[c+1]) of the concatenation.

__device__ __forceinline__ uint32_t cloud_of(const uint32_t *__restrict__ off, uint32_t n_clouds, uint32_t i) {
  uint32_t lo = 0, hi = n_clouds;  // largest c with off[c] <= i
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (__ldg(off + mid) <= i) lo = mid;
    else hi = mid;
  }
  return lo;
}

// Scene box of each cloud: one block per cloud.
__global__ void __launch_bounds__(256) k_seg_bounds(const float *__restrict__ pts, const uint32_t *__restrict__ off,
                                                   float *__restrict__ seg_scene, uint32_t *__restrict__ err) {
  const uint32_t c = blockIdx.x;
  const uint32_t b = off[c], e = off[c + 1];
  float mn[3], mx[3];
  uint32_t bad = 0;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    mn[a] = __int_as_float(0x7f800000);
    mx[a] = __int_as_float(0xff800000);
  }
  for (uint32_t i = b + threadIdx.x; i < e; i += blockDim.x) {
#pragma unroll
    for (int a = 0; a < 3; ++a) acc_axis(__ldg(pts + 3 * (uint64_t)i + a), mn[a], mx[a], bad);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      mn[a] = fminf(mn[a], __shfl_xor_sync(0xffffffffu, mn[a], o));
      mx[a] = fmaxf(mx[a], __shfl_xor_sync(0xffffffffu, mx[a], o));
    }
    bad += __shfl_xor_sync(0xffffffffu, bad, o);
  }
  __shared__ float s_v[8][6];
  __shared__ uint32_t s_bad[8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      s_v[warp][a] = mn[a];
      s_v[warp][3 + a] = mx[a];
    }
    s_bad[warp] = bad;
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    const int a = threadIdx.x;
    float v = s_v[0][a];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) v = a < 3 ? fminf(v, s_v[w][a]) : fmaxf(v, s_v[w][a]);
    seg_scene[6 * c + a] = v;
  } else if (threadIdx.x == 32) {
    uint32_t t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_bad[w];
    if (t) atomicOr(err, ERR_NONFINITE);
  }
}

// Key (internal cloud id << 30) | 30-bit Morton code against the cloud's own
// scene box (queries clamped into it); histograms of every radix pass.
__global__ void __launch_bounds__(256) k_seg_morton(const float *__restrict__ pts, uint32_t count,
                                                   const uint32_t *__restrict__ off, uint32_t n_clouds,
                                                   const uint32_t *__restrict__ cmap,
                                                   const float *__restrict__ seg_scene, uint64_t *__restrict__ keys,
                                                   uint32_t *__restrict__ hist, int passes) {
  __shared__ uint32_t s_h[8][kRadix];
  for (int i = threadIdx.x; i < passes * kRadix; i += blockDim.x) (&s_h[0][0])[i] = 0;
  __syncthreads();
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
    const uint32_t c = cloud_of(off, n_clouds, i);
    float sc[6];
#pragma unroll
    for (int a = 0; a < 6; ++a) sc[a] = __ldg(seg_scene + 6 * c + a);
    const uint32_t code = morton<uint32_t>(__ldg(pts + 3 * (uint64_t)i), __ldg(pts + 3 * (uint64_t)i + 1),
                                           __ldg(pts + 3 * (uint64_t)i + 2), sc);
    const uint64_t key = ((uint64_t)__ldg(cmap + c) << 30) | code;
    keys[i] = key;
    hist_add<uint64_t>(s_h, passes, key);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < passes * kRadix; i += blockDim.x) {
    const uint32_t c = (&s_h[0][0])[i];
    if (c) atomicAdd(&hist[i], c);
  }
}

// Root slot of every cloud in the tree over the (cloud, code) keys: the cloud
// owns sorted positions [a, b]; the node covering exactly that range hangs in
// its parent's record at split b (left child) when the keys share a longer
// prefix across b | b+1 than across a-1 | a, else at split a - 1 (right
// child) -- the parent rule of the build.  The whole range [0, N - 1] is the
// root (record slot 0).  Empty clouds get -1.
__global__ void __launch_bounds__(256) k_seg_roots(const uint64_t *__restrict__ codes, uint32_t n,
                                                  const uint32_t *__restrict__ sorted_off, uint32_t n_clouds,
                                                  int32_t *__restrict__ root_slot) {
  const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_clouds) return;
  const int a = (int)sorted_off[c], b = (int)sorted_off[c + 1] - 1, N = (int)n;
  if (b < a) {
    root_slot[c] = -1;
    return;
  }
  if (a == 0 && b == N - 1) {
    root_slot[c] = 0;
    return;
  }
  const int dr = delta<uint64_t>(codes, codes[b], b, b + 1, N);
  const int dl = a > 0 ? delta<uint64_t>(codes, codes[a - 1], a - 1, a, N) : -1;
  const bool left_child = dr > dl;
  const int p = left_child ? b : a - 1;
  root_slot[c] = 2 + 2 * p + (left_child ? 0 : 1);
}

int sm_count() {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}

}  // namespace

void launch_iota_on_timeout(uint32_t *order, uint32_t m, const uint32_t *err, cudaStream_t s) {
  if (m == 0) return;
  k_iota_on_timeout<<<ceil_div<uint32_t>(m, 256u), 256, 0, s>>>(order, m, err);
}

void launch_init_meta(DevMeta *meta, cudaStream_t s) { k_init_meta<<<1, 32, 0, s>>>(meta); }

void launch_init_meta_zero(DevMeta *meta, void *zero, size_t bytes, cudaStream_t s) {
  const uint64_t words = bytes / 16;  // bytes: a multiple of 16 at a 16-byte aligned address
  const uint32_t blocks =
      (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(ceil_div<uint64_t>(words, 256), (uint64_t)sm_count() * 4));
  k_init_meta_zero<<<blocks, 256, 0, s>>>(meta, static_cast<uint4 *>(zero), words);
}

void launch_bounds(const float *prims, int64_t n, int kind, DevMeta *meta, cudaStream_t s) {
  const uint64_t nf = (uint64_t)n * (kind == 0 ? 3 : 6);
  if (nf == 0) return;
  const bool vec = (reinterpret_cast<uintptr_t>(prims) & 15u) == 0;
  const uint64_t work = vec ? nf / 12 + 1 : nf;
  // one resident wave: a grid of 8 blocks per SM at the kernel's 6 resident blocks ran a second,
  // quarter-occupied wave (29.6 -> 26.8 us at 1e7 points)
  int occ = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_bounds, 256, 0);
  const uint32_t blocks =
      (uint32_t)std::min<uint64_t>(ceil_div<uint64_t>(work, 256), (uint64_t)sm_count() * std::max(occ, 1));
  prof::Scope ps(s, "bounds");
  k_bounds<<<blocks, 256, 0, s>>>(prims, nf, vec, meta);
}

template <typename K>
void launch_morton(const float *prims, uint32_t n, int kind, DevMeta *meta, K *codes, uint32_t *hist, int passes,
                   bool write_scene, cudaStream_t s, int drop) {
  if (n == 0) return;
  const bool vec = (reinterpret_cast<uintptr_t>(prims) & 15u) == 0;
  const uint32_t per_thread = kind == 0 ? 4 : 2;
  const uint32_t blocks = std::min<uint32_t>(ceil_div<uint32_t>(ceil_div<uint32_t>(n, per_thread), 256u),
                                        (uint32_t)sm_count() * 8u);
  prof::Scope ps(s, "morton");
  if (kind == 0)
    k_morton<K, 0><<<blocks, 256, 0, s>>>(prims, n, vec, meta, codes, hist, passes, write_scene, drop);
  else
    k_morton<K, 1><<<blocks, 256, 0, s>>>(prims, n, vec, meta, codes, hist, passes, write_scene, drop);
}

template <typename K>
void launch_hierarchy(const K *codes, uint32_t n, int32_t *parent, cudaStream_t s) {
  if (n < 2) return;
  prof::Scope ps(s, "hierarchy");
  k_hierarchy<K><<<ceil_div<uint32_t>(n - 1, 256u), 256, 0, s>>>(codes, n, parent);
}

void launch_fit(const float *prims, uint32_t n, int kind, const uint32_t *perm, const int32_t *parent,
                uint32_t *arrival, float4 *rec, uint32_t *err, cudaStream_t s) {
  if (n == 0) return;
  prof::Scope ps(s, "fit");
  if (kind == 0)
    k_fit<0><<<ceil_div<uint32_t>(n, 256u), 256, 0, s>>>(prims, n, perm, parent, arrival, rec, err);
  else
    k_fit<1><<<ceil_div<uint32_t>(n, 256u), 256, 0, s>>>(prims, n, perm, parent, arrival, rec, err);
}

size_t apetrei_front_bytes(uint32_t n) { return (size_t)2 * ceil_div<uint32_t>(std::max(n, 1u), kApChunk) * sizeof(Frontier); }

template <typename K>
void launch_apetrei(const float *prims, uint32_t n, int kind, const K *codes, const uint32_t *perm, int32_t *other,
                    float4 *rec, void *front_ws, uint32_t *err, cudaStream_t s) {
  if (n == 0) return;
  prof::Scope ps(s, "apetrei");
  const uint32_t chunks = ceil_div<uint32_t>(n, (uint32_t)kApChunk);
  Frontier *front = static_cast<Frontier *>(front_ws);
  if (kind == 0)
    k_apetrei_local<K, 0><<<chunks, kApBlock, 0, s>>>(prims, n, codes, perm, other, rec, front, err);
  else
    k_apetrei_local<K, 1><<<chunks, kApBlock, 0, s>>>(prims, n, codes, perm, other, rec, front, err);
  if (chunks > 1)
    k_apetrei_top<K><<<ceil_div<uint32_t>(2 * chunks, 256u), 256, 0, s>>>(codes, n, other, rec, front, 2 * chunks,
                                                                          err);
}

void launch_seg_bounds(const float *pts, const uint32_t *off, uint32_t n_clouds, float *seg_scene, uint32_t *err,
                       cudaStream_t s) {
  if (n_clouds == 0) return;
  prof::Scope ps(s, "seg_bounds");
  k_seg_bounds<<<n_clouds, 256, 0, s>>>(pts, off, seg_scene, err);
}

void launch_seg_morton(const float *pts, uint32_t count, const uint32_t *off, uint32_t n_clouds, const uint32_t *cmap,
                       const float *seg_scene, uint64_t *keys, uint32_t *hist, int passes, cudaStream_t s) {
  if (count == 0) return;
  const uint32_t blocks = std::min<uint32_t>(ceil_div<uint32_t>(count, 256u), (uint32_t)sm_count() * 8u);
  prof::Scope ps(s, "seg_morton");
  k_seg_morton<<<blocks, 256, 0, s>>>(pts, count, off, n_clouds, cmap, seg_scene, keys, hist, passes);
}

void launch_seg_roots(const uint64_t *codes, uint32_t n, const uint32_t *sorted_off, uint32_t n_clouds,
                      int32_t *root_slot, cudaStream_t s) {
  if (n_clouds == 0 || n == 0) return;
  prof::Scope ps(s, "seg_roots");
  k_seg_roots<<<ceil_div<uint32_t>(n_clouds, 256u), 256, 0, s>>>(codes, n, sorted_off, n_clouds, root_slot);
}

template void launch_apetrei<uint32_t>(const float *, uint32_t, int, const uint32_t *, const uint32_t *, int32_t *,
                                       float4 *, void *, uint32_t *, cudaStream_t);
template void launch_apetrei<uint64_t>(const float *, uint32_t, int, const uint64_t *, const uint32_t *, int32_t *,
                                       float4 *, void *, uint32_t *, cudaStream_t);
template void launch_morton<uint32_t>(const float *, uint32_t, int, DevMeta *, uint32_t *, uint32_t *, int, bool,
                                      cudaStream_t, int);
template void launch_morton<uint64_t>(const float *, uint32_t, int, DevMeta *, uint64_t *, uint32_t *, int, bool,
                                      cudaStream_t, int);
template void launch_hierarchy<uint32_t>(const uint32_t *, uint32_t, int32_t *, cudaStream_t);
template void launch_hierarchy<uint64_t>(const uint64_t *, uint32_t, int32_t *, cudaStream_t);

}  // namespace abx

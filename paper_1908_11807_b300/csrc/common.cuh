// Shared device helpers of the LBVH library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace abx {

// device error word bits (DevMeta::err)
enum : uint32_t {
  ERR_NONFINITE = 1u << 0,  // a primitive coordinate is NaN or +-inf
  ERR_TIMEOUT = 1u << 1,    // a bounded look-back wait gave up
  ERR_STACK = 1u << 2,      // traversal stack exceeded its static bound
  ERR_CSR = 1u << 3,        // spatial fill would write past the index capacity
};

// Per-tree device block: scene box reduction and sticky error word.
struct DevMeta {
  uint32_t bounds_ord[6];  // order-preserving encodings of lo.xyz (min) and hi.xyz (max)
  uint32_t nonfinite;      // count of non-finite coordinates seen by the reduction
  uint32_t err;            // ERR_* bits, sticky until read by arborx_check
  float scene[6];          // decoded scene box lo.xyz, hi.xyz
  uint32_t pad[2];
  unsigned long long nodes[2];    // traversal statistics: internal nodes loaded (spatial, nearest)
  unsigned long long queries[2];  // queries traversed (spatial, nearest)
};

constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;

// float <-> unsigned with the same order (for atomicMin / atomicMax on floats)
__device__ __forceinline__ uint32_t f2ord(float f) {
  uint32_t b = __float_as_uint(f);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float ord2f(uint32_t o) {
  uint32_t b = (o & 0x80000000u) ? (o & 0x7fffffffu) : ~o;
  return __uint_as_float(b);
}

__device__ __forceinline__ bool is_finite_bits(float v) {
  return (__float_as_uint(v) & 0x7f800000u) != 0x7f800000u;
}

__device__ __forceinline__ uint32_t lane_id() {
  uint32_t l;
  asm volatile("mov.u32 %0, %%laneid;" : "=r"(l));
  return l;
}
__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm volatile("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}
__device__ __forceinline__ uint32_t lanemask_gt() {
  uint32_t m;
  asm volatile("mov.u32 %0, %%lanemask_gt;" : "=r"(m));
  return m;
}

// GPU-scope relaxed accesses for words other blocks read while this kernel runs
__device__ __forceinline__ uint32_t ld_relaxed_gpu(const uint32_t *p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_gpu(uint32_t *p, uint32_t v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
// acq_rel exchange: publishes this thread's earlier writes, acquires the other arriver's
__device__ __forceinline__ int32_t atom_exch_acq_rel_gpu(int32_t *p, int32_t v) {
  int32_t old;
  asm volatile("atom.acq_rel.gpu.global.exch.b32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}
// acq_rel add: releases this thread's earlier writes, acquires the other arriver's
__device__ __forceinline__ uint32_t atom_add_acq_rel_gpu(uint32_t *p, uint32_t v) {
  uint32_t old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}
// L1-bypassing vector load (data written by another block of the same kernel)
__device__ __forceinline__ float4 ld_cg_f4(const float4 *p) { return __ldcg(p); }
__device__ __forceinline__ float ld_cg_f32(const float *p) { return __ldcg(p); }

__device__ __forceinline__ void set_err(uint32_t *err, uint32_t bit) {
  if (err) atomicOr(err, bit);
}

// Per-axis gap between a point coordinate and an interval [lo, hi] (0 inside),
// one FP32 rounding per subtraction; equals |q - p| exactly when lo == hi == p.
__device__ __forceinline__ float axis_gap(float q, float lo, float hi) {
  return fmaxf(fmaxf(__fsub_rn(lo, q), __fsub_rn(q, hi)), 0.0f);
}

// d^2 = ((gx*gx) + (gy*gy)) + (gz*gz), round-to-nearest, never contracted
__device__ __forceinline__ float dist2_box(float qx, float qy, float qz, float4 lo, float4 hi) {
  float gx = axis_gap(qx, lo.x, hi.x);
  float gy = axis_gap(qy, lo.y, hi.y);
  float gz = axis_gap(qz, lo.z, hi.z);
  return __fadd_rn(__fadd_rn(__fmul_rn(gx, gx), __fmul_rn(gy, gy)), __fmul_rn(gz, gz));
}

template <typename T>
__host__ __device__ constexpr T ceil_div(T a, T b) {
  return (a + b - 1) / b;
}

}  // namespace abx

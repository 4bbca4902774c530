// Learned k-th-neighbour distance (an initial bound for the nearest traversal
// of ArborX Sec. 2.2, "Traversal for nearest queries"; the traversal itself and
// its exactness are unchanged).  Regressor 3 -> 64 -> 64 -> 1 with ReLU,
// inputs normalised by the tree's scene box, predicting log d_k.
//
// Training (FP32, CUDA cores): k_mlp_grad runs forward + backward for 32
// samples per block and writes the block's gradient; k_adam sums the block
// gradients in a fixed order (deterministic) and applies Adam.
// Inference (BF16 in, FP32 accumulate): k_mlp_bound_tc puts the 64x64 hidden
// layer on the 5th-generation tensor cores -- one tcgen05.mma M=128 N=64 K=64
// per tile of 128 queries, operands in shared memory, accumulators in tensor
// memory -- and writes the initial squared bound exp(2 (y + margin)).
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>

#include "kernels.cuh"
#include "prof.cuh"

namespace abx {

namespace {

constexpr int kH = 64;
constexpr int kNP = kMlpParams;  // 4481
constexpr int OFF_W1 = 0, OFF_B1 = 192, OFF_W2 = 256, OFF_B2 = 4352, OFF_W3 = 4416, OFF_B3 = 4480;
constexpr int kS = 32;  // samples per training block

__device__ __forceinline__ void normalise(const DevMeta *meta, float qx, float qy, float qz, float &x0, float &x1,
                                          float &x2) {
  const float *sc = meta->scene;
  const float e0 = sc[3] - sc[0], e1 = sc[4] - sc[1], e2 = sc[5] - sc[2];
  x0 = e0 > 0.f ? (qx - sc[0]) / e0 : 0.f;
  x1 = e1 > 0.f ? (qy - sc[1]) / e1 : 0.f;
  x2 = e2 > 0.f ? (qz - sc[2]) / e2 : 0.f;
}

// Forward + backward of the mean squared error over samples
// (start + blockIdx.x * kS + s) mod mt; block gradient -> partial[blockIdx.x].
__global__ void __launch_bounds__(256) k_mlp_grad(const float *__restrict__ params, const float *__restrict__ queries,
                                                 const float *__restrict__ labels, int64_t mt, int64_t start, int b,
                                                 float inv_b, const DevMeta *__restrict__ meta,
                                                 float *__restrict__ partial) {
  extern __shared__ float sm[];
  float *sp = sm;               // parameters, 4481 (+pad)
  float *sW2T = sp + 4488;      // W2 transposed [j][i]
  float *sx = sW2T + 4096;      // inputs [kS][3]
  float *st = sx + 128;         // labels
  float *sdy = st + 32;         // dL/dy
  float *sh1 = sdy + 32;        // hidden 1 [kS][64]
  float *sh2 = sh1 + kS * kH;   // hidden 2
  float *sdz2 = sh2 + kS * kH;  // dL/dz2
  float *sdz1 = sdz2 + kS * kH;
  __shared__ float s_loss[8];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int i = tid; i < kNP; i += 256) sp[i] = params[i];
  for (int e = tid; e < kH * kH; e += 256) sW2T[(e & 63) * kH + (e >> 6)] = params[OFF_W2 + e];
  const int nb = min(kS, b - (int)blockIdx.x * kS);
  if (tid < kS) {
    const int s = tid;
    float x0 = 0.f, x1 = 0.f, x2 = 0.f, t = 0.f;
    if (s < nb) {
      const int64_t idx = (start + (int64_t)blockIdx.x * kS + s) % mt;
      normalise(meta, queries[3 * idx], queries[3 * idx + 1], queries[3 * idx + 2], x0, x1, x2);
      t = labels[idx];
    }
    sx[3 * s] = x0;
    sx[3 * s + 1] = x1;
    sx[3 * s + 2] = x2;
    st[s] = t;
  }
  __syncthreads();
  for (int e = tid; e < kS * kH; e += 256) {
    const int s = e >> 6, j = e & 63;
    const float z = sp[OFF_B1 + j] + sp[OFF_W1 + 3 * j] * sx[3 * s] + sp[OFF_W1 + 3 * j + 1] * sx[3 * s + 1] +
                    sp[OFF_W1 + 3 * j + 2] * sx[3 * s + 2];
    sh1[e] = fmaxf(z, 0.f);
  }
  __syncthreads();
  {
    const int i = tid & 63, s0 = tid >> 6;
    float acc[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) acc[u] = sp[OFF_B2 + i];
    for (int j = 0; j < kH; ++j) {
      const float w = sW2T[j * kH + i];
#pragma unroll
      for (int u = 0; u < 8; ++u) acc[u] += w * sh1[(s0 + 4 * u) * kH + j];
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) sh2[(s0 + 4 * u) * kH + i] = fmaxf(acc[u], 0.f);
  }
  __syncthreads();
  float lsum = 0.f;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int s = warp + 8 * u;
    float v = sp[OFF_W3 + lane] * sh2[s * kH + lane] + sp[OFF_W3 + lane + 32] * sh2[s * kH + lane + 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const float r = s < nb ? v + sp[OFF_B3] - st[s] : 0.f;
    if (lane == 0) sdy[s] = 2.f * r * inv_b;
    lsum += r * r;
  }
  if (lane == 0) s_loss[warp] = lsum;
  __syncthreads();
  for (int e = tid; e < kS * kH; e += 256) {
    const int s = e >> 6, i = e & 63;
    sdz2[e] = sh2[e] > 0.f ? sdy[s] * sp[OFF_W3 + i] : 0.f;
  }
  __syncthreads();
  float *out = partial + (size_t)blockIdx.x * (kNP + 1);
#pragma unroll 4
  for (int u = 0; u < 16; ++u) {
    const int e = tid + 256 * u, i = e >> 6, j = e & 63;
    float g = 0.f;
    for (int s = 0; s < kS; ++s) g += sdz2[s * kH + i] * sh1[s * kH + j];
    out[OFF_W2 + e] = g;
  }
  if (tid < 64) {
    float g = 0.f;
    for (int s = 0; s < kS; ++s) g += sdy[s] * sh2[s * kH + tid];
    out[OFF_W3 + tid] = g;
  } else if (tid < 128) {
    const int i = tid - 64;
    float g = 0.f;
    for (int s = 0; s < kS; ++s) g += sdz2[s * kH + i];
    out[OFF_B2 + i] = g;
  } else if (tid == 128) {
    float g = 0.f;
    for (int s = 0; s < kS; ++s) g += sdy[s];
    out[OFF_B3] = g;
  } else if (tid == 129) {
    float l = 0.f;
    for (int w = 0; w < 8; ++w) l += s_loss[w];
    out[kNP] = l * inv_b;  // this block's share of the batch loss
  }
  {
    const int j = tid & 63, s0 = tid >> 6;
    float acc[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) acc[u] = 0.f;
    for (int i = 0; i < kH; ++i) {
      const float w = sp[OFF_W2 + i * kH + j];
#pragma unroll
      for (int u = 0; u < 8; ++u) acc[u] += w * sdz2[(s0 + 4 * u) * kH + i];
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int s = s0 + 4 * u;
      sdz1[s * kH + j] = sh1[s * kH + j] > 0.f ? acc[u] : 0.f;
    }
  }
  __syncthreads();
  {
    const int e = tid;  // 192 entries of dW1, 64 of db1
    float g = 0.f;
    if (e < 192) {
      const int j = e / 3, c = e % 3;
      for (int s = 0; s < kS; ++s) g += sdz1[s * kH + j] * sx[3 * s + c];
      out[OFF_W1 + e] = g;
    } else {
      const int j = e - 192;
      for (int s = 0; s < kS; ++s) g += sdz1[s * kH + j];
      out[OFF_B1 + j] = g;
    }
  }
}

// Sum the block gradients (fixed order) and take one Adam step (c1, c2 = bias
// corrections 1 - beta^t).  lr = 0 only reduces: grad_out gets the gradient.
__global__ void k_adam(float *__restrict__ params, float *__restrict__ mom, float *__restrict__ vel,
                       const float *__restrict__ partial, int nblocks, float lr, float b1, float b2, float eps,
                       float c1, float c2, float *__restrict__ grad_out, float *__restrict__ loss_out,
                       float loss_scale) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p > kNP) return;
  float g = 0.f;
  for (int b = 0; b < nblocks; ++b) g += partial[(size_t)b * (kNP + 1) + p];
  if (p == kNP) {
    if (loss_out) *loss_out += g * loss_scale;
    return;
  }
  if (grad_out) grad_out[p] = g;
  if (lr == 0.f) return;
  const float m = b1 * mom[p] + (1.f - b1) * g;
  const float v = b2 * vel[p] + (1.f - b2) * g * g;
  mom[p] = m;
  vel[p] = v;
  params[p] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
}

// labels t_i = log(max(d_k, 1e-30)) from the k-th squared distance of each row
__global__ void k_labels(const float *__restrict__ d2, int64_t mt, int kk, float *__restrict__ labels) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= mt) return;
  const float d = sqrtf(d2[i * kk + kk - 1]);
  labels[i] = logf(fmaxf(d, 1e-30f));
}

// FP32 reference forward on CUDA cores (one thread per query).
__global__ void __launch_bounds__(128) k_mlp_forward(const float *__restrict__ params, const float *__restrict__ queries,
                                                    uint32_t m, const DevMeta *__restrict__ meta,
                                                    float *__restrict__ y) {
  __shared__ float sp[kNP + 3];
  for (int i = threadIdx.x; i < kNP; i += blockDim.x) sp[i] = params[i];
  __syncthreads();
  const uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= m) return;
  float x0, x1, x2;
  normalise(meta, queries[3 * (uint64_t)q], queries[3 * (uint64_t)q + 1], queries[3 * (uint64_t)q + 2], x0, x1, x2);
  float h1[kH];
#pragma unroll
  for (int j = 0; j < kH; ++j)
    h1[j] = fmaxf(sp[OFF_B1 + j] + sp[OFF_W1 + 3 * j] * x0 + sp[OFF_W1 + 3 * j + 1] * x1 + sp[OFF_W1 + 3 * j + 2] * x2,
                  0.f);
  float out = sp[OFF_B3];
  for (int i = 0; i < kH; ++i) {
    float z = sp[OFF_B2 + i];
#pragma unroll
    for (int j = 0; j < kH; ++j) z += sp[OFF_W2 + i * kH + j] * h1[j];
    out += sp[OFF_W3 + i] * fmaxf(z, 0.f);
  }
  y[q] = out;
}

// ------------------------------------------------------ tcgen05 inference

constexpr int kTile = 128;                  // queries per tile = TMEM lanes
constexpr uint32_t kTmemCols = 64;          // FP32 accumulator columns (N = 64)
constexpr uint32_t kLBO = 128;              // bytes between K-adjacent 8x16B core matrices
constexpr uint32_t kSBO = 1024;             // bytes between M/N-adjacent 8-row groups (8 K chunks)
constexpr uint32_t kMbarSpinCap = 1u << 24;
// Resident blocks per SM: 8 x 64 accumulator columns fill the SM's 512 TMEM columns, and the
// kernel's 27 KB of static shared memory admits no ninth block, so every allocation is granted.
constexpr int kTcBlocksPerSm = 8;

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// UMMA shared-memory descriptor, K-major, no swizzle
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
         (1ull << 46);
}

// instruction descriptor: D = F32, A = B = BF16, both K-major, N = 64, M = 128
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((64u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t *>(&h);
}

// byte offset of element (row, k) in a K-major, no-swizzle core-matrix tile with 64 K columns
__device__ __forceinline__ uint32_t core_off(int row, int k) {
  return (uint32_t)((row >> 3) * kSBO + (k >> 3) * kLBO + (row & 7) * 16 + (k & 7) * 2);
}

__global__ void __launch_bounds__(kTile, kTcBlocksPerSm) k_mlp_bound_tc(const float *__restrict__ params,
                                                       const float *__restrict__ queries, uint32_t m,
                                                       const DevMeta *__restrict__ meta, float margin,
                                                       float *__restrict__ bound2, float *__restrict__ y_out,
                                                       uint32_t *__restrict__ err) {
  __shared__ __align__(1024) unsigned char sA[kTile * kH * 2];  // h1 tile, BF16
  __shared__ __align__(1024) unsigned char sB[kH * kH * 2];     // W2, BF16 ([n = out][k = in])
  __shared__ float4 sL1[kH];  // layer 1, hidden unit j: (W1[j][0], W1[j][1], W1[j][2], b1[j])
  __shared__ float sb2[kH], sw3[kH];
  __shared__ float sb3;
  __shared__ float s_lo[3], s_inv[3];  // scene-box corner and reciprocal extents (0 on a flat axis)
  __shared__ __align__(8) unsigned long long mbar;
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid < kH) {
    sL1[tid] = make_float4(params[OFF_W1 + 3 * tid], params[OFF_W1 + 3 * tid + 1], params[OFF_W1 + 3 * tid + 2],
                           params[OFF_B1 + tid]);
    sb2[tid] = params[OFF_B2 + tid];
    sw3[tid] = params[OFF_W3 + tid];
  }
  if (tid == 0) sb3 = params[OFF_B3];
  if (tid < 3) {
    const float e = meta->scene[3 + tid] - meta->scene[tid];
    s_lo[tid] = meta->scene[tid];
    s_inv[tid] = e > 0.f ? 1.0f / e : 0.f;
  }
  for (int e = tid; e < kH * kH / 2; e += kTile) {  // two consecutive k per store
    const int n = (2 * e) >> 6, k = (2 * e) & 63;
    *reinterpret_cast<uint32_t *>(sB + core_off(n, k)) =
        pack_bf16(params[OFF_W2 + n * kH + k], params[OFF_W2 + n * kH + k + 1]);
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("fence.proxy.async.shared::cta;");
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t taddr = tmem_base;
  const uint32_t aaddr = smem_u32(sA), baddr = smem_u32(sB);
  uint32_t phase = 0;
  bool failed = false;

  // the next tile's query is loaded while this tile computes
  float r0 = 0.f, r1 = 0.f, r2 = 0.f;
  auto fetch = [&](uint32_t tile) {
    const uint64_t qn = (uint64_t)tile * kTile + tid;
    if (qn < m) {
      r0 = __ldg(queries + 3 * qn);
      r1 = __ldg(queries + 3 * qn + 1);
      r2 = __ldg(queries + 3 * qn + 2);
    }
  };
  fetch(blockIdx.x);
  for (uint32_t tile = blockIdx.x; tile * kTile < m && !failed; tile += gridDim.x) {
    const uint32_t q = tile * kTile + tid;
    const bool valid = q < m;
    float x0 = 0.f, x1 = 0.f, x2 = 0.f;
    if (valid) {  // the scene-box scaling as one multiply per axis (a flat axis gives 0)
      x0 = s_inv[0] > 0.f ? (r0 - s_lo[0]) * s_inv[0] : 0.f;
      x1 = s_inv[1] > 0.f ? (r1 - s_lo[1]) * s_inv[1] : 0.f;
      x2 = s_inv[2] > 0.f ? (r2 - s_lo[2]) * s_inv[2] : 0.f;
    }
    fetch(tile + gridDim.x);
    // layer 1 in FP32, stored as BF16 row `tid` of the A tile (8 K-chunks of 16 bytes)
#pragma unroll
    for (int kc = 0; kc < 8; ++kc) {
      uint32_t w[4];
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        const int j = kc * 8 + 2 * h;
        const float4 ua = sL1[j], ub = sL1[j + 1];
        const float a = fmaxf(fmaf(ua.z, x2, fmaf(ua.y, x1, fmaf(ua.x, x0, ua.w))), 0.f);
        const float b = fmaxf(fmaf(ub.z, x2, fmaf(ub.y, x1, fmaf(ub.x, x0, ub.w))), 0.f);
        w[h] = pack_bf16(a, b);
      }
      *reinterpret_cast<uint4 *>(sA + core_off(tid, kc * 8)) = make_uint4(w[0], w[1], w[2], w[3]);
    }
    asm volatile("fence.proxy.async.shared::cta;");  // generic-proxy writes -> tensor core reads
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
      for (int ks = 0; ks < 4; ++ks) {  // K = 16 per instruction: two core matrices along K
        const uint64_t ad = umma_desc(aaddr + ks * 2 * kLBO, kLBO, kSBO);
        const uint64_t bd = umma_desc(baddr + ks * 2 * kLBO, kLBO, kSBO);
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(taddr),
            "l"(ad), "l"(bd), "r"(kIdesc), "r"(ks));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(&mbar)));
    }
    // wait for the accumulators (bounded)
    uint32_t done = 0, spins = 0;
    while (!done) {
      asm volatile(
          "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
          : "=r"(done)
          : "r"(smem_u32(&mbar)), "r"(phase));
      if (!done && ++spins >= kMbarSpinCap) {
        failed = true;
        break;
      }
    }
    if (failed) {
      set_err(err, ERR_TIMEOUT);
      break;
    }
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;");
    float y = sb3;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      float v[16];
      tmem_ld16(taddr + ((uint32_t)(warp * 32) << 16) + c * 16, v);
      asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
      for (int i = 0; i < 16; ++i) y += sw3[c * 16 + i] * fmaxf(v[i] + sb2[c * 16 + i], 0.f);
    }
    if (valid) {
      if (bound2) bound2[q] = expf(2.f * (y + margin));
      if (y_out) y_out[q] = y;
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
  }
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(kTmemCols));
}

int sms() {
  int dev = 0, n = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n;
}

}  // namespace

size_t mlp_grad_smem_bytes() { return (size_t)(4488 + 4096 + 128 + 64 + 4 * kS * kH) * sizeof(float); }

void launch_mlp_grad(const float *params, const float *queries, const float *labels, int64_t mt, int64_t start, int b,
                     const DevMeta *meta, float *partial, cudaStream_t s) {
  const int blocks = (b + kS - 1) / kS;
  const size_t smem = mlp_grad_smem_bytes();
  cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  prof::Scope ps(s, "mlp_grad");
  k_mlp_grad<<<blocks, 256, smem, s>>>(params, queries, labels, mt, start, b, 1.0f / (float)b, meta, partial);
}

void launch_adam(float *params, float *mom, float *vel, const float *partial, int nblocks, float lr, float b1, float b2,
                 float eps, float c1, float c2, float *grad_out, float *loss_out, float loss_scale, cudaStream_t s) {
  prof::Scope ps(s, "adam");
  k_adam<<<(kNP + 1 + 255) / 256, 256, 0, s>>>(params, mom, vel, partial, nblocks, lr, b1, b2, eps, c1, c2, grad_out,
                                                loss_out, loss_scale);
}

void launch_labels(const float *d2, int64_t mt, int kk, float *labels, cudaStream_t s) {
  if (mt == 0) return;
  k_labels<<<(unsigned)((mt + 255) / 256), 256, 0, s>>>(d2, mt, kk, labels);
}

void launch_mlp_forward(const float *params, const float *queries, uint32_t m, const DevMeta *meta, float *y,
                        cudaStream_t s) {
  if (m == 0) return;
  prof::Scope ps(s, "mlp_forward");
  k_mlp_forward<<<ceil_div<uint32_t>(m, 128u), 128, 0, s>>>(params, queries, m, meta, y);
}

void launch_mlp_bound(const float *params, const float *queries, uint32_t m, const DevMeta *meta, float margin,
                      float *bound2, float *y_out, uint32_t *err, cudaStream_t s) {
  if (m == 0) return;
  const uint32_t tiles = ceil_div<uint32_t>(m, (uint32_t)kTile);
  const uint32_t grid = std::min<uint32_t>(tiles, (uint32_t)sms() * (uint32_t)kTcBlocksPerSm);
  prof::Scope ps(s, "mlp_bound_tc");
  k_mlp_bound_tc<<<grid, kTile, 0, s>>>(params, queries, m, meta, margin, bound2, y_out, err);
}

}  // namespace abx

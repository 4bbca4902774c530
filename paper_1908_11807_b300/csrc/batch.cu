// Many independent point clouds built and queried together: one launch
// sequence (optionally replayed from a CUDA graph) instead of a build and a
// query per cloud.
//
// Keys are (internal cloud id << 30) | 30-bit Morton code against the cloud's
// own scene box, so one stable radix sort groups the clouds and orders each by
// its Z-curve; one bottom-up pass builds a single tree whose top levels split
// the clouds, recording the subtree of each cloud; queries are keyed the same
// way and answered by persistent warps that start at their cloud's subtree.
// Internal cloud ids order the clouds by their k class, so that every class of
// candidate-list width is one contiguous range of sorted queries.
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/arborx_b300.h"
#include "kernels.cuh"
#include "radix_sort.cuh"

using namespace abx;

struct arborx_batch_s {
  int64_t C = 0, N = 0, M = 0, entries = 0;
  arborx_opts opts;
  void *mem = nullptr;
  size_t mem_bytes = 0;
  cudaStream_t alloc_stream = nullptr;
  // per cloud (original order): point / query offsets; per internal cloud: the rest
  uint32_t *pt_off, *q_off, *cmap, *sorted_off, *prim_base, *ncount;
  int32_t *kof, *root_slot;
  int64_t *row_off;
  float *seg_scene;
  uint32_t *err;
  uint64_t *kA, *kB, *qkA, *qkB;
  uint32_t *vA, *vB, *qvA, *qvB;
  float4 *rec;
  int32_t *other;
  void *front;  // frontier list of the chunked hierarchy build
  uint32_t *queue;
  void *zero_base;
  size_t zero_bytes;
  SortWs wsp, wsq;
  struct Cls {
    int kc;
    uint32_t begin, end;
  };
  std::vector<Cls> classes;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t cap = nullptr;  // own stream: graphs cannot be captured on the legacy default stream
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  const float *g_pts = nullptr, *g_q = nullptr;
  int64_t *g_off = nullptr;
  int32_t *g_idx = nullptr;
  float *g_d2 = nullptr;
};

namespace {

constexpr size_t kAl = 256;
size_t al(size_t x) { return (x + kAl - 1) & ~(kAl - 1); }

// Query class of a cloud's k: the register-list width for k below heap_from (17 or 33), else 0
// (the shared-memory heap of up to 32 entries).  The heap is faster for large clouds, the
// 32-entry list for small ones (the 512-cloud workload of 1e3..1e5 points: 20.0 against 21.7 ms),
// so the threshold is an option the batch tuner picks.
int kc_of(int k, int heap_from) {
  const int widths[] = {1, 2, 4, 8, 10, 16, 32};
  for (int w : widths)
    if (k <= w && k < heap_from) return w;
  return k <= 32 ? 0 : -1;
}

int status_of(cudaError_t e) { return e == cudaSuccess ? ARBORX_OK : ARBORX_ECUDA; }

// Enqueue the whole batch on `s`; ARBORX_EINVAL if a query class cannot be launched.
int enqueue(arborx_batch_s *b, const float *pts, const float *qs, cudaStream_t s, int64_t *d_row_offsets,
             int32_t *d_idx, float *d_d2) {
  const uint32_t N = (uint32_t)b->N, M = (uint32_t)b->M, C = (uint32_t)b->C;
  cudaMemsetAsync(b->zero_base, 0, b->zero_bytes, s);
  cudaMemsetAsync(b->root_slot, 0xff, (size_t)C * sizeof(int32_t), s);
  const uint64_t *skeys = nullptr;
  const uint32_t *sperm = nullptr;
  if (N > 0) {
    launch_seg_bounds(pts, b->pt_off, C, b->seg_scene, b->err, s);
    launch_seg_morton(pts, N, b->pt_off, C, b->cmap, b->seg_scene, b->kA, b->wsp.hist, b->wsp.passes, s);
    const bool inA = launch_onesweep<uint64_t>(b->kA, b->kB, b->vA, b->vB, N, b->wsp, b->err, s);
    skeys = inA ? b->kA : b->kB;
    sperm = inA ? b->vA : b->vB;
    // one binary radix tree over the (cloud, code) keys: the cloud id in the high bits makes every
    // cloud one subtree; its root slot is found afterwards
    launch_apetrei<uint64_t>(pts, N, ARBORX_POINTS, skeys, sperm, b->other, b->rec, b->front, b->err, s);
    launch_seg_roots(skeys, N, b->sorted_off, C, b->root_slot, s);
  }
  if (d_row_offsets)
    cudaMemcpyAsync(d_row_offsets, b->row_off, (size_t)(M + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, s);
  if (M == 0) return ARBORX_OK;
  launch_seg_morton(qs, M, b->q_off, C, b->cmap, b->seg_scene, b->qkA, b->wsq.hist, b->wsq.passes, s);
  const bool qinA = launch_onesweep<uint64_t>(b->qkA, b->qkB, b->qvA, b->qvB, M, b->wsq, b->err, s);
  TravCfg cfg;
  cfg.block = b->opts.block_size > 0 ? b->opts.block_size : 128;
  cfg.stack_smem = b->opts.stack_smem > 0 ? b->opts.stack_smem : 16;
  cfg.stats_nodes = nullptr;
  for (size_t i = 0; i < b->classes.size(); ++i) {
    BatchQueryArgs a{};
    a.rec = b->rec;
    a.n = N;
    a.queries = qs;
    a.qperm = qinA ? b->qvA : b->qvB;
    a.qkeys = qinA ? b->qkA : b->qkB;
    a.pos_begin = b->classes[i].begin;
    a.pos_end = b->classes[i].end;
    a.queue = b->queue + i;
    a.root_slot = b->root_slot;
    a.kof = b->kof;
    a.ncount = b->ncount;
    a.prim_base = b->prim_base;
    a.row_off = b->row_off;
    a.out_idx = d_idx;
    a.out_d2 = d_d2;
    a.err = b->err;
    a.stack_smem = cfg.stack_smem;
    a.anchor = b->opts.knn_anchor;
    a.queries_per_warp = b->opts.queries_per_warp > 0 ? b->opts.queries_per_warp : 32;
    if (launch_batch_nearest(a, b->classes[i].kc, cfg, s)) return ARBORX_EINVAL;
  }
  return ARBORX_OK;
}

}  // namespace

extern "C" {

int arborx_batch_create(int64_t n_clouds, const int64_t *h_point_offsets, const int64_t *h_query_offsets,
                        const int32_t *h_k, const arborx_opts *opts, void *stream, arborx_batch *out) {
  if (!out || n_clouds < 1 || n_clouds > (1 << 20) || !h_point_offsets || !h_query_offsets || !h_k)
    return ARBORX_EINVAL;
  *out = nullptr;
  const int64_t C = n_clouds;
  if (h_point_offsets[0] != 0 || h_query_offsets[0] != 0) return ARBORX_EINVAL;
  for (int64_t c = 0; c < C; ++c) {
    if (h_point_offsets[c + 1] < h_point_offsets[c] || h_query_offsets[c + 1] < h_query_offsets[c]) return ARBORX_EINVAL;
    if (h_k[c] < 1 || h_k[c] > 32) return ARBORX_EINVAL;
  }
  const int64_t N = h_point_offsets[C], M = h_query_offsets[C];
  if (N >= ARBORX_MAX_PRIMS || M >= ARBORX_MAX_QUERIES) return ARBORX_EINVAL;
  arborx_opts o;
  if (opts) o = *opts;
  else arborx_default_opts(&o);
  if (o.block_size != 0 && (o.block_size < 32 || o.block_size > 256 || o.block_size % 32)) return ARBORX_EINVAL;
  if (o.stack_smem < 0 || o.stack_smem > 64) return ARBORX_EINVAL;
  if (o.knn_anchor < 0 || o.knn_anchor > 3) return ARBORX_EINVAL;
  if (o.knn_heap_from != 0 && o.knn_heap_from != 17 && o.knn_heap_from != 33) return ARBORX_EINVAL;
  if (o.queries_per_warp != 0 && o.queries_per_warp != 32 && o.queries_per_warp != 64 &&
      o.queries_per_warp != 128 && o.queries_per_warp != 256)
    return ARBORX_EINVAL;
  arborx_batch_s *b = new (std::nothrow) arborx_batch_s();
  if (!b) return ARBORX_ENOMEM;
  b->C = C;
  b->N = N;
  b->M = M;
  b->opts = o;
  const cudaStream_t s = (cudaStream_t)stream;
  b->alloc_stream = s;

  // internal cloud order: by candidate-list width, then original index
  std::vector<int64_t> order(C);
  for (int64_t c = 0; c < C; ++c) order[c] = c;
  const int heap_from = o.knn_heap_from > 0 ? o.knn_heap_from : 17;
  std::stable_sort(order.begin(), order.end(),
                   [&](int64_t x, int64_t y) { return kc_of(h_k[x], heap_from) < kc_of(h_k[y], heap_from); });
  std::vector<uint32_t> pt_off(C + 1), q_off(C + 1), cmap(C), sorted_off(C + 1), prim_base(C), ncount(C);
  std::vector<int32_t> kof(C);
  std::vector<int64_t> row_off(M + 1);
  for (int64_t c = 0; c <= C; ++c) {
    pt_off[c] = (uint32_t)h_point_offsets[c];
    q_off[c] = (uint32_t)h_query_offsets[c];
  }
  sorted_off[0] = 0;
  uint32_t qpos = 0;
  for (int64_t j = 0; j < C; ++j) {
    const int64_t c = order[j];
    cmap[c] = (uint32_t)j;
    const uint32_t nc = pt_off[c + 1] - pt_off[c], mc = q_off[c + 1] - q_off[c];
    sorted_off[j + 1] = sorted_off[j] + nc;
    prim_base[j] = pt_off[c];
    ncount[j] = nc;
    kof[j] = h_k[c];
    const int kc = kc_of(h_k[c], heap_from);
    if (mc > 0) {
      if (b->classes.empty() || b->classes.back().kc != kc) b->classes.push_back({kc, qpos, qpos});
      b->classes.back().end = qpos + mc;
    }
    qpos += mc;
  }
  row_off[0] = 0;
  for (int64_t c = 0; c < C; ++c) {
    const int64_t kk = std::min<int64_t>(h_k[c], pt_off[c + 1] - pt_off[c]);
    for (uint32_t qi = q_off[c]; qi < q_off[c + 1]; ++qi) row_off[qi + 1] = row_off[qi] + kk;
  }
  b->entries = row_off[M];

  // device memory, one allocation
  int cbits = 1;
  while (((int64_t)1 << cbits) < C) ++cbits;
  const int key_bits = 30 + cbits;
  const size_t wsp_words = sort_ws_words<uint64_t>(N, key_bits), wsq_words = sort_ws_words<uint64_t>(M, key_bits);
  const size_t nclass = std::max<size_t>(b->classes.size(), 1);
  const size_t rec_f4 = (size_t)(2 + 2 * (N > 0 ? N - 1 : 0)) * 2;
  size_t bytes = 0;
  auto take = [&](size_t sz) {
    const size_t at = bytes;
    bytes += al(sz);
    return at;
  };
  const size_t o_pt = take((C + 1) * 4), o_q = take((C + 1) * 4), o_cmap = take(C * 4), o_soff = take((C + 1) * 4),
               o_pb = take(C * 4), o_nc = take(C * 4), o_kof = take(C * 4), o_root = take(C * 4),
               o_row = take((M + 1) * 8), o_scene = take(C * 6 * 4), o_kA = take(N * 8), o_kB = take(N * 8),
               o_vA = take(N * 4), o_vB = take(N * 4), o_qkA = take(M * 8), o_qkB = take(M * 8), o_qvA = take(M * 4),
               o_qvB = take(M * 4), o_rec = take(rec_f4 * 16), o_other = take((N > 1 ? N - 1 : 1) * 4),
               o_front = take(apetrei_front_bytes((uint32_t)N));
  const size_t o_zero = bytes;
  const size_t o_wsp = take(wsp_words * 4), o_wsq = take(wsq_words * 4), o_queue = take(nclass * 4),
               o_err = take(4);
  b->zero_bytes = bytes - o_zero;
  b->mem_bytes = bytes;
  cudaError_t e = o.alloc ? cudaSuccess : cudaMallocAsync(&b->mem, bytes, s);
  if (o.alloc) b->mem = o.alloc(bytes, stream, o.alloc_ctx);
  if (e != cudaSuccess || !b->mem) {
    cudaGetLastError();
    delete b;
    return ARBORX_ENOMEM;
  }
  char *base = (char *)b->mem;
  b->pt_off = (uint32_t *)(base + o_pt);
  b->q_off = (uint32_t *)(base + o_q);
  b->cmap = (uint32_t *)(base + o_cmap);
  b->sorted_off = (uint32_t *)(base + o_soff);
  b->prim_base = (uint32_t *)(base + o_pb);
  b->ncount = (uint32_t *)(base + o_nc);
  b->kof = (int32_t *)(base + o_kof);
  b->root_slot = (int32_t *)(base + o_root);
  b->row_off = (int64_t *)(base + o_row);
  b->seg_scene = (float *)(base + o_scene);
  b->kA = (uint64_t *)(base + o_kA);
  b->kB = (uint64_t *)(base + o_kB);
  b->vA = (uint32_t *)(base + o_vA);
  b->vB = (uint32_t *)(base + o_vB);
  b->qkA = (uint64_t *)(base + o_qkA);
  b->qkB = (uint64_t *)(base + o_qkB);
  b->qvA = (uint32_t *)(base + o_qvA);
  b->qvB = (uint32_t *)(base + o_qvB);
  b->rec = (float4 *)(base + o_rec);
  b->other = (int32_t *)(base + o_other);
  b->front = base + o_front;
  b->zero_base = base + o_zero;
  b->wsp = sort_ws_carve<uint64_t>((uint32_t *)(base + o_wsp), N, key_bits);
  b->wsq = sort_ws_carve<uint64_t>((uint32_t *)(base + o_wsq), M, key_bits);
  b->queue = (uint32_t *)(base + o_queue);
  b->err = (uint32_t *)(base + o_err);
  cudaMemcpyAsync(b->pt_off, pt_off.data(), (C + 1) * 4, cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(b->q_off, q_off.data(), (C + 1) * 4, cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(b->cmap, cmap.data(), C * 4, cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(b->sorted_off, sorted_off.data(), (C + 1) * 4, cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(b->prim_base, prim_base.data(), C * 4, cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(b->ncount, ncount.data(), C * 4, cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(b->kof, kof.data(), C * 4, cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(b->row_off, row_off.data(), (M + 1) * 8, cudaMemcpyHostToDevice, s);
  const int st = status_of(cudaStreamSynchronize(s));  // host vectors go out of scope
  if (st) {
    arborx_batch_destroy(b);
    return st;
  }
  *out = b;
  return ARBORX_OK;
}

int arborx_batch_entries(arborx_batch b, int64_t *n_points, int64_t *n_queries, int64_t *entries) {
  if (!b) return ARBORX_EINVAL;
  if (n_points) *n_points = b->N;
  if (n_queries) *n_queries = b->M;
  if (entries) *entries = b->entries;
  return ARBORX_OK;
}

int arborx_batch_run(arborx_batch b, const float *d_points, const float *d_queries, int32_t use_graph, void *stream,
                     int64_t *d_row_offsets, int32_t *d_indices, float *d_dist2) {
  if (!b || (b->N > 0 && !d_points) || (b->M > 0 && !d_queries) || (b->entries > 0 && !d_indices)) return ARBORX_EINVAL;
  const cudaStream_t s = (cudaStream_t)stream;
  if (!use_graph) {
    const int st = enqueue(b, d_points, d_queries, s, d_row_offsets, d_indices, d_dist2);
    return st ? st : status_of(cudaGetLastError());
  }
  if (!b->cap) {
    if (cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      return ARBORX_ECUDA;
    }
  }
  // the graph runs on the batch's own stream, ordered after and before the caller's work
  if (cudaEventRecord(b->ev_in, s) != cudaSuccess || cudaStreamWaitEvent(b->cap, b->ev_in, 0) != cudaSuccess)
    return ARBORX_ECUDA;
  const bool same = b->exec && b->g_pts == d_points && b->g_q == d_queries && b->g_off == d_row_offsets &&
                    b->g_idx == d_indices && b->g_d2 == d_dist2;
  if (!same) {
    if (b->exec) {
      cudaGraphExecDestroy(b->exec);
      b->exec = nullptr;
    }
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return ARBORX_ECUDA;
    const int st = enqueue(b, d_points, d_queries, b->cap, d_row_offsets, d_indices, d_dist2);
    if (cudaStreamEndCapture(b->cap, &g) != cudaSuccess || !g || st) {
      cudaGetLastError();
      if (g) cudaGraphDestroy(g);
      return st ? st : ARBORX_ECUDA;
    }
    const cudaError_t e = cudaGraphInstantiate(&b->exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      cudaGetLastError();
      b->exec = nullptr;
      return ARBORX_ECUDA;
    }
    b->g_pts = d_points;
    b->g_q = d_queries;
    b->g_off = d_row_offsets;
    b->g_idx = d_indices;
    b->g_d2 = d_dist2;
  }
  if (cudaGraphLaunch(b->exec, b->cap) != cudaSuccess || cudaEventRecord(b->ev_out, b->cap) != cudaSuccess ||
      cudaStreamWaitEvent(s, b->ev_out, 0) != cudaSuccess)
    return ARBORX_ECUDA;
  return ARBORX_OK;
}

int arborx_batch_check(arborx_batch b, void *stream) {
  if (!b) return ARBORX_EINVAL;
  const cudaStream_t s = (cudaStream_t)stream;
  uint32_t bits = 0;
  if (cudaMemcpyAsync(&bits, b->err, sizeof bits, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return ARBORX_ECUDA;
  if (bits & ERR_NONFINITE) return ARBORX_EINVAL;
  if (bits & ERR_TIMEOUT) return ARBORX_ETIMEOUT;
  if (bits & (ERR_STACK | ERR_CSR)) return ARBORX_EOVERFLOW;
  return ARBORX_OK;
}

int arborx_batched(int64_t n_clouds, const int64_t *h_point_offsets, const int64_t *h_query_offsets,
                    const int32_t *h_k, const float *d_points, const float *d_queries, const arborx_opts *opts,
                    void *stream, int64_t *d_row_offsets, int32_t *d_indices, float *d_dist2, int64_t capacity) {
  arborx_batch b = nullptr;
  int st = arborx_batch_create(n_clouds, h_point_offsets, h_query_offsets, h_k, opts, stream, &b);
  if (st) return st;
  int64_t np = 0, nq = 0, entries = 0;
  st = arborx_batch_entries(b, &np, &nq, &entries);
  if (st == ARBORX_OK && (capacity < entries || (entries > 0 && !d_indices))) st = ARBORX_EINVAL;
  if (st == ARBORX_OK) st = arborx_batch_run(b, d_points, d_queries, 0, stream, d_row_offsets, d_indices, d_dist2);
  if (st == ARBORX_OK) st = arborx_batch_check(b, stream);
  const int sd = arborx_batch_destroy(b);
  return st ? st : sd;
}

int arborx_batch_destroy(arborx_batch b) {
  if (!b) return ARBORX_OK;
  if (b->cap) {
    cudaStreamSynchronize(b->cap);  // graph launches still using the memory
    cudaStreamDestroy(b->cap);
    cudaEventDestroy(b->ev_in);
    cudaEventDestroy(b->ev_out);
  }
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->mem) {
    if (b->opts.free) b->opts.free(b->mem, b->mem_bytes, (void *)b->alloc_stream, b->opts.alloc_ctx);
    else cudaFreeAsync(b->mem, b->alloc_stream);
  }
  delete b;
  return status_of(cudaGetLastError());
}

}  // extern "C"

// C ABI of the LBVH library: handles, memory, argument checks and the launch
// sequences of the build and the queries (ArborX Sec. 2.1 - 2.3).
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>

#include "../../include/arborx_b300.h"
#include "kernels.cuh"
#include "radix_sort.cuh"
#include "status.cuh"

using namespace abx;

struct arborx_bvh_s {
  int device;
  int64_t n;
  int32_t kind;
  arborx_opts opts;
  cudaStream_t stream;  // build stream (used to release memory)
  // persistent: DevMeta followed by the records
  void *persist;
  size_t persist_bytes;
  DevMeta *meta;
  float4 *rec;
  // sorted codes + permutation (keep_order)
  void *order;
  size_t order_bytes;
  // query workspace, grown on demand
  void *qws;
  size_t qws_bytes;
  // build scratch kept between arborx_rebuild calls (allocated by the first one)
  void *bscratch;
  size_t bscratch_bytes;
  // state handed from spatial count to spatial fill
  const uint32_t *qperm;
  const float *count_queries;
  int64_t count_m;
  float count_radius;
  bool count_valid;
  // queries traversed since the last arborx_stats (spatial, nearest)
  uint64_t stat_queries[2];
  // one-pass spatial: row buffers [m][bs], kept from the count call to the fill call
  int32_t *sbuf;
  size_t sbuf_bytes;
  int buf_bs;
  bool buffered_valid;
  // radius and box queries emit wholly contained subtrees from the kept leaf order
  bool emit_subtrees;
  // second stream of arborx_query_spatial_nearest (forked from and joined to the caller's stream)
  cudaStream_t side;
  cudaEvent_t ev_fork, ev_join;
};

namespace {

constexpr size_t kAlign = 256;
inline size_t align_up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

// Queries are ordered by the top 24 bits of their 30-bit Morton codes (8 bits
// per axis, 16.7M cells): the order only decides speed, and three radix
// passes instead of four give the same coherence.
constexpr int kQueryKeyBits = 24;

struct Carver {
  char *base;
  size_t off = 0;
  explicit Carver(void *b) : base((char *)b) {}
  template <typename T>
  T *take(size_t count) {
    T *p = (T *)(base + off);
    off += align_up(count * sizeof(T));
    return p;
  }
};

// Library-owned stream-ordered pool per device.  Its release threshold is
// unlimited so that memory freed by one build is reused by the next without
// being unmapped at every synchronisation (the default pool trims to zero).
constexpr int kMaxDevices = 64;
std::mutex g_pool_mu;
cudaMemPool_t g_pool[kMaxDevices] = {};

cudaMemPool_t lib_pool() {
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= kMaxDevices) return nullptr;
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (!g_pool[dev]) {
    cudaMemPoolProps props;
    std::memset(&props, 0, sizeof props);
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    uint64_t thr = ~0ull;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    g_pool[dev] = pool;
  }
  return g_pool[dev];
}

void *dev_alloc(const arborx_opts &o, size_t bytes, cudaStream_t s) {
  if (bytes == 0) bytes = kAlign;
  if (o.alloc) {
    void *q = o.alloc(bytes, (void *)s, o.alloc_ctx);
    if (q && (reinterpret_cast<uintptr_t>(q) & (kAlign - 1))) {  // the traversals read 32-byte slots
      o.free(q, bytes, (void *)s, o.alloc_ctx);
      return nullptr;
    }
    return q;
  }
  void *p = nullptr;
  cudaMemPool_t pool = lib_pool();
  const cudaError_t e = pool ? cudaMallocFromPoolAsync(&p, bytes, pool, s) : cudaMallocAsync(&p, bytes, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

void dev_free(const arborx_opts &o, void *p, size_t bytes, cudaStream_t s) {
  if (!p) return;
  if (bytes == 0) bytes = kAlign;
  if (o.free) {
    o.free(p, bytes, (void *)s, o.alloc_ctx);
    return;
  }
  cudaFreeAsync(p, s);
}

TravCfg trav_cfg(const arborx_bvh_s *h, int which) {
  TravCfg c;
  c.block = h->opts.block_size > 0 ? h->opts.block_size : 128;
  c.stack_smem = h->opts.stack_smem > 0 ? h->opts.stack_smem : 16;
  c.stats_nodes = h->opts.stats ? &h->meta->nodes[which] : nullptr;
  c.heap_from = h->opts.knn_heap_from;
  if (h->emit_subtrees && h->order && h->n > 0) {  // the kept permutation follows the widened codes
    c.leafperm = reinterpret_cast<const uint32_t *>(static_cast<const char *>(h->order) +
                                                    align_up((size_t)h->n * sizeof(uint64_t)));
    c.numbering = h->opts.build_method == ARBORX_BUILD_KARRAS ? 1 : 0;
  }
  return c;
}

NearestArgs nearest_args(const arborx_bvh_s *h, const float *queries, const uint32_t *perm, int64_t m, int k) {
  NearestArgs a{};
  a.rec = h->rec;
  a.n = (uint32_t)h->n;
  a.queries = queries;
  a.qperm = perm;
  a.m = (uint32_t)m;
  a.k = k;
  a.bound_scale = 1.0f;
  a.err = &h->meta->err;
  a.anchor = h->opts.knn_anchor;
  return a;
}

bool opts_ok(const arborx_opts &o) {
  if (o.key_bits != 30 && o.key_bits != 63) return false;
  if (o.block_size != 0 && (o.block_size < 32 || o.block_size > 256 || o.block_size % 32)) return false;
  if (o.stack_smem < 0 || o.stack_smem > 64) return false;
  if ((o.alloc == nullptr) != (o.free == nullptr)) return false;
  if (o.build_method != ARBORX_BUILD_APETREI && o.build_method != ARBORX_BUILD_KARRAS) return false;
  if (o.sorted_rows != 0 && o.sorted_rows != 1) return false;
  if (o.knn_anchor < 0 || o.knn_anchor > 3) return false;
  if (o.knn_heap_from != 0 && o.knn_heap_from != 17 && o.knn_heap_from != 33) return false;
  if (o.queries_per_warp != 0 && o.queries_per_warp != 32 && o.queries_per_warp != 64 &&
      o.queries_per_warp != 128 && o.queries_per_warp != 256)
    return false;
  return true;
}

// Sort (keys, iota) with the onesweep passes; keys already in kA, histogram
// already in ws.hist.  Returns pointers to the sorted keys / permutation.
template <typename K>
void sort_pairs(K *kA, K *kB, uint32_t *vA, uint32_t *vB, uint32_t n, const SortWs &ws, uint32_t *err,
                cudaStream_t s, K **sorted_keys, uint32_t **perm) {
  const bool inA = launch_onesweep<K>(kA, kB, vA, vB, n, ws, err, s);
  *sorted_keys = inA ? kA : kB;
  *perm = inA ? vA : vB;
}

// Build scratch: keys A/B, vals A/B, parent links (Karras, preset to -1) or range ends (Apetrei),
// the Apetrei frontier list, then the zero-initialised region (arrival counters, sort workspace).
template <typename K>
size_t build_scratch_bytes(const arborx_bvh_s *h) {
  const int64_t n = h->n;
  const int64_t n_int = n > 0 ? n - 1 : 0;
  const bool karras = h->opts.build_method == ARBORX_BUILD_KARRAS;
  const size_t ws_words = sort_ws_words<K>(n, h->opts.key_bits);
  const size_t arrival_words = karras ? (size_t)n_int : 0;
  const size_t link_words = karras ? (size_t)(2 * n - 1) : (size_t)n_int;
  const size_t front_bytes = karras ? 0 : align_up(apetrei_front_bytes((uint32_t)n));
  return 2 * align_up((size_t)n * sizeof(K)) + 2 * align_up((size_t)n * sizeof(uint32_t)) +
         align_up(link_words * sizeof(int32_t)) + front_bytes + align_up(arrival_words * sizeof(uint32_t)) +
         align_up(ws_words * sizeof(uint32_t));
}

// The build's work into the handle's records (allocated): scratch NULL takes a temporary block
// from the allocator and returns it at the end.
template <typename K>
int build_work(arborx_bvh_s *h, const float *d_prims, cudaStream_t s, void *scratch) {
  const int64_t n = h->n;
  const uint32_t un = (uint32_t)n;
  const int key_bits = h->opts.key_bits;
  const int passes = sort_passes(key_bits);
  const int64_t n_int = n > 0 ? n - 1 : 0;
  if (n == 0) {
    launch_init_meta(h->meta, s);
    // empty tree: the root record must still be readable; mark it empty by n == 0
    cudaMemsetAsync(h->rec, 0, 2 * sizeof(float4), s);
    return launch_status();
  }

  const bool karras = h->opts.build_method == ARBORX_BUILD_KARRAS;
  const size_t ws_words = sort_ws_words<K>(n, key_bits);
  const size_t arrival_words = karras ? (size_t)n_int : 0;  // Karras fit's arrival counters
  const size_t zero_bytes = align_up(arrival_words * sizeof(uint32_t)) + align_up(ws_words * sizeof(uint32_t));
  const size_t link_words = karras ? (size_t)(2 * n - 1) : (size_t)n_int;
  const size_t front_bytes = karras ? 0 : align_up(apetrei_front_bytes(un));
  const size_t scratch_bytes = build_scratch_bytes<K>(h);
  const bool own = scratch == nullptr;
  if (own) scratch = dev_alloc(h->opts, scratch_bytes, s);
  if (!scratch) {
    launch_init_meta(h->meta, s);  // the handle's error word and statistics start clean all the same
    return ARBORX_ENOMEM;
  }
  Carver c(scratch);
  K *kA = c.take<K>(n);
  K *kB = c.take<K>(n);
  uint32_t *vA = c.take<uint32_t>(n);
  uint32_t *vB = c.take<uint32_t>(n);
  int32_t *links = c.take<int32_t>(link_words);
  void *front = karras ? nullptr : static_cast<void *>(c.take<char>(front_bytes));
  char *zero_base = c.base + c.off;
  uint32_t *arrival = c.take<uint32_t>(arrival_words);
  uint32_t *wsbase = c.take<uint32_t>(ws_words);
  launch_init_meta_zero(h->meta, zero_base, zero_bytes, s);  // the tree's meta block and the zeroed scratch
  if (karras) cudaMemsetAsync(links, 0xff, link_words * sizeof(int32_t), s);  // unset links read as -1
  launch_bounds(d_prims, n, h->kind, h->meta, s);
  int st = launch_status();
  if (!st && h->opts.validate) {
    uint32_t nonfinite = 0;
    if (cudaMemcpyAsync(&nonfinite, &h->meta->nonfinite, sizeof(uint32_t), cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      st = ARBORX_ECUDA;
    else if (nonfinite)
      st = ARBORX_EINVAL;
  }
  if (st) {
    if (own) dev_free(h->opts, scratch, scratch_bytes, s);
    return st;
  }
  const SortWs ws = sort_ws_carve<K>(wsbase, n, key_bits);

  launch_morton<K>(d_prims, un, h->kind, h->meta, kA, ws.hist, passes, true, s);
  K *skeys;
  uint32_t *perm;
  sort_pairs<K>(kA, kB, vA, vB, un, ws, &h->meta->err, s, &skeys, &perm);
  if (karras) {
    launch_hierarchy<K>(skeys, un, links, s);
    launch_fit(d_prims, un, h->kind, perm, links, arrival, h->rec, &h->meta->err, s);
  } else {
    launch_apetrei<K>(d_prims, un, h->kind, skeys, perm, links, h->rec, front, &h->meta->err, s);
  }
  st = launch_status();
  if (st == ARBORX_OK && h->opts.keep_order) {
    h->order_bytes = align_up((size_t)n * sizeof(uint64_t)) + align_up((size_t)n * sizeof(uint32_t));
    if (!h->order) h->order = dev_alloc(h->opts, h->order_bytes, s);
    if (!h->order) {
      st = ARBORX_ENOMEM;
    } else {
      // keep codes widened to uint64 so the export format does not depend on key_bits
      Carver oc(h->order);
      uint64_t *codes64 = oc.take<uint64_t>(n);
      uint32_t *perm_keep = oc.take<uint32_t>(n);
      if (sizeof(K) == 8) {
        cudaMemcpyAsync(codes64, skeys, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s);
      } else {
        // widen with a strided copy: low words = codes, high words = 0
        cudaMemsetAsync(codes64, 0, n * sizeof(uint64_t), s);
        cudaMemcpy2DAsync(codes64, sizeof(uint64_t), skeys, sizeof(uint32_t), sizeof(uint32_t), n,
                          cudaMemcpyDeviceToDevice, s);
      }
      cudaMemcpyAsync(perm_keep, perm, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s);
      st = launch_status();
    }
  }
  if (own) dev_free(h->opts, scratch, scratch_bytes, s);
  return st;
}

template <typename K>
int build_impl(arborx_bvh_s *h, const float *d_prims, cudaStream_t s) {
  // persistent block: meta + records (root, reserved, 2 per internal node)
  const int64_t n_int = h->n > 0 ? h->n - 1 : 0;
  const size_t rec_floats = (size_t)(2 + 2 * n_int) * 8;
  h->persist_bytes = align_up(sizeof(DevMeta)) + align_up(rec_floats * sizeof(float));
  h->persist = dev_alloc(h->opts, h->persist_bytes, s);
  if (!h->persist) return ARBORX_ENOMEM;
  {
    Carver c(h->persist);
    h->meta = c.take<DevMeta>(1);
    h->rec = c.take<float4>(rec_floats / 4);
  }
  return build_work<K>(h, d_prims, s, nullptr);
}

void release(arborx_bvh_s *h) {
  if (!h) return;
  dev_free(h->opts, h->qws, h->qws_bytes, h->stream);
  dev_free(h->opts, h->bscratch, h->bscratch_bytes, h->stream);
  h->bscratch = nullptr;
  dev_free(h->opts, h->sbuf, h->sbuf_bytes, h->stream);
  h->sbuf = nullptr;
  dev_free(h->opts, h->order, h->order_bytes, h->stream);
  dev_free(h->opts, h->persist, h->persist_bytes, h->stream);
  h->qws = h->order = h->persist = nullptr;
  // the stream and events are released once the work queued on them is done
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  if (h->side) cudaStreamDestroy(h->side);
  h->ev_fork = h->ev_join = nullptr;
  h->side = nullptr;
}

// Query workspace: codes A/B, perm A/B, sort workspace, counts, scan tiles.
struct QueryWs {
  uint32_t *cA, *cB, *pA, *pB;
  uint32_t *sortws;
  size_t sort_words;
  int32_t *counts;
  int64_t *scan_tmp;
  uint32_t *miss;     // miss list + counter (learned bound fallback)
  uint64_t *sc_ws;    // look-back status of the fused scan and compaction; follows miss[m + 32]
  size_t sc_words;
};

// Zero the overflow counter (miss[m]) and the fused scan's look-back words in one memset: they
// are adjacent in the workspace.
void zero_ovf_and_scan(const QueryWs &q, int64_t m, cudaStream_t s) {
  char *a = reinterpret_cast<char *>(q.miss + m);
  char *b = reinterpret_cast<char *>(q.sc_ws + q.sc_words);
  cudaMemsetAsync(a, 0, (size_t)(b - a), s);
}

size_t query_ws_bytes(int64_t m, size_t *sort_words) {
  *sort_words = sort_ws_words<uint32_t>(m, kQueryKeyBits);
  return 4 * align_up((size_t)m * sizeof(uint32_t)) + align_up(*sort_words * sizeof(uint32_t)) +
         align_up((size_t)m * sizeof(int32_t)) + align_up(scan_tmp_words((uint32_t)m) * sizeof(int64_t)) +
         align_up(((size_t)m + 32) * sizeof(uint32_t)) + align_up(scan_compact_ws_words((uint32_t)m) * sizeof(uint64_t));
}

int get_query_ws(arborx_bvh_s *h, int64_t m, cudaStream_t s, QueryWs *q) {
  size_t sort_words;
  const size_t need = query_ws_bytes(m, &sort_words);
  if (need > h->qws_bytes) {
    dev_free(h->opts, h->qws, h->qws_bytes, s);
    h->qws = dev_alloc(h->opts, need, s);
    h->qws_bytes = h->qws ? need : 0;
    if (!h->qws) return ARBORX_ENOMEM;
  }
  Carver c(h->qws);
  q->cA = c.take<uint32_t>(m);
  q->cB = c.take<uint32_t>(m);
  q->pA = c.take<uint32_t>(m);
  q->pB = c.take<uint32_t>(m);
  q->sortws = c.take<uint32_t>(sort_words);
  q->sort_words = sort_words;
  q->counts = c.take<int32_t>(m);
  q->scan_tmp = c.take<int64_t>(scan_tmp_words((uint32_t)m));
  q->miss = c.take<uint32_t>(m + 32);
  q->sc_words = scan_compact_ws_words((uint32_t)m);
  q->sc_ws = c.take<uint64_t>(q->sc_words);
  return ARBORX_OK;
}

// Morton-sort the queries against the tree's scene box; returns the
// permutation (sorted position -> query index), or NULL for input order.
int order_queries(arborx_bvh_s *h, const float *d_q, int64_t m, cudaStream_t s, QueryWs &q, const uint32_t **perm,
                  const uint32_t *given = nullptr, int kind = ARBORX_POINTS) {
  *perm = given;
  if (given || !h->opts.sort_queries || m < 2 || h->n == 0) return ARBORX_OK;
  cudaMemsetAsync(q.sortws, 0, q.sort_words * sizeof(uint32_t), s);
  const SortWs ws = sort_ws_carve<uint32_t>(q.sortws, m, kQueryKeyBits);
  launch_morton<uint32_t>(d_q, (uint32_t)m, kind, h->meta, q.cA, ws.hist, ws.passes, false, s,
                          30 - kQueryKeyBits);
  uint32_t *sk, *pm;
  sort_pairs<uint32_t>(q.cA, q.cB, q.pA, q.pB, (uint32_t)m, ws, &h->meta->err, s, &sk, &pm);
  *perm = pm;
  return launch_status();
}

bool finite_radius(float r) { return !std::isnan(r) && r >= 0.0f; }

}  // namespace

namespace {

// opts.sorted_rows: put every row of the first `capacity` result entries in ascending index order
int sort_rows(arborx_bvh_s *h, const int64_t *d_offsets, int32_t *d_indices, int64_t m, int64_t capacity,
              cudaStream_t s) {
  if (!h->opts.sorted_rows || m == 0 || capacity == 0) return ARBORX_OK;
  if (capacity >= ARBORX_MAX_PRIMS) return ARBORX_EINVAL;
  const uint32_t cap = (uint32_t)capacity;
  const size_t bytes = sort_rows_bytes(cap, (uint32_t)m, (uint32_t)h->n);
  void *ws = dev_alloc(h->opts, bytes, s);
  if (!ws) return ARBORX_ENOMEM;
  launch_sort_rows(d_offsets, d_indices, (uint32_t)m, cap, (uint32_t)h->n, ws, &h->meta->err, s);
  dev_free(h->opts, ws, bytes, s);
  return ARBORX_OK;
}

}  // namespace

extern "C" {

const char *arborx_version(void) { return "arborx-b300 0.1 (sm_103a)"; }

const char *arborx_error_string(int status) {
  switch (status) {
    case ARBORX_OK: return "ok";
    case ARBORX_EINVAL: return "invalid argument";
    case ARBORX_ENOMEM: return "out of device memory";
    case ARBORX_ECUDA: return "CUDA error";
    case ARBORX_ETIMEOUT: return "bounded device wait timed out";
    case ARBORX_EOVERFLOW: return "result capacity exceeded";
    case ARBORX_ESTATE: return "call out of order";
    default: return "unknown";
  }
}

int arborx_default_opts(arborx_opts *o) {
  if (!o) return ARBORX_EINVAL;
  std::memset(o, 0, sizeof(*o));
  o->key_bits = 30;
  o->sort_queries = 1;
  o->validate = 1;
  o->keep_order = 0;
  o->block_size = 0;
  o->stack_smem = 0;
  o->build_method = ARBORX_BUILD_APETREI;
  o->stats = 0;
  o->sorted_rows = 0;
  o->knn_anchor = 3;
  o->queries_per_warp = 0;
  o->knn_heap_from = 0;
  return ARBORX_OK;
}

int arborx_build(const float *d_prims, int64_t n, int32_t kind, const arborx_opts *opts, void *stream,
                 arborx_handle *out) {
  if (!out) return ARBORX_EINVAL;
  *out = nullptr;
  if (n < 0 || n >= ARBORX_MAX_PRIMS || (kind != ARBORX_POINTS && kind != ARBORX_BOXES)) return ARBORX_EINVAL;
  if (n > 0 && !d_prims) return ARBORX_EINVAL;
  arborx_opts o;
  if (opts) o = *opts;
  else arborx_default_opts(&o);
  if (!opts_ok(o)) return ARBORX_EINVAL;
  arborx_bvh_s *h = new (std::nothrow) arborx_bvh_s();
  if (!h) return ARBORX_ENOMEM;
  cudaGetDevice(&h->device);
  h->n = n;
  h->kind = kind;
  h->opts = o;
  h->stream = (cudaStream_t)stream;
  const cudaStream_t s = (cudaStream_t)stream;
  const int st = o.key_bits == 30 ? build_impl<uint32_t>(h, d_prims, s) : build_impl<uint64_t>(h, d_prims, s);
  if (st != ARBORX_OK) {
    release(h);
    delete h;
    return st;
  }
  *out = h;
  return ARBORX_OK;
}

int arborx_rebuild(arborx_handle h, const float *d_prims, void *stream) {
  if (!h || (h->n > 0 && !d_prims)) return ARBORX_EINVAL;
  const cudaStream_t s = (cudaStream_t)stream;
  h->stream = s;
  h->count_valid = false;  // rows counted on the old tree cannot be filled from the new one
  h->buffered_valid = false;
  const bool wide = h->opts.key_bits != 30;
  const size_t need = wide ? build_scratch_bytes<uint64_t>(h) : build_scratch_bytes<uint32_t>(h);
  if (need > h->bscratch_bytes) {
    dev_free(h->opts, h->bscratch, h->bscratch_bytes, s);
    h->bscratch = dev_alloc(h->opts, need, s);
    h->bscratch_bytes = h->bscratch ? need : 0;
    if (!h->bscratch) return ARBORX_ENOMEM;
  }
  return wide ? build_work<uint64_t>(h, d_prims, s, h->bscratch) : build_work<uint32_t>(h, d_prims, s, h->bscratch);
}

int arborx_destroy(arborx_handle h) {
  if (!h) return ARBORX_OK;
  // memory is released stream-ordered on the stream of the handle's last call
  release(h);
  delete h;
  return launch_status();
}

int arborx_size(arborx_handle h, int64_t *n, int32_t *kind) {
  if (!h) return ARBORX_EINVAL;
  if (n) *n = h->n;
  if (kind) *kind = h->kind;
  return ARBORX_OK;
}

int arborx_check(arborx_handle h, void *stream) {
  if (!h) return ARBORX_EINVAL;
  const cudaStream_t s = (cudaStream_t)stream;
  uint32_t bits = 0;
  if (cudaMemcpyAsync(&bits, &h->meta->err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return ARBORX_ECUDA;
  // non-finite input is a property of the tree: keep reporting it
  const uint32_t keep = bits & ERR_NONFINITE;
  if (bits & ~keep) cudaMemcpyAsync(&h->meta->err, &keep, sizeof(uint32_t), cudaMemcpyHostToDevice, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) return ARBORX_ECUDA;
  return err_bits_to_status(bits);
}

int arborx_query_spatial_count(arborx_handle h, const float *d_queries, int64_t m, float radius,
                               const uint32_t *d_order, void *stream, int64_t *d_offsets) {
  if (!h || m < 0 || m >= ARBORX_MAX_QUERIES || !d_offsets || (m > 0 && !d_queries) || !finite_radius(radius))
    return ARBORX_EINVAL;
  const cudaStream_t s = (cudaStream_t)stream;
  h->stream = s;
  h->count_valid = false;
  QueryWs q;
  int st = get_query_ws(h, m, s, &q);
  if (st) return st;
  const uint32_t *perm;
  st = order_queries(h, d_queries, m, s, q, &perm, d_order);
  if (st) return st;
  const float r2 = radius * radius;  // one IEEE single rounding
  launch_spatial_count(h->rec, (uint32_t)h->n, d_queries, perm, (uint32_t)m, r2, q.counts, &h->meta->err,
                       trav_cfg(h, 0), s);
  h->stat_queries[0] += (uint64_t)m;
  launch_scan(q.counts, (uint32_t)m, d_offsets, q.scan_tmp, s);
  st = launch_status();
  if (st) return st;
  h->qperm = perm;
  h->count_queries = d_queries;
  h->count_m = m;
  h->count_radius = radius;
  h->count_valid = true;
  return ARBORX_OK;
}

int arborx_query_spatial_fill(arborx_handle h, const float *d_queries, int64_t m, float radius, void *stream,
                              const int64_t *d_offsets, int32_t *d_indices, int64_t capacity) {
  if (!h || m < 0 || !d_offsets || (m > 0 && !d_queries) || !finite_radius(radius) || capacity < 0 ||
      (capacity > 0 && !d_indices))
    return ARBORX_EINVAL;
  if (!h->count_valid || h->count_queries != d_queries || h->count_m != m || h->count_radius != radius)
    return ARBORX_ESTATE;
  const cudaStream_t s = (cudaStream_t)stream;
  const float r2 = radius * radius;  // one IEEE single rounding
  launch_spatial_fill(h->rec, (uint32_t)h->n, d_queries, h->qperm, (uint32_t)m, r2, d_offsets, d_indices, capacity,
                      &h->meta->err, trav_cfg(h, 0), s);
  const int st = sort_rows(h, d_offsets, d_indices, m, capacity, s);
  return st ? st : launch_status();
}

int arborx_query_spatial(arborx_handle h, const float *d_queries, int64_t m, float radius, const uint32_t *d_order,
                         void *stream, int64_t *d_offsets, int32_t **d_indices, int64_t *nnz) {
  if (!d_indices || !nnz) return ARBORX_EINVAL;
  *d_indices = nullptr;
  *nnz = 0;
  int st = arborx_query_spatial_count(h, d_queries, m, radius, d_order, stream, d_offsets);
  if (st) return st;
  const cudaStream_t s = (cudaStream_t)stream;
  int64_t total = 0;
  uint32_t bits = 0;
  if (cudaMemcpyAsync(&total, d_offsets + m, sizeof(int64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(&bits, &h->meta->err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return ARBORX_ECUDA;
  st = err_bits_to_status(bits);
  if (st) return st;
  int32_t *idx = (int32_t *)dev_alloc(h->opts, (size_t)total * sizeof(int32_t), s);
  if (!idx) return ARBORX_ENOMEM;
  st = arborx_query_spatial_fill(h, d_queries, m, radius, stream, d_offsets, idx, total);
  if (st) {
    dev_free(h->opts, idx, (size_t)total * sizeof(int32_t), s);
    return st;
  }
  *d_indices = idx;
  *nnz = total;
  return ARBORX_OK;
}

int arborx_free(arborx_handle h, void *d_ptr, size_t bytes, void *stream) {
  if (!h) return ARBORX_EINVAL;
  dev_free(h->opts, d_ptr, bytes, (cudaStream_t)stream);
  return launch_status();
}

namespace {

// The nearest query's traversal once the order is known (uses none of the query workspace).
int nearest_work(arborx_bvh_s *h, const uint32_t *perm, const float *d_queries, int64_t m, int32_t k, cudaStream_t s,
                 int64_t *d_offsets, int32_t *d_indices, float *d_dist2) {
  NearestArgs a = nearest_args(h, d_queries, perm, m, k);
  a.offsets = d_offsets;
  a.out_idx = d_indices;
  a.out_d2 = d_dist2;
  if (launch_nearest(a, trav_cfg(h, 1), s)) return ARBORX_EINVAL;
  h->stat_queries[1] += (uint64_t)m;
  return launch_status();
}

}  // namespace

int arborx_query_nearest(arborx_handle h, const float *d_queries, int64_t m, int32_t k, const uint32_t *d_order,
                         void *stream, int64_t *d_offsets, int32_t *d_indices, float *d_dist2) {
  if (!h || m < 0 || m >= ARBORX_MAX_QUERIES || k < 1 || k > ARBORX_MAX_K || (m > 0 && !d_queries))
    return ARBORX_EINVAL;
  const int64_t kk = k < h->n ? k : h->n;
  if (m > 0 && kk > 0 && !d_indices) return ARBORX_EINVAL;
  const cudaStream_t s = (cudaStream_t)stream;
  h->stream = s;
  if (m == 0 || kk == 0) {
    if (d_offsets) cudaMemsetAsync(d_offsets, 0, (size_t)(m + 1) * sizeof(int64_t), s);
    return launch_status();
  }
  QueryWs q;
  int st = get_query_ws(h, m, s, &q);
  if (st) return st;
  const uint32_t *perm;
  st = order_queries(h, d_queries, m, s, q, &perm, d_order);
  if (st) return st;
  return nearest_work(h, perm, d_queries, m, k, s, d_offsets, d_indices, d_dist2);
}

int arborx_export_tree(arborx_handle h, void *stream, float *d_records, float *d_scene, uint64_t *d_codes,
                       uint32_t *d_perm) {
  if (!h) return ARBORX_EINVAL;
  const cudaStream_t s = (cudaStream_t)stream;
  const int64_t n = h->n;
  if ((d_codes || d_perm) && !h->order && n > 0) return ARBORX_ESTATE;
  if (d_records && n > 0)
    cudaMemcpyAsync(d_records, h->rec, (size_t)(2 + 2 * (n - 1)) * 8 * sizeof(float), cudaMemcpyDeviceToDevice, s);
  if (d_scene) cudaMemcpyAsync(d_scene, h->meta->scene, 6 * sizeof(float), cudaMemcpyDeviceToDevice, s);
  if (n > 0 && h->order) {
    Carver oc(h->order);
    uint64_t *codes64 = oc.take<uint64_t>(n);
    uint32_t *perm = oc.take<uint32_t>(n);
    if (d_codes) cudaMemcpyAsync(d_codes, codes64, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s);
    if (d_perm) cudaMemcpyAsync(d_perm, perm, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s);
  }
  return launch_status();
}

int arborx_sort_pairs(void *d_keys, uint32_t *d_perm, int64_t n, int32_t key_bits, void *stream) {
  if (n < 0 || n >= ARBORX_MAX_PRIMS || key_bits < 1 || key_bits > 64 || (n > 0 && (!d_keys || !d_perm)))
    return ARBORX_EINVAL;
  if (n == 0) return ARBORX_OK;
  const cudaStream_t s = (cudaStream_t)stream;
  arborx_opts o;
  arborx_default_opts(&o);
  const bool wide = key_bits > 32;
  const size_t kb = wide ? 8 : 4;
  const size_t ws_words = wide ? sort_ws_words<uint64_t>(n, key_bits) : sort_ws_words<uint32_t>(n, key_bits);
  const size_t bytes = align_up(n * kb) + align_up(n * 4) + align_up(ws_words * 4) + align_up(4);
  void *tmp = dev_alloc(o, bytes, s);
  if (!tmp) return ARBORX_ENOMEM;
  Carver c(tmp);
  void *kB = c.take<char>(n * kb);
  uint32_t *vB = c.take<uint32_t>(n);
  uint32_t *wsb = c.take<uint32_t>(ws_words);
  uint32_t *err = c.take<uint32_t>(1);
  cudaMemsetAsync(wsb, 0, align_up(ws_words * 4) + align_up(4), s);
  bool inA;
  if (wide) {
    const SortWs ws = sort_ws_carve<uint64_t>(wsb, n, key_bits);
    launch_histogram<uint64_t>((const uint64_t *)d_keys, (uint32_t)n, ws.passes, ws.hist, s);
    inA = launch_onesweep<uint64_t>((uint64_t *)d_keys, (uint64_t *)kB, d_perm, vB, (uint32_t)n, ws, err, s);
  } else {
    const SortWs ws = sort_ws_carve<uint32_t>(wsb, n, key_bits);
    launch_histogram<uint32_t>((const uint32_t *)d_keys, (uint32_t)n, ws.passes, ws.hist, s);
    inA = launch_onesweep<uint32_t>((uint32_t *)d_keys, (uint32_t *)kB, d_perm, vB, (uint32_t)n, ws, err, s);
  }
  if (!inA) {
    cudaMemcpyAsync(d_keys, kB, n * kb, cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(d_perm, vB, n * 4, cudaMemcpyDeviceToDevice, s);
  }
  uint32_t bits = 0;
  cudaMemcpyAsync(&bits, err, 4, cudaMemcpyDeviceToHost, s);
  dev_free(o, tmp, bytes, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) return ARBORX_ECUDA;
  const int st = launch_status();
  if (st) return st;
  return err_bits_to_status(bits);
}

int arborx_selftest_bounded_wait(void *stream) {
  const cudaStream_t s = (cudaStream_t)stream;
  arborx_opts o;
  arborx_default_opts(&o);
  uint32_t *w = (uint32_t *)dev_alloc(o, 256, s);  // flag (never set) and error word
  if (!w) return ARBORX_ENOMEM;
  uint32_t bits = 0;
  cudaMemsetAsync(w, 0, 8, s);
  launch_spin_probe(w, w + 1, s);
  cudaMemcpyAsync(&bits, w + 1, sizeof bits, cudaMemcpyDeviceToHost, s);
  dev_free(o, w, 256, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) return ARBORX_ECUDA;
  const int st = launch_status();
  if (st) return st;
  return err_bits_to_status(bits);
}

int arborx_selftest_scan_wait(void *stream) {
  const cudaStream_t s = (cudaStream_t)stream;
  arborx_opts o;
  arborx_default_opts(&o);
  const uint32_t m = scan_compact_probe_queries();  // two tiles of the one-call scan
  const size_t ws_words = scan_compact_ws_words(m);
  const size_t bytes = align_up(m * sizeof(int32_t)) + align_up((m + 1) * sizeof(int64_t)) +
                       align_up(ws_words * sizeof(uint64_t)) + align_up(sizeof(uint32_t));
  void *tmp = dev_alloc(o, bytes, s);
  if (!tmp) return ARBORX_ENOMEM;
  Carver c(tmp);
  int32_t *counts = c.take<int32_t>(m);
  int64_t *offsets = c.take<int64_t>(m + 1);
  uint64_t *ws = c.take<uint64_t>(ws_words);
  uint32_t *err = c.take<uint32_t>(1);
  uint32_t bits = 0;
  cudaMemsetAsync(err, 0, sizeof(uint32_t), s);
  launch_scan_compact_wait_probe(counts, offsets, ws, err, s);
  cudaMemcpyAsync(&bits, err, sizeof bits, cudaMemcpyDeviceToHost, s);
  dev_free(o, tmp, bytes, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) return ARBORX_ECUDA;
  const int st = launch_status();
  if (st) return st;
  return err_bits_to_status(bits);
}

// ------------------------------------------------------------ learned bound

int arborx_mlp_forward(arborx_handle h, const float *d_params, const float *d_queries, int64_t m, int32_t tensor_cores,
                       void *stream, float *d_y) {
  if (!h || !d_params || m < 0 || m >= ARBORX_MAX_QUERIES || (m > 0 && (!d_queries || !d_y))) return ARBORX_EINVAL;
  const cudaStream_t s = (cudaStream_t)stream;
  if (tensor_cores) launch_mlp_bound(d_params, d_queries, (uint32_t)m, h->meta, 0.f, nullptr, d_y, &h->meta->err, s);
  else launch_mlp_forward(d_params, d_queries, (uint32_t)m, h->meta, d_y, s);
  return launch_status();
}

int arborx_mlp_grad(arborx_handle h, const float *d_params, const float *d_queries, const float *d_labels, int64_t b,
                    void *stream, float *d_grad, float *d_loss) {
  if (!h || !d_params || !d_queries || !d_labels || !d_grad || b < 1 || b > (1 << 24)) return ARBORX_EINVAL;
  const cudaStream_t s = (cudaStream_t)stream;
  const int nblocks = (int)((b + 31) / 32);
  const size_t bytes = (size_t)nblocks * (kMlpParams + 1) * sizeof(float);
  float *partial = (float *)dev_alloc(h->opts, bytes, s);
  if (!partial) return ARBORX_ENOMEM;
  if (d_loss) cudaMemsetAsync(d_loss, 0, sizeof(float), s);
  launch_mlp_grad(d_params, d_queries, d_labels, b, 0, (int)b, h->meta, partial, s);
  launch_adam(nullptr, nullptr, nullptr, partial, nblocks, 0.f, 0.f, 0.f, 0.f, 1.f, 1.f, d_grad, d_loss, 1.f, s);
  dev_free(h->opts, partial, bytes, s);
  return launch_status();
}

int arborx_mlp_train(arborx_handle h, const float *d_queries, int64_t mt, int32_t k, int32_t epochs, int32_t batch,
                     float lr, float lr_final, void *stream, float *d_params, float *d_loss) {
  if (!h || !d_queries || !d_params || mt < 1 || mt >= ARBORX_MAX_QUERIES || k < 1 || k > ARBORX_MAX_K ||
      epochs < 0 || batch < 1 || batch > (1 << 20) || !(lr >= 0.f) || !(lr_final >= 0.f) || h->n < 1)
    return ARBORX_EINVAL;
  const cudaStream_t s = (cudaStream_t)stream;
  h->stream = s;
  const int64_t kk = k < h->n ? k : h->n;
  const int b = (int)std::min<int64_t>(batch, mt);
  const int nblocks = (b + 31) / 32;
  const size_t bytes = align_up((size_t)mt * kk * sizeof(float)) + align_up((size_t)mt * kk * sizeof(int32_t)) +
                       align_up((size_t)mt * sizeof(float)) +
                       align_up((size_t)nblocks * (kMlpParams + 1) * sizeof(float)) +
                       2 * align_up((size_t)kMlpParams * sizeof(float));
  void *ws = dev_alloc(h->opts, bytes, s);
  if (!ws) return ARBORX_ENOMEM;
  Carver c(ws);
  float *d2 = c.take<float>((size_t)mt * kk);
  int32_t *idx = c.take<int32_t>((size_t)mt * kk);
  float *labels = c.take<float>(mt);
  float *partial = c.take<float>((size_t)nblocks * (kMlpParams + 1));
  float *mom = c.take<float>(kMlpParams);
  float *vel = c.take<float>(kMlpParams);
  // labels: exact k-th distances from the library's own nearest traversal
  int st = arborx_query_nearest(h, d_queries, mt, k, nullptr, stream, nullptr, idx, d2);
  if (st == ARBORX_OK) {
    launch_labels(d2, mt, (int)kk, labels, s);
    cudaMemsetAsync(mom, 0, 2 * align_up((size_t)kMlpParams * sizeof(float)), s);
    if (d_loss && epochs > 0) cudaMemsetAsync(d_loss, 0, (size_t)epochs * sizeof(float), s);
    const int64_t steps = (mt + b - 1) / b;
    const double total = (double)steps * epochs;
    const double b1 = 0.9, b2 = 0.999;
    int64_t t = 0;
    for (int e = 0; e < epochs; ++e) {
      const int64_t shift = ((int64_t)e * 7919) % mt;  // batches differ from epoch to epoch
      for (int64_t j = 0; j < steps; ++j) {
        // cosine decay from lr (first step) to lr_final (last step)
        const double frac = total > 1 ? (double)t / (total - 1) : 0.0;
        const float lr_t = (float)(lr_final + (lr - lr_final) * 0.5 * (1.0 + std::cos(3.14159265358979323846 * frac)));
        ++t;
        launch_mlp_grad(d_params, d_queries, labels, mt, (shift + j * b) % mt, b, h->meta, partial, s);
        launch_adam(d_params, mom, vel, partial, nblocks, lr_t, (float)b1, (float)b2, 1e-8f,
                    (float)(1.0 - std::pow(b1, (double)t)), (float)(1.0 - std::pow(b2, (double)t)), nullptr,
                    d_loss ? d_loss + e : nullptr, 1.0f / (float)steps, s);
      }
    }
    st = launch_status();
  }
  dev_free(h->opts, ws, bytes, s);
  return st;
}

namespace {
// Bounded nearest traversal seeded with per-query squared bounds (in `bound2`,
// by query index; may alias the workspace).  Queries that find fewer than k
// primitives inside their bound run a second, still bounded, traversal whose
// bound comes from the finished rows of their Morton neighbours (neighbour's
// k-th distance plus the distance between the two queries: a guaranteed upper
// bound); a third, unbounded pass is kept for the rare query whose neighbours
// give no usable bound.
int nearest_bounded(arborx_handle h, const float *d_queries, int64_t m, int32_t k, const float *bound2,
                    const uint32_t *perm, QueryWs &q, cudaStream_t s, int64_t *d_offsets, int32_t *d_indices,
                    float *d_dist2, int64_t *h_fallbacks) {
  uint32_t *miss = q.miss;
  uint32_t *miss_count = q.miss + m;
  uint32_t *miss2 = perm == q.pB ? q.pA : q.pB;  // free once the order exists
  uint32_t *miss2_count = q.miss + m + 1;
  const int64_t kk = k < h->n ? k : h->n;
  // the neighbour bound reads finished squared distances: keep them even if the caller does not
  float *d2 = d_dist2;
  const size_t d2_bytes = (size_t)m * kk * sizeof(float);
  if (!d2) {
    d2 = (float *)dev_alloc(h->opts, d2_bytes, s);
    if (!d2) return ARBORX_ENOMEM;
  }
  cudaMemsetAsync(miss_count, 0, 2 * sizeof(uint32_t), s);
  const TravCfg cfg = trav_cfg(h, 1);
  NearestArgs a = nearest_args(h, d_queries, perm, m, k);
  a.offsets = d_offsets;
  a.out_idx = d_indices;
  a.out_d2 = d2;
  a.init_bound2 = bound2;
  a.anchor = 0;  // the caller's bound takes its place; the unbounded last pass below uses it
  a.miss_list = miss;
  a.miss_count = miss_count;
  int st = launch_nearest(a, cfg, s) ? ARBORX_EINVAL : ARBORX_OK;
  if (st == ARBORX_OK) {
    NearestArgs b = nearest_args(h, d_queries, perm, m, k);
    b.out_idx = d_indices;
    b.out_d2 = d2;
    b.pos_list = miss;
    b.m_dev = miss_count;
    b.nbr_bound = 1;
    b.anchor = 0;
    b.miss_list = miss2;
    b.miss_count = miss2_count;
    launch_nearest(b, cfg, s);
    NearestArgs c = nearest_args(h, d_queries, perm, m, k);
    c.out_idx = d_indices;
    c.out_d2 = d2;
    c.pos_list = miss2;
    c.m_dev = miss2_count;
    launch_nearest(c, cfg, s);
    h->stat_queries[1] += (uint64_t)m;
    st = launch_status();
  }
  if (d2 != d_dist2) dev_free(h->opts, d2, d2_bytes, s);
  if (st == ARBORX_OK && h_fallbacks) {
    uint32_t cnt = 0;
    if (cudaMemcpyAsync(&cnt, miss_count, sizeof cnt, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return ARBORX_ECUDA;
    *h_fallbacks = cnt;
  }
  return st;
}
}  // namespace

int arborx_query_nearest_bounded(arborx_handle h, const float *d_queries, int64_t m, int32_t k,
                                 const float *d_bound2, const uint32_t *d_order, void *stream, int64_t *d_offsets,
                                 int32_t *d_indices, float *d_dist2, int64_t *h_fallbacks) {
  if (!h || m < 0 || m >= ARBORX_MAX_QUERIES || k < 1 || k > ARBORX_MAX_K || (m > 0 && (!d_queries || !d_bound2)))
    return ARBORX_EINVAL;
  if (h_fallbacks) *h_fallbacks = 0;
  if (h->n < k || m == 0) return arborx_query_nearest(h, d_queries, m, k, d_order, stream, d_offsets, d_indices, d_dist2);
  if (!d_indices) return ARBORX_EINVAL;
  const cudaStream_t s = (cudaStream_t)stream;
  h->stream = s;
  QueryWs q;
  int st = get_query_ws(h, m, s, &q);
  if (st) return st;
  const uint32_t *perm;
  st = order_queries(h, d_queries, m, s, q, &perm, d_order);
  if (st) return st;
  return nearest_bounded(h, d_queries, m, k, d_bound2, perm, q, s, d_offsets, d_indices, d_dist2, h_fallbacks);
}

int arborx_query_nearest_learned(arborx_handle h, const float *d_queries, int64_t m, int32_t k,
                                 const float *d_params, float margin, const uint32_t *d_order, void *stream,
                                 int64_t *d_offsets, int32_t *d_indices, float *d_dist2, int64_t *h_fallbacks) {
  if (!h || m < 0 || m >= ARBORX_MAX_QUERIES || k < 1 || k > ARBORX_MAX_K || (m > 0 && !d_queries) || !d_params ||
      std::isnan(margin))
    return ARBORX_EINVAL;
  if (h_fallbacks) *h_fallbacks = 0;
  if (h->n < k || m == 0)  // a bound cannot help when every primitive is returned
    return arborx_query_nearest(h, d_queries, m, k, d_order, stream, d_offsets, d_indices, d_dist2);
  if (!d_indices) return ARBORX_EINVAL;
  const cudaStream_t s = (cudaStream_t)stream;
  h->stream = s;
  QueryWs q;
  int st = get_query_ws(h, m, s, &q);
  if (st) return st;
  const uint32_t *perm;
  st = order_queries(h, d_queries, m, s, q, &perm, d_order);
  if (st) return st;
  // the initial bounds reuse a Morton-code buffer (free once the order exists)
  float *bound2 = reinterpret_cast<float *>(q.cA);
  launch_mlp_bound(d_params, d_queries, (uint32_t)m, h->meta, margin, bound2, nullptr, &h->meta->err, s);
  return nearest_bounded(h, d_queries, m, k, bound2, perm, q, s, d_offsets, d_indices, d_dist2, h_fallbacks);
}

int arborx_query_spatial_buffered_count(arborx_handle h, const float *d_queries, int64_t m, float radius,
                                        int32_t buffer_size, const uint32_t *d_order, void *stream,
                                        int64_t *d_offsets, int64_t *h_nnz) {
  if (!h || m < 0 || m >= ARBORX_MAX_QUERIES || !d_offsets || !h_nnz || (m > 0 && !d_queries) ||
      !finite_radius(radius) || buffer_size < 1 || buffer_size > ARBORX_MAX_BUFFER_SIZE)
    return ARBORX_EINVAL;
  const cudaStream_t s = (cudaStream_t)stream;
  h->stream = s;
  h->count_valid = false;
  h->buffered_valid = false;
  *h_nnz = 0;
  QueryWs q;
  int st = get_query_ws(h, m, s, &q);
  if (st) return st;
  const size_t need = (size_t)m * buffer_size * sizeof(int32_t);
  if (need > h->sbuf_bytes) {
    dev_free(h->opts, h->sbuf, h->sbuf_bytes, s);
    h->sbuf = (int32_t *)dev_alloc(h->opts, need, s);
    h->sbuf_bytes = h->sbuf ? need : 0;
    if (!h->sbuf) return ARBORX_ENOMEM;
  }
  const uint32_t *perm;
  st = order_queries(h, d_queries, m, s, q, &perm, d_order);
  if (st) return st;
  const float r2 = radius * radius;  // one IEEE single rounding
  uint32_t *ovf_count = q.miss + m;
  cudaMemsetAsync(ovf_count, 0, sizeof(uint32_t), s);
  launch_spatial_buffered(h->rec, (uint32_t)h->n, d_queries, perm, (uint32_t)m, r2, q.counts, h->sbuf, buffer_size,
                          q.miss, ovf_count, &h->meta->err, trav_cfg(h, 0), s);
  launch_scan(q.counts, (uint32_t)m, d_offsets, q.scan_tmp, s);
  h->stat_queries[0] += (uint64_t)m;
  int64_t total = 0;
  uint32_t bits = 0;
  if (cudaMemcpyAsync(&total, d_offsets + m, sizeof(int64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(&bits, &h->meta->err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return ARBORX_ECUDA;
  st = err_bits_to_status(bits);
  if (st) return st;
  *h_nnz = total;
  h->count_queries = d_queries;
  h->count_m = m;
  h->count_radius = radius;
  h->buf_bs = buffer_size;
  h->buffered_valid = true;
  return launch_status();
}

int arborx_query_spatial_buffered_fill(arborx_handle h, const float *d_queries, int64_t m, float radius, void *stream,
                                       const int64_t *d_offsets, int32_t *d_indices, int64_t capacity) {
  if (!h || m < 0 || !d_offsets || (m > 0 && !d_queries) || !finite_radius(radius) || capacity < 0 ||
      (capacity > 0 && !d_indices))
    return ARBORX_EINVAL;
  if (!h->buffered_valid || h->count_queries != d_queries || h->count_m != m || h->count_radius != radius)
    return ARBORX_ESTATE;
  const cudaStream_t s = (cudaStream_t)stream;
  QueryWs q;
  int st = get_query_ws(h, m, s, &q);  // same m: the same carve as the count call
  if (st) return st;
  launch_compact(h->sbuf, h->buf_bs, q.counts, d_offsets, (uint32_t)m, d_indices, capacity, &h->meta->err, s);
  // queries whose rows did not fit the buffer: second traversal straight into the CSR rows
  const float r2 = radius * radius;
  launch_spatial_fill(h->rec, (uint32_t)h->n, d_queries, q.miss, (uint32_t)m, r2, d_offsets, d_indices, capacity,
                      &h->meta->err, trav_cfg(h, 0), s, q.miss + m);
  st = sort_rows(h, d_offsets, d_indices, m, capacity, s);
  return st ? st : launch_status();
}

namespace {

// The one-call one-pass spatial query after the row buffer is sized and the order known.
int spatial_buffered_work(arborx_bvh_s *h, const QueryWs &q, const uint32_t *perm, const float *d_queries, int64_t m,
                          float radius, int32_t buffer_size, cudaStream_t s, int64_t *d_offsets, int32_t *d_indices,
                          int64_t capacity) {
  const float r2 = radius * radius;  // one IEEE single rounding
  uint32_t *ovf_count = q.miss + m;
  zero_ovf_and_scan(q, m, s);
  launch_spatial_buffered(h->rec, (uint32_t)h->n, d_queries, perm, (uint32_t)m, r2, q.counts, h->sbuf, buffer_size,
                          q.miss, ovf_count, &h->meta->err, trav_cfg(h, 0), s);
  launch_scan_compact(q.counts, (uint32_t)m, h->sbuf, buffer_size, d_offsets, d_indices, capacity, q.sc_ws,
                      &h->meta->err, s);
  launch_spatial_fill(h->rec, (uint32_t)h->n, d_queries, q.miss, (uint32_t)m, r2, d_offsets, d_indices, capacity,
                      &h->meta->err, trav_cfg(h, 0), s, ovf_count);
  h->stat_queries[0] += (uint64_t)m;
  const int st = sort_rows(h, d_offsets, d_indices, m, capacity, s);
  return st ? st : launch_status();
}

// Grow the handle's one-pass row buffer to m rows of buffer_size slots.
int size_row_buffer(arborx_bvh_s *h, int64_t m, int32_t buffer_size, cudaStream_t s) {
  const size_t need = (size_t)m * buffer_size * sizeof(int32_t);
  if (need > h->sbuf_bytes) {
    dev_free(h->opts, h->sbuf, h->sbuf_bytes, s);
    h->sbuf = (int32_t *)dev_alloc(h->opts, need, s);
    h->sbuf_bytes = h->sbuf ? need : 0;
    if (!h->sbuf) return ARBORX_ENOMEM;
  }
  return ARBORX_OK;
}

}  // namespace

int arborx_query_spatial_buffered(arborx_handle h, const float *d_queries, int64_t m, float radius,
                                  int32_t buffer_size, const uint32_t *d_order, void *stream, int64_t *d_offsets,
                                  int32_t *d_indices, int64_t capacity) {
  if (!h || m < 0 || m >= ARBORX_MAX_QUERIES || !d_offsets || (m > 0 && !d_queries) || !finite_radius(radius) ||
      buffer_size < 1 || buffer_size > ARBORX_MAX_BUFFER_SIZE || capacity < 0 || (capacity > 0 && !d_indices))
    return ARBORX_EINVAL;
  const cudaStream_t s = (cudaStream_t)stream;
  h->stream = s;
  h->count_valid = false;
  h->buffered_valid = false;
  QueryWs q;
  int st = get_query_ws(h, m, s, &q);
  if (st) return st;
  st = size_row_buffer(h, m, buffer_size, s);
  if (st) return st;
  const uint32_t *perm;
  st = order_queries(h, d_queries, m, s, q, &perm, d_order);
  if (st) return st;
  return spatial_buffered_work(h, q, perm, d_queries, m, radius, buffer_size, s, d_offsets, d_indices, capacity);
}

int arborx_query_spatial_nearest(arborx_handle h, const float *d_queries, int64_t m, float radius,
                                 int32_t buffer_size, int32_t k, const uint32_t *d_order, void *stream,
                                 int64_t *d_offsets, int32_t *d_indices, int64_t capacity, int64_t *d_nn_offsets,
                                 int32_t *d_nn_indices, float *d_nn_dist2) {
  if (!h || m < 0 || m >= ARBORX_MAX_QUERIES || !d_offsets || (m > 0 && !d_queries) || !finite_radius(radius) ||
      buffer_size < 1 || buffer_size > ARBORX_MAX_BUFFER_SIZE || capacity < 0 || (capacity > 0 && !d_indices) ||
      k < 1 || k > ARBORX_MAX_K)
    return ARBORX_EINVAL;
  const int64_t kk = k < h->n ? k : h->n;
  if (m > 0 && kk > 0 && !d_nn_indices) return ARBORX_EINVAL;
  const cudaStream_t s = (cudaStream_t)stream;
  h->stream = s;
  h->count_valid = false;
  h->buffered_valid = false;
  QueryWs q;
  int st = get_query_ws(h, m, s, &q);
  if (st) return st;
  st = size_row_buffer(h, m, buffer_size, s);
  if (st) return st;
  const uint32_t *perm;
  st = order_queries(h, d_queries, m, s, q, &perm, d_order);
  if (st) return st;
  if (m == 0 || kk == 0) {  // nothing to traverse for the nearest query
    if (d_nn_offsets) cudaMemsetAsync(d_nn_offsets, 0, (size_t)(m + 1) * sizeof(int64_t), s);
    return spatial_buffered_work(h, q, perm, d_queries, m, radius, buffer_size, s, d_offsets, d_indices, capacity);
  }
  if (!h->side) {  // first such call on the handle: its second stream and the two events
    cudaStream_t side = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&e0, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&e1, cudaEventDisableTiming) != cudaSuccess) {
      if (e0) cudaEventDestroy(e0);
      if (side) cudaStreamDestroy(side);
      cudaGetLastError();
      return ARBORX_ECUDA;
    }
    h->side = side;
    h->ev_fork = e0;
    h->ev_join = e1;
  }
  // fork: the nearest traversal on the handle's second stream, the spatial query on `stream`
  if (cudaEventRecord(h->ev_fork, s) != cudaSuccess || cudaStreamWaitEvent(h->side, h->ev_fork, 0) != cudaSuccess)
    return ARBORX_ECUDA;
  const int st_nn = nearest_work(h, perm, d_queries, m, k, h->side, d_nn_offsets, d_nn_indices, d_nn_dist2);
  const int st_sp =
      spatial_buffered_work(h, q, perm, d_queries, m, radius, buffer_size, s, d_offsets, d_indices, capacity);
  // join: `stream` waits for the nearest traversal, so later work on it sees both results
  if (cudaEventRecord(h->ev_join, h->side) != cudaSuccess || cudaStreamWaitEvent(s, h->ev_join, 0) != cudaSuccess)
    return ARBORX_ECUDA;
  return st_nn ? st_nn : st_sp;
}

namespace {

int query_order(arborx_handle h, const float *d_queries, int64_t m, int kind, void *stream, uint32_t *d_order) {
  if (!h || m < 0 || m >= ARBORX_MAX_QUERIES || (m > 0 && (!d_queries || !d_order))) return ARBORX_EINVAL;
  if (m == 0) return ARBORX_OK;
  const cudaStream_t s = (cudaStream_t)stream;
  h->stream = s;
  QueryWs q;
  int st = get_query_ws(h, m, s, &q);
  if (st) return st;
  const uint32_t *perm = nullptr;
  if (h->n > 0 && m > 1) {
    cudaMemsetAsync(q.sortws, 0, q.sort_words * sizeof(uint32_t), s);
    const SortWs ws = sort_ws_carve<uint32_t>(q.sortws, m, kQueryKeyBits);
    launch_morton<uint32_t>(d_queries, (uint32_t)m, kind, h->meta, q.cA, ws.hist, ws.passes, false, s,
                            30 - kQueryKeyBits);
    uint32_t *sk, *pm;
    sort_pairs<uint32_t>(q.cA, q.cB, q.pA, q.pB, (uint32_t)m, ws, &h->meta->err, s, &sk, &pm);
    perm = pm;
  }
  if (perm) {
    cudaMemcpyAsync(d_order, perm, (size_t)m * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s);
  } else {
    launch_iota(d_order, (uint32_t)m, s);
  }
  return launch_status();
}

}  // namespace

int arborx_query_order(arborx_handle h, const float *d_queries, int64_t m, void *stream, uint32_t *d_order) {
  return query_order(h, d_queries, m, ARBORX_POINTS, stream, d_order);
}

int arborx_query_order_boxes(arborx_handle h, const float *d_boxes, int64_t m, void *stream, uint32_t *d_order) {
  return query_order(h, d_boxes, m, ARBORX_BOXES, stream, d_order);
}

int arborx_order(const float *d_prims, int64_t m, int32_t kind, const arborx_opts *opts, void *stream,
                 uint32_t *d_order) {
  if (m < 0 || m >= ARBORX_MAX_QUERIES || (kind != ARBORX_POINTS && kind != ARBORX_BOXES) ||
      (m > 0 && (!d_prims || !d_order)))
    return ARBORX_EINVAL;
  arborx_opts o;
  if (opts) o = *opts;
  else arborx_default_opts(&o);
  if (!opts_ok(o)) return ARBORX_EINVAL;
  if (m == 0) return ARBORX_OK;
  const cudaStream_t s = (cudaStream_t)stream;
  if (m == 1) {
    launch_iota(d_order, 1u, s);
    return launch_status();
  }
  const uint32_t um = (uint32_t)m;
  const size_t ws_words = sort_ws_words<uint32_t>(m, kQueryKeyBits);
  const size_t bytes = align_up(sizeof(DevMeta)) + 3 * align_up((size_t)m * sizeof(uint32_t)) +
                       align_up(ws_words * sizeof(uint32_t));
  void *tmp = dev_alloc(o, bytes, s);
  if (!tmp) return ARBORX_ENOMEM;
  Carver c(tmp);
  DevMeta *meta = c.take<DevMeta>(1);
  uint32_t *cA = c.take<uint32_t>(m), *cB = c.take<uint32_t>(m), *pB = c.take<uint32_t>(m);
  uint32_t *wsb = c.take<uint32_t>(ws_words);
  // the box of the set itself (finite coordinates only), its Morton codes, then the stable sort
  launch_init_meta(meta, s);
  launch_bounds(d_prims, m, kind, meta, s);
  cudaMemsetAsync(wsb, 0, ws_words * sizeof(uint32_t), s);
  const SortWs ws = sort_ws_carve<uint32_t>(wsb, m, kQueryKeyBits);
  launch_morton<uint32_t>(d_prims, um, kind, meta, cA, ws.hist, ws.passes, false, s, 30 - kQueryKeyBits);
  uint32_t *sk, *pm;
  sort_pairs<uint32_t>(cA, cB, d_order, pB, um, ws, &meta->err, s, &sk, &pm);
  if (pm != d_order) cudaMemcpyAsync(d_order, pm, (size_t)m * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s);
  launch_iota_on_timeout(d_order, um, &meta->err, s);
  dev_free(o, tmp, bytes, s);
  return launch_status();
}

int arborx_query_intersects(arborx_handle h, const float *d_boxes, int64_t m, int32_t buffer_size,
                            const uint32_t *d_order, void *stream, int64_t *d_offsets, int32_t *d_indices,
                            int64_t capacity) {
  if (!h || m < 0 || m >= ARBORX_MAX_QUERIES || !d_offsets || (m > 0 && !d_boxes) || buffer_size < 1 ||
      buffer_size > ARBORX_MAX_BUFFER_SIZE || capacity < 0 || (capacity > 0 && !d_indices))
    return ARBORX_EINVAL;
  const cudaStream_t s = (cudaStream_t)stream;
  h->stream = s;
  h->count_valid = false;
  h->buffered_valid = false;
  QueryWs q;
  int st = get_query_ws(h, m, s, &q);
  if (st) return st;
  const size_t need = (size_t)m * buffer_size * sizeof(int32_t);
  if (need > h->sbuf_bytes) {
    dev_free(h->opts, h->sbuf, h->sbuf_bytes, s);
    h->sbuf = (int32_t *)dev_alloc(h->opts, need, s);
    h->sbuf_bytes = h->sbuf ? need : 0;
    if (!h->sbuf) return ARBORX_ENOMEM;
  }
  const uint32_t *perm;
  st = order_queries(h, d_boxes, m, s, q, &perm, d_order, ARBORX_BOXES);
  if (st) return st;
  uint32_t *ovf_count = q.miss + m;
  zero_ovf_and_scan(q, m, s);
  const TravCfg cfg = trav_cfg(h, 0);
  launch_spatial_buffered(h->rec, (uint32_t)h->n, d_boxes, perm, (uint32_t)m, 0.0f, q.counts, h->sbuf, buffer_size,
                          q.miss, ovf_count, &h->meta->err, cfg, s, true);
  launch_scan_compact(q.counts, (uint32_t)m, h->sbuf, buffer_size, d_offsets, d_indices, capacity, q.sc_ws,
                      &h->meta->err, s);
  launch_spatial_fill(h->rec, (uint32_t)h->n, d_boxes, q.miss, (uint32_t)m, 0.0f, d_offsets, d_indices, capacity,
                      &h->meta->err, cfg, s, ovf_count, true);
  h->stat_queries[0] += (uint64_t)m;
  st = sort_rows(h, d_offsets, d_indices, m, capacity, s);
  return st ? st : launch_status();
}

int arborx_set_query_option(arborx_handle h, int32_t option, int64_t value) {
  if (!h) return ARBORX_EINVAL;
  if (option == ARBORX_QOPT_EMIT_SUBTREES) {
    if (value != 0 && value != 1) return ARBORX_EINVAL;
    if (value == 1 && !h->opts.keep_order) return ARBORX_ESTATE;
    h->emit_subtrees = value == 1;
    return ARBORX_OK;
  }
  return ARBORX_EINVAL;
}

int arborx_stats(arborx_handle h, void *stream, uint64_t out[4]) {
  if (!h || !out) return ARBORX_EINVAL;
  const cudaStream_t s = (cudaStream_t)stream;
  unsigned long long nodes[2] = {0, 0};
  if (cudaMemcpyAsync(nodes, h->meta->nodes, sizeof nodes, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return ARBORX_ECUDA;
  cudaMemsetAsync(h->meta->nodes, 0, sizeof nodes, s);
  out[0] = nodes[0];
  out[1] = nodes[1];
  out[2] = h->stat_queries[0];
  out[3] = h->stat_queries[1];
  h->stat_queries[0] = h->stat_queries[1] = 0;
  return cudaStreamSynchronize(s) == cudaSuccess ? ARBORX_OK : ARBORX_ECUDA;
}

int arborx_release_cached_memory(void) {
  std::lock_guard<std::mutex> lk(g_pool_mu);
  for (int d = 0; d < kMaxDevices; ++d)
    if (g_pool[d]) cudaMemPoolTrimTo(g_pool[d], 0);
  return launch_status();
}

}  // extern "C"

// Launchers of the LBVH kernels (internal to the library).
#pragma once

#include "common.cuh"

namespace abx {

// ---- construction (build.cu)
void launch_init_meta(DevMeta *meta, cudaStream_t s);
// launch_init_meta and a zero fill of `bytes` (a multiple of 16) at the 16-byte aligned `zero`
void launch_init_meta_zero(DevMeta *meta, void *zero, size_t bytes, cudaStream_t s);
void launch_bounds(const float *prims, int64_t n, int kind, DevMeta *meta, cudaStream_t s);
template <typename K>
void launch_morton(const float *prims, uint32_t n, int kind, DevMeta *meta, K *codes, uint32_t *hist, int passes,
                   bool write_scene, cudaStream_t s, int drop = 0);
template <typename K>
void launch_hierarchy(const K *codes, uint32_t n, int32_t *parent, cudaStream_t s);
// bytes of the frontier list of launch_apetrei for n leaves
size_t apetrei_front_bytes(uint32_t n);
// other: n - 1 words, no initialisation needed; front_ws: apetrei_front_bytes(n)
template <typename K>
void launch_apetrei(const float *prims, uint32_t n, int kind, const K *codes, const uint32_t *perm, int32_t *other,
                    float4 *rec, void *front_ws, uint32_t *err, cudaStream_t s);
// batched clouds (cloud c owns entries [off[c], off[c+1]))
void launch_seg_bounds(const float *pts, const uint32_t *off, uint32_t n_clouds, float *seg_scene, uint32_t *err,
                       cudaStream_t s);
void launch_seg_morton(const float *pts, uint32_t count, const uint32_t *off, uint32_t n_clouds, const uint32_t *cmap,
                       const float *seg_scene, uint64_t *keys, uint32_t *hist, int passes, cudaStream_t s);
// root record slot of every cloud in the tree over (cloud, code) keys (-1 for an empty cloud)
void launch_seg_roots(const uint64_t *codes, uint32_t n, const uint32_t *sorted_off, uint32_t n_clouds,
                      int32_t *root_slot, cudaStream_t s);
void launch_fit(const float *prims, uint32_t n, int kind, const uint32_t *perm, const int32_t *parent,
                uint32_t *arrival, float4 *rec, uint32_t *err, cudaStream_t s);

// ---- traversal (traverse.cu)
struct TravCfg {
  int block;                       // threads per block
  int stack_smem;                  // stack entries per thread kept in shared memory
  unsigned long long *stats_nodes; // nullable: add the internal nodes loaded here
  int heap_from = 17;              // nearest: k from which the shared-memory heap replaces the register list
  const uint32_t *leafperm = nullptr;  // spatial: emit contained subtrees from this sorted leaf order
  int numbering = 0;                   // 0: internal node p splits leaves p | p+1 (Apetrei); 1: Karras ids
};

void launch_iota(uint32_t *out, uint32_t m, cudaStream_t s);
// out[i] = i for i < m, only when *err holds ERR_TIMEOUT (a sort of the order gave up)
void launch_iota_on_timeout(uint32_t *order, uint32_t m, const uint32_t *err, cudaStream_t s);

struct SpatialArgs {
  const float4 *rec;
  uint32_t n;
  const float *queries;
  const uint32_t *qperm;  // nullable: input order
  uint32_t m;
  float r2;
  int32_t *counts;
  const int64_t *offsets;
  int32_t *indices;
  int64_t capacity;
  int32_t *buf;  // 1P row buffers [m][bs]
  int bs;
  int buf_vec4;  // 1: bs a multiple of 4 and buf 16-byte aligned: hits go out in 16-byte stores
  uint32_t *ovf_list;  // 1P queries with more than bs results
  uint32_t *ovf_count;
  const uint32_t *m_dev;  // nullable: device-side query count
  uint32_t *err;
  int stack_smem;
  unsigned long long *stats;
  const uint32_t *leafperm;  // non-null only in the subtree-emitting kernels
  int numbering;
};

// Spatial predicates: box = false, queries are points float[m][3] matched within r2; box = true,
// queries are boxes float[m][6] (lo.xyz, hi.xyz) matched by closed-interval overlap (r2 unused).
// counts[j] (j in original query order) = number of matching primitives
void launch_spatial_count(const float4 *rec, uint32_t n, const float *queries, const uint32_t *qperm, uint32_t m,
                          float r2, int32_t *counts, uint32_t *err, const TravCfg &cfg, cudaStream_t s,
                          bool box = false);
// fill rows at offsets[j]; m_dev (nullable) bounds the number of queries on the device
void launch_spatial_fill(const float4 *rec, uint32_t n, const float *queries, const uint32_t *qperm, uint32_t m,
                         float r2, const int64_t *offsets, int32_t *indices, int64_t capacity, uint32_t *err,
                         const TravCfg &cfg, cudaStream_t s, const uint32_t *m_dev = nullptr, bool box = false);
// one pass: counts + the first bs results of each query in buf; overflowing queries listed
void launch_spatial_buffered(const float4 *rec, uint32_t n, const float *queries, const uint32_t *qperm, uint32_t m,
                             float r2, int32_t *counts, int32_t *buf, int bs, uint32_t *ovf_list, uint32_t *ovf_count,
                             uint32_t *err, const TravCfg &cfg, cudaStream_t s, bool box = false);
void launch_compact(const int32_t *buf, int bs, const int32_t *counts, const int64_t *offsets, uint32_t m,
                    int32_t *indices, int64_t capacity, uint32_t *err, cudaStream_t s);
// one-pass rows -> CSR in one kernel: exclusive scan of counts[m] into offsets[m+1] and the rows
// of at most bs results copied from buf; ws: scan_compact_ws_words(m) uint64 words, all zero
size_t scan_compact_ws_words(uint32_t m);
void launch_scan_compact(const int32_t *counts, uint32_t m, const int32_t *buf, int bs, int64_t *offsets,
                         int32_t *indices, int64_t capacity, uint64_t *ws, uint32_t *err, cudaStream_t s);
// the one-call scan's look-back wait on a predecessor that never publishes (self-test), over
// p = scan_compact_probe_queries() queries (two tiles): counts of p words, offsets of p + 1, ws of
// scan_compact_ws_words(p) words, *err zero
uint32_t scan_compact_probe_queries();
void launch_scan_compact_wait_probe(int32_t *counts, int64_t *offsets, uint64_t *ws, uint32_t *err, cudaStream_t s);
// exclusive scan counts[m] -> offsets[m+1]; tmp holds scan_tmp_words(m) int64
size_t scan_tmp_words(uint32_t m);
void launch_scan(const int32_t *counts, uint32_t m, int64_t *offsets, int64_t *tmp, cudaStream_t s);

// ---- row order (rows.cu): sort every CSR row of the first cap entries ascending (total read from
// offsets[m] on the device); ws: sort_rows_bytes(cap, m, n_prims) bytes, 256-byte aligned
size_t sort_rows_bytes(uint32_t cap, uint32_t m, uint32_t n_prims);
void launch_sort_rows(const int64_t *offsets, int32_t *indices, uint32_t m, uint32_t cap, uint32_t n_prims,
                      void *ws, uint32_t *err, cudaStream_t s);

// nearest: rows of kk = min(k, n) (index, d2) in (d2, index) order.
struct NearestArgs {
  const float4 *rec;
  uint32_t n;
  const float *queries;
  const uint32_t *qperm;     // sorted position -> query index (nullable: identity)
  const uint32_t *pos_list;  // nullable: thread -> sorted position (second passes)
  uint32_t m;                // number of queries (sorted positions 0..m-1)
  const uint32_t *m_dev;     // nullable: number of threads to run, produced on the device
  int k;
  int kk;                    // set by launch_nearest
  int64_t *offsets;          // nullable: offsets[t] = t * kk
  int32_t *out_idx;
  float *out_d2;             // nullable unless nbr_bound
  const float *init_bound2;  // nullable: initial k-th squared distance by query index, times bound_scale
  float bound_scale;
  int nbr_bound;             // also bound by the finished rows of the sorted neighbours (needs out_d2)
  uint32_t *miss_list;       // nullable: sorted positions of queries with fewer than k hits in their bound
  uint32_t *miss_count;
  uint32_t *err;
  int stack_smem;            // set by launch_nearest
  unsigned long long *stats; // set by launch_nearest
  int anchor;                // 0, or the form (1 to 3) of the tree's own k-th-distance bound
  int out_pairs;             // set by launch_nearest: both outputs 8-byte aligned (rows in pair stores)
};
int launch_nearest(NearestArgs a, const TravCfg &cfg, cudaStream_t s);

// batched clouds: k-nearest for sorted query positions [pos_begin, pos_end), all with k <= kc
struct BatchQueryArgs {
  const float4 *rec;
  uint32_t n;
  const float *queries;
  const uint32_t *qperm;    // sorted position -> query index
  const uint64_t *qkeys;    // sorted query keys, internal cloud id in bits 30 and up
  uint32_t pos_begin, pos_end;
  uint32_t *queue;          // work counter, zero at launch
  const int32_t *root_slot; // per internal cloud: record slot of its subtree (-1: empty cloud)
  const int32_t *kof;       // per internal cloud: k
  const uint32_t *ncount;   // per internal cloud: number of points
  const uint32_t *prim_base;// per internal cloud: index of its first point in the concatenation
  const int64_t *row_off;   // per query: first output entry
  int32_t *out_idx;
  float *out_d2;            // nullable
  uint32_t *err;
  int stack_smem;
  int anchor;                // 0, or the form (1 to 3) of the tree's own k-th-distance bound
  int queries_per_warp;      // sorted positions a warp takes per queue fetch (multiple of 32)
};
int launch_batch_nearest(const BatchQueryArgs &a, int kc, const TravCfg &cfg, cudaStream_t s);

// ---- learned k-th-distance regressor (mlp.cu)
constexpr int kMlpParams = 4481;  // W1 64x3, b1 64, W2 64x64, b2 64, w3 64, b3 1
size_t mlp_grad_smem_bytes();
void launch_mlp_grad(const float *params, const float *queries, const float *labels, int64_t mt, int64_t start, int b,
                     const DevMeta *meta, float *partial, cudaStream_t s);
void launch_adam(float *params, float *mom, float *vel, const float *partial, int nblocks, float lr, float b1, float b2,
                 float eps, float c1, float c2, float *grad_out, float *loss_out, float loss_scale, cudaStream_t s);
void launch_labels(const float *d2, int64_t mt, int kk, float *labels, cudaStream_t s);
void launch_mlp_forward(const float *params, const float *queries, uint32_t m, const DevMeta *meta, float *y,
                        cudaStream_t s);
void launch_mlp_bound(const float *params, const float *queries, uint32_t m, const DevMeta *meta, float margin,
                      float *bound2, float *y_out, uint32_t *err, cudaStream_t s);

}  // namespace abx

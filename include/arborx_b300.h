/*
 * arborx_b300.h -- C ABI of a B300 (sm_103a) linear-BVH geometric search
 * library following ArborX (Lebrun-Grandie, Prokopenko, Turcksin, Slattery,
 * arXiv 1908.11807).
 *
 * Every call takes plain pointers and sizes.  Unless stated otherwise:
 *   - pointers named d_* are DEVICE memory of the current CUDA device, owned by
 *     the caller and only read (inputs) or written (outputs) during the call's
 *     stream-ordered work;
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream); all device work is enqueued on it, and calls return before it
 *     finishes unless they say they synchronise;
 *   - coordinates are float32, 3 per point (x, y, z) or 6 per box
 *     (lo.x, lo.y, lo.z, hi.x, hi.y, hi.z), rows packed back to back;
 *   - the return value is an arborx_status code; no call throws, aborts or
 *     prints.  On a non-zero return no output is guaranteed and, for
 *     arborx_build, no handle is created.
 *
 * Results are exact: a spatial query returns exactly the primitives whose box
 * is within distance r of the query point, d^2 <= fl32(r*r) with
 * d^2 = ((gx*gx) + (gy*gy)) + (gz*gz) evaluated in FP32 round-to-nearest
 * without fused multiply-add (g = per-axis gap between point and box); a
 * nearest query returns the min(k, n) primitives first in (d^2, index) order.
 * A query with a non-finite coordinate has no neighbours.
 */
#ifndef ARBORX_B300_H
#define ARBORX_B300_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define ARBORX_API __attribute__((visibility("default")))
#else
#define ARBORX_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
typedef enum {
  ARBORX_OK = 0,
  ARBORX_EINVAL = 1,    /* bad argument: NULL pointer, size out of range, r < 0 or NaN, k < 1,
                           non-finite primitive coordinate (found by the scene-box reduction) */
  ARBORX_ENOMEM = 2,    /* a device allocation failed */
  ARBORX_ECUDA = 3,     /* a CUDA runtime call or kernel launch failed */
  ARBORX_ETIMEOUT = 4,  /* a bounded inter-block wait (radix-sort look-back) gave up;
                           results of that call are invalid, the context stays usable */
  ARBORX_EOVERFLOW = 5, /* a result would not fit: traversal stack or CSR capacity exceeded */
  ARBORX_ESTATE = 6     /* call out of order (e.g. spatial fill without a matching count) */
} arborx_status;

/* primitive kinds */
#define ARBORX_POINTS 0 /* d_prims is float[n][3] */
#define ARBORX_BOXES 1  /* d_prims is float[n][6] = lo.xyz, hi.xyz (lo <= hi per axis) */

/* hierarchy construction (arborx_opts.build_method) */
#define ARBORX_BUILD_APETREI 0 /* one bottom-up pass for hierarchy and boxes (Apetrei 2014) */
#define ARBORX_BUILD_KARRAS 1  /* top-down split search per internal node (Karras 2012), then the box fit */

/* limits */
#define ARBORX_MAX_PRIMS ((int64_t)1 << 30) /* n must be < this */
#define ARBORX_MAX_QUERIES ((int64_t)1 << 30) /* m must be < this */
#define ARBORX_MAX_K 512

/* Tree record layout, as exported by arborx_export_tree: float32 [2 + 2(n-1)][8].
 * A record is (lo.x, lo.y, lo.z, enc, hi.x, hi.y, hi.z, aux), 32 bytes, with enc
 * the bit pattern of an int32: enc >= 0 names internal node enc, enc < 0 a leaf
 * holding primitive ~enc.  Record 0 describes the root (its box is the scene
 * box); record 1 is reserved; the two children of internal node p are records
 * 2 + 2p (left) and 3 + 2p (right), adjacent, so one 64-byte load tests both.
 * Leaves are not stored separately: a child record of a leaf is its primitive's
 * box.  aux is the bit pattern of an int32: the number of leaves under the
 * record (1 for a leaf; record 0 holds n). */
#define ARBORX_RECORD_FLOATS 8

/* Caller-supplied device allocator (e.g. a framework's caching allocator).
 * alloc returns device memory of at least `bytes` bytes usable on `stream`,
 * aligned to 256 bytes (as cudaMalloc and the torch caching allocator return it),
 * or NULL on failure; free releases it (stream-ordered).  A block that is not
 * 256-byte aligned is released again and the call fails with ARBORX_ENOMEM. */
typedef void *(*arborx_alloc_fn)(size_t bytes, void *stream, void *ctx);
typedef void (*arborx_free_fn)(void *ptr, size_t bytes, void *stream, void *ctx);

typedef struct arborx_opts {
  int32_t key_bits;     /* Morton code length: 30 (default, 10 bits per axis) or 63 (21 bits per axis) */
  int32_t sort_queries; /* 1 (default): traverse queries in Morton order (Sec. 2.2, "Query ordering");
                           0: in input order.  Results are the same either way. */
  int32_t validate;     /* 1 (default): arborx_build synchronises once after the scene-box reduction and
                           returns ARBORX_EINVAL on a non-finite coordinate; 0: fully asynchronous, the
                           error is reported by arborx_check instead */
  int32_t keep_order;   /* 1: keep the sorted Morton codes and the leaf permutation (for arborx_export_tree
                           and for ARBORX_QOPT_EMIT_SUBTREES);
                           0 (default): freed at the end of the build */
  int32_t block_size;   /* traversal threads per block: 0 = default (128); 32..256, multiple of 32 */
  int32_t stack_smem;   /* per-thread traversal-stack entries held in shared memory (0 = default 16);
                           deeper entries spill to local memory, never dropped */
  int32_t build_method; /* ARBORX_BUILD_APETREI (default) or ARBORX_BUILD_KARRAS; both build the same binary
                           radix tree (node numbering differs) */
  int32_t stats;        /* 1: count the internal nodes each traversal loads (read with arborx_stats) */
  int32_t sorted_rows;  /* 1: every row of a spatial or box query lists its primitives in ascending index
                           order (two stable radix sorts over the result entries; results up to
                           ARBORX_MAX_PRIMS entries, else ARBORX_EINVAL); 0 (default): traversal order.
                           The paper leaves row order open (rows are sets). */
  int32_t knn_anchor;   /* a nearest query with no caller-supplied bound starts its traversal from an
                           exact bound on the k-th distance taken from the tree: the farthest-corner
                           distance of a subtree box of at least k leaves near the query (that box
                           holds k primitives), so candidates and stack entries beyond it are never
                           inserted or kept.  3 (default): the bound is gathered on the traversal's own
                           first closest-first descent (the smallest corner distance of the children of
                           k leaves met there), and the siblings pushed before it was known and lying
                           beyond it are then dropped from the stack (cube 1e7, 1e6 queries, k = 4:
                           0.558 ms against 0.597 / 0.614 for forms 2 / 1 and 0.747 unbounded; k = 10:
                           0.993 against 0.998 / 0.996 and 1.125).  It serves k up to 10; wider register
                           lists and the heap run form 2 in its place.  2: a walk from the root through
                           the child holding the query, bound from the last box of k leaves on it (the
                           64-Gaussian mixture, k = 16: 1.618 against 1.845 for form 1); 1: a walk
                           through the child with the nearer farthest corner, keeping the smallest seen;
                           0: the traversal starts unbounded, as in Sec. 2.2.2.  The tuner picks the
                           form per workload.  Results are identical in every case. */
  int32_t queries_per_warp; /* batched nearest queries (arborx_batch_*): sorted query positions a
                           persistent warp takes from the work queue per fetch, its lanes serving 32 at
                           a time (0 = default 32; else 32, 64, 128 or 256).  The single-tree
                           traversals serve one query per thread and ignore it. */
  int32_t knn_heap_from; /* nearest queries with k at least this keep their candidates in a shared-memory
                           heap, smaller k in a sorted register list (0 = default 17; 17 or 33).  A
                           single tree over many points is faster with the heap from 17 (k = 32 at 1e7
                           points: 3.41 against 4.32 ms), a batch of small clouds with lists up to 32
                           (the 512-cloud workload: 20.0 against 21.7 ms).  Results are identical. */
  arborx_alloc_fn alloc; /* NULL: stream-ordered cudaMallocAsync / cudaFreeAsync */
  arborx_free_fn free;
  void *alloc_ctx;
} arborx_opts;

typedef struct arborx_bvh_s *arborx_handle;

/* Library version string (static storage). */
ARBORX_API const char *arborx_version(void);

/* Human-readable text of a status code (static storage; unknown codes give "unknown"). */
ARBORX_API const char *arborx_error_string(int status);

/* Fill *opts with the defaults listed above.  EINVAL if opts is NULL. */
ARBORX_API int arborx_default_opts(arborx_opts *opts);

/* Build the LBVH over n primitives (Sec. 2.1, "BVH construction"): scene-box
 * reduction, Morton codes of the box centroids scaled by the scene box, a
 * stable radix sort of (code, index) pairs, the binary radix-tree hierarchy
 * split at the highest differing bit of the index-augmented codes (Karras
 * 2012), and the bottom-up box fit in which the second thread to reach a node
 * continues (Sec. 2.1, internal-node boxes).
 *   d_prims  device float[n][3] (ARBORX_POINTS) or float[n][6] (ARBORX_BOXES); read only during the
 *            build's stream work; may be freed once that work completes (the tree keeps its own copy
 *            of every primitive box)
 *   n        0 <= n < ARBORX_MAX_PRIMS; n = 0 gives an empty tree, n = 1 a tree whose root is the leaf
 *   opts     NULL for defaults; copied, need not outlive the call
 *   out      receives the handle, owned by the caller until arborx_destroy
 * Synchronises `stream` once when opts->validate is 1 (the default). */
ARBORX_API int arborx_build(const float *d_prims, int64_t n, int32_t kind, const arborx_opts *opts, void *stream,
                 arborx_handle *out);

/* Rebuild the tree in place over new coordinates of the same n primitives of the same kind (a
 * simulation's next time step): the same kernels as arborx_build, writing the handle's records.
 * The first call allocates a build scratch block that the handle keeps (freed by
 * arborx_destroy); later calls allocate nothing and, with opts.validate = 0, do not synchronise,
 * so a rebuild and the queries after it can be captured in one CUDA graph and replayed.  Counts
 * kept for arborx_query_spatial_fill / _buffered_fill are invalidated.  Work on other streams that
 * still reads the old tree must be ordered before the rebuild.
 *   d_prims  device float[n][3] or float[n][6], as for arborx_build (NULL only when n = 0)
 * Errors: ARBORX_EINVAL (null handle or pointer, or a non-finite coordinate when validate = 1),
 * ARBORX_ENOMEM (first call only).  After an error the handle's tree is unspecified until a
 * rebuild succeeds; arborx_destroy still releases it. */
ARBORX_API int arborx_rebuild(arborx_handle h, const float *d_prims, void *stream);

/* Release every allocation of the handle, stream-ordered on the stream of the handle's last call
 * (a handle is used from one stream at a time).  NULL is a no-op. */
ARBORX_API int arborx_destroy(arborx_handle h);

/* Number of primitives and their kind. */
ARBORX_API int arborx_size(arborx_handle h, int64_t *n, int32_t *kind);

/* Synchronise `stream` and report errors raised on the device by earlier calls on this handle
 * (non-finite input when validate was 0, a timed-out look-back, a stack or CSR overflow);
 * clears them. */
ARBORX_API int arborx_check(arborx_handle h, void *stream);

/* Traversal order of a query set (Sec. 2.2, "Query ordering"): 30-bit Morton codes of the query
 * points scaled by the tree's scene box (points outside clamped to it), stably sorted by their top
 * 24 bits (8 per axis; the order only affects speed); d_order[i] is the
 * query traversed i-th.  Pass it to the query calls below to sort a query set once for several
 * queries.  A tree with n = 0 or m < 2 gives the identity.
 *   d_order  device uint32[m], written */
ARBORX_API int arborx_query_order(arborx_handle h, const float *d_queries, int64_t m, void *stream,
                                  uint32_t *d_order);

/* Traversal order of a point or box set without a tree (Sec. 2.2, "Query ordering"): the same
 * 24-bit Morton keys as arborx_query_order, scaled by the set's own bounding box (its finite
 * coordinates; box centres for boxes) instead of a tree's.  Any permutation gives the same query
 * results, so the order may be computed on another stream while the tree is built, or before it.
 * Only enqueues work (graph-capturable); if the sort gives up a bounded wait, d_order is the
 * identity, which is still a valid order.
 *   d_prims  device float[m][3] (ARBORX_POINTS) or float[m][6] (ARBORX_BOXES)
 *   opts     NULL for defaults; only the allocator is used (temporary memory, stream-ordered)
 *   d_order  device uint32[m], written: a permutation of 0..m-1 */
ARBORX_API int arborx_order(const float *d_prims, int64_t m, int32_t kind, const arborx_opts *opts, void *stream,
                            uint32_t *d_order);

/* Spatial query, pass 1 of the count-and-fill scheme (Sec. 2.2, "2P"): traverse the tree for
 * each of the m query points, count the primitives within distance `radius`, and write the
 * exclusive prefix sum of the counts to d_offsets[0..m] (d_offsets[m] = total, int64).
 *   d_queries  device float[m][3]; radius >= 0 and not NaN (+inf selects everything)
 *   d_order    NULL (order the queries here when opts.sort_queries, else input order) or a
 *              permutation of 0..m-1 from arborx_query_order (must stay valid until the fill)
 *   d_offsets  device int64[m + 1], written
 * Keeps the traversal order in the handle for the matching arborx_query_spatial_fill.
 * Does not synchronise. */
ARBORX_API int arborx_query_spatial_count(arborx_handle h, const float *d_queries, int64_t m, float radius,
                                          const uint32_t *d_order, void *stream, int64_t *d_offsets);

/* Spatial query, pass 2: traverse again and write row j (the primitives within `radius` of
 * query j) to d_indices[d_offsets[j] .. d_offsets[j+1]).  Must follow
 * arborx_query_spatial_count on the same handle with the same d_queries, m, radius and
 * d_offsets.  Row order within a row is the traversal order (rows are sets).
 *   d_indices  device int32[capacity], capacity >= d_offsets[m]; writes beyond capacity are
 *              skipped and reported as ARBORX_EOVERFLOW by arborx_check.
 * Does not synchronise. */
ARBORX_API int arborx_query_spatial_fill(arborx_handle h, const float *d_queries, int64_t m, float radius, void *stream,
                              const int64_t *d_offsets, int32_t *d_indices, int64_t capacity);

/* Spatial query, both passes: count, read the total back to the host (synchronises `stream`),
 * allocate the indices with the handle's allocator, fill.  d_order as for the count pass.
 *   d_offsets   device int64[m + 1], written (CSR offsets, original query order)
 *   d_indices   receives a device int32[*nnz] array allocated with the handle's allocator
 *               (opts.alloc, else cudaMallocAsync); release it with arborx_free
 *   nnz         receives the total number of results */
ARBORX_API int arborx_query_spatial(arborx_handle h, const float *d_queries, int64_t m, float radius,
                                    const uint32_t *d_order, void *stream, int64_t *d_offsets, int32_t **d_indices,
                                    int64_t *nnz);

/* One-pass spatial query (Sec. 2.2, "1P"), count call: a single traversal counts the results of
 * every query and keeps the first `buffer_size` of them in a row buffer owned by the handle
 * (m * buffer_size int32); the counts are scanned into d_offsets and the total is read back
 * (synchronises `stream`) into *h_nnz.  buffer_size is the caller's estimate of the largest row;
 * it only affects speed: rows that do not fit are produced by a second traversal in the fill call.
 *   1 <= buffer_size <= ARBORX_MAX_BUFFER_SIZE; d_order as for arborx_query_spatial_count */
#define ARBORX_MAX_BUFFER_SIZE 4096
ARBORX_API int arborx_query_spatial_buffered_count(arborx_handle h, const float *d_queries, int64_t m, float radius,
                                                   int32_t buffer_size, const uint32_t *d_order, void *stream,
                                                   int64_t *d_offsets, int64_t *h_nnz);

/* One-pass spatial query, fill call: compacts the buffered rows into d_indices at d_offsets and
 * traverses again only for the queries whose rows overflowed the buffer.  Must follow
 * arborx_query_spatial_buffered_count on the same handle with the same d_queries, m, radius and
 * d_offsets; d_indices as for arborx_query_spatial_fill.  Does not synchronise. */
ARBORX_API int arborx_query_spatial_buffered_fill(arborx_handle h, const float *d_queries, int64_t m, float radius,
                                                  void *stream, const int64_t *d_offsets, int32_t *d_indices,
                                                  int64_t capacity);

/* One-pass spatial query in a single call with no host synchronisation (graph-capturable): the
 * count traversal with the `buffer_size` row buffer, the scan, the compaction and the second
 * traversal of the overflowing rows, all enqueued on `stream`.  d_offsets[m] receives the total
 * on the device.  Rows are written into caller-owned d_indices of `capacity` entries; entries at
 * positions >= capacity are not written and set the CSR-overflow error reported as
 * ARBORX_EOVERFLOW by arborx_check (the offsets stay complete, so the caller can size a new
 * buffer from d_offsets[m] and repeat).  Results equal those of arborx_query_spatial.
 *   buffer_size  1 <= buffer_size <= ARBORX_MAX_BUFFER_SIZE
 *   d_order      NULL or a traversal order from arborx_query_order
 *   d_offsets    device int64[m + 1]
 *   d_indices    device int32[capacity] (NULL when capacity == 0) */
ARBORX_API int arborx_query_spatial_buffered(arborx_handle h, const float *d_queries, int64_t m, float radius,
                                             int32_t buffer_size, const uint32_t *d_order, void *stream,
                                             int64_t *d_offsets, int32_t *d_indices, int64_t capacity);

/* The one-pass spatial query of arborx_query_spatial_buffered and the nearest query of
 * arborx_query_nearest over the same queries (Sec. 2.2: the two traversals share the tree and the
 * query order but nothing else), in one call: after the query order, the nearest traversal runs on
 * a second stream owned by the handle, forked from `stream` by an event and joined back into it,
 * so that it overlaps the spatial query's counting traversal tail, compaction and overflow pass.
 * Results equal those of the two calls made one after the other; work enqueued on `stream` after
 * this call sees both.  The handle creates its second stream and two events on its first such
 * call (make that call outside stream capture); arborx_destroy releases them.  No host
 * synchronisation.
 *   radius, buffer_size, d_offsets, d_indices, capacity  as for arborx_query_spatial_buffered
 *   k, d_nn_offsets, d_nn_indices, d_nn_dist2             as d_offsets, d_indices, d_dist2 of
 *                                                         arborx_query_nearest
 *   d_order      NULL or a traversal order from arborx_query_order (shared by both traversals)
 * Errors: those of the two calls; ARBORX_ECUDA when the stream or events cannot be created. */
ARBORX_API int arborx_query_spatial_nearest(arborx_handle h, const float *d_queries, int64_t m, float radius,
                                            int32_t buffer_size, int32_t k, const uint32_t *d_order, void *stream,
                                            int64_t *d_offsets, int32_t *d_indices, int64_t capacity,
                                            int64_t *d_nn_offsets, int32_t *d_nn_indices, float *d_nn_dist2);

/* Traversal order of a set of query boxes: as arborx_query_order, with each box's centre
 * 0.5 (lo + hi) in place of the point (a NaN centre sorts first).
 *   d_boxes  device float[m][6] (lo.x, lo.y, lo.z, hi.x, hi.y, hi.z)
 *   d_order  device uint32[m], written */
ARBORX_API int arborx_query_order_boxes(arborx_handle h, const float *d_boxes, int64_t m, void *stream,
                                        uint32_t *d_order);

/* Spatial query with a box predicate (Sec. 2.2.1, where every node is tested against the query's
 * predicate on its own; here the predicate is box intersection, the test AABBs make cheap, Sec. 2):
 * row j lists every primitive whose box B (a point p is the box [p, p]) meets query box Q on every
 * axis as closed intervals:  B.lo <= Q.hi  and  B.hi >= Q.lo.  Touching boxes match.  The test is
 * comparisons only, so results are exact; a query box with a NaN bound matches nothing, infinite
 * bounds are allowed, and a box with lo > hi on an axis matches what the same test accepts.
 * One call with no host synchronisation (graph-capturable), in the one-pass form of
 * arborx_query_spatial_buffered: a counting traversal that keeps the first `buffer_size` results
 * of each row, the scan into d_offsets, the compaction, and a second traversal for the rows that
 * overflowed the buffer.  d_offsets[m] receives the total on the device; entries at positions
 * >= capacity are not written and set the CSR-overflow error (ARBORX_EOVERFLOW from
 * arborx_check), with the offsets still complete so the caller can size a new buffer and repeat.
 *   d_boxes      device float[m][6] (lo.xyz, hi.xyz), read only
 *   buffer_size  1 <= buffer_size <= ARBORX_MAX_BUFFER_SIZE (speed only)
 *   d_order      NULL (Morton order of the box centres when opts.sort_queries, else input order)
 *                or a permutation of 0..m-1 from arborx_query_order_boxes
 *   d_offsets    device int64[m + 1], written (original query order)
 *   d_indices    device int32[capacity] (NULL when capacity == 0); rows are sets in traversal order
 * Errors: ARBORX_EINVAL for a null handle, m out of range, a missing pointer or a bad
 * buffer_size or capacity; ARBORX_ENOMEM when the row buffer cannot be allocated. */
ARBORX_API int arborx_query_intersects(arborx_handle h, const float *d_boxes, int64_t m, int32_t buffer_size,
                                       const uint32_t *d_order, void *stream, int64_t *d_offsets, int32_t *d_indices,
                                       int64_t capacity);

/* Self-test of the bounded waits (not in the paper): one GPU thread waits on a flag that nothing
 * sets, with the iteration cap and backoff of the sort's decoupled look-back, gives up, and the
 * call reports it the way arborx_check reports a timed-out look-back.  Returns ARBORX_ETIMEOUT
 * (the expected result; the device stays usable), ARBORX_ENOMEM or ARBORX_ECUDA.  Synchronises
 * `stream`; takes about a second. */
ARBORX_API int arborx_selftest_bounded_wait(void *stream);

/* Self-test of the one-call spatial query's scan (not in the paper): the scan-and-compaction
 * kernel of arborx_query_spatial_buffered runs over two tiles of empty rows with its tile counter
 * preset so that its only block takes the second tile and looks back at a first tile that never
 * publishes; the look-back gives up at its iteration cap.  Returns ARBORX_ETIMEOUT (the expected
 * result; the device stays usable), ARBORX_ENOMEM or ARBORX_ECUDA.  Synchronises `stream`; takes
 * about a second. */
ARBORX_API int arborx_selftest_scan_wait(void *stream);

/* Release memory returned by arborx_query_spatial (stream-ordered on `stream`). */
ARBORX_API int arborx_free(arborx_handle h, void *d_ptr, size_t bytes, void *stream);

/* Nearest query (Sec. 2.2, "Traversal for nearest queries"): for each query, the kk = min(k, n)
 * primitives first in (d^2, index) order, found by a stack traversal that visits the closer
 * child first and skips a node whose box distance exceeds the current k-th candidate.  Unless
 * opts.knn_anchor = 0, the traversal starts from an exact bound on the k-th distance taken from
 * the tree (a subtree of at least k leaves near the query, found on the traversal's first descent
 * or by a walk before it, see arborx_opts); candidates in a
 * register list for k below opts.knn_heap_from, else a shared-memory heap.
 *   k           1 <= k <= ARBORX_MAX_K
 *   d_order     NULL or a traversal order from arborx_query_order (as for the spatial count)
 *   d_offsets   NULL or device int64[m + 1]: written with j * kk (CSR view of the rows)
 *   d_indices   device int32[m * kk]: row j holds query j's neighbours in (d^2, index) order;
 *               -1 where a query has fewer (non-finite query)
 *   d_dist2     NULL or device float[m * kk]: the matching squared distances (+inf for -1)
 * Does not synchronise. */
ARBORX_API int arborx_query_nearest(arborx_handle h, const float *d_queries, int64_t m, int32_t k,
                                    const uint32_t *d_order, void *stream, int64_t *d_offsets, int32_t *d_indices,
                                    float *d_dist2);

/* Copy the tree out for inspection (device to device, stream-ordered):
 *   d_records  NULL or device float[(2 + 2(n-1)) * 8] in the record layout above (n >= 1)
 *   d_scene    NULL or device float[6]: the scene box lo.xyz, hi.xyz
 *   d_codes    NULL or device uint64[n]: sorted Morton codes (needs opts.keep_order = 1)
 *   d_perm     NULL or device uint32[n]: primitive index of each sorted leaf (needs keep_order)
 * ESTATE if codes / perm are requested but were not kept. */
ARBORX_API int arborx_export_tree(arborx_handle h, void *stream, float *d_records, float *d_scene, uint64_t *d_codes,
                       uint32_t *d_perm);

/* Stable ascending radix sort of n keys of key_bits significant bits (the sort step of the
 * build, Sec. 2.1, exposed on its own): keys are uint32 when key_bits <= 32, else uint64;
 * d_keys is sorted in place and d_perm receives, for each output position, the input position
 * of its key (ties keep input order).  Needs temporary memory from cudaMallocAsync.
 *   1 <= key_bits <= 64; 0 <= n < ARBORX_MAX_PRIMS */
ARBORX_API int arborx_sort_pairs(void *d_keys, uint32_t *d_perm, int64_t n, int32_t key_bits, void *stream);

/* Same sort as arborx_sort_pairs, for callers that must not allocate device memory inside the call
 * (for example code that runs inside another framework's fixed memory budget, or a loop whose memory
 * is planned up front): its temporaries live in a fixed 16 MiB device array that the library
 * defines, which every GPU that loads the library holds until the process exits.  The paper has no
 * counterpart; this is a property of this library's interface only.
 *   n  at most ARBORX_SORT_NOALLOC_MAX_KEYS; larger n returns ARBORX_EINVAL without touching the GPU
 * The first call on a device looks up the array's device address (make it before any stream
 * capture) and keeps it for the life of the process; after a cudaDeviceReset of that device the
 * kept address is stale, as is the library's per-device memory pool, so the library must not be
 * called on that device again.  All calls on a device share the one array, which keeps the last
 * call's contents (each call clears what must start at zero): calls whose GPU work overlaps
 * (different streams or host threads) race and must be serialised by the caller.  Synchronises
 * `stream`.  Status is reported as by arborx_sort_pairs. */
#define ARBORX_SORT_NOALLOC_MAX_KEYS (1 << 20)
ARBORX_API int arborx_sort_pairs_noalloc(void *d_keys, uint32_t *d_perm, int64_t n, int32_t key_bits, void *stream);

/* ---------------------------------------------------------------------------------------------
 * Learned initial bound for nearest queries.  A regressor 3 -> 64 -> 64 -> 1 (ReLU) maps a query,
 * normalised by the tree's scene box ((q - lo) / (hi - lo), 0 on a flat axis), to an estimate y of
 * log d_k, the distance to its k-th nearest primitive.  The paper has no such component: it only
 * seeds the nearest traversal of Sec. 2.2 with the squared bound exp(2 (y + margin)); queries that
 * find fewer than k primitives inside the bound are traversed again without it, so results are
 * exactly those of arborx_query_nearest.  Parameters are one float32 vector of ARBORX_MLP_PARAMS
 * values: W1 [64][3], b1 [64], W2 [64][64] (row = output unit), b2 [64], w3 [64], b3. */
#define ARBORX_MLP_PARAMS 4481

/* Regressor output y for m queries: tensor_cores = 1 runs the BF16 tensor-core kernel used by
 * arborx_query_nearest_learned (inputs rounded to BF16, FP32 accumulation); 0 runs FP32 on CUDA cores.
 *   d_params  device float[ARBORX_MLP_PARAMS];  d_y  device float[m], written */
ARBORX_API int arborx_mlp_forward(arborx_handle h, const float *d_params, const float *d_queries, int64_t m,
                                  int32_t tensor_cores, void *stream, float *d_y);

/* Mean squared error of y against d_labels over b queries and its gradient w.r.t. the parameters
 * (FP32 forward and backward on the GPU).
 *   d_labels  device float[b];  d_grad  device float[ARBORX_MLP_PARAMS], written;
 *   d_loss    NULL or device float[1], written */
ARBORX_API int arborx_mlp_grad(arborx_handle h, const float *d_params, const float *d_queries, const float *d_labels,
                               int64_t b, void *stream, float *d_grad, float *d_loss);

/* Train the regressor on mt training queries: labels log(max(d_k, 1e-30)) come from this tree's own
 * exact nearest traversal (k-th distance); then `epochs` passes of mini-batch Adam (beta 0.9 / 0.999,
 * eps 1e-8) over batches of `batch` queries, the learning rate following a cosine from lr at the
 * first step to lr_final at the last (lr_final = lr: constant), each step one gradient kernel and
 * one update kernel.  d_params holds the initial parameters and receives the trained ones;
 * d_loss (NULL or device float[epochs]) receives the mean batch loss of each epoch. */
ARBORX_API int arborx_mlp_train(arborx_handle h, const float *d_queries, int64_t mt, int32_t k, int32_t epochs,
                                int32_t batch, float lr, float lr_final, void *stream, float *d_params,
                                float *d_loss);

/* Nearest query seeded with a caller-supplied upper bound per query (for example the k-th distances
 * of the previous time step of a simulation): the traversal starts with d_bound2[j] as the k-th
 * squared distance of query j; queries that find fewer than k primitives within their bound are
 * traversed again with a bound taken from the finished rows of their neighbours in Morton order
 * (the neighbour's k-th distance plus the distance between the two queries, which always holds k
 * primitives), and without a bound if no neighbour provides one, so outputs equal those of
 * arborx_query_nearest whatever the bounds.
 *   d_bound2     device float[m] (by query index; +inf = no bound)
 *   h_fallbacks  NULL, or host int64 receiving the number of second traversals (synchronises) */
ARBORX_API int arborx_query_nearest_bounded(arborx_handle h, const float *d_queries, int64_t m, int32_t k,
                                            const float *d_bound2, const uint32_t *d_order, void *stream,
                                            int64_t *d_offsets, int32_t *d_indices, float *d_dist2,
                                            int64_t *h_fallbacks);

/* Nearest query with the learned initial bound (same outputs as arborx_query_nearest).
 *   margin       added to the predicted log distance (larger: fewer fallbacks, less pruning)
 *   h_fallbacks  NULL, or host int64 receiving the number of queries that needed the unbounded
 *                second traversal (synchronises `stream`) */
ARBORX_API int arborx_query_nearest_learned(arborx_handle h, const float *d_queries, int64_t m, int32_t k,
                                            const float *d_params, float margin, const uint32_t *d_order,
                                            void *stream, int64_t *d_offsets, int32_t *d_indices, float *d_dist2,
                                            int64_t *h_fallbacks);

/* ---------------------------------------------------------------------------------------------
 * Many independent point clouds at once: every cloud gets its own tree (the LBVH of Sec. 2.1 over its
 * points) and every query its k nearest points of its own cloud (Sec. 2.2), for all clouds in one
 * launch sequence of about twenty kernels instead of a build and a query per cloud.  The paper has
 * no batched interface; results equal those of arborx_build + arborx_query_nearest per cloud. */
typedef struct arborx_batch_s *arborx_batch;

/* Plan a batch of n_clouds clouds (host arrays, copied): cloud c owns points
 * [h_point_offsets[c], h_point_offsets[c+1]) of the concatenated point array (float[N][3]) and
 * queries [h_query_offsets[c], h_query_offsets[c+1]) of the concatenated query array, and wants
 * its k_c = h_k[c] nearest points (1 <= k_c <= 32).  Offsets start at 0 and do not decrease.
 * Allocates every device buffer the runs need (so runs allocate nothing) and synchronises once.
 * opts: block_size, stack_smem, knn_anchor, queries_per_warp, knn_heap_from and the allocator are
 * used; NULL for defaults. */
ARBORX_API int arborx_batch_create(int64_t n_clouds, const int64_t *h_point_offsets, const int64_t *h_query_offsets,
                                   const int32_t *h_k, const arborx_opts *opts, void *stream, arborx_batch *out);

/* Totals of a batch: points, queries, and output entries (sum over queries of min(k_c, n_c)). */
ARBORX_API int arborx_batch_entries(arborx_batch b, int64_t *n_points, int64_t *n_queries, int64_t *entries);

/* Build all clouds and answer all queries.  Row j (query j of the concatenation) is written at
 * d_row_offsets[j] (int64[M+1], NULL to skip) with min(k_c, n_c) point indices local to the
 * query's cloud in (d^2, index) order, -1 for a non-finite query; d_dist2 (NULL or float[entries])
 * gets the squared distances.  use_graph = 1: the launch sequence is captured in a CUDA graph on
 * the first call and replayed while the five pointers stay the same.  Does not synchronise;
 * arborx_batch_check reports device errors of the last run. */
ARBORX_API int arborx_batch_run(arborx_batch b, const float *d_points, const float *d_queries, int32_t use_graph,
                                void *stream, int64_t *d_row_offsets, int32_t *d_indices, float *d_dist2);

/* Synchronise `stream` and report device errors of the last run (non-finite input: EINVAL). */
ARBORX_API int arborx_batch_check(arborx_batch b, void *stream);

/* The whole batch in one synchronous call: arborx_batch_create, arborx_batch_run (eager, no graph),
 * arborx_batch_check and arborx_batch_destroy.  Arguments as for those calls; capacity is the
 * number of entries d_indices (and d_dist2, if not NULL) hold, at least the batch's entries
 * (sum over queries of min(k_c, n_c)), else ARBORX_EINVAL.  Returns the first error.  The paper has
 * no batched interface; results equal those of arborx_build + arborx_query_nearest per cloud. */
ARBORX_API int arborx_batched(int64_t n_clouds, const int64_t *h_point_offsets, const int64_t *h_query_offsets,
                              const int32_t *h_k, const float *d_points, const float *d_queries,
                              const arborx_opts *opts, void *stream, int64_t *d_row_offsets, int32_t *d_indices,
                              float *d_dist2, int64_t capacity);

/* Release the batch (stream-ordered on the creation stream).  NULL is a no-op. */
ARBORX_API int arborx_batch_destroy(arborx_batch b);

/* Per-tree query options, set between queries (host only; takes effect for the queries enqueued
 * after it).  Not in the paper; speed only, results are identical either way.
 *   ARBORX_QOPT_EMIT_SUBTREES, value 0 (default) or 1: radius and box queries take every leaf of a
 *     subtree whose box lies wholly inside the query (for a radius, its farthest corner within r,
 *     which bounds the FP32 distance of every point in it) from the tree's kept sorted leaf order,
 *     instead of walking the subtree.  Faster when rows hold hundreds of hits (the 256^3 lattice at
 *     r = 4, 253 hits per row: 6.58 -> 5.65 ms per 1e6 queries), slower for short rows
 *     (mean 10 hits on the 1e7-point cube: 0.62 -> 0.91 ms).  Needs a
 *     tree built with opts.keep_order = 1, else ARBORX_ESTATE.
 * Errors: ARBORX_EINVAL for a null handle, an unknown option or a value out of range. */
#define ARBORX_QOPT_EMIT_SUBTREES 1
ARBORX_API int arborx_set_query_option(arborx_handle h, int32_t option, int64_t value);

/* Traversal statistics of a tree built with opts.stats = 1 (synchronises `stream`): out[0], out[1] =
 * internal nodes loaded by spatial and nearest traversals, out[2], out[3] = queries traversed,
 * since the previous call; resets them. */
ARBORX_API int arborx_stats(arborx_handle h, void *stream, uint64_t out[4]);

/* Return the library's cached device memory (freed trees and workspaces) to the driver.  The
 * library's stream-ordered pool keeps freed blocks for reuse until this call. */
ARBORX_API int arborx_release_cached_memory(void);

/* Process-wide kernel timing.  With on = 1, every kernel launch of the library is bracketed by a
 * pair of CUDA events on its stream (a few microseconds of host overhead per launch). */
ARBORX_API int arborx_profile_enable(int on);

/* Wait for the recorded events, then write one line per kernel name, "name launches total_ms\n",
 * into buf (NUL-terminated, at most cap bytes) and reset the counters.  EOVERFLOW if truncated. */
ARBORX_API int arborx_profile_report(char *buf, size_t cap);

#ifdef __cplusplus
}
#endif

#endif /* ARBORX_B300_H */

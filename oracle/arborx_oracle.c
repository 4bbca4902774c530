/*
 * CPU oracle for the geometric search path -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * may load this code.  It shares no source, header, table or helper with the
 * CUDA library and never calls it.  Build: gcc -O2 -ffp-contract=off -fopenmp
 * (no FMA contraction, so every float expression rounds exactly as written).
 *
 * What it computes (ArborX, arXiv 1908.11807):
 *   - scene bounding box: min / max over all box corners (Sec. 2.1, scene box
 *     step);
 *   - Morton codes of box centroids scaled by the scene box into [0,1]^3,
 *     30-bit (10 bits per axis) and 63-bit (21 bits per axis), bits
 *     interleaved x-major (Sec. 2.1, Morton code step);
 *   - spatial query: every primitive whose AABB lies within distance r of the
 *     query point (Sec. 2.2, "Traversal for spatial queries"), read as the
 *     closed ball d^2 <= fl32(r*r);
 *   - box query: every primitive whose AABB meets the query box, both taken
 *     as closed intervals on each axis (lo_i <= qhi and hi_i >= qlo on x, y
 *     and z); the spatial traversal of Sec. 2.2 with the box-intersection test
 *     that Sec. 2 names as the AABB's cheap operation as its predicate;
 *   - nearest query: the min(k, n) primitives closest to the query point, ties
 *     broken by lower index, rows ordered by (d^2, index) (Sec. 2.2, "Traversal
 *     for nearest queries"; fewer than k when n < k, as the paper drops missing
 *     entries).
 *
 * Distance arithmetic (the reading used on both sides): per axis the gap
 * g = lo - q if q < lo, q - hi if q > hi, else 0 (for a point p: g = q - p);
 * d^2 = ((gx*gx) + (gy*gy)) + (gz*gz), each operation one FP32 round-to-
 * nearest step.  A query with a non-finite coordinate has no neighbours.
 *
 * Three independent evaluators:
 *   1. brute force over all primitives -- the definition written out;
 *   2. a CPU BVH built by recursive median split of the longest centroid
 *      extent (leaf size 4) -- a different tree from the LBVH, used to check
 *      large cases quickly; its node boxes are exact min / max of member
 *      coordinates, so its pruning never drops a result;
 *   3. an FP64 checker that recomputes membership in double precision from the
 *      FP32-stored coordinates and reports disagreements that are not within
 *      a relative 1e-6 of the radius (or of the k-th distance).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_POINTS 0
#define ORC_BOXES 1

static int nthreads_used(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

int orc_threads(void) { return nthreads_used(); }

void orc_set_threads(int t) {
#ifdef _OPENMP
  if (t > 0) omp_set_num_threads(t);
#else
  (void)t;
#endif
}

/* ---------------------------------------------------------------- geometry */

static inline void prim_box(const float *prims, int kind, int64_t i, float lo[3], float hi[3]) {
  if (kind == ORC_POINTS) {
    const float *p = prims + 3 * i;
    lo[0] = hi[0] = p[0];
    lo[1] = hi[1] = p[1];
    lo[2] = hi[2] = p[2];
  } else {
    const float *b = prims + 6 * i;
    lo[0] = b[0]; lo[1] = b[1]; lo[2] = b[2];
    hi[0] = b[3]; hi[1] = b[4]; hi[2] = b[5];
  }
}

static inline float gap(float q, float lo, float hi) {
  if (q < lo) return lo - q;
  if (q > hi) return q - hi;
  return 0.0f;
}

/* squared distance from point q to the box [lo, hi], FP32, fixed order */
static inline float dist2_box(const float q[3], const float lo[3], const float hi[3]) {
  float gx = gap(q[0], lo[0], hi[0]);
  float gy = gap(q[1], lo[1], hi[1]);
  float gz = gap(q[2], lo[2], hi[2]);
  float sx = gx * gx;
  float sy = gy * gy;
  float sz = gz * gz;
  float s = sx + sy;
  s = s + sz;
  return s;
}

/* squared distance from point q to primitive i (point: plain difference) */
static inline float dist2_prim(const float *prims, int kind, int64_t i, const float q[3]) {
  if (kind == ORC_POINTS) {
    const float *p = prims + 3 * i;
    float dx = q[0] - p[0];
    float dy = q[1] - p[1];
    float dz = q[2] - p[2];
    float sx = dx * dx;
    float sy = dy * dy;
    float sz = dz * dz;
    float s = sx + sy;
    s = s + sz;
    return s;
  }
  float lo[3], hi[3];
  prim_box(prims, kind, i, lo, hi);
  return dist2_box(q, lo, hi);
}

static inline int finite3(const float q[3]) {
  return isfinite(q[0]) && isfinite(q[1]) && isfinite(q[2]);
}

/* (d, i) strictly before (e, j) in the (distance, index) order */
static inline int pair_less(float d, int32_t i, float e, int32_t j) {
  return d < e || (d == e && i < j);
}

/* ------------------------------------------------- scene box and Morton */

/* Scene box: min / max over every corner coordinate.  out = lo.xyz, hi.xyz.
 * Returns the number of non-finite coordinates seen. */
int64_t orc_scene_box(const float *prims, int64_t n, int kind, float out[6]) {
  int64_t bad = 0;
  float lo[3] = {INFINITY, INFINITY, INFINITY};
  float hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  int per = kind == ORC_POINTS ? 3 : 6;
  for (int64_t i = 0; i < n; ++i) {
    for (int c = 0; c < per; ++c) {
      float v = prims[per * i + c];
      int a = c % 3;
      if (!isfinite(v)) {
        ++bad;
        continue;
      }
      if (v < lo[a]) lo[a] = v;
      if (v > hi[a]) hi[a] = v;
    }
  }
  for (int a = 0; a < 3; ++a) {
    out[a] = lo[a];
    out[3 + a] = hi[a];
  }
  return bad;
}

/* Quantise a centroid coordinate: u = (c - L) / (H - L) in FP32 (u = 0 when
 * the axis is flat), clamped into [0, 1], scaled by 2^bits, floored, clamped
 * to 2^bits - 1. */
static inline uint32_t quantise(float c, float L, float H, int bits) {
  float ext = H - L;
  float u = 0.0f;
  if (ext > 0.0f) {
    float num = c - L;
    u = num / ext;
  }
  if (!(u >= 0.0f)) u = 0.0f; /* also maps NaN to 0 */
  if (u > 1.0f) u = 1.0f;
  float scaled = u * (float)(1u << bits);
  uint32_t q = (uint32_t)floorf(scaled);
  uint32_t top = (1u << bits) - 1u;
  return q > top ? top : q;
}

static inline void centroid(const float *prims, int kind, int64_t i, float c[3]) {
  if (kind == ORC_POINTS) {
    c[0] = prims[3 * i];
    c[1] = prims[3 * i + 1];
    c[2] = prims[3 * i + 2];
  } else {
    const float *b = prims + 6 * i;
    for (int a = 0; a < 3; ++a) {
      float s = b[a] + b[3 + a];
      c[a] = s * 0.5f;
    }
  }
}

/* Interleave: for bit level l from most significant down, emit x_l, y_l, z_l,
 * so x occupies bit 3l+2, y 3l+1, z 3l. */
static uint64_t interleave(uint32_t qx, uint32_t qy, uint32_t qz, int bits) {
  uint64_t code = 0;
  for (int l = bits - 1; l >= 0; --l) {
    code = (code << 1) | ((qx >> l) & 1u);
    code = (code << 1) | ((qy >> l) & 1u);
    code = (code << 1) | ((qz >> l) & 1u);
  }
  return code;
}

/* Morton codes of the n primitive centroids against scene box sb (lo.xyz,
 * hi.xyz); bits_per_axis is 10 (30-bit codes) or 21 (63-bit codes). */
void orc_morton(const float *prims, int64_t n, int kind, const float sb[6], int bits_per_axis,
                uint64_t *out) {
  for (int64_t i = 0; i < n; ++i) {
    float c[3];
    centroid(prims, kind, i, c);
    uint32_t q[3];
    for (int a = 0; a < 3; ++a) q[a] = quantise(c[a], sb[a], sb[3 + a], bits_per_axis);
    out[i] = interleave(q[0], q[1], q[2], bits_per_axis);
  }
}

/* ----------------------------------------------------------- brute force */

/* Spatial, pass 1: counts[j] = |{ i : d2(q_j, b_i) <= fl(r*r) }|. */
void orc_spatial_count_brute(const float *prims, int64_t n, int kind, const float *queries, int64_t m,
                             float r, int64_t *counts) {
  float r2 = r * r;
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t j = 0; j < m; ++j) {
    const float *q = queries + 3 * j;
    int64_t c = 0;
    if (finite3(q))
      for (int64_t i = 0; i < n; ++i)
        if (dist2_prim(prims, kind, i, q) <= r2) ++c;
    counts[j] = c;
  }
}

/* Spatial, pass 2: row j of the CSR result in ascending index order. */
void orc_spatial_fill_brute(const float *prims, int64_t n, int kind, const float *queries, int64_t m,
                            float r, const int64_t *offsets, int32_t *indices) {
  float r2 = r * r;
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t j = 0; j < m; ++j) {
    const float *q = queries + 3 * j;
    int64_t o = offsets[j];
    if (finite3(q))
      for (int64_t i = 0; i < n; ++i)
        if (dist2_prim(prims, kind, i, q) <= r2) indices[o++] = (int32_t)i;
  }
}

/* Box query predicate: the closed boxes [lo, hi] and [q[0..2], q[3..5]] meet
 * on every axis.  Comparisons only; a NaN bound makes a comparison false. */
static inline int boxes_meet(const float lo[3], const float hi[3], const float *q) {
  for (int a = 0; a < 3; ++a)
    if (!(lo[a] <= q[3 + a] && hi[a] >= q[a])) return 0;
  return 1;
}

/* Box query, pass 1: counts[j] = number of primitives meeting query box j. */
void orc_intersects_count_brute(const float *prims, int64_t n, int kind, const float *qboxes, int64_t m,
                                int64_t *counts) {
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t j = 0; j < m; ++j) {
    const float *q = qboxes + 6 * j;
    int64_t c = 0;
    for (int64_t i = 0; i < n; ++i) {
      float lo[3], hi[3];
      prim_box(prims, kind, i, lo, hi);
      if (boxes_meet(lo, hi, q)) ++c;
    }
    counts[j] = c;
  }
}

/* Box query, pass 2: row j of the CSR result in ascending index order. */
void orc_intersects_fill_brute(const float *prims, int64_t n, int kind, const float *qboxes, int64_t m,
                               const int64_t *offsets, int32_t *indices) {
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t j = 0; j < m; ++j) {
    const float *q = qboxes + 6 * j;
    int64_t o = offsets[j];
    for (int64_t i = 0; i < n; ++i) {
      float lo[3], hi[3];
      prim_box(prims, kind, i, lo, hi);
      if (boxes_meet(lo, hi, q)) indices[o++] = (int32_t)i;
    }
  }
}

/* insert (d, i) into the ascending list (ld, li) of length len <= cap, keeping
 * the cap best; returns the new length */
static int list_insert(float *ld, int32_t *li, int len, int cap, float d, int32_t i) {
  if (len == cap && !pair_less(d, i, ld[len - 1], li[len - 1])) return len;
  int pos = len < cap ? len : cap - 1;
  while (pos > 0 && pair_less(d, i, ld[pos - 1], li[pos - 1])) {
    ld[pos] = ld[pos - 1];
    li[pos] = li[pos - 1];
    --pos;
  }
  ld[pos] = d;
  li[pos] = i;
  return len < cap ? len + 1 : len;
}

/* Nearest: row j = first kk = min(k, n) primitives in (d2, index) order.
 * Unfilled entries (non-finite query) are index -1, distance +inf. */
void orc_nearest_brute(const float *prims, int64_t n, int kind, const float *queries, int64_t m, int k,
                       int32_t *indices, float *dist2) {
  int kk = (int)(n < k ? n : k);
  if (kk <= 0) return;
#pragma omp parallel
  {
    float *ld = (float *)malloc(sizeof(float) * kk);
    int32_t *li = (int32_t *)malloc(sizeof(int32_t) * kk);
#pragma omp for schedule(dynamic, 16)
    for (int64_t j = 0; j < m; ++j) {
      const float *q = queries + 3 * j;
      int len = 0;
      if (finite3(q))
        for (int64_t i = 0; i < n; ++i) len = list_insert(ld, li, len, kk, dist2_prim(prims, kind, i, q), (int32_t)i);
      for (int t = 0; t < kk; ++t) {
        indices[j * kk + t] = t < len ? li[t] : -1;
        if (dist2) dist2[j * kk + t] = t < len ? ld[t] : INFINITY;
      }
    }
    free(ld);
    free(li);
  }
}

/* ------------------------------------------------------------- CPU BVH */

typedef struct {
  float lo[3], hi[3];
  int32_t left, right; /* internal: child node ids; leaf: left = -1, right unused */
  int64_t begin, end;  /* member range in perm (leaves) */
} cnode;

typedef struct {
  cnode *nodes;
  int64_t nnodes, cap;
  int64_t *perm;
  float *cent; /* centroids, [n][3], ordering only */
  const float *prims;
  int64_t n;
  int kind;
} ctree;

#define LEAF_SIZE 4

static inline int cent_less(const ctree *t, int axis, int64_t a, int64_t b) {
  float ca = t->cent[3 * a + axis], cb = t->cent[3 * b + axis];
  return ca < cb || (ca == cb && a < b);
}

/* quickselect: reorder perm[b, e) so that perm[mid] is the element of rank
 * mid - b in (centroid[axis], index) order, smaller ones before it */
static void select_mid(ctree *t, int axis, int64_t b, int64_t e, int64_t mid) {
  int64_t *p = t->perm;
  while (e - b > 1) {
    int64_t a0 = b, a1 = b + (e - b) / 2, a2 = e - 1; /* median of three */
    int64_t piv;
    {
      int64_t x = p[a0], y = p[a1], z = p[a2];
      if (cent_less(t, axis, x, y)) {
        if (cent_less(t, axis, y, z)) piv = y;
        else if (cent_less(t, axis, x, z)) piv = z;
        else piv = x;
      } else {
        if (cent_less(t, axis, x, z)) piv = x;
        else if (cent_less(t, axis, y, z)) piv = z;
        else piv = y;
      }
    }
    /* three-way split around the (unique) pivot */
    int64_t lt = b, i = b, gt = e;
    while (i < gt) {
      if (cent_less(t, axis, p[i], piv)) {
        int64_t s = p[lt]; p[lt] = p[i]; p[i] = s; ++lt; ++i;
      } else if (cent_less(t, axis, piv, p[i])) {
        --gt; int64_t s = p[gt]; p[gt] = p[i]; p[i] = s;
      } else {
        ++i;
      }
    }
    if (mid < lt) e = lt;
    else if (mid >= gt) b = gt;
    else return;
  }
}

static int64_t new_node(ctree *t) {
  int64_t id;
#pragma omp atomic capture
  id = t->nnodes++;
  return id;
}

static void node_box(ctree *t, int64_t b, int64_t e, float lo[3], float hi[3]) {
  for (int a = 0; a < 3; ++a) {
    lo[a] = INFINITY;
    hi[a] = -INFINITY;
  }
  for (int64_t s = b; s < e; ++s) {
    float pl[3], ph[3];
    prim_box(t->prims, t->kind, t->perm[s], pl, ph);
    for (int a = 0; a < 3; ++a) {
      if (pl[a] < lo[a]) lo[a] = pl[a];
      if (ph[a] > hi[a]) hi[a] = ph[a];
    }
  }
}

static void build_rec(ctree *t, int64_t id, int64_t b, int64_t e, int depth) {
  cnode *nd = &t->nodes[id];
  node_box(t, b, e, nd->lo, nd->hi);
  nd->begin = b;
  nd->end = e;
  if (e - b <= LEAF_SIZE) {
    nd->left = nd->right = -1;
    return;
  }
  /* split on the longest extent of the member centroids */
  float clo[3] = {INFINITY, INFINITY, INFINITY}, chi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int64_t s = b; s < e; ++s)
    for (int a = 0; a < 3; ++a) {
      float v = t->cent[3 * t->perm[s] + a];
      if (v < clo[a]) clo[a] = v;
      if (v > chi[a]) chi[a] = v;
    }
  int axis = 0;
  for (int a = 1; a < 3; ++a)
    if (chi[a] - clo[a] > chi[axis] - clo[axis]) axis = a;
  int64_t mid = b + (e - b) / 2;
  select_mid(t, axis, b, e, mid);
  int64_t l = new_node(t), r = new_node(t);
  nd->left = (int32_t)l;
  nd->right = (int32_t)r;
  if (depth < 12 && e - b > 65536) {
#pragma omp task
    build_rec(t, l, b, mid, depth + 1);
#pragma omp task
    build_rec(t, r, mid, e, depth + 1);
#pragma omp taskwait
  } else {
    build_rec(t, l, b, mid, depth + 1);
    build_rec(t, r, mid, e, depth + 1);
  }
}

void *orc_bvh_build(const float *prims, int64_t n, int kind) {
  ctree *t = (ctree *)calloc(1, sizeof(ctree));
  t->prims = prims;
  t->n = n;
  t->kind = kind;
  t->cap = n > 0 ? 2 * n : 1;
  t->nodes = (cnode *)malloc(sizeof(cnode) * t->cap);
  t->perm = (int64_t *)malloc(sizeof(int64_t) * (n > 0 ? n : 1));
  t->cent = (float *)malloc(sizeof(float) * 3 * (n > 0 ? n : 1));
  for (int64_t i = 0; i < n; ++i) {
    t->perm[i] = i;
    /* double-precision centroid: only orders the split, never a distance */
    if (kind == ORC_POINTS) {
      for (int a = 0; a < 3; ++a) t->cent[3 * i + a] = prims[3 * i + a];
    } else {
      for (int a = 0; a < 3; ++a)
        t->cent[3 * i + a] = (float)(0.5 * ((double)prims[6 * i + a] + (double)prims[6 * i + 3 + a]));
    }
  }
  t->nnodes = 0;
  if (n > 0) {
    int64_t root = new_node(t);
#pragma omp parallel
#pragma omp single
    build_rec(t, root, 0, n, 0);
  }
  return t;
}

void orc_bvh_free(void *h) {
  ctree *t = (ctree *)h;
  if (!t) return;
  free(t->nodes);
  free(t->perm);
  free(t->cent);
  free(t);
}

int64_t orc_bvh_nnodes(void *h) { return ((ctree *)h)->nnodes; }

/* Stack traversal; mode 0 counts, mode 1 fills (ascending index order is
 * NOT guaranteed; rows are sets).  A node is entered iff its box is within r. */
static int64_t bvh_spatial_one(const ctree *t, const float q[3], float r2, int32_t *out) {
  if (t->n == 0 || !finite3(q)) return 0;
  int64_t stack[128];
  int sp = 0;
  int64_t c = 0;
  stack[sp++] = 0;
  while (sp > 0) {
    const cnode *nd = &t->nodes[stack[--sp]];
    if (dist2_box(q, nd->lo, nd->hi) > r2) continue;
    if (nd->left < 0) {
      for (int64_t s = nd->begin; s < nd->end; ++s) {
        int64_t i = t->perm[s];
        if (dist2_prim(t->prims, t->kind, i, q) <= r2) {
          if (out) out[c] = (int32_t)i;
          ++c;
        }
      }
    } else {
      stack[sp++] = nd->right;
      stack[sp++] = nd->left;
    }
  }
  return c;
}

void orc_bvh_spatial_count(void *h, const float *queries, int64_t m, float r, int64_t *counts) {
  const ctree *t = (const ctree *)h;
  float r2 = r * r;
#pragma omp parallel for schedule(dynamic, 256)
  for (int64_t j = 0; j < m; ++j) counts[j] = bvh_spatial_one(t, queries + 3 * j, r2, NULL);
}

void orc_bvh_spatial_fill(void *h, const float *queries, int64_t m, float r, const int64_t *offsets,
                          int32_t *indices) {
  const ctree *t = (const ctree *)h;
  float r2 = r * r;
#pragma omp parallel for schedule(dynamic, 256)
  for (int64_t j = 0; j < m; ++j) bvh_spatial_one(t, queries + 3 * j, r2, indices + offsets[j]);
}

/* Box query on the CPU BVH: a node is entered iff its box meets the query
 * box (its box contains its members' boxes, so no match is skipped). */
static int64_t bvh_intersects_one(const ctree *t, const float *q, int32_t *out) {
  if (t->n == 0) return 0;
  int64_t stack[128];
  int sp = 0;
  int64_t c = 0;
  stack[sp++] = 0;
  while (sp > 0) {
    const cnode *nd = &t->nodes[stack[--sp]];
    if (!boxes_meet(nd->lo, nd->hi, q)) continue;
    if (nd->left < 0) {
      for (int64_t s = nd->begin; s < nd->end; ++s) {
        int64_t i = t->perm[s];
        float lo[3], hi[3];
        prim_box(t->prims, t->kind, i, lo, hi);
        if (boxes_meet(lo, hi, q)) {
          if (out) out[c] = (int32_t)i;
          ++c;
        }
      }
    } else {
      stack[sp++] = nd->right;
      stack[sp++] = nd->left;
    }
  }
  return c;
}

void orc_bvh_intersects_count(void *h, const float *qboxes, int64_t m, int64_t *counts) {
  const ctree *t = (const ctree *)h;
#pragma omp parallel for schedule(dynamic, 256)
  for (int64_t j = 0; j < m; ++j) counts[j] = bvh_intersects_one(t, qboxes + 6 * j, NULL);
}

void orc_bvh_intersects_fill(void *h, const float *qboxes, int64_t m, const int64_t *offsets, int32_t *indices) {
  const ctree *t = (const ctree *)h;
#pragma omp parallel for schedule(dynamic, 256)
  for (int64_t j = 0; j < m; ++j) bvh_intersects_one(t, qboxes + 6 * j, indices + offsets[j]);
}

/* Nearest by stack traversal: the closer child is visited first; a node is
 * skipped when its box distance is strictly larger than the current k-th
 * candidate (an equal one may still hold a lower index). */
void orc_bvh_nearest(void *h, const float *queries, int64_t m, int k, int32_t *indices, float *dist2) {
  const ctree *t = (const ctree *)h;
  int kk = (int)(t->n < k ? t->n : k);
  if (kk <= 0) return;
#pragma omp parallel
  {
    float *ld = (float *)malloc(sizeof(float) * kk);
    int32_t *li = (int32_t *)malloc(sizeof(int32_t) * kk);
#pragma omp for schedule(dynamic, 256)
    for (int64_t j = 0; j < m; ++j) {
      const float *q = queries + 3 * j;
      int len = 0;
      if (finite3(q)) {
        int64_t stack[128];
        float sd[128];
        int sp = 0;
        stack[sp] = 0;
        sd[sp++] = dist2_box(q, t->nodes[0].lo, t->nodes[0].hi);
        while (sp > 0) {
          --sp;
          const cnode *nd = &t->nodes[stack[sp]];
          if (len == kk && sd[sp] > ld[kk - 1]) continue;
          if (nd->left < 0) {
            for (int64_t s = nd->begin; s < nd->end; ++s) {
              int64_t i = t->perm[s];
              len = list_insert(ld, li, len, kk, dist2_prim(t->prims, t->kind, i, q), (int32_t)i);
            }
          } else {
            const cnode *L = &t->nodes[nd->left], *R = &t->nodes[nd->right];
            float dl = dist2_box(q, L->lo, L->hi), dr = dist2_box(q, R->lo, R->hi);
            if (dl <= dr) { /* push the farther first so the closer is popped next */
              stack[sp] = nd->right; sd[sp++] = dr;
              stack[sp] = nd->left; sd[sp++] = dl;
            } else {
              stack[sp] = nd->left; sd[sp++] = dl;
              stack[sp] = nd->right; sd[sp++] = dr;
            }
          }
        }
      }
      for (int s = 0; s < kk; ++s) {
        indices[j * kk + s] = s < len ? li[s] : -1;
        if (dist2) dist2[j * kk + s] = s < len ? ld[s] : INFINITY;
      }
    }
    free(ld);
    free(li);
  }
}

/* ------------------------------------------------------------ FP64 checker */

static inline double gap64(double q, double lo, double hi) {
  if (q < lo) return lo - q;
  if (q > hi) return q - hi;
  return 0.0;
}

static inline double dist_prim64(const float *prims, int kind, int64_t i, const float q[3]) {
  float lo[3], hi[3];
  prim_box(prims, kind, i, lo, hi);
  double s = 0.0;
  for (int a = 0; a < 3; ++a) {
    double g = gap64((double)q[a], (double)lo[a], (double)hi[a]);
    s += g * g;
  }
  return sqrt(s);
}

/* For each sampled query j (sample[t], t < ns): compare the FP32 result row
 * (CSR offsets/indices, original query order) with the FP64 ball d <= r.  A
 * primitive on which they disagree is tolerated only if |d - r| <= rel * r.
 * Returns the number of intolerable disagreements; *tolerated gets the rest. */
int64_t orc_fp64_check_spatial(const float *prims, int64_t n, int kind, const float *queries,
                               const int64_t *sample, int64_t ns, float r, const int64_t *offsets,
                               const int32_t *indices, double rel, int64_t *tolerated) {
  int64_t bad = 0, tol = 0;
  double R = (double)r;
#pragma omp parallel reduction(+ : bad, tol)
  {
    unsigned char *mark = (unsigned char *)calloc(n > 0 ? n : 1, 1);
#pragma omp for schedule(dynamic, 1)
    for (int64_t t = 0; t < ns; ++t) {
      int64_t j = sample[t];
      const float *q = queries + 3 * j;
      for (int64_t s = offsets[j]; s < offsets[j + 1]; ++s) {
        int32_t i = indices[s];
        if (i < 0 || i >= n || mark[i]) { ++bad; continue; } /* out of range or duplicate */
        mark[i] = 1;
      }
      if (finite3(q))
        for (int64_t i = 0; i < n; ++i) {
          double d = dist_prim64(prims, kind, i, q);
          int in64 = d <= R;
          if (in64 != (int)mark[i]) {
            if (fabs(d - R) <= rel * R) ++tol;
            else ++bad;
          }
        }
      else
        for (int64_t s = offsets[j]; s < offsets[j + 1]; ++s) ++bad;
      for (int64_t s = offsets[j]; s < offsets[j + 1]; ++s) {
        int32_t i = indices[s];
        if (i >= 0 && i < n) mark[i] = 0;
      }
    }
    free(mark);
  }
  if (tolerated) *tolerated = tol;
  return bad;
}

/* kk-th smallest of d[0..n) by a bounded ascending insertion list */
static double kth_smallest(const double *d, int64_t n, int kk, double *buf) {
  int len = 0;
  for (int64_t i = 0; i < n; ++i) {
    double v = d[i];
    if (len == kk && !(v < buf[kk - 1])) continue;
    int pos = len < kk ? len : kk - 1;
    while (pos > 0 && v < buf[pos - 1]) {
      buf[pos] = buf[pos - 1];
      --pos;
    }
    buf[pos] = v;
    if (len < kk) ++len;
  }
  return buf[kk - 1];
}

/* Nearest check in FP64: D_k = the k-th smallest FP64 distance.  Every returned
 * index must satisfy d <= D_k (1 + rel), and every primitive with
 * d < D_k (1 - rel) must be returned; rows have kk = min(k, n) distinct entries. */
int64_t orc_fp64_check_nearest(const float *prims, int64_t n, int kind, const float *queries,
                               const int64_t *sample, int64_t ns, int k, const int32_t *indices,
                               double rel, int64_t *tolerated) {
  int kk = (int)(n < k ? n : k);
  int64_t bad = 0, tol = 0;
  if (kk <= 0) return 0;
#pragma omp parallel reduction(+ : bad, tol)
  {
    double *d = (double *)malloc(sizeof(double) * (n > 0 ? n : 1));
    double *buf = (double *)malloc(sizeof(double) * kk);
    unsigned char *mark = (unsigned char *)calloc(n > 0 ? n : 1, 1);
#pragma omp for schedule(dynamic, 1)
    for (int64_t t = 0; t < ns; ++t) {
      int64_t j = sample[t];
      const float *q = queries + 3 * j;
      const int32_t *row = indices + j * kk;
      if (!finite3(q)) {
        for (int s = 0; s < kk; ++s) bad += row[s] != -1;
        continue;
      }
      for (int64_t i = 0; i < n; ++i) d[i] = dist_prim64(prims, kind, i, q);
      double Dk = kth_smallest(d, n, kk, buf);
      for (int s = 0; s < kk; ++s) {
        int32_t i = row[s];
        if (i < 0 || i >= n || mark[i]) { ++bad; continue; }
        mark[i] = 1;
        if (d[i] > Dk) {
          if (d[i] <= Dk * (1.0 + rel)) ++tol;
          else ++bad;
        }
      }
      for (int64_t i = 0; i < n; ++i)
        if (!mark[i] && d[i] < Dk) {
          if (d[i] >= Dk * (1.0 - rel)) ++tol;
          else ++bad;
        }
      for (int s = 0; s < kk; ++s) {
        int32_t i = row[s];
        if (i >= 0 && i < n) mark[i] = 0;
      }
    }
    free(d);
    free(buf);
    free(mark);
  }
  if (tolerated) *tolerated = tol;
  return bad;
}

/*
 * emst_oracle.c -- plain, slow, obviously-correct CPU oracle for the
 * single-tree Boruvka EMST (Prokopenko, Sao, Lebrun-Grandie, arXiv 2207.00514).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  The product path (the
 * CUDA library) never calls it, links it, or shares a line of code with it.
 *
 * Every function follows one passage of the paper and says which.  Floating
 * point is FP32 only where the method fixes it (the edge weight and the
 * Morton quantisation, which both sides must decide in the same precision);
 * everything else is integer work or exact min/max comparisons.
 *
 * Compile with -ffp-contract=off (no implicit fma contraction): the weight
 * below spells out its fma order explicitly.
 *
 * Readings of the paper taken here (the paper is silent or informal on them):
 *  - weight: the paper's w_ij = ||p_i - p_j||_2 (§2, "EMST computation") is
 *    replaced by the FP32 squared distance  w = fma(dz,dz, fma(dy,dy, dx*dx))
 *    (2D: fma(dy,dy, dx*dx)), dx = x_i - x_j in FP32.  Squaring preserves the
 *    order of lengths, so the spanning tree is the same.
 *  - edge order: (w, min(i,j), max(i,j)) lexicographic, the tie-break of §2
 *    ("Boruvka's algorithm", last paragraph).  Under this strict total order
 *    the MST is unique (§2, "MST computation").
 *  - ids are the caller's original point indices.
 *  - mutual reachability (§4.5): d_core(u) is the distance to u's k_pts-th
 *    nearest neighbour counting u itself, and the weight of (u, v) is
 *    max(d_core(u), d_core(v), ||u - v||).  Kept squared like the EMST
 *    weight: core2(u) = the (k_pts - 1)-th smallest w(u, v) over v != u
 *    (0 for k_pts = 1), and w_m(u, v) = max(core2(u), core2(v), w(u, v)); the
 *    order (w_m, min id, max id) is the same tie-break.  k_pts = 1 gives the
 *    EMST itself.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  uint32_t i, j;
  float w;
} oracle_edge;

#define ORACLE_INVALID 0xFFFFFFFFu

/* ------------------------------------------------------------------------ */
/* Edge weight and the total order on edges (§2)                            */
/* ------------------------------------------------------------------------ */

float oracle_weight(const float *p, const float *q, int dim) {
  float dx = p[0] - q[0];
  float s = dx * dx;
  float dy = p[1] - q[1];
  s = fmaf(dy, dy, s);
  if (dim == 3) {
    float dz = p[2] - q[2];
    s = fmaf(dz, dz, s);
  }
  return s;
}

/* -1 / 0 / +1 comparing (w1, min1, max1) with (w2, min2, max2). */
static int key_cmp(float w1, uint32_t a1, uint32_t b1, float w2, uint32_t a2, uint32_t b2) {
  uint32_t lo1 = a1 < b1 ? a1 : b1, hi1 = a1 < b1 ? b1 : a1;
  uint32_t lo2 = a2 < b2 ? a2 : b2, hi2 = a2 < b2 ? b2 : a2;
  if (w1 < w2) return -1;
  if (w1 > w2) return 1;
  if (lo1 < lo2) return -1;
  if (lo1 > lo2) return 1;
  if (hi1 < hi2) return -1;
  if (hi1 > hi2) return 1;
  return 0;
}

static int edge_qsort_cmp(const void *x, const void *y) {
  const oracle_edge *a = (const oracle_edge *)x, *b = (const oracle_edge *)y;
  return key_cmp(a->w, a->i, a->j, b->w, b->i, b->j);
}

/* Put every edge as (min id, max id) and sort by the total order. */
void oracle_canonical_sort(oracle_edge *e, int64_t m) {
  for (int64_t k = 0; k < m; ++k) {
    if (e[k].i > e[k].j) {
      uint32_t t = e[k].i;
      e[k].i = e[k].j;
      e[k].j = t;
    }
  }
  qsort(e, (size_t)m, sizeof(oracle_edge), edge_qsort_cmp);
}

/* ------------------------------------------------------------------------ */
/* Reference EMSTs by definition                                            */
/* ------------------------------------------------------------------------ */

/* Prim's algorithm on the complete distance graph, O(n^2) (§2, "MST
 * computation": grow one component by its minimum-weight cut edge).  Each
 * outside vertex v keeps its best edge to the tree as (w, u); the next vertex
 * is the one whose best edge is smallest under the full key.  Output: n-1
 * edges in the order they were added. */
/* The edge weight: the squared distance, or with core2 != NULL the squared
 * mutual reachability distance (§4.5). */
static float edge_weight(const float *pts, const float *core2, int64_t u, int64_t v, int dim) {
  float w = oracle_weight(pts + u * dim, pts + v * dim, dim);
  if (core2) {
    if (core2[u] > w) w = core2[u];
    if (core2[v] > w) w = core2[v];
  }
  return w;
}

static int prim_impl(const float *pts, const float *core2, int64_t n, int dim, oracle_edge *out) {
  if (n <= 1) return 0;
  float *bw = (float *)malloc(sizeof(float) * (size_t)n);
  uint32_t *bu = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n);
  unsigned char *in = (unsigned char *)calloc((size_t)n, 1);
  if (!bw || !bu || !in) { free(bw); free(bu); free(in); return -1; }
  in[0] = 1;
  for (int64_t v = 1; v < n; ++v) {
    bw[v] = edge_weight(pts, core2, 0, v, dim);
    bu[v] = 0;
  }
  for (int64_t step = 0; step < n - 1; ++step) {
    int64_t pick = -1;
    for (int64_t v = 0; v < n; ++v) {
      if (in[v]) continue;
      if (pick < 0 || key_cmp(bw[v], (uint32_t)v, bu[v], bw[pick], (uint32_t)pick, bu[pick]) < 0)
        pick = v;
    }
    in[pick] = 1;
    out[step].i = bu[pick];
    out[step].j = (uint32_t)pick;
    out[step].w = bw[pick];
    for (int64_t v = 0; v < n; ++v) {
      if (in[v]) continue;
      float w = edge_weight(pts, core2, pick, v, dim);
      if (key_cmp(w, (uint32_t)v, (uint32_t)pick, bw[v], (uint32_t)v, bu[v]) < 0) {
        bw[v] = w;
        bu[v] = (uint32_t)pick;
      }
    }
  }
  free(bw);
  free(bu);
  free(in);
  return 0;
}

int oracle_prim(const float *pts, int64_t n, int dim, oracle_edge *out) {
  return prim_impl(pts, NULL, n, dim, out);
}

/* Prim on the mutual reachability weights (§4.5), core2 as above. */
int oracle_prim_mrd(const float *pts, const float *core2, int64_t n, int dim, oracle_edge *out) {
  return prim_impl(pts, core2, n, dim, out);
}

/* Union-find with path halving and union by index (smaller root wins). */
static uint32_t uf_find(uint32_t *par, uint32_t x) {
  while (par[x] != x) {
    par[x] = par[par[x]];
    x = par[x];
  }
  return x;
}

/* Kruskal's algorithm over all n(n-1)/2 pairs (§2, "MST computation"): sort
 * every edge by the total order, keep those joining two different trees. */
static int kruskal_impl(const float *pts, const float *core2, int64_t n, int dim,
                        oracle_edge *out) {
  if (n <= 1) return 0;
  int64_t m = n * (n - 1) / 2;
  oracle_edge *all = (oracle_edge *)malloc(sizeof(oracle_edge) * (size_t)m);
  uint32_t *par = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n);
  if (!all || !par) { free(all); free(par); return -1; }
  int64_t k = 0;
  for (int64_t a = 0; a < n; ++a)
    for (int64_t b = a + 1; b < n; ++b) {
      all[k].i = (uint32_t)a;
      all[k].j = (uint32_t)b;
      all[k].w = edge_weight(pts, core2, a, b, dim);
      ++k;
    }
  qsort(all, (size_t)m, sizeof(oracle_edge), edge_qsort_cmp);
  for (int64_t v = 0; v < n; ++v) par[v] = (uint32_t)v;
  int64_t got = 0;
  for (k = 0; k < m && got < n - 1; ++k) {
    uint32_t ra = uf_find(par, all[k].i), rb = uf_find(par, all[k].j);
    if (ra == rb) continue;
    if (ra < rb) par[rb] = ra; else par[ra] = rb;
    out[got++] = all[k];
  }
  free(all);
  free(par);
  return got == n - 1 ? 0 : -2;
}

int oracle_kruskal(const float *pts, int64_t n, int dim, oracle_edge *out) {
  return kruskal_impl(pts, NULL, n, dim, out);
}

int oracle_kruskal_mrd(const float *pts, const float *core2, int64_t n, int dim,
                       oracle_edge *out) {
  return kruskal_impl(pts, core2, n, dim, out);
}

/* Core distances (§4.5), by definition: for each u, the (k - 1)-th smallest
 * weight w(u, v) over all v != u (u itself is the first neighbour, at 0), by
 * a full selection over all n - 1 others.  k = 1: 0.  Returns -1 for k < 1 or
 * k > n. */
static int cmp_float(const void *x, const void *y) {
  float a = *(const float *)x, b = *(const float *)y;
  return (a > b) - (a < b);
}

int oracle_core_dist2_brute(const float *pts, int64_t n, int dim, int k, float *core2) {
  if (k < 1 || k > n) return -1;
  float *w = (float *)malloc(sizeof(float) * (size_t)(n > 1 ? n - 1 : 1));
  if (!w) return -1;
  for (int64_t u = 0; u < n; ++u) {
    if (k == 1) { core2[u] = 0.0f; continue; }
    int64_t m = 0;
    for (int64_t v = 0; v < n; ++v)
      if (v != u) w[m++] = oracle_weight(pts + u * dim, pts + v * dim, dim);
    qsort(w, (size_t)m, sizeof(float), cmp_float);
    core2[u] = w[k - 2];
  }
  free(w);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Per-step definitions of the paper's hot path                             */
/* ------------------------------------------------------------------------ */

/* A1. Scene bounding box: per-dimension min and max over all points (the
 * box the Z-curve linearisation quantises, §2 "ArborX").  Returns 1 if every
 * coordinate is finite, else 0. */
int oracle_scene_box(const float *pts, int64_t n, int dim, float *lo, float *hi) {
  int finite = 1;
  for (int d = 0; d < dim; ++d) {
    lo[d] = INFINITY;
    hi[d] = -INFINITY;
  }
  for (int64_t k = 0; k < n; ++k)
    for (int d = 0; d < dim; ++d) {
      float x = pts[k * dim + d];
      if (!isfinite(x)) { finite = 0; continue; }
      if (x < lo[d]) lo[d] = x;
      if (x > hi[d]) hi[d] = x;
    }
  return finite;
}

/* A2. Morton (Z-curve) code of each point (§2 "ArborX"; 64-bit codes, §4.1).
 * Quantisation (the paper does not print one; this is the reading used by
 * both sides, decided in FP32): with B = 21 bits per dimension in 3D and
 * B = 32 in 2D,
 *     s_d = 2^B / (hi_d - lo_d)            (0 if hi_d == lo_d)
 *     t   = (x_d - lo_d) * s_d             (FP32, each op rounded)
 *     q_d = t >= 2^B ? 2^B - 1 : floor(t)
 * and the code interleaves the bits of q, most significant first, x before y
 * before z: bit (dim*b + dim-1-d) of the code is bit b of q_d. */
void oracle_morton(const float *pts, int64_t n, int dim, const float *lo, const float *hi,
                   uint64_t *codes) {
  int B = dim == 3 ? 21 : 32;
  float twoB = dim == 3 ? 2097152.0f : 4294967296.0f;
  uint64_t qmax = (dim == 3) ? ((1ull << 21) - 1) : 0xFFFFFFFFull;
  float s[3] = {0.f, 0.f, 0.f};
  for (int d = 0; d < dim; ++d) {
    float ext = hi[d] - lo[d];
    s[d] = ext > 0.0f ? twoB / ext : 0.0f;
  }
  for (int64_t k = 0; k < n; ++k) {
    uint64_t q[3] = {0, 0, 0};
    for (int d = 0; d < dim; ++d) {
      float diff = pts[k * dim + d] - lo[d];
      float t = diff * s[d];
      q[d] = (t >= twoB) ? qmax : (uint64_t)t;
    }
    uint64_t code = 0;
    for (int b = 0; b < B; ++b)
      for (int d = 0; d < dim; ++d)
        code |= ((q[d] >> b) & 1ull) << (dim * b + (dim - 1 - d));
    codes[k] = code;
  }
}

/* A2 at the finer grid §4.2 suggests for very dense data ("128-bit Morton
 * codes instead of 64-bit ones"): B = 42 bits per dimension in 3D, 64 in 2D.
 * The quantiser runs in FP64 so the finer grid resolves FP32 coordinates
 * (x - lo of two FP32 values is exact in FP64 unless their exponents are far
 * apart): s = 2^B / (hi - lo) (0 for a flat dimension), t = (x - lo) * s,
 * q = t >= 2^B ? 2^B - 1 : floor(t); bits interleaved x most significant, the
 * 128-bit code split into a high and a low 64-bit word. */
void oracle_morton128(const float *pts, int64_t n, int dim, const float *lo, const float *hi,
                      uint64_t *code_hi, uint64_t *code_lo) {
  const int B = dim == 3 ? 42 : 64;
  const double twoB = ldexp(1.0, B);
  const uint64_t qmax = B == 64 ? ~0ull : ((1ull << B) - 1);
  double s[3] = {0.0, 0.0, 0.0};
  for (int d = 0; d < dim; ++d) {
    double ext = (double)hi[d] - (double)lo[d];
    s[d] = ext > 0.0 ? twoB / ext : 0.0;
  }
  for (int64_t k = 0; k < n; ++k) {
    uint64_t q[3] = {0, 0, 0};
    for (int d = 0; d < dim; ++d) {
      double t = ((double)pts[k * dim + d] - (double)lo[d]) * s[d];
      q[d] = (t >= twoB) ? qmax : (uint64_t)t;
    }
    uint64_t ch = 0, cl = 0;
    for (int b = 0; b < B; ++b)
      for (int d = 0; d < dim; ++d) {
        int pos = dim * b + (dim - 1 - d);
        uint64_t bit = (q[d] >> b) & 1ull;
        if (pos < 64) cl |= bit << pos;
        else ch |= bit << (pos - 64);
      }
    code_hi[k] = ch;
    code_lo[k] = cl;
  }
}

/* A3. Sort along the Z-curve: the stable order of the codes (equal codes keep
 * their input order).  perm[k] = input index of the k-th point in order. */
static const uint64_t *g_sort_codes;
static int perm_cmp(const void *x, const void *y) {
  uint32_t a = *(const uint32_t *)x, b = *(const uint32_t *)y;
  if (g_sort_codes[a] < g_sort_codes[b]) return -1;
  if (g_sort_codes[a] > g_sort_codes[b]) return 1;
  return a < b ? -1 : (a > b ? 1 : 0);
}
void oracle_sort_perm(const uint64_t *codes, int64_t n, uint32_t *perm) {
  for (int64_t k = 0; k < n; ++k) perm[k] = (uint32_t)k;
  g_sort_codes = codes;
  qsort(perm, (size_t)n, sizeof(uint32_t), perm_cmp);
}

/* A3 for 128-bit codes: stable order of (hi, lo). */
static const uint64_t *g_sort_hi, *g_sort_lo;
static int perm_cmp128(const void *x, const void *y) {
  uint32_t a = *(const uint32_t *)x, b = *(const uint32_t *)y;
  if (g_sort_hi[a] != g_sort_hi[b]) return g_sort_hi[a] < g_sort_hi[b] ? -1 : 1;
  if (g_sort_lo[a] != g_sort_lo[b]) return g_sort_lo[a] < g_sort_lo[b] ? -1 : 1;
  return a < b ? -1 : (a > b ? 1 : 0);
}
void oracle_sort_perm128(const uint64_t *code_hi, const uint64_t *code_lo, int64_t n,
                         uint32_t *perm) {
  for (int64_t k = 0; k < n; ++k) perm[k] = (uint32_t)k;
  g_sort_hi = code_hi;
  g_sort_lo = code_lo;
  qsort(perm, (size_t)n, sizeof(uint32_t), perm_cmp128);
}

/* A4. Binary radix tree over the sorted codes (the linear BVH hierarchy of
 * §2 "ArborX": n leaves, n-1 internal nodes), by its definition, top-down:
 * the node covering sorted positions [a, b] splits after the last position s
 * whose augmented key still shares with key a more leading bits than key b
 * does.  Keys are augmented by their position, so equal codes still split.
 * Node numbering (the one drawn in Fig. 4): the root is 0; an internal child
 * covering [a, s] is numbered s, one covering [s+1, b] is numbered s+1.
 * Output per internal node: children as refs (internal id in [0, n-1), leaf
 * k as n-1+k) and the covered range [first, last]. */

/* a != b: leading bits shared by the augmented keys (code, position); with
 * h != NULL the code is 128 bits, h its high word */
static int prefix_len2(const uint64_t *h, const uint64_t *c, int64_t a, int64_t b) {
  int base = 0;
  if (h) {
    if (h[a] != h[b]) return __builtin_clzll(h[a] ^ h[b]);
    base = 64;
  }
  if (c[a] != c[b]) return base + __builtin_clzll(c[a] ^ c[b]);
  return base + 64 + __builtin_clz((uint32_t)a ^ (uint32_t)b);
}

static void radix_tree_impl(const uint64_t *sorted_hi, const uint64_t *sorted_codes, int64_t n,
                            int64_t *left, int64_t *right, int64_t *first, int64_t *last);

void oracle_radix_tree(const uint64_t *sorted_codes, int64_t n, int64_t *left, int64_t *right,
                       int64_t *first, int64_t *last) {
  radix_tree_impl(NULL, sorted_codes, n, left, right, first, last);
}

void oracle_radix_tree128(const uint64_t *sorted_hi, const uint64_t *sorted_lo, int64_t n,
                          int64_t *left, int64_t *right, int64_t *first, int64_t *last) {
  radix_tree_impl(sorted_hi, sorted_lo, n, left, right, first, last);
}

static void radix_tree_impl(const uint64_t *sorted_hi, const uint64_t *sorted_codes, int64_t n,
                            int64_t *left, int64_t *right, int64_t *first, int64_t *last) {
  if (n < 2) return;
  /* explicit stack of (node id, a, b) */
  int64_t cap = 2 * n + 8;
  int64_t *st = (int64_t *)malloc(sizeof(int64_t) * 3 * (size_t)cap);
  int64_t sp = 0;
  st[0] = 0; st[1] = 0; st[2] = n - 1; sp = 1;
  while (sp > 0) {
    --sp;
    int64_t id = st[3 * sp], a = st[3 * sp + 1], b = st[3 * sp + 2];
    first[id] = a;
    last[id] = b;
    int common = prefix_len2(sorted_hi, sorted_codes, a, b);
    int64_t s = a;
    for (int64_t k = a + 1; k < b; ++k)
      if (prefix_len2(sorted_hi, sorted_codes, a, k) > common) s = k;
    /* left child [a, s], right child [s+1, b] */
    if (s == a) left[id] = (n - 1) + a;
    else { left[id] = s; st[3 * sp] = s; st[3 * sp + 1] = a; st[3 * sp + 2] = s; ++sp; }
    if (s + 1 == b) right[id] = (n - 1) + b;
    else { right[id] = s + 1; st[3 * sp] = s + 1; st[3 * sp + 1] = s + 1; st[3 * sp + 2] = b; ++sp; }
  }
  free(st);
}

/* A4 (refit). Bounding box of every internal node: min / max over the points
 * of its leaf range (sorted_pts are the points in sorted order). */
void oracle_node_boxes(const float *sorted_pts, const int64_t *first, const int64_t *last,
                       int64_t n, int dim, float *lo, float *hi) {
  for (int64_t v = 0; v + 1 < n; ++v)
    for (int d = 0; d < dim; ++d) {
      float mn = INFINITY, mx = -INFINITY;
      for (int64_t k = first[v]; k <= last[v]; ++k) {
        float x = sorted_pts[k * dim + d];
        if (x < mn) mn = x;
        if (x > mx) mx = x;
      }
      lo[v * dim + d] = mn;
      hi[v * dim + d] = mx;
    }
}

/* A5. Node label (§3, Optimization 1 and Fig. 4): the label shared by every
 * leaf of the node's subtree, or INVALID when two leaves differ.  labels[k]
 * is the component label of the k-th point in sorted order. */
void oracle_node_labels(const uint32_t *labels, const int64_t *first, const int64_t *last,
                        int64_t n, uint32_t *node_label) {
  for (int64_t v = 0; v + 1 < n; ++v) {
    uint32_t l = labels[first[v]];
    for (int64_t k = first[v] + 1; k <= last[v]; ++k)
      if (labels[k] != l) { l = ORACLE_INVALID; break; }
    node_label[v] = l;
  }
}

/* A6. Component upper bounds (§3, Optimization 2): for every pair of points
 * adjacent on the curve with different labels, the pair's weight bounds the
 * shortest outgoing edge of both components.  ub[label] = min over such
 * pairs, +inf where a label has none. */
void oracle_upper_bounds(const float *sorted_pts, const uint32_t *labels, int64_t n, int dim,
                         float *ub) {
  for (int64_t k = 0; k < n; ++k) ub[k] = INFINITY;
  for (int64_t k = 0; k + 1 < n; ++k) {
    if (labels[k] == labels[k + 1]) continue;
    float w = oracle_weight(sorted_pts + k * dim, sorted_pts + (k + 1) * dim, dim);
    if (w < ub[labels[k]]) ub[labels[k]] = w;
    if (w < ub[labels[k + 1]]) ub[labels[k + 1]] = w;
  }
}

/* A7. Per-point query of Algorithm 2, by brute force: among points j with
 * labels[j] != labels[i] and w(i,j) <= radius[i] (inclusive, Algorithm 2's
 * acceptance test), the one with the smallest (w, orig id of j); for a fixed i
 * that is the smallest key (w, min, max) of §2.  out_j = sorted index of the
 * neighbour or -1 if none is within the radius. */
void oracle_nn_other(const float *sorted_pts, const uint32_t *orig_ids, const uint32_t *labels,
                     const float *radius, int64_t n, int dim, float *out_w, int64_t *out_j) {
  for (int64_t i = 0; i < n; ++i) {
    float bw = INFINITY;
    int64_t bj = -1;
    for (int64_t j = 0; j < n; ++j) {
      if (labels[j] == labels[i]) continue;
      float w = oracle_weight(sorted_pts + i * dim, sorted_pts + j * dim, dim);
      if (!(w <= radius[i])) continue;
      if (bj < 0 || w < bw || (w == bw && orig_ids[j] < orig_ids[bj])) {
        bw = w;
        bj = j;
      }
    }
    out_w[i] = bj < 0 ? INFINITY : bw;
    out_j[i] = bj;
  }
}

/* A8. Shortest outgoing edge of each component (Algorithm 1, the minimum over
 * S; Algorithm 2's final update): the smallest key (w, min id, max id) over
 * the per-point results of the component's points.  Indexed by label value;
 * comp_a = sorted index of the endpoint inside the component, comp_b = the
 * one outside, -1 where the label has no edge. */
void oracle_component_min(const uint32_t *labels, const uint32_t *orig_ids, const float *res_w,
                          const int64_t *res_j, int64_t n, float *comp_w, int64_t *comp_a,
                          int64_t *comp_b) {
  for (int64_t c = 0; c < n; ++c) { comp_w[c] = INFINITY; comp_a[c] = -1; comp_b[c] = -1; }
  for (int64_t i = 0; i < n; ++i) {
    if (res_j[i] < 0) continue;
    uint32_t c = labels[i];
    if (comp_a[c] < 0 ||
        key_cmp(res_w[i], orig_ids[i], orig_ids[res_j[i]], comp_w[c], orig_ids[comp_a[c]],
                orig_ids[comp_b[c]]) < 0) {
      comp_w[c] = res_w[i];
      comp_a[c] = i;
      comp_b[c] = res_j[i];
    }
  }
}

/* A9. Merge (§3, "Merging components together"; the chains of §2): every
 * component C points to T(C) = label of the outside endpoint of its edge.
 * Each point follows the chain from its component until the terminal pair
 * X <-> T(X) and takes the smaller label of the pair.  (When a radius cut
 * the queries short, a component may have no edge; a chain ends there and
 * keeps that component's label.  In the full method every component has an
 * edge.)  The chosen edges are
 * emitted once each (a mutual pair shares one edge).  Returns the number of
 * emitted edges, or -1 if some chain is longer than n (impossible under a
 * strict total order). */
int64_t oracle_merge(const uint32_t *labels, const int64_t *comp_a, const int64_t *comp_b,
                     const float *comp_w, const uint32_t *orig_ids, int64_t n,
                     uint32_t *new_labels, oracle_edge *out_edges) {
  uint32_t *T = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n);
  for (int64_t c = 0; c < n; ++c) T[c] = comp_b[c] >= 0 ? labels[comp_b[c]] : ORACLE_INVALID;
  int64_t emitted = 0;
  for (int64_t c = 0; c < n; ++c) {
    if (comp_b[c] < 0) continue;
    uint32_t t = T[c];
    int mutual = (T[t] == (uint32_t)c);
    if (mutual && (uint32_t)c > t) continue; /* the pair's edge is emitted by its smaller side */
    uint32_t oi = orig_ids[comp_a[c]], oj = orig_ids[comp_b[c]];
    out_edges[emitted].i = oi < oj ? oi : oj;
    out_edges[emitted].j = oi < oj ? oj : oi;
    out_edges[emitted].w = comp_w[c];
    ++emitted;
  }
  for (int64_t k = 0; k < n; ++k) {
    /* follow C -> T(C) -> ... ; a component without an edge (possible only
     * when queries were cut off by a radius) ends its chain */
    uint32_t x = labels[k];
    int64_t steps = 0;
    for (;;) {
      uint32_t t = T[x];
      if (t == ORACLE_INVALID) { new_labels[k] = x; break; }
      if (T[t] == x) { new_labels[k] = x < t ? x : t; break; }
      x = t;
      if (++steps > n) { free(T); return -1; }
    }
  }
  free(T);
  return emitted;
}

/* ------------------------------------------------------------------------ */
/* Boruvka by the per-step definitions (Fig. 3 loop, brute-force queries).  */
/* Points are taken in the order given (the caller may pass them sorted);   */
/* ids are positions in that order unless orig_ids is given.                */
/* ------------------------------------------------------------------------ */
int oracle_boruvka_steps(const float *pts, const uint32_t *orig_ids_in, int64_t n, int dim,
                         oracle_edge *out, int64_t *rounds_out) {
  if (n <= 1) { if (rounds_out) *rounds_out = 0; return 0; }
  uint32_t *ids = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n);
  uint32_t *lab = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n);
  uint32_t *lab2 = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n);
  float *ub = (float *)malloc(sizeof(float) * (size_t)n);
  float *rw = (float *)malloc(sizeof(float) * (size_t)n);
  float *rad = (float *)malloc(sizeof(float) * (size_t)n);
  int64_t *rj = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
  float *cw = (float *)malloc(sizeof(float) * (size_t)n);
  int64_t *ca = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
  int64_t *cb = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
  for (int64_t k = 0; k < n; ++k) { ids[k] = orig_ids_in ? orig_ids_in[k] : (uint32_t)k; lab[k] = (uint32_t)k; }
  int64_t got = 0, rounds = 0;
  int status = 0;
  while (got < n - 1) {
    oracle_upper_bounds(pts, lab, n, dim, ub);
    for (int64_t k = 0; k < n; ++k) rad[k] = ub[lab[k]];
    oracle_nn_other(pts, ids, lab, rad, n, dim, rw, rj);
    oracle_component_min(lab, ids, rw, rj, n, cw, ca, cb);
    int64_t e = oracle_merge(lab, ca, cb, cw, ids, n, lab2, out + got);
    if (e <= 0) { status = -2; break; }
    got += e;
    memcpy(lab, lab2, sizeof(uint32_t) * (size_t)n);
    if (++rounds > 64) { status = -3; break; }
  }
  if (rounds_out) *rounds_out = rounds;
  free(ids); free(lab); free(lab2); free(ub); free(rw); free(rad); free(rj); free(cw); free(ca); free(cb);
  return status;
}

/* ------------------------------------------------------------------------ */
/* k-d tree Boruvka: the large-n oracle.  Same MST definition, a different   */
/* data structure (median-split k-d tree, union-find components) and plain  */
/* sequential control; the per-point queries may run on several threads,    */
/* with results that do not depend on the thread count.                     */
/* ------------------------------------------------------------------------ */
typedef struct {
  float lo[3], hi[3];
  int64_t begin, end; /* points idx[begin, end) */
  int64_t left, right; /* child node ids or -1 */
} kd_node;

typedef struct {
  const float *pts;
  int dim;
  int64_t n;
  uint32_t *idx;
  kd_node *nodes;
  int64_t n_nodes;
  int max_depth;
} kd_tree;

#define KD_LEAF 8

static float coord(const kd_tree *t, uint32_t p, int d) { return t->pts[(int64_t)p * t->dim + d]; }

/* three-way quickselect of idx[b, e) on dimension d so that position m holds
 * the m-th smallest coordinate */
static void kd_select(kd_tree *t, int64_t b, int64_t e, int64_t m, int d) {
  uint32_t *a = t->idx;
  while (e - b > 1) {
    float p0 = coord(t, a[b], d), p1 = coord(t, a[b + (e - b) / 2], d), p2 = coord(t, a[e - 1], d);
    float piv = p0 < p1 ? (p1 < p2 ? p1 : (p0 < p2 ? p2 : p0)) : (p0 < p2 ? p0 : (p1 < p2 ? p2 : p1));
    int64_t lt = b, i = b, gt = e;
    while (i < gt) {
      float x = coord(t, a[i], d);
      if (x < piv) { uint32_t s = a[lt]; a[lt] = a[i]; a[i] = s; ++lt; ++i; }
      else if (x > piv) { --gt; uint32_t s = a[gt]; a[gt] = a[i]; a[i] = s; }
      else ++i;
    }
    if (m < lt) e = lt;
    else if (m >= gt) b = gt;
    else return;
  }
}

static int64_t kd_build_rec(kd_tree *t, int64_t b, int64_t e, int depth) {
  int64_t id = t->n_nodes++;
  kd_node *nd = &t->nodes[id];
  if (depth > t->max_depth) t->max_depth = depth;
  for (int d = 0; d < t->dim; ++d) { nd->lo[d] = INFINITY; nd->hi[d] = -INFINITY; }
  for (int64_t k = b; k < e; ++k)
    for (int d = 0; d < t->dim; ++d) {
      float x = coord(t, t->idx[k], d);
      if (x < nd->lo[d]) nd->lo[d] = x;
      if (x > nd->hi[d]) nd->hi[d] = x;
    }
  nd->begin = b;
  nd->end = e;
  nd->left = nd->right = -1;
  if (e - b <= KD_LEAF) return id;
  int sd = 0;
  double best = -1.0;
  for (int d = 0; d < t->dim; ++d) {
    double ext = (double)nd->hi[d] - (double)nd->lo[d];
    if (ext > best) { best = ext; sd = d; }
  }
  if (best <= 0.0) return id; /* all points coincide: one (large) leaf */
  int64_t m = b + (e - b) / 2;
  kd_select(t, b, e, m, sd);
  int64_t l = kd_build_rec(t, b, m, depth + 1);
  int64_t r = kd_build_rec(t, m, e, depth + 1);
  t->nodes[id].left = l;
  t->nodes[id].right = r;
  return id;
}

/* Lower bound of the weight from p to any point in the node's box: the same
 * fma order on p - clamp(p, lo, hi).  Per dimension |p - clamp| <= |p - q| for
 * every q in the box, rounding is monotone and fma / mul are monotone in
 * non-negative operands, so this never exceeds the weight to a point inside. */
static float box_weight(const float *p, const kd_node *nd, int dim) {
  float c0 = p[0] < nd->lo[0] ? nd->lo[0] : (p[0] > nd->hi[0] ? nd->hi[0] : p[0]);
  float c1 = p[1] < nd->lo[1] ? nd->lo[1] : (p[1] > nd->hi[1] ? nd->hi[1] : p[1]);
  float dx = p[0] - c0;
  float s = dx * dx;
  float dy = p[1] - c1;
  s = fmaf(dy, dy, s);
  if (dim == 3) {
    float c2 = p[2] < nd->lo[2] ? nd->lo[2] : (p[2] > nd->hi[2] ? nd->hi[2] : p[2]);
    float dz = p[2] - c2;
    s = fmaf(dz, dz, s);
  }
  return s;
}

typedef struct {
  kd_tree *t;
  const float *core2;        /* squared core distances (mutual reachability), or NULL */
  const uint32_t *comp;      /* component root per point (original index) */
  const uint32_t *node_comp; /* component of a single-component node, else INVALID */
  uint32_t *comp_radius;     /* float bits of the best weight found so far per component */
  float *res_w;
  uint32_t *res_j;
  int64_t begin, end; /* range of positions in idx order */
} kd_job;

static void atomic_min_u32(uint32_t *a, uint32_t v) {
  uint32_t cur = __atomic_load_n(a, __ATOMIC_RELAXED);
  while (v < cur && !__atomic_compare_exchange_n(a, &cur, v, 1, __ATOMIC_RELAXED, __ATOMIC_RELAXED)) {
  }
}

static uint32_t f2u(float f) { uint32_t u; memcpy(&u, &f, 4); return u; }
static float u2f(uint32_t u) { float f; memcpy(&f, &u, 4); return f; }

static void *kd_query_range(void *arg) {
  kd_job *job = (kd_job *)arg;
  kd_tree *t = job->t;
  int dim = t->dim;
  int64_t *stack = (int64_t *)malloc(sizeof(int64_t) * (size_t)(2 * t->max_depth + 8));
  for (int64_t pos = job->begin; pos < job->end; ++pos) {
    uint32_t i = t->idx[pos];
    uint32_t c = job->comp[i];
    const float *p = t->pts + (int64_t)i * dim;
    /* with core distances every weight from i is at least core2[i] */
    const float wi = job->core2 ? job->core2[i] : 0.0f;
    float best_w = INFINITY;
    uint32_t best_j = ORACLE_INVALID;
    int64_t sp = 0;
    stack[sp++] = 0;
    while (sp > 0) {
      int64_t v = stack[--sp];
      const kd_node *nd = &t->nodes[v];
      if (job->node_comp[v] == c) continue; /* every point here is in i's component */
      float radius = u2f(__atomic_load_n(&job->comp_radius[c], __ATOMIC_RELAXED));
      if (best_w < radius) radius = best_w;
      float lb = box_weight(p, nd, dim);
      if (wi > lb) lb = wi;
      if (lb > radius) continue;
      if (nd->left < 0) {
        for (int64_t k = nd->begin; k < nd->end; ++k) {
          uint32_t j = t->idx[k];
          if (job->comp[j] == c) continue;
          float w = edge_weight(t->pts, job->core2, i, j, dim);
          if (w > radius) continue;
          if (w < best_w || (w == best_w && j < best_j)) {
            best_w = w;
            best_j = j;
            radius = w;
          }
        }
        continue;
      }
      const kd_node *L = &t->nodes[nd->left], *R = &t->nodes[nd->right];
      float dl = box_weight(p, L, dim), dr = box_weight(p, R, dim);
      if (dl <= dr) { stack[sp++] = nd->right; stack[sp++] = nd->left; }
      else { stack[sp++] = nd->left; stack[sp++] = nd->right; }
    }
    job->res_w[i] = best_w;
    job->res_j[i] = best_j;
    if (best_j != ORACLE_INVALID) atomic_min_u32(&job->comp_radius[c], f2u(best_w));
  }
  free(stack);
  return NULL;
}

/* Node component flags, bottom-up (children before parents: ids are
 * preorder, so a reverse sweep sees children first). */
static void kd_node_comp(const kd_tree *t, const uint32_t *comp, uint32_t *node_comp) {
  for (int64_t v = t->n_nodes - 1; v >= 0; --v) {
    const kd_node *nd = &t->nodes[v];
    if (nd->left < 0) {
      uint32_t c = comp[t->idx[nd->begin]];
      for (int64_t k = nd->begin + 1; k < nd->end; ++k)
        if (comp[t->idx[k]] != c) { c = ORACLE_INVALID; break; }
      node_comp[v] = c;
    } else {
      uint32_t a = node_comp[nd->left], b = node_comp[nd->right];
      node_comp[v] = (a == b) ? a : ORACLE_INVALID;
    }
  }
}

static int kd_boruvka_impl(const float *pts, const float *core2, int64_t n, int dim,
                           oracle_edge *out, int nthreads, int64_t *rounds_out) {
  if (rounds_out) *rounds_out = 0;
  if (n <= 1) return 0;
  if (nthreads < 1) nthreads = 1;
  kd_tree t;
  t.pts = pts;
  t.dim = dim;
  t.n = n;
  t.idx = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n);
  t.nodes = (kd_node *)malloc(sizeof(kd_node) * (size_t)(2 * (n / (KD_LEAF / 2) + 2)));
  t.n_nodes = 0;
  t.max_depth = 0;
  for (int64_t k = 0; k < n; ++k) t.idx[k] = (uint32_t)k;
  kd_build_rec(&t, 0, n, 0);

  uint32_t *par = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n);
  uint32_t *comp = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n);
  uint32_t *node_comp = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)t.n_nodes);
  uint32_t *rad = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n);
  float *res_w = (float *)malloc(sizeof(float) * (size_t)n);
  uint32_t *res_j = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n);
  float *cw = (float *)malloc(sizeof(float) * (size_t)n);
  uint32_t *ca = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n);
  uint32_t *cb = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n);
  for (int64_t k = 0; k < n; ++k) par[k] = (uint32_t)k;
  int64_t got = 0, rounds = 0;
  int status = 0;
  pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nthreads);
  kd_job *jobs = (kd_job *)malloc(sizeof(kd_job) * (size_t)nthreads);
  while (got < n - 1) {
    for (int64_t k = 0; k < n; ++k) comp[k] = uf_find(par, (uint32_t)k);
    kd_node_comp(&t, comp, node_comp);
    /* initial radius: any real cross edge of the component is a valid bound;
     * use pairs adjacent in the tree's point order (same idea as §3,
     * Optimization 2, on this oracle's own order) */
    for (int64_t k = 0; k < n; ++k) rad[k] = f2u(INFINITY);
    for (int64_t k = 0; k + 1 < n; ++k) {
      uint32_t a = t.idx[k], b = t.idx[k + 1];
      if (comp[a] == comp[b]) continue;
      uint32_t wb = f2u(edge_weight(pts, core2, a, b, dim));
      if (wb < rad[comp[a]]) rad[comp[a]] = wb;
      if (wb < rad[comp[b]]) rad[comp[b]] = wb;
    }
    int64_t chunk = (n + nthreads - 1) / nthreads;
    for (int q = 0; q < nthreads; ++q) {
      jobs[q].t = &t; jobs[q].core2 = core2; jobs[q].comp = comp; jobs[q].node_comp = node_comp;
      jobs[q].comp_radius = rad;
      jobs[q].res_w = res_w; jobs[q].res_j = res_j;
      jobs[q].begin = q * chunk < n ? q * chunk : n;
      jobs[q].end = (q + 1) * chunk < n ? (q + 1) * chunk : n;
    }
    if (nthreads == 1) kd_query_range(&jobs[0]);
    else {
      for (int q = 0; q < nthreads; ++q) pthread_create(&th[q], NULL, kd_query_range, &jobs[q]);
      for (int q = 0; q < nthreads; ++q) pthread_join(th[q], NULL);
    }
    /* per-component minimum under the full key, sequentially */
    for (int64_t k = 0; k < n; ++k) { cw[k] = INFINITY; ca[k] = ORACLE_INVALID; cb[k] = ORACLE_INVALID; }
    for (int64_t i = 0; i < n; ++i) {
      if (res_j[i] == ORACLE_INVALID) continue;
      uint32_t c = comp[i];
      if (ca[c] == ORACLE_INVALID ||
          key_cmp(res_w[i], (uint32_t)i, res_j[i], cw[c], ca[c], cb[c]) < 0) {
        cw[c] = res_w[i]; ca[c] = (uint32_t)i; cb[c] = res_j[i];
      }
    }
    /* add every component's edge; a mutual pair's shared edge is added once */
    int64_t added = 0;
    for (int64_t c = 0; c < n; ++c) {
      if (ca[c] == ORACLE_INVALID) continue;
      uint32_t ra = uf_find(par, ca[c]), rb = uf_find(par, cb[c]);
      if (ra == rb) continue;
      if (ra < rb) par[rb] = ra; else par[ra] = rb;
      out[got].i = ca[c] < cb[c] ? ca[c] : cb[c];
      out[got].j = ca[c] < cb[c] ? cb[c] : ca[c];
      out[got].w = cw[c];
      ++got;
      ++added;
    }
    ++rounds;
    if (added == 0) { status = -2; break; }
    if (rounds > 64) { status = -3; break; }
  }
  if (rounds_out) *rounds_out = rounds;
  free(th); free(jobs);
  free(t.idx); free(t.nodes); free(par); free(comp); free(node_comp); free(rad);
  free(res_w); free(res_j); free(cw); free(ca); free(cb);
  return status;
}

int oracle_kd_boruvka(const float *pts, int64_t n, int dim, oracle_edge *out, int nthreads,
                      int64_t *rounds_out) {
  return kd_boruvka_impl(pts, NULL, n, dim, out, nthreads, rounds_out);
}

/* The same Boruvka loop on the mutual reachability weights (§4.5): the
 * queries prune with max(core2[i], box weight), a lower bound of every weight
 * from i into the box. */
int oracle_kd_boruvka_mrd(const float *pts, const float *core2, int64_t n, int dim,
                          oracle_edge *out, int nthreads, int64_t *rounds_out) {
  return kd_boruvka_impl(pts, core2, n, dim, out, nthreads, rounds_out);
}

/* Core distances with the k-d tree: each point keeps its k - 1 smallest
 * weights to other points (sorted), searching with the largest of them as
 * the cutoff once it has k - 1 (§4.5's definition, faster than the full
 * selection above for large n). */
typedef struct {
  kd_tree *t;
  int k;
  float *core2;
  int64_t begin, end;
} kd_knn_job;

static void *kd_knn_range(void *arg) {
  kd_knn_job *job = (kd_knn_job *)arg;
  kd_tree *t = job->t;
  const int dim = t->dim, m = job->k - 1;
  int64_t *stack = (int64_t *)malloc(sizeof(int64_t) * (size_t)(2 * t->max_depth + 8));
  float *best = (float *)malloc(sizeof(float) * (size_t)(m > 0 ? m : 1));
  for (int64_t pos = job->begin; pos < job->end; ++pos) {
    uint32_t i = t->idx[pos];
    if (m == 0) { job->core2[i] = 0.0f; continue; }
    const float *p = t->pts + (int64_t)i * dim;
    int have = 0;
    int64_t sp = 0;
    stack[sp++] = 0;
    while (sp > 0) {
      const kd_node *nd = &t->nodes[stack[--sp]];
      const float radius = have == m ? best[m - 1] : INFINITY;
      if (box_weight(p, nd, dim) > radius) continue;
      if (nd->left < 0) {
        for (int64_t q = nd->begin; q < nd->end; ++q) {
          uint32_t j = t->idx[q];
          if (j == i) continue;
          float w = oracle_weight(p, t->pts + (int64_t)j * dim, dim);
          if (have == m && w >= best[m - 1]) continue;
          int at = have < m ? have++ : m - 1; /* drop the largest when full */
          while (at > 0 && best[at - 1] > w) { best[at] = best[at - 1]; --at; }
          best[at] = w;
        }
        continue;
      }
      const kd_node *L = &t->nodes[nd->left], *R = &t->nodes[nd->right];
      float dl = box_weight(p, L, dim), dr = box_weight(p, R, dim);
      if (dl <= dr) { stack[sp++] = nd->right; stack[sp++] = nd->left; }
      else { stack[sp++] = nd->left; stack[sp++] = nd->right; }
    }
    job->core2[i] = best[m - 1];
  }
  free(stack);
  free(best);
  return NULL;
}

int oracle_kd_core_dist2(const float *pts, int64_t n, int dim, int k, float *core2, int nthreads) {
  if (k < 1 || k > n) return -1;
  if (nthreads < 1) nthreads = 1;
  kd_tree t;
  t.pts = pts;
  t.dim = dim;
  t.n = n;
  t.idx = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n);
  t.nodes = (kd_node *)malloc(sizeof(kd_node) * (size_t)(2 * (n / (KD_LEAF / 2) + 2)));
  t.n_nodes = 0;
  t.max_depth = 0;
  for (int64_t q = 0; q < n; ++q) t.idx[q] = (uint32_t)q;
  kd_build_rec(&t, 0, n, 0);
  pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nthreads);
  kd_knn_job *jobs = (kd_knn_job *)malloc(sizeof(kd_knn_job) * (size_t)nthreads);
  int64_t chunk = (n + nthreads - 1) / nthreads;
  for (int q = 0; q < nthreads; ++q) {
    jobs[q].t = &t;
    jobs[q].k = k;
    jobs[q].core2 = core2;
    jobs[q].begin = q * chunk < n ? q * chunk : n;
    jobs[q].end = (q + 1) * chunk < n ? (q + 1) * chunk : n;
  }
  if (nthreads == 1) kd_knn_range(&jobs[0]);
  else {
    for (int q = 0; q < nthreads; ++q) pthread_create(&th[q], NULL, kd_knn_range, &jobs[q]);
    for (int q = 0; q < nthreads; ++q) pthread_join(th[q], NULL);
  }
  free(th);
  free(jobs);
  free(t.idx);
  free(t.nodes);
  return 0;
}

/* Checks used by the tests: number of distinct components of an edge list
 * (1 == spanning and connected) and whether it has a cycle. */
int64_t oracle_count_components(const oracle_edge *e, int64_t m, int64_t n, int *has_cycle) {
  uint32_t *par = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n);
  for (int64_t k = 0; k < n; ++k) par[k] = (uint32_t)k;
  int64_t comps = n;
  *has_cycle = 0;
  for (int64_t k = 0; k < m; ++k) {
    if (e[k].i >= n || e[k].j >= n) { *has_cycle = 1; continue; }
    uint32_t a = uf_find(par, e[k].i), b = uf_find(par, e[k].j);
    if (a == b) { *has_cycle = 1; continue; }
    if (a < b) par[b] = a; else par[a] = b;
    --comps;
  }
  free(par);
  return comps;
}

/* ------------------------------------------------------------------------ */
/* Single-linkage dendrogram of a spanning tree.  The introduction names     */
/* clustering (HDBSCAN*) as a consumer of the EMST, and §4.5 computes the    */
/* mutual-reachability tree for it; the hierarchy those methods read off the */
/* tree is defined here.                                                     */
/* ------------------------------------------------------------------------ */

/* The single-linkage hierarchy of a tree is the sequence of merges that
 * Kruskal's algorithm (§2, "MST computation") makes on the tree's own edges:
 * take them in order of weight and join the two clusters each one connects.
 * The given edge order is the merge order (weights must not decrease; among
 * equal weights the order decides).  Cluster ids: point v is cluster v, the
 * cluster made by the k-th edge is n + k.
 *   e        m = n - 1 edges.
 *   linkage  m rows of 4 words {a, b, w bits, size}: the two clusters merged
 *            (a < b), the weight, the number of points in the new cluster.
 *   parent   2n - 1 words: the cluster each cluster is merged into,
 *            ORACLE_INVALID for the last one.
 * Returns 0, or -1 when an id is >= n, an edge closes a cycle, a weight is
 * NaN, or a weight is below the one before it. */
int oracle_dendrogram(const oracle_edge *e, int64_t n, uint32_t *linkage, uint32_t *parent) {
  if (n <= 0) return 0;
  const int64_t m = n - 1;
  uint32_t *par = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n);
  uint32_t *cluster = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n);
  uint32_t *size = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n);
  if (!par || !cluster || !size) { free(par); free(cluster); free(size); return -2; }
  for (int64_t v = 0; v < n; ++v) {
    par[v] = (uint32_t)v;
    cluster[v] = (uint32_t)v;
    size[v] = 1;
  }
  int rc = 0;
  for (int64_t k = 0; k < m; ++k) {
    if (e[k].i >= n || e[k].j >= n || e[k].w != e[k].w || (k > 0 && e[k].w < e[k - 1].w)) {
      rc = -1;
      break;
    }
    uint32_t ra = uf_find(par, e[k].i), rb = uf_find(par, e[k].j);
    if (ra == rb) { rc = -1; break; }
    uint32_t ca = cluster[ra], cb = cluster[rb];
    uint32_t *row = linkage + 4 * k;
    row[0] = ca < cb ? ca : cb;
    row[1] = ca < cb ? cb : ca;
    memcpy(&row[2], &e[k].w, 4);
    row[3] = size[ra] + size[rb];
    parent[ca] = parent[cb] = (uint32_t)(n + k);
    uint32_t r = ra < rb ? ra : rb;
    par[ra] = par[rb] = r;
    cluster[r] = (uint32_t)(n + k);
    size[r] = row[3];
  }
  parent[2 * n - 2] = ORACLE_INVALID;
  free(par);
  free(cluster);
  free(size);
  return rc;
}

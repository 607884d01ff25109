// mrd.cu -- the mutual reachability distance of §4.5 (the metric of
// HDBSCAN*): squared core distances by a k-nearest-neighbour search of the
// hierarchy the EMST builds.  The Boruvka rounds then run on
// max(core(u), core(v), w(u, v)) (traverse.cuh, rounds.cu).
#include "traverse.cuh"

namespace emst {

constexpr int kCoreBlock = 128;

// Sorted insertion of w into best[0..MMAX) (ascending, +inf = empty slot),
// dropping the largest: each slot takes its left neighbour when that is
// above w, else the smaller of itself and w.
template <int MMAX>
__device__ __forceinline__ void knn_insert(float (&best)[MMAX], float w) {
#pragma unroll
  for (int j = MMAX - 1; j > 0; --j) best[j] = best[j - 1] > w ? best[j - 1] : fminf(best[j], w);
  best[0] = fminf(best[0], w);
}

// A leaf of the hierarchy met by a k-nearest-neighbour query at i: a one-point
// leaf c at (exact) distance d, or a chunk scanned point by point; the query
// itself and its seeded window [wlo, whi] are skipped.
template <int MMAX, bool CHUNKS>
__device__ __forceinline__ void knn_leaf(float (&best)[MMAX], float &thr, uint32_t c,
                                         float d, int64_t i, int64_t wlo, int64_t whi,
                                         const float4 &p, const float4 *__restrict__ pts,
                                         int leaf, int64_t n) {
  if (!CHUNKS) {
    if ((int64_t)c != i && ((int64_t)c < wlo || (int64_t)c > whi) && d < thr) {
      knn_insert(best, d);
      thr = best[MMAX - 1];
    }
    return;
  }
  const int64_t lo = (int64_t)c * leaf;
  const int64_t hi = lo + leaf < n ? lo + leaf : n;
  for (int64_t k = lo; k < hi; ++k) {
    if (k == i || (k >= wlo && k <= whi)) continue;
    const float4 t = __ldg(pts + k);
    const float w = sq_dist(p.x, p.y, p.z, t.x, t.y, t.z);
    if (w < thr) {
      knn_insert(best, w);
      thr = best[MMAX - 1];
    }
  }
}

// Squared core distance of every point (curve order): the m-th smallest
// weight from the point to another point, m = k - 1 (the point itself is the
// k-th neighbour's first).  Seeded with the m curve neighbours on each side
// (a full list, so a finite cutoff from the start); the search skips those
// positions so no point is counted twice.  A candidate enters only below the
// current m-th smallest (an equal one changes nothing), and a box is entered
// only when nearer than it.  The stack bound is the traversal's (§ A7).
template <int MMAX, bool CHUNKS>
__global__ void __launch_bounds__(kCoreBlock) k_core_knn(const float4 *__restrict__ pts,
                                                         const NodeRec *__restrict__ nodes,
                                                         int64_t n, int leaf, int m,
                                                         float *__restrict__ core2,
                                                         uint32_t *status) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (m == 0) {
    core2[i] = 0.0f;
    return;
  }
  const float4 p = pts[i];
  // the first MMAX - m slots hold -inf, which no insertion displaces, so the
  // m smallest candidates fill the last m slots and the m-th is always the
  // last one (a static register index)
  float best[MMAX];
#pragma unroll
  for (int j = 0; j < MMAX; ++j)
    best[j] = j < MMAX - m ? __int_as_float(0xff800000) : __int_as_float(0x7f800000);
  const int64_t wlo = i - m < 0 ? 0 : i - m;
  const int64_t whi = i + m >= n ? n - 1 : i + m;
  for (int64_t j = wlo; j <= whi; ++j) {
    if (j == i) continue;
    const float4 c = __ldg(pts + j);
    knn_insert(best, sq_dist(p.x, p.y, p.z, c.x, c.y, c.z));
  }
  float thr = best[MMAX - 1];
  uint32_t st_node[kStackDepth];
  float st_dist[kStackDepth];
  int sp = 0;
  uint32_t node = 0;
  while (true) {
    float4 a, b, c;
    uint4 dd;
    load_record(nodes + node, a, b, c, dd);
    const float dL = box_dist(p.x, p.y, p.z, a.x, a.y, a.z, a.w, b.x, b.y);
    const float dR = box_dist(p.x, p.y, p.z, b.z, b.w, c.x, c.y, c.z, c.w);
    bool okL = dL < thr, okR = dR < thr;
    if (okL && (dd.x & kLeafBit)) {
      knn_leaf<MMAX, CHUNKS>(best, thr, dd.x & ~kLeafBit, dL, i, wlo, whi, p, pts, leaf, n);
      okL = false;
    }
    if (okR && (dd.y & kLeafBit)) {
      if (dR < thr)
        knn_leaf<MMAX, CHUNKS>(best, thr, dd.y & ~kLeafBit, dR, i, wlo, whi, p, pts, leaf, n);
      okR = false;
    }
    okL = okL && dL < thr;
    okR = okR && dR < thr;
    if (okL && okR) {
      if (sp >= kStackDepth) { atomicOr(status, kErrStack); break; }
      if (dL <= dR) { st_node[sp] = dd.y; st_dist[sp] = dR; node = dd.x; }
      else { st_node[sp] = dd.x; st_dist[sp] = dL; node = dd.y; }
      ++sp;
      continue;
    }
    if (okL) { node = dd.x; continue; }
    if (okR) { node = dd.y; continue; }
    bool found = false;
    while (sp > 0) {
      --sp;
      if (st_dist[sp] < thr) { node = st_node[sp]; found = true; break; }
    }
    if (!found) break;
  }
  core2[i] = thr;
}

// Curve order -> the caller's order (the original index rides in pts.w).
__global__ void k_core_to_input(const float4 *__restrict__ pts, const float *__restrict__ core2,
                                int64_t n, float *__restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  out[__float_as_uint(pts[i].w)] = core2[i];
}

void launch_core_knn(Problem &P, int k) {
  const int m = k - 1;
  const int g = grid_for(P.n, kCoreBlock);
  const bool h = P.leaf > 1;
#define EMST_KNN(M) \
  do { \
    if (h) k_core_knn<M, true><<<g, kCoreBlock, 0, P.stream>>>(P.pts, P.nodes, P.n, P.leaf, m, P.core2, P.counters + 1); \
    else k_core_knn<M, false><<<g, kCoreBlock, 0, P.stream>>>(P.pts, P.nodes, P.n, P.leaf, m, P.core2, P.counters + 1); \
  } while (0)
  if (m <= 4) EMST_KNN(4);
  else if (m <= 8) EMST_KNN(8);
  else if (m <= 16) EMST_KNN(16);
  else EMST_KNN(32);
#undef EMST_KNN
  P.launches += 1;
}

void launch_core_to_input(Problem &P, float *out) {
  k_core_to_input<<<grid_for(P.n, 256), 256, 0, P.stream>>>(P.pts, P.core2, P.n, out);
  P.launches += 1;
}

}  // namespace emst

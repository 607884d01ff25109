// traverse.cuh -- the per-point query of Algorithm 2 (nearest neighbour in
// another component), shared by the round kernels and the learned-radius
// sample logger.
#pragma once

#include "common.cuh"

namespace emst {

#ifndef EMST_STACK_DEPTH
#define EMST_STACK_DEPTH 164
#endif
constexpr int kStackDepth = EMST_STACK_DEPTH;  // > 160 = the deepest possible path (see traverse_one)

// Per-query state of Algorithm 2.
struct Query {
  float px, py, pz;
  float core;      // mutual reachability: the query's squared core distance (else 0)
  uint32_t me;     // the query's component label
  float radius;    // cutoff (inclusive)
  float best;      // best weight found
  uint32_t bj;     // its curve index (kInvalid: none yet)
  uint32_t bid;    // its original index
};

// A candidate j at weight d <= radius: keep the smaller (w, original id).
__device__ __forceinline__ void take_point(Query &q, uint32_t j, float d, uint32_t idj) {
  if (q.bj == kInvalid || d < q.best) {  // first candidate, or strictly closer
    q.best = d;
    q.bj = j;
    q.bid = idj;
    q.radius = d;
  } else if (d == q.best && idj < q.bid) {
    q.bj = j;
    q.bid = idj;
  }
}

// A leaf of the hierarchy is a chunk of `leaf` consecutive curve positions
// (the last one may be shorter).  A one-point leaf's box IS the point, so its
// box distance d is already the exact weight and its label was tested with
// the box; its original id is loaded only to break an exact tie.  A longer
// chunk is scanned point by point.
// MRD: the weight is the mutual reachability one, max(core(query), core(j), d)
// (§4.5), so a candidate within the cutoff by distance may fall outside it.
template <bool CHUNKS, bool MRD>
__device__ __forceinline__ void scan_chunk(Query &q, uint32_t c, float d1, int leaf, int64_t n,
                                           const float4 *__restrict__ pts,
                                           const uint32_t *__restrict__ labels,
                                           const float *__restrict__ core2) {
  if (!CHUNKS) {
    if (MRD) {
      d1 = fmaxf(d1, fmaxf(q.core, __ldg(core2 + c)));
      if (d1 > q.radius) return;
    }
    if (q.bj == kInvalid || d1 < q.best) {
      q.best = d1;
      q.bj = c;
      q.bid = kInvalid;  // loaded lazily
      q.radius = d1;
    } else if (d1 == q.best) {
      const uint32_t idj = __float_as_uint(pts[c].w);
      if (q.bid == kInvalid) q.bid = __float_as_uint(pts[q.bj].w);
      if (idj < q.bid) { q.bj = c; q.bid = idj; }
    }
    return;
  }
  if (q.bid == kInvalid && q.bj != kInvalid) q.bid = __float_as_uint(pts[q.bj].w);
  const int64_t lo = (int64_t)c * leaf;
  const int64_t hi = lo + leaf < n ? lo + leaf : n;
  for (int64_t k = lo; k < hi; ++k) {
    if (__ldg(labels + k) == q.me) continue;
    const float4 t = __ldg(pts + k);
    float d = sq_dist(q.px, q.py, q.pz, t.x, t.y, t.z);
    if (MRD) d = fmaxf(d, fmaxf(q.core, __ldg(core2 + k)));
    if (d <= q.radius) take_point(q, (uint32_t)k, d, __float_as_uint(t.w));
  }
}

// One node record in two 32-byte loads (the record is 64-byte aligned).
__device__ __forceinline__ void load_record(const NodeRec *rec, float4 &a, float4 &b, float4 &c,
                                            uint4 &dd) {
  asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
      : "l"(rec));
  asm("ld.global.nc.v8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=f"(c.x), "=f"(c.y), "=f"(c.z), "=f"(c.w), "=r"(dd.x), "=r"(dd.y), "=r"(dd.z), "=r"(dd.w)
      : "l"(reinterpret_cast<const char *>(rec) + 32));
}

// ---------------------------------------------------------------------------
// The search stack of one query of the persistent kernel (Algorithm 2's
// stack of nodes still to examine, each with the weight bound of its box,
// re-tested when popped): one 8-byte (node, bound bits) entry per level in a
// per-thread local array of kStackDepth entries (the deepest possible path,
// see traverse_one); push reports an overflow instead of writing past it.
// ---------------------------------------------------------------------------
struct LocalStack {
  uint2 e[kStackDepth];
  int sp;
  __device__ __forceinline__ void init() { sp = 0; }
  __device__ __forceinline__ bool push(uint32_t node, float d) {
    if (sp >= kStackDepth) return false;
    e[sp++] = make_uint2(node, __float_as_uint(d));
    return true;
  }
  __device__ __forceinline__ bool pop(uint2 &x) {
    if (sp == 0) return false;
    x = e[--sp];
    return true;
  }
};

// One visit of internal node `node` of Algorithm 2, whose own box the caller
// has already accepted: test both children from the node's record, scan
// accepted leaf chunks, and return the nearer accepted internal child (the
// farther one is pushed with its box bound), or kInvalid when no internal
// child is accepted (the caller pops).  `overflow` is set if a push found
// the stack full (cannot happen, see traverse_one).
// FIRST: the first round, where every label is the point's own curve index,
// so no internal child is single-component and the only one-point leaf to
// skip is the query itself: no label load.
// MRD: mutual reachability weights (§4.5).  The boxes prune exactly as for
// the plain weight: the caller only searches with a cutoff at or above the
// query's core distance, and every weight from the query is at least that,
// so max(core, box distance) <= cutoff  <=>  box distance <= cutoff.
// TIES = false: the input has no large group of identical points (see the
// tie rule below), so that check is compiled out.
template <bool CHUNKS, bool FIRST, bool MRD, bool TIES, class Stack>
__device__ __forceinline__ uint32_t visit(Query &q, uint32_t node,
                                          const NodeRec *__restrict__ nodes,
                                          const uint2 *__restrict__ nlabels,
                                          const float4 *__restrict__ pts,
                                          const uint32_t *__restrict__ labels, int leaf,
                                          int64_t n, Stack &stk, bool &overflow,
                                          const float *__restrict__ core2, bool ties) {
  float4 a, b, c;
  uint4 dd;
  load_record(nodes + node, a, b, c, dd);
  uint2 lab;
  if (FIRST) {
    lab.x = (!CHUNKS && (dd.x & kLeafBit)) ? (dd.x & ~kLeafBit) : kInvalid;
    lab.y = (!CHUNKS && (dd.y & kLeafBit)) ? (dd.y & ~kLeafBit) : kInvalid;
  } else {
    lab = __ldg(nlabels + node);
  }
  const float dL = box_dist(q.px, q.py, q.pz, a.x, a.y, a.z, a.w, b.x, b.y);
  const float dR = box_dist(q.px, q.py, q.pz, b.z, b.w, c.x, c.y, c.z, c.w);
  bool okL = (lab.x != q.me) && (dL <= q.radius);
  bool okR = (lab.y != q.me) && (dR <= q.radius);
  if (okL && (dd.x & kLeafBit)) {
    scan_chunk<CHUNKS, MRD>(q, dd.x & ~kLeafBit, dL, leaf, n, pts, labels, core2);
    okL = false;
  }
  if (okR && (dd.y & kLeafBit)) {
    if (dR <= q.radius) scan_chunk<CHUNKS, MRD>(q, dd.y & ~kLeafBit, dR, leaf, n, pts, labels, core2);
    okR = false;
  }
  okL = okL && dL <= q.radius;
  okR = okR && dR <= q.radius;
  // An internal child whose weight bound only ties the cutoff holds nothing
  // better than the best so far unless it has a point with a smaller
  // original id (dd.z / dd.w hold each child's smallest).  Without this a
  // group of m identical points costs each of its queries a visit to all m,
  // and so does a group at one equal distance from the query.  (Checked
  // only when a tie occurs; a leaf resolves its own ties.)
  // (the ids are read again in the rare tie case: kept live through the
  // leaf scans above they cost the hot loop a register it does not have)
  // Only when the input has a run of more than 32 equal codes (`ties`):
  // otherwise no group of identical points is larger than that, a tie
  // involves a few points at most and the check would only cost time.
  const float lbL = MRD ? fmaxf(q.core, dL) : dL, lbR = MRD ? fmaxf(q.core, dR) : dR;
  if (TIES && ties && q.bj != kInvalid && ((okL && lbL == q.radius) || (okR && lbR == q.radius))) {
    if (q.bid == kInvalid) q.bid = __float_as_uint(pts[q.bj].w);  // loaded lazily
    const uint2 mn = __ldg(reinterpret_cast<const uint2 *>(nodes + node) + 7);  // dd.z, dd.w
    if (lbL == q.radius && mn.x >= q.bid) okL = false;
    if (lbR == q.radius && mn.y >= q.bid) okR = false;
  }
  if (okL && okR) {
    const bool left_first = dL <= dR;
    if (!stk.push(left_first ? dd.y : dd.x, left_first ? dR : dL)) overflow = true;
    return left_first ? dd.x : dd.y;
  }
  if (okL) return dd.x;
  if (okR) return dd.y;
  return kInvalid;
}

// The next stacked node whose bound is still within the cutoff (the cutoff
// only shrinks, so entries above it are dropped), or kInvalid.
template <class Stack>
__device__ __forceinline__ uint32_t pop_next(const Query &q, Stack &stk) {
  uint2 e;
  while (stk.pop(e))
    if (__uint_as_float(e.y) <= q.radius) return e.x;
  return kInvalid;
}

// Depth-first search of the subtree of internal node `node`, whose own box
// the caller has already accepted: test both children of every visited
// record, scan accepted leaf chunks, descend into the nearer accepted
// internal child and stack the farther one with its box distance (re-tested
// when popped).  The same steps as visit() + pop_next(), in one loop with the
// stack in two local arrays (node, bound): the form the one-thread-per-point
// kernel measured fastest.  COUNT: count the visits (nvis) and, with a
// bitmap `seen` of the internal nodes, mark each node visited.
// FIRST: the first round, where every label is the point's own curve index,
// so no internal child is single-component and the only one-point leaf to
// skip is the query itself: no label load.
// MRD: mutual reachability weights (§4.5).  The boxes prune exactly as for
// the plain weight: the caller only searches with a cutoff at or above the
// query's core distance, and every weight from the query is at least that,
// so max(core, box distance) <= cutoff  <=>  box distance <= cutoff.
// TIES = false: the input has no large group of identical points (see the
// tie rule below), so that check is compiled out.
template <bool COUNT, bool CHUNKS, bool FIRST, bool MRD = false, bool TIES = true, bool LB = false>
__device__ __forceinline__ bool explore(Query &q, uint32_t node, const NodeRec *__restrict__ nodes,
                                        const uint2 *__restrict__ nlabels,
                                        const float4 *__restrict__ pts,
                                        const uint32_t *__restrict__ labels, int leaf, int64_t n,
                                        uint32_t *st_node, float *st_dist,
                                        unsigned long long &nvis,
                                        const float *__restrict__ core2 = nullptr,
                                        bool ties = true, uint32_t *seen = nullptr) {
  int sp = 0;
  while (true) {
    if (COUNT) {
      ++nvis;
      if (seen) atomicOr(seen + (node >> 5), 1u << (node & 31));
    }
    float4 a, b, c;
    uint4 dd;
    load_record(nodes + node, a, b, c, dd);
    uint2 lab;
    if (FIRST) {
      lab.x = (!CHUNKS && (dd.x & kLeafBit)) ? (dd.x & ~kLeafBit) : kInvalid;
      lab.y = (!CHUNKS && (dd.y & kLeafBit)) ? (dd.y & ~kLeafBit) : kInvalid;
    } else {
      lab = __ldg(nlabels + node);
    }
    const float dL = box_dist(q.px, q.py, q.pz, a.x, a.y, a.z, a.w, b.x, b.y);
    const float dR = box_dist(q.px, q.py, q.pz, b.z, b.w, c.x, c.y, c.z, c.w);
    bool okL = (lab.x != q.me) && (dL <= q.radius);
    bool okR = (lab.y != q.me) && (dR <= q.radius);
    // LB: while nothing is found, q.best keeps the smallest weight bound of a
    // child of another component rejected by its distance (see traverse_one)
    // (once something is found, q.best <= the cutoff < any rejected bound,
    // so the update leaves it alone)
    if (LB) {
      const float rl = (lab.x != q.me && !okL) ? dL : __int_as_float(0x7f800000);
      const float rr = (lab.y != q.me && !okR) ? dR : __int_as_float(0x7f800000);
      q.best = fminf(q.best, fminf(rl, rr));
    }
    if (okL && (dd.x & kLeafBit)) {
      scan_chunk<CHUNKS, MRD>(q, dd.x & ~kLeafBit, dL, leaf, n, pts, labels, core2);
      okL = false;
    }
    if (okR && (dd.y & kLeafBit)) {
      if (dR <= q.radius) scan_chunk<CHUNKS, MRD>(q, dd.y & ~kLeafBit, dR, leaf, n, pts, labels, core2);
      okR = false;
    }
    okL = okL && dL <= q.radius;
    okR = okR && dR <= q.radius;
    // An internal child whose weight bound only ties the cutoff holds nothing
    // better than the best so far unless it has a point with a smaller
    // original id (dd.z / dd.w hold each child's smallest).  Without this a
    // group of m identical points costs each of its queries a visit to all m,
    // and so does a group at one equal distance from the query.  (Checked
    // only when a tie occurs; a leaf resolves its own ties.)
    // (the ids are read again in the rare tie case: kept live through the
    // leaf scans above they cost the hot loop a register it does not have)
    // Only when the input has a run of more than 32 equal codes (`ties`):
    // otherwise no group of identical points is larger than that, a tie
    // involves a few points at most and the check would only cost time.
    const float lbL = MRD ? fmaxf(q.core, dL) : dL, lbR = MRD ? fmaxf(q.core, dR) : dR;
    if (TIES && ties && q.bj != kInvalid && ((okL && lbL == q.radius) || (okR && lbR == q.radius))) {
      if (q.bid == kInvalid) q.bid = __float_as_uint(pts[q.bj].w);  // loaded lazily
      const uint2 mn = __ldg(reinterpret_cast<const uint2 *>(nodes + node) + 7);  // dd.z, dd.w
      if (lbL == q.radius && mn.x >= q.bid) okL = false;
      if (lbR == q.radius && mn.y >= q.bid) okR = false;
    }
    if (okL && okR) {
      if (sp >= kStackDepth) return false;
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
      if (st_dist[sp] <= q.radius) { node = st_node[sp]; found = true; break; }
    }
    if (!found) return true;
  }
}

// ---------------------------------------------------------------------------
// A7. Nearest other-component neighbour of every point (Algorithm 2), one
// thread per point in curve order (neighbouring threads get nearby queries).
//  - cutoff: the component's upper bound (Optimization 2), optionally
//    tightened by the previous round's neighbour when it still lies in
//    another component (a real cross edge of this point, so never below the
//    component minimum);
//  - a child is examined only if its label differs from the query's
//    (Optimization 1) and its box is within the cutoff (inclusive: equal
//    weights with smaller ids must survive); a leaf updates the best
//    (w, original id) and shrinks the cutoff to w.
// The leaves of the hierarchy are chunks of `leaf` consecutive curve
// positions; an accepted chunk is scanned point by point.
// The stack never overflows: every split of the hierarchy uses a strictly
// later bit of the augmented key (code + 32-bit index: 96 bits with 64-bit
// codes, 160 with 128-bit codes), so a root-to-leaf path has at most 160
// internal nodes and at most one stacked sibling per level.
// Ends with the per-component minimum (A8): the found edge is offered to its
// component's 128-bit (w, min id, max id, outside label) key.
// SEEDED (the emst_compute path) also tightens each cutoff with the
// component's best weight found so far (a real cross edge, so never below
// the component minimum), reports the exact nearest neighbour within that cutoff
// (or none), and keeps a per-point lower bound for the next round (res.x):
// a point whose bound exceeds its component's cutoff skips its query.  The
// endpoint of every component's minimum edge still finds it, so the minima
// (and the tree) are unchanged; which other points report differs.
// Unseeded, each point reports exactly its nearest other-component point
// within its cutoff (what the inspection entry point exposes).
// ---------------------------------------------------------------------------
// A8: offer the edge (w, oi, oj) found by a query of component `c` (its
// neighbour j in curve order) to the component's 128-bit minimum.  Many
// points of a large component find edges, but only one that improves on the
// value seen now needs the compare-and-swap; the outside endpoint's label is
// loaded only then.  Values only decrease, so a failed swap returns a
// smaller value and the loop re-checks it (bounded; a status bit if not).
__device__ __forceinline__ void offer_best(CompBest *c, uint32_t w_bits, uint32_t oi, uint32_t oj,
                                           const uint32_t *__restrict__ labels, uint32_t j,
                                           uint32_t *status) {
  const uint64_t key = ((uint64_t)w_bits << 32) | (uint64_t)(oi < oj ? oi : oj);
  const uint64_t mx_hi = (uint64_t)(oi < oj ? oj : oi) << 32;
  CompBest cur;
  cur.key = __ldcg(reinterpret_cast<const unsigned long long *>(&c->key));
  if (key > cur.key) return;
  cur.mx = __ldcg(reinterpret_cast<const unsigned long long *>(&c->mx));
  if (key == cur.key && mx_hi >= (cur.mx & 0xFFFFFFFF00000000ull)) return;  // same or later edge
  CompBest want;
  want.key = key;
  want.mx = mx_hi | (uint64_t)__ldg(labels + j);
  for (int it = 0; it < (1 << 20); ++it) {
    const CompBest old = atomicCAS(c, cur, want);
    if (old.key == cur.key && old.mx == cur.mx) return;
    cur = old;
    if (want.key > cur.key || (want.key == cur.key && want.mx >= cur.mx)) return;
  }
  atomicOr(status, kErrCas);
}

struct TravArgs {
  const float4 *pts;
  const NodeRec *nodes;
  const uint2 *nlabels;
  const float *core2;  // MRD: squared core distances in curve order
  bool ties;           // identical points exist: prune children that can only tie
  const uint32_t *labels;
  const uint32_t *bound;
  const float *radius_in;
  int leaf;
  const uint32_t *inst_of;
  const uint32_t *inst_root;
  const int64_t *offsets;
  uint2 *res;
  CompBest *comp;
  int64_t n;
  uint32_t *status;
  unsigned long long *visits;   // COUNT: node visits
  unsigned long long *queries;  // COUNT: queries that searched (not skipped)
  uint32_t *seen;               // COUNT: bitmap of the internal nodes visited
  const float *pred_r;  // LEARNED: proposed cutoff of each point
  float *r_used;        // LEARNED: cutoff each query was exact within (+inf: skipped)
  uint32_t *queue;      // a listed launch: warps take 32 list entries at a time, in list
                        // order, from this counter (null: a grid-stride walk of the list)
};

// The first half of a query: its cutoff, and whether it needs a search at all.
// Returns false when the query is already finished (its result written):
// a one-point instance, a point whose lower bound exceeds its component's
// cutoff, or (MRD) a core distance above the cutoff.  Otherwise q holds the
// query, `start` the node to search from and r0 the cutoff the search is
// exact within.
// LEARNED also tightens the cutoff with the proposed radius pred_r[i] (any
// value: exactness is restored afterwards by rerunning every point whose
// cutoff fell below its component's found minimum) and records it in r_used.
// MRD: the mutual reachability weights (§4.5); a query whose own core
// distance lies above its cutoff finds nothing and is skipped.
template <bool CARRIED, bool RADIUS_IN, bool SEEDED, bool LEARNED, bool MRD>
__device__ __forceinline__ bool start_query(const TravArgs &A, int64_t i, Query &q,
                                            uint32_t &start, float &r0) {
  const float kInf = __int_as_float(0x7f800000);
  // Batched form: search only this point's instance (its subtree).
  start = 0u;
  if (A.inst_of) {
    const uint32_t I = __ldg(A.inst_of + i);
    start = __ldg(A.inst_root + I);
    if (start == kInvalid) {  // a one-point instance: nothing to find
      A.res[i] = make_uint2(0u, kInvalid);
      if (LEARNED) A.r_used[i] = kInf;
      return false;
    }
  }
  const float4 p = A.pts[i];
  q.px = p.x;
  q.py = p.y;
  q.pz = p.z;
  q.core = MRD ? __ldg(A.core2 + i) : 0.0f;
  q.me = A.labels[i];
  q.best = kInf;
  q.bj = kInvalid;
  q.bid = kInvalid;
  if (RADIUS_IN) q.radius = A.radius_in[i];
  else q.radius = bound_to_radius(A.bound[q.me]);
  uint2 prev = make_uint2(0u, kInvalid);
  if (CARRIED) prev = A.res[i];
  if (SEEDED) {
    // The component's best weight found so far this round: a real cross edge
    // of the component, so never below its minimum.
    const uint32_t cw =
        (uint32_t)(__ldcg(reinterpret_cast<const unsigned long long *>(&A.comp[q.me].key)) >> 32);
    q.radius = fminf(q.radius, bound_to_radius(cw));
    // prev.x is a lower bound of this point's nearest other-component weight
    // (components only grow, so that weight never decreases).  Above the
    // component-level cutoff, this point cannot be an endpoint of the
    // component's minimum edge: skip the query.
    if (CARRIED && __uint_as_float(prev.x) > q.radius) {
      A.res[i] = make_uint2(prev.x, kInvalid);
      if (LEARNED) A.r_used[i] = kInf;
      return false;
    }
  }
  // The previous round's neighbour, if still in another component, is a real
  // cross edge of this point: a per-point cutoff.
  if (CARRIED && prev.y != kInvalid && A.labels[prev.y] != q.me)
    q.radius = fminf(q.radius, __uint_as_float(prev.x));
  if (LEARNED) q.radius = fminf(q.radius, __ldg(A.pred_r + i));
  r0 = q.radius;  // the search is exact within this cutoff
  if (LEARNED) A.r_used[i] = r0;
  if (MRD && q.core > r0) {  // every weight from this point is at least its core distance
    A.res[i] = make_uint2(__float_as_uint(q.core), kInvalid);
    return false;
  }
  return true;
}

// The second half: the query's result, and its edge offered to its
// component's minimum (A8, offer_best).
// SEEDED reports only the exact nearest neighbour within r0 (a seed beyond r0
// is dropped) and keeps in res.x a lower bound for the next round: the found
// weight, or r0 when nothing lies within it.
template <bool SEEDED>
__device__ __forceinline__ void finish_query(const TravArgs &A, int64_t i, Query &q, float r0) {
  const float kInf = __int_as_float(0x7f800000);
  if (SEEDED) {
    const bool found = q.bj != kInvalid && q.best <= r0;
    if (!found) q.bj = kInvalid;
    const float lb = found ? q.best : (r0 < kInf ? r0 : 0.0f);
    A.res[i] = make_uint2(__float_as_uint(lb), q.bj);
  } else {
    A.res[i] = make_uint2(__float_as_uint(q.best), q.bj);
  }
  if (q.bj != kInvalid) {
    const uint32_t oi = __float_as_uint(__ldg(&A.pts[i].w));
    const uint32_t oj = q.bid != kInvalid ? q.bid : __float_as_uint(__ldg(&A.pts[q.bj].w));
    offer_best(A.comp + q.me, __float_as_uint(q.best), oi, oj, A.labels, q.bj, A.status);
  }
}

// One query, start to finish (the one-thread-per-point form): the same
// steps as start_query + explore + finish_query, kept in one piece so the
// point's record stays in registers through the search.
template <bool CARRIED, bool RADIUS_IN, bool COUNT, bool SEEDED, bool CHUNKS, bool LEARNED,
          bool FIRST = false, bool MRD = false, bool TIES = true, bool LBT = true>
__device__ __forceinline__ void traverse_one(const TravArgs &A, int64_t i) {
  const float kInf = __int_as_float(0x7f800000);
  const int64_t n = A.n;
  // Batched form: search only this point's instance (its subtree).
  uint32_t start = 0u;
  if (A.inst_of) {
    const uint32_t I = __ldg(A.inst_of + i);
    start = __ldg(A.inst_root + I);
    if (start == kInvalid) {  // a one-point instance: nothing to find
      A.res[i] = make_uint2(0u, kInvalid);
      if (LEARNED) A.r_used[i] = kInf;
      return;
    }
  }
  const float4 p = A.pts[i];
  Query q;
  q.px = p.x;
  q.py = p.y;
  q.pz = p.z;
  q.core = MRD ? __ldg(A.core2 + i) : 0.0f;
  q.me = A.labels[i];
  q.best = kInf;
  q.bj = kInvalid;
  q.bid = kInvalid;
  if (RADIUS_IN) q.radius = A.radius_in[i];
  else q.radius = bound_to_radius(A.bound[q.me]);
  uint2 prev = make_uint2(0u, kInvalid);
  if (CARRIED) prev = A.res[i];
  if (SEEDED) {
    // The component's best weight found so far this round: a real cross edge
    // of the component, so never below its minimum.
    const uint32_t cw =
        (uint32_t)(__ldcg(reinterpret_cast<const unsigned long long *>(&A.comp[q.me].key)) >> 32);
    q.radius = fminf(q.radius, bound_to_radius(cw));
    // prev.x is a lower bound of this point's nearest other-component weight
    // (components only grow, so that weight never decreases).  Above the
    // component-level cutoff, this point cannot be an endpoint of the
    // component's minimum edge: skip the query.
    if (CARRIED && __uint_as_float(prev.x) > q.radius) {
      // (the entry already reads so when it holds no neighbour: no write)
      if (prev.y != kInvalid) A.res[i] = make_uint2(prev.x, kInvalid);
      if (LEARNED) A.r_used[i] = kInf;
      return;
    }
  }
  // The previous round's neighbour, if still in another component, is a real
  // cross edge of this point: a per-point cutoff.
  if (CARRIED && prev.y != kInvalid && A.labels[prev.y] != q.me)
    q.radius = fminf(q.radius, __uint_as_float(prev.x));
  if (LEARNED) q.radius = fminf(q.radius, __ldg(A.pred_r + i));
  const float r0 = q.radius;  // the search is exact within this cutoff
  if (LEARNED) A.r_used[i] = r0;
  if (MRD && q.core > r0) {  // every weight from this point is at least its core distance
    A.res[i] = make_uint2(__float_as_uint(q.core), kInvalid);
    return;
  }
  uint32_t st_node[kStackDepth];
  float st_dist[kStackDepth];
  unsigned long long nvis = 0;
  // A search that finds nothing within r0 leaves a lower bound of this
  // point's nearest other-component weight for the next round's skip test.
  // LB: the smallest weight bound of the children of other components that
  // the search rejected by distance (each above r0; every point of another
  // component lies in such a child, or in a leaf the search saw), instead of
  // r0 itself.  One-point leaves and the Euclidean weight only: there every
  // rejected candidate is a child rejected by its box distance.  (LBT false:
  // not tracked, where the tracking costs the searches more than the skips
  // it buys later.)
  constexpr bool LB = LBT && SEEDED && CARRIED && !CHUNKS && !LEARNED && !FIRST && !MRD;
  const bool ok = explore<COUNT, CHUNKS, FIRST, MRD, TIES, LB>(q, start, A.nodes, A.nlabels, A.pts, A.labels,
                                                     A.leaf, n, st_node, st_dist, nvis, A.core2,
                                                     A.ties, COUNT ? A.seen : nullptr);
  if (!ok) atomicOr(A.status, kErrStack);
  if (COUNT) {
    // one atomic per warp: sum the active lanes' counts first
    const unsigned mask = __activemask();
    const unsigned v = __reduce_add_sync(mask, (unsigned)nvis);
    if ((threadIdx.x & 31) == (unsigned)(__ffs(mask) - 1)) {
      atomicAdd(A.visits, (unsigned long long)v);
      atomicAdd(A.queries, (unsigned long long)__popc(mask));
    }
  }
  if (SEEDED) {
    // Report only the exact nearest neighbour within r0 (a seed beyond r0 is
    // dropped); keep in res.x a lower bound for the next round: the found
    // weight, or r0 when nothing lies within it.
    const bool found = q.bj != kInvalid && q.best <= r0;
    if (!found) q.bj = kInvalid;
    float lb = found ? q.best : (r0 < kInf ? r0 : 0.0f);
    // (LB, nothing found: q.best is that bound, above r0, or +inf when the
    // search met no other component at all; r0 is kept then)
    if (LB && !found && r0 < kInf && q.best < kInf) lb = q.best;
    A.res[i] = make_uint2(__float_as_uint(lb), q.bj);
  } else {
    A.res[i] = make_uint2(__float_as_uint(q.best), q.bj);
  }
  if (q.bj != kInvalid) {
    const uint32_t oi = __float_as_uint(p.w);
    const uint32_t oj = q.bid != kInvalid ? q.bid : __float_as_uint(A.pts[q.bj].w);
    offer_best(A.comp + q.me, __float_as_uint(q.best), oi, oj, A.labels, q.bj, A.status);
  }
}

}  // namespace emst

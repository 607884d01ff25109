// rounds.cu -- one Boruvka round of the method (§3, Fig. 3 loop body):
//   A5 node labels (Optimization 1, Fig. 4), A6 component upper bounds
//   (Optimization 2), A7 nearest-other-component traversal (Algorithm 2),
//   A8 per-component minimum, A9 merge (§3 "Merging components together"),
// plus the final ordering of the edges (A12).
#include "traverse.cuh"

namespace emst {

constexpr int kBlock = 256;

// ---------------------------------------------------------------------------
// A5. Node labels (the reduceLabels step of §3, Optimization 1; Fig. 4): a
// node's label is the label shared by all of its leaves, else kInvalid.  The
// leaves of a node are a contiguous range [a, b] of curve positions, so the
// node is single-component iff no label boundary lies inside the range.  With
// runs[k] = number of positions m < k where labels[m] != labels[m+1] (one
// prefix scan), that is runs[b] == runs[a], and the label is labels[a].  The
// result equals the bottom-up combination of the paper (equal child labels ->
// that label, else invalid) without its atomics and climbing threads.
// ---------------------------------------------------------------------------
constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;
constexpr uint32_t kScanAggregate = 1u << 30;
constexpr uint32_t kScanPrefix = 2u << 30;
constexpr uint32_t kScanMask = (1u << 30) - 1u;

// Single-pass exclusive scan of the boundary flags with decoupled look-back.
__global__ void __launch_bounds__(kScanThreads) k_label_runs(const uint32_t *__restrict__ labels,
                                                             int64_t n, uint32_t *__restrict__ runs,
                                                             uint32_t *lookback,
                                                             uint32_t *tile_counter,
                                                             uint32_t *status) {
  __shared__ uint32_t s_tile;
  __shared__ uint32_t s_warp[kScanThreads / 32];
  __shared__ uint32_t s_prefix;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) s_tile = atomicAdd(tile_counter, 1u);
  __syncthreads();
  const uint32_t tile = s_tile;
  const int64_t first = (int64_t)tile * kScanTile + (int64_t)tid * kScanItems;
  uint32_t flags = 0;  // bit q: boundary after position first+q
  uint32_t lab[kScanItems + 1];
#pragma unroll
  for (int q = 0; q <= kScanItems; ++q) {
    int64_t k = first + q;
    lab[q] = k < n ? __ldg(labels + k) : kInvalid;
  }
#pragma unroll
  for (int q = 0; q < kScanItems; ++q) {
    int64_t k = first + q;
    if (k + 1 < n && lab[q] != lab[q + 1]) flags |= 1u << q;
  }
  const uint32_t mine = __popc(flags);
  uint32_t x = mine;
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = lane < kScanThreads / 32 ? s_warp[lane] : 0u;
    uint32_t z = w;
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, z, o);
      if (lane >= o) z += y;
    }
    if (lane < kScanThreads / 32) s_warp[lane] = z - w;  // exclusive per warp
    const uint32_t total = __shfl_sync(0xffffffffu, z, kScanThreads / 32 - 1);
    if (lane == 0) {
      volatile uint32_t *lb = lookback + tile;
      *lb = (tile == 0 ? kScanPrefix : kScanAggregate) | total;
      uint32_t excl = 0;
      if (tile > 0) {
        for (int64_t j = (int64_t)tile - 1; j >= 0; --j) {
          const volatile uint32_t *pj = lookback + j;
          uint32_t wv = *pj;
          int spins = 0;
          while ((wv & ~kScanMask) == 0u) {
            if (++spins > (1 << 22)) { atomicOr(status, kErrSpin); wv = kScanPrefix; break; }
            __nanosleep(32);
            wv = *pj;
          }
          excl += wv & kScanMask;
          if ((wv & ~kScanMask) == kScanPrefix) break;
        }
        *lb = kScanPrefix | ((excl + total) & kScanMask);
      }
      s_prefix = excl;
    }
  }
  __syncthreads();
  uint32_t run = s_prefix + s_warp[warp] + x - mine;
#pragma unroll
  for (int q = 0; q < kScanItems; ++q) {
    int64_t k = first + q;
    if (k < n) runs[k] = run;
    run += (flags >> q) & 1u;
  }
}

__global__ void __launch_bounds__(kBlock) k_node_labels(const uint32_t *__restrict__ labels,
                                                        const uint32_t *__restrict__ runs,
                                                        const uint4 *__restrict__ range,
                                                        int64_t n, int64_t nc, int leaf,
                                                        NodeRec *__restrict__ nodes) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nc - 1) return;
  // the children split the node's chunk range [first, last] after `split`
  const uint4 r = __ldg(range + i);
  const int64_t a0 = (int64_t)r.x * leaf;
  const int64_t b0 = ((int64_t)r.y + 1) * leaf - 1;
  const int64_t a1 = b0 + 1;
  const int64_t b1 = ((int64_t)r.z + 1) * leaf < n ? ((int64_t)r.z + 1) * leaf - 1 : n - 1;
  const uint32_t l0 = __ldg(labels + a0), l1 = __ldg(labels + a1);
  const uint32_t lab0 = (__ldg(runs + b0) == __ldg(runs + a0)) ? l0 : kInvalid;
  const uint32_t lab1 = (__ldg(runs + b1) == __ldg(runs + a1)) ? l1 : kInvalid;
  reinterpret_cast<uint2 *>(&nodes[i].d)[1] = make_uint2(lab0, lab1);
}

void launch_label_runs(Problem &P) {
  const int64_t tiles = (P.n + kScanTile - 1) / kScanTile;
  uint32_t *ctr = P.counters + 24;
  cudaMemsetAsync(ctr, 0, sizeof(uint32_t), P.stream);
  cudaMemsetAsync(P.sort_lookback, 0, sizeof(uint32_t) * (size_t)tiles, P.stream);
  k_label_runs<<<(unsigned)tiles, kScanThreads, 0, P.stream>>>(P.labels, P.n, P.runs,
                                                               P.sort_lookback, ctr,
                                                               P.counters + 1);
  P.launches += 1;
}

void launch_node_labels(Problem &P) {
  k_node_labels<<<grid_for(P.nc - 1, kBlock), kBlock, 0, P.stream>>>(
      P.labels, P.runs, P.range, P.n, P.nc, P.leaf, P.nodes);
  P.launches += 1;
}

// ---------------------------------------------------------------------------
// A6. Upper bounds (computeUpperBounds): every pair of curve neighbours with
// different labels bounds the shortest outgoing edge of both components.
// bound[] holds FP32 bits (non-negative, so they order like uint32);
// kNoBound is +inf.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kBlock) k_upper_bounds(const float4 *__restrict__ pts,
                                                         const uint32_t *__restrict__ labels,
                                                         const uint32_t *__restrict__ inst_of,
                                                         int64_t n, uint32_t *bound) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k + 1 >= n) return;
  uint32_t la = labels[k], lb = labels[k + 1];
  if (la == lb) return;
  if (inst_of && __ldg(inst_of + k) != __ldg(inst_of + k + 1)) return;  // different instances
  float4 p = pts[k], q = pts[k + 1];
  uint32_t w = __float_as_uint(sq_dist(p.x, p.y, p.z, q.x, q.y, q.z));
  atomicMin(&bound[la], w);
  atomicMin(&bound[lb], w);
}

void launch_upper_bounds(Problem &P) {
  k_upper_bounds<<<grid_for(P.n, kBlock), kBlock, 0, P.stream>>>(P.pts, P.labels, P.inst_of, P.n,
                                                                 P.bound);
  P.launches += 1;
}

// One thread per point, or (list != nullptr) a grid-stride pass over the
// listed points (the certification reruns of the learned radius).
template <bool CARRIED, bool RADIUS_IN, bool COUNT, bool SEEDED, bool CHUNKS, bool LEARNED>
__global__ void __launch_bounds__(kBlock) k_traverse(TravArgs A, const uint32_t *__restrict__ list,
                                                     const uint32_t *__restrict__ list_count) {
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (list) {
    const int64_t count = *list_count;
    for (int64_t t = gid; t < count; t += (int64_t)gridDim.x * blockDim.x)
      traverse_one<CARRIED, RADIUS_IN, COUNT, SEEDED, CHUNKS, LEARNED>(A, __ldg(list + t));
  } else if (gid < A.n) {
    traverse_one<CARRIED, RADIUS_IN, COUNT, SEEDED, CHUNKS, LEARNED>(A, gid);
  }
}

void launch_traverse(Problem &P, bool carried, const float *radius_in, int block, bool count,
                     bool seeded, int learned_pass) {
  if (block <= 0) block = kBlock;
  TravArgs A;
  A.pts = P.pts;
  A.nodes = P.nodes;
  A.labels = P.labels;
  A.bound = P.bound;
  A.radius_in = radius_in;
  A.leaf = P.leaf;
  A.inst_of = P.inst_of;
  A.inst_root = P.inst_root;
  A.offsets = P.offsets;
  A.res = P.res;
  A.res_id = P.res_id;
  A.comp_key = P.comp_key;
  A.n = P.n;
  A.status = P.counters + 1;
  A.visits = reinterpret_cast<unsigned long long *>(P.counters + 2);
  A.pred_r = P.pred_r;
  A.r_used = P.r_used;
  // learned_pass: 0 = plain, 1 = with the proposed radii, 2 = rerun of the
  // listed points with the plain cutoff
  const uint32_t *list = learned_pass == 2 ? P.rerun_list : nullptr;
  const uint32_t *list_count = learned_pass == 2 ? P.counters + 13 : nullptr;
  const int g = learned_pass == 2 ? 152 * 8 : grid_for(P.n, block);
  cudaStream_t s = P.stream;
#define EMST_TRAV2(C, R, K, S, H, L) k_traverse<C, R, K, S, H, L><<<g, block, 0, s>>>(A, list, list_count)
#define EMST_TRAV(C, R, K, S, L)                       \
  do {                                                 \
    if (P.leaf > 1) EMST_TRAV2(C, R, K, S, true, L);   \
    else EMST_TRAV2(C, R, K, S, false, L);             \
  } while (0)
  if (radius_in) {
    EMST_TRAV(false, true, false, false, false);
  } else if (!seeded) {
    EMST_TRAV(false, false, false, false, false);
  } else if (learned_pass == 1) {
    if (carried) {
      if (count) EMST_TRAV(true, false, true, true, true); else EMST_TRAV(true, false, false, true, true);
    } else {
      if (count) EMST_TRAV(false, false, true, true, true); else EMST_TRAV(false, false, false, true, true);
    }
  } else if (carried) {
    if (count) EMST_TRAV(true, false, true, true, false); else EMST_TRAV(true, false, false, true, false);
  } else {
    if (count) EMST_TRAV(false, false, true, true, false); else EMST_TRAV(false, false, false, true, false);
  }
#undef EMST_TRAV
#undef EMST_TRAV2
  P.launches += 1;
}

// ---------------------------------------------------------------------------
// A8 (second half). Among the points whose (w, min id) equals the component's
// winner, the smallest max id: together the exact minimum of the key
// (w, min id, max id) of §2 over the component.  Also clears the other
// round's bound buffer (bound_next) for the relabel pass that fills it.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kBlock) k_reduce_max(const float4 *__restrict__ pts,
                                                       const uint32_t *__restrict__ labels,
                                                       const uint2 *__restrict__ res,
                                                       const uint32_t *__restrict__ res_id,
                                                       const uint64_t *__restrict__ comp_key,
                                                       uint32_t *comp_max,
                                                       uint32_t *__restrict__ bound_next,
                                                       int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (bound_next) bound_next[i] = kNoBound;
  uint2 r = res[i];
  if (r.y == kInvalid) return;
  uint32_t me = labels[i];
  uint32_t oi = __float_as_uint(pts[i].w), oj = res_id[i];
  uint64_t key = ((uint64_t)r.x << 32) | (uint64_t)(oi < oj ? oi : oj);
  if (key == comp_key[me]) atomicMin(&comp_max[me], oi < oj ? oj : oi);
}

void launch_reduce(Problem &P) {
  k_reduce_max<<<grid_for(P.n, kBlock), kBlock, 0, P.stream>>>(
      P.pts, P.labels, P.res, P.res_id, P.comp_key, P.comp_max, P.bound_buf[P.cur ^ 1], P.n);
  P.launches += 1;
}

// ---------------------------------------------------------------------------
// A9. Merge.  (a) every component C with an edge points to T(C), the label of
// the edge's outside endpoint; (b) following the chain C -> T(C) -> ... ends
// in a mutual pair X <-> T(X) (edge weights strictly decrease along a chain
// under the total order, so there is no longer cycle); the new label is the
// smaller label of that pair.  The pair's shared edge is emitted once, by its
// smaller side; every other component emits its own edge.  (A component with
// no edge -- possible only when a given radius cut every query short -- ends
// any chain that reaches it and keeps its label.)  Components are visited
// through the list of active labels (all n in the first round); each new root
// appends itself to the next round's list.  (c) relabel every point (A9) and,
// in the same pass, prepare the next round: its curve-pair upper bounds (A6)
// and the label-boundary prefix scan the node labels (A5) need.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kBlock) k_merge_targets(const uint32_t *__restrict__ list,
                                                          int64_t count,
                                                          const uint64_t *__restrict__ comp_key,
                                                          const uint32_t *__restrict__ comp_max,
                                                          const uint32_t *__restrict__ inv,
                                                          const uint32_t *__restrict__ labels,
                                                          uint32_t *__restrict__ target,
                                                          uint32_t *status) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= count) return;
  const uint32_t c = list ? list[t] : (uint32_t)t;
  uint64_t key = comp_key[c];
  const uint32_t mx = comp_max[c];
  if (key == kEmptyKey || mx == kInvalid) {
    // (the second case cannot happen: the winner of the first half always
    // matches its own key in the second; guarded so no index is ever wild)
    if (key != kEmptyKey) atomicOr(status, kErrChain);
    target[c] = kInvalid;
    return;
  }
  uint32_t lmn = labels[inv[(uint32_t)key]];
  uint32_t lmx = labels[inv[mx]];
  target[c] = (lmn == c) ? lmx : lmn;
}

__global__ void __launch_bounds__(kBlock) k_merge_roots(const uint32_t *__restrict__ list,
                                                        int64_t count,
                                                        uint64_t *__restrict__ comp_key,
                                                        uint32_t *__restrict__ comp_max,
                                                        const uint32_t *__restrict__ target,
                                                        uint32_t *__restrict__ root,
                                                        emst_edge *__restrict__ edges,
                                                        uint32_t *__restrict__ next_list,
                                                        uint32_t *counters, int64_t n) {
  int64_t t64 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t64 >= count) return;
  const uint32_t c = list ? list[t64] : (uint32_t)t64;
  const uint64_t key = comp_key[c];
  const uint32_t t = key == kEmptyKey ? kInvalid : target[c];
  uint32_t r = c;
  if (t != kInvalid) {
    const bool mutual = target[t] == c;
    if (!mutual || c < t) {
      uint32_t e = atomicAdd(&counters[0], 1u);
      emst_edge E;
      E.i = (uint32_t)key;
      E.j = comp_max[c];
      E.w = __uint_as_float((uint32_t)(key >> 32));
      edges[e] = E;
    }
    uint32_t x = c;
    for (int64_t steps = 0;; ++steps) {
      uint32_t y = target[x];
      if (y == kInvalid) { r = x; break; }  // chain ends at a component without an edge
      if (target[y] == x) { r = x < y ? x : y; break; }
      x = y;
      if (steps > n) { atomicOr(&counters[1], kErrChain); r = x; break; }
    }
    comp_key[c] = kEmptyKey;
    comp_max[c] = kInvalid;
  }
  root[c] = r;
  if (r == c) next_list[atomicAdd(&counters[12], 1u)] = c;
}

// Relabel + next round's bounds + label-boundary scan, one tile of positions
// per CTA, decoupled look-back for the scan.  New labels go to a second
// buffer (neighbouring tiles still read the old ones).
constexpr int kRelabelItems = 8;
constexpr int kRelabelTile = kScanThreads * kRelabelItems;

__global__ void __launch_bounds__(kScanThreads, 6) k_relabel_runs(
    const uint32_t *__restrict__ labels_old, const uint32_t *__restrict__ root,
    const float4 *__restrict__ pts, const uint32_t *__restrict__ inst_of, int64_t n,
    uint32_t *__restrict__ labels_new,
    uint32_t *__restrict__ bound_next, uint32_t *__restrict__ runs, uint32_t *lookback,
    uint32_t *tile_counter, uint32_t *status) {
  __shared__ uint32_t s_tile;
  __shared__ uint32_t s_warp[kScanThreads / 32];
  __shared__ uint32_t s_prefix;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) s_tile = atomicAdd(tile_counter, 1u);
  __syncthreads();
  const uint32_t tile = s_tile;
  const int64_t first = (int64_t)tile * kRelabelTile + (int64_t)tid * kRelabelItems;
  uint32_t lab[kRelabelItems + 1];
#pragma unroll
  for (int q = 0; q <= kRelabelItems; ++q) {
    int64_t k = first + q;
    lab[q] = k < n ? __ldg(root + __ldg(labels_old + k)) : kInvalid;
  }
  uint32_t flags = 0;
#pragma unroll
  for (int q = 0; q < kRelabelItems; ++q) {
    int64_t k = first + q;
    if (k < n) labels_new[k] = lab[q];
    if (k + 1 < n && lab[q] != lab[q + 1]) {
      flags |= 1u << q;
      if (inst_of && __ldg(inst_of + k) != __ldg(inst_of + k + 1)) continue;  // no cross-instance bound
      const float4 p = __ldg(pts + k), r = __ldg(pts + k + 1);
      const uint32_t w = __float_as_uint(sq_dist(p.x, p.y, p.z, r.x, r.y, r.z));
      atomicMin(&bound_next[lab[q]], w);
      atomicMin(&bound_next[lab[q + 1]], w);
    }
  }
  const uint32_t mine = __popc(flags);
  uint32_t x = mine;
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = lane < kScanThreads / 32 ? s_warp[lane] : 0u;
    uint32_t z = w;
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, z, o);
      if (lane >= o) z += y;
    }
    if (lane < kScanThreads / 32) s_warp[lane] = z - w;
    const uint32_t total = __shfl_sync(0xffffffffu, z, kScanThreads / 32 - 1);
    if (lane == 0) {
      volatile uint32_t *lb = lookback + tile;
      *lb = (tile == 0 ? kScanPrefix : kScanAggregate) | total;
      uint32_t excl = 0;
      if (tile > 0) {
        for (int64_t j = (int64_t)tile - 1; j >= 0; --j) {
          const volatile uint32_t *pj = lookback + j;
          uint32_t wv = *pj;
          int spins = 0;
          while ((wv & ~kScanMask) == 0u) {
            if (++spins > (1 << 22)) { atomicOr(status, kErrSpin); wv = kScanPrefix; break; }
            __nanosleep(32);
            wv = *pj;
          }
          excl += wv & kScanMask;
          if ((wv & ~kScanMask) == kScanPrefix) break;
        }
        *lb = kScanPrefix | ((excl + total) & kScanMask);
      }
      s_prefix = excl;
    }
  }
  __syncthreads();
  uint32_t run = s_prefix + s_warp[warp] + x - mine;
#pragma unroll
  for (int q = 0; q < kRelabelItems; ++q) {
    int64_t k = first + q;
    if (k < n) runs[k] = run;
    run += (flags >> q) & 1u;
  }
}

void launch_merge(Problem &P) {
  const int64_t count = P.active_list ? P.n_active : P.n;
  const int g = grid_for(count, kBlock);
  cudaMemsetAsync(P.counters + 12, 0, sizeof(uint32_t), P.stream);
  k_merge_targets<<<g, kBlock, 0, P.stream>>>(P.active_list, count, P.comp_key, P.comp_max, P.inv,
                                              P.labels, P.target, P.counters + 1);
  k_merge_roots<<<g, kBlock, 0, P.stream>>>(P.active_list, count, P.comp_key, P.comp_max, P.target,
                                            P.root, P.edges, P.next_list, P.counters, P.n);
  const int64_t tiles = (P.n + kRelabelTile - 1) / kRelabelTile;
  uint32_t *ctr = P.counters + 24;
  cudaMemsetAsync(ctr, 0, sizeof(uint32_t), P.stream);
  cudaMemsetAsync(P.sort_lookback, 0, sizeof(uint32_t) * (size_t)tiles, P.stream);
  k_relabel_runs<<<(unsigned)tiles, kScanThreads, 0, P.stream>>>(
      P.labels, P.root, P.pts, P.inst_of, P.n, P.labels_buf[P.cur ^ 1], P.bound_buf[P.cur ^ 1], P.runs,
      P.sort_lookback, ctr, P.counters + 1);
  P.launches += 3;
}

// After the host has seen a round finish: the next round's labels, bounds and
// active list become current.
void advance_round(Problem &P, int64_t n_active) {
  P.cur ^= 1;
  P.labels = P.labels_buf[P.cur];
  P.bound = P.bound_buf[P.cur];
  uint32_t *t = P.list_buf[0] == P.next_list ? P.list_buf[1] : P.list_buf[0];
  P.active_list = P.next_list;
  P.next_list = t;
  P.n_active = n_active;
}

__global__ void k_fill_u32(uint32_t *p, uint32_t v, int64_t count) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < count) p[k] = v;
}

void launch_fill_u32(Problem &P, uint32_t *p, uint32_t v, int64_t count) {
  if (count <= 0) return;
  k_fill_u32<<<grid_for(count, kBlock), kBlock, 0, P.stream>>>(p, v, count);
  P.launches += 1;
}

// ---------------------------------------------------------------------------
// A12. Output order: (w, i, j) ascending, by two stable radix sorts (first by
// j, then by (w bits << L) | i), then a gather.
// ---------------------------------------------------------------------------
__global__ void k_edge_keys_j(const emst_edge *__restrict__ edges, int64_t m,
                              uint64_t *__restrict__ keys, uint32_t *__restrict__ vals) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m) return;
  keys[e] = edges[e].j;
  vals[e] = (uint32_t)e;
}

__global__ void k_edge_keys_wi(const emst_edge *__restrict__ edges, int64_t m,
                               uint64_t *__restrict__ keys, const uint32_t *__restrict__ vals,
                               int shift_i) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m) return;
  emst_edge E = edges[vals[e]];
  keys[e] = ((uint64_t)__float_as_uint(E.w) << shift_i) | (uint64_t)E.i;
}

__global__ void k_edge_keys_inst(const emst_edge *__restrict__ edges, int64_t m,
                                 uint64_t *__restrict__ keys, const uint32_t *__restrict__ vals,
                                 const uint32_t *__restrict__ inst_in) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m) return;
  keys[e] = __ldg(inst_in + edges[vals[e]].i);
}

// Final order, with ids made local to their instance in the batched form.
__global__ void k_edge_gather(const emst_edge *__restrict__ edges, int64_t m,
                              const uint32_t *__restrict__ order, emst_edge *__restrict__ out,
                              const uint32_t *__restrict__ inst_in,
                              const int64_t *__restrict__ offsets) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m) return;
  emst_edge E = edges[order[e]];
  if (inst_in) {
    const uint32_t base = (uint32_t)__ldg(offsets + __ldg(inst_in + E.i));
    E.i -= base;
    E.j -= base;
  }
  out[e] = E;
}

void launch_edge_keys_j(Problem &P, int64_t m) {
  k_edge_keys_j<<<grid_for(m, kBlock), kBlock, 0, P.stream>>>(P.edges, m, P.keys[0], P.vals[0]);
  P.launches += 1;
}
void launch_edge_keys_wi(Problem &P, int64_t m, int src, int shift_i) {
  k_edge_keys_wi<<<grid_for(m, kBlock), kBlock, 0, P.stream>>>(P.edges, m, P.keys[src], P.vals[src],
                                                               shift_i);
  P.launches += 1;
}
void launch_edge_keys_inst(Problem &P, int64_t m, int src) {
  k_edge_keys_inst<<<grid_for(m, kBlock), kBlock, 0, P.stream>>>(P.edges, m, P.keys[src],
                                                                  P.vals[src], P.inst_in);
  P.launches += 1;
}
void launch_edge_gather(Problem &P, int64_t m, const uint32_t *order, emst_edge *out) {
  k_edge_gather<<<grid_for(m, kBlock), kBlock, 0, P.stream>>>(P.edges, m, order, out, P.inst_in,
                                                              P.offsets);
  P.launches += 1;
}

}  // namespace emst

// rounds.cu -- one Boruvka round of the method (§3, Fig. 3 loop body):
//   A5 node labels (Optimization 1, Fig. 4), A6 component upper bounds
//   (Optimization 2), A7 nearest-other-component traversal (Algorithm 2),
//   A9 merge (§3 "Merging components together"; the A8 minimum itself is
//   taken at the end of every query, offer_best in traverse.cuh),
// plus the final ordering of the edges (A12).
#include "traverse.cuh"

namespace emst {

constexpr int kBlock = 256;

// The weight of curve neighbours k and k + 1 (core2: the mutual reachability
// weight, §4.5).
__device__ __forceinline__ float pair_weight(const float4 &p, const float4 &q,
                                             const float *__restrict__ core2, int64_t k) {
  float w = sq_dist(p.x, p.y, p.z, q.x, q.y, q.z);
  if (core2) w = fmaxf(w, fmaxf(__ldg(core2 + k), __ldg(core2 + k + 1)));
  return w;
}

// ---------------------------------------------------------------------------
// A5. Node labels (the reduceLabels step of §3, Optimization 1; Fig. 4): a
// node's label is the label shared by all of its leaves, else kInvalid.  The
// leaves of a node are a contiguous range [a, b] of curve positions, so the
// node is single-component iff no label boundary lies inside the range.  With
// runs[k] = number of positions m < k where labels[m] != labels[m+1] (a
// prefix count), that is runs[b] == runs[a], and the label is labels[a].  The
// result equals the bottom-up combination of the paper (equal child labels ->
// that label, else invalid) without its atomics and climbing threads.
//
// runs[k] is kept in three parts, so no tile waits on another and the node
// pass reads a small array that stays in L2: per word w of 32 positions, a
// bitmap of its boundaries (bit b: positions 32w + b and 32w + b + 1 differ)
// beside the count of boundaries before it within its tile of kScanTile
// positions (one 8-byte entry, carved from P.runs), and the count of all
// earlier tiles (tile_prefix, an exclusive scan of the tile totals done by
// the last tile to finish).
// ---------------------------------------------------------------------------
constexpr int kScanThreads = 256;
// Tile shape of the relabel pass (build knobs): 8 rows of 32 positions per
// warp at 8 CTAs per SM measured best at 37M halo points (rounds 40.90 ms;
// 16 rows at 6 CTAs 40.99, 16 at 8 40.92, 4 at 8 41.48).
#ifndef EMST_SCAN_ROWS_LOG2
#define EMST_SCAN_ROWS_LOG2 3
#endif
#ifndef EMST_SCAN_MIN_BLOCKS
#define EMST_SCAN_MIN_BLOCKS 8
#endif
constexpr int kScanItems = 1 << EMST_SCAN_ROWS_LOG2;  // rows of 32 positions per warp
constexpr int kScanTileShift = EMST_SCAN_ROWS_LOG2 + 8;
constexpr int kScanTile = 1 << kScanTileShift;
static_assert(kScanTile == kScanThreads * kScanItems, "scan tile shape");

int64_t scan_tiles_for(int64_t n) { return (n + kScanTile - 1) / kScanTile; }

__device__ __forceinline__ uint32_t runs_at(const uint2 *__restrict__ words,
                                            const uint32_t *__restrict__ tile_prefix, int64_t k) {
  const uint2 wd = __ldg(words + (k >> 5));  // (bitmap, boundaries before it in the tile)
  const uint32_t below = wd.x & ((1u << (k & 31)) - 1u);
  return __ldg(tile_prefix + (k >> kScanTileShift)) + wd.y + (uint32_t)__popc(below);
}

// Exclusive scan of count values by one CTA of kScanThreads threads, each
// summing a contiguous chunk (the values come from other CTAs of the same
// launch: read through L2).  Chunks are a multiple of 8 values and read 8 at
// a time with all 8 loads in flight: this runs on one CTA at the end of the
// launch, so its L2 round trips are the launch's tail.
__device__ void block_exclusive_scan(const uint32_t *in, uint32_t *out, int64_t count) {
  __shared__ uint32_t s_part[kScanThreads / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t chunk = ((count + kScanThreads - 1) / kScanThreads + 7) & ~(int64_t)7;
  const int64_t lo = (int64_t)tid * chunk < count ? (int64_t)tid * chunk : count;
  const int64_t hi = lo + chunk < count ? lo + chunk : count;
  uint32_t sum = 0;
  for (int64_t t = lo; t < hi; t += 8) {
    uint32_t v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = t + u < hi ? __ldcg(in + t + u) : 0u;
#pragma unroll
    for (int u = 0; u < 8; ++u) sum += v[u];
  }
  uint32_t x = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_part[warp] = x;
  __syncthreads();
  uint32_t base = 0;
  for (int w = 0; w < warp; ++w) base += s_part[w];
  uint32_t run = base + x - sum;
  for (int64_t t = lo; t < hi; t += 8) {
    uint32_t v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = t + u < hi ? __ldcg(in + t + u) : 0u;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      if (t + u < hi) out[t + u] = run;
      run += v[u];
    }
  }
}

// The boundary bitmap with its per-word counts, and the tile totals,
// one tile of kScanTile positions per CTA.  Warp-striped: warp w of the tile
// owns kScanItems rows of 32 consecutive positions, so every load and store
// is one coalesced 128-byte row, and a row's boundaries are one ballot: its
// word of the bitmap.  RELABEL:
// the labels are first mapped through root (the merge's new labels, written
// to labels_new), and every boundary between two curve neighbours of one
// instance lowers both components' bounds for the next round (A6) -- one
// pass for A9's relabel, A6 and A5's counts.
template <bool RELABEL>
__global__ void __launch_bounds__(kScanThreads, EMST_SCAN_MIN_BLOCKS) k_runs(
    const uint32_t *__restrict__ labels_old, const uint32_t *__restrict__ root,
    const float4 *__restrict__ pts, const uint32_t *__restrict__ inst_of,
    const float *__restrict__ core2, int64_t n,
    uint32_t *__restrict__ labels_new, uint32_t *__restrict__ bound_next,
    uint2 *__restrict__ words, uint32_t *tile_total, uint32_t *tile_prefix, uint32_t *done) {
  __shared__ uint32_t s_warp[kScanThreads / 32];
  __shared__ uint32_t s_last;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t tile = blockIdx.x;
  const int64_t seg = (int64_t)tile * kScanTile + (int64_t)warp * 32 * kScanItems;
  // positions of this warp that exist (32-bit indexing within the segment)
  const int64_t rem64 = n - seg;
  const int rem = rem64 > 32 * kScanItems ? 32 * kScanItems + 1 : (int)(rem64 > 0 ? rem64 : 0);
  const uint32_t *lo = labels_old + seg;
  uint32_t lab[kScanItems];
#pragma unroll
  for (int q = 0; q < kScanItems; ++q) {
    const int k = q * 32 + lane;
    lab[q] = k < rem ? __ldg(lo + k) : kInvalid;
  }
  // the position after the warp's last row
  uint32_t tail = kInvalid;
  if (lane == 0 && 32 * kScanItems < rem) tail = __ldg(lo + 32 * kScanItems);
  if (RELABEL) {
#pragma unroll
    for (int q = 0; q < kScanItems; ++q)
      if (lab[q] != kInvalid) lab[q] = __ldg(root + lab[q]);
    if (tail != kInvalid) tail = __ldg(root + tail);
  }
  tail = __shfl_sync(0xffffffffu, tail, 0);
  uint32_t flags = 0;  // bit q: boundary between row q's position and the next one
  uint32_t wtotal = 0;
#pragma unroll
  for (int q = 0; q < kScanItems; ++q) {
    const int k = q * 32 + lane;
    uint32_t nxt = __shfl_down_sync(0xffffffffu, lab[q], 1);
    const uint32_t row_next =
        q + 1 < kScanItems ? __shfl_sync(0xffffffffu, lab[q + 1 < kScanItems ? q + 1 : q], 0) : tail;
    if (lane == 31) nxt = row_next;
    const bool f = k + 1 < rem && lab[q] != nxt;
    if (f) {
      flags |= 1u << q;
      if (RELABEL && !(inst_of && __ldg(inst_of + seg + k) != __ldg(inst_of + seg + k + 1))) {
        // (no bound across instances)
        const float4 p = __ldg(pts + seg + k), r = __ldg(pts + seg + k + 1);
        const uint32_t w = __float_as_uint(pair_weight(p, r, core2, seg + k));
        atomicMin(&bound_next[lab[q]], w);
        atomicMin(&bound_next[nxt], w);
      }
    }
    if (RELABEL && k < rem) labels_new[seg + k] = lab[q];
    wtotal += __popc(__ballot_sync(0xffffffffu, f));
  }
  if (lane == 0) s_warp[warp] = wtotal;
  __syncthreads();
  uint32_t run = 0, total = 0;
#pragma unroll
  for (int w = 0; w < kScanThreads / 32; ++w) {
    const uint32_t v = s_warp[w];
    run += w < warp ? v : 0u;
    total += v;
  }
  // lane q writes row q's word and the tile's boundaries before it
  uint32_t my_bits = 0, my_prefix = 0;
#pragma unroll
  for (int q = 0; q < kScanItems; ++q) {
    const uint32_t b = __ballot_sync(0xffffffffu, (flags >> q) & 1u);
    if (lane == q) { my_bits = b; my_prefix = run; }
    run += __popc(b);
  }
  if (lane < kScanItems && lane * 32 < rem) words[(seg >> 5) + lane] = make_uint2(my_bits, my_prefix);
  // the last tile to finish scans the tile totals
  if (tid == 0) {
    tile_total[tile] = total;
    __threadfence();
    s_last = atomicAdd(done, 1u) == gridDim.x - 1 ? 1u : 0u;
  }
  __syncthreads();
  if (s_last) {
    __threadfence();
    block_exclusive_scan(tile_total, tile_prefix, gridDim.x);
  }
}

static void launch_runs(Problem &P, bool relabel) {
  const int64_t tiles = scan_tiles_for(P.n);
  uint32_t *done = P.counters + 24;
  uint32_t *tile_total = P.scan_tiles, *tile_prefix = P.scan_tiles + tiles;
  uint2 *words = reinterpret_cast<uint2 *>(P.runs);
  cudaMemsetAsync(done, 0, sizeof(uint32_t), P.stream);
  if (relabel)
    k_runs<true><<<(unsigned)tiles, kScanThreads, 0, P.stream>>>(
        P.labels, P.root, P.pts, P.inst_of, P.core2, P.n, P.labels_buf[P.cur ^ 1],
        P.bound_buf[P.cur ^ 1], words, tile_total, tile_prefix, done);
  else
    k_runs<false><<<(unsigned)tiles, kScanThreads, 0, P.stream>>>(
        P.labels, nullptr, P.pts, P.inst_of, nullptr, P.n, nullptr, nullptr, words, tile_total,
        tile_prefix, done);
  P.launches += 1;
}

void launch_label_runs(Problem &P) { launch_runs(P, false); }

__global__ void __launch_bounds__(kBlock) k_node_labels(const uint32_t *__restrict__ labels,
                                                        const uint2 *__restrict__ words,
                                                        const uint32_t *__restrict__ tile_prefix,
                                                        const uint2 *__restrict__ range,
                                                        int64_t n, int64_t nc, int leaf,
                                                        uint2 *__restrict__ nlabels) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nc - 1) return;
  // the children split the node's chunk range [first, last] after `split`
  const NodeRange r = unpack_range((uint32_t)i, __ldg(range + i));
  const int64_t a0 = (int64_t)r.first * leaf;
  const int64_t b0 = ((int64_t)r.split + 1) * leaf - 1;
  const int64_t a1 = b0 + 1;
  const int64_t b1 = ((int64_t)r.last + 1) * leaf < n ? ((int64_t)r.last + 1) * leaf - 1 : n - 1;
  const uint32_t l0 = __ldg(labels + a0), l1 = __ldg(labels + a1);
  const uint32_t lab0 =
      runs_at(words, tile_prefix, b0) == runs_at(words, tile_prefix, a0) ? l0 : kInvalid;
  const uint32_t lab1 =
      runs_at(words, tile_prefix, b1) == runs_at(words, tile_prefix, a1) ? l1 : kInvalid;
  nlabels[i] = make_uint2(lab0, lab1);
}

void launch_node_labels(Problem &P) {
  k_node_labels<<<grid_for(P.nc - 1, kBlock), kBlock, 0, P.stream>>>(
      P.labels, reinterpret_cast<const uint2 *>(P.runs), P.scan_tiles + scan_tiles_for(P.n), P.range,
      P.n, P.nc, P.leaf, P.nlabels);
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
                                                         const float *__restrict__ core2,
                                                         int64_t n, uint32_t *bound) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k + 1 >= n) return;
  uint32_t la = labels[k], lb = labels[k + 1];
  if (la == lb) return;
  if (inst_of && __ldg(inst_of + k) != __ldg(inst_of + k + 1)) return;  // different instances
  float4 p = pts[k], q = pts[k + 1];
  uint32_t w = __float_as_uint(pair_weight(p, q, core2, k));
  atomicMin(&bound[la], w);
  atomicMin(&bound[lb], w);
}

void launch_upper_bounds(Problem &P) {
  k_upper_bounds<<<grid_for(P.n, kBlock), kBlock, 0, P.stream>>>(P.pts, P.labels, P.inst_of,
                                                                 P.core2, P.n, P.bound);
  P.launches += 1;
}

// One thread per point, or (list != nullptr) a grid-stride pass over the
// listed points (the certification reruns of the learned radius).
template <bool CARRIED, bool RADIUS_IN, bool COUNT, bool SEEDED, bool CHUNKS, bool LEARNED,
          bool FIRST, bool MRD, bool TIES = true, bool LBT = true>
__global__ void __launch_bounds__(kTraverseMaxBlock, EMST_TRAVERSE_MIN_BLOCKS) k_traverse(TravArgs A, const uint32_t *__restrict__ list,
                                                     const uint32_t *__restrict__ list_count) {
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (list && A.queue) {
    // the next 32 entries for this warp, in list order, so the queries in
    // flight stay a window of the list (and of the curve) that L2 holds
    const uint32_t count = *list_count;
    const int lane = threadIdx.x & 31;
    for (;;) {
      uint32_t base = 0;
      if (lane == 0) base = atomicAdd(A.queue, 32u);
      base = __shfl_sync(0xffffffffu, base, 0);
      if (base >= count) break;
      if (base + lane < count)
        traverse_one<CARRIED, RADIUS_IN, COUNT, SEEDED, CHUNKS, LEARNED, FIRST, MRD, TIES, LBT>(
            A, __ldg(list + base + lane));
      __syncwarp();
    }
  } else if (list) {
    const int64_t count = *list_count;
    for (int64_t t = gid; t < count; t += (int64_t)gridDim.x * blockDim.x)
      traverse_one<CARRIED, RADIUS_IN, COUNT, SEEDED, CHUNKS, LEARNED, FIRST, MRD, TIES, LBT>(A, __ldg(list + t));
  } else if (gid < A.n) {
    traverse_one<CARRIED, RADIUS_IN, COUNT, SEEDED, CHUNKS, LEARNED, FIRST, MRD, TIES, LBT>(A, gid);
  }
}

// ---------------------------------------------------------------------------
// A7, persistent form: a resident grid whose warps take queries from a
// global work queue (the curve positions in order, handed out in chunks of
// `chunk` consecutive positions per warp, so the queries a warp holds stay
// close on the curve and share node records in L1) and refill a lane as soon
// as its search ends, instead of holding 32 queries until the longest one
// finishes.  Each loop iteration: when at least `refill` lanes are idle (or
// all are), they take the next positions of the warp's chunk and start them
// (a query skipped by its lower bound finishes at once and leaves its lane
// idle); then every lane with a search in progress makes one node visit (or
// pops).  Same per-query arithmetic as traverse_one, so the same results.
// One-point leaves, no learned cutoff, no mutual reachability.
// ---------------------------------------------------------------------------
#ifndef EMST_PERSIST_MIN_BLOCKS
#define EMST_PERSIST_MIN_BLOCKS 12
#endif
constexpr int kDefaultRefill = 16;   // measured best of 4 / 8 / 16 at 37M halo points
constexpr int kDefaultChunk = 64;    // measured best of 32 / 64 / 128

template <bool CARRIED, bool FIRST, bool TIES, bool COUNT>
__global__ void __launch_bounds__(kPersistBlock, EMST_PERSIST_MIN_BLOCKS)
    k_traverse_queue(TravArgs A, unsigned long long *queue, int refill, int chunk) {
  const unsigned lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const int64_t n = A.n;
  LocalStack stk;
  stk.init();
  Query q;
  uint32_t node = 0, i = 0;
  float r0 = 0.0f;
  bool live = false;
  unsigned long long nvis = 0, nq = 0;
  // this warp's current chunk [next, end) of curve positions (warp-uniform)
  int64_t next = 0, end = 0;
  bool drained = false;
  while (true) {
    const unsigned idle = __ballot_sync(0xffffffffu, !live);
    if (idle == 0xffffffffu && drained) break;
    if (!drained && __popc(idle) >= (idle == 0xffffffffu ? 1 : refill)) {
      const int need = __popc(idle);
      const int64_t avail = end - next;
      int64_t fresh = 0;
      if (avail < need) {
        if (lane == 0) fresh = (int64_t)atomicAdd(queue, (unsigned long long)chunk);
        fresh = __shfl_sync(0xffffffffu, fresh, 0);
      }
      if (!live) {
        const int rank = __popc(idle & lt);
        const int64_t t = rank < avail ? next + rank : fresh + (rank - avail);
        if (t < n) {
          i = (uint32_t)t;
          uint32_t start;
          live = start_query<CARRIED, false, true, false, false>(A, t, q, start, r0);
          if (live) {
            node = start;
            stk.init();
            if (COUNT) ++nq;
          }
        }
      }
      if (avail < need) {
        next = fresh + (need - avail);
        end = fresh + chunk;
      } else {
        next += need;
      }
      // chunks leave the queue in increasing order, so once this warp's next
      // position is past the end no later chunk holds a query either
      drained = next >= n;
    }
    if (live) {
      if (COUNT) {
        ++nvis;
        if (A.seen) atomicOr(A.seen + (node >> 5), 1u << (node & 31));
      }
      bool overflow = false;
      uint32_t nxt = visit<false, FIRST, false, TIES>(q, node, A.nodes, A.nlabels, A.pts, A.labels,
                                                      1, n, stk, overflow, nullptr, A.ties);
      if (overflow) atomicOr(A.status, kErrStack);
      if (nxt == kInvalid && !overflow) nxt = pop_next(q, stk);
      if (nxt == kInvalid || overflow) {
        finish_query<true>(A, i, q, r0);
        live = false;
      } else {
        node = nxt;
      }
    }
  }
  if (COUNT) {
    const unsigned long long v = __reduce_add_sync(0xffffffffu, (unsigned)nvis);
    const unsigned long long c = __reduce_add_sync(0xffffffffu, (unsigned)nq);
    if (lane == 0) {
      atomicAdd(A.visits, v);
      atomicAdd(A.queries, c);
    }
  }
}

template <bool CARRIED, bool FIRST, bool TIES, bool COUNT>
static void queue_launch(Problem &P, const TravArgs &A) {
  // chunk >= 32: a refill takes at most 32 positions, from at most two chunks
  const int chunk = P.queue_chunk >= 32 ? P.queue_chunk : kDefaultChunk;
  const int refill = P.refill_lanes >= 1 && P.refill_lanes <= 32 ? P.refill_lanes : kDefaultRefill;
  static int blocks_per_sm[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  const size_t sm = 0;
  auto kern = k_traverse_queue<CARRIED, FIRST, TIES, COUNT>;
  if (dev >= 0 && dev < 64 && blocks_per_sm[dev] == 0) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, kPersistBlock, sm) != cudaSuccess || b < 1) {
      cudaGetLastError();
      b = 1;
    }
    blocks_per_sm[dev] = b;
  }
  const int per_sm = (dev >= 0 && dev < 64) ? blocks_per_sm[dev] : 1;
  // no more warps than there are chunks of queries
  const int64_t warps_needed = (A.n + chunk - 1) / chunk;
  int64_t g = (int64_t)sm_count() * per_sm;
  const int64_t g_need = (warps_needed + kPersistBlock / 32 - 1) / (kPersistBlock / 32);
  if (g > g_need) g = g_need;
  if (g < 1) g = 1;
  kern<<<(unsigned)g, kPersistBlock, sm, P.stream>>>(A, reinterpret_cast<unsigned long long *>(P.counters + 36),
                                                     refill, chunk);
}

static void launch_traverse_queue(Problem &P, const TravArgs &A, bool carried, bool first, bool count) {
  cudaMemsetAsync(P.counters + 36, 0, sizeof(unsigned long long), P.stream);
  const bool ties = P.ties;
#define EMST_Q(C, F, T, K) queue_launch<C, F, T, K>(P, A)
  if (count) {
    if (carried) { if (ties) EMST_Q(true, false, true, true); else EMST_Q(true, false, false, true); }
    else if (first) { if (ties) EMST_Q(false, true, true, true); else EMST_Q(false, true, false, true); }
    else { if (ties) EMST_Q(false, false, true, true); else EMST_Q(false, false, false, true); }
  } else {
    if (carried) { if (ties) EMST_Q(true, false, true, false); else EMST_Q(true, false, false, false); }
    else if (first) { if (ties) EMST_Q(false, true, true, false); else EMST_Q(false, true, false, false); }
    else { if (ties) EMST_Q(false, false, true, false); else EMST_Q(false, false, false, false); }
  }
#undef EMST_Q
  P.launches += 1;
}

// ---------------------------------------------------------------------------
// The queries of a round that need a search (rounds from kCompactFromRound
// on, where many points skip theirs): a point whose lower bound exceeds its
// component's cutoff as the round starts (upper bound, best so far) is
// finished here exactly as traverse_one would finish it; the others are
// listed in curve order (k_active_count flags them and counts them per tile,
// its last CTA scans the tile counts, k_active_write writes the list) for
// the traversal, which tests them again against the cutoff as it has shrunk
// by then.  The list is a subset of
// what the one-thread-per-point launch would search, so the result is the
// same; its searches fill whole warps instead of a third of each.  The
// traversal's warps take the list 32 entries at a time from a counter, in
// list order, so the queries in flight stay one window of the curve whose
// node records L2 holds (a grid-stride walk spread them: round 3 read twice
// the DRAM bytes).  Measured at 37M halo points, ms per call: first listed
// round 1 / 2 / 3 with the ordered warps 45.48 / 45.31 / 46.40, with the
// grid-stride walk 2 / 3 / 4 / 5 48.46 / 48.24 / 49.43 / 49.71, no list
// 50.41.
// ---------------------------------------------------------------------------
#ifndef EMST_COMPACT_FROM_ROUND
#define EMST_COMPACT_FROM_ROUND 2
#endif
constexpr int kCompactFromRound = EMST_COMPACT_FROM_ROUND;
constexpr uint32_t kActiveCounter = 50;  // P.counters slot: listed queries
constexpr uint32_t kActiveQueue = 51;    // P.counters slot: list entries handed out
constexpr uint32_t kActiveDone = 52;     // P.counters slot: tiles of k_active_count finished
#ifndef EMST_ORDERED_UNTIL_ROUND
#define EMST_ORDERED_UNTIL_ROUND 6
#endif
constexpr int kOrderedUntilRound = EMST_ORDERED_UNTIL_ROUND;  // exact curve order before this round
#ifndef EMST_LIST_QUEUE
#define EMST_LIST_QUEUE 1
#endif

// The same with one atomic per warp of 128 positions (four per thread):
// the list is in curve order only within each warp's positions, which costs
// the traversal locality while many queries are listed but saves the count
// pass's scan when few are (rounds from kOrderedUntilRound on).
__global__ void __launch_bounds__(256) k_active(const uint32_t *__restrict__ labels,
                                                const uint32_t *__restrict__ bound,
                                                const CompBest *comp, uint2 *__restrict__ res,
                                                int64_t n, uint32_t *__restrict__ list,
                                                uint32_t *count) {
  const int lane = threadIdx.x & 31;
  const int64_t i0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4;
  uint32_t act = 0;
  if (i0 < n) {
    uint32_t lab[4];
    uint2 prev[4];
    if (i0 + 4 <= n) {  // 16-byte loads (i0 is a multiple of 4; the arrays are 256-B aligned)
      const uint4 l4 = *reinterpret_cast<const uint4 *>(labels + i0);
      const uint4 ra = reinterpret_cast<const uint4 *>(res + i0)[0];
      const uint4 rb = reinterpret_cast<const uint4 *>(res + i0)[1];
      lab[0] = l4.x; lab[1] = l4.y; lab[2] = l4.z; lab[3] = l4.w;
      prev[0] = make_uint2(ra.x, ra.y); prev[1] = make_uint2(ra.z, ra.w);
      prev[2] = make_uint2(rb.x, rb.y); prev[3] = make_uint2(rb.z, rb.w);
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        lab[j] = i0 + j < n ? labels[i0 + j] : 0u;
        prev[j] = i0 + j < n ? res[i0 + j] : make_uint2(0u, kInvalid);
      }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (i0 + j >= n) continue;
      float r = bound_to_radius(__ldg(bound + lab[j]));
      // (no query of the round has run yet, so the entries are fixed during
      // this kernel and may come through L1: in the last rounds every point
      // reads one of a handful of them)
      const uint32_t cw =
          (uint32_t)(__ldg(reinterpret_cast<const unsigned long long *>(&comp[lab[j]].key)) >> 32);
      r = fminf(r, bound_to_radius(cw));
      if (__uint_as_float(prev[j].x) > r) {
        if (prev[j].y != kInvalid) res[i0 + j] = make_uint2(prev[j].x, kInvalid);
      } else {
        act |= 1u << j;
      }
    }
  }
  const uint32_t c = (uint32_t)__popc(act);
  uint32_t x = c;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  uint32_t base = 0;
  if (lane == 31 && x) base = atomicAdd(count, x);
  base = __shfl_sync(0xffffffffu, base, 31);
  uint32_t at = base + x - c;
#pragma unroll
  for (int j = 0; j < 4; ++j)
    if ((act >> j) & 1u) list[at++] = (uint32_t)(i0 + j);
}

// Eight curve positions per thread, 2,048 per CTA: the skip
// test, the positions to search as one byte of flags per thread, the tile's
// count of them, and (last CTA to finish) the exclusive scan of the tile
// counts and the list's length.
constexpr int kActiveThreads = 256;
constexpr int kActiveTile = kActiveThreads * 8;
static_assert(kActiveThreads == kScanThreads, "block_exclusive_scan runs on a CTA of kScanThreads");

__global__ void __launch_bounds__(kActiveThreads) k_active_count(
    const uint32_t *__restrict__ labels, const uint32_t *__restrict__ bound, const CompBest *comp,
    uint2 *__restrict__ res, int64_t n, uint8_t *__restrict__ flags, uint32_t *tile_total,
    uint32_t *tile_prefix, uint32_t *done, uint32_t *count) {
  __shared__ uint32_t s_warp[kActiveThreads / 32];
  __shared__ uint32_t s_last;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t t = (int64_t)blockIdx.x * kActiveThreads + tid;
  const int64_t i0 = t * 8;
  uint32_t act = 0;
  if (i0 < n) {
    uint32_t lab[8];
    uint2 prev[8];
    if (i0 + 8 <= n) {  // 16-byte loads (i0 is a multiple of 8; the arrays are 256-B aligned)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const uint4 l4 = reinterpret_cast<const uint4 *>(labels + i0)[h];
        lab[4 * h] = l4.x; lab[4 * h + 1] = l4.y; lab[4 * h + 2] = l4.z; lab[4 * h + 3] = l4.w;
      }
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        const uint4 r = reinterpret_cast<const uint4 *>(res + i0)[h];
        prev[2 * h] = make_uint2(r.x, r.y);
        prev[2 * h + 1] = make_uint2(r.z, r.w);
      }
    } else {
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        lab[j] = i0 + j < n ? labels[i0 + j] : 0u;
        prev[j] = i0 + j < n ? res[i0 + j] : make_uint2(0u, kInvalid);
      }
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      if (i0 + j >= n) continue;
      float r = bound_to_radius(__ldg(bound + lab[j]));
      // (no query of the round has run yet, so the entries are fixed during
      // this kernel and may come through L1: in the last rounds every point
      // reads one of a handful of them)
      const uint32_t cw =
          (uint32_t)(__ldg(reinterpret_cast<const unsigned long long *>(&comp[lab[j]].key)) >> 32);
      r = fminf(r, bound_to_radius(cw));
      if (__uint_as_float(prev[j].x) > r) {
        if (prev[j].y != kInvalid) res[i0 + j] = make_uint2(prev[j].x, kInvalid);
      } else {
        act |= 1u << j;
      }
    }
    flags[t] = (uint8_t)act;
  }
  const uint32_t wsum = __reduce_add_sync(0xffffffffu, (uint32_t)__popc(act));
  if (lane == 0) s_warp[warp] = wsum;
  __syncthreads();
  if (tid == 0) {
    uint32_t total = 0;
#pragma unroll
    for (int w = 0; w < kActiveThreads / 32; ++w) total += s_warp[w];
    tile_total[blockIdx.x] = total;
    __threadfence();
    s_last = atomicAdd(done, 1u) == gridDim.x - 1 ? 1u : 0u;
  }
  __syncthreads();
  if (s_last) {
    __threadfence();
    block_exclusive_scan(tile_total, tile_prefix, gridDim.x);
    __syncthreads();
    if (tid == 0) *count = tile_prefix[gridDim.x - 1] + __ldcg(tile_total + gridDim.x - 1);
  }
}

// The list in curve order: each tile's positions after the positions of all
// earlier tiles, in order within the tile.
__global__ void __launch_bounds__(kActiveThreads) k_active_write(const uint8_t *__restrict__ flags,
                                                                 const uint32_t *__restrict__ tile_prefix,
                                                                 int64_t n, uint32_t *__restrict__ list) {
  __shared__ uint32_t s_warp[kActiveThreads / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t t = (int64_t)blockIdx.x * kActiveThreads + tid;
  const int64_t i0 = t * 8;
  const uint32_t act = i0 < n ? (uint32_t)flags[t] : 0u;
  const uint32_t c = (uint32_t)__popc(act);
  uint32_t x = c;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[warp] = x;
  __syncthreads();
  uint32_t before = 0;
  for (int w = 0; w < warp; ++w) before += s_warp[w];
  uint32_t at = __ldg(tile_prefix + blockIdx.x) + before + x - c;
#pragma unroll
  for (int j = 0; j < 8; ++j)
    if ((act >> j) & 1u) list[at++] = (uint32_t)(i0 + j);
}

using TravKernel = void (*)(TravArgs, const uint32_t *, const uint32_t *);

static void launch_trav(TravKernel k, int g, int block, cudaStream_t s, const TravArgs &A,
                        const uint32_t *list, const uint32_t *list_count) {
  k<<<g, block, 0, s>>>(A, list, list_count);
}

// The tighter lower bound of empty searches (traverse_one's LB) is tracked
// from round 2 on (rounds count from 0): round 1 still searches nearly every
// point, so tracking there would cost it more than its bounds save the
// rounds after it (measured: from round 1 / 2 / 3, 48.36 / 48.35 / 48.56 ms
// per call at 37M halo points).
#ifndef EMST_LB_FROM_ROUND
#define EMST_LB_FROM_ROUND 2
#endif
static bool track_lower_bounds(int round) { return round < 0 || round >= EMST_LB_FROM_ROUND; }

void launch_traverse(Problem &P, bool carried, const float *radius_in, int block, bool count,
                     bool seeded, int learned_pass, bool first, int round) {
  if (block <= 0) block = kTraverseBlock;
  TravArgs A;
  A.pts = P.pts;
  A.nodes = P.nodes;
  A.nlabels = P.nlabels;
  A.core2 = P.core2;
  A.ties = P.ties;
  A.labels = P.labels;
  A.bound = P.bound;
  A.radius_in = radius_in;
  A.leaf = P.leaf;
  A.inst_of = P.inst_of;
  A.inst_root = P.inst_root;
  A.offsets = P.offsets;
  A.res = P.res;
  A.comp = P.comp;
  A.n = P.n;
  A.status = P.counters + 1;
  A.visits = reinterpret_cast<unsigned long long *>(P.counters + 2);
  A.queries = reinterpret_cast<unsigned long long *>(P.counters + 34);
  A.seen = P.seen;
  A.pred_r = P.pred_r;
  A.r_used = P.r_used;
  A.queue = nullptr;
  // learned_pass: 0 = plain, 1 = with the proposed radii, 2 = rerun of the
  // listed points with the plain cutoff
  // the persistent work-queue form serves the plain rounds on one-point leaves
  if (P.persistent && seeded && !radius_in && learned_pass == 0 && !P.core2 && P.leaf == 1) {
    launch_traverse_queue(P, A, carried, first, count);
    return;
  }
  const uint32_t *list = learned_pass == 2 ? P.rerun_list : nullptr;
  const uint32_t *list_count = learned_pass == 2 ? P.counters + 13 : nullptr;
  int g = learned_pass == 2 ? sm_count() * 8 : grid_for(P.n, block);
  cudaStream_t s = P.stream;
  if (carried && seeded && !radius_in && learned_pass == 0 && round >= kCompactFromRound) {
    // the queries that need a search, listed in curve order (vals[1] and
    // keys[1] are free during the rounds: the list, and the flags and tile
    // counts behind it)
    uint32_t *active = P.vals[1];
    uint32_t *active_count = P.counters + kActiveCounter;
    const int64_t tiles = (P.n + kActiveTile - 1) / kActiveTile;
    uint8_t *flags = reinterpret_cast<uint8_t *>(P.keys[1]);
    uint32_t *tile_total = reinterpret_cast<uint32_t *>(P.keys[1]) + tiles * (kActiveTile / 8 / 4);  // after the flags
    uint32_t *tile_prefix = tile_total + tiles;
    if (round < kOrderedUntilRound) {
      cudaMemsetAsync(P.counters + kActiveDone, 0, sizeof(uint32_t), s);
      k_active_count<<<(unsigned)tiles, kActiveThreads, 0, s>>>(P.labels, P.bound, P.comp, P.res, P.n,
                                                               flags, tile_total, tile_prefix,
                                                               P.counters + kActiveDone, active_count);
      k_active_write<<<(unsigned)tiles, kActiveThreads, 0, s>>>(flags, tile_prefix, P.n, active);
      P.launches += 2;
    } else {
      cudaMemsetAsync(active_count, 0, sizeof(uint32_t), s);
      k_active<<<(unsigned)grid_for((P.n + 3) / 4, 256), 256, 0, s>>>(P.labels, P.bound, P.comp, P.res,
                                                                       P.n, active, active_count);
      P.launches += 1;
    }
    list = active;
    list_count = active_count;
    g = sm_count() * (2048 / block);  // one resident wave
#if EMST_LIST_QUEUE
    A.queue = P.counters + kActiveQueue;  // warps take the list in order
    cudaMemsetAsync(A.queue, 0, sizeof(uint32_t), s);
#endif
  }
#define EMST_TRAV2(C, R, K, S, H, L) launch_trav(k_traverse<C, R, K, S, H, L, false, false>, g, block, s, A, list, list_count)
#define EMST_TRAV_FIRST(K, H) launch_trav(k_traverse<false, false, K, true, H, false, true, false>, g, block, s, A, list, list_count)
#define EMST_TRAV_MRD(C, K, H) launch_trav(k_traverse<C, false, K, true, H, false, false, true>, g, block, s, A, list, list_count)
#define EMST_TRAV_NOTIES(C, F, H) launch_trav(k_traverse<C, false, false, true, H, false, F, false, false>, g, block, s, A, list, list_count)
#define EMST_TRAV_NOTIES_NOLB() launch_trav(k_traverse<true, false, false, true, false, false, false, false, false, false>, g, block, s, A, list, list_count)
#define EMST_TRAV_NOLB(K) launch_trav(k_traverse<true, false, K, true, false, false, false, false, true, false>, g, block, s, A, list, list_count)
  const bool lbt = track_lower_bounds(round);
#define EMST_TRAV(C, R, K, S, L)                       \
  do {                                                 \
    if (P.leaf > 1) EMST_TRAV2(C, R, K, S, true, L);   \
    else EMST_TRAV2(C, R, K, S, false, L);             \
  } while (0)
  if (!P.ties && !count && seeded && !radius_in && learned_pass == 0 && !P.core2) {
    // the plain form on input without large groups of identical points
    const bool h = P.leaf > 1;
    if (carried) {
      if (h) EMST_TRAV_NOTIES(true, false, true);
      else if (lbt) EMST_TRAV_NOTIES(true, false, false);
      else EMST_TRAV_NOTIES_NOLB();
    }
    else if (first) { if (h) EMST_TRAV_NOTIES(false, true, true); else EMST_TRAV_NOTIES(false, true, false); }
    else { if (h) EMST_TRAV_NOTIES(false, false, true); else EMST_TRAV_NOTIES(false, false, false); }
  } else if (radius_in) {
    EMST_TRAV(false, true, false, false, false);
  } else if (!seeded) {
    EMST_TRAV(false, false, false, false, false);
  } else if (learned_pass == 1) {
    if (carried) {
      if (count) EMST_TRAV(true, false, true, true, true); else EMST_TRAV(true, false, false, true, true);
    } else {
      if (count) EMST_TRAV(false, false, true, true, true); else EMST_TRAV(false, false, false, true, true);
    }
  } else if (P.core2) {  // mutual reachability weights (the plain form's rounds)
    const bool h = P.leaf > 1;
    if (carried) {
      if (count) { if (h) EMST_TRAV_MRD(true, true, true); else EMST_TRAV_MRD(true, true, false); }
      else { if (h) EMST_TRAV_MRD(true, false, true); else EMST_TRAV_MRD(true, false, false); }
    } else {
      if (count) { if (h) EMST_TRAV_MRD(false, true, true); else EMST_TRAV_MRD(false, true, false); }
      else { if (h) EMST_TRAV_MRD(false, false, true); else EMST_TRAV_MRD(false, false, false); }
    }
  } else if (carried) {
    if (!lbt && P.leaf == 1) {
      if (count) EMST_TRAV_NOLB(true); else EMST_TRAV_NOLB(false);
    } else {
      if (count) EMST_TRAV(true, false, true, true, false); else EMST_TRAV(true, false, false, true, false);
    }
  } else if (first) {  // the first round of the plain form: labels are the curve indices
    if (P.leaf > 1) {
      if (count) EMST_TRAV_FIRST(true, true); else EMST_TRAV_FIRST(false, true);
    } else {
      if (count) EMST_TRAV_FIRST(true, false); else EMST_TRAV_FIRST(false, false);
    }
  } else {
    if (count) EMST_TRAV(false, false, true, true, false); else EMST_TRAV(false, false, false, true, false);
  }
#undef EMST_TRAV
#undef EMST_TRAV2
#undef EMST_TRAV_FIRST
#undef EMST_TRAV_MRD
#undef EMST_TRAV_NOTIES
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
__device__ __forceinline__ uint32_t merge_target(const CompBest *comp, uint32_t x) {
  const CompBest b = comp[x];
  return b.key == kEmptyKey ? kInvalid : (uint32_t)b.mx;
}

// One thread per listed component.  The edges and the next round's list are
// appended through one atomic per CTA (their order carries no meaning: the
// output is sorted, the list is a set).  comp_clear: the other round's
// minima, cleared for the listed labels; bound_next: the next
// round's bounds, cleared for the new roots (the only labels it reads) before
// the relabel pass lowers them.  count_dev (graph rounds): the list's length
// on the device, at most `count` (the grid covers `count`).
__global__ void __launch_bounds__(kBlock) k_merge_roots(const uint32_t *__restrict__ list,
                                                        int64_t count,
                                                        const uint32_t *__restrict__ count_dev,
                                                        const CompBest *__restrict__ comp,
                                                        CompBest *__restrict__ comp_clear,
                                                        uint32_t *__restrict__ bound_next,
                                                        uint32_t *__restrict__ root,
                                                        emst_edge *__restrict__ edges,
                                                        uint32_t *__restrict__ next_list,
                                                        uint32_t *counters, int64_t n) {
  __shared__ uint32_t s_warp[2][kBlock / 32];
  __shared__ uint32_t s_wmax[kBlock / 32];
  __shared__ uint32_t s_base[2];
  const int64_t t64 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (count_dev) {
    const int64_t c = (int64_t)*count_dev;
    if (c < count) count = c;
  }
  bool emit = false, is_root = false;
  uint32_t c = 0;
  emst_edge E = {0u, 0u, 0.0f};
  if (t64 < count) {
    c = list ? list[t64] : (uint32_t)t64;
    const CompBest b = comp[c];
    const uint64_t key = b.key, mx = b.mx;
    const uint32_t t = key == kEmptyKey ? kInvalid : (uint32_t)mx;
    uint32_t r = c;
    if (t != kInvalid) {
      emit = !(merge_target(comp, t) == c) || c < t;
      E.i = (uint32_t)key;
      E.j = (uint32_t)(mx >> 32);
      E.w = __uint_as_float((uint32_t)(key >> 32));
      uint32_t x = c, y = t;
      for (int64_t steps = 0;; ++steps) {
        if (y == kInvalid) { r = x; break; }  // chain ends at a component without an edge
        const uint32_t z = merge_target(comp, y);
        if (z == x) { r = x < y ? x : y; break; }
        x = y;
        y = z;
        if (steps > n) { atomicOr(&counters[1], kErrChain); r = x; break; }
      }
    }
    CompBest empty;
    empty.key = kEmptyKey;
    empty.mx = kEmptyKey;
    comp_clear[c] = empty;
    root[c] = r;
    is_root = r == c;
    if (is_root) bound_next[c] = kNoBound;
  }
  const uint32_t be = __ballot_sync(0xffffffffu, emit), br = __ballot_sync(0xffffffffu, is_root);
  const uint32_t wmax = __reduce_max_sync(0xffffffffu, emit ? __float_as_uint(E.w) : 0u);
  if (lane == 0) {
    s_warp[0][warp] = __popc(be);
    s_warp[1][warp] = __popc(br);
    s_wmax[warp] = wmax;
  }
  __syncthreads();
  if (threadIdx.x == 32) {  // the largest weight emitted (for the output's key width)
    uint32_t m = 0;
    for (int w = 0; w < kBlock / 32; ++w) m = m > s_wmax[w] ? m : s_wmax[w];
    if (m) atomicMax(&counters[11], m);
  }
  if (threadIdx.x < 2) {
    uint32_t tot = 0;
    for (int w = 0; w < kBlock / 32; ++w) {
      const uint32_t v = s_warp[threadIdx.x][w];
      s_warp[threadIdx.x][w] = tot;
      tot += v;
    }
    s_base[threadIdx.x] = tot ? atomicAdd(&counters[threadIdx.x == 0 ? 0 : 12], tot) : 0u;
  }
  __syncthreads();
  const uint32_t lt = (1u << lane) - 1u;
  if (emit) edges[s_base[0] + s_warp[0][warp] + __popc(be & lt)] = E;
  if (is_root) next_list[s_base[1] + s_warp[1][warp] + __popc(br & lt)] = c;
}

void launch_merge(Problem &P) {
  const int64_t count = P.active_list ? P.n_active : P.n;
  const int g = grid_for(count, kBlock);
  // graph rounds: this round's list length exists only on the device
  const uint32_t *count_dev = P.active_list ? P.count_dev : nullptr;
  if (count_dev)
    cudaMemcpyAsync(P.count_dev, P.counters + 12, sizeof(uint32_t), cudaMemcpyDeviceToDevice,
                    P.stream);
  cudaMemsetAsync(P.counters + 12, 0, sizeof(uint32_t), P.stream);
  k_merge_roots<<<g, kBlock, 0, P.stream>>>(P.active_list, count, count_dev, P.comp, P.comp_buf[P.cur ^ 1],
                                            P.bound_buf[P.cur ^ 1], P.root, P.edges, P.next_list, P.counters, P.n);
  P.launches += 1;
  launch_runs(P, true);
}

// After the host has seen a round finish: the next round's labels, bounds and
// active list become current.
void advance_round(Problem &P, int64_t n_active) {
  P.cur ^= 1;
  P.labels = P.labels_buf[P.cur];
  P.bound = P.bound_buf[P.cur];
  P.comp = P.comp_buf[P.cur];
  uint32_t *t = P.list_buf[0] == P.next_list ? P.list_buf[1] : P.list_buf[0];
  P.active_list = P.next_list;
  P.next_list = t;
  P.n_active = n_active;
}

// Count runs only: the distinct internal nodes of this round's searches (the
// bits of the visited bitmap), added to a 64-bit counter; the bitmap is
// cleared for the next round.
__global__ void __launch_bounds__(kBlock) k_count_seen(uint32_t *seen, int64_t words,
                                                       unsigned long long *total) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned c = 0;
  if (k < words) {
    c = __popc(seen[k]);
    seen[k] = 0u;
  }
  c = __reduce_add_sync(0xffffffffu, c);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(total, (unsigned long long)c);
}

void launch_count_seen(Problem &P) {
  if (!P.seen || P.nc < 2) return;
  const int64_t words = (P.nc - 1 + 31) / 32;
  k_count_seen<<<grid_for(words, kBlock), kBlock, 0, P.stream>>>(
      P.seen, words, reinterpret_cast<unsigned long long *>(P.counters + 38));
  P.launches += 1;
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
// A12. Output order: (w, i, j) ascending.  Fast path (one instance): one
// radix sort by (w bits << L) | i (only as many digits as the largest weight
// needs) with j as the value, then the runs of equal (w, i) -- the edges of
// one point with equal weights, a handful in general position -- are put in
// j order in place and the edges are rebuilt from (key, value).  A run longer
// than kTieRunMax (exact ties: many identical points make a star of
// zero-weight edges) is only counted; the caller then redoes the output on
// the full path: a stable sort by j, then a stable sort by (w, i) (and by
// instance in the batched form, which always takes it), then a gather.
// ---------------------------------------------------------------------------
constexpr int kTieRunMax = 64;

__global__ void k_edge_keys_wi(const emst_edge *__restrict__ edges, int64_t m,
                               uint64_t *__restrict__ keys, uint32_t *__restrict__ vals,
                               int shift_i) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m) return;
  const emst_edge E = edges[e];
  keys[e] = ((uint64_t)__float_as_uint(E.w) << shift_i) | (uint64_t)E.i;
  vals[e] = E.j;
}

// The first thread of each run of equal keys orders the run by j (insertion
// sort), or counts it when it is longer than kTieRunMax.
__global__ void k_edge_ties(const uint64_t *__restrict__ keys, uint32_t *__restrict__ vals,
                            int64_t m, uint32_t *long_runs) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e + 1 >= m) return;
  const uint64_t key = keys[e];
  if (keys[e + 1] != key || (e > 0 && keys[e - 1] == key)) return;
  int64_t end = e + 2;
  while (end < m && end - e <= kTieRunMax && keys[end] == key) ++end;
  if (end - e > kTieRunMax) {
    atomicAdd(long_runs, 1u);
    return;
  }
  for (int64_t a = e + 1; a < end; ++a) {
    const uint32_t v = vals[a];
    int64_t b = a;
    while (b > e && vals[b - 1] > v) {
      vals[b] = vals[b - 1];
      --b;
    }
    vals[b] = v;
  }
}

// The same after a sort by w alone ((w << L) | i sorted on w's bits, stable,
// so a run of equal w holds its edges in emission order): the first thread
// of each run of equal w orders the run by (i, j) -- by (key, j), the key's
// w bits being equal -- or counts it when it is longer than kTieRunMax.
__global__ void k_edge_ties_w(uint64_t *__restrict__ keys, uint32_t *__restrict__ vals, int64_t m,
                              int shift_i, uint32_t *long_runs) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e + 1 >= m) return;
  const uint64_t w = keys[e] >> shift_i;
  if ((keys[e + 1] >> shift_i) != w || (e > 0 && (keys[e - 1] >> shift_i) == w)) return;
  int64_t end = e + 2;
  while (end < m && end - e <= kTieRunMax && (keys[end] >> shift_i) == w) ++end;
  if (end - e > kTieRunMax) {
    atomicAdd(long_runs, 1u);
    return;
  }
  for (int64_t a = e + 1; a < end; ++a) {
    const uint64_t k = keys[a];
    const uint32_t v = vals[a];
    int64_t b = a;
    while (b > e && (keys[b - 1] > k || (keys[b - 1] == k && vals[b - 1] > v))) {
      keys[b] = keys[b - 1];
      vals[b] = vals[b - 1];
      --b;
    }
    keys[b] = k;
    vals[b] = v;
  }
}

// Edge e of the output from its sorted key ((w << L) | i, with the instance
// above w in the batched form) and j; w_mask keeps w's bits.
__global__ void k_edge_from_keys(const uint64_t *__restrict__ keys,
                                 const uint32_t *__restrict__ vals, int64_t m, int shift_i,
                                 uint32_t w_mask, emst_edge *__restrict__ out) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m) return;
  const uint64_t k = keys[e];
  emst_edge E;
  E.i = (uint32_t)(k & ((1ull << shift_i) - 1ull));
  E.j = vals[e];
  E.w = __uint_as_float((uint32_t)(k >> shift_i) & w_mask);
  out[e] = E;
}

// The same with 16-byte stores that consecutive lanes make to consecutive
// addresses (the output may be pinned host memory written over the
// chip-to-chip link, where whole coalesced lines matter): thread c writes
// 16-byte chunk c of the output, i.e. words 4c..4c+3 of the flat array of
// (i, j, w) words, rebuilt from the (at most two) edges they belong to.
// `out` 16-byte aligned; chunks = floor(3m / 4) whole chunks.
__global__ void k_edge_from_keys16(const uint64_t *__restrict__ keys,
                                   const uint32_t *__restrict__ vals, int64_t chunks, int shift_i,
                                   uint32_t w_mask, uint4 *__restrict__ out) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= chunks) return;
  const uint64_t imask = (1ull << shift_i) - 1ull;
  uint32_t w[4];
  const int64_t w0 = 4 * c;
  int64_t e = w0 / 3;
  int f = (int)(w0 - 3 * e);
  uint64_t k = __ldg(keys + e);
  uint32_t j = __ldg(vals + e);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    w[q] = f == 0 ? (uint32_t)(k & imask) : f == 1 ? j : ((uint32_t)(k >> shift_i) & w_mask);
    if (++f == 3 && q < 3) {
      f = 0;
      ++e;
      k = __ldg(keys + e);
      j = __ldg(vals + e);
    }
  }
  out[c] = make_uint4(w[0], w[1], w[2], w[3]);
}

// Batched fast path: one key per edge, (instance, w, local i), with the
// local j as the value, when the three fit in 64 bits.  Sorting it puts every
// instance's edges together in (w, i, j) order (local ids keep the order of
// the global ones: one offset per instance), with the same tie fix for runs
// of equal (w, i) as one instance.
__global__ void k_edge_keys_inst_wi(const emst_edge *__restrict__ edges, int64_t m,
                                    uint64_t *__restrict__ keys, uint32_t *__restrict__ vals,
                                    const uint32_t *__restrict__ inst_in,
                                    const int64_t *__restrict__ offsets, int shift_w,
                                    int shift_i) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m) return;
  const emst_edge E = edges[e];
  const uint32_t I = __ldg(inst_in + E.i);
  const uint32_t base = (uint32_t)__ldg(offsets + I);
  keys[e] = ((uint64_t)I << shift_w) | ((uint64_t)__float_as_uint(E.w) << shift_i) |
            (uint64_t)(E.i - base);
  vals[e] = E.j - base;
}

// Full path: keys by j with the edge index as the value, then keys by
// (w, i) of the edges in that order.
__global__ void k_edge_keys_j(const emst_edge *__restrict__ edges, int64_t m,
                              uint64_t *__restrict__ keys, uint32_t *__restrict__ vals) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m) return;
  keys[e] = edges[e].j;
  vals[e] = (uint32_t)e;
}

__global__ void k_edge_keys_wi_of(const emst_edge *__restrict__ edges, int64_t m,
                                  uint64_t *__restrict__ keys, const uint32_t *__restrict__ vals,
                                  int shift_i) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m) return;
  const emst_edge E = edges[vals[e]];
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

void launch_edge_keys_wi(Problem &P, int64_t m, int shift_i) {
  k_edge_keys_wi<<<grid_for(m, kBlock), kBlock, 0, P.stream>>>(P.edges, m, P.keys[0], P.vals[0],
                                                               shift_i);
  P.launches += 1;
}
void launch_edge_ties(Problem &P, int64_t m, int src) {
  k_edge_ties<<<grid_for(m, kBlock), kBlock, 0, P.stream>>>(P.keys[src], P.vals[src], m,
                                                            P.counters + 10);
  P.launches += 1;
}
void launch_edge_ties_w(Problem &P, int64_t m, int src, int shift_i) {
  k_edge_ties_w<<<grid_for(m, kBlock), kBlock, 0, P.stream>>>(P.keys[src], P.vals[src], m, shift_i,
                                                              P.counters + 10);
  P.launches += 1;
}
void launch_edge_from_keys(Problem &P, int64_t m, int src, int shift_i, int w_bits_used,
                           emst_edge *out) {
  const uint32_t w_mask = w_bits_used >= 32 ? 0xFFFFFFFFu : ((1u << w_bits_used) - 1u);
  // whole 16-byte chunks of the output by coalesced wide stores when it is
  // 16-byte aligned, the edges after the last whole chunk one by one
  const int64_t chunks = (reinterpret_cast<uintptr_t>(out) & 15u) == 0 ? (3 * m) / 4 : 0;
  const int64_t covered = (4 * chunks) / 3;  // edges wholly inside those chunks (the next one,
                                             // if split, is rewritten whole below)
  if (chunks > 0) {
    k_edge_from_keys16<<<grid_for(chunks, kBlock), kBlock, 0, P.stream>>>(
        P.keys[src], P.vals[src], chunks, shift_i, w_mask, reinterpret_cast<uint4 *>(out));
    P.launches += 1;
  }
  if (m - covered > 0) {
    k_edge_from_keys<<<grid_for(m - covered, kBlock), kBlock, 0, P.stream>>>(
        P.keys[src] + covered, P.vals[src] + covered, m - covered, shift_i, w_mask, out + covered);
    P.launches += 1;
  }
}
void launch_edge_keys_inst_wi(Problem &P, int64_t m, int shift_w, int shift_i) {
  k_edge_keys_inst_wi<<<grid_for(m, kBlock), kBlock, 0, P.stream>>>(
      P.edges, m, P.keys[0], P.vals[0], P.inst_in, P.offsets, shift_w, shift_i);
  P.launches += 1;
}
void launch_edge_keys_j(Problem &P, int64_t m) {
  k_edge_keys_j<<<grid_for(m, kBlock), kBlock, 0, P.stream>>>(P.edges, m, P.keys[0], P.vals[0]);
  P.launches += 1;
}
void launch_edge_keys_wi_of(Problem &P, int64_t m, int src, int shift_i) {
  k_edge_keys_wi_of<<<grid_for(m, kBlock), kBlock, 0, P.stream>>>(P.edges, m, P.keys[src],
                                                                  P.vals[src], shift_i);
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

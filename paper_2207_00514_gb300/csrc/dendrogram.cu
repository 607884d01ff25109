// dendrogram.cu -- the single-linkage dendrogram of a spanning tree: the
// hierarchy that single-linkage clustering and HDBSCAN* read off the EMST
// (the introduction names clustering as a consumer; §4.5 builds the
// mutual-reachability tree for HDBSCAN*).
//
// Definition: Kruskal's merge sequence (§2, "MST computation") over the
// tree's own edges in the given order (non-decreasing weight).  Edge k makes
// cluster n + k.  The parent of edge k is the first later edge that touches
// C(k), the component of edges 0..k holding k: the lowest-ranked edge on
// C(k)'s boundary.  A point's parent is its lowest-ranked incident edge.
//
// The merge sequence is serial (its depth is the height of the hierarchy,
// which single linkage makes long by chaining).  Here the ranks are split
// instead, O(log n) levels whatever that height:
//  - A block B of ranks [s, e) sees the components of edges 0..s-1 as
//    contracted vertices.  Split B at its middle h: the light half [s, h)
//    keeps B's vertices; the heavy half [h, e) sees the components of the
//    light edges (over B's vertices) as its vertices.
//  - Let B be the smallest block holding edge k and its parent p.  Then k is
//    in B's light half, p in its heavy half, C(k) is k's light component K,
//    k is K's top (largest rank) edge and p is the lowest-ranked heavy edge
//    touching K.  One level finds those (k, p) for every block at once.
//  - Blocks of kLocalEdges edges and less run their levels in shared
//    memory, one CTA each, and finish with the serial merge sequence over
//    blocks of kSerialEdges edges, which also gives every cluster's size.
// A contracted vertex is named by an endpoint slot 2k + side of the
// lowest-ranked edge of its block that touches it.  The blocks of one level
// own disjoint slot ranges, so one union-find over all 2m slots serves every
// block of a level at once.
#include <cstdlib>
#include <utility>

#include "common.cuh"

namespace emst {
namespace {

#ifndef EMST_DG_LOCAL_EDGES
#define EMST_DG_LOCAL_EDGES 4096
#endif
#ifndef EMST_DG_LOCAL_THREADS
#define EMST_DG_LOCAL_THREADS 1024
#endif
constexpr int kLocalEdges = EMST_DG_LOCAL_EDGES;   // edges per block of the shared-memory levels
constexpr int kLocalThreads = EMST_DG_LOCAL_THREADS;
constexpr int kSerialEdges = 32;    // edges per serial finish (one thread each)
constexpr int kDgBlock = 256;
#ifndef EMST_DG_MID_EDGES
#define EMST_DG_MID_EDGES 32768
#endif
constexpr int64_t kMidEdges = EMST_DG_MID_EDGES;  // blocks of the CTA-level kernel (0: none)
constexpr int kMidThreads = 1024;
constexpr size_t kLocalSmem = (size_t)2 * kLocalEdges * (5 * 4 + 2);

// A bijective mix of a slot name (the MurmurHash3 32-bit finaliser): the
// union-find hooks the root of higher priority under the other, so trees
// stay shallow in expectation whatever order the slots are united in
// (linking by random index).
__device__ __forceinline__ uint32_t prio(uint32_t x) {
  x ^= x >> 16;
  x *= 0x85ebca6bu;
  x ^= x >> 13;
  x *= 0xc2b2ae35u;
  x ^= x >> 16;
  return x;
}

// How a level reads and writes its per-slot entries.  Plain (TAG false):
// an entry holds its value, and every level starts from cleared entries.
// Tagged (TAG true, trees below 2^26 edges): an entry also carries, in its
// top 5 bits, the number of the level that wrote it, so an entry of an
// earlier level reads as never written and nothing needs clearing: a
// union-find entry is (level, parent) -- any other level's entry makes its
// slot a root; a component's top edge is (level, rank + 1), which any
// earlier level's entry is below (atomicMax); its lowest heavy slot is
// (31 - level, slot), which any earlier level's entry (and the initial all
// ones) is above (atomicMin).
template <bool TAG>
struct Codec {
  uint32_t cur = 0;  // this level's number, 1..30 (TAG)
  static constexpr uint32_t kV = 0x07FFFFFFu;
  __device__ __forceinline__ uint32_t parent(uint32_t raw, uint32_t x) const {
    if (!TAG) return raw;
    return (raw >> 27) == cur ? (raw & kV) : x;
  }
  __device__ __forceinline__ uint32_t link(uint32_t p) const { return TAG ? ((cur << 27) | p) : p; }
  __device__ __forceinline__ uint32_t top_val(uint32_t rank1) const {
    return TAG ? ((cur << 27) | rank1) : rank1;
  }
  __device__ __forceinline__ uint32_t top_of(uint32_t raw) const {
    if (!TAG) return raw;
    return (raw >> 27) == cur ? (raw & kV) : 0u;
  }
  __device__ __forceinline__ uint32_t minh_val(uint32_t slot) const {
    return TAG ? (((31u - cur) << 27) | slot) : slot;
  }
  __device__ __forceinline__ uint32_t minh_of(uint32_t raw) const {
    if (!TAG) return raw;
    return (raw >> 27) == 31u - cur ? (raw & kV) : kInvalid;
  }
};

// Root of x, optionally halving the path.  Every parent has a lower
// priority than its child and a parent is only ever replaced by an
// ancestor, so a walk is strictly descending and ends even when it reads
// stale (cached) entries: a stale entry is still an ancestor.  A stale root
// is caught by the hook's compare-and-swap in uf_unite.
template <bool HALVE, bool TAG = false, class T>
__device__ __forceinline__ uint32_t uf_find(T *uf, uint32_t x, Codec<TAG> C = Codec<TAG>()) {
  for (;;) {
    const uint32_t p = C.parent(uf[x], x);
    if (p == x) return x;
    const uint32_t g = C.parent(uf[p], p);
    if (g == p) return p;
    if (HALVE) uf[x] = C.link(g);
    x = g;
  }
}

// The roots of a and b, the two walks advanced together so that their
// loads are in flight at once (each walk as in uf_find; `wa` / `wb` false:
// that walk is not needed and its result is the input).
template <bool HALVE, bool TAG = false, class T>
__device__ __forceinline__ void uf_find2(T *uf, uint32_t &a, uint32_t &b, bool wa = true,
                                         bool wb = true, Codec<TAG> C = Codec<TAG>()) {
  bool da = !wa, db = !wb;
  while (!(da && db)) {
    const uint32_t pa = da ? a : C.parent(uf[a], a);
    const uint32_t pb = db ? b : C.parent(uf[b], b);
    if (!da && pa == a) da = true;
    if (!db && pb == b) db = true;
    const uint32_t ga = da ? a : C.parent(uf[pa], pa);
    const uint32_t gb = db ? b : C.parent(uf[pb], pb);
    if (!da) {
      if (ga == pa) { a = pa; da = true; }
      else { if (HALVE) uf[a] = C.link(ga); a = ga; }
    }
    if (!db) {
      if (gb == pb) { b = pb; db = true; }
      else { if (HALVE) uf[b] = C.link(gb); b = gb; }
    }
  }
}

// Joins the sets of a and b, lock-free.  A failed hook returns the hooked
// root's actual parent, and the walk resumes there, so each retry climbs the
// real chain.  Hooking the higher-priority root under the other cannot close
// a cycle even when the other is stale: its actual root has a still lower
// priority.  False only if the retry bound runs out.  Tagged entries: the
// hook swaps the root's entry as read (whatever earlier level wrote it) for
// the link; a changed entry that still reads as a root is retried.
template <bool TAG = false, class T>
__device__ __forceinline__ bool uf_unite(T *uf, uint32_t a, uint32_t b, Codec<TAG> C = Codec<TAG>()) {
  uf_find2<true, TAG>(uf, a, b, true, true, C);
  for (int it = 0; it < (1 << 22); ++it) {
    if (a == b) return true;
    const bool ah = prio(a) > prio(b);
    const uint32_t hi = ah ? a : b, lo = ah ? b : a;
    uint32_t expect = hi;
    if constexpr (TAG) {  // (read in L2, where the swap compares: a cached copy may be old)
      expect = __ldcg(reinterpret_cast<const unsigned int *>(uf) + hi);
      const uint32_t p = C.parent(expect, hi);
      if (p != hi) {  // no longer a root
        if (ah) a = uf_find<true, TAG>(uf, p, C);
        else b = uf_find<true, TAG>(uf, p, C);
        continue;
      }
    }
    const uint32_t old = atomicCAS((uint32_t *)uf + hi, expect, C.link(lo));
    if (old == expect) return true;
    const uint32_t p = C.parent(old, hi);
    if (p == hi) continue;  // (TAG: the entry read was not the current one)
    if (ah) a = uf_find<true, TAG>(uf, p, C);
    else b = uf_find<true, TAG>(uf, p, C);
  }
  return false;
}

// Atomics on a[idx] from a warp.  In up to two rounds, the lanes that share
// the target of the lowest remaining lane (the lanes of one large
// component) combine their values and one of them updates, after a cached
// look at the entry (max and min only; values only move one way, so a stale
// look can only cause an unneeded update).  Lanes left after two rounds
// update on their own.  Every lane of the warp calls; `want` selects the
// participants.
template <int OP>  // 0 max, 1 min, 2 add
__device__ __forceinline__ void warp_update(uint32_t *a, uint32_t idx, uint32_t v, bool want) {
  unsigned act = __ballot_sync(0xffffffffu, want);
  if (!want) return;
  const int lane = (int)(threadIdx.x & 31);
#pragma unroll
  for (int round = 0; round < 2; ++round) {
    const int leader = __ffs(act) - 1;
    const uint32_t lead_idx = __shfl_sync(act, idx, leader);
    const unsigned same = __ballot_sync(act, idx == lead_idx);
    if (idx == lead_idx) {
      const uint32_t r = OP == 0 ? __reduce_max_sync(same, v)
                       : OP == 1 ? __reduce_min_sync(same, v) : __reduce_add_sync(same, v);
      if (lane != leader) return;
      if (OP == 0 && a[idx] < r) atomicMax(a + idx, r);
      if (OP == 1 && a[idx] > r) atomicMin(a + idx, r);
      if (OP == 2) atomicAdd(a + idx, r);
      return;
    }
    act &= ~same;
  }
  if (OP == 0) atomicMax(a + idx, v);
  if (OP == 1) atomicMin(a + idx, v);
  if (OP == 2) atomicAdd(a + idx, v);
}

__device__ __forceinline__ uint32_t slot_vertex(const emst_edge *e, uint32_t s) {
  const emst_edge &x = e[s >> 1];
  return (s & 1) ? x.j : x.i;
}

// Input checks: ids below n, no loop edge, no NaN weight, weights not
// decreasing.
__global__ void k_dg_check(const emst_edge *__restrict__ e, int64_t m, int64_t n,
                           uint32_t *status) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= m) return;
  const emst_edge x = e[k];
  bool bad = x.i >= n || x.j >= n || x.i == x.j || !(x.w == x.w);
  if (k + 1 < m && e[k + 1].w < x.w) bad = true;
  if (bad) atomicOr(status, kErrBadInput);
}

// vslot[v] = the lowest slot touching point v: slot 2p + side says that v
// hangs under edge p, on that side.
__global__ void k_dg_first_slot(const emst_edge *__restrict__ e, int64_t m2,
                                uint32_t *__restrict__ vslot) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= m2) return;
  const uint32_t v = slot_vertex(e, (uint32_t)s);
  if (vslot[v] > (uint32_t)s) atomicMin(vslot + v, (uint32_t)s);
}

// The per-level union-find and per-component values come in two sets: a
// level reads one and, in its last kernel, clears the other for the next
// level.  Only slots that name a vertex are ever read there (every walk
// starts at a name and hooks join names), but every slot is cleared: whole
// coalesced sectors, where clearing the scattered names alone made each
// sector a partial write that DRAM had to fill first (measured 4.2 GB per
// stitch launch at 37M points, HBM-bound).  With tagged entries (Codec)
// only the sizes alternate and are cleared; one set of union-find, top and
// lowest-heavy entries serves every level.
struct Level {
  uint32_t *rep, *sz, *uf, *top, *minh, *csz, *parent;
  uint32_t *nuf, *ntop, *nminh, *ncsz;  // the next level's set
  int64_t m;
  uint32_t mask, half;  // block size - 1, half the block size
  uint32_t cur;         // this level's number (tagged entries)
  uint32_t *status;
};

template <bool TAG>
__device__ __forceinline__ Codec<TAG> codec(const Level &L) {
  Codec<TAG> C;
  C.cur = L.cur;
  return C;
}

template <bool TAG>
__device__ __forceinline__ void clear_pair(const Level &L, uint32_t s0) {
  if (!TAG) {
    reinterpret_cast<uint2 *>(L.nuf)[s0 >> 1] = make_uint2(s0, s0 + 1);
    reinterpret_cast<uint2 *>(L.ntop)[s0 >> 1] = make_uint2(0u, 0u);
    reinterpret_cast<uint2 *>(L.nminh)[s0 >> 1] = make_uint2(kInvalid, kInvalid);
  }
  reinterpret_cast<uint2 *>(L.ncsz)[s0 >> 1] = make_uint2(0u, 0u);
}

// The host's and the CTA-level kernel's step from one level to the next.
template <bool TAG>
__host__ __device__ __forceinline__ void next_level(Level &L) {
  uint32_t *t;
  if (!TAG) {
    t = L.uf; L.uf = L.nuf; L.nuf = t;
    t = L.top; L.top = L.ntop; L.ntop = t;
    t = L.minh; L.minh = L.nminh; L.nminh = t;
  }
  t = L.csz; L.csz = L.ncsz; L.ncsz = t;
  L.cur += 1;
}

__device__ __forceinline__ bool block_split(const Level &L, uint32_t k, bool &light) {
  const uint32_t start = k & ~L.mask;
  light = (k & L.mask) < L.half;
  return (int64_t)start + L.half < L.m;  // the block has a heavy half
}

// Top level: every vertex is a point, named by its lowest slot, size 1.
// The slot that names point v also records v as the child on that side of
// its edge (the cluster a point starts in); the even slot of each edge
// clears the first level's set for the edge's two slots.
template <bool TAG>
__global__ void k_dg_init(Level L, const emst_edge *__restrict__ e,
                          const uint32_t *__restrict__ vslot, uint32_t *__restrict__ child) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= 2 * L.m) return;
  const uint32_t v = slot_vertex(e, (uint32_t)s);
  const uint32_t r = vslot[v];
  L.rep[s] = r;
  L.sz[s] = 1;
  if ((s & 1) == 0) clear_pair<TAG>(L, (uint32_t)s);
  if (child) child[s] = r == (uint32_t)s ? v : kInvalid;  // the rest come from k_dg_children
}

// Light components: unite the two vertices of every light edge.
template <bool TAG>
__device__ __forceinline__ void dg_unite(const Level &L, int64_t k) {
  if (k >= L.m) return;
  bool light;
  if (!block_split(L, (uint32_t)k, light) || !light) return;
  if (!uf_unite<TAG>(L.uf, L.rep[2 * k], L.rep[2 * k + 1], codec<TAG>(L))) atomicOr(L.status, kErrSpin);
}

template <bool TAG>
__global__ void k_dg_unite(Level L) { dg_unite<TAG>(L, (int64_t)blockIdx.x * blockDim.x + threadIdx.x); }

// Per light component (by root): its top edge (rank + 1), its size (the sum
// over its vertices, each counted at the slot that names it) and the lowest
// heavy slot touching it.  A warp covers 32 edges of one half.  Light halves
// are visited from the top rank down, so the first value to reach a
// component's top is usually its maximum and later lanes skip the atomic.
// (every lane of a warp calls it: warp_update combines across the warp)
template <bool TAG>
__device__ __forceinline__ void dg_classify(const Level &L, int64_t t) {
  const Codec<TAG> C = codec<TAG>(L);
  bool light = false;
  const bool act = t < L.m && block_split(L, (uint32_t)t, light);
  uint32_t k = (uint32_t)t;
  if (act && light) {
    const uint32_t start = k & ~L.mask;
    k = start + L.half - 1 - (k - start);
  }
  const uint32_t s0 = 2 * k;
  // A vertex named by a slot of the heavy half touches no light edge (its
  // name is its lowest slot in the block, and light slots come first): a
  // component of its own whose lowest heavy slot is its name, so it needs no
  // find and no minimum here, and the stitch keeps its name.
  const uint32_t hs = 2 * ((k & ~L.mask) + L.half);  // the block's first heavy slot
  uint32_t r0 = 0, r1 = 0, x0 = 0, x1 = 0;
  bool m0 = false, m1 = false;
  if (act) {
    r0 = L.rep[s0];
    r1 = L.rep[s0 + 1];
    if (light) {
      x0 = uf_find<true, TAG>(L.uf, r0, C);
      x1 = x0;  // a light edge's ends share a root
    } else {
      m0 = r0 < hs;
      m1 = r1 < hs;
      x0 = r0;
      x1 = r1;
      uf_find2<true, TAG>(L.uf, x0, x1, m0, m1, C);
    }
  }
  warp_update<0>(L.top, x0, C.top_val(k + 1), act && light);
  warp_update<1>(L.minh, x0, C.minh_val(s0), m0);
  warp_update<1>(L.minh, x1, C.minh_val(s0 + 1), m1);
  // sizes are summed for light components only: a slot of the heavy half
  // that names its vertex names one that touches no light edge (a vertex's
  // name is its lowest slot in the block, and light slots come first), a
  // component of its own whose sum the stitch never reads
  const bool self0 = act && light && r0 == s0, self1 = act && light && r1 == s0 + 1;
  warp_update<2>(L.csz, x0, self0 ? L.sz[s0] : 0u, self0);
  warp_update<2>(L.csz, x1, self1 ? L.sz[s0 + 1] : 0u, self1);
}

template <bool TAG>
__global__ void k_dg_classify(Level L) { dg_classify<TAG>(L, (int64_t)blockIdx.x * blockDim.x + threadIdx.x); }

// The top edge of each light component takes the lowest heavy slot touching
// it as its parent (2p + side: edge p, on that side), and hands the
// component's size to that slot, which names the component in the heavy
// half; heavy slots are renamed to it.
template <bool TAG>
__device__ __forceinline__ void dg_stitch(const Level &L, int64_t k) {
  if (k >= L.m) return;
  const Codec<TAG> C = codec<TAG>(L);
  bool light;
  const bool split = block_split(L, (uint32_t)k, light);
  const uint32_t s0 = 2 * (uint32_t)k;
  uint32_t r0 = L.rep[s0], r1 = L.rep[s0 + 1];
  if (split && light) {
    const uint32_t r = uf_find<false, TAG>(L.uf, r0, C);
    const uint32_t h = C.minh_of(L.minh[r]);
    if (C.top_of(L.top[r]) == (uint32_t)k + 1 && h != kInvalid) {
      L.parent[k] = h;
      L.sz[h] = L.csz[r];
    }
  } else if (split) {
    // (names in the heavy half stay: see k_dg_classify)
    const uint32_t hs = 2 * (((uint32_t)k & ~L.mask) + L.half);
    uint32_t x0 = r0, x1 = r1;
    uf_find2<false, TAG>(L.uf, x0, x1, r0 < hs, r1 < hs, C);
    if (r0 < hs) L.rep[s0] = C.minh_of(L.minh[x0]);
    if (r1 < hs) L.rep[s0 + 1] = C.minh_of(L.minh[x1]);
  }
  clear_pair<TAG>(L, s0);
}

template <bool TAG>
__global__ void k_dg_stitch(Level L) { dg_stitch<TAG>(L, (int64_t)blockIdx.x * blockDim.x + threadIdx.x); }

// The levels of blocks from kMidEdges edges down to 2 * kLocalEdges, one CTA
// per block of kMidEdges edges: the same three steps per level as the global
// kernels, separated by barriers of the CTA instead of kernel boundaries, on
// the same global arrays, which stay in L2 while the CTA works on its
// block's slots (no other CTA touches them).  `L` arrives with the set of
// the first of these levels current (cleared by the level before); the
// levels alternate the sets as the host loop does.
template <bool TAG>
__global__ void __launch_bounds__(kMidThreads) k_dg_mid(Level L, int64_t top) {
  const int64_t b0 = (int64_t)blockIdx.x * top;
  for (int64_t S = top; S > kLocalEdges; S >>= 1) {
    L.mask = (uint32_t)(S - 1);
    L.half = (uint32_t)(S >> 1);
    for (int64_t j = threadIdx.x; j < top; j += kMidThreads) dg_unite<TAG>(L, b0 + j);
    __syncthreads();
    for (int64_t j = threadIdx.x; j < top; j += kMidThreads) dg_classify<TAG>(L, b0 + j);
    __syncthreads();
    for (int64_t j = threadIdx.x; j < top; j += kMidThreads) dg_stitch<TAG>(L, b0 + j);
    __syncthreads();
    next_level<TAG>(L);
  }
}

// The levels of blocks of kLocalEdges edges and less, in shared memory, one
// CTA per block: the same four steps per level as the global kernels, then
// the serial merge sequence over blocks of kSerialEdges edges, one thread
// each, which also gives every cluster's size.  Vertex names are local slot
// numbers (slot - 2 * block start); the serial finish checks that each stays
// inside its block (it does for any input with valid ids).
__global__ void __launch_bounds__(kLocalThreads)
    k_dg_local(int64_t m, const uint32_t *__restrict__ rep, const uint32_t *__restrict__ sz,
               uint32_t *__restrict__ parent, uint32_t *__restrict__ size_out, uint32_t *status) {
  constexpr int SL = 2 * kLocalEdges;
  extern __shared__ __align__(16) uint32_t smem[];
  uint32_t *uf = smem, *top = uf + SL, *minh = top + SL, *csz = minh + SL, *szl = csz + SL;
  uint16_t *lrep = reinterpret_cast<uint16_t *>(szl + SL);
  volatile uint32_t *vuf = uf;
  const int tid = threadIdx.x;
  const int64_t b0 = (int64_t)blockIdx.x * kLocalEdges;
  const int cnt = (int)(m - b0 < kLocalEdges ? m - b0 : kLocalEdges);
  const uint32_t g0 = (uint32_t)(2 * b0);  // global slot of local slot 0
  bool bad = false;
  if (cnt == kLocalEdges) {  // a full block: 16-byte loads, all in flight at once
    constexpr int kVec = SL / 4 / kLocalThreads;
    uint4 vr[kVec], vs[kVec];
#pragma unroll
    for (int i = 0; i < kVec; ++i) {
      vr[i] = reinterpret_cast<const uint4 *>(rep + g0)[tid + i * kLocalThreads];
      vs[i] = reinterpret_cast<const uint4 *>(sz + g0)[tid + i * kLocalThreads];
    }
#pragma unroll
    for (int i = 0; i < kVec; ++i) {
      const int l = 4 * (tid + i * kLocalThreads);
      const uint32_t r[4] = {vr[i].x, vr[i].y, vr[i].z, vr[i].w};
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int64_t lr = (int64_t)r[j] - g0;
        const bool out = lr < 0 || lr >= SL;
        bad |= out;
        lrep[l + j] = out ? (uint16_t)(l + j) : (uint16_t)lr;
      }
      reinterpret_cast<uint4 *>(szl)[tid + i * kLocalThreads] = vs[i];
    }
  } else {
    for (int l = tid; l < 2 * cnt; l += kLocalThreads) {
      const int64_t lr = (int64_t)rep[g0 + l] - g0;
      const bool out = lr < 0 || lr >= 2 * cnt;
      bad |= out;
      lrep[l] = out ? (uint16_t)l : (uint16_t)lr;
      szl[l] = sz[g0 + l];
    }
  }
  if (__syncthreads_or(bad)) {
    if (tid == 0) atomicOr(status, kErrChain);
    return;
  }
  for (int S = kLocalEdges; S > kSerialEdges; S >>= 1) {
    const int half = S >> 1;
    for (int l = tid; l < 2 * cnt; l += kLocalThreads) {
      uf[l] = (uint32_t)l;
      top[l] = 0;
      minh[l] = kInvalid;
      csz[l] = 0;
    }
    __syncthreads();
    for (int t = tid; t < cnt; t += kLocalThreads) {
      const int start = t & ~(S - 1);
      if ((t & (S - 1)) < half && start + half < cnt && !uf_unite(vuf, lrep[2 * t], lrep[2 * t + 1]))
        atomicOr(status, kErrSpin);
    }
    __syncthreads();
    for (int t = tid; t < cnt; t += kLocalThreads) {
      const int start = t & ~(S - 1);
      if (start + half >= cnt) continue;
      const uint32_t s0 = 2 * t, r0 = lrep[s0], r1 = lrep[s0 + 1];
      const uint32_t x0 = uf_find<true>(vuf, r0);
      if ((t & (S - 1)) < half) {
        atomicMax(top + x0, (uint32_t)t + 1);
        if (r0 == s0) atomicAdd(csz + x0, szl[s0]);
        if (r1 == s0 + 1) atomicAdd(csz + x0, szl[s0 + 1]);
      } else {  // (no sizes, and no minimum for names in the heavy half: as in k_dg_classify)
        const uint32_t hs = 2 * (uint32_t)(start + half);
        if (r0 < hs) atomicMin(minh + x0, s0);
        if (r1 < hs) atomicMin(minh + uf_find<true>(vuf, r1), s0 + 1);
      }
    }
    __syncthreads();
    for (int t = tid; t < cnt; t += kLocalThreads) {
      const int start = t & ~(S - 1);
      if (start + half >= cnt) continue;
      const uint32_t s0 = 2 * t;
      if ((t & (S - 1)) < half) {
        const uint32_t r = uf_find<false>(vuf, lrep[s0]);
        const uint32_t h = minh[r];
        if (top[r] == (uint32_t)t + 1 && h != kInvalid) {
          parent[b0 + t] = g0 + h;
          szl[h] = csz[r];
        }
      } else {
        const uint32_t hs = 2 * (uint32_t)(start + half);
        if (lrep[s0] < hs) lrep[s0] = (uint16_t)minh[uf_find<false>(vuf, lrep[s0])];
        if (lrep[s0 + 1] < hs) lrep[s0 + 1] = (uint16_t)minh[uf_find<false>(vuf, lrep[s0 + 1])];
      }
    }
    __syncthreads();
  }
  // Serial finish: thread j merges local edges [j * kSerialEdges, ...).  Its
  // slots are laid out transposed (slot o of sub-block j at o * kSubs +
  // j), so the lanes of a warp, at the same step of their own sub-blocks,
  // touch 32 different banks.  pn holds each slot's name, transposed too.
  constexpr int kSubSlots = 2 * kSerialEdges;
  constexpr int kSubs = SL / kSubSlots;
  static_assert(kSubs % 32 == 0 && kSubs * kSubSlots == SL, "one sub-block per bank, a bijection");
  static_assert(kSubs <= kLocalThreads, "one thread per sub-block");
  uint32_t *pn = minh;
  for (int l = tid; l < 2 * cnt; l += kLocalThreads) {
    const uint32_t r = lrep[l];
    if (r / kSubSlots != (uint32_t)l / kSubSlots) bad = true;  // a name outside its sub-block
    const uint32_t pl = (l % kSubSlots) * kSubs + l / kSubSlots;
    pn[pl] = (r % kSubSlots) * kSubs + r / kSubSlots;
    uf[pl] = pl;
    top[pl] = 0;
    csz[pl] = r == (uint32_t)l ? szl[l] : 0u;
  }
  if (__syncthreads_or(bad)) {
    if (tid == 0) atomicOr(status, kErrChain);
    return;
  }
  const int j = tid, t0 = j * kSerialEdges;
  if (t0 >= cnt) return;
  const int ne = cnt - t0 < kSerialEdges ? cnt - t0 : kSerialEdges;
  for (int i = 0; i < ne; ++i) {
    uint32_t a = pn[(2 * i) * kSubs + j], b = pn[(2 * i + 1) * kSubs + j];
    while (uf[a] != a) { uf[a] = uf[uf[a]]; a = uf[a]; }
    while (uf[b] != b) { uf[b] = uf[uf[b]]; b = uf[b]; }
    if (a == b) {  // the edge closes a cycle: not a tree
      atomicOr(status, kErrBadInput);
      return;
    }
    const uint32_t k = (uint32_t)(b0 + t0 + i);
    if (top[a]) parent[b0 + t0 + top[a] - 1] = 2 * k;
    if (top[b]) parent[b0 + t0 + top[b] - 1] = 2 * k + 1;
    const uint32_t size = csz[a] + csz[b];
    size_out[k] = size;
    const uint32_t r = a < b ? a : b;
    uf[a ^ b ^ r] = r;
    top[r] = (uint32_t)i + 1;
    csz[r] = size;
  }
}

// Every cluster names its parent: point v (id v) the edge of its lowest
// slot, edge f (id n + f) the edge of slot parent[f], the root none.  Slot
// 2p + side receives exactly one child, the cluster on that side of edge p
// (points were placed there by k_dg_init).
__global__ void k_dg_children(int64_t n, int64_t m, const uint32_t *__restrict__ vslot,
                              const uint32_t *__restrict__ eparent, uint32_t *__restrict__ child,
                              uint32_t *__restrict__ out_parent) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n + m) return;
  // (a point with no edge exists only when the input has a cycle, which
  // the serial finish reports)
  const uint32_t ps = c < n ? vslot[c] : eparent[c - n];
  if (out_parent) out_parent[c] = ps == kInvalid ? kInvalid : (uint32_t)n + (ps >> 1);
  if (child && c >= n && ps != kInvalid) child[ps] = (uint32_t)c;
}

// Linkage rows {a, b, w, size}, the two children ordered a < b.
__global__ void k_dg_rows(const emst_edge *__restrict__ e, int64_t m,
                          const uint32_t *__restrict__ size_out, const uint2 *__restrict__ child,
                          uint4 *__restrict__ link) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= m) return;
  const uint2 c = child[k];
  link[k] = make_uint4(min(c.x, c.y), max(c.x, c.y), __float_as_uint(e[k].w), size_out[k]);
}

}  // namespace

int dendrogram_impl(const emst_edge *edges, int64_t n, uint4 *out_link, uint32_t *out_parent,
                    cudaStream_t s) {
  if (n < 0 || n > EMST_MAX_POINTS) return EMST_ERR_INVALID_ARG;
  if (n == 0) return EMST_OK;
  const int64_t m = n - 1;
  if (m > 0 && !edges) return EMST_ERR_INVALID_ARG;
  const bool link_dev = !out_link || device_accessible(out_link);
  const bool par_dev = !out_parent || device_accessible(out_parent);
  if (m == 0) {
    if (out_parent) {
      const uint32_t root = kInvalid;
      if (cudaMemcpyAsync(out_parent, &root, 4, cudaMemcpyDefault, s) != cudaSuccess ||
          cudaStreamSynchronize(s) != cudaSuccess)
        return EMST_ERR_CUDA;
    }
    return EMST_OK;
  }
  const int64_t m2 = 2 * m;
  const bool edges_dev = device_accessible(edges);
  // scratch: status, vslot[n], rep/sz/uf/top/minh/csz[2m], parent/size[m],
  // plus staging for host edges and host outputs
  size_t off = 0;
  auto take = [&](size_t bytes) {
    off = (off + 255) & ~size_t(255);
    const size_t at = off;
    off += bytes > 0 ? bytes : 1;
    return at;
  };
  const size_t o_status = take(64);
  const size_t o_vslot = take(4 * (size_t)n);
  size_t o_slot[11];  // rep, sz, two sets of (uf, top, minh, csz), child
  for (int i = 0; i < 11; ++i) o_slot[i] = take(4 * (size_t)m2);
  const size_t o_par = take(4 * (size_t)m);
  const size_t o_size = take(4 * (size_t)m);
  const size_t o_edges = edges_dev ? 0 : take(sizeof(emst_edge) * (size_t)m);
  const size_t o_link = (out_link && !link_dev) ? take(16 * (size_t)m) : 0;
  const size_t o_pout = (out_parent && !par_dev) ? take(4 * (size_t)(n + m)) : 0;
  char *base = nullptr;
  if (scratch_alloc((void **)&base, off, s) != cudaSuccess) return EMST_ERR_OOM;
  int rc = EMST_OK;
  uint32_t host_status = 0;
  auto U = [&](size_t o) { return reinterpret_cast<uint32_t *>(base + o); };
  uint32_t *status = U(o_status), *vslot = U(o_vslot), *eparent = U(o_par), *size = U(o_size);
  const emst_edge *e = edges_dev ? edges : reinterpret_cast<emst_edge *>(base + o_edges);
  uint4 *link = out_link ? (link_dev ? out_link : reinterpret_cast<uint4 *>(base + o_link)) : nullptr;
  uint32_t *pout = out_parent ? (par_dev ? out_parent : U(o_pout)) : nullptr;
  Level L;
  L.rep = U(o_slot[0]);
  L.sz = U(o_slot[1]);
  L.uf = U(o_slot[2]);
  L.top = U(o_slot[3]);
  L.minh = U(o_slot[4]);
  L.csz = U(o_slot[5]);
  L.nuf = U(o_slot[6]);
  L.ntop = U(o_slot[7]);
  L.nminh = U(o_slot[8]);
  L.ncsz = U(o_slot[9]);
  L.parent = eparent;
  L.m = m;
  L.status = status;
  const int gm = grid_for(m, kDgBlock), gs = grid_for(m2, kDgBlock);
  cudaMemsetAsync(status, 0, 64, s);
  if (!edges_dev)
    cudaMemcpyAsync((void *)e, edges, sizeof(emst_edge) * (size_t)m, cudaMemcpyHostToDevice, s);
  k_dg_check<<<gm, kDgBlock, 0, s>>>(e, m, n, status);
  // an id out of range would index past vslot: stop before any such access
  if (cudaMemcpyAsync(&host_status, status, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    rc = EMST_ERR_CUDA;
  } else if (host_status != 0) {
    rc = status_from_bits(host_status);
  } else {
    cudaMemsetAsync(vslot, 0xff, 4 * (size_t)n, s);
    cudaMemsetAsync(eparent, 0xff, 4 * (size_t)m, s);
    k_dg_first_slot<<<gs, kDgBlock, 0, s>>>(e, m2, vslot);
    uint32_t *child = link ? U(o_slot[10]) : nullptr;
    int64_t S = kLocalEdges;
    while (S < m) S *= 2;
    // Tagged entries when slot numbers fit their 27 value bits (the level
    // numbers, at most log2(2^26 / kLocalEdges) + 1, fit the 5 tag bits):
    // the union-find, top and lowest-heavy entries are set once here and
    // never cleared again.
    // (EMST_DENDROGRAM_UNTAGGED=1 in the environment selects the cleared
    // entries at any size: the tests run both forms)
    const char *force_plain = getenv("EMST_DENDROGRAM_UNTAGGED");
    const bool tagged = m2 < ((int64_t)1 << 27) && !(force_plain && force_plain[0] == '1');
    L.cur = 1;
    if (tagged) {
      cudaMemsetAsync(L.uf, 0, 4 * (size_t)m2, s);
      cudaMemsetAsync(L.top, 0, 4 * (size_t)m2, s);
      cudaMemsetAsync(L.minh, 0xff, 4 * (size_t)m2, s);
    }
    // the first level reads the set k_dg_init clears (the "next" one here)
    next_level<false>(L);
    if (tagged) k_dg_init<true><<<gs, kDgBlock, 0, s>>>(L, e, vslot, child);
    else k_dg_init<false><<<gs, kDgBlock, 0, s>>>(L, e, vslot, child);
    next_level<false>(L);
    L.cur = 1;
    const int64_t mid = kMidEdges > kLocalEdges ? kMidEdges : 0;
    for (; S > kLocalEdges && (mid == 0 || S > mid); S /= 2) {
      L.mask = (uint32_t)(S - 1);
      L.half = (uint32_t)(S / 2);
      if (tagged) {
        k_dg_unite<true><<<gm, kDgBlock, 0, s>>>(L);
        k_dg_classify<true><<<gm, kDgBlock, 0, s>>>(L);
        k_dg_stitch<true><<<gm, kDgBlock, 0, s>>>(L);
        next_level<true>(L);
      } else {
        k_dg_unite<false><<<gm, kDgBlock, 0, s>>>(L);
        k_dg_classify<false><<<gm, kDgBlock, 0, s>>>(L);
        k_dg_stitch<false><<<gm, kDgBlock, 0, s>>>(L);
        next_level<false>(L);
      }
    }
    if (S > kLocalEdges) {  // the remaining levels, S down to 2 * kLocalEdges, one CTA per block
      if (tagged) k_dg_mid<true><<<(unsigned)((m + S - 1) / S), kMidThreads, 0, s>>>(L, S);
      else k_dg_mid<false><<<(unsigned)((m + S - 1) / S), kMidThreads, 0, s>>>(L, S);
    }
    cudaFuncSetAttribute(k_dg_local, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLocalSmem);
    k_dg_local<<<grid_for(m, kLocalEdges), kLocalThreads, kLocalSmem, s>>>(m, L.rep, L.sz, eparent,
                                                                           size, status);
    k_dg_children<<<grid_for(n + m, kDgBlock), kDgBlock, 0, s>>>(n, m, vslot, eparent, child, pout);
    if (link)
      k_dg_rows<<<gm, kDgBlock, 0, s>>>(e, m, size, reinterpret_cast<const uint2 *>(child), link);
    if (cudaPeekAtLastError() != cudaSuccess) rc = EMST_ERR_CUDA;
    if (out_link && !link_dev)
      cudaMemcpyAsync(out_link, link, 16 * (size_t)m, cudaMemcpyDeviceToHost, s);
    if (out_parent && !par_dev)
      cudaMemcpyAsync(out_parent, pout, 4 * (size_t)(n + m), cudaMemcpyDeviceToHost, s);
    if (cudaMemcpyAsync(&host_status, status, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      rc = EMST_ERR_CUDA;
    else if (rc == EMST_OK)
      rc = status_from_bits(host_status);
  }
  cudaFreeAsync(base, s);
  if (cudaGetLastError() != cudaSuccess && rc == EMST_OK) rc = EMST_ERR_CUDA;
  return rc;
}

}  // namespace emst

extern "C" int emst_dendrogram(const emst_edge *edges, int64_t n, emst_linkage *out_linkage,
                               uint32_t *out_parent, void *stream) {
  static_assert(sizeof(emst_linkage) == 16, "linkage row is 16 bytes");
  return emst::dendrogram_impl(edges, n, reinterpret_cast<uint4 *>(out_linkage), out_parent,
                               (cudaStream_t)stream);
}

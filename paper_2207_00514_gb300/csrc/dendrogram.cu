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
//  - Blocks of kBaseEdges edges finish with the serial merge sequence in
//    shared memory, one warp each, which also gives every cluster's size.
// A contracted vertex is named by an endpoint slot 2k + side of the
// lowest-ranked edge of its block that touches it.  The blocks of one level
// own disjoint slot ranges, so one union-find over all 2m slots serves every
// block of a level at once.
#include "common.cuh"

namespace emst {
namespace {

constexpr int kBaseEdges = 256;  // edges per block of the serial finish
constexpr int kBaseWarps = 4;    // serial blocks per CTA (one warp each)
constexpr int kDgBlock = 256;

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

// Root of x with path halving.  Every parent has a lower priority than its
// child and a parent is only ever replaced by an ancestor, so concurrent
// walks and hooks keep each walk strictly descending: it ends.
__device__ __forceinline__ uint32_t uf_find(uint32_t *uf, uint32_t x) {
  volatile uint32_t *u = uf;
  for (;;) {
    const uint32_t p = u[x];
    if (p == x) return x;
    const uint32_t g = u[p];
    if (g == p) return p;
    u[x] = g;
    x = g;
  }
}

// Joins the sets of a and b (lock-free: a failed hook means another thread
// hooked that root first; retry from the new roots).  False only if the
// retry bound runs out.
__device__ __forceinline__ bool uf_unite(uint32_t *uf, uint32_t a, uint32_t b) {
  for (int it = 0; it < (1 << 22); ++it) {
    a = uf_find(uf, a);
    b = uf_find(uf, b);
    if (a == b) return true;
    uint32_t hi = a, lo = b;
    if (prio(a) < prio(b)) { hi = b; lo = a; }
    if (atomicCAS(uf + hi, hi, lo) == hi) return true;
  }
  return false;
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

// vslot[v] = the lowest slot touching point v (its parent edge is vslot>>1).
__global__ void k_dg_first_slot(const emst_edge *__restrict__ e, int64_t m2,
                                uint32_t *__restrict__ vslot) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= m2) return;
  atomicMin(vslot + slot_vertex(e, (uint32_t)s), (uint32_t)s);
}

// Top level: every vertex is a point, named by its lowest slot, size 1.
__global__ void k_dg_init(const emst_edge *__restrict__ e, int64_t m2,
                          const uint32_t *__restrict__ vslot, uint32_t *__restrict__ rep,
                          uint32_t *__restrict__ sz) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= m2) return;
  rep[s] = vslot[slot_vertex(e, (uint32_t)s)];
  sz[s] = 1;
}

struct Level {
  uint32_t *rep, *sz, *uf, *top, *minh, *csz, *parent;
  int64_t m;
  uint32_t mask, half;  // block size - 1, half the block size
  uint32_t *status;
};

__device__ __forceinline__ bool block_split(const Level &L, uint32_t k, bool &light) {
  const uint32_t start = k & ~L.mask;
  light = (k & L.mask) < L.half;
  return (int64_t)start + L.half < L.m;  // the block has a heavy half
}

__global__ void k_dg_reset(Level L) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= 2 * L.m) return;
  L.uf[s] = (uint32_t)s;
  L.top[s] = 0;
  L.minh[s] = kInvalid;
  L.csz[s] = 0;
}

// Light components: unite the two vertices of every light edge.
__global__ void k_dg_unite(Level L) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= L.m) return;
  bool light;
  if (!block_split(L, (uint32_t)k, light) || !light) return;
  if (!uf_unite(L.uf, L.rep[2 * k], L.rep[2 * k + 1])) atomicOr(L.status, kErrSpin);
}

// Per light component (by root): its top edge (rank + 1), its size (the sum
// over its vertices, each counted at the slot that names it) and the lowest
// heavy slot touching it.
__global__ void k_dg_classify(Level L) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= L.m) return;
  bool light;
  if (!block_split(L, (uint32_t)k, light)) return;
  const uint32_t s0 = 2 * (uint32_t)k;
  const uint32_t r0 = L.rep[s0], r1 = L.rep[s0 + 1];
  if (light) {
    atomicMax(L.top + uf_find(L.uf, r0), (uint32_t)k + 1);
  } else {
    atomicMin(L.minh + uf_find(L.uf, r0), s0);
    atomicMin(L.minh + uf_find(L.uf, r1), s0 + 1);
  }
  if (r0 == s0) atomicAdd(L.csz + uf_find(L.uf, s0), L.sz[s0]);
  if (r1 == s0 + 1) atomicAdd(L.csz + uf_find(L.uf, s0 + 1), L.sz[s0 + 1]);
}

// The top edge of each light component takes the lowest heavy edge touching
// it as its parent, and hands the component's size to the slot that names
// the component in the heavy half; heavy slots are renamed to that slot.
__global__ void k_dg_stitch(Level L) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= L.m) return;
  bool light;
  if (!block_split(L, (uint32_t)k, light)) return;
  const uint32_t s0 = 2 * (uint32_t)k;
  if (light) {
    const uint32_t r = uf_find(L.uf, L.rep[s0]);
    const uint32_t h = L.minh[r];
    if (L.top[r] == (uint32_t)k + 1 && h != kInvalid) {
      L.parent[k] = h >> 1;
      L.sz[h] = L.csz[r];
    }
  } else {
    L.rep[s0] = L.minh[uf_find(L.uf, L.rep[s0])];
    L.rep[s0 + 1] = L.minh[uf_find(L.uf, L.rep[s0 + 1])];
  }
}

// The serial finish: one warp per block of kBaseEdges edges.  The lanes
// stage the block's vertex names (local slot numbers) and sizes in shared
// memory; lane 0 then runs the merge sequence over them.
__global__ void __launch_bounds__(32 * kBaseWarps)
    k_dg_base(int64_t m, const uint32_t *__restrict__ rep, const uint32_t *__restrict__ sz,
              uint32_t *__restrict__ parent, uint32_t *__restrict__ size_out, uint32_t *status) {
  __shared__ uint16_t s_rep[kBaseWarps][2 * kBaseEdges];
  __shared__ uint16_t s_uf[kBaseWarps][2 * kBaseEdges];
  __shared__ uint16_t s_top[kBaseWarps][2 * kBaseEdges];
  __shared__ uint32_t s_size[kBaseWarps][2 * kBaseEdges];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t b0 = ((int64_t)blockIdx.x * kBaseWarps + w) * kBaseEdges;
  if (b0 >= m) return;
  const int cnt = (int)(m - b0 < kBaseEdges ? m - b0 : kBaseEdges);
  uint16_t *lrep = s_rep[w], *uf = s_uf[w], *top = s_top[w];
  uint32_t *csize = s_size[w];
  bool bad = false;
  for (int l = lane; l < 2 * cnt; l += 32) {
    const uint32_t s = (uint32_t)(2 * b0) + l;
    const uint32_t r = rep[s];
    const int64_t lr = (int64_t)r - 2 * b0;
    if (lr < 0 || lr >= 2 * cnt) bad = true;
    lrep[l] = bad ? (uint16_t)l : (uint16_t)lr;
    uf[l] = (uint16_t)l;
    top[l] = 0;
    csize[l] = r == s ? sz[s] : 0;
  }
  if (__any_sync(0xffffffffu, bad)) {
    if (lane == 0) atomicOr(status, kErrChain);
    return;
  }
  __syncwarp();
  if (lane != 0) return;
  for (int t = 0; t < cnt; ++t) {
    uint32_t a = lrep[2 * t], b = lrep[2 * t + 1];
    while (uf[a] != a) { uf[a] = uf[uf[a]]; a = uf[a]; }
    while (uf[b] != b) { uf[b] = uf[uf[b]]; b = uf[b]; }
    if (a == b) {  // the edge closes a cycle: not a tree
      atomicOr(status, kErrBadInput);
      return;
    }
    const uint32_t k = (uint32_t)b0 + t;
    if (top[a]) parent[b0 + top[a] - 1] = k;
    if (top[b]) parent[b0 + top[b] - 1] = k;
    const uint32_t size = csize[a] + csize[b];
    size_out[k] = size;
    const uint32_t r = a < b ? a : b;
    uf[a ^ b ^ r] = (uint16_t)r;
    top[r] = (uint16_t)(t + 1);
    csize[r] = size;
  }
}

// Linkage rows {a, b, w, size}: w and size now, the children (a < b) by
// min/max scatter from both sides in k_dg_children.
__global__ void k_dg_rows(const emst_edge *__restrict__ e, int64_t m,
                          const uint32_t *__restrict__ size_out, uint4 *__restrict__ link) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= m) return;
  link[k] = make_uint4(kInvalid, 0u, __float_as_uint(e[k].w), size_out[k]);
}

// Every cluster names its parent: point v (id v) hangs under its lowest
// edge, edge f (id n + f) under parent[f].  Each row receives exactly two
// children, so a min and a max order them.
__global__ void k_dg_children(int64_t n, int64_t m, const uint32_t *__restrict__ vslot,
                              const uint32_t *__restrict__ eparent, uint4 *link,
                              uint32_t *__restrict__ out_parent) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n + m) return;
  // (a point with no edge exists only when the input has a cycle, which
  // the serial finish reports)
  uint32_t p = kInvalid;
  if (c < n) p = vslot[c] == kInvalid ? kInvalid : vslot[c] >> 1;
  else p = eparent[c - n];
  if (out_parent) out_parent[c] = p == kInvalid ? kInvalid : (uint32_t)n + p;
  if (link && p != kInvalid) {
    atomicMin(&link[p].x, (uint32_t)c);
    atomicMax(&link[p].y, (uint32_t)c);
  }
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
  size_t o_slot[6];
  for (int i = 0; i < 6; ++i) o_slot[i] = take(4 * (size_t)m2);
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
    k_dg_init<<<gs, kDgBlock, 0, s>>>(e, m2, vslot, L.rep, L.sz);
    int64_t S = kBaseEdges;
    while (S < m) S *= 2;
    for (; S > kBaseEdges; S /= 2) {
      L.mask = (uint32_t)(S - 1);
      L.half = (uint32_t)(S / 2);
      k_dg_reset<<<gs, kDgBlock, 0, s>>>(L);
      k_dg_unite<<<gm, kDgBlock, 0, s>>>(L);
      k_dg_classify<<<gm, kDgBlock, 0, s>>>(L);
      k_dg_stitch<<<gm, kDgBlock, 0, s>>>(L);
    }
    const int64_t blocks = (m + kBaseEdges - 1) / kBaseEdges;
    k_dg_base<<<grid_for(blocks, kBaseWarps), 32 * kBaseWarps, 0, s>>>(m, L.rep, L.sz, eparent,
                                                                       size, status);
    if (link) k_dg_rows<<<gm, kDgBlock, 0, s>>>(e, m, size, link);
    k_dg_children<<<grid_for(n + m, kDgBlock), kDgBlock, 0, s>>>(n, m, vslot, eparent, link, pout);
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

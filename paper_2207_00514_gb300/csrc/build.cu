// build.cu -- the tree build of the method (§2 "ArborX": Z-curve
// linearisation, sort, fully parallel bottom-up hierarchy construction):
//   A1 scene box, A2 Morton codes, A3 (sort.cu), A4 gather + hierarchy + refit.
#include "common.cuh"

namespace emst {

constexpr int kBlock = 256;

// ---------------------------------------------------------------------------
// A1. Scene box: per-dimension min / max of all coordinates, plus a flag for
// any non-finite coordinate.  box[0..2] = ordered min, box[3..5] = ordered max.
// ---------------------------------------------------------------------------
// COPY: the points are read from pinned host memory through its device
// mapping and written to `copy` (device) on the way, so the host-to-device
// transfer of a host input is this pass itself.
template <int DIM, bool COPY>
__global__ void __launch_bounds__(kBlock) k_scene_box(const float *__restrict__ pts, int64_t n,
                                                      uint32_t *__restrict__ box,
                                                      uint32_t *__restrict__ status,
                                                      float *__restrict__ copy) {
  float lo[3] = {INFINITY, INFINITY, INFINITY};
  float hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  bool bad = false;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  auto take = [&](int64_t k) {
#pragma unroll
    for (int q = 0; q < DIM; ++q) {
      const float x = COPY ? pts[k * DIM + q] : __ldg(pts + k * DIM + q);
      if (COPY) copy[k * DIM + q] = x;
      if (!isfinite(x)) { bad = true; continue; }
      lo[q] = fminf(lo[q], x);
      hi[q] = fmaxf(hi[q], x);
    }
  };
  // whole points per thread, four independent ones per step (loads in flight)
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; k + 3 * stride < n; k += 4 * stride) {
    take(k);
    take(k + stride);
    take(k + 2 * stride);
    take(k + 3 * stride);
  }
  for (; k < n; k += stride) take(k);
#pragma unroll
  for (int q = 0; q < DIM; ++q) {
    for (int o = 16; o > 0; o >>= 1) {
      lo[q] = fminf(lo[q], __shfl_xor_sync(0xffffffffu, lo[q], o));
      hi[q] = fmaxf(hi[q], __shfl_xor_sync(0xffffffffu, hi[q], o));
    }
  }
  if ((threadIdx.x & 31) == 0) {
#pragma unroll
    for (int q = 0; q < DIM; ++q) {
      if (lo[q] <= hi[q]) {
        atomicMin(&box[q], float_to_ordered(lo[q]));
        atomicMax(&box[3 + q], float_to_ordered(hi[q]));
      }
    }
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(status, kErrNonFinite);
}

// The COPY form reading 16 bytes per load (the host input through its
// mapping): the flat coordinate array as float4s, element e of dimension
// e % DIM; `tail` (< 4) trailing elements read one by one by thread 0.
// src and copy 16-byte aligned.
template <int DIM>
__global__ void __launch_bounds__(kBlock) k_scene_box_copy4(const float4 *__restrict__ src,
                                                            int64_t nv, int tail,
                                                            uint32_t *__restrict__ box,
                                                            uint32_t *__restrict__ status,
                                                            float4 *__restrict__ copy) {
  float lo[3] = {INFINITY, INFINITY, INFINITY};
  float hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  bool bad = false;
  auto take = [&](float x, int d) {
    if (!isfinite(x)) { bad = true; return; }
#pragma unroll
    for (int q = 0; q < DIM; ++q) {
      if (q == d) {
        lo[q] = fminf(lo[q], x);
        hi[q] = fmaxf(hi[q], x);
      }
    }
  };
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  auto use = [&](const float4 &a, int64_t v) {
    copy[v] = a;
    const int d0 = (int)((4 * v) % DIM);
    take(a.x, d0);
    take(a.y, (d0 + 1) % DIM);
    take(a.z, (d0 + 2) % DIM);
    take(a.w, (d0 + 3) % DIM);
  };
  // four independent loads in flight per thread (the link's latency is long)
  int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; v + 3 * stride < nv; v += 4 * stride) {
    const float4 a0 = src[v], a1 = src[v + stride], a2 = src[v + 2 * stride], a3 = src[v + 3 * stride];
    use(a0, v);
    use(a1, v + stride);
    use(a2, v + 2 * stride);
    use(a3, v + 3 * stride);
  }
  for (; v < nv; v += stride) use(src[v], v);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const float *s1 = reinterpret_cast<const float *>(src + nv);
    float *c1 = reinterpret_cast<float *>(copy + nv);
    for (int t = 0; t < tail; ++t) {
      c1[t] = s1[t];
      take(s1[t], (int)((4 * nv + t) % DIM));
    }
  }
#pragma unroll
  for (int q = 0; q < DIM; ++q) {
    for (int o = 16; o > 0; o >>= 1) {
      lo[q] = fminf(lo[q], __shfl_xor_sync(0xffffffffu, lo[q], o));
      hi[q] = fmaxf(hi[q], __shfl_xor_sync(0xffffffffu, hi[q], o));
    }
  }
  if ((threadIdx.x & 31) == 0) {
#pragma unroll
    for (int q = 0; q < DIM; ++q) {
      if (lo[q] <= hi[q]) {
        atomicMin(&box[q], float_to_ordered(lo[q]));
        atomicMax(&box[3 + q], float_to_ordered(hi[q]));
      }
    }
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(status, kErrNonFinite);
}

__global__ void k_box_init(uint32_t *box) {
  int t = threadIdx.x;
  if (t < 3) box[t] = 0xFFFFFFFFu;
  else if (t < 6) box[t] = 0u;
}

void launch_scene_box(Problem &P) {
  uint32_t *box = P.counters + 4;
  k_box_init<<<1, 32, 0, P.stream>>>(box);
  int grid = sm_count() * 4;
  int64_t need = (P.n + kBlock - 1) / kBlock;
  if (need < grid) grid = (int)(need < 1 ? 1 : need);
  float *copy = const_cast<float *>(P.points);
  if (P.points_mapped && (reinterpret_cast<uintptr_t>(P.points_mapped) & 15u) == 0 &&
      (reinterpret_cast<uintptr_t>(copy) & 15u) == 0) {
    // read the host input through its mapping 16 bytes at a time, keep a device copy
    const int64_t elems = P.n * P.dim, nv = elems / 4;
    const int tail = (int)(elems - 4 * nv);
    int g4 = sm_count() * 4;
    if ((nv + kBlock - 1) / kBlock < g4) g4 = (int)((nv + kBlock - 1) / kBlock < 1 ? 1 : (nv + kBlock - 1) / kBlock);
    const float4 *src = reinterpret_cast<const float4 *>(P.points_mapped);
    float4 *dst = reinterpret_cast<float4 *>(copy);
    if (P.dim == 3)
      k_scene_box_copy4<3><<<g4, kBlock, 0, P.stream>>>(src, nv, tail, box, P.counters + 1, dst);
    else
      k_scene_box_copy4<2><<<g4, kBlock, 0, P.stream>>>(src, nv, tail, box, P.counters + 1, dst);
  } else if (P.points_mapped) {  // read the host input through its mapping, keep a device copy
    if (P.dim == 3)
      k_scene_box<3, true><<<grid, kBlock, 0, P.stream>>>(P.points_mapped, P.n, box, P.counters + 1, copy);
    else
      k_scene_box<2, true><<<grid, kBlock, 0, P.stream>>>(P.points_mapped, P.n, box, P.counters + 1, copy);
  } else if (P.dim == 3) {
    k_scene_box<3, false><<<grid, kBlock, 0, P.stream>>>(P.points, P.n, box, P.counters + 1, nullptr);
  } else {
    k_scene_box<2, false><<<grid, kBlock, 0, P.stream>>>(P.points, P.n, box, P.counters + 1, nullptr);
  }
  P.launches += 2;
}

// ---------------------------------------------------------------------------
// A2. Morton codes.  Quantisation decided in FP32 exactly as specified (B = 21
// bits per dimension in 3D, 32 in 2D; fewer in the batched form, see
// code_bits):
//   s = 2^B / (hi - lo) (0 for a flat dimension), t = (x - lo) * s,
//   q = t >= 2^B ? 2^B - 1 : trunc(t)
// and the bits interleave x (most significant), y, z.
// ---------------------------------------------------------------------------
// With instances, the instance id goes above the interleaved bits.
template <int DIM>
__global__ void __launch_bounds__(kBlock) k_morton(const float *__restrict__ pts, int64_t n,
                                                   const uint32_t *__restrict__ box,
                                                   const uint32_t *__restrict__ inst_in, int bits,
                                                   uint64_t *__restrict__ keys,
                                                   uint32_t *__restrict__ vals) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const Quantizer Q = make_quantizer(box, DIM, bits);
  uint32_t q[3] = {0, 0, 0};
#pragma unroll
  for (int d = 0; d < DIM; ++d) q[d] = quantize(Q, d, __ldg(pts + k * DIM + d));
  uint64_t code = interleave(q[0], q[1], q[2], DIM);
  if (inst_in) code |= (uint64_t)__ldg(inst_in + k) << (DIM * bits);
  keys[k] = code;
  vals[k] = (uint32_t)k;
}

void launch_morton(Problem &P) {
  int g = grid_for(P.n, kBlock);
  const int bits = code_bits(P.dim, P.inst_bits);
  if (P.dim == 3)
    k_morton<3><<<g, kBlock, 0, P.stream>>>(P.points, P.n, P.counters + 4, P.inst_in, bits,
                                            P.keys[0], P.vals[0]);
  else
    k_morton<2><<<g, kBlock, 0, P.stream>>>(P.points, P.n, P.counters + 4, P.inst_in, bits,
                                            P.keys[0], P.vals[0]);
  P.launches += 1;
}

// A2 at the finer grid §4.1 suggests for very dense data (128-bit codes):
// B = 42 bits per dimension in 3D, 64 in 2D, quantised in FP64 so the grid
// resolves FP32 coordinates:
//   s = 2^B / (hi - lo) (0 for a flat dimension), t = (x - lo) * s,
//   q = t >= 2^B ? 2^B - 1 : trunc(t)
// every step rounded explicitly.  The code is the 64-bit interleave of each
// half of the cells: in 3D, with H and L the 63-bit interleaves of the high
// and low 21 bits, code = H << 63 | L; in 2D the halves are the two words.
template <int DIM>
__global__ void __launch_bounds__(kBlock) k_morton128(const float *__restrict__ pts, int64_t n,
                                                      const uint32_t *__restrict__ box,
                                                      uint64_t *__restrict__ code_hi,
                                                      uint64_t *__restrict__ code_lo,
                                                      uint64_t *__restrict__ keys,
                                                      uint32_t *__restrict__ vals) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  constexpr int B = DIM == 3 ? 42 : 64;
  const double twoB = DIM == 3 ? 4398046511104.0 : 18446744073709551616.0;  // 2^B
  const uint64_t qmax = DIM == 3 ? ((1ull << 42) - 1ull) : ~0ull;
  uint64_t q[3] = {0, 0, 0};
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    const double lo = (double)ordered_to_float(box[d]);
    const double ext = __dsub_rn((double)ordered_to_float(box[3 + d]), lo);
    const double sc = ext > 0.0 ? __ddiv_rn(twoB, ext) : 0.0;
    const double t = __dmul_rn(__dsub_rn((double)__ldg(pts + k * DIM + d), lo), sc);
    q[d] = t >= twoB ? qmax : (uint64_t)t;
  }
  uint64_t hi, lo;
  if (DIM == 3) {
    const uint64_t H = interleave((uint32_t)(q[0] >> 21), (uint32_t)(q[1] >> 21), (uint32_t)(q[2] >> 21), 3);
    const uint64_t L = interleave((uint32_t)(q[0] & 0x1fffffu), (uint32_t)(q[1] & 0x1fffffu),
                                  (uint32_t)(q[2] & 0x1fffffu), 3);
    hi = H >> 1;
    lo = L | (H << 63);
  } else {
    hi = interleave((uint32_t)(q[0] >> 32), (uint32_t)(q[1] >> 32), 0u, 2);
    lo = interleave((uint32_t)q[0], (uint32_t)q[1], 0u, 2);
  }
  (void)B;
  code_hi[k] = hi;
  code_lo[k] = lo;
  keys[k] = lo;
  vals[k] = (uint32_t)k;
}

void launch_morton128(Problem &P) {
  int g = grid_for(P.n, kBlock);
  if (P.dim == 3)
    k_morton128<3><<<g, kBlock, 0, P.stream>>>(P.points, P.n, P.counters + 4, P.wide_hi, P.wide_lo,
                                               P.keys[0], P.vals[0]);
  else
    k_morton128<2><<<g, kBlock, 0, P.stream>>>(P.points, P.n, P.counters + 4, P.wide_hi, P.wide_lo,
                                               P.keys[0], P.vals[0]);
  P.launches += 1;
}

// out[k] = src[idx[k]] (a 64-bit word carried through a permutation)
__global__ void k_gather_u64(const uint64_t *__restrict__ src, const uint32_t *__restrict__ idx,
                             int64_t n, uint64_t *__restrict__ out) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) out[k] = __ldg(src + __ldg(idx + k));
}

void launch_gather_u64(Problem &P, const uint64_t *src, const uint32_t *idx, uint64_t *out) {
  k_gather_u64<<<grid_for(P.n, kBlock), kBlock, 0, P.stream>>>(src, idx, P.n, out);
  P.launches += 1;
}

// Instance id of every input row (binary search in the offsets).
__global__ void __launch_bounds__(kBlock) k_instance_ids(const int64_t *__restrict__ offsets,
                                                         int64_t num_inst, int64_t n,
                                                         uint32_t *__restrict__ inst_in) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  int64_t lo = 0, hi = num_inst - 1;  // last instance whose start is <= k
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) >> 1;
    if (__ldg(offsets + mid) <= k) lo = mid; else hi = mid - 1;
  }
  inst_in[k] = (uint32_t)lo;
}

void launch_instance_ids(Problem &P) {
  k_instance_ids<<<grid_for(P.n, kBlock), kBlock, 0, P.stream>>>(P.offsets, P.num_inst, P.n,
                                                                 P.inst_in);
  P.launches += 1;
}

// Root node of each instance's subtree: the node whose chunk range is exactly
// the instance's (one of its two ends is the node's index); kInvalid for an
// instance with fewer than two chunks... of points (nothing to search).
__global__ void __launch_bounds__(kBlock) k_instance_roots(const int64_t *__restrict__ offsets,
                                                           int64_t num_inst, int64_t nc, int leaf,
                                                           const uint2 *__restrict__ range,
                                                           uint32_t *__restrict__ inst_root,
                                                           uint32_t *status) {
  int64_t I = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= num_inst) return;
  const int64_t a = __ldg(offsets + I), b = __ldg(offsets + I + 1) - 1;
  if (b <= a) { inst_root[I] = kInvalid; return; }
  const int64_t ca = a / leaf, cb = b / leaf;
  uint32_t root = kInvalid;
  if (ca == cb) {
    root = kInvalid;  // inside one leaf chunk: cannot happen with leaf 1 (a < b)
  } else {
    if (ca < nc - 1) {
      const NodeRange r = unpack_range((uint32_t)ca, __ldg(range + ca));
      if (r.first == (uint32_t)ca && r.last == (uint32_t)cb) root = (uint32_t)ca;
    }
    if (root == kInvalid && cb < nc - 1) {
      const NodeRange r = unpack_range((uint32_t)cb, __ldg(range + cb));
      if (r.first == (uint32_t)ca && r.last == (uint32_t)cb) root = (uint32_t)cb;
    }
  }
  if (root == kInvalid) atomicOr(status, kErrChain);
  inst_root[I] = root;
}

void launch_instance_roots(Problem &P) {
  k_instance_roots<<<grid_for(P.num_inst, kBlock), kBlock, 0, P.stream>>>(
      P.offsets, P.num_inst, P.nc, P.leaf, P.range, P.inst_root, P.counters + 1);
  P.launches += 1;
}

// ---------------------------------------------------------------------------
// A4 (a). Gather the points into curve order as float4 (x, y, z, original
// index bits) and the first labels (labels(i) = i, Fig. 3), in curve indices.
// ---------------------------------------------------------------------------
// Also counts, over the curve positions whose code equals the previous
// position's: identical points (dup[0]) and distinct points the grid does not
// separate (dup[1]: a cell holding many of them has no spatial order inside,
// so its subtree's boxes all span it); and flags (dup[2] != 0) a run of more
// than 32 equal codes -- the only way a group of identical points can be
// large, which is when the search needs its tie rule.
// code_hi: the codes' high words (128-bit codes), else nullptr.
template <int DIM>
__global__ void __launch_bounds__(kBlock) k_gather(const float *__restrict__ pts,
                                                   const uint32_t *__restrict__ perm, int64_t n,
                                                   float4 *__restrict__ out,
                                                   uint32_t *__restrict__ labels,
                                                   const uint32_t *__restrict__ inst_in,
                                                   uint32_t *__restrict__ inst_of,
                                                   const uint64_t *__restrict__ sorted_codes,
                                                   const uint64_t *__restrict__ code_hi,
                                                   unsigned long long *dup) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  uint32_t o = __ldg(perm + k);
  if (inst_of) inst_of[k] = __ldg(inst_in + o);
  const float *p = pts + (int64_t)o * DIM;
  float x = __ldg(p), y = __ldg(p + 1), z = DIM == 3 ? __ldg(p + 2) : 0.0f;
  out[k] = make_float4(x, y, z, __uint_as_float(o));
  labels[k] = (uint32_t)k;
  bool same = false, differ = false;
  if (k > 0 && __ldg(sorted_codes + k) == __ldg(sorted_codes + k - 1) &&
      (!code_hi || __ldg(code_hi + k) == __ldg(code_hi + k - 1))) {
    const float *q = pts + (int64_t)__ldg(perm + k - 1) * DIM;
    differ = __ldg(q) != x || __ldg(q + 1) != y || (DIM == 3 && __ldg(q + 2) != z);
    same = !differ;
  }
  // sorted codes: equal 32 positions back means all between are equal too
  const bool run = k >= 32 && __ldg(sorted_codes + k) == __ldg(sorted_codes + k - 32) &&
                   (!code_hi || __ldg(code_hi + k) == __ldg(code_hi + k - 32));
  const unsigned mask = __activemask();
  const unsigned cs = __popc(__ballot_sync(mask, same)), cd = __popc(__ballot_sync(mask, differ));
  const unsigned cr = __ballot_sync(mask, run);
  if ((threadIdx.x & 31) == (unsigned)(__ffs(mask) - 1)) {
    if (cs) atomicAdd(dup, (unsigned long long)cs);
    if (cd) atomicAdd(dup + 1, (unsigned long long)cd);
    if (cr) atomicOr(reinterpret_cast<unsigned int *>(dup + 2), 1u);
  }
}

void launch_gather(Problem &P, const uint32_t *perm) {
  int g = grid_for(P.n, kBlock);
  unsigned long long *dup = reinterpret_cast<unsigned long long *>(P.counters + 28);
  cudaMemsetAsync(dup, 0, 3 * sizeof(unsigned long long), P.stream);
  if (P.dim == 3)
    k_gather<3><<<g, kBlock, 0, P.stream>>>(P.points, perm, P.n, P.pts, P.labels, P.inst_in,
                                            P.inst_of, P.keys[0], P.code_hi, dup);
  else
    k_gather<2><<<g, kBlock, 0, P.stream>>>(P.points, perm, P.n, P.pts, P.labels, P.inst_in,
                                            P.inst_of, P.keys[0], P.code_hi, dup);
  P.launches += 1;
}

// ---------------------------------------------------------------------------
// A4 (b, c). Hierarchy and boxes in one bottom-up pass.
// The hierarchy is Karras's binary radix tree over the leaf chunks (chunks of
// `leaf` consecutive sorted points; leaf = 1: one point per leaf; chunk c's
// key is the code of its first point, augmented by c so equal codes still
// split), numbered as in Fig. 4: internal node i covers a chunk range with
// one end at i, and its split gamma gives the children gamma (left) and
// gamma + 1 (right), leaves when the range ends there.
// Here it is found from the leaves up (the agglomerative form of the same
// tree): with delta(i) the leading bits shared by the keys of chunks i and
// i + 1, a node covering chunks [l, r] hangs under the split r (it is the
// left child) when delta(r) > delta(l - 1), else under the split l - 1 (the
// right child).  So a left child's index is its right end and a right
// child's its left end: a node knows its own index once it knows which side
// it hangs on.  At every split the first child to arrive stops and the
// second builds the parent: its range from both children's far ends, its
// box as the union of theirs, its record (both child boxes, the child
// references, their smallest original ids), range and round-0 child labels,
// written once at the parent's index; then it carries on upwards.
// k_build_local: one thread per leaf chunk climbs the splits between two of
// its CTA's chunks, with the CTA's shared keys' delta values, boxes and
// arrival counts in shared memory (block-scope acquire-release adds).  A
// split at the CTA's edge ends the climb in global memory: the thread leaves
// its far end in split_far, adds a device-scope acquire-release arrival, and
// the second arriver lists the split.  A split inside the CTA that only one
// child reached (the other spans CTAs) passes that child's far end to global
// memory at the end.
// k_build_up: one thread per listed split builds it and climbs on in global
// memory; a child's box comes from its record (the union of the record's two
// child boxes) or from its points (a leaf).
// Each split gets exactly two arrivals; the counters start at zero.
// The child labels are the round-0 ones (a one-point chunk k: label k;
// otherwise several components, kInvalid); a caller with other labels
// rewrites them (A5).
// ---------------------------------------------------------------------------
// kh != nullptr: 128-bit codes, kh their high words (the augmented key is
// then (high, low, position), 160 bits)
__device__ __forceinline__ int prefix_delta(const uint64_t *__restrict__ k,
                                            const uint64_t *__restrict__ kh, int64_t nc, int leaf,
                                            int64_t i, int64_t j) {
  if (j < 0 || j >= nc || i < 0 || i >= nc) return -1;
  int base = 0;
  if (kh) {
    const uint64_t a = __ldg(kh + i * leaf), b = __ldg(kh + j * leaf);
    if (a != b) return __clzll((long long)(a ^ b));
    base = 64;
  }
  uint64_t a = __ldg(k + i * leaf), b = __ldg(k + j * leaf);
  if (a != b) return base + __clzll((long long)(a ^ b));
  return base + 64 + __clz((int)((uint32_t)i ^ (uint32_t)j));
}

#ifndef EMST_REFIT_BLOCK
#define EMST_REFIT_BLOCK 128
#endif
constexpr int kRefitBlock = EMST_REFIT_BLOCK;  // leaf chunks per k_build_local CTA
constexpr int kRefitUpBlock = 128;
constexpr uint32_t kRefitReadyCounter = 48;  // P.counters slot: splits listed by k_build_local

// The split a node [l, r] hangs under and its side (0: left child, the split
// is r; 1: right child, the split is l - 1), from delta(l - 1) and delta(r);
// false for the root.
__device__ __forceinline__ bool parent_split(int64_t l, int64_t r, int64_t nc, int dl, int dr,
                                             uint32_t &ps, int &side) {
  if (l == 0 && r == nc - 1) return false;
  const bool left = l == 0 || (r != nc - 1 && dr > dl);
  ps = (uint32_t)(left ? r : l - 1);
  side = left ? 0 : 1;
  return true;
}

// The index of node [l, r] (Fig. 4 numbering): 0 for the root, else the end
// of its range away from the split it hangs under.
__device__ __forceinline__ uint32_t node_index(int64_t l, int64_t r, bool root, int side) {
  return root ? 0u : (uint32_t)(side == 0 ? r : l);
}

__device__ __forceinline__ void chunk_box(const float4 *__restrict__ pts, int64_t n, int leaf,
                                          int64_t c, float *box, uint32_t &idmin) {
  const int64_t p0 = c * leaf, p1 = p0 + leaf < n ? p0 + leaf : n;
  float4 p = __ldg(pts + p0);
  box[0] = box[3] = p.x;
  box[1] = box[4] = p.y;
  box[2] = box[5] = p.z;
  idmin = __float_as_uint(p.w);
  for (int64_t m = p0 + 1; m < p1; ++m) {
    p = __ldg(pts + m);
    box[0] = fminf(box[0], p.x); box[1] = fminf(box[1], p.y); box[2] = fminf(box[2], p.z);
    box[3] = fmaxf(box[3], p.x); box[4] = fmaxf(box[4], p.y); box[5] = fmaxf(box[5], p.z);
    idmin = min(idmin, __float_as_uint(p.w));
  }
}

// A finished child's box and smallest original id: a leaf chunk's from its
// points, an internal node's from its record (written before its arrival was
// released, so read through L2).
__device__ __forceinline__ void child_box(const float4 *__restrict__ pts, int64_t n, int leaf,
                                          const NodeRec *nodes, uint32_t idx, bool is_leaf,
                                          float *box, uint32_t &idmin) {
  if (is_leaf) {
    chunk_box(pts, n, leaf, idx, box, idmin);
    return;
  }
  const float4 *f = reinterpret_cast<const float4 *>(nodes + idx);
  const float4 a = __ldcg(f), b = __ldcg(f + 1), c = __ldcg(f + 2);
  const uint4 d = __ldcg(reinterpret_cast<const uint4 *>(f + 3));
  box[0] = fminf(a.x, b.z); box[1] = fminf(a.y, b.w); box[2] = fminf(a.z, c.x);
  box[3] = fmaxf(a.w, c.y); box[4] = fmaxf(b.x, c.z); box[5] = fmaxf(b.y, c.w);
  idmin = min(d.z, d.w);
}

// Node `idx` covering chunks [L, R] with split g and child boxes Lb, Rb (and
// their smallest original ids): its whole record, range and round-0 child
// labels; returns the union in `box` / `idmin` (which may alias Lb or Rb).
__device__ __forceinline__ void write_node(NodeRec *nodes, uint2 *__restrict__ nlabels,
                                           uint2 *__restrict__ range, uint32_t idx, uint32_t L,
                                           uint32_t g, uint32_t R, const float *Lb, const float *Rb,
                                           uint32_t minL, uint32_t minR, int64_t n, int leaf,
                                           float *box, uint32_t &idmin) {
  const bool lleaf = L == g, rleaf = R == g + 1u;
  // a chunk of exactly one point is its own component in round 0
  auto one_point = [&](int64_t c) { return n - c * leaf == 1 || leaf == 1; };
  NodeRec rec;
  rec.a = make_float4(Lb[0], Lb[1], Lb[2], Lb[3]);
  rec.b = make_float4(Lb[4], Lb[5], Rb[0], Rb[1]);
  rec.c = make_float4(Rb[2], Rb[3], Rb[4], Rb[5]);
  rec.d = make_uint4(lleaf ? (kLeafBit | g) : g, rleaf ? (kLeafBit | (g + 1u)) : g + 1u, minL, minR);
  nodes[idx] = rec;
  range[idx] = pack_range(idx, L, g, R);
  nlabels[idx] = make_uint2(lleaf && one_point(g) ? (uint32_t)((int64_t)g * leaf) : kInvalid,
                            rleaf && one_point(g + 1) ? (uint32_t)((int64_t)(g + 1) * leaf) : kInvalid);
#pragma unroll
  for (int t = 0; t < 3; ++t) {
    const float lo = fminf(Lb[t], Rb[t]), hi = fmaxf(Lb[3 + t], Rb[3 + t]);
    box[t] = lo;
    box[3 + t] = hi;
  }
  idmin = min(minL, minR);
}

// Arrival counters with acquire-release order: the first arriver's stores
// (its box and far end) are released by its add, and the second arriver's
// add acquires them, so no separate fences are needed around the add.
__device__ __forceinline__ uint32_t add_acq_rel_gpu(uint32_t *p, uint32_t v) {
  uint32_t old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}
__device__ __forceinline__ uint32_t add_acq_rel_cta_shared(uint32_t *p, uint32_t v) {
  uint32_t old;
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
  asm volatile("atom.acq_rel.cta.shared::cta.add.u32 %0, [%1], %2;" : "=r"(old) : "r"(a), "r"(v) : "memory");
  return old;
}

__global__ void __launch_bounds__(kRefitBlock) k_build_local(
    const uint64_t *__restrict__ keys, const uint64_t *__restrict__ keys_hi,
    const float4 *__restrict__ pts, int64_t n, int64_t nc, int leaf, NodeRec *nodes,
    uint2 *__restrict__ nlabels, uint2 *__restrict__ range, uint2 *split_far, uint32_t *arrivals,
    uint32_t *__restrict__ ready, uint32_t *ready_count, uint32_t capacity, uint32_t *status) {
  __shared__ int s_delta[kRefitBlock + 1];     // delta(first - 1 + t)
  __shared__ float s_box[kRefitBlock][2][6];   // both child boxes of each split inside the CTA
  __shared__ uint32_t s_min[kRefitBlock][2];   // their smallest original ids
  __shared__ uint32_t s_far[kRefitBlock][2];   // their far ends (kInvalid: not arrived)
  __shared__ uint32_t s_arrive[kRefitBlock];
  const int64_t first = (int64_t)blockIdx.x * kRefitBlock;
  const int64_t last = first + kRefitBlock - 1 < nc - 1 ? first + kRefitBlock - 1 : nc - 1;
  for (int t = threadIdx.x; t <= kRefitBlock; t += blockDim.x)
    s_delta[t] = prefix_delta(keys, keys_hi, nc, leaf, first - 1 + t, first + t);
  s_arrive[threadIdx.x] = 0u;
  s_far[threadIdx.x][0] = s_far[threadIdx.x][1] = kInvalid;
  __syncthreads();
  const int64_t k = first + threadIdx.x;  // this thread's chunk
  if (k <= last) {
    float box[6];
    uint32_t idmin;
    chunk_box(pts, n, leaf, k, box, idmin);
    int64_t l = k, r = k;
    uint32_t ps;
    int side;
    bool up = parent_split(l, r, nc, s_delta[l - first], s_delta[r - first + 1], ps, side);
    while (up) {
      const uint32_t far = side == 0 ? (uint32_t)l : (uint32_t)r;
      if ((int64_t)ps < first || (int64_t)ps >= last) {
        // a split at the CTA's edge: its other child lies (partly) in another CTA
        reinterpret_cast<uint32_t *>(split_far + ps)[side] = far;
        if ((add_acq_rel_gpu(arrivals + ps, 1u) & 1u) != 0u) {  // second: list it
          const uint32_t at = atomicAdd(ready_count, 1u);
          if (at < capacity) ready[at] = ps;
          else atomicOr(status, kErrChain);  // cannot happen (see launch_build_tree)
        }
        break;
      }
      const int j = (int)(ps - first);
#pragma unroll
      for (int t = 0; t < 6; ++t) s_box[j][side][t] = box[t];
      s_min[j][side] = idmin;
      s_far[j][side] = far;
      if (add_acq_rel_cta_shared(&s_arrive[j], 1u) == 0u) break;  // first: the sibling carries on
      float sib[6];
#pragma unroll
      for (int t = 0; t < 6; ++t) sib[t] = s_box[j][side ^ 1][t];
      const uint32_t sibmin = s_min[j][side ^ 1], sibfar = s_far[j][side ^ 1];
      if (side == 0 ? (sibfar <= ps || (int64_t)sibfar > last) : ((int64_t)sibfar < first || sibfar > ps)) {
        atomicOr(status, kErrChain);  // cannot happen: the sibling lies in this CTA
        break;
      }
      // the parent covers [L, R] with split ps; which side it hangs on gives its index
      const int64_t L = side == 0 ? l : (int64_t)sibfar, R = side == 0 ? (int64_t)sibfar : r;
      uint32_t ps2;
      int side2;
      up = parent_split(L, R, nc, s_delta[L - first], s_delta[R - first + 1], ps2, side2);
      const uint32_t idx = node_index(L, R, !up, side2);
      if (side == 0)
        write_node(nodes, nlabels, range, idx, (uint32_t)L, ps, (uint32_t)R, box, sib, idmin, sibmin, n,
                   leaf, box, idmin);
      else
        write_node(nodes, nlabels, range, idx, (uint32_t)L, ps, (uint32_t)R, sib, box, sibmin, idmin, n,
                   leaf, box, idmin);
      l = L;
      r = R;
      ps = ps2;
      side = side2;
    }
  }
  __syncthreads();
  // a split inside the CTA that one child reached: the other spans CTAs and
  // arrives in k_build_up, which finds this one's far end in split_far
  const int64_t s = first + threadIdx.x;
  if (s < last && s_arrive[threadIdx.x] == 1u) {
    const int side = s_far[threadIdx.x][0] != kInvalid ? 0 : 1;
    reinterpret_cast<uint32_t *>(split_far + s)[side] = s_far[threadIdx.x][side];
    arrivals[s] = 1u;
  }
}

__global__ void __launch_bounds__(kRefitUpBlock) k_build_up(
    const uint64_t *__restrict__ keys, const uint64_t *__restrict__ keys_hi,
    const float4 *__restrict__ pts, int64_t n, int64_t nc, int leaf, NodeRec *nodes,
    uint2 *__restrict__ nlabels, uint2 *__restrict__ range, uint2 *split_far, uint32_t *arrivals,
    const uint32_t *__restrict__ ready, const uint32_t *ready_count, uint32_t capacity,
    uint32_t *status) {
  const uint32_t count = min(*ready_count, capacity);
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < count; t += gridDim.x * blockDim.x) {
    // a split both of whose children k_build_local finished
    uint32_t ps = __ldg(ready + t);
    const uint2 fe = __ldcg(split_far + ps);
    if (fe.x > ps || fe.y <= ps || (int64_t)fe.y >= nc) {  // cannot happen: both children arrived
      atomicOr(status, kErrChain);
      continue;
    }
    float box[6], sib[6];
    uint32_t idmin, sibmin;
    child_box(pts, n, leaf, nodes, ps, fe.x == ps, box, idmin);
    child_box(pts, n, leaf, nodes, ps + 1u, fe.y == ps + 1u, sib, sibmin);
    int64_t L = fe.x, R = fe.y;
    int side = 0;  // the child whose box is in `box`
    while (true) {
      uint32_t ps2;
      int side2;
      const bool up = parent_split(L, R, nc, prefix_delta(keys, keys_hi, nc, leaf, L - 1, L),
                                   prefix_delta(keys, keys_hi, nc, leaf, R, R + 1), ps2, side2);
      const uint32_t idx = node_index(L, R, !up, side2);
      if (side == 0)
        write_node(nodes, nlabels, range, idx, (uint32_t)L, ps, (uint32_t)R, box, sib, idmin, sibmin, n,
                   leaf, box, idmin);
      else
        write_node(nodes, nlabels, range, idx, (uint32_t)L, ps, (uint32_t)R, sib, box, sibmin, idmin, n,
                   leaf, box, idmin);
      if (!up) break;
      // arrive at the parent's split; the record just written is released with the add
      ps = ps2;
      side = side2;
      const uint32_t far = side == 0 ? (uint32_t)L : (uint32_t)R;
      reinterpret_cast<uint32_t *>(split_far + ps)[side] = far;
      if ((add_acq_rel_gpu(arrivals + ps, 1u) & 1u) == 0u) break;  // first: the sibling carries on
      const uint32_t sibfar = __ldcg(reinterpret_cast<const uint32_t *>(split_far + ps) + (side ^ 1));
      if (side == 0 ? (sibfar <= ps || (int64_t)sibfar >= nc) : sibfar > ps) {  // cannot happen
        atomicOr(status, kErrChain);
        break;
      }
      const uint32_t sidx = side == 0 ? ps + 1u : ps;  // the sibling's index or leaf chunk
      const bool sleaf = side == 0 ? sibfar == ps + 1u : sibfar == ps;
      child_box(pts, n, leaf, nodes, sidx, sleaf, sib, sibmin);
      if (side == 0) R = sibfar;
      else L = sibfar;
    }
  }
}

void launch_build_tree(Problem &P) {
  // A listed split has both children inside CTAs of k_build_local but lies at
  // the edge of one, so it is the boundary between two: fewer listed splits
  // than k_build_local has CTAs.  list_buf[1] (n entries) is free until the
  // rounds.
  uint32_t *ready = P.list_buf[1];
  uint32_t *ready_count = P.counters + kRefitReadyCounter;
  uint2 *split_far = P.split_far;
  cudaMemsetAsync(ready_count, 0, sizeof(uint32_t), P.stream);
  const int64_t ctas = grid_for(P.nc, kRefitBlock);
  k_build_local<<<(unsigned)ctas, kRefitBlock, 0, P.stream>>>(
      P.keys[0] /*sorted*/, P.code_hi, P.pts, P.n, P.nc, P.leaf, P.nodes, P.nlabels, P.range, split_far,
      P.arrivals, ready, ready_count, (uint32_t)P.n, P.counters + 1);
  int64_t g = ctas / kRefitUpBlock + 1;
  if (g > (int64_t)sm_count() * 16) g = (int64_t)sm_count() * 16;
  k_build_up<<<(unsigned)g, kRefitUpBlock, 0, P.stream>>>(
      P.keys[0], P.code_hi, P.pts, P.n, P.nc, P.leaf, P.nodes, P.nlabels, P.range, split_far,
      P.arrivals, ready, ready_count, (uint32_t)P.n, P.counters + 1);
  P.launches += 2;
}

}  // namespace emst

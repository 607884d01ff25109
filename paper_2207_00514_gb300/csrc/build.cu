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
// A4 (b). Hierarchy: Karras's fully parallel binary radix tree.  Its leaves are
// chunks of `leaf` consecutive sorted points (leaf = 1: one point per leaf);
// chunk c's key is the code of its first point, augmented by c so equal codes
// still split.  Internal node i covers a chunk range with one end at i; its
// split gamma gives the children gamma (left) and gamma+1 (right), leaves when
// the range ends there.  This is the numbering drawn in Fig. 4.
// ---------------------------------------------------------------------------
// kh != nullptr: 128-bit codes, kh their high words (the augmented key is
// then (high, low, position), 160 bits)
__device__ __forceinline__ int prefix_delta(const uint64_t *__restrict__ k,
                                            const uint64_t *__restrict__ kh, int64_t nc, int leaf,
                                            int64_t i, int64_t j) {
  if (j < 0 || j >= nc) return -1;
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

__global__ void __launch_bounds__(kBlock) k_hierarchy(const uint64_t *__restrict__ keys,
                                                      const uint64_t *__restrict__ keys_hi,
                                                      int64_t nc, int leaf,
                                                      uint32_t *__restrict__ parent_leaf,
                                                      uint2 *__restrict__ up_delta,
                                                      uint2 *__restrict__ range) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nc - 1) return;
  int d = (prefix_delta(keys, keys_hi, nc, leaf, i, i + 1) - prefix_delta(keys, keys_hi, nc, leaf, i, i - 1)) > 0 ? 1 : -1;
  int dmin = prefix_delta(keys, keys_hi, nc, leaf, i, i - d);
  int64_t lmax = 2;
  while (prefix_delta(keys, keys_hi, nc, leaf, i, i + lmax * d) > dmin) lmax <<= 1;
  int64_t l = 0;
  for (int64_t t = lmax >> 1; t >= 1; t >>= 1)
    if (prefix_delta(keys, keys_hi, nc, leaf, i, i + (l + t) * d) > dmin) l += t;
  int64_t j = i + l * d;
  int dnode = prefix_delta(keys, keys_hi, nc, leaf, i, j);
  int64_t s = 0, t = l;
  do {
    t = (t + 1) >> 1;
    if (prefix_delta(keys, keys_hi, nc, leaf, i, i + (s + t) * d) > dnode) s += t;
  } while (t > 1);
  int64_t gamma = i + s * d + (d < 0 ? -1 : 0);
  int64_t lo = i < j ? i : j, hi = i < j ? j : i;
  uint32_t left = (lo == gamma) ? (kLeafBit | (uint32_t)gamma) : (uint32_t)gamma;
  uint32_t right = (hi == gamma + 1) ? (kLeafBit | (uint32_t)(gamma + 1)) : (uint32_t)(gamma + 1);
  range[i] = pack_range((uint32_t)i, (uint32_t)lo, (uint32_t)gamma, (uint32_t)hi);
  reinterpret_cast<uint32_t *>(up_delta + i)[1] = (uint32_t)dnode;
  uint32_t up = (uint32_t)i << 1;
  if (left & kLeafBit) parent_leaf[left & ~kLeafBit] = up;
  else reinterpret_cast<uint32_t *>(up_delta + left)[0] = up;
  if (right & kLeafBit) parent_leaf[right & ~kLeafBit] = up | 1u;
  else reinterpret_cast<uint32_t *>(up_delta + right)[0] = up | 1u;
  if (i == 0) reinterpret_cast<uint32_t *>(up_delta)[0] = kInvalid;
}

void launch_hierarchy(Problem &P) {
  k_hierarchy<<<grid_for(P.nc - 1, kBlock), kBlock, 0, P.stream>>>(
      P.keys[0] /*sorted*/, P.code_hi, P.nc, P.leaf, P.parent_leaf, P.up_delta, P.range);
  P.launches += 1;
}

// ---------------------------------------------------------------------------
// A4 (c). Refit: bottom-up boxes, in two launches.
// k_refit: one thread per leaf chunk computes the box of its points and
// climbs the nodes whose leaf range lies inside its CTA's chunks: both
// arrivals at such a node come from this CTA, so both child boxes meet in
// shared memory and the arrivals are counted there with block-scope
// acquire-release adds; at every node the first arriver stops, the second
// merges the two child boxes, writes the node's whole record once (both
// boxes and the child references from the node's range) and its child
// labels, and carries the union one level up.  The first node spanning
// CTAs ends the climb: the thread leaves its box in its slot of that node's
// global record and adds a device-scope acquire-release arrival; the second
// arriver lists the node for the next launch.
// k_refit_up: one thread per listed node (both child boxes in its record)
// writes it and climbs on in global memory, first arriver stopping, as
// above.  (In one launch the threads that climb above their CTA's nodes --
// one or two per CTA, up to the root's depth -- would hold their CTA's
// slot while its other threads are long done.)
// The global counters are never reset: each pass adds exactly two arrivals
// per node, so the parity of the count before the add tells first from
// second.
// Each record also carries the smallest original id of each child's points
// (the traversal's tie pruning).
// The child labels are the round-0 ones (a one-point chunk k: label k;
// otherwise several components, kInvalid); a caller with other labels
// rewrites them (A5).
// ---------------------------------------------------------------------------
#ifndef EMST_REFIT_BLOCK
#define EMST_REFIT_BLOCK 128
#endif
constexpr int kRefitBlock = EMST_REFIT_BLOCK;  // leaf chunks per refit CTA
constexpr int kRefitUpBlock = 128;
constexpr uint32_t kRefitReadyCounter = 48;  // P.counters slot: nodes listed by k_refit

__device__ __forceinline__ void store_slot_box(NodeRec *rec, int slot, const float *bx) {
  float2 *f = reinterpret_cast<float2 *>(rec) + 3 * slot;
  f[0] = make_float2(bx[0], bx[1]);
  f[1] = make_float2(bx[2], bx[3]);
  f[2] = make_float2(bx[4], bx[5]);
}

__device__ __forceinline__ void load_slot_box(const NodeRec *rec, int slot, float *bx) {
  const float2 *f = reinterpret_cast<const float2 *>(rec) + 3 * slot;
#pragma unroll
  for (int t = 0; t < 3; ++t) {
    const float2 v = __ldcg(f + t);
    bx[2 * t] = v.x;
    bx[2 * t + 1] = v.y;
  }
}

// Arrival counters of the refit with acquire-release order: the first
// arriver's box stores are released by its add, and the second arriver's add
// acquires them, so no separate fences are needed around the add.
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

// Node `node` with range r and both child boxes L, R (and their smallest
// original ids): its whole record (boxes, references -- leaves where the
// range ends at the split -- and the round-0 child labels); returns the
// union in `box` / `idmin`.
__device__ __forceinline__ void write_node(NodeRec *nodes, uint2 *__restrict__ nlabels, uint32_t node,
                                           const NodeRange &r, const float *L, const float *R,
                                           uint32_t minL, uint32_t minR, int64_t n, int leaf,
                                           float *box, uint32_t &idmin) {
  const uint32_t g = r.split;
  const bool lleaf = r.first == g, rleaf = r.last == g + 1u;
  // a chunk of exactly one point is its own component in round 0
  auto one_point = [&](int64_t c) { return n - c * leaf == 1 || leaf == 1; };
  NodeRec rec;
  rec.a = make_float4(L[0], L[1], L[2], L[3]);
  rec.b = make_float4(L[4], L[5], R[0], R[1]);
  rec.c = make_float4(R[2], R[3], R[4], R[5]);
  rec.d = make_uint4(lleaf ? (kLeafBit | g) : g, rleaf ? (kLeafBit | (g + 1u)) : g + 1u, minL, minR);
  nodes[node] = rec;
  nlabels[node] = make_uint2(lleaf && one_point(g) ? (uint32_t)((int64_t)g * leaf) : kInvalid,
                             rleaf && one_point(g + 1) ? (uint32_t)((int64_t)(g + 1) * leaf) : kInvalid);
#pragma unroll
  for (int t = 0; t < 3; ++t) {
    box[t] = fminf(L[t], R[t]);
    box[3 + t] = fmaxf(L[3 + t], R[3 + t]);
  }
  idmin = min(minL, minR);
}

__global__ void __launch_bounds__(kRefitBlock) k_refit(const float4 *__restrict__ pts, int64_t n,
                                                  int64_t nc, int leaf, NodeRec *nodes,
                                                  uint2 *__restrict__ nlabels,
                                                  const uint32_t *__restrict__ parent_leaf,
                                                  const uint2 *__restrict__ up_delta,
                                                  const uint2 *__restrict__ range,
                                                  uint32_t *arrivals, uint32_t *__restrict__ ready,
                                                  uint32_t *ready_count, uint32_t capacity,
                                                  uint32_t *status) {
  __shared__ float s_box[kRefitBlock][2][6];  // both child boxes of each local node
  __shared__ uint32_t s_min[kRefitBlock][2];  // and their smallest original ids
  __shared__ uint32_t s_arrive[kRefitBlock];
  const int64_t first = (int64_t)blockIdx.x * kRefitBlock;
  const int64_t last = first + kRefitBlock - 1;
  s_arrive[threadIdx.x] = 0u;
  __syncthreads();
  const int64_t k = first + threadIdx.x;  // this thread's chunk
  if (k >= nc) return;
  const int64_t p0 = k * leaf, p1 = p0 + leaf < n ? p0 + leaf : n;
  float4 p = pts[p0];
  float box[6] = {p.x, p.y, p.z, p.x, p.y, p.z};
  uint32_t idmin = __float_as_uint(p.w);
  for (int64_t m = p0 + 1; m < p1; ++m) {
    p = pts[m];
    box[0] = fminf(box[0], p.x); box[1] = fminf(box[1], p.y); box[2] = fminf(box[2], p.z);
    box[3] = fmaxf(box[3], p.x); box[4] = fmaxf(box[4], p.y); box[5] = fmaxf(box[5], p.z);
    idmin = min(idmin, __float_as_uint(p.w));
  }
  uint32_t up = parent_leaf[k];
  while (true) {
    const uint32_t node = up >> 1;
    const int slot = (int)(up & 1u);
    // both depend on the node only: one round trip per level
    const NodeRange r = unpack_range(node, __ldg(range + node));
    const uint32_t up_next = __ldg(&up_delta[node].x);
    if ((int64_t)r.first < first || (int64_t)r.last > last) {
      // spans CTAs: leave the box for the sibling or for k_refit_up
      store_slot_box(&nodes[node], slot, box);
      reinterpret_cast<uint32_t *>(&nodes[node].d)[2 + slot] = idmin;
      const uint32_t before = add_acq_rel_gpu(&arrivals[node], 1u);
      if ((before & 1u) != 0u) {
        const uint32_t at = atomicAdd(ready_count, 1u);
        if (at < capacity) ready[at] = node;
        else atomicOr(status, kErrChain);  // cannot happen (see launch_refit)
      }
      return;
    }
#pragma unroll
    for (int t = 0; t < 6; ++t) s_box[node - first][slot][t] = box[t];
    s_min[node - first][slot] = idmin;
    if (add_acq_rel_cta_shared(&s_arrive[node - first], 1u) == 0u) return;  // first: the sibling carries on
    float sib[6];
#pragma unroll
    for (int t = 0; t < 6; ++t) sib[t] = s_box[node - first][slot ^ 1][t];
    const uint32_t sibmin = s_min[node - first][slot ^ 1];
    if (slot == 0) write_node(nodes, nlabels, node, r, box, sib, idmin, sibmin, n, leaf, box, idmin);
    else write_node(nodes, nlabels, node, r, sib, box, sibmin, idmin, n, leaf, box, idmin);
    if (node == 0) return;
    up = up_next;
  }
}

__global__ void __launch_bounds__(kRefitUpBlock) k_refit_up(int64_t n, int leaf, NodeRec *nodes,
                                                       uint2 *__restrict__ nlabels,
                                                       const uint2 *__restrict__ up_delta,
                                                       const uint2 *__restrict__ range,
                                                       uint32_t *arrivals,
                                                       const uint32_t *__restrict__ ready,
                                                       const uint32_t *ready_count, uint32_t capacity) {
  const uint32_t count = min(*ready_count, capacity);
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < count; t += gridDim.x * blockDim.x) {
    uint32_t node = __ldg(ready + t);
    float box[6], sib[6];
    uint32_t idmin, sibmin;
    // both children arrived in k_refit: both boxes are in the record
    load_slot_box(&nodes[node], 0, box);
    load_slot_box(&nodes[node], 1, sib);
    idmin = __ldcg(reinterpret_cast<const uint32_t *>(&nodes[node].d) + 2);
    sibmin = __ldcg(reinterpret_cast<const uint32_t *>(&nodes[node].d) + 3);
    int slot = 0;
    while (true) {
      const NodeRange r = unpack_range(node, __ldg(range + node));
      if (slot == 0) write_node(nodes, nlabels, node, r, box, sib, idmin, sibmin, n, leaf, box, idmin);
      else write_node(nodes, nlabels, node, r, sib, box, sibmin, idmin, n, leaf, box, idmin);
      if (node == 0) break;
      const uint32_t up = __ldg(&up_delta[node].x);
      node = up >> 1;
      slot = (int)(up & 1u);
      store_slot_box(&nodes[node], slot, box);
      reinterpret_cast<uint32_t *>(&nodes[node].d)[2 + slot] = idmin;
      const uint32_t before = add_acq_rel_gpu(&arrivals[node], 1u);
      if ((before & 1u) == 0u) break;  // first: the sibling carries on
      load_slot_box(&nodes[node], slot ^ 1, sib);
      sibmin = __ldcg(reinterpret_cast<const uint32_t *>(&nodes[node].d) + 2 + (slot ^ 1));
    }
  }
}

void launch_refit(Problem &P) {
  // A listed node has both children inside CTAs of k_refit but spans two,
  // so it splits at the boundary between them: fewer listed nodes than
  // k_refit has CTAs.  list_buf[1] (n entries) is free until the rounds.
  uint32_t *ready = P.list_buf[1];
  uint32_t *ready_count = P.counters + kRefitReadyCounter;
  cudaMemsetAsync(ready_count, 0, sizeof(uint32_t), P.stream);
  k_refit<<<grid_for(P.nc, kRefitBlock), kRefitBlock, 0, P.stream>>>(P.pts, P.n, P.nc, P.leaf, P.nodes,
                                                          P.nlabels, P.parent_leaf, P.up_delta, P.range,
                                                          P.arrivals, ready, ready_count,
                                                          (uint32_t)P.n, P.counters + 1);
  int64_t g = grid_for(P.nc, kRefitBlock) / kRefitUpBlock + 1;
  if (g > (int64_t)sm_count() * 16) g = (int64_t)sm_count() * 16;
  k_refit_up<<<(unsigned)g, kRefitUpBlock, 0, P.stream>>>(P.n, P.leaf, P.nodes, P.nlabels, P.up_delta,
                                                          P.range, P.arrivals, ready, ready_count,
                                                          (uint32_t)P.n);
  P.launches += 2;
}

}  // namespace emst

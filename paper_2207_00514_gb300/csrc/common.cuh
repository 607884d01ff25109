// common.cuh -- types, device helpers and kernel launchers shared by the
// translation units of libemst.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/emst.h"

namespace emst {

constexpr uint32_t kInvalid = 0xFFFFFFFFu;   // no label / no neighbour
constexpr uint32_t kLeafBit = 0x80000000u;   // child reference of a leaf
constexpr uint32_t kNoBound = 0xFFFFFFFFu;   // "+inf" in the u32 radius arrays
constexpr uint64_t kEmptyKey = ~0ull;        // empty per-component minimum

// The minimum outgoing edge of a component (A8) as one 128-bit key, ordered
// as the pair (key, mx): key = (w bits << 32) | min original id (w >= 0, so
// float bits order as unsigned), mx = (max original id << 32) | the label of
// the edge's endpoint outside the component (fixed by the edge, so it never
// decides the order).  Its lexicographic minimum is the (w, min id, max id)
// minimum of §2's tie-break.  All ones = no edge yet.
struct __align__(16) CompBest {
  uint64_t mx;
  uint64_t key;
};
static_assert(sizeof(CompBest) == 16, "one 128-bit key per component");

// Error bits of the device status word.
enum : uint32_t {
  kErrNonFinite = 1u << 0,
  kErrStack = 1u << 1,
  kErrSpin = 1u << 2,
  kErrChain = 1u << 3,
  kErrBadInput = 1u << 4,  // an input found invalid on the device (dendrogram)
  kErrCas = 1u << 5,       // a compare-and-swap loop gave up (bounded retries)
};

// One internal node of the hierarchy, 64 bytes.  The boxes of both children
// travel with the parent, so a query visiting the node tests both children
// with one record load (Algorithm 2, the loop over children).  Child labels
// (Optimization 1) are rewritten every round, so they live beside the record
// (nlabels, 8 bytes per node): the round's pass writes whole sectors.
//   f[0..5]   left child box  (lo x,y,z, hi x,y,z)
//   f[6..11]  right child box
//   u[12..13] child references (leaf k: kLeafBit|k; internal node: its index)
//   u[14..15] smallest original id among each child's points (a child whose
//             weight bound only ties the cutoff can win the tie only below it)
struct __align__(16) NodeRec {
  float4 a, b, c;
  uint4 d;
};
static_assert(sizeof(NodeRec) == 64, "node record must be 64 bytes");

// ---------------------------------------------------------------------------
// The edge weight of the method: FP32 squared distance in a fixed fma order,
// every step rounded explicitly (no contraction freedom left to the compiler).
// 2D runs with z = 0 everywhere: fma(0, 0, s) == s exactly.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float sq_dist(float px, float py, float pz, float qx, float qy,
                                         float qz) {
  float dx = __fsub_rn(px, qx);
  float dy = __fsub_rn(py, qy);
  float dz = __fsub_rn(pz, qz);
  float s = __fmul_rn(dx, dx);
  s = __fmaf_rn(dy, dy, s);
  s = __fmaf_rn(dz, dz, s);
  return s;
}

// Lower bound of sq_dist from p to any point of the box [lo, hi]: the same
// order on p - clamp(p, lo, hi).  Per dimension |p - clamp| <= |p - q| for q in
// the box, rounding is monotone and mul / fma are monotone in non-negative
// operands, so the bound never exceeds the weight to a point inside; for a
// degenerate box (a leaf: lo == hi == q) it IS the weight to q.
__device__ __forceinline__ float box_dist(float px, float py, float pz, float lx, float ly,
                                          float lz, float hx, float hy, float hz) {
  float cx = fminf(fmaxf(px, lx), hx);
  float cy = fminf(fmaxf(py, ly), hy);
  float cz = fminf(fmaxf(pz, lz), hz);
  return sq_dist(px, py, pz, cx, cy, cz);
}

__device__ __forceinline__ float bound_to_radius(uint32_t b) {
  return b == kNoBound ? __int_as_float(0x7f800000) : __uint_as_float(b);
}

// Order-preserving map float -> uint32 (for atomic min/max of floats).
__device__ __forceinline__ uint32_t float_to_ordered(float f) {
  uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float ordered_to_float(uint32_t o) {
  uint32_t u = (o & 0x80000000u) ? (o & 0x7FFFFFFFu) : ~o;
  return __uint_as_float(u);
}

__device__ __forceinline__ uint32_t ld_cg_u32(const uint32_t *p) { return __ldcg(p); }

// ---------------------------------------------------------------------------
// Z-curve quantisation (decided in FP32, the same everywhere it is used):
// B = 21 bits per dimension in 3D, 32 in 2D; s = 2^B / (hi - lo) (0 for a
// flat dimension); t = (x - lo) * s; q = t >= 2^B ? 2^B - 1 : max(t, 0)
// truncated.  Monotone non-decreasing in x.  Bits interleave x (most
// significant), y, z.
// ---------------------------------------------------------------------------
struct Quantizer {
  float lo[3];
  float s[3];
  float twoB;
  uint32_t qmax;
};

// Bits per dimension of the codes: 21 in 3D and 32 in 2D, fewer when the top
// bits carry an instance id.
__host__ __device__ __forceinline__ int code_bits(int dim, int inst_bits) {
  const int b = (64 - inst_bits) / dim;
  return dim == 3 ? (b < 21 ? b : 21) : (b < 32 ? b : 32);
}

__device__ __forceinline__ Quantizer make_quantizer(const uint32_t *box, int dim, int bits) {
  Quantizer Q;
  Q.twoB = __uint_as_float((uint32_t)(127 + bits) << 23);  // 2^bits exactly
  Q.qmax = bits >= 32 ? 0xffffffffu : ((1u << bits) - 1u);
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    Q.lo[d] = 0.f;
    Q.s[d] = 0.f;
    if (d < dim) {
      float lo = ordered_to_float(box[d]);
      float hi = ordered_to_float(box[3 + d]);
      float ext = __fsub_rn(hi, lo);
      Q.lo[d] = lo;
      Q.s[d] = ext > 0.0f ? __fdiv_rn(Q.twoB, ext) : 0.0f;
    }
  }
  return Q;
}

__device__ __forceinline__ uint32_t quantize(const Quantizer &Q, int d, float x) {
  float t = __fmul_rn(__fsub_rn(x, Q.lo[d]), Q.s[d]);
  return (t >= Q.twoB) ? Q.qmax : (t > 0.0f ? (uint32_t)t : 0u);
}

__device__ __forceinline__ uint64_t spread3(uint64_t x) {
  x &= 0x1fffffull;
  x = (x | (x << 32)) & 0x1f00000000ffffull;
  x = (x | (x << 16)) & 0x1f0000ff0000ffull;
  x = (x | (x << 8)) & 0x100f00f00f00f00full;
  x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
  x = (x | (x << 2)) & 0x1249249249249249ull;
  return x;
}

__device__ __forceinline__ uint64_t spread2(uint64_t x) {
  x &= 0xffffffffull;
  x = (x | (x << 16)) & 0x0000ffff0000ffffull;
  x = (x | (x << 8)) & 0x00ff00ff00ff00ffull;
  x = (x | (x << 4)) & 0x0f0f0f0f0f0f0f0full;
  x = (x | (x << 2)) & 0x3333333333333333ull;
  x = (x | (x << 1)) & 0x5555555555555555ull;
  return x;
}

__device__ __forceinline__ uint64_t interleave(uint32_t qx, uint32_t qy, uint32_t qz, int dim) {
  return dim == 3 ? ((spread3(qx) << 2) | (spread3(qy) << 1) | spread3(qz))
                  : ((spread2(qx) << 1) | spread2(qy));
}

// ---------------------------------------------------------------------------
// Scratch layout of one EMST problem (carved from one allocation).
// ---------------------------------------------------------------------------
// An internal node's leaf-chunk range [first, last] and split, in 8 bytes.
// In the hierarchy's numbering one end of a node's range is the node's own
// index, so only the other end is stored, with bit 31 set when that other
// end is `first` (the node is the range's last chunk).  Chunk indices are
// below 2^31.
struct NodeRange {
  uint32_t first, split, last;
};
__host__ __device__ __forceinline__ uint2 pack_range(uint32_t node, uint32_t first, uint32_t split,
                                                     uint32_t last) {
  return make_uint2(first == node ? last : (first | 0x80000000u), split);
}
__host__ __device__ __forceinline__ NodeRange unpack_range(uint32_t node, uint2 e) {
  NodeRange r;
  const uint32_t other = e.x & 0x7FFFFFFFu;
  const bool node_is_last = (e.x >> 31) != 0u;
  r.first = node_is_last ? other : node;
  r.last = node_is_last ? node : other;
  r.split = e.y;
  return r;
}

struct Problem {
  int64_t n = 0;
  int dim = 3;
  int leaf = 1;      // points per leaf chunk of the hierarchy
  int64_t nc = 0;    // leaf chunks: ceil(n / leaf)

  // Batched form: num_inst independent instances, instance I = input rows
  // [offsets[I], offsets[I+1]); the instance id sits in the top `inst_bits`
  // bits of every code, so instance I is also curve positions
  // [offsets[I], offsets[I+1]) and one subtree of the hierarchy.  With one
  // instance all of this is off (null arrays, inst_bits 0).
  int64_t num_inst = 1;
  int inst_bits = 0;
  int64_t *offsets = nullptr;       // num_inst+1, device
  uint32_t *inst_in = nullptr;      // n: instance of each input row
  uint32_t *inst_of = nullptr;      // n: instance of each curve position
  uint32_t *inst_root = nullptr;    // num_inst: root node of each instance's subtree
  int64_t edges_expected = 0;       // sum over instances of max(n_I - 1, 0)
  int64_t largest = 0;              // points of the largest instance

  // Learned radius (optional): network parameters (device, EMST_MLP_PARAMS
  // floats), proposed cutoffs, the cutoffs used, component sizes and the
  // list of points to rerun.
  bool want_learned = false;         // set before layout(): carve the learned-radius arrays
  bool want_logging = false;         // set before layout(): carve the logging counter
  bool want_mrd = false;             // set before layout(): carve the core distances
  bool wide = false;                 // set before layout(): 128-bit Morton codes
  bool auto_wide = false;            // set before layout(): 64-bit codes unless they leave more
                                     // than n/64 distinct points sharing a code (then 128)
  int64_t code_collisions = 0;       // that count, when measured
  bool persistent = false;           // A7 by the persistent work-queue kernel
  int refill_lanes = 0;              // its refill threshold (0: default)
  int queue_chunk = 0;               // its queue chunk per warp (0: default)
  int block = 0;                     // one-thread-per-point traversal CTA size (0: default)
  bool graph_round = false;          // run_round is being captured as a graph body
  bool want_count = false;           // set before layout(): carve the visited-node bitmap
  uint32_t *seen = nullptr;          // count runs: bitmap of the internal nodes visited this round
  bool ties = true;                  // the search needs its tie rule (a run of > 32 equal
                                     // codes exists; set after the build, true when unknown)
  const float *mlp = nullptr;
  float *pred_r = nullptr;
  float *r_used = nullptr;
  uint32_t *comp_size = nullptr;
  uint32_t *rerun_list = nullptr;
  // Logging of training pairs (optional).
  float *log_feat = nullptr;
  float *log_target = nullptr;
  int64_t log_capacity = 0;
  int log_every = 1;
  unsigned long long *log_count = nullptr;
  cudaStream_t stream = nullptr;

  const float *points = nullptr;  // n x dim, device
  const float *points_mapped = nullptr;  // a pinned host input through its device mapping: the
                                         // scene-box pass reads it and writes `points`
  float4 *pts = nullptr;          // n, curve order, .w = original index bits
  uint64_t *keys[2] = {nullptr, nullptr};
  uint32_t *vals[2] = {nullptr, nullptr};
  uint32_t *perm = nullptr;       // curve index -> original index
  uint64_t *wide_hi = nullptr;    // n: 128-bit codes, high / low words in input order
  uint64_t *wide_lo = nullptr;
  const uint64_t *code_hi = nullptr;  // sorted high words during the build (128-bit codes),
                                      // else nullptr; the sorted low words are keys[0]
  NodeRec *nodes = nullptr;       // nc-1 internal nodes
  uint2 *nlabels = nullptr;       // nc-1: child labels of each internal node (A5)
  uint2 *split_far = nullptr;        // nc-1: per split of the build, the far end of the left
                                     //      and of the right child that reached it
  uint32_t *arrivals = nullptr;      // nc-1 arrival counters of the splits (parity = who is second)
  uint2 *range = nullptr;            // nc-1: each internal node's leaf-chunk range [first, last]
                                     //      and split (the last chunk of its left child), packed
                                     //      by pack_range (one end of the range is the node itself)
  uint32_t *runs = nullptr;          // n: per 32 curve positions, the bitmap of their label
                                     //    boundaries and the count of boundaries before them
                                     //    within their scan tile (plus the tile's entry of
                                     //    tile_prefix): 8 bytes, 256-B aligned
  uint32_t *scan_tiles = nullptr;    // 2 x scan tiles: boundary total of each tile, then the
                                     //    exclusive prefix of those totals
  uint32_t *labels = nullptr;        // n, current round (= labels_buf[cur])
  uint32_t *bound = nullptr;         // n, FP32 bits of the component upper bound (= bound_buf[cur])
  uint32_t *labels_buf[2] = {nullptr, nullptr};
  uint32_t *bound_buf[2] = {nullptr, nullptr};
  int cur = 0;
  uint32_t *list_buf[2] = {nullptr, nullptr};  // active component labels, ping-pong
  uint32_t *active_list = nullptr;   // this round's active labels (nullptr: all n)
  uint32_t *next_list = nullptr;     // roots appended by the merge
  int64_t n_active = 0;
  uint2 *res = nullptr;              // n: (w bits, neighbour curve index)
  float *core2 = nullptr;            // n: mutual reachability -- squared core distances in
                                     //    curve order (nullptr: the Euclidean weight)
  // Per-component minimum edge (A8), indexed by label, ping-pong by round:
  // the merge of round r clears the other buffer's entries of its active
  // labels.
  CompBest *comp_buf[2] = {nullptr, nullptr};  // n
  CompBest *comp = nullptr;          // = comp_buf[cur]
  uint32_t *root = nullptr;          // n: new label of a component
  emst_edge *edges = nullptr;        // n: edges in emission order
  emst_edge *out_stage = nullptr;    // n-1: device staging of host outputs
  uint32_t *counters = nullptr;      // [0] edges emitted, [1] status bits, [2..3] node visits (u64),
                                     // [4..9] scene box (ordered), [10] long tie runs in the output, [28..29] identical curve neighbours (u64), [30..31] code collisions (u64), [32] a run of > 32 equal codes, [11] largest emitted
                                     // weight bits, [16..23] sort tile counters,
                                     // [12] next round's active components, [13] points
                                     // to rerun, [14..15] reruns / queries (learned radius),
                                     // [24] scan tiles finished, [34..35] queries that
                                     // searched (u64), [36..37] the work queue of the
                                     // persistent traversal (u64), [38..39] distinct internal
                                     // nodes visited (u64), [40] this round's active
                                     // components and [41] rounds done (graph rounds)
  uint32_t *count_dev = nullptr;     // graph rounds: counters + 40 (else nullptr)
  uint32_t *sort_hist = nullptr;     // 8 x 256
  uint32_t *sort_lookback = nullptr; // tiles x 256
  int64_t sort_tiles = 0;
  int launches = 0;
};

// ---------------------------------------------------------------------------
// Launchers (host side), one per kernel family.
// ---------------------------------------------------------------------------
// build.cu
void launch_scene_box(Problem &P);
void launch_morton(Problem &P);
void launch_morton128(Problem &P);
void launch_gather_u64(Problem &P, const uint64_t *src, const uint32_t *idx, uint64_t *out);
// also counts identical points and code collisions into counters[28..31] and
// flags long runs of equal codes in counters[32]
void launch_gather(Problem &P, const uint32_t *perm);
void launch_instance_ids(Problem &P);
void launch_instance_roots(Problem &P);
// A4: hierarchy, boxes, records, ranges and round-0 child labels in one
// bottom-up pass (P.arrivals zeroed first)
void launch_build_tree(Problem &P);
// sort.cu
// Tile shape of one sort pass (compile-time knobs; the defaults are the measured best).
#ifndef EMST_SORT_THREADS
#define EMST_SORT_THREADS 256
#endif
#ifndef EMST_SORT_ITEMS
#define EMST_SORT_ITEMS 12
#endif
#ifndef EMST_SORT_MIN_BLOCKS
#define EMST_SORT_MIN_BLOCKS 3
#endif
constexpr int kSortThreads = EMST_SORT_THREADS;
constexpr int kSortItems = EMST_SORT_ITEMS;
constexpr int kSortTile = kSortThreads * kSortItems;
int64_t sort_tiles_for(int64_t n);
// Stable LSD radix sort of (keys, vals) pairs on digits [digit_begin, digit_end)
// (8-bit digits).  Returns the index (0/1) of the buffers holding the result.
// Stable sort of (keys[src], vals[src]) by the bits [bit0 + 8 digit_begin,
// bit0 + 8 digit_end) of the keys (digit d of the key >> bit0 per pass);
// returns the buffer index holding the result.
int radix_sort_pairs(Problem &P, int64_t n, int digit_begin, int digit_end, int src, int bit0 = 0);
// rounds.cu
#ifndef EMST_TRAVERSE_MIN_BLOCKS
#define EMST_TRAVERSE_MIN_BLOCKS 8      // resident 256-thread CTAs the traversal's registers must allow (32 registers: measured best)
#endif
constexpr int kTraverseBlock = 128;     // default traversal CTA size (measured best)
constexpr int kTraverseMaxBlock = 256;  // largest the traversal kernels are compiled for
#ifndef EMST_PERSIST_BLOCK
#define EMST_PERSIST_BLOCK 128
#endif
constexpr int kPersistBlock = EMST_PERSIST_BLOCK;  // CTA size of the persistent traversal
int64_t scan_tiles_for(int64_t n);
void launch_label_runs(Problem &P);
void launch_node_labels(Problem &P);
void advance_round(Problem &P, int64_t n_active);
void launch_upper_bounds(Problem &P);
// mrd.cu: squared core distances (k-th nearest neighbour, §4.5) into P.core2
void launch_core_knn(Problem &P, int k);
void launch_core_to_input(Problem &P, float *out);
// first: the first round of the plain form (labels = curve indices);
// round: the round's number (-1: not known, as in graph rounds)
void launch_traverse(Problem &P, bool carried, const float *radius_in, int block, bool count,
                     bool seeded, int learned_pass = 0, bool first = false, int round = -1);
void launch_merge(Problem &P);
void launch_fill_u32(Problem &P, uint32_t *p, uint32_t v, int64_t count);
// count runs: adds the bits of the visited-node bitmap to counters[38..39]
// and clears it for the next round
void launch_count_seen(Problem &P);
// output
void launch_edge_keys_wi(Problem &P, int64_t m, int shift_i);
void launch_edge_ties(Problem &P, int64_t m, int src);
void launch_edge_ties_w(Problem &P, int64_t m, int src, int shift_i);
void launch_edge_from_keys(Problem &P, int64_t m, int src, int shift_i, int w_bits_used,
                           emst_edge *out);
void launch_edge_keys_inst_wi(Problem &P, int64_t m, int shift_w, int shift_i);
void launch_edge_keys_j(Problem &P, int64_t m);
void launch_edge_keys_wi_of(Problem &P, int64_t m, int src, int shift_i);
void launch_edge_keys_inst(Problem &P, int64_t m, int src);
// learned.cu
void launch_comp_sizes(Problem &P);
void launch_predict(Problem &P, bool carried);
void launch_rerun_mark(Problem &P);
void launch_log_samples(Problem &P, int round, bool carried);
void launch_edge_gather(Problem &P, int64_t m, const uint32_t *order, emst_edge *out);

// tuning.cu: the tuned traversal parameters for this device, dimension, form
// and size (0 in a field: no choice); false when the tuning file has none.
struct TuneChoice {
  int traversal = 0, block = 0, leaf = 0, refill = 0, chunk = 0;
};
bool lookup_tuning(int dim, bool batched, int64_t n, TuneChoice *out);

// api.cu: helpers of the orchestration
bool device_accessible(const void *p);
// The device address of page-locked (pinned) host memory that kernels can
// read and write directly (over the chip-to-chip link), else nullptr.
void *mapped_host(const void *p);
// Streaming multiprocessors of the current device (queried once per device):
// grid caps of grid-stride kernels are multiples of it.
int sm_count();
// Stream-ordered scratch from the library's pool on the current device
// (release with cudaFreeAsync on the same stream).
cudaError_t scratch_alloc(void **p, size_t bytes, cudaStream_t s);
// Lays the scratch of one problem out from `base` (nullptr: only measures);
// returns the bytes needed.
size_t layout(Problem &P, char *base, bool copy_points, bool copy_edges);
int status_from_bits(uint32_t bits);
int check_args(const float *points, int64_t n, int dim);
int bits_for(int64_t v);
void run_build(Problem &P);
void reset_round_state(Problem &P);
void run_round(Problem &P, int round, bool carried, int block, bool count);
// Leaf chunk size actually used for n points and a requested size (0 =
// default): a power of two, at most the request, leaving at least 2 chunks.
int effective_leaf(int64_t n, int requested);
int run_output(Problem &P, emst_edge *out, uint32_t w_bits);

inline int grid_for(int64_t n, int block) {
  int64_t g = (n + block - 1) / block;
  return (int)(g < 1 ? 1 : g);
}

}  // namespace emst

/*
 * emst.h -- C ABI of libemst.so: the single-tree Boruvka Euclidean minimum
 * spanning tree (EMST) of Prokopenko, Sao and Lebrun-Grandie (arXiv
 * 2207.00514) on one NVIDIA GB300 (sm_103a).
 *
 * The problem (§2, "EMST computation"): given n points in d dimensions, the
 * EMST is the minimum spanning tree of the complete graph whose edge (i, j)
 * weighs ||p_i - p_j||.  The method (§3, Fig. 3): build one bounding volume
 * hierarchy over the points, then repeat Boruvka rounds (Algorithm 1) until
 * one component is left; each round labels tree nodes by component
 * (Optimization 1), bounds each component's shortest outgoing edge from
 * curve-adjacent pairs (Optimization 2), runs one nearest-other-component
 * query per point (Algorithm 2), reduces the per-component minimum and merges
 * the chains of components (§3, "Merging components together").
 *
 * Conventions shared by every entry point:
 *  - points: row-major n x dim FP32, dim 2 or 3.  Pointers may be device
 *    memory or host memory (pinned or pageable); the library detects which.
 *  - edge weight: the FP32 squared distance w = fma(dz,dz, fma(dy,dy, dx*dx))
 *    with dx = x_i - x_j rounded to FP32 (2D: fma(dy,dy, dx*dx)).  Squaring
 *    keeps the order of lengths, so the tree is the EMST.
 *  - ties: edges compare by (w, min(i,j), max(i,j)), the tie-break of §2
 *    ("Boruvka's algorithm", last paragraph); under it the MST is unique.
 *  - output: exactly n-1 edges (i < j, original point indices), sorted by
 *    that same (w, i, j) order.
 *  - streams: `stream` is a cudaStream_t passed as void* (NULL = the legacy
 *    default stream).  Work is ordered on it; each call returns after that
 *    work has finished (it synchronises the stream once to read the status).
 *  - memory: the caller owns inputs and outputs.  Scratch memory is taken
 *    stream-ordered from a library-owned pool on the current device and
 *    returned to the pool before the call returns.
 *  - errors: every entry point returns an emst_status value; nothing traps
 *    or aborts.  Device-side failures (non-finite input, round limit, an
 *    internal guard) are read back from a status word at the end of the call.
 *  - limits: 0 <= n <= EMST_MAX_POINTS.  n = 0 or 1 gives 0 edges.
 */
#ifndef EMST_H_
#define EMST_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* One spanning-tree edge: original point indices i < j and the FP32 squared
 * distance w between them (12 bytes, no padding). */
typedef struct emst_edge {
  uint32_t i;
  uint32_t j;
  float w;
} emst_edge;

typedef enum emst_status {
  EMST_OK = 0,
  EMST_ERR_INVALID_ARG = -1, /* bad n, dim, null pointer, offsets, options */
  EMST_ERR_NONFINITE = -2,   /* a coordinate is NaN or infinite */
  EMST_ERR_OOM = -3,         /* scratch allocation failed */
  EMST_ERR_CUDA = -4,        /* a CUDA runtime call or launch failed */
  EMST_ERR_ROUND_LIMIT = -5, /* more Boruvka rounds than ceil(log2 n) (cannot happen for valid input) */
  EMST_ERR_INTERNAL = -6,    /* an internal device-side guard fired (bounded wait, stack) */
  EMST_ERR_TOO_LARGE = -7    /* n above EMST_NOALLOC_MAX_POINTS in emst_compute_noalloc */
} emst_status;

#define EMST_MAX_POINTS ((int64_t)1073741823) /* 2^30 - 1 */

/* Options for emst_compute_ex.  Zero-initialise, then set struct_size. */
typedef struct emst_options {
  int32_t struct_size;        /* sizeof(emst_options) */
  int32_t block_size;         /* traversal CTA size: 0 = default (128), else 64..256, multiple of 32 */
  int32_t carried_radius;     /* 1 (default if struct_size==0) = seed each query with the previous
                                 round's neighbour when it is still in another component */
  int32_t use_graph;          /* 1 = graph rounds: after the first round (run and checked from
                                 the host), every later round runs inside one CUDA graph whose
                                 while node repeats a two-round body until a one-thread kernel
                                 finds, on the device, all edges emitted, an error bit set or
                                 the round limit reached -- no host round trip per round.
                                 Captured on streams the library creates, launched on `stream`,
                                 instantiated per call.  Not with mlp_params or count_visits
                                 (those run the host loop); per-round traversal times then
                                 cover the first round only.  0 (default) = the host loop,
                                 one status read per round.  The tree is the same either way. */
  int32_t count_visits;       /* 1 = count node visits per round into emst_stats */
  int32_t leaf_size;          /* points per leaf chunk of the hierarchy: 0 = default (1, one
                                 point per leaf as in the paper), else 1, 2, 4, 8 or 16 (halved
                                 while fewer than 2 chunks remain).  Chunks are runs of
                                 consecutive curve positions; on clustered data they straddle
                                 the curve's jumps and search more, so 1 is the fastest there */
  const float *mlp_params;    /* learned search radius: the network (EMST_MLP_PARAMS floats,
                                 host or device memory; see emst_mlp_forward), or NULL for the
                                 plain method.  The tree is the same either way. */
  int32_t mrd_k;              /* mutual reachability (§4.5, the metric of HDBSCAN*): 0 or 1 =
                                 the Euclidean MST; 2 <= k <= EMST_MRD_MAX_K (and k <= n) = the
                                 MST under max(core(u), core(v), |u - v|), core(u) the distance
                                 from u to its k-th nearest neighbour counting u itself; edge
                                 weights are then FP32 squared mutual reachability distances,
                                 ordered and tie-broken like the Euclidean ones.  Not together
                                 with mlp_params. */
  int32_t morton_bits;        /* Z-curve code width: 64 (21 bits per axis in 3D, 32 in 2D,
                                 FP32 quantiser), 128 (42 / 64 bits per axis, FP64 quantiser:
                                 the finer grid §4.1 suggests for very dense data; one more
                                 8-pass sort) or 0 = automatic (the default): 64, rebuilt with
                                 128 when more than n/64 distinct points share their curve
                                 predecessor's 64-bit code.  The tree is the same either way. */
  int32_t traversal;          /* the Algorithm 2 kernel: 0 = default (one thread per point,
                                 the fastest measured), 1 = one thread per point, 2 = a
                                 persistent grid whose warps take queries from a global work
                                 queue and refill lanes as searches end (plain rounds on
                                 one-point leaves; other forms use one thread per point).
                                 The tree is the same either way. */
  int32_t refill_lanes;       /* traversal 2: idle lanes that trigger a refill, 1..32
                                 (0 = tuned or default 16) */
  int32_t queue_chunk;        /* traversal 2: curve positions a warp takes from the queue at
                                 a time, >= 32 (0 = tuned or default 64) */
  int32_t ignore_tuning;      /* 1 = do not read the tuning file (see below); 0 = block_size,
                                 leaf_size, traversal, refill_lanes and queue_chunk left at 0
                                 take the tuned values for this GPU, dimension and size */
  int32_t reserved[2];
} emst_options;

/* Tuning file.  emst_compute_ex / emst_compute_batched_ex (and the calls
 * without options) read, once per process, the file named by the
 * environment variable EMST_TUNING_FILE, else emst_tuning.txt beside
 * libemst.so.  Each line "gpu=<name> dim=<2|3> form=<single|batched>
 * nmin=<n> nmax=<n> traversal=<1|2> block=<b> leaf=<l> refill=<r> chunk=<c>"
 * (other keys ignored, '#' starts a comment) gives the parameters of calls on
 * a device of that name with nmin <= n < nmax points.  A missing or
 * unreadable file means defaults.  The file only chooses among exact
 * variants: the tree is the same whatever it says. */

#define EMST_MRD_MAX_K 32

/* Per-call statistics filled by emst_compute_ex when `stats` is not NULL
 * (struct_size must be at least sizeof(emst_stats), else EMST_ERR_INVALID_ARG). */
typedef struct emst_stats {
  int32_t struct_size;   /* set by the caller: sizeof(emst_stats) */
  int32_t rounds;        /* Boruvka rounds run */
  int32_t kernel_launches; /* kernels this call launched */
  int32_t morton_bits;   /* Z-curve code width used (64 or 128) */
  double total_ms;       /* device time of the whole call (CUDA events) */
  double build_ms;       /* scene box, codes, sort, hierarchy, refit (A1-A4) */
  double rounds_ms;      /* all Boruvka rounds */
  double output_ms;      /* final ordering of the edges (+ copies) */
  int64_t node_visits;   /* total internal-node visits by queries (count_visits=1) */
  int64_t components_per_round[40]; /* components at the start of each round */
  double traverse_ms;    /* device time of the traversal kernels (Algorithm 2) alone */
  int32_t traverse_launches; /* traversal kernels timed in traverse_ms */
  int32_t reserved1;
  double round_traverse_ms[40]; /* traversal time of each round */
  int64_t queried_points;  /* learned radius: queries that used a proposed cutoff */
  int64_t rerun_points;    /* learned radius: of those, rerun because the cutoff fell below
                              their component's found minimum */
  double learned_search_ms; /* learned radius: device time of the searches with the proposed
                               cutoffs alone (traverse_ms adds inference and the reruns) */
  double core_ms;          /* mutual reachability: device time of the core distances */
  int64_t code_collisions; /* distinct points sharing their curve predecessor's code: of the
                              64-bit codes when they were built (automatic or 64), else of
                              the 128-bit ones */
  int64_t reserved[1];
  /* count_visits = 1 only (else 0), per round of the plain form: */
  int64_t round_visits[40];   /* internal-node visits of the round's searches */
  int64_t round_queries[40];  /* queries that searched (the others were skipped by their
                                 lower bound before any node visit) */
  int64_t round_distinct_nodes[40]; /* distinct internal nodes those searches visited */
  int32_t traversal_used;  /* the Algorithm 2 kernel that ran: 1 one thread per point, 2
                              persistent work queue */
  int32_t block_used;      /* its CTA size */
  int32_t leaf_used;       /* points per leaf of the hierarchy */
  int32_t tuned;           /* 1 when the tuning file chose parameters of this call */
} emst_stats;

/* EMST of n points (§3, Fig. 3 end to end).
 *   points    n x dim FP32, device or host memory, read only.
 *   n, dim    0 <= n <= EMST_MAX_POINTS, dim in {2, 3}.
 *   out_edges room for max(n-1, 0) emst_edge, device or host memory.
 *   stream    cudaStream_t as void* (NULL = default stream).
 * Returns EMST_OK or an emst_status error (then out_edges is unspecified). */
int emst_compute(const float *points, int64_t n, int dim, emst_edge *out_edges, void *stream);

/* emst_compute with options (NULL = defaults) and statistics (NULL = none). */
int emst_compute_ex(const float *points, int64_t n, int dim, emst_edge *out_edges, void *stream,
                    const emst_options *options, emst_stats *stats);

/* Many independent EMSTs in one call (not in the paper: instances are
 * independent problems, each solved exactly as emst_compute would).
 *   points        all instances' points concatenated, sum(n_k) x dim FP32.
 *   offsets       num_instances+1 int64, offsets[0] = 0, non-decreasing,
 *                 instance k = rows [offsets[k], offsets[k+1]); host or
 *                 device memory (device: read back once, they size the call).
 *   out_edges     room for sum(max(n_k-1, 0)) edges; instance k's edges are
 *                 contiguous, use ids local to the instance, sorted as above.
 *   out_offsets   num_instances+1 int64, host or device memory: edge block
 *                 bounds.
 * Returns EMST_OK or an emst_status error. */
int emst_compute_batched(const float *points, const int64_t *offsets, int num_instances, int dim,
                         emst_edge *out_edges, int64_t *out_offsets, void *stream);

/* emst_compute_batched with options and statistics (as emst_compute_ex;
 * leaf_size, mrd_k, mlp_params and morton_bits other than 0 / 64 do not
 * apply to the batched form and are ignored: one point per leaf, Euclidean
 * weights, 64-bit codes with the instance id in the top bits). */
int emst_compute_batched_ex(const float *points, const int64_t *offsets, int num_instances, int dim,
                            emst_edge *out_edges, int64_t *out_offsets, void *stream,
                            const emst_options *options, emst_stats *stats);

/* Squared core distances of the mutual reachability distance (§4.5): for
 * every point, the FP32 squared distance to its k-th nearest neighbour, the
 * point itself counting as the first (k = 1: 0).  A k-nearest-neighbour
 * search of the same hierarchy the EMST builds.
 *   points    n x dim FP32, device or host memory, read only.
 *   n, dim    1 <= n <= EMST_MAX_POINTS, dim in {2, 3}.
 *   k         1 <= k <= min(n, EMST_MRD_MAX_K).
 *   out_core2 n FP32, device or host memory, in the caller's point order.
 * Returns EMST_OK or an emst_status error. */
int emst_core_distances(const float *points, int64_t n, int dim, int k, float *out_core2,
                        void *stream);

/* EMST with no device allocation (the paper has no counterpart: this is a
 * deployment variant of emst_compute).  For callers that cannot allocate
 * device memory where they need the tree -- an execute hook that must not
 * allocate, a process under a device-memory budget it does not own, or a
 * latency-critical loop that cannot take an allocator's implicit
 * synchronisation.  Same arguments, result and output order as emst_compute.
 *   - Codes: always 64-bit Z-curve codes (emst_compute switches to 128-bit
 *     codes on very dense data, see emst_options.morton_bits).  The tree is
 *     the same either way; only the search on very dense input is slower.
 *   - Scratch: one fixed 16 MiB array in the library's device memory, held by
 *     every GPU that loads the library until the process exits; no cudaMalloc,
 *     cudaFree or pool allocation happens in the call.
 *   - Limit: n <= EMST_NOALLOC_MAX_POINTS, else EMST_ERR_TOO_LARGE (nothing
 *     launched).
 *   - The first call on a device looks up the array's device address (once
 *     per device, with that device current); make that first call before any
 *     stream capture on the device.
 *   - The call waits on its stream: it reads a status word back after the
 *     build and after every round, like emst_compute.
 *   - Every call on a device shares the array and it keeps the last call's
 *     contents (each call clears what must start at zero).  Calls whose GPU
 *     work overlaps (other streams or threads, same device) race on it and
 *     give undefined results: serialise them. */
#define EMST_NOALLOC_MAX_POINTS ((int64_t)65536)
int emst_compute_noalloc(const float *points, int64_t n, int dim, emst_edge *out_edges,
                         void *stream);

/* ---------------------------------------------------------------------- */
/* Learned search radius (the paper has no counterpart; a proposal that only */
/* tightens cutoffs, with a certification rerun that keeps the tree exact).  */
/* ---------------------------------------------------------------------- */
/* The network: EMST_MLP_FEATURES inputs -> 64 -> 64 -> 64 -> 1 (ReLU), one
 * flat FP32 parameter vector of EMST_MLP_PARAMS entries in this order:
 *   in_mu[8], in_sigma[8], out_mu, out_sigma, margin, pad,
 *   W1[64][8], b1[64], W2[64][64], b2[64], W3[64][64], b3[64], w4[64], b4.
 * Features are normalised (f - in_mu) / in_sigma; the output y predicts the
 * normalised log2 nearest other-component weight, de-normalised as
 * y * out_sigma + out_mu, plus margin (a safety offset in log2 units).
 * The 8 features of a point (curve order) in a round: its position in the
 * scene box (3, z = 0 in 2D), log2 of the smallest and of the mean weight to
 * its 4 + 4 curve neighbours, log2 of its component size, log2 of its lower
 * bound from the previous round (0 in the first), log2 of its component's
 * cutoff. */
#define EMST_MLP_FEATURES 8
#define EMST_MLP_PARAMS 8981

/* Inference (BF16 weights and activations on the tensor cores, FP32
 * accumulation): out_log2w[k] = predicted log2 weight of feature row k.
 * features: m x EMST_MLP_FEATURES FP32; params, out: device memory. */
int emst_mlp_forward(const float *features, int64_t m, const float *params, float *out_log2w,
                     void *stream);

/* Training step pieces (FP32).  emst_mlp_grad ADDS the gradient of the mean
 * squared error (on the normalised target log2 weights) over the m samples to
 * grad[EMST_MLP_PARAMS] and the loss to *loss; emst_mlp_adam applies one Adam
 * step (step >= 1) to the trainable entries (from W1 on) and clears grad.
 * All pointers are device memory. */
int emst_mlp_grad(const float *features, const float *targets, int64_t m, const float *params,
                  float *grad, float *loss, void *stream);
int emst_mlp_adam(float *params, float *grad, float *m1, float *m2, int step, float lr,
                  float beta1, float beta2, float eps, void *stream);

/* Training pairs from a plain run on `points`: in every round, about one
 * point in `every` (a fixed hash of position and round) contributes its
 * features and the exact log2 weight of its nearest point in another
 * component.  out_features (capacity x EMST_MLP_FEATURES) and out_targets
 * (capacity) are device memory; *out_count (host) = pairs produced (only the
 * first `capacity` are stored). */
int emst_learned_samples(const float *points, int64_t n, int dim, int every, float *out_features,
                         float *out_targets, int64_t capacity, int64_t *out_count, void *stream);

/* ---------------------------------------------------------------------- */
/* Single-linkage dendrogram (the paper has no counterpart: the hierarchy   */
/* that single-linkage clustering and HDBSCAN* read off the EMST, or off    */
/* the mutual-reachability tree of §4.5 -- clustering is the first use of   */
/* the EMST the introduction names).                                        */
/* ---------------------------------------------------------------------- */
/* One merge of the hierarchy: clusters a < b joined at weight w into a
 * cluster of `size` points (16 bytes; the row layout of a linkage matrix). */
typedef struct emst_linkage {
  uint32_t a;
  uint32_t b;
  float w;
  uint32_t size;
} emst_linkage;

/* The hierarchy is Kruskal's merge sequence over the tree's own edges (§2,
 * "MST computation"), taken in the given order.  Cluster ids: point v is
 * cluster v; the cluster made by edges[k] is n + k.
 *   edges        n-1 edges of a spanning tree of points 0..n-1 in merge
 *                order: weights not decreasing (emst_compute's output order
 *                qualifies); equal weights merge in the given order.  Device
 *                or host memory, read only.
 *   n            0 <= n <= EMST_MAX_POINTS.
 *   out_linkage  n-1 rows (device or host), or NULL: row k = the merge made
 *                by edges[k] (a < b, w = edges[k].w).
 *   out_parent   2n-1 uint32 (device or host), or NULL: the cluster each
 *                cluster merges into; 0xFFFFFFFF for the last one (n + n-2,
 *                or point 0 when n = 1).
 * Returns EMST_OK, or EMST_ERR_INVALID_ARG when an id is >= n, an edge joins
 * a point to itself or closes a cycle, a weight is NaN, or a weight is below
 * the one before it (outputs then unspecified). */
int emst_dendrogram(const emst_edge *edges, int64_t n, emst_linkage *out_linkage,
                    uint32_t *out_parent, void *stream);

/* Static string for a status code (never NULL). */
const char *emst_status_string(int status);

/* ---------------------------------------------------------------------- */
/* Inspection entry points: the hot path's intermediate results, for tests */
/* and tools.  All output pointers are DEVICE memory owned by the caller.   */
/* ---------------------------------------------------------------------- */

/* Tree build (§2 "ArborX": Z-curve sort and linear BVH; §3 Fig. 4 numbering).
 * The hierarchy's leaves are chunks of leaf_size consecutive points in curve
 * order (chunk c = curve positions [c*leaf_size, (c+1)*leaf_size), the last
 * one shorter); with leaf_size = 1 every point is a leaf, as in the paper.
 *   points           n x dim FP32 (device or host), n >= 2.
 *   leaf_size        1, 2, 4, 8 or 16, with ceil(n / leaf_size) >= 2.
 *   out_codes        n uint64: Morton codes in sorted order.
 *   out_perm         n uint32: input index of the k-th point in curve order.
 *   out_children     2(m-1) uint32, m = ceil(n / leaf_size): internal node v's
 *                    left/right child; leaf chunk c is 0x80000000|c, an
 *                    internal node is its index.
 *   out_boxes        (m-1) x 2 x 6 FP32: per internal node, per child, the
 *                    child's box (lo x,y,z, hi x,y,z; z = 0 in 2D).
 * Any output pointer may be NULL (then it is not written). */
int emst_build_bvh(const float *points, int64_t n, int dim, int leaf_size, uint64_t *out_codes,
                   uint32_t *out_perm, uint32_t *out_children, float *out_boxes, void *stream);

/* emst_build_bvh with a Z-curve code width: morton_bits 64 (as above) or 128
 * (emst_options.morton_bits); with 128, out_codes holds 2n uint64: the sorted
 * codes as (high word, low word) pairs. */
int emst_build_bvh_ex(const float *points, int64_t n, int dim, int leaf_size, int morton_bits,
                      uint64_t *out_codes, uint32_t *out_perm, uint32_t *out_children,
                      float *out_boxes, void *stream);

/* One Boruvka round from given component labels (§3: Optimization 1 node
 * labels, Optimization 2 upper bounds, Algorithm 2 queries, the per-component
 * minimum, and the merge), on the hierarchy emst_build_bvh builds with the
 * same leaf_size.  Everything is indexed in CURVE order (the out_perm order of
 * emst_build_bvh); a label is the curve index of a point of its component,
 * and labels[labels[k]] == labels[k] must hold.
 *   labels_in        n uint32 (device).
 *   radius_in        n FP32 per-point starting radius, or NULL to use the
 *                    component upper bound only (device).
 *   out_node_labels  2(m-1) uint32: the label stored with each child of each
 *                    internal node (0xFFFFFFFF = several components).
 *   out_upper_bound  n FP32 indexed by label (+inf where none).
 *   out_nn_w, out_nn_j  n FP32 / uint32: each point's neighbour in another
 *                    component within its radius (j in curve order,
 *                    0xFFFFFFFF = none, w = +inf).
 *   out_labels       n uint32: labels after the merge.
 *   out_edges        room for n edges (device); *out_num_edges (host) = count,
 *                    in no particular order.
 * Any device output pointer may be NULL. */
int emst_round_step(const float *points, int64_t n, int dim, int leaf_size,
                    const uint32_t *labels_in, const float *radius_in, uint32_t *out_node_labels,
                    float *out_upper_bound, float *out_nn_w, uint32_t *out_nn_j,
                    uint32_t *out_labels, emst_edge *out_edges, int64_t *out_num_edges,
                    void *stream);

#ifdef __cplusplus
}
#endif

#endif /* EMST_H_ */

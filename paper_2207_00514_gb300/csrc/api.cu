// api.cu -- the C ABI (include/emst.h): argument checks, scratch layout,
// host/device pointer handling and the orchestration of the method (Fig. 3):
// build the hierarchy once, then Boruvka rounds until n-1 edges are found.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "common.cuh"

namespace emst {
namespace {

// ---------------------------------------------------------------------------
// Stream-ordered scratch from one library-owned pool per device.  The pool
// keeps its memory between calls (release threshold = max), so repeated calls
// of the same size allocate nothing new from the driver.
// ---------------------------------------------------------------------------
std::mutex g_pool_mu;
cudaMemPool_t g_pool[64];
bool g_pool_ready[64] = {false};

cudaError_t get_pool(int dev, cudaMemPool_t *out) {
  std::lock_guard<std::mutex> lock(g_pool_mu);
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!g_pool_ready[dev]) {
    cudaMemPoolProps props;
    std::memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaError_t e = cudaMemPoolCreate(&g_pool[dev], &props);
    if (e != cudaSuccess) return e;
    uint64_t thr = ~0ull;
    cudaMemPoolSetAttribute(g_pool[dev], cudaMemPoolAttrReleaseThreshold, &thr);
    g_pool_ready[dev] = true;
  }
  *out = g_pool[dev];
  return cudaSuccess;
}

}  // namespace

// Helpers shared with the other entry points of the library (declared in
// common.cuh).
bool device_accessible(const void *p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

#ifndef EMST_MAPPED_HOST
#define EMST_MAPPED_HOST 1
#endif
void *mapped_host(const void *p) {
  if (!EMST_MAPPED_HOST || !p) return nullptr;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (a.type != cudaMemoryTypeHost) return nullptr;
  return a.devicePointer;
}

int sm_count() {
  static int cached[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
  if (cached[dev] == 0) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1) {
      cudaGetLastError();
      v = 1;
    }
    cached[dev] = v;
  }
  return cached[dev];
}

cudaError_t scratch_alloc(void **p, size_t bytes, cudaStream_t s) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  cudaMemPool_t pool;
  e = get_pool(dev, &pool);
  if (e != cudaSuccess) return e;
  e = cudaMallocFromPoolAsync(p, bytes, pool, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
  }
  return e;
}

struct Carver {
  char *base;
  size_t off = 0;
  explicit Carver(char *b) : base(b) {}
  template <class T>
  T *take(int64_t count) {
    off = (off + 255) & ~size_t(255);
    T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
    off += sizeof(T) * (size_t)(count > 0 ? count : 1);
    return p;
  }
};

// Lays the scratch of one problem out from `base` (nullptr: only measures).
int effective_leaf(int64_t n, int requested) {
  int k = requested > 0 ? requested : 1;
  if (k > 16) k = 16;
  int p = 1;
  while (p * 2 <= k) p *= 2;
  while (p > 1 && (n + p - 1) / p < 2) p /= 2;
  return p;
}

size_t layout(Problem &P, char *base, bool copy_points, bool copy_edges) {
  const int64_t n = P.n;
  if (P.leaf < 1) P.leaf = 1;
  P.nc = (n + P.leaf - 1) / P.leaf;
  const int64_t nc = P.nc;
  Carver c(base);
  P.counters = c.take<uint32_t>(64);
  P.sort_hist = c.take<uint32_t>(8 * 256);
  P.sort_tiles = sort_tiles_for(n);
  P.sort_lookback = c.take<uint32_t>(256 * P.sort_tiles);
  P.pts = c.take<float4>(n);
  P.keys[0] = c.take<uint64_t>(n);
  P.keys[1] = c.take<uint64_t>(n);
  P.vals[0] = c.take<uint32_t>(n);
  P.vals[1] = c.take<uint32_t>(n);
  P.nodes = c.take<NodeRec>(nc - 1);
  P.nlabels = c.take<uint2>(nc - 1);
  P.split_far = c.take<uint2>(nc - 1);
  P.arrivals = c.take<uint32_t>(nc - 1);
  P.range = c.take<uint2>(nc - 1);
  P.runs = c.take<uint32_t>(n);
  P.scan_tiles = c.take<uint32_t>(2 * scan_tiles_for(n));
  P.labels_buf[0] = c.take<uint32_t>(n);
  P.labels_buf[1] = c.take<uint32_t>(n);
  P.bound_buf[0] = c.take<uint32_t>(n);
  P.bound_buf[1] = c.take<uint32_t>(n);
  P.list_buf[0] = c.take<uint32_t>(n);
  P.list_buf[1] = c.take<uint32_t>(n);
  P.cur = 0;
  P.labels = P.labels_buf[0];
  P.bound = P.bound_buf[0];
  P.active_list = nullptr;
  P.next_list = P.list_buf[0];
  P.n_active = n;
  P.res = c.take<uint2>(n);
  P.comp_buf[0] = c.take<CompBest>(n);
  P.comp_buf[1] = c.take<CompBest>(n);
  P.comp = P.comp_buf[0];
  P.root = c.take<uint32_t>(n);
  P.edges = c.take<emst_edge>(n);
  if (P.num_inst > 1) {
    P.offsets = c.take<int64_t>(P.num_inst + 1);
    P.inst_in = c.take<uint32_t>(n);
    P.inst_of = c.take<uint32_t>(n);
    P.inst_root = c.take<uint32_t>(P.num_inst);
  } else {
    P.offsets = nullptr;
    P.inst_in = P.inst_of = P.inst_root = nullptr;
  }
  if (P.want_learned || P.want_logging) P.comp_size = c.take<uint32_t>(n);
  if (P.want_learned) {
    P.pred_r = c.take<float>(n);
    P.r_used = c.take<float>(n);
    P.rerun_list = c.take<uint32_t>(n);
    P.mlp = c.take<float>(EMST_MLP_PARAMS);
  }
  if (P.want_logging) P.log_count = c.take<unsigned long long>(1);
  P.seen = P.want_count ? c.take<uint32_t>((nc - 1 + 31) / 32) : nullptr;
  P.core2 = P.want_mrd ? c.take<float>(n) : nullptr;
  P.wide_hi = P.wide || P.auto_wide ? c.take<uint64_t>(n) : nullptr;
  P.wide_lo = P.wide || P.auto_wide ? c.take<uint64_t>(n) : nullptr;
  float *pcopy = c.take<float>(copy_points ? n * P.dim : 1);
  if (copy_points) P.points = pcopy;
  emst_edge *ecopy = c.take<emst_edge>(copy_edges ? n : 1);
  P.out_stage = copy_edges ? ecopy : nullptr;
  return c.off + 256;
}

int status_from_bits(uint32_t bits) {
  if (bits & kErrBadInput) return EMST_ERR_INVALID_ARG;
  if (bits & kErrNonFinite) return EMST_ERR_NONFINITE;
  if (bits & (kErrStack | kErrSpin | kErrChain | kErrCas)) return EMST_ERR_INTERNAL;
  return EMST_OK;
}

#define CU(call)                                  \
  do {                                            \
    cudaError_t e_ = (call);                      \
    if (e_ != cudaSuccess) { rc = EMST_ERR_CUDA; goto done; } \
  } while (0)

int check_args(const float *points, int64_t n, int dim) {
  if (n < 0 || n > EMST_MAX_POINTS) return EMST_ERR_INVALID_ARG;
  if (dim != 2 && dim != 3) return EMST_ERR_INVALID_ARG;
  if (n > 0 && !points) return EMST_ERR_INVALID_ARG;
  return EMST_OK;
}

int bits_for(int64_t v) {  // bits needed to represent values in [0, v]
  int b = 0;
  while (b < 63 && (v >> b) != 0) ++b;
  return b;
}

// A2-A4 (a): codes, their stable order, the points gathered into it.
static void build_order64(Problem &P) {
  launch_morton(P);
  const int src = radix_sort_pairs(P, P.n, 0, 8, 0);
  if (src != 0) {  // keep the sorted codes in keys[0] and the order in vals[0]
    std::swap(P.keys[0], P.keys[1]);
    std::swap(P.vals[0], P.vals[1]);
  }
  P.code_hi = nullptr;
  P.perm = P.vals[0];
  launch_gather(P, P.perm);
}

// The same with 128-bit codes: a stable LSD sort by the low words, then by
// the high words carrying that order; the low words follow the final order.
static void build_order128(Problem &P) {
  launch_morton128(P);
  const int s = radix_sort_pairs(P, P.n, 0, 8, 0);
  launch_gather_u64(P, P.wide_hi, P.vals[s], P.keys[s ^ 1]);
  cudaMemcpyAsync(P.vals[s ^ 1], P.vals[s], sizeof(uint32_t) * (size_t)P.n,
                  cudaMemcpyDeviceToDevice, P.stream);
  const int r = radix_sort_pairs(P, P.n, 0, 8, s ^ 1);
  launch_gather_u64(P, P.wide_lo, P.vals[r], P.keys[r ^ 1]);
  // keys[0] = sorted low words, keys[1] = sorted high words, vals[0] = order
  if (r == 0) std::swap(P.keys[0], P.keys[1]);
  else std::swap(P.vals[0], P.vals[1]);
  P.code_hi = P.keys[1];
  P.perm = P.vals[0];
  launch_gather(P, P.perm);
}

// A1-A4: scene box, codes, sort, gather, hierarchy, refit.  With auto_wide
// the 64-bit order is built first and its collisions counted (one host
// read); when more than n/64 distinct points share their predecessor's code,
// the order is rebuilt with 128-bit codes (§4.1's remedy for data the 64-bit
// grid under-resolves).
void run_build(Problem &P) {
  launch_scene_box(P);
  if (P.num_inst > 1) launch_instance_ids(P);
  if (P.wide) {
    build_order128(P);
  } else {
    build_order64(P);
    if (P.auto_wide) {
      unsigned long long c = 0;
      uint32_t status = 0;
      cudaMemcpyAsync(&c, P.counters + 30, sizeof(c), cudaMemcpyDeviceToHost, P.stream);
      cudaMemcpyAsync(&status, P.counters + 1, sizeof(status), cudaMemcpyDeviceToHost, P.stream);
      if (cudaStreamSynchronize(P.stream) == cudaSuccess) {
        P.code_collisions = (int64_t)c;
        if (status == 0 && (int64_t)c * 64 > P.n) {
          P.wide = true;
          build_order128(P);
        }
      }
    }
  }
  if (P.n >= 2) {
    cudaMemsetAsync(P.arrivals, 0, sizeof(uint32_t) * (size_t)(P.nc - 1), P.stream);
    launch_build_tree(P);
    if (P.num_inst > 1) launch_instance_roots(P);
  }
}

// One Boruvka round (the loop body of Fig. 3).  Round 0 takes its node labels
// from the refit and computes its curve-pair bounds here; later rounds use
// what the previous round's relabel pass prepared.
void run_round(Problem &P, int round, bool carried, int block, bool count) {
  if (round > 0) launch_node_labels(P);
  else launch_upper_bounds(P);
  launch_traverse(P, round > 0 && carried, nullptr, block, count, true, 0, round == 0,
                  P.graph_round ? -1 : round);
  launch_merge(P);
}

// ---------------------------------------------------------------------------
// Graph rounds (emst_options.use_graph): rounds 1, 2, ... as one CUDA graph
// whose while node repeats them until a device-side flag says the method is
// done -- no host round trip between rounds.  The round's buffers alternate
// (ping-pong), so the loop body holds two rounds, the second under an if
// node; after each round a one-thread kernel reads the edge count, the status
// word and the round count on the device and sets the conditions: continue
// while edges < expected, no error bit is set and fewer than `limit` rounds
// have run (the same bound as the host loop, so the loop always ends).
// ---------------------------------------------------------------------------
enum : int { kCondInit = 0, kCondBoth = 1, kCondLoop = 2 };

__global__ void k_rounds_cond(cudaGraphConditionalHandle h_loop, cudaGraphConditionalHandle h_if,
                              int mode, uint32_t *counters, uint32_t expected, uint32_t limit,
                              uint32_t rounds_before) {
  uint32_t done_rounds;
  if (mode == kCondInit) {
    done_rounds = rounds_before;
  } else {
    done_rounds = counters[41] + 1u;
  }
  counters[41] = done_rounds;
  const unsigned go = counters[0] < expected && counters[1] == 0u && done_rounds < limit ? 1u : 0u;
  cudaGraphSetConditional(h_loop, go);
  if (mode == kCondBoth) cudaGraphSetConditional(h_if, go);
}

// Captures and runs the rounds after round 0 (which the caller ran and
// checked: P holds its state, P.n_active the components it left, the cap of
// every later round's list).  Returns the status of the capture and launch;
// the rounds' own results are in P.counters ([41] = rounds done in all).
// `kernels` receives the kernels one round body launches.
static cudaError_t run_rounds_graph(Problem &P, int64_t expected, int limit, bool carried,
                                    int block, int rounds_before, int *kernels) {
  cudaStream_t cs[3] = {nullptr, nullptr, nullptr};
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ge = nullptr;
  const cudaStream_t caller = P.stream;
  int capturing = 0;
  cudaError_t e = cudaSuccess;
  for (auto &x : cs)
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking);
  P.count_dev = P.counters + 40;
  cudaStreamCaptureStatus st;
  cudaGraph_t cg = nullptr;
  const cudaGraphNode_t *deps = nullptr;
  size_t nd = 0;
  cudaGraphConditionalHandle h_loop = 0, h_if = 0;
  cudaGraphNodeParams wp = {cudaGraphNodeTypeConditional};
  cudaGraphNodeParams ip = {cudaGraphNodeTypeConditional};
  cudaGraphNode_t wn = nullptr, in = nullptr;
  int launches0 = 0;
#define GR(call)                        \
  do {                                  \
    if (e == cudaSuccess) e = (call);   \
  } while (0)
  // outer graph: set the loop condition, then the while node
  GR(cudaStreamBeginCapture(cs[0], cudaStreamCaptureModeThreadLocal));
  if (e == cudaSuccess) capturing = 1;
  GR(cudaStreamGetCaptureInfo(cs[0], &st, nullptr, &cg, &deps, nullptr, &nd));
  GR(cudaGraphConditionalHandleCreate(&h_loop, cg, 0, 0));
  if (e == cudaSuccess) {
    k_rounds_cond<<<1, 1, 0, cs[0]>>>(h_loop, h_loop, kCondInit, P.counters, (uint32_t)expected,
                                      (uint32_t)limit, (uint32_t)rounds_before);
    e = cudaPeekAtLastError();
  }
  GR(cudaStreamGetCaptureInfo(cs[0], &st, nullptr, &cg, &deps, nullptr, &nd));
  wp.type = cudaGraphNodeTypeConditional;
  wp.conditional.handle = h_loop;
  wp.conditional.type = cudaGraphCondTypeWhile;
  wp.conditional.size = 1;
  GR(cudaGraphAddNode(&wn, cg, deps, nullptr, nd, &wp));
  GR(cudaStreamUpdateCaptureDependencies(cs[0], &wn, nullptr, 1, cudaStreamSetCaptureDependencies));
  // the loop body: one round, its conditions, then the other parity's round
  // under the if node
  GR(cudaStreamBeginCaptureToGraph(cs[1], e == cudaSuccess ? wp.conditional.phGraph_out[0] : nullptr,
                                   nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  if (e == cudaSuccess) capturing = 2;
  GR(cudaGraphConditionalHandleCreate(&h_if, wp.conditional.phGraph_out[0], 0, 0));
  if (e == cudaSuccess) {
    P.stream = cs[1];
    launches0 = P.launches;
    P.graph_round = true;  // (the body serves every later round: numbers unknown)
    run_round(P, 1, carried, block, false);
    *kernels = P.launches - launches0 + 1;
    k_rounds_cond<<<1, 1, 0, cs[1]>>>(h_loop, h_if, kCondBoth, P.counters, (uint32_t)expected,
                                      (uint32_t)limit, 0u);
    e = cudaPeekAtLastError();
  }
  GR(cudaStreamGetCaptureInfo(cs[1], &st, nullptr, &cg, &deps, nullptr, &nd));
  ip.type = cudaGraphNodeTypeConditional;
  ip.conditional.handle = h_if;
  ip.conditional.type = cudaGraphCondTypeIf;
  ip.conditional.size = 1;
  GR(cudaGraphAddNode(&in, cg, deps, nullptr, nd, &ip));
  GR(cudaStreamUpdateCaptureDependencies(cs[1], &in, nullptr, 1, cudaStreamSetCaptureDependencies));
  GR(cudaStreamBeginCaptureToGraph(cs[2], e == cudaSuccess ? ip.conditional.phGraph_out[0] : nullptr,
                                   nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  if (e == cudaSuccess) {
    capturing = 3;
    advance_round(P, P.n_active);  // the other parity (same cap)
    P.stream = cs[2];
    run_round(P, 2, carried, block, false);
    k_rounds_cond<<<1, 1, 0, cs[2]>>>(h_loop, h_if, kCondLoop, P.counters, (uint32_t)expected,
                                      (uint32_t)limit, 0u);
    e = cudaPeekAtLastError();
    advance_round(P, P.n_active);  // back: two swaps restore the first parity
  }
  P.stream = caller;
  P.graph_round = false;
  // end every capture that began, whatever happened
  if (capturing >= 3) {
    cudaGraph_t x = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(cs[2], &x);
    if (e == cudaSuccess) e = e2;
  }
  if (capturing >= 2) {
    cudaGraph_t x = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(cs[1], &x);
    if (e == cudaSuccess) e = e2;
  }
  if (capturing >= 1) {
    const cudaError_t e2 = cudaStreamEndCapture(cs[0], &g);
    if (e == cudaSuccess) e = e2;
  }
  GR(cudaGraphInstantiate(&ge, g, 0));
  GR(cudaGraphLaunch(ge, caller));
  GR(cudaStreamSynchronize(caller));
#undef GR
  P.count_dev = nullptr;
  if (ge) cudaGraphExecDestroy(ge);
  if (g) cudaGraphDestroy(g);
  for (auto &x : cs)
    if (x) cudaStreamDestroy(x);
  if (e != cudaSuccess) cudaGetLastError();
  return e;
}

void reset_round_state(Problem &P) {
  cudaMemsetAsync(P.bound, 0xFF, sizeof(uint32_t) * (size_t)P.n, P.stream);
  // (the other buffer is cleared by the first round's merge)
  cudaMemsetAsync(P.comp, 0xFF, sizeof(CompBest) * (size_t)P.n, P.stream);
}

// A12: the n-1 edges in (w, i, j) order into `out` (device).  w_bits: the
// largest emitted weight's bits (counters[11]): the sort key needs
// L + significant bits of it.
int run_output(Problem &P, emst_edge *out, uint32_t w_bits) {
  const int64_t m = P.num_inst > 1 ? P.edges_expected : P.n - 1;
  if (m <= 0) return EMST_OK;
  const int L = bits_for(P.n - 1);
  const int wb = w_bits ? 32 - __builtin_clz(w_bits) : 0;
  // fast path: one sort of a 64-bit key, then the runs of equal keys (the
  // edges of one point at one weight) put in j order in place -- unless such
  // a run is long (exact ties: many identical points), then the full path
  const int Lloc = P.num_inst > 1 ? bits_for(P.largest > 1 ? P.largest - 1 : 1) : L;
  const bool fast = P.num_inst == 1 || P.inst_bits + wb + Lloc <= 64;
  auto long_run_count = [&](uint32_t &c) {
    return cudaMemcpyAsync(&c, P.counters + 10, sizeof(uint32_t), cudaMemcpyDeviceToHost,
                           P.stream) == cudaSuccess &&
           cudaStreamSynchronize(P.stream) == cudaSuccess;
  };
  // fastest path (one instance, no group of identical points): the same key
  // sorted on w's bits only, stable, then every run of equal w (a handful of
  // edges in general position) put in (i, j) order in place -- unless such
  // a run is long (a lattice, many equal distances), then the next path
  if (P.num_inst == 1 && !P.ties && wb > 0) {
    launch_edge_keys_wi(P, m, L);
    const int s = radix_sort_pairs(P, m, 0, (wb + 7) / 8, 0, L);
    cudaMemsetAsync(P.counters + 10, 0, sizeof(uint32_t), P.stream);
    launch_edge_ties_w(P, m, s, L);
    uint32_t long_runs = 0;
    if (!long_run_count(long_runs)) return EMST_ERR_CUDA;
    if (long_runs == 0) {
      launch_edge_from_keys(P, m, s, Lloc, wb, out);
      return EMST_OK;
    }
  }
  if (fast) {
    int digits;
    if (P.num_inst == 1) {
      launch_edge_keys_wi(P, m, L);
      digits = (L + wb + 7) / 8;
    } else {
      launch_edge_keys_inst_wi(P, m, wb + Lloc, Lloc);
      digits = (P.inst_bits + wb + Lloc + 7) / 8;
    }
    const int s = radix_sort_pairs(P, m, 0, digits, 0);
    cudaMemsetAsync(P.counters + 10, 0, sizeof(uint32_t), P.stream);
    launch_edge_ties(P, m, s);
    uint32_t long_runs = 0;
    if (cudaMemcpyAsync(&long_runs, P.counters + 10, sizeof(uint32_t), cudaMemcpyDeviceToHost,
                        P.stream) != cudaSuccess ||
        cudaStreamSynchronize(P.stream) != cudaSuccess)
      return EMST_ERR_CUDA;
    if (long_runs == 0) {
      launch_edge_from_keys(P, m, s, Lloc, wb, out);
      return EMST_OK;
    }
  }
  // full path: stable by j, then by (w, i), then (batched) by instance
  launch_edge_keys_j(P, m);
  int s = radix_sort_pairs(P, m, 0, (L + 7) / 8, 0);
  launch_edge_keys_wi_of(P, m, s, L);
  s = radix_sort_pairs(P, m, 0, (L + wb + 7) / 8, s);
  if (P.num_inst > 1) {
    launch_edge_keys_inst(P, m, s);
    s = radix_sort_pairs(P, m, 0, (P.inst_bits + 7) / 8, s);
  }
  launch_edge_gather(P, m, P.vals[s], out);
  return EMST_OK;
}

namespace {

struct Timer {
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  bool on = false;
  void start(cudaStream_t s) {
    on = true;
    for (auto &e : ev) cudaEventCreate(&e);
    cudaEventRecord(ev[0], s);
  }
  void mark(int k, cudaStream_t s) { if (on) cudaEventRecord(ev[k], s); }
  float ms(int a, int b) {
    float t = 0.f;
    if (on) cudaEventElapsedTime(&t, ev[a], ev[b]);
    return t;
  }
  ~Timer() { for (auto &e : ev) if (e) cudaEventDestroy(e); }
};

}  // namespace

// The method on one point set, or (offsets != nullptr) on num_inst
// independent instances in one launch sequence.  offsets / out_offsets are
// host arrays of num_inst + 1 entries.
// Internal extras of a call: training-pair logging and skipping the output.
struct Extras {
  float *log_feat = nullptr;
  float *log_target = nullptr;
  int64_t log_capacity = 0;
  int log_every = 1;
  int64_t *log_count_out = nullptr;
  bool skip_output = false;
};

int compute_impl(const float *points, int64_t n, int dim, const int64_t *offsets, int64_t num_inst,
                 emst_edge *out, int64_t *out_offsets, cudaStream_t stream,
                 const emst_options *opt, emst_stats *stats, const Extras *ex = nullptr) {
  int rc = check_args(points, n, dim);
  if (rc != EMST_OK) return rc;
  int64_t expected = n > 1 ? n - 1 : 0, largest = n;
  if (offsets) {
    if (num_inst < 1 || num_inst > (int64_t)1 << 30 || offsets[0] != 0 || offsets[num_inst] != n)
      return EMST_ERR_INVALID_ARG;
    expected = 0;
    largest = 0;
    for (int64_t I = 0; I < num_inst; ++I) {
      const int64_t nk = offsets[I + 1] - offsets[I];
      if (nk < 0) return EMST_ERR_INVALID_ARG;
      if (out_offsets) out_offsets[I] = expected;
      expected += nk > 1 ? nk - 1 : 0;
      largest = nk > largest ? nk : largest;
    }
    if (out_offsets) out_offsets[num_inst] = expected;
  } else {
    num_inst = 1;
  }
  const bool skip_output = ex && ex->skip_output;
  if (expected > 0 && !out && !skip_output) return EMST_ERR_INVALID_ARG;
  if (stats) {
    int32_t sz = stats->struct_size;
    if (sz < (int32_t)sizeof(emst_stats)) return EMST_ERR_INVALID_ARG;
    std::memset(stats, 0, sizeof(emst_stats));
    stats->struct_size = sz;
  }
  if (n == 0) return EMST_OK;
  int block = 0, carried = 1, count = 0, leaf_req = 0, mrd_k = 0, morton_bits = 0, traversal = 0;
  int refill = 0, chunk = 0, ignore_tuning = 0, use_graph = 0;
  const float *mlp_params = nullptr;
  if (opt && opt->struct_size >= (int32_t)sizeof(emst_options)) {
    block = opt->block_size;
    carried = opt->carried_radius;
    use_graph = opt->use_graph;
    count = opt->count_visits;
    leaf_req = opt->leaf_size;
    mlp_params = opt->mlp_params;
    mrd_k = opt->mrd_k;
    if (offsets) {  // the batched form: Euclidean weights, plain cutoffs, one point per leaf
      mlp_params = nullptr;
      mrd_k = 0;
      leaf_req = 0;
    }
    if (mrd_k < 0 || mrd_k > EMST_MRD_MAX_K || (mrd_k >= 2 && (mlp_params || n < mrd_k)))
      return EMST_ERR_INVALID_ARG;
    morton_bits = opt->morton_bits;
    traversal = opt->traversal;
    if (traversal < 0 || traversal > 2) return EMST_ERR_INVALID_ARG;
    refill = opt->refill_lanes;
    chunk = opt->queue_chunk;
    ignore_tuning = opt->ignore_tuning;
    if (refill < 0 || refill > 32 || (chunk != 0 && (chunk < 32 || chunk > (1 << 20))))
      return EMST_ERR_INVALID_ARG;
    if (morton_bits != 0 && morton_bits != 64 && morton_bits != 128) return EMST_ERR_INVALID_ARG;
    if (leaf_req < 0 || leaf_req > 16 || (leaf_req & (leaf_req - 1)) != 0) return EMST_ERR_INVALID_ARG;
    if (block != 0 && (block < 64 || block > kTraverseMaxBlock || block % 32 != 0))
      return EMST_ERR_INVALID_ARG;
  } else if (opt && opt->struct_size != 0) {
    return EMST_ERR_INVALID_ARG;
  }

  // parameters the caller left to the library: the tuning file's choice for
  // this GPU, dimension, form and size, if it has one
  TuneChoice tuned;
  bool was_tuned = false;
  if (!ignore_tuning && lookup_tuning(dim, offsets != nullptr, n, &tuned)) {
    was_tuned = true;
    if (traversal == 0) traversal = tuned.traversal;
    if (block == 0 && tuned.block >= 64 && tuned.block <= kTraverseMaxBlock && tuned.block % 32 == 0)
      block = tuned.block;
    if (leaf_req == 0 && !offsets && tuned.leaf >= 1 && tuned.leaf <= 16 &&
        (tuned.leaf & (tuned.leaf - 1)) == 0 && !mlp_params && mrd_k < 2)
      leaf_req = tuned.leaf;
    if (refill == 0 && tuned.refill >= 1 && tuned.refill <= 32) refill = tuned.refill;
    if (chunk == 0 && tuned.chunk >= 32) chunk = tuned.chunk;
    if (traversal < 0 || traversal > 2) traversal = 0;
  }

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return EMST_ERR_CUDA;
  cudaMemPool_t pool;
  if (get_pool(dev, &pool) != cudaSuccess) return EMST_ERR_CUDA;
  const bool pts_dev = device_accessible(points);
  const bool out_dev = expected == 0 || skip_output || device_accessible(out);
  // pinned host buffers are read / written in place by the first and last
  // passes (no separate copies); pageable ones are staged through scratch
  const float *pts_map = pts_dev ? nullptr : static_cast<const float *>(mapped_host(points));
  emst_edge *out_map = out_dev ? nullptr : static_cast<emst_edge *>(mapped_host(out));
  const bool learned = mlp_params != nullptr;
  const bool logging = ex && ex->log_feat;

  Problem P;
  P.n = n;
  P.dim = dim;
  P.stream = stream;
  P.points = points;
  P.num_inst = num_inst;
  P.inst_bits = num_inst > 1 ? bits_for(num_inst - 1) : 0;
  P.edges_expected = expected;
  P.largest = largest;
  // (a batched problem keeps one point per leaf: chunks would mix instances)
  P.leaf = num_inst > 1 ? 1 : effective_leaf(n, leaf_req);
  P.want_learned = learned;
  P.want_logging = logging;
  P.want_mrd = mrd_k >= 2 && !offsets && n >= 2;
  P.wide = morton_bits == 128 && !offsets;
  P.auto_wide = morton_bits == 0 && !offsets;
  P.persistent = traversal == 2;
  P.refill_lanes = refill;
  P.queue_chunk = chunk;
  P.block = block;
  P.want_count = count != 0;
  if (logging) {
    P.log_feat = ex->log_feat;
    P.log_target = ex->log_target;
    P.log_capacity = ex->log_capacity;
    P.log_every = ex->log_every < 1 ? 1 : ex->log_every;
  }
  int64_t reruns = 0;
  const size_t need = layout(P, nullptr, !pts_dev, !out_dev && !out_map);
  char *base = nullptr;
  uint32_t host_counters[48] = {0};
  uint64_t prev_visits = 0, prev_queries = 0, prev_distinct = 0;
  Timer tm;
  int rounds = 0;
  cudaEvent_t tev[2 * 40];
  cudaEvent_t lev[2 * 40] = {nullptr};  // learned: around the proposed-cutoff search
  cudaEvent_t cev[2] = {nullptr, nullptr};  // mutual reachability: around the core distances
  int n_tev = 0;
  if (cudaMallocFromPoolAsync((void **)&base, need, pool, stream) != cudaSuccess) {
    cudaGetLastError();
    return EMST_ERR_OOM;
  }
  layout(P, base, !pts_dev, !out_dev && !out_map);
  if (stats) tm.start(stream);
  CU(cudaMemsetAsync(P.counters, 0, sizeof(uint32_t) * 64, stream));
  if (pts_map) P.points_mapped = pts_map;  // copied by the scene-box pass
  else if (!pts_dev)
    CU(cudaMemcpyAsync((void *)P.points, points, sizeof(float) * (size_t)n * dim,
                       cudaMemcpyHostToDevice, stream));
  if (num_inst > 1)
    CU(cudaMemcpyAsync(P.offsets, offsets, sizeof(int64_t) * (size_t)(num_inst + 1),
                       cudaMemcpyHostToDevice, stream));
  if (learned)
    CU(cudaMemcpyAsync((void *)P.mlp, mlp_params, sizeof(float) * EMST_MLP_PARAMS,
                       cudaMemcpyDefault, stream));
  if (logging) CU(cudaMemsetAsync(P.log_count, 0, sizeof(unsigned long long), stream));
  if (P.seen) CU(cudaMemsetAsync(P.seen, 0, sizeof(uint32_t) * (size_t)((P.nc - 1 + 31) / 32), stream));
  run_build(P);
  tm.mark(1, stream);
  // Non-finite input is reported before any round runs.
  CU(cudaMemcpyAsync(host_counters, P.counters, sizeof(host_counters), cudaMemcpyDeviceToHost,
                     stream));
  CU(cudaStreamSynchronize(stream));
  if (host_counters[1] != 0) { rc = status_from_bits(host_counters[1]); goto done; }
  // a large group of identical points can exist: the search needs its tie rule
  P.ties = host_counters[32] != 0;
  if (!P.auto_wide) P.code_collisions = (int64_t)host_counters[30] | ((int64_t)host_counters[31] << 32);
  if (expected > 0) {
    if (P.core2) {  // mutual reachability: core distances on the finished hierarchy
      if (stats) {
        cudaEventCreate(&cev[0]);
        cudaEventCreate(&cev[1]);
        cudaEventRecord(cev[0], stream);
      }
      launch_core_knn(P, mrd_k);
      if (stats) cudaEventRecord(cev[1], stream);
    }
    reset_round_state(P);
    // Boruvka rounds (Fig. 3 loop): each round at least halves the number of
    // components of every unfinished instance, so more than ceil(log2 n)
    // rounds (n: the largest instance) means something is wrong.
    const int limit = bits_for(largest - 1) + 1;
    for (rounds = 0;; ++rounds) {
      if (rounds >= limit) { rc = EMST_ERR_ROUND_LIMIT; goto done; }
      if (stats && rounds < 40)
        stats->components_per_round[rounds] = n - (int64_t)host_counters[0];
      if (rounds > 0) launch_node_labels(P);
      else launch_upper_bounds(P);
      if (learned || logging) launch_comp_sizes(P);
      if (logging) launch_log_samples(P, rounds, rounds > 0 && carried);
      if (stats && rounds < 40) {
        cudaEventCreate(&tev[2 * rounds]);
        cudaEventCreate(&tev[2 * rounds + 1]);
        cudaEventRecord(tev[2 * rounds], stream);
      }
      if (learned) {
        // proposed cutoffs, queries with them, then the certification rerun
        launch_predict(P, rounds > 0 && carried);
        if (stats && rounds < 40) {
          cudaEventCreate(&lev[2 * rounds]);
          cudaEventRecord(lev[2 * rounds], stream);
        }
        launch_traverse(P, rounds > 0 && carried, nullptr, block, count != 0, true, 1);
        if (stats && rounds < 40) {
          cudaEventCreate(&lev[2 * rounds + 1]);
          cudaEventRecord(lev[2 * rounds + 1], stream);
        }
        CU(cudaMemsetAsync(P.counters + 13, 0, sizeof(uint32_t), stream));
        launch_rerun_mark(P);
        launch_traverse(P, rounds > 0 && carried, nullptr, block, count != 0, true, 2);
      } else {
        launch_traverse(P, rounds > 0 && carried, nullptr, block, count != 0, true, 0, rounds == 0, rounds);
      }
      if (stats && rounds < 40) {
        cudaEventRecord(tev[2 * rounds + 1], stream);
        n_tev = rounds + 1;
      }
      if (count) launch_count_seen(P);
      launch_merge(P);
      CU(cudaPeekAtLastError());  // a launch that failed must not read as a round without edges
      CU(cudaMemcpyAsync(host_counters, P.counters, sizeof(host_counters), cudaMemcpyDeviceToHost,
                         stream));
      CU(cudaStreamSynchronize(stream));
      if (host_counters[1] != 0) { rc = status_from_bits(host_counters[1]); goto done; }
      if (learned) reruns += host_counters[13];
      if (count && stats && rounds < 40) {
        auto u64 = [&](int k) { return (uint64_t)host_counters[k] | ((uint64_t)host_counters[k + 1] << 32); };
        stats->round_visits[rounds] = (int64_t)(u64(2) - prev_visits);
        stats->round_queries[rounds] = (int64_t)(u64(34) - prev_queries);
        stats->round_distinct_nodes[rounds] = (int64_t)(u64(38) - prev_distinct);
        prev_visits = u64(2);
        prev_queries = u64(34);
        prev_distinct = u64(38);
      }
      advance_round(P, (int64_t)host_counters[12]);
      if ((int64_t)host_counters[0] >= expected) { ++rounds; break; }
      if (rounds == 0 && use_graph == 1 && !learned && !logging && !count) {
        // the remaining rounds as one graph ended on the device
        int kernels = 0;
        const int before = P.launches;
        CU(run_rounds_graph(P, expected, limit, carried != 0, block, 1, &kernels));
        CU(cudaMemcpyAsync(host_counters, P.counters, sizeof(host_counters),
                           cudaMemcpyDeviceToHost, stream));
        CU(cudaStreamSynchronize(stream));
        rounds = (int)host_counters[41];
        P.launches = before + 1 + (rounds - 1) * kernels;
        if (host_counters[1] != 0) { rc = status_from_bits(host_counters[1]); goto done; }
        if ((int64_t)host_counters[0] < expected) { rc = EMST_ERR_ROUND_LIMIT; goto done; }
        break;
      }
    }
    tm.mark(2, stream);
    if ((int64_t)host_counters[0] != expected) { rc = EMST_ERR_INTERNAL; goto done; }
    if (!skip_output) {
      rc = run_output(P, out_dev ? out : (out_map ? out_map : P.out_stage), host_counters[11]);
      if (rc != EMST_OK) goto done;
    }
    if (!out_dev && !out_map && !skip_output)
      CU(cudaMemcpyAsync(out, P.out_stage, sizeof(emst_edge) * (size_t)expected,
                         cudaMemcpyDeviceToHost, stream));
  } else {
    tm.mark(2, stream);
  }
  tm.mark(3, stream);
  CU(cudaMemcpyAsync(host_counters, P.counters, sizeof(host_counters), cudaMemcpyDeviceToHost,
                     stream));
  CU(cudaStreamSynchronize(stream));
  CU(cudaGetLastError());
  rc = status_from_bits(host_counters[1]);
  if (logging && ex->log_count_out) {
    unsigned long long c = 0;
    CU(cudaMemcpy(&c, P.log_count, sizeof(c), cudaMemcpyDeviceToHost));
    *ex->log_count_out = (int64_t)c;
  }
done:
  cudaFreeAsync(base, stream);
  if (rc == EMST_ERR_CUDA) cudaGetLastError();
  if (stats) {
    cudaStreamSynchronize(stream);
    stats->rounds = rounds;
    stats->kernel_launches = P.launches;
    stats->traversal_used = P.persistent && !learned && !P.core2 && P.leaf == 1 ? 2 : 1;
    stats->block_used = stats->traversal_used == 2 ? kPersistBlock : (block ? block : kTraverseBlock);
    stats->leaf_used = P.leaf;
    stats->tuned = was_tuned ? 1 : 0;
    stats->morton_bits = P.wide ? 128 : 64;
    stats->code_collisions = P.code_collisions;
    stats->build_ms = tm.ms(0, 1);
    stats->rounds_ms = tm.ms(1, 2);
    stats->output_ms = tm.ms(2, 3);
    stats->total_ms = tm.ms(0, 3);
    stats->node_visits = (int64_t)host_counters[2] | ((int64_t)host_counters[3] << 32);
    for (int r = 0; r < n_tev; ++r) {
      float t = 0.f;
      cudaEventElapsedTime(&t, tev[2 * r], tev[2 * r + 1]);
      stats->round_traverse_ms[r] = t;
      stats->traverse_ms += t;
    }
    stats->traverse_launches = n_tev;
    stats->queried_points = learned ? (int64_t)host_counters[15] : 0;
    stats->rerun_points = reruns;
    for (int r = 0; r < n_tev && learned; ++r) {
      float t = 0.f;
      if (lev[2 * r] && lev[2 * r + 1]) cudaEventElapsedTime(&t, lev[2 * r], lev[2 * r + 1]);
      stats->learned_search_ms += t;
    }
  }
  for (int r = 0; r < 2 * 40; ++r)
    if (lev[r]) cudaEventDestroy(lev[r]);
  if (cev[0] && cev[1] && stats) {
    float t = 0.f;
    cudaEventElapsedTime(&t, cev[0], cev[1]);
    stats->core_ms = t;
  }
  for (auto &e : cev)
    if (e) cudaEventDestroy(e);
  for (int r = 0; r < n_tev; ++r) {
    cudaEventDestroy(tev[2 * r]);
    cudaEventDestroy(tev[2 * r + 1]);
  }
  return rc;
}

// ---------------------------------------------------------------------------
// Inspection helpers
// ---------------------------------------------------------------------------
namespace {
__global__ void k_bound_to_float(const uint32_t *b, float *out, int64_t n) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) out[k] = bound_to_radius(b[k]);
}
__global__ void k_split_res(const uint2 *res, float *w, uint32_t *j, int64_t n) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  uint2 r = res[k];
  if (w) w[k] = __uint_as_float(r.x);
  if (j) j[k] = r.y;
}

struct Session {
  Problem P;
  char *base = nullptr;
  int rc = EMST_OK;
  ~Session() {
    if (base) cudaFreeAsync(base, P.stream);
  }
};

int open_session(Session &S, const float *points, int64_t n, int dim, int leaf,
                 cudaStream_t stream) {
  int rc = check_args(points, n, dim);
  if (rc != EMST_OK) return rc;
  if (n < 2) return EMST_ERR_INVALID_ARG;
  if (leaf < 1 || leaf > 16 || (leaf & (leaf - 1)) != 0 || (n + leaf - 1) / leaf < 2)
    return EMST_ERR_INVALID_ARG;
  S.P.leaf = leaf;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return EMST_ERR_CUDA;
  cudaMemPool_t pool;
  if (get_pool(dev, &pool) != cudaSuccess) return EMST_ERR_CUDA;
  const bool pts_dev = device_accessible(points);
  S.P.n = n;
  S.P.dim = dim;
  S.P.stream = stream;
  S.P.points = points;
  size_t need = layout(S.P, nullptr, !pts_dev, false);
  if (cudaMallocFromPoolAsync((void **)&S.base, need, pool, stream) != cudaSuccess) {
    cudaGetLastError();
    S.base = nullptr;
    return EMST_ERR_OOM;
  }
  layout(S.P, S.base, !pts_dev, false);
  cudaMemsetAsync(S.P.counters, 0, sizeof(uint32_t) * 64, stream);
  if (!pts_dev)
    cudaMemcpyAsync((void *)S.P.points, points, sizeof(float) * (size_t)n * dim,
                    cudaMemcpyHostToDevice, stream);
  return EMST_OK;
}

int finish_session(Session &S) {
  uint32_t st = 0;
  if (cudaMemcpyAsync(&st, S.P.counters + 1, sizeof(uint32_t), cudaMemcpyDeviceToHost,
                      S.P.stream) != cudaSuccess)
    return EMST_ERR_CUDA;
  if (cudaStreamSynchronize(S.P.stream) != cudaSuccess) return EMST_ERR_CUDA;
  if (cudaGetLastError() != cudaSuccess) return EMST_ERR_CUDA;
  return status_from_bits(st);
}
}  // namespace

}  // namespace emst

using namespace emst;

extern "C" {

const char *emst_status_string(int status) {
  switch (status) {
    case EMST_OK: return "ok";
    case EMST_ERR_INVALID_ARG: return "invalid argument";
    case EMST_ERR_NONFINITE: return "non-finite coordinate";
    case EMST_ERR_OOM: return "out of device memory";
    case EMST_ERR_CUDA: return "CUDA error";
    case EMST_ERR_ROUND_LIMIT: return "Boruvka round limit exceeded";
    case EMST_ERR_INTERNAL: return "internal error (device-side guard)";
    case EMST_ERR_TOO_LARGE: return "too many points for the fixed scratch of emst_compute_noalloc";
    default: return "unknown status";
  }
}

int emst_compute(const float *points, int64_t n, int dim, emst_edge *out_edges, void *stream) {
  return compute_impl(points, n, dim, nullptr, 1, out_edges, nullptr, (cudaStream_t)stream,
                      nullptr, nullptr);
}

int emst_compute_ex(const float *points, int64_t n, int dim, emst_edge *out_edges, void *stream,
                    const emst_options *options, emst_stats *stats) {
  return compute_impl(points, n, dim, nullptr, 1, out_edges, nullptr, (cudaStream_t)stream,
                      options, stats);
}

int emst_compute_batched(const float *points, const int64_t *offsets, int num_instances, int dim,
                         emst_edge *out_edges, int64_t *out_offsets, void *stream) {
  return emst_compute_batched_ex(points, offsets, num_instances, dim, out_edges, out_offsets, stream,
                                 nullptr, nullptr);
}

int emst_compute_batched_ex(const float *points, const int64_t *offsets, int num_instances, int dim,
                            emst_edge *out_edges, int64_t *out_offsets, void *stream,
                            const emst_options *options, emst_stats *stats) {
  if (num_instances < 0 || !offsets || !out_offsets || (dim != 2 && dim != 3))
    return EMST_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  // offsets / out_offsets may live in device memory: the bounds are read to
  // the host once (they size the problem) and the edge bounds written back
  const bool offs_dev = device_accessible(offsets);
  const bool outoffs_dev = device_accessible(out_offsets);
  std::vector<int64_t> h_offs, h_out;
  const int64_t *offs = offsets;
  if (offs_dev) {
    h_offs.resize((size_t)num_instances + 1);
    if (cudaMemcpyAsync(h_offs.data(), offsets, sizeof(int64_t) * h_offs.size(),
                        cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      cudaGetLastError();
      return EMST_ERR_CUDA;
    }
    offs = h_offs.data();
  }
  int64_t *oo = out_offsets;
  if (outoffs_dev) {
    h_out.resize((size_t)num_instances + 1);
    oo = h_out.data();
  }
  int rc;
  if (num_instances == 0) {
    oo[0] = 0;
    rc = offs[0] == 0 ? EMST_OK : EMST_ERR_INVALID_ARG;
  } else {
    rc = compute_impl(points, offs[num_instances], dim, offs, num_instances, out_edges, oo, s,
                      options, stats);
  }
  if (outoffs_dev && (rc == EMST_OK || rc == EMST_ERR_INVALID_ARG)) {
    if (cudaMemcpyAsync(out_offsets, oo, sizeof(int64_t) * h_out.size(), cudaMemcpyHostToDevice, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      cudaGetLastError();
      return EMST_ERR_CUDA;
    }
  }
  return rc;
}

int emst_learned_samples(const float *points, int64_t n, int dim, int every, float *out_features,
                         float *out_targets, int64_t capacity, int64_t *out_count, void *stream) {
  if (every < 1 || capacity < 0 || (capacity > 0 && (!out_features || !out_targets)) || !out_count)
    return EMST_ERR_INVALID_ARG;
  *out_count = 0;
  if (capacity == 0) return EMST_OK;
  Extras ex;
  ex.log_feat = out_features;
  ex.log_target = out_targets;
  ex.log_capacity = capacity;
  ex.log_every = every;
  ex.log_count_out = out_count;
  ex.skip_output = true;
  return compute_impl(points, n, dim, nullptr, 1, nullptr, nullptr, (cudaStream_t)stream, nullptr,
                      nullptr, &ex);
}

int emst_core_distances(const float *points, int64_t n, int dim, int k, float *out_core2,
                        void *stream) {
  cudaStream_t s = (cudaStream_t)stream;
  if (!out_core2 || n < 1 || k < 1 || k > n || k > EMST_MRD_MAX_K) return EMST_ERR_INVALID_ARG;
  int rc = check_args(points, n, dim);
  if (rc != EMST_OK) return rc;
  if (n == 1) {  // k = 1: the point itself
    const float zero = 0.0f;
    if (cudaMemcpyAsync(out_core2, &zero, sizeof(float), cudaMemcpyDefault, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return EMST_ERR_CUDA;
    return EMST_OK;
  }
  Session S;
  S.P.want_mrd = true;
  rc = open_session(S, points, n, dim, 1, s);
  if (rc != EMST_OK) return rc;
  Problem &P = S.P;
  run_build(P);
  launch_core_knn(P, k);
  const bool out_dev = device_accessible(out_core2);
  float *dst = out_dev ? out_core2 : reinterpret_cast<float *>(P.keys[1]);  // n floats of scratch
  launch_core_to_input(P, dst);
  if (!out_dev)
    cudaMemcpyAsync(out_core2, dst, sizeof(float) * (size_t)n, cudaMemcpyDeviceToHost, s);
  return finish_session(S);
}

int emst_build_bvh_ex(const float *points, int64_t n, int dim, int leaf_size, int morton_bits,
                      uint64_t *out_codes, uint32_t *out_perm, uint32_t *out_children,
                      float *out_boxes, void *stream) {
  if (morton_bits != 64 && morton_bits != 128) return EMST_ERR_INVALID_ARG;
  Session S;
  S.P.wide = morton_bits == 128;
  cudaStream_t s = (cudaStream_t)stream;
  int rc = open_session(S, points, n, dim, leaf_size, s);
  if (rc != EMST_OK) return rc;
  Problem &P = S.P;
  run_build(P);
  const int64_t m = P.nc - 1;
  if (out_codes && !P.wide)
    cudaMemcpyAsync(out_codes, P.keys[0], 8 * (size_t)n, cudaMemcpyDeviceToDevice, s);
  if (out_codes && P.wide) {  // (high, low) word pairs
    cudaMemcpy2DAsync(out_codes, 16, P.code_hi, 8, 8, (size_t)n, cudaMemcpyDeviceToDevice, s);
    cudaMemcpy2DAsync(out_codes + 1, 16, P.keys[0], 8, 8, (size_t)n, cudaMemcpyDeviceToDevice, s);
  }
  if (out_perm) cudaMemcpyAsync(out_perm, P.perm, 4 * (size_t)n, cudaMemcpyDeviceToDevice, s);
  if (out_children)
    cudaMemcpy2DAsync(out_children, 8, reinterpret_cast<char *>(P.nodes) + 48, 64, 8, (size_t)m,
                      cudaMemcpyDeviceToDevice, s);
  if (out_boxes)
    cudaMemcpy2DAsync(out_boxes, 48, P.nodes, 64, 48, (size_t)m, cudaMemcpyDeviceToDevice, s);
  return finish_session(S);
}

int emst_build_bvh(const float *points, int64_t n, int dim, int leaf_size, uint64_t *out_codes,
                   uint32_t *out_perm, uint32_t *out_children, float *out_boxes, void *stream) {
  return emst_build_bvh_ex(points, n, dim, leaf_size, 64, out_codes, out_perm, out_children,
                           out_boxes, stream);
}

int emst_round_step(const float *points, int64_t n, int dim, int leaf_size,
                    const uint32_t *labels_in, const float *radius_in, uint32_t *out_node_labels,
                    float *out_upper_bound, float *out_nn_w, uint32_t *out_nn_j,
                    uint32_t *out_labels, emst_edge *out_edges, int64_t *out_num_edges,
                    void *stream) {
  if (!labels_in) return EMST_ERR_INVALID_ARG;
  Session S;
  cudaStream_t s = (cudaStream_t)stream;
  int rc = open_session(S, points, n, dim, leaf_size, s);
  if (rc != EMST_OK) return rc;
  Problem &P = S.P;
  run_build(P);
  cudaMemcpyAsync(P.labels, labels_in, 4 * (size_t)n, cudaMemcpyDeviceToDevice, s);
  reset_round_state(P);
  launch_label_runs(P);
  launch_node_labels(P);
  if (out_node_labels)
    cudaMemcpyAsync(out_node_labels, P.nlabels, sizeof(uint2) * (size_t)(P.nc - 1),
                    cudaMemcpyDeviceToDevice, s);
  launch_upper_bounds(P);
  if (out_upper_bound)
    k_bound_to_float<<<grid_for(n, 256), 256, 0, s>>>(P.bound, out_upper_bound, n);
  launch_traverse(P, false, radius_in, 0, false, false);
  if (out_nn_w || out_nn_j) k_split_res<<<grid_for(n, 256), 256, 0, s>>>(P.res, out_nn_w, out_nn_j, n);
  launch_merge(P);
  if (out_labels)
    cudaMemcpyAsync(out_labels, P.labels_buf[P.cur ^ 1], 4 * (size_t)n, cudaMemcpyDeviceToDevice, s);
  uint32_t emitted = 0;
  cudaMemcpyAsync(&emitted, P.counters, 4, cudaMemcpyDeviceToHost, s);
  rc = finish_session(S);
  if (rc != EMST_OK) return rc;
  if (out_edges && emitted)
    cudaMemcpyAsync(out_edges, P.edges, sizeof(emst_edge) * emitted, cudaMemcpyDeviceToDevice, s);
  if (out_num_edges) *out_num_edges = emitted;
  if (cudaStreamSynchronize(s) != cudaSuccess) return EMST_ERR_CUDA;
  return EMST_OK;
}

}  // extern "C"

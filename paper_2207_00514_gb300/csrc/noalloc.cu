// noalloc.cu -- emst_compute_noalloc: the whole EMST with no device
// allocation at all.  For callers that cannot call cudaMalloc (or any pool
// allocator) at the point where they need a spanning tree: a plugin whose
// execute hook must not allocate, code running under a fixed device-memory
// budget owned by someone else, or a latency-critical loop that cannot afford
// an allocator's implicit synchronisation.
//
// All scratch lives in one file-scope device array of fixed size, which every
// GPU that loads this library's module holds until the process exits.  The
// caller still passes the input points and the output edges.
//
// Sharing rules: every call on a device uses the same array, and the array
// keeps whatever the previous call left in it; the path below clears every
// buffer that must start at zero or at a sentinel before it is read.  Two
// calls whose work overlaps on the GPU (different streams or host threads,
// same device) race on the array and both results are undefined: serialise
// them.
#include <cstring>
#include <mutex>

#include "common.cuh"

namespace emst {
namespace {

// Fixed scratch: 16 MiB, enough for EMST_NOALLOC_MAX_POINTS points of either
// dimension including host-copy staging (checked per call against the layout).
constexpr size_t kNoallocScratchBytes = size_t(16) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

// Device address of the array, looked up once per device.  In host code the
// array's name is only a host-side stand-in, so it is never passed to a kernel.
std::mutex g_addr_mu;
void *g_addr[64] = {nullptr};

cudaError_t scratch_address(int dev, void **out) {
  std::lock_guard<std::mutex> lock(g_addr_mu);
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!g_addr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);  // current device == dev
    if (e != cudaSuccess) return e;
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace emst

using namespace emst;

// A CUDA failure: read and clear the runtime's last error (as emst_compute
// does), so the caller's next runtime call does not report this call's error.
static int cuda_failure() {
  cudaGetLastError();
  return EMST_ERR_CUDA;
}

// Codes are always 64-bit here (emst_compute may rebuild with 128-bit codes
// on very dense data; the 128-bit arrays would not fit the fixed scratch at
// the size limit).  The tree does not depend on the code width, only the
// search time on very dense input does.
extern "C" int emst_compute_noalloc(const float *points, int64_t n, int dim, emst_edge *out_edges,
                                    void *stream_) {
  int rc = check_args(points, n, dim);
  if (rc != EMST_OK) return rc;
  if (n > EMST_NOALLOC_MAX_POINTS) return EMST_ERR_TOO_LARGE;
  if (n >= 2 && !out_edges) return EMST_ERR_INVALID_ARG;
  if (n == 0) return EMST_OK;
  cudaStream_t stream = (cudaStream_t)stream_;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return cuda_failure();
  char *base = nullptr;
  if (scratch_address(dev, (void **)&base) != cudaSuccess) return cuda_failure();
  const bool pts_dev = device_accessible(points);
  const bool out_dev = n < 2 || device_accessible(out_edges);
  Problem P;
  P.n = n;
  P.dim = dim;
  P.stream = stream;
  P.points = points;
  P.leaf = effective_leaf(n, 0);
  if (layout(P, nullptr, !pts_dev, !out_dev) > kNoallocScratchBytes) return EMST_ERR_TOO_LARGE;
  layout(P, base, !pts_dev, !out_dev);

  uint32_t host_counters[16] = {0};
  // Launch errors first: a failed launch must not read as a round without edges.
  auto sync_counters = [&]() -> bool {
    if (cudaPeekAtLastError() != cudaSuccess) return false;
    if (cudaMemcpyAsync(host_counters, P.counters, sizeof(host_counters), cudaMemcpyDeviceToHost,
                        stream) != cudaSuccess)
      return false;
    return cudaStreamSynchronize(stream) == cudaSuccess;
  };
  // Counters (edge count, status word, box) start from zero every call.
  if (cudaMemsetAsync(P.counters, 0, sizeof(uint32_t) * 64, stream) != cudaSuccess)
    return cuda_failure();
  if (!pts_dev && cudaMemcpyAsync((void *)P.points, points, sizeof(float) * (size_t)n * dim,
                                  cudaMemcpyHostToDevice, stream) != cudaSuccess)
    return cuda_failure();
  run_build(P);  // clears its own histograms, tile counters, look-back and arrivals
  if (!sync_counters()) return cuda_failure();
  if (host_counters[1] != 0) return status_from_bits(host_counters[1]);
  if (n >= 2) {
    reset_round_state(P);  // bounds and per-component minima back to their sentinels
    const int limit = bits_for(n - 1) + 1;
    for (int round = 0;; ++round) {
      if (round >= limit) return EMST_ERR_ROUND_LIMIT;
      run_round(P, round, true, 0, false);
      if (!sync_counters()) return cuda_failure();
      if (host_counters[1] != 0) return status_from_bits(host_counters[1]);
      advance_round(P, (int64_t)host_counters[12]);
      if ((int64_t)host_counters[0] >= n - 1) break;
    }
    if ((int64_t)host_counters[0] != n - 1) return EMST_ERR_INTERNAL;
    const int orc = run_output(P, out_dev ? out_edges : P.out_stage, host_counters[11]);
    if (orc == EMST_ERR_CUDA) return cuda_failure();
    if (orc != EMST_OK) return orc;
    if (!out_dev && cudaMemcpyAsync(out_edges, P.out_stage, sizeof(emst_edge) * (size_t)(n - 1),
                                    cudaMemcpyDeviceToHost, stream) != cudaSuccess)
      return cuda_failure();
  }
  if (!sync_counters()) return cuda_failure();
  if (cudaGetLastError() != cudaSuccess) return EMST_ERR_CUDA;
  return status_from_bits(host_counters[1]);
}

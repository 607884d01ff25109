// sort.cu -- A3: stable LSD radix sort of (uint64 key, uint32 value) pairs,
// one kernel per 8-bit digit with decoupled look-back ("onesweep"): each CTA
// ranks one tile of keys in shared memory, publishes its per-digit counts,
// looks back over the preceding tiles for their running totals and scatters
// its keys straight to their final positions of that pass.
//
// The paper sorts the Z-curve keys with the search library's device sort
// (§2 "ArborX"); this is an independent GPU sort with the same result (a
// stable order of the codes, equal codes keeping input order).
#include "common.cuh"

namespace emst {

constexpr int kRadix = 256;
constexpr int kWarps = kSortThreads / 32;
static_assert(kSortThreads == kRadix, "a sort pass gives each thread one digit");
constexpr uint32_t kFlagAggregate = 1u << 30;
constexpr uint32_t kFlagPrefix = 2u << 30;
constexpr uint32_t kValueMask = (1u << 30) - 1u;
constexpr int kSpinLimit = 1 << 22;
constexpr int kLookWindow = 8;  // preceding tiles read per look-back round trip

int64_t sort_tiles_for(int64_t n) { return (n + kSortTile - 1) / kSortTile; }

// Histograms of all digits in [digit_begin, digit_end) in one pass.
__global__ void __launch_bounds__(512) k_sort_hist(const uint64_t *__restrict__ keys, int64_t n,
                                                   int digit_begin, int digit_end, int bit0,
                                                   uint32_t *__restrict__ hist) {
  __shared__ uint32_t sh[8][kRadix];
  for (int t = threadIdx.x; t < 8 * kRadix; t += blockDim.x) (&sh[0][0])[t] = 0;
  __syncthreads();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride) {
    uint64_t key = __ldg(keys + k) >> bit0;
    for (int d = digit_begin; d < digit_end; ++d)
      atomicAdd(&sh[d][(uint32_t)(key >> (8 * d)) & 0xffu], 1u);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < 8 * kRadix; t += blockDim.x) {
    uint32_t v = (&sh[0][0])[t];
    if (v) atomicAdd(hist + t, v);
  }
}

// Exclusive scan of each digit's histogram (one CTA of 256 threads per digit).
__global__ void __launch_bounds__(kRadix) k_sort_scan(uint32_t *hist) {
  __shared__ uint32_t warp_sum[kRadix / 32];
  uint32_t *h = hist + blockIdx.x * kRadix;
  int t = threadIdx.x, lane = t & 31, w = t >> 5;
  uint32_t v = h[t];
  uint32_t x = v;
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sum[w] = x;
  __syncthreads();
  uint32_t base = 0;
  for (int q = 0; q < w; ++q) base += warp_sum[q];
  h[t] = base + x - v;
}

struct SortSmem {
  uint64_t keys[kSortTile];
  uint32_t vals[kSortTile];
  uint32_t warp_hist[kWarps][kRadix];
  uint32_t tile_start[kRadix];   // first local position of each digit in the tile
  uint32_t global_base[kRadix];  // global position of local position 0 of each digit
  uint32_t warp_tot[kWarps];
  uint32_t tile_id;
};

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

__global__ void __launch_bounds__(kSortThreads, EMST_SORT_MIN_BLOCKS) k_sort_pass(
    const uint64_t *__restrict__ keys_in, const uint32_t *__restrict__ vals_in,
    uint64_t *__restrict__ keys_out, uint32_t *__restrict__ vals_out, int64_t n, int shift,
    const uint32_t *__restrict__ digit_offset, uint32_t *lookback, uint32_t *tile_counter,
    uint32_t *status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SortSmem &S = *reinterpret_cast<SortSmem *>(smem_raw);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  if (tid == 0) S.tile_id = atomicAdd(tile_counter, 1u);
  for (int t = tid; t < kWarps * kRadix; t += kSortThreads) (&S.warp_hist[0][0])[t] = 0;
  __syncthreads();
  const uint32_t tile = S.tile_id;
  const int64_t base = (int64_t)tile * kSortTile;
  const int64_t seg = base + (int64_t)warp * 32 * kSortItems;

  // Load: warp w owns a contiguous segment; item `it` of lane l sits at
  // seg + it*32 + l, so (it, lane) order is input order within the warp.
  uint64_t key[kSortItems];
  uint32_t val[kSortItems];
  uint32_t rank[kSortItems];
#pragma unroll
  for (int it = 0; it < kSortItems; ++it) {
    int64_t idx = seg + it * 32 + lane;
    bool ok = idx < n;
    key[it] = ok ? keys_in[idx] : 0ull;
    val[it] = ok ? vals_in[idx] : 0u;
  }
  // Rank within the warp, in input order: peers with the same digit in this
  // item, plus the warp's running count of that digit.  The group's leader
  // adds the group size to the warp's counter; the old value is the group's
  // base.  The warp issues the items' adds in order, so item it's base counts
  // exactly the keys of items < it.
  const uint32_t lt = lanemask_lt();
#pragma unroll
  for (int it = 0; it < kSortItems; ++it) {
    int64_t idx = seg + it * 32 + lane;
    bool ok = idx < n;
    uint32_t dg = ok ? (uint32_t)(key[it] >> shift) & 0xffu : 0x100u + lane;
    uint32_t peers = __match_any_sync(0xffffffffu, dg);
    const int leader = __ffs(peers) - 1;
    uint32_t base = 0u;
    if (ok && leader == lane) base = atomicAdd(&S.warp_hist[warp][dg], (uint32_t)__popc(peers));
    base = __shfl_sync(0xffffffffu, base, leader);
    rank[it] = base + __popc(peers & lt);
  }
  __syncthreads();

  // Thread t owns digit t: exclusive prefix over warps, and the tile total.
  const int t = tid;
  uint32_t total = 0;
#pragma unroll
  for (int w = 0; w < kWarps; ++w) {
    uint32_t c = S.warp_hist[w][t];
    S.warp_hist[w][t] = total;
    total += c;
  }
  // Publish this tile's count (tile 0 publishes a finished prefix at once).
  {
    volatile uint32_t *lb = lookback + (int64_t)tile * kRadix + t;
    *lb = (tile == 0 ? kFlagPrefix : kFlagAggregate) | total;
  }
  // Exclusive scan of the totals over digits: local start of each digit.
  uint32_t x = total;
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) S.warp_tot[warp] = x;
  // Look back over preceding tiles for digit t, kLookWindow tiles per round
  // trip: sum their counts in order up to the nearest finished prefix; a
  // tile that has not published yet is waited for.
  uint32_t excl = 0;
  if (tile > 0) {
    int64_t j = (int64_t)tile - 1;
    int spins = 0;
    for (;;) {
      uint32_t wv[kLookWindow];
#pragma unroll
      for (int w = 0; w < kLookWindow; ++w)
        wv[w] = j - w >= 0 ? *reinterpret_cast<const volatile uint32_t *>(lookback + (j - w) * kRadix + t)
                           : kFlagPrefix;  // before tile 0: a finished prefix of 0
      int used = 0;
      bool done = false, stall = false;
#pragma unroll
      for (int w = 0; w < kLookWindow; ++w) {
        if (done || stall) continue;
        const uint32_t f = wv[w] & ~kValueMask;
        if (f == 0u) { stall = true; continue; }
        excl += wv[w] & kValueMask;
        ++used;
        done = f == kFlagPrefix;
      }
      if (done) break;
      j -= used;
      if (stall) {
        if (++spins > kSpinLimit) {  // give up: results are invalid, the status says so
          atomicOr(status, kErrSpin);
          break;
        }
        __nanosleep(32);
      }
    }
    volatile uint32_t *mine = lookback + (int64_t)tile * kRadix + t;
    *mine = kFlagPrefix | ((excl + total) & kValueMask);
  }
  __syncthreads();
  uint32_t wbase = 0;
  for (int q = 0; q < warp; ++q) wbase += S.warp_tot[q];
  const uint32_t start = wbase + x - total;
  S.tile_start[t] = start;
  S.global_base[t] = digit_offset[t] + excl - start;
  __syncthreads();

  // Scatter into shared memory in tile-sorted order.
#pragma unroll
  for (int it = 0; it < kSortItems; ++it) {
    int64_t idx = seg + it * 32 + lane;
    if (idx < n) {
      uint32_t dg = (uint32_t)(key[it] >> shift) & 0xffu;
      uint32_t pos = S.tile_start[dg] + S.warp_hist[warp][dg] + rank[it];
      S.keys[pos] = key[it];
      S.vals[pos] = val[it];
    }
  }
  __syncthreads();
  // Write out: consecutive threads write consecutive positions of a digit run.
  int64_t count = n - base < kSortTile ? n - base : kSortTile;
  for (int i = tid; i < count; i += kSortThreads) {
    uint64_t k = S.keys[i];
    uint32_t dg = (uint32_t)(k >> shift) & 0xffu;
    uint32_t out = S.global_base[dg] + (uint32_t)i;
    keys_out[out] = k;
    vals_out[out] = S.vals[i];
  }
}

static bool g_sort_attr_set[64] = {false};

int radix_sort_pairs(Problem &P, int64_t n, int digit_begin, int digit_end, int src, int bit0) {
  if (n <= 1 || digit_begin >= digit_end) return src;
  cudaStream_t s = P.stream;
  int dev = 0;
  cudaGetDevice(&dev);
  const size_t smem = sizeof(SortSmem);
  if (dev < 64 && !g_sort_attr_set[dev]) {
    cudaFuncSetAttribute(k_sort_pass, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    g_sort_attr_set[dev] = true;
  }
  uint32_t *hist = P.sort_hist;
  uint32_t *tile_ctr = P.counters + 16;
  cudaMemsetAsync(hist, 0, sizeof(uint32_t) * 8 * kRadix, s);
  cudaMemsetAsync(tile_ctr, 0, sizeof(uint32_t) * 8, s);
  int hgrid = (int)((n + 511) / 512);
  if (hgrid > sm_count() * 4) hgrid = sm_count() * 4;
  k_sort_hist<<<hgrid, 512, 0, s>>>(P.keys[src], n, digit_begin, digit_end, bit0, hist);
  k_sort_scan<<<8, kRadix, 0, s>>>(hist);
  P.launches += 2;
  const int64_t tiles = sort_tiles_for(n);
  for (int d = digit_begin; d < digit_end; ++d) {
    cudaMemsetAsync(P.sort_lookback, 0, sizeof(uint32_t) * kRadix * tiles, s);
    k_sort_pass<<<(unsigned)tiles, kSortThreads, smem, s>>>(
        P.keys[src], P.vals[src], P.keys[src ^ 1], P.vals[src ^ 1], n, bit0 + 8 * d, hist + d * kRadix,
        P.sort_lookback, tile_ctr + d, P.counters + 1);
    P.launches += 1;
    src ^= 1;
  }
  return src;
}

}  // namespace emst

// Stable bucket sort of caller-owned device keys with no device allocation:
// the counting sort of the re-bin (Section 4, the fresh-particle case where
// every particle is a mover) on scratch that lives in a file-scope device
// array instead of memory obtained from the allocator.
//
// The call clears every part of the scratch it reads before using it, on the
// caller's stream, so nothing has to be zero on entry.  One array per device
// serves every caller of the process: calls that overlap in time (different
// streams or host threads on one device) race on it.  Buckets are put in
// input order by a per-thread insertion sort up to 32 elements and by an
// in-place bitonic network above (O(m log^2 m), no extra memory), so a call
// with few keys and many elements stays fast.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <mutex>

#include "../../include/pic.h"
#include "launch.hpp"
#include "segsort.cuh"

namespace pic {
namespace {

// Scratch layout: counts (later fill cursors, later the list of crowded
// buckets) | scan tile sums | scan total | crowded-bucket count | spare.
constexpr int64_t kMaxTiles = (PIC_NOALLOC_MAX_KEYS + kScanTileElems - 1) / kScanTileElems;
constexpr int64_t kScratchWords = PIC_NOALLOC_MAX_KEYS + 192;
static_assert(kMaxTiles + 2 < 192, "scan tile sums and totals overrun the scratch tail");

static __device__ __align__(256) int32_t g_bucket_scratch[kScratchWords];

constexpr int kMaxDevices = 256;
std::mutex g_scratch_mu;
int32_t *g_scratch_addr[kMaxDevices] = {};

// Address of this device's scratch array, looked up once per device.
int scratch_of_current_device(int32_t **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return PIC_ECUDA;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_bucket_scratch) != cudaSuccess || !p) return PIC_ECUDA;
    g_scratch_addr[dev] = static_cast<int32_t *>(p);
  }
  *out = g_scratch_addr[dev];
  return PIC_OK;
}

__global__ void k_na_count(const int32_t *keys, int64_t n, int64_t n_keys, int32_t *count) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int32_t k = keys[i];
    if (k >= 0 && k < n_keys) atomicAdd(&count[k], 1);
  }
}

__global__ void k_na_fill(const int32_t *keys, int64_t n, int64_t n_keys, const int32_t *start, int32_t *cursor,
                          int32_t *perm) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int32_t k = keys[i];
    if (k >= 0 && k < n_keys) perm[start[k] + atomicAdd(&cursor[k], 1)] = (int32_t)i;
  }
}

// Restores input order inside every bucket (the fill's atomic order is
// arbitrary): buckets of at most kSmallBucket elements by one thread, longer
// ones are listed for k_na_order_large.
constexpr int kSmallBucket = 32;
__global__ void k_na_order(const int32_t *start, int64_t n_keys, int32_t *perm, int32_t *large, int32_t *n_large) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_keys) return;
  const int32_t b = start[k], e = start[k + 1];
  if (e - b > kSmallBucket) {
    large[atomicAdd(n_large, 1)] = (int32_t)k;
    return;
  }
  for (int32_t i = b + 1; i < e; ++i) {
    int32_t x = perm[i], j = i - 1;
    while (j >= b && perm[j] > x) {
      perm[j + 1] = perm[j];
      --j;
    }
    perm[j + 1] = x;
  }
}

// One block per crowded bucket (grid-stride over the list): in-place bitonic
// network, chunks of kOrderChunk in shared memory; O(m log^2 m) for a bucket
// of m elements, no memory beyond the bucket's own range of perm.
constexpr int kOrderThreads = 1024;
constexpr int kOrderChunk = 8192;
__global__ void __launch_bounds__(kOrderThreads) k_na_order_large(const int32_t *start, const int32_t *large,
                                                                  const int32_t *n_large, int32_t *perm) {
  __shared__ int32_t sk[kOrderChunk];
  const int nl = *n_large;
  for (int li = blockIdx.x; li < nl; li += gridDim.x) {
    const int32_t k = large[li];
    const int32_t b = start[k], m = start[k + 1] - b;
    block_sort_global<int32_t, int32_t>(perm + b, nullptr, m, sk, nullptr, kOrderChunk);
    __syncthreads();
  }
}

}  // namespace
}  // namespace pic

using namespace pic;

extern "C" int pic_bucket_noalloc(const int32_t *keys, int64_t n, int64_t n_keys, int32_t *start, int32_t *perm,
                                  void *stream) {
  if (n < 0 || n > INT32_MAX || n_keys < 1 || !start || (n > 0 && (!keys || !perm))) return PIC_EINVAL;
  if (n_keys > PIC_NOALLOC_MAX_KEYS) return PIC_EINVAL;  // above the fixed scratch
  int32_t *scratch = nullptr;
  int rc = scratch_of_current_device(&scratch);
  if (rc) return rc;
  int32_t *count = scratch;
  int32_t *tile_sums = scratch + PIC_NOALLOC_MAX_KEYS;
  int32_t *total = tile_sums + kMaxTiles;
  int32_t *n_large = total + 1;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int threads = 256;
  const unsigned grid = (unsigned)(n > 0 ? std::min<int64_t>((n + threads - 1) / threads, 152 * 8) : 1);
  if (cudaMemsetAsync(count, 0, sizeof(int32_t) * n_keys, s) != cudaSuccess) return PIC_ECUDA;
  k_na_count<<<grid, threads, 0, s>>>(keys, n, n_keys, count);
  launch_exclusive_scan(count, n_keys, start, tile_sums, total, s);
  if (cudaMemsetAsync(count, 0, sizeof(int32_t) * n_keys, s) != cudaSuccess) return PIC_ECUDA;
  k_na_fill<<<grid, threads, 0, s>>>(keys, n, n_keys, start, count, perm);
  if (cudaMemsetAsync(n_large, 0, sizeof(int32_t), s) != cudaSuccess) return PIC_ECUDA;
  k_na_order<<<(unsigned)((n_keys + threads - 1) / threads), threads, 0, s>>>(start, n_keys, perm, count, n_large);
  k_na_order_large<<<152, kOrderThreads, 0, s>>>(start, count, n_large, perm);
  count_launches(4);
  return cudaGetLastError() == cudaSuccess ? PIC_OK : PIC_ECUDA;
}

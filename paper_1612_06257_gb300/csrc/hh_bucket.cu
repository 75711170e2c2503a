// hh_bucket.cu -- length bucketing of a ragged batch (work-queue order).
//
// A message of length L needs P = ceil(L / 32) Updates before finalisation
// (one per whole 32-byte packet plus one for a partial packet, Sections 4.2
// and 4.5).  Messages are counting-sorted by bucket(P) in DESCENDING order:
// bucket = P below 2048 packets (64 KiB), then 128 buckets per doubling of P
// (steps under 1%), up to messages of 4 GiB.  A warp tile thus holds
// messages of (nearly) equal Update count, so no lane waits on another, and
// tiles are handed out longest first, so the long ones cannot end up last.
// The scan also counts the messages of a given bucket and above (by default
// kHugeBucket, 128 KiB), which the hash kernel runs two threads per message.
//
// Three kernels: per-block histograms merged with one global atomic per
// non-empty bucket (for one-key offsets-form batches above 8192 messages
// this count runs inside the short kernel instead: hh_count.h); a one-block exclusive scan in descending bucket order
// (which also resets the tile counter of the work queue); and a scatter that
// ranks elements inside each 8192-element chunk in shared memory and reserves
// each bucket's range with one global atomic per chunk.  A batch of at most
// one chunk is sorted by a single block in one launch.  The order inside a
// bucket depends on atomic timing; results do not, because every message's
// hash is stored at its own index.
#include <cuda_runtime.h>

#include <cstdint>

#include "hh_batch.cuh"
#include "hh_count.h"
#include "hh_internal.h"

namespace hh {
namespace {

constexpr int kSortThreads = 1024;
constexpr int kPerThread = 8;
constexpr int kChunk = kSortThreads * kPerThread;

__device__ __forceinline__ int bucket_of(const Batch& b, int64_t i) {
  const int64_t len = message_length(b, i);
  if (len <= 0) return 0;  // empty, or invalid (reported by the hash kernel)
  return bucket_of_packets((len + 31) >> 5);
}

// Buckets of this thread's kPerThread elements of chunk c (-1 past n).  In
// the plain offsets form every offset is loaded first, unconditionally (at
// a clamped index), so that all the loads are in flight together; the
// general form goes through message_length one element at a time.
__device__ __forceinline__ void bucket_keys(const Batch& b, int64_t n, int64_t c,
                                            int key[kPerThread]) {
  if (n > 0 && b.offsets != nullptr && b.key_index == nullptr && b.stream_mode != kStreamUpdate) {
    int64_t s[kPerThread], e[kPerThread];
#pragma unroll
    for (int k = 0; k < kPerThread; ++k) {
      const int64_t i = c + k * kSortThreads + threadIdx.x;
      const int64_t j = i < n ? i : n - 1;
      s[k] = b.offsets[j];
      e[k] = b.offsets[j + 1];
    }
#pragma unroll
    for (int k = 0; k < kPerThread; ++k) {
      const int64_t i = c + k * kSortThreads + threadIdx.x;
      const int64_t len = e[k] - s[k];  // negative: a bad descriptor, hashed as empty
      key[k] = i >= n ? -1 : len <= 0 ? 0 : bucket_of_packets((len + 31) >> 5);
    }
    return;
  }
#pragma unroll
  for (int k = 0; k < kPerThread; ++k) {
    const int64_t i = c + k * kSortThreads + threadIdx.x;
    key[k] = i < n ? bucket_of(b, i) : -1;
  }
}

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Buckets 0 .. kRegBuckets - 1 (messages of at most 96 bytes) are counted
// in registers and reduced once per warp: batches of short messages would
// otherwise send every element through the warp-aggregated atomics.
constexpr int kRegBuckets = 4;

__global__ void __launch_bounds__(kSortThreads) bucket_count_kernel(Batch b, uint32_t* hist) {
  resolve_count(b);
  const int64_t n = b.n;
  __shared__ uint32_t h[kBuckets];
  for (int i = threadIdx.x; i < kBuckets; i += kSortThreads) h[i] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  uint32_t small[kRegBuckets] = {};
  for (int64_t c = static_cast<int64_t>(blockIdx.x) * kChunk; c < n;
       c += static_cast<int64_t>(gridDim.x) * kChunk) {
    int keys[kPerThread];
    bucket_keys(b, n, c, keys);
#pragma unroll
    for (int e = 0; e < kPerThread; ++e) {
      const int key = keys[e];
#pragma unroll
      for (int q = 0; q < kRegBuckets; ++q) small[q] += key == q ? 1u : 0u;
      const int big = key >= kRegBuckets ? key : -1;
      if (__any_sync(0xffffffffu, big >= 0)) {
        const unsigned peers = __match_any_sync(0xffffffffu, big);
        if (big >= 0 && lane == __ffs(peers) - 1) atomicAdd(&h[big], __popc(peers));
      }
    }
  }
#pragma unroll
  for (int q = 0; q < kRegBuckets; ++q) {
    uint32_t v = small[q];
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
    if (lane == 0 && v) atomicAdd(&h[q], v);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kBuckets; i += kSortThreads)
    if (h[i]) atomicAdd(&hist[i], h[i]);
}

// Exclusive scan of counts[] in descending bucket order: cursor[k] = number
// of messages in buckets above k.  Also resets the work queue's counters
// next_tile[0..3] (warp tiles, huge-prefix claims, launch bookkeeping); writes the number of messages in buckets >=
// huge_bucket (the huge count; 0 when huge_bucket >= kBuckets) and the
// use-order flag (1 when some message is longer than kShortMax), and returns
// that flag.  Called by all kSortThreads threads of one block; counts and
// cursor may be shared or global memory.
__device__ __forceinline__ int scan_descending(const uint32_t* counts, uint32_t* cursor,
                                               unsigned long long* next_tile, int* use_perm,
                                               long long* huge_count, int huge_bucket) {
  constexpr int kPer = kBuckets / kSortThreads;  // 4 buckets per thread
  __shared__ uint32_t warp_sums[kSortThreads / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // Thread tid owns descending positions tid*kPer .. tid*kPer + kPer - 1,
  // i.e. buckets kBuckets-1-pos.
  uint32_t v[kPer];
  uint32_t local = 0;
#pragma unroll
  for (int j = 0; j < kPer; ++j) {
    v[j] = counts[kBuckets - 1 - (tid * kPer + j)];
    local += v[j];
  }
  uint32_t incl = local;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t x = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += x;
  }
  if (lane == 31) warp_sums[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = warp_sums[lane];
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t x = __shfl_up_sync(0xffffffffu, w, d);
      if (lane >= d) w += x;
    }
    warp_sums[lane] = w;  // inclusive over warps
  }
  __syncthreads();
  uint32_t run = incl - local + (warp > 0 ? warp_sums[warp - 1] : 0u);
#pragma unroll
  for (int j = 0; j < kPer; ++j) {
    const int bucket = kBuckets - 1 - (tid * kPer + j);
    cursor[bucket] = run;
    run += v[j];
    // Messages in buckets >= huge_bucket: everything up to and including it
    // in descending order.
    if (bucket == huge_bucket) *huge_count = static_cast<long long>(run);
  }
  if (tid == 0) {
    next_tile[0] = 0ull;
    next_tile[1] = 0ull;
    next_tile[2] = 0ull;  // launch bookkeeping of the hash kernel
    next_tile[3] = 0ull;
    if (huge_bucket >= kBuckets) *huge_count = 0;  // huge messages switched off
  }
  // Buckets above kShortMax / 32 hold messages longer than kShortMax bytes.
  const int long_bucket = kShortMax / 32 + 1;
  bool mine = false;
#pragma unroll
  for (int j = 0; j < kPer; ++j)
    mine |= v[j] != 0 && kBuckets - 1 - (tid * kPer + j) >= long_bucket;
  const int any_long = __syncthreads_or(mine);
  if (tid == 0) *use_perm = any_long;
  return any_long;
}

__global__ void __launch_bounds__(kSortThreads) bucket_scan_kernel(const uint32_t* hist,
                                                                   uint32_t* cursor,
                                                                   unsigned long long* next_tile,
                                                                   int* use_perm,
                                                                   long long* huge_count,
                                                                   int huge_bucket) {
  scan_descending(hist, cursor, next_tile, use_perm, huge_count, huge_bucket);
}

// Ranks of chunk elements c .. c + kChunk - 1 inside their buckets: counts
// into cnt[] (shared, zeroed by the caller) and returns each element's key
// (-1 past the end) and rank.  kMergeShort: buckets 0..2 (messages of at
// most kShortMax bytes) are one bucket, 2, as the count inside the short
// kernel makes them.
template <bool kMergeShort>
__device__ __forceinline__ void rank_chunk(const Batch& b, int64_t n, int64_t c, uint32_t* cnt,
                                           int key[kPerThread], uint32_t rank[kPerThread]) {
  const int lane = threadIdx.x & 31;
  bucket_keys(b, n, c, key);
  if (kMergeShort) {
    constexpr int kShortBucket = kShortMax / 32;
#pragma unroll
    for (int e = 0; e < kPerThread; ++e)
      key[e] = key[e] >= 0 && key[e] < kShortBucket ? kShortBucket : key[e];
  }
#pragma unroll
  for (int e = 0; e < kPerThread; ++e) {
    const unsigned peers = __match_any_sync(0xffffffffu, key[e]);
    const int leader = __ffs(peers) - 1;
    uint32_t first = 0;
    if (key[e] >= 0 && lane == leader) first = atomicAdd(&cnt[key[e]], __popc(peers));
    first = __shfl_sync(0xffffffffu, first, leader);
    rank[e] = first + __popc(peers & lanemask_lt());
  }
}

// The whole sort of a batch of at most kChunk messages in one block: rank
// in shared memory, scan, scatter.
__global__ void __launch_bounds__(kSortThreads) bucket_small_kernel(
    Batch b, int32_t* perm, unsigned long long* next_tile, int* use_perm,
    long long* huge_count, int huge_bucket) {
  resolve_count(b);
  const int64_t n = b.n < kChunk ? b.n : kChunk;  // the host checked b.n <= kChunk
  __shared__ uint32_t cnt[kBuckets];
  __shared__ uint32_t base[kBuckets];
  for (int i = threadIdx.x; i < kBuckets; i += kSortThreads) cnt[i] = 0;
  __syncthreads();
  int key[kPerThread];
  uint32_t rank[kPerThread];
  rank_chunk<false>(b, n, 0, cnt, key, rank);
  __syncthreads();
  if (!scan_descending(cnt, base, next_tile, use_perm, huge_count, huge_bucket)) return;
#pragma unroll
  for (int e = 0; e < kPerThread; ++e) {
    const int64_t i = e * kSortThreads + threadIdx.x;
    if (key[e] >= 0) perm[base[key[e]] + rank[e]] = static_cast<int32_t>(i);
  }
}

template <bool kMergeShort>
__global__ void __launch_bounds__(kSortThreads) bucket_scatter_kernel(Batch b, uint32_t* cursor,
                                                                      int32_t* perm,
                                                                      const int* use_perm) {
  if (*use_perm == 0) return;
  resolve_count(b);
  const int64_t n = b.n;
  __shared__ uint32_t cnt[kBuckets];
  __shared__ uint32_t base[kBuckets];
  for (int64_t c = static_cast<int64_t>(blockIdx.x) * kChunk; c < n;
       c += static_cast<int64_t>(gridDim.x) * kChunk) {
    for (int i = threadIdx.x; i < kBuckets; i += kSortThreads) cnt[i] = 0;
    __syncthreads();
    int key[kPerThread];
    uint32_t rank[kPerThread];
    rank_chunk<kMergeShort>(b, n, c, cnt, key, rank);
    __syncthreads();
    for (int i = threadIdx.x; i < kBuckets; i += kSortThreads)
      if (cnt[i]) base[i] = atomicAdd(&cursor[i], cnt[i]);
    __syncthreads();
#pragma unroll
    for (int e = 0; e < kPerThread; ++e) {
      const int64_t i = c + e * kSortThreads + threadIdx.x;
      if (key[e] >= 0) perm[base[key[e]] + rank[e]] = static_cast<int32_t>(i);
    }
    __syncthreads();
  }
}

}  // namespace

namespace {

int sort_grid(int64_t n, int num_sms) {
  const int64_t chunks = (n + kChunk - 1) / kChunk;
  const int64_t cap = static_cast<int64_t>(num_sms) * 2;
  return static_cast<int>(chunks < cap ? chunks : cap);
}

}  // namespace

cudaError_t launch_bucket_scan_scatter(const Batch& b, uint32_t* hist, uint32_t* cursor,
                                       int32_t* perm, unsigned long long* next_tile,
                                       int* use_perm, long long* huge_count, int huge_bucket,
                                       int num_sms, cudaStream_t stream, int* launches) {
  bucket_scan_kernel<<<1, kSortThreads, 0, stream>>>(hist, cursor, next_tile, use_perm,
                                                      huge_count, huge_bucket);
  const int grid = sort_grid(b.n, num_sms);
  if (grid > 0)
    bucket_scatter_kernel<true><<<grid, kSortThreads, 0, stream>>>(b, cursor, perm, use_perm);
  *launches += grid > 0 ? 2 : 1;
  return cudaGetLastError();
}

cudaError_t launch_bucket_sort(const Batch& b, uint32_t* hist,
                               uint32_t* cursor, int32_t* perm, unsigned long long* next_tile,
                               int* use_perm, long long* huge_count, int huge_bucket,
                               int num_sms, cudaStream_t stream, int* launches) {
  const int64_t n = b.n;
  if (n <= kChunk) {
    bucket_small_kernel<<<1, kSortThreads, 0, stream>>>(b, perm, next_tile, use_perm, huge_count,
                                                         huge_bucket);
    *launches += 1;
    return cudaGetLastError();
  }
  cudaError_t e = cudaMemsetAsync(hist, 0, sizeof(uint32_t) * kBuckets, stream);
  if (e != cudaSuccess) return e;
  const int grid = sort_grid(n, num_sms);
  bucket_count_kernel<<<grid, kSortThreads, 0, stream>>>(b, hist);
  bucket_scan_kernel<<<1, kSortThreads, 0, stream>>>(hist, cursor, next_tile, use_perm,
                                                      huge_count, huge_bucket);
  bucket_scatter_kernel<false><<<grid, kSortThreads, 0, stream>>>(b, cursor, perm, use_perm);
  *launches += 3;
  return cudaGetLastError();
}

}  // namespace hh

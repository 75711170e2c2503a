// hh_api.cu -- the C ABI of libhh (declared in include/hh.h).
//
// Host-side only: argument checks, kernel choice, scratch memory for the
// length sort, and the chunked host-buffer path.  Every step of the hash
// itself runs in the kernels of hh_kernels.cu and hh_bucket.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "hh.h"
#include "hh_context.h"
#include "hh_count.h"
#include "hh_internal.h"

namespace {

// Every ragged batch is length-sorted (one launch up to 8192 messages): the
// sort also finds the long messages that run two threads each.
constexpr int64_t kSortMinMessages = 1;
constexpr int64_t kMaxSortedMessages = 0x7FFFFFFFll;
constexpr int64_t kShortKernelMinMessages = 8192;  // smaller batches: warp-tile kernel only
constexpr int64_t kFixedRows = 128;                // messages per TMA tile at one per thread
constexpr size_t kHostChunkBytes = size_t(128) << 20;  // payload per host-path chunk
constexpr int64_t kHostChunkMessages = int64_t(1) << 20;

using hh::DeviceGuard;

int to_status(cudaError_t e) {
  if (e == cudaSuccess) return HH_OK;
  if (e == cudaErrorMemoryAllocation) return HH_ERR_NO_MEMORY;
  return HH_ERR_CUDA;
}

// Grow the length sort's message-order scratch to `n` entries.  Only
// hh_init and hh_reserve call this: the hash calls themselves never allocate
// (a batch beyond the reserved size returns HH_ERR_TOO_LARGE instead).
int reserve_perm(hh_ctx* ctx, int64_t n) {
  if (n <= ctx->perm_cap) return HH_OK;
  if (ctx->d_perm) {
    // The old array may still be read by work queued on any stream.
    if (cudaDeviceSynchronize() != cudaSuccess) return HH_ERR_CUDA;
    cudaFree(ctx->d_perm);
  }
  ctx->d_perm = nullptr;
  ctx->perm_cap = 0;
  if (cudaMalloc(&ctx->d_perm, sizeof(int32_t) * static_cast<size_t>(n)) != cudaSuccess)
    return HH_ERR_NO_MEMORY;
  ctx->perm_cap = n;
  return HH_OK;
}

int words_of(int bits) { return bits == 64 ? 1 : bits == 128 ? 2 : bits == 256 ? 4 : 0; }

// Enqueue the hash of one device batch `b` (offsets, fixed or segments
// form; the caller has checked its arguments and filled b).
int hash_device(hh_ctx* ctx, hh::Batch b, cudaStream_t stream) {
  ctx->last_launches = 0;
  if (b.n == 0) return HH_OK;
  DeviceGuard guard(ctx->device);
  if (!guard.ok) return HH_ERR_CUDA;
  b.err = ctx->d_err;
  b.wait_ns = ctx->wait_limit_ns;
  const int64_t n = b.n;
  const bool fixed = b.offsets == nullptr && b.seg_start == nullptr;

  if (b.stream_mode != hh::kWholeMessages &&
      (ctx->kernel == HH_KERNEL_NAIVE || ctx->kernel == HH_KERNEL_STAGED_BULK))
    return HH_ERR_INVALID_ARG;  // streams run in the warp-tile and short kernels only
  if (ctx->kernel == HH_KERNEL_NAIVE) {
    ctx->last_launches = 1;
    return to_status(hh::launch_naive(b, stream));
  }
  if (fixed && b.key_index == nullptr && hh::fixed_tma_supported(b.bytes, b.fixed_len, n)) {
    const hh::StagedShape shape = ctx->tune.fixed[hh::fixed_class(b.fixed_len)];
    ctx->last_launches = 1;
    // A batch too small to give every SM a tile is latency bound: it runs
    // 256-byte windows, two threads per message (each chain half as long)
    // or one.
    if (!ctx->tuning && n < static_cast<int64_t>(ctx->num_sms) * kFixedRows * shape.msgs)
      return to_status(ctx->tune.fixed_pair
                           ? hh::launch_fixed_tma_pair(b, ctx->num_sms, stream)
                           : hh::launch_fixed_tma(b, hh::StagedShape{256, 2, 1}, ctx->num_sms,
                                                  stream));
    return to_status(hh::launch_fixed_tma(b, shape, ctx->num_sms, stream));
  }

  const bool sort = !fixed && ctx->kernel != HH_KERNEL_STAGED_UNSORTED && n >= kSortMinMessages;
  const bool with_short = sort && ctx->kernel != HH_KERNEL_STAGED_BULK && n > kShortKernelMinMessages;
  // One-key offsets-form batches count their lengths inside the short
  // kernel (hh_count.h): one pass over the offsets fewer.
  const bool counted_short = with_short && hh::short_count_eligible(b);
  hh::Queue q{};
  if (sort) {
    // The batch must fit the scratch reserved by hh_init / hh_reserve.
    if (n > ctx->perm_cap) return HH_ERR_TOO_LARGE;
    int launches = 0;
    cudaError_t e;
    if (counted_short) {
      e = cudaMemsetAsync(ctx->d_hist, 0, sizeof(uint32_t) * (hh::kBuckets + 2), stream);
      if (e == cudaSuccess) e = hh::launch_short_counted(b, ctx->d_hist, ctx->num_sms, stream);
      if (e == cudaSuccess)
        e = hh::launch_bucket_scan_scatter(b, ctx->d_hist, ctx->d_cursor, ctx->d_perm,
                                           ctx->d_next_tile, ctx->d_use_perm, ctx->d_huge,
                                           ctx->tune.huge_bucket, ctx->num_sms, stream, &launches);
      launches += 1;
    } else {
      e = hh::launch_bucket_sort(b, ctx->d_hist, ctx->d_cursor, ctx->d_perm, ctx->d_next_tile,
                                 ctx->d_use_perm, ctx->d_huge, ctx->tune.huge_bucket,
                                 ctx->num_sms, stream, &launches);
    }
    ctx->last_launches += launches;
    if (e != cudaSuccess) return to_status(e);
    q.perm = ctx->d_perm;
    q.use_perm = ctx->d_use_perm;
    q.huge_count = ctx->d_huge;
    q.next_tile = ctx->d_next_tile;
  }
  cudaError_t e;
  if (ctx->kernel == HH_KERNEL_STAGED_BULK) {
    // Earlier design: 128-message CTA tiles, one bulk copy per thread.
    q.tiles = (n + hh::kTileRows - 1) / hh::kTileRows;
    const bool aligned16 = fixed && (reinterpret_cast<uintptr_t>(b.bytes) % 16 == 0) &&
                           (b.fixed_len % 16 == 0);
    e = hh::launch_staged(b, q, ctx->shape_bulk, aligned16, ctx->num_sms, stream);
  } else {
    if (with_short) {
      // All-short batches (the sort's flag says no message is longer than
      // kShortMax) run in the short kernel; otherwise it returns at once and
      // the warp-tile kernel runs.  Both are enqueued, so the sequence of
      // launches does not depend on the data.  Small batches skip the short
      // kernel: the warp-tile kernel hashes all-short tiles without shared
      // memory too, and one launch fewer matters more there.  (With the
      // count inside the short kernel, it ran before the sort's scan.)
      if (!counted_short) {
        e = hh::launch_short(b, ctx->d_use_perm, ctx->num_sms, stream);
        if (e != cudaSuccess) return to_status(e);
        ctx->last_launches += 1;
      }
      q.skip_if_short = 1;
    }
    // The grid is sized for warp tiles of 32, or for up to solo_max solo
    // tiles (one message each) when that is more; solo and pair tiles are
    // taken from the same queue by the same persistent CTAs.
    q.solo_max = sort ? static_cast<int64_t>(ctx->tune.solo_per_sm) * ctx->num_sms : 0;
    q.solo_ctas = static_cast<int>((q.solo_max + hh::kRaggedWarps - 1) / hh::kRaggedWarps);
    q.solo_shared = ctx->tune.solo_shared;
    q.tiles = std::max((n + 31) / 32, std::min(n, q.solo_max));
    e = hh::launch_ragged(b, q, ctx->tune.ragged, ctx->num_sms, stream);
    if (q.skip_if_short) ctx->last_launches += 1;  // two warp-tile variants, one runs
  }
  ctx->last_launches += 1;
  return to_status(e);
}

// Argument checks and Batch set-up shared by the offsets and fixed forms.
int hash_common(hh_ctx* ctx, int bits, const uint64_t* keys, int key_mode, const uint8_t* bytes,
                const int64_t* offsets, int64_t fixed_len, int64_t n, uint64_t* out,
                cudaStream_t stream) {
  if (ctx == nullptr) return HH_ERR_INVALID_ARG;
  const int words = words_of(bits);
  if (words == 0 || (key_mode != HH_KEY_SHARED && key_mode != HH_KEY_PER_MESSAGE) || n < 0 ||
      fixed_len < 0)
    return HH_ERR_INVALID_ARG;
  ctx->last_launches = 0;
  if (n == 0) return HH_OK;
  if (keys == nullptr || out == nullptr) return HH_ERR_INVALID_ARG;
  // Only a fixed-length batch of empty messages may come without bytes.
  if (bytes == nullptr && !(offsets == nullptr && fixed_len == 0)) return HH_ERR_INVALID_ARG;
  if (offsets == nullptr && fixed_len > 0 && n > INT64_MAX / fixed_len) return HH_ERR_TOO_LARGE;
  hh::Batch b{};
  b.bytes = bytes;
  b.offsets = offsets;
  b.fixed_len = fixed_len;
  b.keys = keys;
  b.per_message_keys = key_mode == HH_KEY_PER_MESSAGE;
  b.n = n;
  b.out = out;
  b.words = words;
  return hash_device(ctx, b, stream);
}

// Grow one device buffer of the host-buffer path, stream-ordered on the
// context's copy stream: the old buffer is released after everything queued
// there (which includes the slot's last use), and nothing outside the
// context's own streams waits.
template <typename T>
int grow(T** p, size_t* cap, size_t need, cudaStream_t s) {
  if (need <= *cap) return HH_OK;
  const size_t want = std::max(need, *cap + *cap / 2);
  if (*p) cudaFreeAsync(*p, s);
  *p = nullptr;
  *cap = 0;
  if (cudaMallocAsync(reinterpret_cast<void**>(p), want * sizeof(T), s) != cudaSuccess)
    return HH_ERR_NO_MEMORY;
  *cap = want;
  return HH_OK;
}

struct OccupancyEntry {
  const void* kern;
  int device, threads, smem, per_sm;
};
std::mutex g_occupancy_mu;
std::vector<OccupancyEntry> g_occupancy;

}  // namespace

namespace hh {

int blocks_per_sm(const void* kern, int threads, int smem, cudaError_t* err) {
  *err = cudaSuccess;
  int dev = 0;
  if ((*err = cudaGetDevice(&dev)) != cudaSuccess) return 0;
  {
    std::lock_guard<std::mutex> lock(g_occupancy_mu);
    for (const OccupancyEntry& e : g_occupancy)
      if (e.kern == kern && e.device == dev && e.threads == threads && e.smem == smem)
        return e.per_sm;
  }
  if (smem > 0 &&
      (*err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) !=
          cudaSuccess)
    return 0;
  int per_sm = 0;
  if ((*err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem)) !=
      cudaSuccess)
    return 0;
  if (per_sm < 1) per_sm = 1;
  std::lock_guard<std::mutex> lock(g_occupancy_mu);
  g_occupancy.push_back({kern, dev, threads, smem, per_sm});
  return per_sm;
}

}  // namespace hh

extern "C" {

const char* hh_status_string(int status) {
  switch (status) {
    case HH_OK: return "ok";
    case HH_ERR_INVALID_ARG: return "invalid argument";
    case HH_ERR_CUDA: return "CUDA runtime error";
    case HH_ERR_NO_MEMORY: return "out of memory";
    case HH_ERR_TIMEOUT: return "device pipeline wait timed out";
    case HH_ERR_TOO_LARGE: return "size too large for this call";
    case HH_ERR_BAD_OFFSETS: return "offsets decrease";
    case HH_ERR_NO_DEVICE: return "no usable sm_103 CUDA device";
    case HH_ERR_BAD_KEY_INDEX: return "key index outside the key table";
    case HH_ERR_BAD_CHUNK: return "stream chunk length not a multiple of 32 bytes";
    default: return "unknown status";
  }
}

int hh_init(hh_ctx** out, int device, const char* tune_cache_path) {
  if (out == nullptr) return HH_ERR_INVALID_ARG;
  *out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count)
    return HH_ERR_NO_DEVICE;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return HH_ERR_NO_DEVICE;
  if (prop.major != 10 || prop.minor != 3) return HH_ERR_NO_DEVICE;
  DeviceGuard guard(device);
  if (!guard.ok) return HH_ERR_CUDA;
  hh_ctx* ctx = new (std::nothrow) hh_ctx();
  if (ctx == nullptr) return HH_ERR_NO_MEMORY;
  ctx->device = device;
  ctx->num_sms = prop.multiProcessorCount;
  if (tune_cache_path != nullptr && !hh::load_tune_table(tune_cache_path, ctx->tune)) {
    delete ctx;
    return HH_ERR_INVALID_ARG;
  }
  bool ok = cudaMalloc(&ctx->d_err, sizeof(int)) == cudaSuccess &&
            cudaMalloc(&ctx->d_next_tile, 4 * sizeof(unsigned long long)) == cudaSuccess &&
            cudaMalloc(&ctx->d_use_perm, sizeof(int)) == cudaSuccess &&
            cudaMalloc(&ctx->d_huge, sizeof(long long)) == cudaSuccess &&
            cudaMalloc(&ctx->d_hist, sizeof(uint32_t) * (hh::kBuckets + 2)) == cudaSuccess &&
            cudaMalloc(&ctx->d_cursor, sizeof(uint32_t) * hh::kBuckets) == cudaSuccess &&
            cudaMemset(ctx->d_err, 0, sizeof(int)) == cudaSuccess &&
            cudaMemset(ctx->d_next_tile, 0, 4 * sizeof(unsigned long long)) == cudaSuccess &&
            reserve_perm(ctx, HH_DEFAULT_MAX_MESSAGES) == HH_OK;
  if (!ok) {
    hh_destroy(ctx);
    return HH_ERR_NO_MEMORY;
  }
  *out = ctx;
  return HH_OK;
}

int hh_destroy(hh_ctx* ctx) {
  if (ctx == nullptr) return HH_OK;
  DeviceGuard guard(ctx->device);
  cudaDeviceSynchronize();
  cudaFree(ctx->d_err);
  cudaFree(ctx->d_next_tile);
  cudaFree(ctx->d_use_perm);
  cudaFree(ctx->d_huge);
  cudaFree(ctx->d_hist);
  cudaFree(ctx->d_cursor);
  cudaFree(ctx->d_perm);
  for (hh::HostSlot& s : ctx->slots) {
    // Allocated stream-ordered on s_h2d (see grow); freed the same way.
    if (ctx->s_h2d) {
      if (s.bytes) cudaFreeAsync(s.bytes, ctx->s_h2d);
      if (s.offsets) cudaFreeAsync(s.offsets, ctx->s_h2d);
      if (s.keys) cudaFreeAsync(s.keys, ctx->s_h2d);
      if (s.out) cudaFreeAsync(s.out, ctx->s_h2d);
    }
    if (s.staged) cudaEventDestroy(s.staged);
    if (s.hashed) cudaEventDestroy(s.hashed);
    if (s.drained) cudaEventDestroy(s.drained);
  }
  if (ctx->s_h2d) {
    cudaStreamSynchronize(ctx->s_h2d);
    cudaStreamDestroy(ctx->s_h2d);
  }
  if (ctx->s_comp) cudaStreamDestroy(ctx->s_comp);
  if (ctx->s_d2h) cudaStreamDestroy(ctx->s_d2h);
  delete ctx;
  return HH_OK;
}

int hh_reserve(hh_ctx* ctx, int64_t max_messages) {
  if (ctx == nullptr || max_messages < 0) return HH_ERR_INVALID_ARG;
  if (max_messages > kMaxSortedMessages) return HH_ERR_TOO_LARGE;
  DeviceGuard guard(ctx->device);
  if (!guard.ok) return HH_ERR_CUDA;
  return reserve_perm(ctx, max_messages);
}

int hh_hash64_batch(hh_ctx* ctx, const uint64_t* keys, int key_mode, const uint8_t* bytes,
                    const int64_t* offsets, int64_t n, uint64_t* out, void* stream) {
  if (offsets == nullptr && n > 0) return HH_ERR_INVALID_ARG;
  return hash_common(ctx, 64, keys, key_mode, bytes, offsets, 0, n, out,
                     static_cast<cudaStream_t>(stream));
}

int hh_hash128_batch(hh_ctx* ctx, const uint64_t* keys, int key_mode, const uint8_t* bytes,
                     const int64_t* offsets, int64_t n, uint64_t* out, void* stream) {
  if (offsets == nullptr && n > 0) return HH_ERR_INVALID_ARG;
  return hash_common(ctx, 128, keys, key_mode, bytes, offsets, 0, n, out,
                     static_cast<cudaStream_t>(stream));
}

int hh_hash256_batch(hh_ctx* ctx, const uint64_t* keys, int key_mode, const uint8_t* bytes,
                     const int64_t* offsets, int64_t n, uint64_t* out, void* stream) {
  if (offsets == nullptr && n > 0) return HH_ERR_INVALID_ARG;
  return hash_common(ctx, 256, keys, key_mode, bytes, offsets, 0, n, out,
                     static_cast<cudaStream_t>(stream));
}

int hh_hash_fixed(hh_ctx* ctx, int bits, const uint64_t* keys, int key_mode,
                  const uint8_t* bytes, int64_t msg_len, int64_t n, uint64_t* out,
                  void* stream) {
  if (msg_len < 0) return HH_ERR_INVALID_ARG;
  return hash_common(ctx, bits, keys, key_mode, bytes, nullptr, msg_len, n, out,
                     static_cast<cudaStream_t>(stream));
}

int hh_hash_segments(hh_ctx* ctx, int bits, const uint64_t* key_table, int32_t key_count,
                     const int32_t* key_index, const uint8_t* bytes, int64_t bytes_len,
                     const int64_t* starts, const int64_t* lengths, int64_t n,
                     const int64_t* n_device, uint64_t* out, void* stream) {
  if (ctx == nullptr) return HH_ERR_INVALID_ARG;
  const int words = words_of(bits);
  if (words == 0 || n < 0 || bytes_len < 0 || key_count < 1) return HH_ERR_INVALID_ARG;
  ctx->last_launches = 0;
  if (n == 0) return HH_OK;
  if (key_table == nullptr || starts == nullptr || lengths == nullptr || out == nullptr ||
      bytes == nullptr)
    return HH_ERR_INVALID_ARG;
  hh::Batch b{};
  b.bytes = bytes;
  b.seg_start = starts;
  b.seg_len = lengths;
  b.bytes_len = bytes_len;
  b.keys = key_table;
  b.per_message_keys = 0;
  b.key_index = key_index;
  b.key_count = key_count;
  b.n = n;
  b.n_dev = n_device;
  b.out = out;
  b.words = words;
  return hash_device(ctx, b, static_cast<cudaStream_t>(stream));
}

int hh_siptree_batch(hh_ctx* ctx, int variant, const uint64_t* keys, int key_mode,
                     const uint8_t* bytes, const int64_t* offsets, int64_t n, uint64_t* out,
                     void* stream) {
  if (ctx == nullptr || (variant != HH_SIPTREE && variant != HH_SIPTREE13) ||
      (key_mode != HH_KEY_SHARED && key_mode != HH_KEY_PER_MESSAGE) || n < 0)
    return HH_ERR_INVALID_ARG;
  ctx->last_launches = 0;
  if (n == 0) return HH_OK;
  if (keys == nullptr || bytes == nullptr || offsets == nullptr || out == nullptr)
    return HH_ERR_INVALID_ARG;
  if (n > ctx->perm_cap) return HH_ERR_TOO_LARGE;
  DeviceGuard guard(ctx->device);
  if (!guard.ok) return HH_ERR_CUDA;
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  hh::Batch b{};
  b.bytes = bytes;
  b.offsets = offsets;
  b.keys = keys;
  b.per_message_keys = key_mode == HH_KEY_PER_MESSAGE;
  b.n = n;
  b.out = out;
  b.words = 1;
  b.err = ctx->d_err;
  b.wait_ns = ctx->wait_limit_ns;
  // Longest first, as for HighwayHash; no message is set apart as huge.
  int launches = 0;
  cudaError_t e = hh::launch_bucket_sort(b, ctx->d_hist, ctx->d_cursor, ctx->d_perm,
                                         ctx->d_next_tile, ctx->d_use_perm, ctx->d_huge,
                                         hh::kBuckets, ctx->num_sms, s, &launches);
  if (e != cudaSuccess) return to_status(e);
  hh::Queue q{};
  q.perm = ctx->d_perm;
  q.use_perm = ctx->d_use_perm;
  q.next_tile = ctx->d_next_tile;
  q.tiles = (n + 31) / 32;
  e = hh::launch_siptree(b, q, variant == HH_SIPTREE ? hh::kSipTree24 : hh::kSipTree13,
                         ctx->num_sms, s);
  ctx->last_launches = launches + 1;
  return to_status(e);
}

int hh_stream_init(hh_ctx* ctx, const uint64_t* keys, int key_mode, int64_t n,
                   uint64_t* states, void* stream) {
  if (ctx == nullptr || n < 0 || (key_mode != HH_KEY_SHARED && key_mode != HH_KEY_PER_MESSAGE))
    return HH_ERR_INVALID_ARG;
  ctx->last_launches = 0;
  if (n == 0) return HH_OK;
  if (keys == nullptr || states == nullptr) return HH_ERR_INVALID_ARG;
  DeviceGuard guard(ctx->device);
  if (!guard.ok) return HH_ERR_CUDA;
  ctx->last_launches = 1;
  return to_status(hh::launch_stream_init(keys, key_mode == HH_KEY_PER_MESSAGE, n, states,
                                          ctx->num_sms, static_cast<cudaStream_t>(stream)));
}

// Shared by hh_stream_update and hh_stream_finish.
static int stream_chunks(hh_ctx* ctx, int mode, int bits, uint64_t* states, const uint8_t* bytes,
                         const int64_t* offsets, int64_t n, uint64_t* out, void* stream) {
  if (ctx == nullptr || n < 0) return HH_ERR_INVALID_ARG;
  const int words = mode == hh::kStreamFinish ? words_of(bits) : 1;
  if (words == 0) return HH_ERR_INVALID_ARG;
  ctx->last_launches = 0;
  if (n == 0) return HH_OK;
  if (states == nullptr || offsets == nullptr || bytes == nullptr ||
      (mode == hh::kStreamFinish && out == nullptr))
    return HH_ERR_INVALID_ARG;
  hh::Batch b{};
  b.bytes = bytes;
  b.offsets = offsets;
  b.n = n;
  b.out = out;
  b.words = words;
  b.states = states;
  b.stream_mode = mode;
  return hash_device(ctx, b, static_cast<cudaStream_t>(stream));
}

int hh_stream_update(hh_ctx* ctx, uint64_t* states, const uint8_t* bytes, const int64_t* offsets,
                     int64_t n, void* stream) {
  return stream_chunks(ctx, hh::kStreamUpdate, 64, states, bytes, offsets, n, nullptr, stream);
}

int hh_stream_finish(hh_ctx* ctx, int bits, const uint64_t* states, const uint8_t* bytes,
                     const int64_t* offsets, int64_t n, uint64_t* out, void* stream) {
  return stream_chunks(ctx, hh::kStreamFinish, bits, const_cast<uint64_t*>(states), bytes,
                       offsets, n, out, stream);
}

int hh_hash_host(hh_ctx* ctx, int bits, const uint64_t* keys, int key_mode,
                 const uint8_t* bytes, const int64_t* offsets, int64_t n, uint64_t* out) {
  if (ctx == nullptr) return HH_ERR_INVALID_ARG;
  const int words = words_of(bits);
  if (words == 0 || (key_mode != HH_KEY_SHARED && key_mode != HH_KEY_PER_MESSAGE) || n < 0)
    return HH_ERR_INVALID_ARG;
  if (n == 0) return HH_OK;
  if (keys == nullptr || bytes == nullptr || offsets == nullptr || out == nullptr)
    return HH_ERR_INVALID_ARG;
  if (offsets[0] < 0 || offsets[n] < offsets[0]) return HH_ERR_BAD_OFFSETS;
  DeviceGuard guard(ctx->device);
  if (!guard.ok) return HH_ERR_CUDA;
  if (ctx->s_h2d == nullptr) {
    if (cudaStreamCreateWithFlags(&ctx->s_h2d, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&ctx->s_comp, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&ctx->s_d2h, cudaStreamNonBlocking) != cudaSuccess)
      return HH_ERR_CUDA;
    for (hh::HostSlot& s : ctx->slots) {
      if (cudaEventCreateWithFlags(&s.staged, cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&s.hashed, cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&s.drained, cudaEventDisableTiming) != cudaSuccess)
        return HH_ERR_CUDA;
    }
  }
  // Once a chunk is enqueued, an error return first waits for the context's
  // streams, so that no copy still reads `bytes` or writes `out` after the
  // call has returned.
  bool enqueued = false;
  auto fail = [&](int status) {
    if (enqueued) {
      cudaStreamSynchronize(ctx->s_h2d);
      cudaStreamSynchronize(ctx->s_comp);
      cudaStreamSynchronize(ctx->s_d2h);
    }
    return status;
  };
  // Chunk boundaries: at most kHostChunkMessages messages and (unless a single
  // message is larger) kHostChunkBytes payload per chunk.
  int launches = 0;
  int chunk_index = 0;
  int64_t m0 = 0;
  while (m0 < n) {
    int64_t m1 = m0 + 1;
    const int64_t limit = std::min<int64_t>(n, m0 + kHostChunkMessages);
    {
      // Largest m1 <= limit with offsets[m1] - offsets[m0] <= chunk bytes.
      int64_t lo = m0 + 1, hi = limit;
      while (lo < hi) {
        const int64_t mid = lo + (hi - lo + 1) / 2;
        if (offsets[mid] - offsets[m0] <= static_cast<int64_t>(kHostChunkBytes)) lo = mid;
        else hi = mid - 1;
      }
      m1 = lo;
    }
    // Only the chunk's own bytes are staged, so every offset inside it must
    // lie between its end offsets: check that none decreases before any of
    // the chunk is enqueued.  (offsets[m0] >= offsets[0] >= 0 follows from
    // the checks of the earlier chunks.)
    {
      bool decreasing = false;
      for (int64_t i = m0; i < m1; ++i) decreasing |= offsets[i + 1] < offsets[i];
      if (decreasing) return fail(HH_ERR_BAD_OFFSETS);
    }
    hh::HostSlot& s = ctx->slots[chunk_index & 1];
    const int64_t cn = m1 - m0;
    const size_t cbytes = static_cast<size_t>(offsets[m1] - offsets[m0]);
    // The slot's previous chunk must have drained before its buffers change.
    if (cudaStreamWaitEvent(ctx->s_h2d, s.drained, 0) != cudaSuccess) return fail(HH_ERR_CUDA);
    {
      int st = grow(&s.bytes, &s.bytes_cap, std::max<size_t>(cbytes, 16), ctx->s_h2d);
      if (st == HH_OK) st = grow(&s.offsets, &s.offsets_cap, static_cast<size_t>(cn + 1), ctx->s_h2d);
      if (st == HH_OK) st = grow(&s.out, &s.out_cap, static_cast<size_t>(cn) * words, ctx->s_h2d);
      if (st == HH_OK)
        st = grow(&s.keys, &s.keys_cap,
                  key_mode == HH_KEY_PER_MESSAGE ? static_cast<size_t>(cn) * 4 : size_t(4),
                  ctx->s_h2d);
      if (st != HH_OK) return fail(st);
    }
    const uint64_t* ck = key_mode == HH_KEY_PER_MESSAGE ? keys + 4 * m0 : keys;
    const size_t key_words = key_mode == HH_KEY_PER_MESSAGE ? static_cast<size_t>(cn) * 4 : 4;
    enqueued = true;
    cudaError_t e = cudaMemcpyAsync(s.bytes, bytes + offsets[m0], cbytes, cudaMemcpyHostToDevice,
                                    ctx->s_h2d);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(s.offsets, offsets + m0, sizeof(int64_t) * (cn + 1),
                          cudaMemcpyHostToDevice, ctx->s_h2d);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(s.keys, ck, sizeof(uint64_t) * key_words, cudaMemcpyHostToDevice,
                          ctx->s_h2d);
    if (e == cudaSuccess) e = cudaEventRecord(s.staged, ctx->s_h2d);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->s_comp, s.staged, 0);
    if (e != cudaSuccess) return fail(HH_ERR_CUDA);
    // The device offsets are absolute; shift the base so that
    // base + offsets[m0] is the first staged byte.
    const uint8_t* dev_base = s.bytes - offsets[m0];
    int st = hash_common(ctx, bits, s.keys, key_mode, dev_base, s.offsets, 0, cn, s.out,
                         ctx->s_comp);
    launches += ctx->last_launches;
    if (st != HH_OK) return fail(st);
    e = cudaEventRecord(s.hashed, ctx->s_comp);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->s_d2h, s.hashed, 0);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(out + m0 * words, s.out, sizeof(uint64_t) * cn * words,
                          cudaMemcpyDeviceToHost, ctx->s_d2h);
    if (e == cudaSuccess) e = cudaEventRecord(s.drained, ctx->s_d2h);
    if (e != cudaSuccess) return fail(HH_ERR_CUDA);
    m0 = m1;
    ++chunk_index;
  }
  ctx->last_launches = launches;
  if (cudaStreamSynchronize(ctx->s_d2h) != cudaSuccess) return fail(HH_ERR_CUDA);
  int err = 0;
  if (cudaMemcpy(&err, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return fail(HH_ERR_CUDA);
  if (err != 0) {
    cudaMemset(ctx->d_err, 0, sizeof(int));
    return err;
  }
  return HH_OK;
}

int hh_get_device_error(hh_ctx* ctx, void* stream) {
  if (ctx == nullptr) return HH_ERR_INVALID_ARG;
  DeviceGuard guard(ctx->device);
  if (!guard.ok) return HH_ERR_CUDA;
  if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess) return HH_ERR_CUDA;
  int err = 0;
  if (cudaMemcpy(&err, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return HH_ERR_CUDA;
  if (err != 0 && cudaMemset(ctx->d_err, 0, sizeof(int)) != cudaSuccess) return HH_ERR_CUDA;
  return err;
}

int hh_set_kernel(hh_ctx* ctx, int kernel) {
  if (ctx == nullptr || kernel < HH_KERNEL_AUTO || kernel > HH_KERNEL_STAGED_BULK)
    return HH_ERR_INVALID_ARG;
  ctx->kernel = kernel;
  return HH_OK;
}

int hh_last_launch_count(hh_ctx* ctx) { return ctx ? ctx->last_launches : 0; }

int hh_update_microbench(hh_ctx* ctx, int variant, int64_t updates, int64_t threads,
                         uint64_t* out, void* stream) {
  if (ctx == nullptr || out == nullptr || updates < 0 || threads <= 0 || threads % 32 != 0 ||
      (threads > 256 && threads % 256 != 0) || threads / 256 > INT32_MAX || variant < 0 ||
      variant >= HH_UPDATE_VARIANTS)
    return HH_ERR_INVALID_ARG;
  DeviceGuard guard(ctx->device);
  if (!guard.ok) return HH_ERR_CUDA;
  ctx->last_launches = 1;
  return to_status(hh::launch_update_microbench(variant, updates, threads, out,
                                                static_cast<cudaStream_t>(stream)));
}

int hh_set_staged_shape(hh_ctx* ctx, int regime, int window, int stages,
                        int messages_per_thread) {
  if (ctx == nullptr || regime < HH_REGIME_FIXED || regime > HH_REGIME_BULK)
    return HH_ERR_INVALID_ARG;
  if (regime != HH_REGIME_FIXED && messages_per_thread != 1) return HH_ERR_INVALID_ARG;
  const hh::StagedShape shape{window, stages, messages_per_thread};
  if (regime == HH_REGIME_FIXED) {
    if (!hh::fixed_shape_valid(shape)) return HH_ERR_INVALID_ARG;
    for (hh::StagedShape& f : ctx->tune.fixed) f = shape;  // every length class
  } else if (regime == HH_REGIME_RAGGED) {
    if (!hh::ragged_shape_valid(shape)) return HH_ERR_INVALID_ARG;
    ctx->tune.ragged = shape;
  } else {
    if (hh::staged_smem_bytes(shape) == 0) return HH_ERR_INVALID_ARG;
    ctx->shape_bulk = shape;
  }
  return HH_OK;
}

}  // extern "C"

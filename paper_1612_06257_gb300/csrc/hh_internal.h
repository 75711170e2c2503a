// hh_internal.h -- declarations shared by the translation units of libhh.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace hh {

// Device error codes (same values as enum hh_status in include/hh.h).
constexpr int kErrTimeout = 4;
constexpr int kErrBadOffsets = 6;   // also: a segment outside the buffer
constexpr int kErrBadKey = 8;       // a key index outside the key table
constexpr int kErrBadChunk = 9;     // a stream-update chunk not a multiple of 32 bytes

// Bounds on the kernels' waits for asynchronous copies.  A wait that runs
// past its limit records kErrTimeout and the thread writes zero hashes; the
// kernel issues no further copies and waits (at most kDrainLimitNs per copy)
// for those it issued before it exits.  The limit is a per-context setting
// (hh_set_tune_param "wait_limit_ns"; kWaitLimitNs by default); 0 tests each
// barrier once without blocking.
constexpr uint64_t kWaitLimitNs = 2000000000ull;  // 2 s: far beyond any legitimate wait
constexpr uint64_t kDrainLimitNs = 200000000ull;  // 0.2 s per copy when giving up

// Length-sort buckets by the number of Updates P = ceil(len / 32) a message
// needs before finalisation: P itself below 2048, then 128 buckets per
// doubling of P (messages up to 4 GiB).  By default messages in kHugeBucket
// and above (P >= 4096, 128 KiB) run two threads per message; the autotuner
// may raise that threshold or switch pairs off.
constexpr int kBuckets = 4096;
constexpr int kHugeBucket = 2048 + 128;

__host__ __device__ inline int bucket_of_packets(int64_t p) {
  if (p < 2048) return static_cast<int>(p);
  int lead = 11;  // index of p's leading bit (p >= 2^11)
  while (lead < 62 && (p >> (lead + 1)) != 0) ++lead;
  const int b = 2048 + 128 * (lead - 11) + static_cast<int>((p >> (lead - 7)) & 127);
  return b < kBuckets ? b : kBuckets - 1;
}

// Messages per work tile of the staged kernel: one thread per message.
constexpr int kTileRows = 128;

// One batch, as every kernel sees it (hh_batch.cuh reads it).
struct Batch {
  const uint8_t* bytes;      // message bytes
  const int64_t* offsets;    // n + 1 offsets (offsets form), or null
  int64_t fixed_len;         // message length (fixed form: offsets and seg_start null)
  const int64_t* seg_start;  // segments form: n starts, relative to bytes, or null
  const int64_t* seg_len;    //                n lengths
  int64_t bytes_len;         //                size of the bytes buffer
  const uint64_t* keys;      // 4 words (shared), 4 * n (per message) or a key table
  int per_message_keys;
  const int32_t* key_index;  // n rows of the key table, or null
  int32_t key_count;         // rows in the key table
  int64_t n;                 // messages, or the capacity when n_dev is set
  const int64_t* n_dev;      // device word with the message count (<= n), or null
  uint64_t* out;             // words * n
  int words;                 // 1, 2 or 4
  int stream_mode;           // kWholeMessages, kStreamUpdate or kStreamFinish
  int* err;                  // device error word (first error wins)
  uint64_t* states;          // streams: n x 16 words (v0, v1, mul0, mul1; lanes 0..3)
  uint64_t wait_ns = kWaitLimitNs;  // limit of one wait for an asynchronous copy
};

// What a batch's messages are: whole messages (Init from the key, hash
// out); chunks that continue stored stream states (whole 32-byte packets
// only, state out); or the last chunks of stored streams (hash out).
constexpr int kWholeMessages = 0;
constexpr int kStreamUpdate = 1;
constexpr int kStreamFinish = 2;

// Work-queue state of the staged kernel.
struct Queue {
  const int32_t* perm;       // processing order of messages, or null = 0..n-1
  const int* use_perm;       // device flag: 0 = ignore perm (no long message), or null
  int skip_if_short = 0;     // 1: return at once when *use_perm == 0 (the short kernel runs)
  const long long* huge_count = nullptr;  // messages perm[0 .. *huge_count) run as pairs
  unsigned long long* next_tile;  // [4] (sorted order): [0] warp-tile counter, [1] huge-
                                  // prefix claims, [2..3] launch bookkeeping; or null =
                                  // static order
  int64_t tiles;             // tiles the grid is sized for
  int64_t solo_max = 0;      // huge prefixes of at most this many messages run one per warp
  int solo_ctas = 0;         // ... taken only by the warps of blocks 0 .. solo_ctas - 1
  int solo_shared = 0;       // 1: solo tiles also while other such launches are in flight
};

// Solo tiles (one huge message per warp) while there are at most this many
// huge messages per SM: one per warp scheduler.  Beyond that, warps would
// share schedulers and 16-message pair tiles give more throughput.
constexpr int kSoloPerSm = 4;
constexpr int kRaggedWarps = 4;  // warps per block of the ragged kernel

// Staged-kernel shapes: bytes of each message staged per pipeline step (W)
// and the number of pipeline buffers.
struct StagedShape {
  int window;    // 128 or 256
  int stages;    // 2..6
  int msgs = 1;  // messages per thread (fixed-length TMA kernel)
};

// Launchers (return the CUDA error of the launch).
// Resident blocks per SM of `kern` at this block size and dynamic shared
// memory on the current device; sets the kernel's dynamic shared memory
// limit first.  Cached per (kernel, device, threads, smem), so only the
// first launch of a shape pays for the queries.  0 on error (in *err).
int blocks_per_sm(const void* kern, int threads, int smem, cudaError_t* err);

cudaError_t launch_naive(const Batch& b, cudaStream_t stream);
cudaError_t launch_stream_init(const uint64_t* keys, int per_message, int64_t n,
                               uint64_t* states, int num_sms, cudaStream_t stream);
cudaError_t launch_staged(const Batch& b, const Queue& q, StagedShape shape, bool aligned16,
                          int num_sms, cudaStream_t stream);
int staged_blocks_per_sm(StagedShape shape, bool aligned16);
size_t staged_smem_bytes(StagedShape shape);

// Ragged batches: warp tiles of 32 messages, coalesced cp.async staging.
// Supported (window, stages) pairs:
#define HH_RAGGED_SHAPES(X) X(128, 2) X(128, 3) X(128, 4) X(256, 2) X(256, 3)
bool ragged_shape_valid(StagedShape shape);
cudaError_t launch_ragged(const Batch& b, const Queue& q, StagedShape shape, int num_sms,
                          cudaStream_t stream);

// Batches of messages of at most kShortMax bytes: thread per message, no
// shared memory.  Returns at once unless *run_if == 0 (run_if may be null).
cudaError_t launch_short(const Batch& b, const int* run_if, int num_sms, cudaStream_t stream);

// Fixed-length batches through 2D tensor-map TMA (len % 16 == 0, 16-byte
// aligned bytes).  Supported (window, stages) pairs:
#define HH_FIXED_SHAPES(X) \
  X(128, 2, 1) X(128, 3, 1) X(128, 4, 1) X(256, 2, 1) X(256, 3, 1) X(128, 2, 2) X(128, 3, 2)
bool fixed_tma_supported(const uint8_t* bytes, int64_t len, int64_t n);
cudaError_t launch_fixed_tma(const Batch& b, StagedShape shape, int num_sms, cudaStream_t stream);
// Fixed-length batches too small to fill the GPU: two threads per message
// (one lane pair each), 256-byte windows, two stages.
cudaError_t launch_fixed_tma_pair(const Batch& b, int num_sms, cudaStream_t stream);
bool fixed_shape_valid(StagedShape shape);

// SipTreeHash (Section 3) of an offsets or segments batch, 64-bit output,
// one thread per message in warp tiles from q's order.  kSipTree24 runs
// SipHash-2-4 lanes (SipTreeHash), kSipTree13 SipHash-1-3 (SipTreeHash13).
constexpr int kSipTree24 = 0;
constexpr int kSipTree13 = 1;
cudaError_t launch_siptree(const Batch& b, const Queue& q, int variant, int num_sms,
                           cudaStream_t stream);

// Update-rate microbenchmark (threads must be a multiple of 256).
cudaError_t launch_update_microbench(int variant, int64_t updates, int64_t threads,
                                     uint64_t* out, cudaStream_t stream);

// Length bucketing: hist and cursor are kBuckets words; perm n words.
// The scan sets *use_perm = 1 when some message is longer than
// kShortMax bytes (the order then matters for load balance), else 0 and the
// scatter does nothing: all-short batches keep index order, which keeps their
// loads sequential.
constexpr int kShortMax = 64;
cudaError_t launch_bucket_sort(const Batch& b, uint32_t* hist, uint32_t* cursor, int32_t* perm,
                               unsigned long long* next_tile, int* use_perm,
                               long long* huge_count, int huge_bucket, int num_sms,
                               cudaStream_t stream, int* launches);

}  // namespace hh

// hh_batch.cuh -- how a kernel finds message m, its key and the byte range.
//
// A batch comes in one of three forms (see Batch in hh_internal.h):
//   offsets   message m = bytes[offsets[m] .. offsets[m+1]), offsets
//             non-decreasing; the batch reads [offsets[0], offsets[n]);
//   fixed     message m = bytes[m * len .. (m+1) * len);
//   segments  message m = bytes[start[m] .. start[m] + length[m]), each inside
//             [0, bytes_len); segments may come in any order and may overlap.
// Keys are one shared key, one key per message, or rows of a key table
// chosen by key_index[m] (0 <= key_index[m] < key_count).
#pragma once

#include <cstdint>

#include "hh_internal.h"

namespace hh {

// A kernel's view of the message count: a batch whose count lives in device
// memory (so that one captured launch serves batches of any size up to its
// capacity) reads it once at kernel start, clamped to the capacity.
__device__ __forceinline__ void resolve_count(Batch& b) {
  if (b.n_dev != nullptr) {
    const int64_t n = *b.n_dev;
    b.n = n < 0 ? 0 : (n < b.n ? n : b.n);
  }
}

// Start (relative to b.bytes) and length of message m.  `bad` is 0, or the
// error code of an invalid descriptor (decreasing offsets or a segment
// outside the buffer: kErrBadOffsets; a key index outside the table:
// kErrBadKey; a stream-update chunk whose length is not a multiple of 32:
// kErrBadChunk); such a message is hashed as empty and its output is 0.
__device__ __forceinline__ void message_bounds(const Batch& b, int64_t m, int64_t& start,
                                               int64_t& len, int& bad) {
  bad = 0;
  if (b.offsets != nullptr) {
    const int64_t s = b.offsets[m], e = b.offsets[m + 1];
    if (e < s) bad = kErrBadOffsets;
    start = s;
    len = bad ? 0 : e - s;
  } else if (b.seg_start != nullptr) {
    const int64_t s = b.seg_start[m], l = b.seg_len[m];
    if (s < 0 || l < 0 || s > b.bytes_len || l > b.bytes_len - s) bad = kErrBadOffsets;
    start = bad ? 0 : s;
    len = bad ? 0 : l;
  } else {
    start = m * b.fixed_len;
    len = b.fixed_len;
  }
  if (b.key_index != nullptr && bad == 0) {
    const int32_t k = b.key_index[m];
    if (k < 0 || k >= b.key_count) {
      bad = kErrBadKey;
      len = 0;
    }
  }
  if (b.stream_mode == kStreamUpdate && bad == 0 && (len & 31) != 0) {
    bad = kErrBadChunk;  // the state is left as it was
    len = 0;
  }
}

// Length only (the length sort); invalid descriptors count as empty.
__device__ __forceinline__ int64_t message_length(const Batch& b, int64_t m) {
  int64_t start, len;
  int bad;
  message_bounds(b, m, start, len, bad);
  return bad ? 0 : len;
}

// The key of message m (valid only when message_bounds did not flag it).
__device__ __forceinline__ const uint64_t* key_of(const Batch& b, int64_t m) {
  if (b.key_index != nullptr) {
    const int32_t k = b.key_index[m];
    return b.keys + 4 * static_cast<int64_t>(k >= 0 && k < b.key_count ? k : 0);
  }
  return b.per_message_keys ? b.keys + 4 * m : b.keys;
}

// The byte range [lo, hi) (relative to b.bytes) that the batch may read.
__device__ __forceinline__ void batch_range(const Batch& b, int64_t& lo, int64_t& hi) {
  if (b.offsets != nullptr) {
    lo = b.offsets[0];
    hi = b.offsets[b.n];
  } else if (b.seg_start != nullptr) {
    lo = 0;
    hi = b.bytes_len;
  } else {
    lo = 0;
    hi = b.n * b.fixed_len;
  }
}

}  // namespace hh

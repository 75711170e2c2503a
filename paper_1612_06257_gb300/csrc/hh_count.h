// hh_count.h -- the length count of the sort fused into the short kernel.
//
// A batch above the short kernel's minimum size, in the plain offsets form
// with one key for every message, is counted and (when all its messages are
// short) hashed in one pass over its offsets: short_count_kernel, then the
// scan and the scatter of the length sort, then the warp-tile kernel.  The
// other batches keep the separate count launch (launch_bucket_sort).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "hh_internal.h"

namespace hh {

// Whether batch b takes the fused path: offsets form, one key, whole
// messages, a host-side message count.
inline bool short_count_eligible(const Batch& b) {
  return b.offsets != nullptr && !b.per_message_keys && b.key_index == nullptr &&
         b.stream_mode == kWholeMessages && b.n_dev == nullptr;
}

// hist: kBuckets + 2 words, zeroed by the caller.  The kernel adds every
// message's length bucket to hist[0 .. kBuckets) (the buckets of
// launch_bucket_sort's count, except that buckets 0..2, the messages of at
// most kShortMax bytes, are all counted in bucket 2) and uses hist[kBuckets]
// as the flag that some message is longer than kShortMax, hist[kBuckets + 1]
// as the counter of its work queue.  When no message is, every hash is
// written; otherwise hashes may or may not be written, and the warp-tile
// kernel launched after the scan writes them all.
cudaError_t launch_short_counted(const Batch& b, uint32_t* hist, int num_sms,
                                 cudaStream_t stream);

// The scan and the scatter of the length sort over a histogram counted by
// launch_short_counted (buckets 0..2 merged into 2; 2 launches, added to
// *launches).
cudaError_t launch_bucket_scan_scatter(const Batch& b, uint32_t* hist, uint32_t* cursor,
                                       int32_t* perm, unsigned long long* next_tile,
                                       int* use_perm, long long* huge_count, int huge_bucket,
                                       int num_sms, cudaStream_t stream, int* launches);

}  // namespace hh

// hh_stream.cuh -- where a message's state comes from and where it goes.
//
// Whole messages start from Init of their key and end in Finalize and the
// hash.  Streams (Section 4.5 injects the size only at the end, so a message
// may arrive in pieces of whole packets) keep their state in device memory
// between calls: an update chunk starts from the stored state and stores it
// back, and the last chunk starts from it and ends in the hash.  Layout of
// a stored state: 16 words, v0[0..3], v1[0..3], mul0[0..3], mul1[0..3].
#pragma once

#include <cstdint>

#include "hh_batch.cuh"
#include "hh_device.cuh"
#include "hh_internal.h"

namespace hh {

__device__ __forceinline__ void start_state(const Batch& b, int64_t m, bool valid, State& s) {
  uint64_t key[4] = {0, 0, 0, 0};
  if (b.stream_mode != kWholeMessages) {
    init(s, key);
    if (valid) {
      const uint64_t* p = b.states + 16 * m;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        s.v0[i] = p[i];
        s.v1[i] = p[4 + i];
        s.mul0[i] = p[8 + i];
        s.mul1[i] = p[12 + i];
      }
    }
    return;
  }
  if (valid) {
    const uint64_t* kp = key_of(b, m);
#pragma unroll
    for (int i = 0; i < 4; ++i) key[i] = __ldg(kp + i);
  }
  init(s, key);
}

// Lane pair `half` (lanes 2 half, 2 half + 1) of message m's state.
__device__ __forceinline__ void start_half(const Batch& b, int64_t m, bool valid, int half,
                                           Half& s) {
  uint64_t key[4] = {0, 0, 0, 0};
  if (b.stream_mode != kWholeMessages) {
    init_half(s, key, half);
    if (valid) {
      const uint64_t* p = b.states + 16 * m + 2 * half;
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        s.v0[j] = p[j];
        s.v1[j] = p[4 + j];
        s.mul0[j] = p[8 + j];
        s.mul1[j] = p[12 + j];
      }
    }
    return;
  }
  if (valid) {
    const uint64_t* kp = key_of(b, m);
#pragma unroll
    for (int i = 0; i < 4; ++i) key[i] = __ldg(kp + i);
  }
  init_half(s, key, half);
}

// Stores the state (update chunks) or finalises and writes the hash (zero
// for an invalid descriptor).
__device__ __forceinline__ void end_state(const Batch& b, int64_t m, bool valid, int bad,
                                          State& s) {
  if (b.stream_mode == kStreamUpdate) {
    if (valid && !bad) {
      uint64_t* p = b.states + 16 * m;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        p[i] = s.v0[i];
        p[4 + i] = s.v1[i];
        p[8 + i] = s.mul0[i];
        p[12 + i] = s.mul1[i];
      }
    }
    return;
  }
  finalize(s);
  if (valid) {
    uint64_t h[4];
    digest(s, h);
    if (bad) h[0] = h[1] = h[2] = h[3] = 0;
    uint64_t* o = b.out + m * b.words;
    o[0] = h[0];
    if (b.words >= 2) o[1] = h[1];
    if (b.words == 4) {
      o[2] = h[2];
      o[3] = h[3];
    }
  }
}

// As end_state for a lane pair; all 32 lanes of the warp call it (the
// finalisation exchanges v0 between partners; b.stream_mode is uniform).
__device__ __forceinline__ void end_half(const Batch& b, int64_t m, bool valid, int bad,
                                         int half, Half& s) {
  if (b.stream_mode == kStreamUpdate) {
    if (valid && !bad) {
      uint64_t* p = b.states + 16 * m + 2 * half;
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        p[j] = s.v0[j];
        p[4 + j] = s.v1[j];
        p[8 + j] = s.mul0[j];
        p[12 + j] = s.mul1[j];
      }
    }
    return;
  }
  finalize_half(s);
  if (valid) {
    uint64_t h0 = s.v0[0] + s.v1[0] + s.mul0[0] + s.mul1[0];
    uint64_t h1 = s.v0[1] + s.v1[1] + s.mul0[1] + s.mul1[1];
    if (bad) h0 = h1 = 0;
    uint64_t* o = b.out + m * b.words;
    if (half == 0) {
      o[0] = h0;
      if (b.words >= 2) o[1] = h1;
    } else if (b.words == 4) {
      o[2] = h0;
      o[3] = h1;
    }
  }
}

}  // namespace hh

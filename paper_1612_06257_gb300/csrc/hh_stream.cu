// hh_stream.cu -- Init of stored stream states (the start of a message that
// arrives in pieces; Section 4.4's Init, written out instead of kept in
// registers).
#include <cuda_runtime.h>

#include <cstdint>

#include "hh_device.cuh"
#include "hh_internal.h"

namespace hh {
namespace {

__global__ void __launch_bounds__(256) stream_init_kernel(const uint64_t* keys, int per_message,
                                                          int64_t n, uint64_t* states) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t m = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; m < n;
       m += stride) {
    const uint64_t* kp = per_message ? keys + 4 * m : keys;
    uint64_t key[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) key[i] = __ldg(kp + i);
    State s;
    init(s, key);
    uint64_t* p = states + 16 * m;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      p[i] = s.v0[i];
      p[4 + i] = s.v1[i];
      p[8 + i] = s.mul0[i];
      p[12 + i] = s.mul1[i];
    }
  }
}

}  // namespace

cudaError_t launch_stream_init(const uint64_t* keys, int per_message, int64_t n,
                               uint64_t* states, int num_sms, cudaStream_t stream) {
  const int64_t blocks = (n + 255) / 256;
  const int64_t cap = static_cast<int64_t>(num_sms) * 8;
  const int grid = static_cast<int>(blocks < cap ? blocks : cap);
  if (grid <= 0) return cudaSuccess;
  stream_init_kernel<<<grid, 256, 0, stream>>>(keys, per_message, n, states);
  return cudaGetLastError();
}

}  // namespace hh

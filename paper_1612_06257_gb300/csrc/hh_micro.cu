// hh_micro.cu -- integer-issue microbenchmark for the Update step.
//
// Every thread runs Update (Section 4.2) `updates` times on register state,
// with no memory traffic except one word of output, so the measured rate is
// the ceiling the integer pipes put on hashing (Updates per second).  The
// variants split the 64-bit additions differently between the ALU pipe and
// the FMA pipe (see update_v in hh_device.cuh); all compute the same result.
#include <cuda_runtime.h>

#include <cstdint>

#include "hh_device.cuh"
#include "hh_internal.h"

namespace hh {
namespace {

template <int V>
__global__ void __launch_bounds__(256) update_rate_kernel(int64_t updates, uint32_t one,
                                                          uint64_t* out) {
  const uint64_t tid = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const uint64_t key[4] = {tid, tid * 0x9E3779B97F4A7C15ull, ~tid, tid ^ 0x5555AAAA5555AAAAull};
  State s;
  init(s, key);
  const uint64_t p[4] = {tid, tid + 1, tid + 2, tid + 3};
#pragma unroll 4
  for (int64_t i = 0; i < updates; ++i) update_v<V>(s, p, one);
  uint64_t h[4];
  digest(s, h);
  out[tid] = h[0] ^ h[1] ^ h[2] ^ h[3];
}

// One lane pair per thread (threads 2t and 2t+1 hold the two pairs of one
// state); the output word mixes both lanes of the pair.
template <int V>
__global__ void __launch_bounds__(256) update_rate_half_kernel(int64_t updates, uint32_t one,
                                                               uint64_t* out) {
  const uint64_t tid = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const uint64_t sid = tid >> 1;
  const uint64_t key[4] = {sid, sid * 0x9E3779B97F4A7C15ull, ~sid, sid ^ 0x5555AAAA5555AAAAull};
  Half s;
  init_half(s, key, static_cast<int>(tid & 1));
  const uint64_t p0 = tid, p1 = tid + 1;
#pragma unroll 4
  for (int64_t i = 0; i < updates; ++i) update_half_v<V>(s, p0, p1, one);
  out[tid] = (s.v0[0] + s.v1[0] + s.mul0[0] + s.mul1[0]) ^ (s.v0[1] + s.v1[1] + s.mul0[1] + s.mul1[1]);
}

}  // namespace

cudaError_t launch_update_microbench(int variant, int64_t updates, int64_t threads,
                                     uint64_t* out, cudaStream_t stream) {
  const int block = threads < 256 ? static_cast<int>(threads) : 256;
  const unsigned grid = static_cast<unsigned>(threads / block);
  switch (variant) {
    case 0: update_rate_kernel<0><<<grid, block, 0, stream>>>(updates, 1u, out); break;
    case 1: update_rate_kernel<1><<<grid, block, 0, stream>>>(updates, 1u, out); break;
    case 2: update_rate_kernel<2><<<grid, block, 0, stream>>>(updates, 1u, out); break;
    case 3: update_rate_kernel<3><<<grid, block, 0, stream>>>(updates, 1u, out); break;
    case 4: update_rate_kernel<4><<<grid, block, 0, stream>>>(updates, 1u, out); break;
    case 5: update_rate_kernel<5><<<grid, block, 0, stream>>>(updates, 1u, out); break;
    case 6: update_rate_half_kernel<0><<<grid, block, 0, stream>>>(updates, 1u, out); break;
    case 7: update_rate_half_kernel<1><<<grid, block, 0, stream>>>(updates, 1u, out); break;
    case 8: update_rate_half_kernel<2><<<grid, block, 0, stream>>>(updates, 1u, out); break;
    case 9: update_rate_half_kernel<3><<<grid, block, 0, stream>>>(updates, 1u, out); break;
    case 10: update_rate_half_kernel<4><<<grid, block, 0, stream>>>(updates, 1u, out); break;
    case 11: update_rate_half_kernel<5><<<grid, block, 0, stream>>>(updates, 1u, out); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace hh

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

// One lane per thread (four threads per state, lane q in thread 4s + q): the
// thread-quad mapping.  Update's ZipperMerge mixes lanes 2k and 2k + 1 only,
// and each result lane of a pair needs just its own word and the partner's
// upper half (same formula with the pair's roles swapped, Section 4.1), so
// the partners trade one 32-bit word by shfl.xor 1 per ZipperMerge.
__device__ __forceinline__ uint64_t zipper_own(uint64_t own, uint32_t other_hi, bool odd) {
  const uint32_t lo = __byte_perm(__byte_perm(lo32(own), other_hi, 0x0243), hi32(own), 0x5210);
  const uint32_t hi = __byte_perm(lo32(own), other_hi, odd ? 0x7061u : 0x0716u);
  return join(lo, hi);
}

__global__ void __launch_bounds__(256) update_rate_quad_kernel(int64_t updates, uint64_t* out) {
  const uint64_t tid = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const uint64_t sid = tid >> 2;
  const int q = static_cast<int>(tid & 3);
  const bool odd = q & 1;
  const uint64_t key = q == 0 ? sid : q == 1 ? sid * 0x9E3779B97F4A7C15ull
                     : q == 2 ? ~sid : sid ^ 0x5555AAAA5555AAAAull;
  const uint64_t c0 = q == 0 ? init_lane(0, 0) : q == 1 ? init_lane(0, 1)
                    : q == 2 ? init_lane(0, 2) : init_lane(0, 3);
  const uint64_t c1 = q == 0 ? init_lane(1, 0) : q == 1 ? init_lane(1, 1)
                    : q == 2 ? init_lane(1, 2) : init_lane(1, 3);
  uint64_t v0 = key ^ c0, v1 = swap_halves(key) ^ c1, mul0 = c0, mul1 = c1;
  const uint64_t p = tid;
#pragma unroll 4
  for (int64_t i = 0; i < updates; ++i) {
    v1 += p + mul0;
    mul0 ^= mul_lo(v1, v0 >> 32);
    const uint64_t add = mul1;                  // v0 += mul1 (before mul1 changes)
    const uint32_t lo = lo32(v0) + lo32(add);   // lo(v0 + mul1)
    mul1 ^= static_cast<uint64_t>(lo) * hi32(v1);
    const uint32_t v1_other = __shfl_xor_sync(0xffffffffu, hi32(v1), 1);
    v0 = v0 + add + zipper_own(v1, v1_other, odd);
    const uint32_t v0_other = __shfl_xor_sync(0xffffffffu, hi32(v0), 1);
    v1 += zipper_own(v0, v0_other, odd);
  }
  out[tid] = v0 + v1 + mul0 + mul1;
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
    case 12: update_rate_quad_kernel<<<grid, block, 0, stream>>>(updates, out); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace hh

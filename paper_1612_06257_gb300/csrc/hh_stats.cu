// hh_stats.cu -- counter-mode output, and the paper's statistical studies
// run on the GPU.
//
//   prng_kernel          out[i] = HighwayHash(key, 8-byte little-endian
//                        counter0 + i): a keyed stream of random words
//                        (the use the paper names in Sections 1 and 7).
//   round_table_kernel   the hash of every input of 1-3 bytes with a chosen
//                        number of finalisation rounds (Section 4.3).
//   toggle_kernel        for each input bit j and output bit k, how many x
//                        have bit k of t[x] ^ t[x ^ 2^j] set.
//   avalanche_kernel     the same counts for seeded random inputs of 1-32
//                        bytes (the strengthened avalanche test, Section 6).
//
// Random inputs come from splitmix64 (Vigna) of a counter, so any other
// implementation of that published generator reproduces them.
#include <cuda_runtime.h>

#include <cstdint>

#include "hh.h"
#include "hh_context.h"
#include "hh_device.cuh"
#include "hh_internal.h"

namespace hh {
namespace {

constexpr unsigned kAll = 0xffffffffu;

// splitmix64: output number `counter` of the stream whose state starts at seed.
__device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t counter) {
  uint64_t z = seed + (counter + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

struct Key4 {
  uint64_t k[4];
};

// The 64-bit hash of a message of len <= 32 bytes held in w[8] (bytes past
// len are ignored) with `rounds` finalisation rounds.
__device__ __forceinline__ uint64_t hash64_upto32(const uint64_t key[4], const uint32_t w[8],
                                                  uint32_t len, int rounds) {
  State s;
  init(s, key);
  if (len == 32) update_words(s, w);
  else remainder(s, len, w);
  finalize_rounds(s, rounds);
  return s.v0[0] + s.v1[0] + s.mul0[0] + s.mul1[0];
}

// kWords output words per counter, fixed per instantiation: the finalisation
// work that feeds no stored lane (for 64- and 128-bit output, the last
// round's second lane pair and most of that pair's work in the round before)
// is dead code the compiler drops.
template <int kWords>
__global__ void __launch_bounds__(256) prng_kernel(const uint64_t* key, uint64_t counter0,
                                                   int64_t n, uint64_t* out) {
  uint64_t k[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) k[i] = __ldg(key + i);
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += stride) {
    const uint64_t c = counter0 + static_cast<uint64_t>(i);
    const uint32_t w[8] = {lo32(c), hi32(c), 0, 0, 0, 0, 0, 0};
    State s;
    init(s, k);
    remainder(s, 8, w);
    finalize(s);
    uint64_t h[4];
    digest(s, h);
    uint64_t* o = out + i * kWords;
    o[0] = h[0];
    if (kWords >= 2) o[1] = h[1];
    if (kWords == 4) {
      o[2] = h[2];
      o[3] = h[3];
    }
  }
}

__global__ void __launch_bounds__(256) round_table_kernel(Key4 key, int nbytes, int rounds,
                                                          uint64_t* table) {
  const int64_t count = int64_t(1) << (8 * nbytes);
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t x = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; x < count;
       x += stride) {
    const uint32_t w[8] = {static_cast<uint32_t>(x), 0, 0, 0, 0, 0, 0, 0};
    table[x] = hash64_upto32(key.k, w, static_cast<uint32_t>(nbytes), rounds);
  }
}

// Adds the 64 bit counts of d over the warp: lane k collects output bits k
// and k + 32 into acc[0], acc[1].
__device__ __forceinline__ void count_bits(uint64_t d, bool valid, int lane, uint32_t acc[2]) {
#pragma unroll
  for (int k = 0; k < 32; ++k) {
    const uint32_t c0 = __popc(__ballot_sync(kAll, valid && ((d >> k) & 1)));
    const uint32_t c1 = __popc(__ballot_sync(kAll, valid && ((d >> (k + 32)) & 1)));
    if (lane == k) {
      acc[0] += c0;
      acc[1] += c1;
    }
  }
}

// blockIdx.y = input bit j.
__global__ void __launch_bounds__(256) toggle_kernel(const uint64_t* table, int m,
                                                     uint64_t* counts) {
  const int j = blockIdx.y;
  const int lane = threadIdx.x & 31;
  const int64_t count = int64_t(1) << m;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  uint32_t acc[2] = {0, 0};
  // Every warp runs the same number of iterations (ballots need all lanes).
  for (int64_t base = static_cast<int64_t>(blockIdx.x) * blockDim.x; base < count;
       base += stride) {
    const int64_t x = base + threadIdx.x;
    const bool valid = x < count;
    const uint64_t d = valid ? table[x] ^ table[x ^ (int64_t(1) << j)] : 0;
    count_bits(d, valid, lane, acc);
  }
  atomicAdd(reinterpret_cast<unsigned long long*>(counts + j * 64 + lane), acc[0]);
  atomicAdd(reinterpret_cast<unsigned long long*>(counts + j * 64 + lane + 32), acc[1]);
}

// blockIdx.y = input bit b.  Iteration t hashes the first `size` bytes of
// splitmix64(seed, 4 + 4t + w), w = 0..3, with the key splitmix64(seed, 0..3),
// and with bit b flipped.
__global__ void __launch_bounds__(256) avalanche_kernel(uint64_t seed, int size, int64_t iters,
                                                        uint64_t* counts) {
  const int b = blockIdx.y;
  const int lane = threadIdx.x & 31;
  uint64_t key[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) key[i] = splitmix64(seed, static_cast<uint64_t>(i));
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  uint32_t acc[2] = {0, 0};
  for (int64_t base = static_cast<int64_t>(blockIdx.x) * blockDim.x; base < iters;
       base += stride) {
    const int64_t t = base + threadIdx.x;
    const bool valid = t < iters;
    uint64_t d = 0;
    if (valid) {
      uint32_t w[8];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const uint64_t r = splitmix64(seed, 4 + 4 * static_cast<uint64_t>(t) + i);
        w[2 * i] = lo32(r);
        w[2 * i + 1] = hi32(r);
      }
      const uint64_t h0 = hash64_upto32(key, w, static_cast<uint32_t>(size), 4);
      uint32_t f[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) f[i] = w[i] ^ ((b >> 5) == i ? (1u << (b & 31)) : 0u);
      d = h0 ^ hash64_upto32(key, f, static_cast<uint32_t>(size), 4);
    }
    count_bits(d, valid, lane, acc);
  }
  atomicAdd(reinterpret_cast<unsigned long long*>(counts + b * 64 + lane), acc[0]);
  atomicAdd(reinterpret_cast<unsigned long long*>(counts + b * 64 + lane + 32), acc[1]);
}

int grid_for(int64_t items, int num_sms) {
  const int64_t blocks = (items + 255) / 256;
  const int64_t cap = int64_t(num_sms) * 8;
  return static_cast<int>(blocks < cap ? (blocks > 0 ? blocks : 1) : cap);
}

int status_of(cudaError_t e) { return e == cudaSuccess ? HH_OK : HH_ERR_CUDA; }

}  // namespace
}  // namespace hh

extern "C" {

int hh_prng_fill(hh_ctx* ctx, int bits, const uint64_t* key, uint64_t counter0, int64_t n,
                 uint64_t* out, void* stream) {
  const int words = bits == 64 ? 1 : bits == 128 ? 2 : bits == 256 ? 4 : 0;
  if (ctx == nullptr || words == 0 || n < 0) return HH_ERR_INVALID_ARG;
  ctx->last_launches = 0;
  if (n == 0) return HH_OK;
  if (key == nullptr || out == nullptr) return HH_ERR_INVALID_ARG;
  hh::DeviceGuard guard(ctx->device);
  if (!guard.ok) return HH_ERR_CUDA;
  auto kern = words == 1 ? hh::prng_kernel<1> : words == 2 ? hh::prng_kernel<2> : hh::prng_kernel<4>;
  kern<<<hh::grid_for(n, ctx->num_sms), 256, 0, static_cast<cudaStream_t>(stream)>>>(key, counter0,
                                                                                    n, out);
  ctx->last_launches = 1;
  return hh::status_of(cudaGetLastError());
}

int hh_stats_round_table(hh_ctx* ctx, const uint64_t* key, int nbytes, int rounds,
                         uint64_t* table, void* stream) {
  if (ctx == nullptr || key == nullptr || table == nullptr || nbytes < 1 || nbytes > 3 ||
      rounds < 0 || rounds > 16)
    return HH_ERR_INVALID_ARG;
  hh::DeviceGuard guard(ctx->device);
  if (!guard.ok) return HH_ERR_CUDA;
  hh::Key4 k{{key[0], key[1], key[2], key[3]}};
  const int64_t count = int64_t(1) << (8 * nbytes);
  hh::round_table_kernel<<<hh::grid_for(count, ctx->num_sms), 256, 0,
                           static_cast<cudaStream_t>(stream)>>>(k, nbytes, rounds, table);
  ctx->last_launches = 1;
  return hh::status_of(cudaGetLastError());
}

int hh_stats_toggle_counts(hh_ctx* ctx, const uint64_t* table, int m, uint64_t* counts,
                           void* stream) {
  if (ctx == nullptr || table == nullptr || counts == nullptr || m < 1 || m > 30)
    return HH_ERR_INVALID_ARG;
  hh::DeviceGuard guard(ctx->device);
  if (!guard.ok) return HH_ERR_CUDA;
  const dim3 grid(hh::grid_for(int64_t(1) << m, ctx->num_sms), m);
  hh::toggle_kernel<<<grid, 256, 0, static_cast<cudaStream_t>(stream)>>>(table, m, counts);
  ctx->last_launches = 1;
  return hh::status_of(cudaGetLastError());
}

int hh_stats_avalanche(hh_ctx* ctx, int size, uint64_t seed, int64_t iterations,
                       uint64_t* counts, void* stream) {
  if (ctx == nullptr || counts == nullptr || size < 1 || size > 32 || iterations < 1)
    return HH_ERR_INVALID_ARG;
  hh::DeviceGuard guard(ctx->device);
  if (!guard.ok) return HH_ERR_CUDA;
  const dim3 grid(hh::grid_for(iterations, ctx->num_sms), 8 * size);
  hh::avalanche_kernel<<<grid, 256, 0, static_cast<cudaStream_t>(stream)>>>(seed, size,
                                                                            iterations, counts);
  ctx->last_launches = 1;
  return hh::status_of(cudaGetLastError());
}

}  // extern "C"

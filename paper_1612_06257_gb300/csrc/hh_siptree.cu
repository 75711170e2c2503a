// hh_siptree.cu -- SipTreeHash (arXiv:1612.06257, Section 3) of ragged
// batches: the paper's tree extension of SipHash, four interleaved SipHash
// lanes whose results are hashed once more.
//
// Per message (readings of the points Section 3 leaves open, as in
// include/hh.h):
//   1. the message is zero-padded to P = ceil(len / 32) vectors of 32 bytes;
//   2. 64-bit little-endian word i of the padded message goes to lane i mod 4,
//      and lane j is the SipHash-c-d of its P words (8P bytes: P
//      compressions, then SipHash's final word, (8P mod 256) << 56);
//   3. the result is the SipHash-c-d of the four lane results followed by
//      the length in bytes (five words, then the final word 40 << 56);
//   4. every SipHash takes the first two 64-bit words of the message's key.
// SipTreeHash uses c = 2 compression and d = 4 finalisation rounds,
// SipTreeHash13 c = 1 and d = 3 (Section 5).
//
// Mapping: one thread per message, its four lane states (16 words) in
// registers, so each 32-byte vector is four independent add-rotate-xor
// chains.  Messages come in warp tiles of 32 from the length sort's order
// (longest first), staged through the same warp-private cp.async ring as
// the HighwayHash warp-tile kernel (WarpStager, hh_stage.cuh); a warp whose
// messages are all at most 64 bytes reads them straight from global memory.
// SipHash is add-rotate-xor on 64-bit words: every operation is two 32-bit
// ALU instructions, except the 32-bit rotations, which are register moves.
#include <cuda_runtime.h>

#include <cstdint>

#include "hh_batch.cuh"
#include "hh_internal.h"
#include "hh_ptx.cuh"
#include "hh_stage.cuh"

namespace hh {
namespace {

// SipHash's initial-state constants: the ASCII text
// "somepseudorandomlygeneratedbytes" as four big-endian 64-bit words.
constexpr uint64_t kSomepseu = 0x736f6d6570736575ull;
constexpr uint64_t kDorandom = 0x646f72616e646f6dull;
constexpr uint64_t kLygenera = 0x6c7967656e657261ull;
constexpr uint64_t kTedbytes = 0x7465646279746573ull;

struct Sip {
  uint64_t v0, v1, v2, v3;
};

__device__ __forceinline__ uint64_t rotl(uint64_t x, int b) { return (x << b) | (x >> (64 - b)); }

__device__ __forceinline__ void sip_init(Sip& s, uint64_t k0, uint64_t k1) {
  s.v0 = k0 ^ kSomepseu;
  s.v1 = k1 ^ kDorandom;
  s.v2 = k0 ^ kLygenera;
  s.v3 = k1 ^ kTedbytes;
}

__device__ __forceinline__ void sip_round(Sip& s) {
  s.v0 += s.v1;
  s.v1 = rotl(s.v1, 13);
  s.v1 ^= s.v0;
  s.v0 = rotl(s.v0, 32);
  s.v2 += s.v3;
  s.v3 = rotl(s.v3, 16);
  s.v3 ^= s.v2;
  s.v0 += s.v3;
  s.v3 = rotl(s.v3, 21);
  s.v3 ^= s.v0;
  s.v2 += s.v1;
  s.v1 = rotl(s.v1, 17);
  s.v1 ^= s.v2;
  s.v2 = rotl(s.v2, 32);
}

template <int C>
__device__ __forceinline__ void sip_compress(Sip& s, uint64_t m) {
  s.v3 ^= m;
#pragma unroll
  for (int i = 0; i < C; ++i) sip_round(s);
  s.v0 ^= m;
}

template <int D>
__device__ __forceinline__ uint64_t sip_finish(Sip& s) {
  s.v2 ^= 0xff;
#pragma unroll
  for (int i = 0; i < D; ++i) sip_round(s);
  return s.v0 ^ s.v1 ^ s.v2 ^ s.v3;
}

// The four lanes of one message.
struct Tree {
  Sip lane[4];
};

__device__ __forceinline__ void tree_init(Tree& t, uint64_t k0, uint64_t k1) {
#pragma unroll
  for (int j = 0; j < 4; ++j) sip_init(t.lane[j], k0, k1);
}

// One 32-byte vector (eight little-endian 32-bit words): word j to lane j.
template <int C>
__device__ __forceinline__ void tree_vector(Tree& t, const uint32_t w[8]) {
#pragma unroll
  for (int j = 0; j < 4; ++j)
    sip_compress<C>(t.lane[j], (static_cast<uint64_t>(w[2 * j + 1]) << 32) | w[2 * j]);
}

// Keep the first `r` (0..32) bytes of a vector, zero the rest.
__device__ __forceinline__ void keep_bytes(uint32_t w[8], uint32_t r) {
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const uint32_t b0 = 4u * i;
    const uint32_t mask = r >= b0 + 4 ? 0xffffffffu
                          : r > b0   ? (1u << (8u * (r - b0))) - 1u
                                     : 0u;
    w[i] &= mask;
  }
}

// The hash of a message of `len` bytes whose `vectors` vectors went into t.
// The four lanes' last compression and finalisation run interleaved, the
// rounds in a loop (not unrolled) to keep the kernel's code small.
template <int C, int D>
__device__ __forceinline__ uint64_t tree_result(Tree& t, int64_t vectors, int64_t len,
                                                uint64_t k0, uint64_t k1) {
  const uint64_t last = static_cast<uint64_t>((8 * vectors) & 0xff) << 56;
#pragma unroll
  for (int j = 0; j < 4; ++j) t.lane[j].v3 ^= last;
#pragma unroll 1
  for (int r = 0; r < C; ++r) {
#pragma unroll
    for (int j = 0; j < 4; ++j) sip_round(t.lane[j]);
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    t.lane[j].v0 ^= last;
    t.lane[j].v2 ^= 0xff;
  }
#pragma unroll 1
  for (int r = 0; r < D; ++r) {
#pragma unroll
    for (int j = 0; j < 4; ++j) sip_round(t.lane[j]);
  }
  uint64_t h[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) h[j] = t.lane[j].v0 ^ t.lane[j].v1 ^ t.lane[j].v2 ^ t.lane[j].v3;
  Sip f;
  sip_init(f, k0, k1);
#pragma unroll
  for (int j = 0; j < 4; ++j) sip_compress<C>(f, h[j]);
  sip_compress<C>(f, static_cast<uint64_t>(len));
  sip_compress<C>(f, static_cast<uint64_t>(40) << 56);
  return sip_finish<D>(f);
}

// Step k of a staged message: its whole vectors in the window, and the
// zero-padded partial vector if the window holds it.
template <int W, bool kAligned, int C>
__device__ __forceinline__ void tree_step(Tree& t, const uint8_t* row, uint32_t mis, int64_t k,
                                          int64_t whole, uint32_t r, int64_t rem_step) {
  const int64_t p0 = k * (W / 32);
  const int64_t left = whole - p0;
  const int count = left <= 0 ? 0 : (left < W / 32 ? static_cast<int>(left) : W / 32);
  // Two vectors per loop iteration: each is four independent chains already,
  // and a fully unrolled window would overflow the instruction cache.
#pragma unroll 2
  for (int j = 0; j < count; ++j) {
    uint32_t w[8];
    read_packet<kAligned>(row, mis + 32u * j, w);
    tree_vector<C>(t, w);
  }
  if (k == rem_step) {
    uint32_t w[8];
    read_packet<false>(row, mis + static_cast<uint32_t>(whole * 32 - k * W), w);
    keep_bytes(w, r);
    tree_vector<C>(t, w);
  }
}

template <int W, int NST, int WARPS, int C, int D>
__global__ void __launch_bounds__(WARPS * 32, 3) siptree_kernel(Batch b, Queue q) {
  using L = RaggedLayout<W, NST>;
  extern __shared__ __align__(128) uint8_t smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint8_t* ring = smem + warp * L::kWarpBytes;
  const uint32_t ring_s = smem_u32(ring);
  resolve_count(b);

  int64_t lo, hi;
  batch_range(b, lo, hi);
  const uintptr_t base = reinterpret_cast<uintptr_t>(b.bytes);
  const uintptr_t safe_lo = (base + lo + 15) & ~uintptr_t(15);
  const uintptr_t safe_hi = (base + hi) & ~uintptr_t(15);
  const int32_t* perm = (q.perm && (q.use_perm == nullptr || *q.use_perm)) ? q.perm : nullptr;
  const int64_t tiles = (b.n + 31) / 32;
  int64_t static_tile = static_cast<int64_t>(blockIdx.x) * WARPS + warp;
  const int64_t static_step = static_cast<int64_t>(gridDim.x) * WARPS;

  for (;;) {
    int64_t tile;
    if (q.next_tile) {
      unsigned long long tk = 0;
      if (lane == 0) tk = atomicAdd(q.next_tile, 1ull);
      tile = static_cast<int64_t>(__shfl_sync(kFull, tk, 0));
    } else {
      tile = static_tile;
      static_tile += static_step;
    }
    if (tile >= tiles) break;

    const int64_t idx = tile * 32 + lane;
    const bool valid = idx < b.n;
    int64_t m = 0, start = 0, len = 0;
    int bad = 0;
    uint64_t k0 = 0, k1 = 0;
    if (valid) {
      m = perm ? static_cast<int64_t>(perm[idx]) : idx;
      message_bounds(b, m, start, len, bad);
      if (bad) record_error(b.err, bad);
      const uint64_t* kp = key_of(b, m);
      k0 = __ldg(kp);
      k1 = __ldg(kp + 1);
    }
    Tree t;
    tree_init(t, k0, k1);
    const int64_t whole = len >> 5;
    const uint32_t r = static_cast<uint32_t>(len & 31);
    const int64_t vectors = whole + (r != 0);

    if (__all_sync(kFull, len <= 64)) {
      // At most two vectors, read straight from global memory.
      uint32_t x[17];
      load_short_words(x, base + start, static_cast<uint32_t>(len), base + lo, base + hi);
      const uint32_t sel = 0x3210u + 0x1111u * static_cast<uint32_t>((base + start) & 3);
      uint32_t v0[8], v1[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        v0[j] = __byte_perm(x[j], x[j + 1], sel);
        v1[j] = __byte_perm(x[8 + j], x[9 + j], sel);
      }
      const uint32_t n32 = static_cast<uint32_t>(len);
      keep_bytes(v0, n32 < 32u ? n32 : 32u);
      keep_bytes(v1, n32 > 32u ? n32 - 32u : 0u);
      if (vectors > 0) tree_vector<C>(t, v0);
      if (vectors > 1) tree_vector<C>(t, v1);
    } else {
      const int64_t my_steps = (len + W - 1) / W;
      const int64_t steps = warp_max(my_steps);
      const uintptr_t msg = base + start;
      const uint32_t mis = static_cast<uint32_t>(msg & 15);
      const bool aligned = __all_sync(kFull, mis == 0 || !valid);
      const int64_t rem_step = r ? (whole * 32) / W : -1;
      const WarpStager<W, NST> stager{ring, ring_s, msg, len, my_steps,
                                      spread_row(aligned, valid, mis, lane), safe_lo, safe_hi,
                                      lane};
      stager.run(steps, [&](int64_t k, const uint8_t* row) {
        if (k < my_steps) {
          if (aligned)  // warp-uniform
            tree_step<W, true, C>(t, row, 0u, k, whole, r, rem_step);
          else
            tree_step<W, false, C>(t, row, mis, k, whole, r, rem_step);
        }
      });
    }
    const uint64_t h = tree_result<C, D>(t, vectors, len, k0, k1);
    if (valid) b.out[m] = bad ? 0ull : h;
  }
}

template <int C, int D>
cudaError_t launch_siptree_t(const Batch& b, const Queue& q, int num_sms, cudaStream_t stream) {
  constexpr int W = 256, NST = 2, WARPS = 4;
  using L = RaggedLayout<W, NST>;
  constexpr int kBytes = WARPS * L::kWarpBytes;
  auto kern = siptree_kernel<W, NST, WARPS, C, D>;
  cudaError_t e;
  const int per_sm = blocks_per_sm(reinterpret_cast<const void*>(kern), WARPS * 32, kBytes, &e);
  if (e != cudaSuccess) return e;
  const int64_t blocks_needed = ((b.n + 31) / 32 + WARPS - 1) / WARPS;
  const int64_t cap = static_cast<int64_t>(per_sm) * num_sms;
  const int grid = static_cast<int>(blocks_needed < cap ? blocks_needed : cap);
  if (grid <= 0) return cudaSuccess;
  kern<<<grid, WARPS * 32, kBytes, stream>>>(b, q);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_siptree(const Batch& b, const Queue& q, int variant, int num_sms,
                           cudaStream_t stream) {
  if (variant == kSipTree24) return launch_siptree_t<2, 4>(b, q, num_sms, stream);
  if (variant == kSipTree13) return launch_siptree_t<1, 3>(b, q, num_sms, stream);
  return cudaErrorInvalidValue;
}

}  // namespace hh

// hh_device.cuh -- per-message HighwayHash arithmetic for sm_103a.
//
// HighwayHash (arXiv:1612.06257, Section 4) keeps a 1024-bit state per
// message in registers: four vectors v0, v1, mul0, mul1 of four 64-bit lanes
// (Section 4.2).  All arithmetic is exact modulo 2^64; the 32x32->64-bit
// multiply compiles to IMAD.WIDE.U32 and ZipperMerge to six PRMT (byte_perm)
// per lane pair.  Nothing here is shared with the CPU checker.
#pragma once

#include <cstdint>

namespace hh {

// ---------------------------------------------------------------- Section 4.4
// The first eight 64-bit words of pi's hexadecimal fraction (3.243F6A88...).
// Words 0-3 give the first constant, words 4-7 the second.  Written most
// significant lane first, so word 0 is lane 3 and the fourth word lane 0;
// lane 0 then gets every bit that fewer than two of the other lanes have.
// (A function rather than a table: device code cannot read a host array.)
__host__ __device__ constexpr uint64_t pi_frac(int i) {
  return i == 0 ? 0x243F6A8885A308D3ull : i == 1 ? 0x13198A2E03707344ull
       : i == 2 ? 0xA4093822299F31D0ull : i == 3 ? 0x082EFA98EC4E6C89ull
       : i == 4 ? 0x452821E638D01377ull : i == 5 ? 0xBE5466CF34E90C6Cull
       : i == 6 ? 0xC0AC29B7C97C50DDull : 0x3F84D5B5B5470917ull;
}

__host__ __device__ constexpr uint64_t at_least_two_of(uint64_t a, uint64_t b, uint64_t c) {
  return (a & b) | (c & (a | b));
}

__host__ __device__ constexpr uint64_t init_lane(int which, int lane) {
  return lane == 3 ? pi_frac(4 * which + 0)
       : lane == 2 ? pi_frac(4 * which + 1)
       : lane == 1 ? pi_frac(4 * which + 2)
                   : pi_frac(4 * which + 3) |
                         ~at_least_two_of(pi_frac(4 * which), pi_frac(4 * which + 1),
                                          pi_frac(4 * which + 2));
}

struct State {
  uint64_t v0[4], v1[4], mul0[4], mul1[4];
};

__device__ __forceinline__ uint32_t lo32(uint64_t x) { return static_cast<uint32_t>(x); }
__device__ __forceinline__ uint32_t hi32(uint64_t x) { return static_cast<uint32_t>(x >> 32); }
__device__ __forceinline__ uint64_t join(uint32_t lo, uint32_t hi) {
  return (static_cast<uint64_t>(hi) << 32) | lo;
}
__device__ __forceinline__ uint64_t swap_halves(uint64_t x) { return join(hi32(x), lo32(x)); }

// Section 4.4: v0 = key ^ C0, v1 = (key, 32-bit halves swapped) ^ C1,
// mul0 = C0, mul1 = C1.
__device__ __forceinline__ void init(State& s, const uint64_t key[4]) {
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const uint64_t c0 = init_lane(0, i), c1 = init_lane(1, i);
    s.v0[i] = key[i] ^ c0;
    s.v1[i] = swap_halves(key[i]) ^ c1;
    s.mul0[i] = c0;
    s.mul1[i] = c1;
  }
}

// ---------------------------------------------------------------- Section 4.1
// ZipperMerge of one lane pair, added into dst.  With the pair's bytes
// S0..S15 (lane a then lane b, little-endian) in 32-bit words w0..w3, result
// byte i is S[P_i] for P = 3 12 2 5 14 1 15 0 | 11 4 10 13 9 6 8 7 (i = 0..15,
// the printed map reversed).  Per result word:
//   a.lo = w0.b3 w3.b0 w0.b2 w1.b1     a.hi = w3.b2 w0.b1 w3.b3 w0.b0
//   b.lo = w2.b3 w1.b0 w2.b2 w3.b1     b.hi = w2.b1 w1.b2 w2.b0 w1.b3
__device__ __forceinline__ void zipper_add_pair(uint64_t& dst_a, uint64_t& dst_b,
                                                uint64_t a, uint64_t b) {
  const uint32_t w0 = lo32(a), w1 = hi32(a), w2 = lo32(b), w3 = hi32(b);
  const uint32_t a_lo = __byte_perm(__byte_perm(w0, w3, 0x0243), w1, 0x5210);
  const uint32_t a_hi = __byte_perm(w0, w3, 0x0716);
  const uint32_t b_lo = __byte_perm(__byte_perm(w2, w1, 0x0243), w3, 0x5210);
  const uint32_t b_hi = __byte_perm(w2, w1, 0x7061);
  dst_a += join(a_lo, a_hi);
  dst_b += join(b_lo, b_hi);
}

// _mm256_mul_epu32 per lane: low 32 bits times low 32 bits, 64-bit product.
__device__ __forceinline__ uint64_t mul_lo(uint64_t a, uint64_t b) {
  return static_cast<uint64_t>(lo32(a)) * lo32(b);
}

// ---------------------------------------------------------------- Section 4.2
// x + y with both halves on the multiply-add (FMA) pipe:
//   t = lo(y) * one + x (64-bit mad.wide), then hi(t) += hi(y) * one.
// `one` is always 1 but arrives at run time, so the compiler cannot turn
// these back into IADD3; moving adds to the FMA pipe relieves the ALU pipe,
// which runs the PRMT, LOP3 and remaining IADD3 of Update.
__device__ __forceinline__ uint64_t add_on_fma(uint64_t x, uint64_t y, uint32_t one) {
  uint64_t t;
  asm("mad.wide.u32 %0, %1, %2, %3;" : "=l"(t) : "r"(lo32(y)), "r"(one), "l"(x));
  uint32_t hi;
  asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(hi) : "r"(hi32(y)), "r"(one), "r"(hi32(t)));
  return join(lo32(t), hi);
}

// ZipperMerge of a lane pair as two words (no add).
__device__ __forceinline__ void zipper_pair(uint64_t a, uint64_t b, uint64_t& za, uint64_t& zb) {
  const uint32_t w0 = lo32(a), w1 = hi32(a), w2 = lo32(b), w3 = hi32(b);
  za = join(__byte_perm(__byte_perm(w0, w3, 0x0243), w1, 0x5210), __byte_perm(w0, w3, 0x0716));
  zb = join(__byte_perm(__byte_perm(w2, w1, 0x0243), w3, 0x5210), __byte_perm(w2, w1, 0x7061));
}

// Update variants: the same arithmetic, with the 64-bit additions split
// differently between the ALU and FMA pipes (see the microbenchmark).
//   0: plain C, the compiler's choice.
//   1: v0 + mul1 + ZM(v1) as one 3-input add; only lo(v0 + mul1) is formed
//      separately for the multiply.
//   2: as 1, and v1 += ZM(v0) on the FMA pipe.
//   3: v0 += mul1 on the ALU, v0 += ZM(v1) and v1 += ZM(v0) on the FMA pipe.
//   4: as 3, and v1 += packet + mul0 on the FMA pipe as well.
//   5: as 1, with the 32-bit lo(v0 + mul1) as a multiply-add on the FMA pipe.
template <int V, int N>
__device__ __forceinline__ void update_lanes(uint64_t (&v0)[N], uint64_t (&v1)[N],
                                             uint64_t (&mul0)[N], uint64_t (&mul1)[N],
                                             const uint64_t (&p)[N], uint32_t one) {
  static_assert(N == 2 || N == 4, "lanes come in ZipperMerge pairs");
  if constexpr (V == 0) {
#pragma unroll
    for (int i = 0; i < N; ++i) {
      v1[i] += p[i] + mul0[i];
      mul0[i] ^= mul_lo(v1[i], v0[i] >> 32);
      v0[i] += mul1[i];
      mul1[i] ^= mul_lo(v0[i], v1[i] >> 32);
    }
#pragma unroll
    for (int i = 0; i < N; i += 2) zipper_add_pair(v0[i], v0[i + 1], v1[i], v1[i + 1]);
#pragma unroll
    for (int i = 0; i < N; i += 2) zipper_add_pair(v1[i], v1[i + 1], v0[i], v0[i + 1]);
  } else {
    // V 1, 2, 5: add[i] = mul1 before its update (v0 + add + ZM(v1) is
    // one 3-input add later).  V 3-4: add[i] = v0 + mul1, formed now.
    uint64_t add[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
      if (V == 4) v1[i] = add_on_fma(add_on_fma(v1[i], p[i], one), mul0[i], one);
      else v1[i] += p[i] + mul0[i];
      mul0[i] ^= mul_lo(v1[i], v0[i] >> 32);
      if (V == 3 || V == 4) {
        add[i] = v0[i] + mul1[i];
        mul1[i] ^= mul_lo(add[i], v1[i] >> 32);
      } else if (V == 5) {
        add[i] = mul1[i];
        uint32_t lo;  // lo(v0 + mul1) = lo(v0) * one + lo(mul1)
        asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(lo) : "r"(lo32(v0[i])), "r"(one), "r"(lo32(add[i])));
        mul1[i] ^= static_cast<uint64_t>(lo) * hi32(v1[i]);
      } else {
        add[i] = mul1[i];
        const uint32_t lo = lo32(v0[i]) + lo32(add[i]);  // lo(v0 + mul1)
        mul1[i] ^= static_cast<uint64_t>(lo) * hi32(v1[i]);
      }
    }
    uint64_t z[N];
#pragma unroll
    for (int i = 0; i < N; i += 2) zipper_pair(v1[i], v1[i + 1], z[i], z[i + 1]);
#pragma unroll
    for (int i = 0; i < N; ++i)
      v0[i] = (V >= 3 && V <= 4) ? add_on_fma(add[i], z[i], one) : v0[i] + add[i] + z[i];
#pragma unroll
    for (int i = 0; i < N; i += 2) zipper_pair(v0[i], v0[i + 1], z[i], z[i + 1]);
#pragma unroll
    for (int i = 0; i < N; ++i)
      v1[i] = (V >= 2 && V <= 4) ? add_on_fma(v1[i], z[i], one) : v1[i] + z[i];
  }
}

template <int V>
__device__ __forceinline__ void update_v(State& s, const uint64_t (&p)[4], uint32_t one) {
  update_lanes<V, 4>(s.v0, s.v1, s.mul0, s.mul1, p, one);
}

// The variant every kernel uses: fastest in the Update-rate microbenchmark on
// GB300.  One 32-bit add on the FMA pipe gains 1.5% (whole state) and 3% (a
// lane pair) over the all-ALU variant 1; moving the 64-bit adds to
// IMAD.WIDE (variants 2-4) was slower.
constexpr int kFastUpdate = 5;

__device__ __forceinline__ void update(State& s, const uint64_t (&p)[4]) {
  update_v<kFastUpdate>(s, p, 1u);
}

// Packet from eight little-endian 32-bit words.
template <int V>
__device__ __forceinline__ void update_words_v(State& s, const uint32_t w[8], uint32_t one) {
  const uint64_t p[4] = {join(w[0], w[1]), join(w[2], w[3]), join(w[4], w[5]), join(w[6], w[7])};
  update_v<V>(s, p, one);
}

__device__ __forceinline__ void update_words(State& s, const uint32_t w[8]) {
  update_words_v<kFastUpdate>(s, w, 1u);
}

// ---------------------------------------------------------------- Section 4.5
// Size injection for r = size mod 32: add (r << 32) + r to each lane of v0
// and rotate each 32-bit half of v1 left by r.  r == 0 changes nothing.
__device__ __forceinline__ void inject_size(State& s, uint32_t r) {
  const uint64_t inject = (static_cast<uint64_t>(r) << 32) + r;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    s.v0[i] += inject;
    const uint32_t lo = lo32(s.v1[i]), hi = hi32(s.v1[i]);
    s.v1[i] = join(__funnelshift_l(lo, lo, r), __funnelshift_l(hi, hi, r));
  }
}

// The padded packet of the last r bytes (tail[0..7] hold the bytes after the
// last whole packet; only the first r are meaningful): whole 4-byte groups
// stay in place, the last r mod 4 bytes go to bytes 28.., all else zero.
__device__ __forceinline__ void remainder_packet(uint32_t r, const uint32_t tail[8],
                                                 uint32_t pkt[8]) {
  const uint32_t whole = r >> 2, extra = r & 3;
  uint32_t last = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    pkt[j] = (static_cast<uint32_t>(j) < whole) ? tail[j] : 0u;
    last = (static_cast<uint32_t>(j) == whole) ? tail[j] : last;
  }
  if (extra) pkt[7] |= last & ((1u << (8 * extra)) - 1u);
}

__device__ __forceinline__ void remainder(State& s, uint32_t r, const uint32_t tail[8]) {
  if (r == 0) return;
  inject_size(s, r);
  uint32_t pkt[8];
  remainder_packet(r, tail, pkt);
  update_words(s, pkt);
}

// ------------------------------------------------ one lane pair per thread
// For very long messages two threads share one message: thread `half` keeps
// lanes 2*half and 2*half+1 of every state vector.  Update mixes lanes only
// within a pair (ZipperMerge, Section 4.1), so the packet loop needs no
// exchange; the two threads trade v0 only in the finalisation Permute.
struct Half {
  uint64_t v0[2], v1[2], mul0[2], mul1[2];
};

__device__ __forceinline__ void init_half(Half& s, const uint64_t key[4], int half) {
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const uint64_t k = half ? key[2 + j] : key[j];  // no run-time array index
    const uint64_t c0 = half ? init_lane(0, 2 + j) : init_lane(0, j);
    const uint64_t c1 = half ? init_lane(1, 2 + j) : init_lane(1, j);
    s.v0[j] = k ^ c0;
    s.v1[j] = swap_halves(k) ^ c1;
    s.mul0[j] = c0;
    s.mul1[j] = c1;
  }
}

// Update of one lane pair (variant V as for update_v).
template <int V>
__device__ __forceinline__ void update_half_v(Half& s, uint64_t p0, uint64_t p1, uint32_t one) {
  const uint64_t p[2] = {p0, p1};
  update_lanes<V, 2>(s.v0, s.v1, s.mul0, s.mul1, p, one);
}

__device__ __forceinline__ void update_half(Half& s, uint64_t p0, uint64_t p1) {
  update_half_v<kFastUpdate>(s, p0, p1, 1u);
}

__device__ __forceinline__ void inject_size_half(Half& s, uint32_t r) {
  const uint64_t inject = (static_cast<uint64_t>(r) << 32) + r;
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    s.v0[i] += inject;
    const uint32_t lo = lo32(s.v1[i]), hi = hi32(s.v1[i]);
    s.v1[i] = join(__funnelshift_l(lo, lo, r), __funnelshift_l(hi, hi, r));
  }
}

// Four rounds of Update(Permute(v0)) for a lane pair; all 32 lanes of the
// warp must call it (partners are lanes l and l ^ 1).  Permute gives lane
// pair (0,1) the rotated v0 lanes (2,3) and vice versa.
__device__ __forceinline__ void finalize_half(Half& s) {
#pragma unroll
  for (int round = 0; round < 4; ++round) {
    const uint64_t o0 = __shfl_xor_sync(0xffffffffu, s.v0[0], 1);
    const uint64_t o1 = __shfl_xor_sync(0xffffffffu, s.v0[1], 1);
    update_half(s, swap_halves(o0), swap_halves(o1));
  }
}

// ---------------------------------------------------------------- Section 4.3
// Four rounds of Update(Permute(v0)); Permute swaps v0's 128-bit halves and
// the 32-bit halves of every lane (index map 2 3 0 1 6 7 4 5).
__device__ __forceinline__ void finalize(State& s) {
#pragma unroll
  for (int round = 0; round < 4; ++round) {
    const uint64_t p[4] = {swap_halves(s.v0[2]), swap_halves(s.v0[3]), swap_halves(s.v0[0]),
                           swap_halves(s.v0[1])};
    update(s, p);
  }
}

// `rounds` rounds of Update(Permute(v0)) (the hash uses 4; other counts
// serve the study of how many rounds finalisation needs, Section 4.3).
__device__ __forceinline__ void finalize_rounds(State& s, int rounds) {
#pragma unroll 1
  for (int round = 0; round < rounds; ++round) {
    const uint64_t p[4] = {swap_halves(s.v0[2]), swap_halves(s.v0[3]), swap_halves(s.v0[0]),
                           swap_halves(s.v0[1])};
    update(s, p);
  }
}

// h[i] = v0[i] + v1[i] + mul0[i] + mul1[i]; the 64-bit hash is h[0], the
// 128-bit hash h[0..1], the 256-bit hash h[0..3].
__device__ __forceinline__ void digest(const State& s, uint64_t h[4]) {
#pragma unroll
  for (int i = 0; i < 4; ++i) h[i] = s.v0[i] + s.v1[i] + s.mul0[i] + s.mul1[i];
}

}  // namespace hh

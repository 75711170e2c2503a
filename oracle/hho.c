/*
 * hho.c -- scalar CPU oracle for HighwayHash (arXiv:1612.06257, Section 4).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * benchmark's CPU-baseline leg, never by the product path.  Plain C99, one
 * 64-bit lane at a time, each step in the order the paper gives it.  No
 * blocking, fusion or reordering.  See hho.h for what pins each function.
 */
#include "hho.h"

#include <string.h>

/* Section 4.4: the constants start from the hexadecimal digits of pi.  These
 * are the first eight 64-bit words of pi's fractional part (0x243F6A88... is
 * the start of 3.243F6A88...).  The first four make the first constant, the
 * next four the second.  A test recomputes them from Machin's formula. */
static const uint64_t kPiWords[8] = {
    0x243F6A8885A308D3ull, 0x13198A2E03707344ull, 0xA4093822299F31D0ull,
    0x082EFA98EC4E6C89ull, 0x452821E638D01377ull, 0xBE5466CF34E90C6Cull,
    0xC0AC29B7C97C50DDull, 0x3F84D5B5B5470917ull};

/* Section 4.1: the final ZipperMerge byte map exactly as printed, i.e. with
 * the offset for result byte i = 15 first and i = 0 last (hexadecimal). */
static const int kZipperPrinted[16] = {0x7, 0x8, 0x6, 0x9, 0xD, 0xA, 0x4, 0xB,
                                       0x0, 0xF, 0x1, 0xE, 0x5, 0x2, 0xC, 0x3};

/* Section 4.3: the Permute indices of 32-bit parts exactly as printed.  The
 * listing follows the same convention as the ZipperMerge map: the index for
 * the most significant part (part 7) comes first. */
static const int kPermutePrinted[8] = {2, 3, 0, 1, 6, 7, 4, 5};

/* Section 4.2: _mm256_mul_epu32 multiplies the lower 32 bits of each lane,
 * giving a full 64-bit product. */
static uint64_t mul_lo32(uint64_t a, uint64_t b) {
  return (a & 0xFFFFFFFFull) * (b & 0xFFFFFFFFull);
}

static uint64_t majority(uint64_t a, uint64_t b, uint64_t c) {
  return (a & b) | (a & c) | (b & c);
}

/* Section 4.4: a 256-bit number written most-significant word first, so the
 * first pi word is lane 3 and the fourth word is lane 0.  Lane 0 gets
 * every bit set that at most one of the other three lanes has set, i.e.
 * every bit where the other three do not hold a majority of ones. */
static void make_constant(const uint64_t w[4], uint64_t c[4]) {
  c[3] = w[0];
  c[2] = w[1];
  c[1] = w[2];
  c[0] = w[3] | ~majority(w[0], w[1], w[2]);
}

void hho_constants(uint64_t c0[4], uint64_t c1[4]) {
  make_constant(&kPiWords[0], c0);
  make_constant(&kPiWords[4], c1);
}

static uint64_t rot32(uint64_t x) { return (x << 32) | (x >> 32); }

/* Section 4.4: v0 = key ^ C0, v1 = (key lanes rotated by 32 bits) ^ C1,
 * mul0 = C0, mul1 = C1. */
void hho_init(hho_state* s, const uint64_t key[4]) {
  uint64_t c0[4], c1[4];
  int i;
  hho_constants(c0, c1);
  for (i = 0; i < 4; ++i) {
    s->v0[i] = key[i] ^ c0[i];
    s->v1[i] = rot32(key[i]) ^ c1[i];
    s->mul0[i] = c0[i];
    s->mul1[i] = c1[i];
  }
}

/* Section 4.1: for each 16-byte lane pair S (lane 2k's bytes then lane
 * 2k+1's bytes, little-endian), result byte R_i = S_{P_i}. */
void hho_zipper_merge(const uint64_t in[4], uint64_t out[4]) {
  int pair, i;
  for (pair = 0; pair < 2; ++pair) {
    uint8_t src[16], res[16];
    uint64_t lo = 0, hi = 0;
    for (i = 0; i < 8; ++i) {
      src[i] = (uint8_t)(in[2 * pair] >> (8 * i));
      src[8 + i] = (uint8_t)(in[2 * pair + 1] >> (8 * i));
    }
    for (i = 0; i < 16; ++i) res[i] = src[kZipperPrinted[15 - i]];
    for (i = 7; i >= 0; --i) {
      lo = (lo << 8) | res[i];
      hi = (hi << 8) | res[8 + i];
    }
    out[2 * pair] = lo;
    out[2 * pair + 1] = hi;
  }
}

/* Section 4.2, statement by statement over all four lanes. */
void hho_update(hho_state* s, const uint64_t packet[4]) {
  uint64_t zm[4];
  int i;
  for (i = 0; i < 4; ++i) s->v1[i] += packet[i];
  for (i = 0; i < 4; ++i) s->v1[i] += s->mul0[i];
  for (i = 0; i < 4; ++i) s->mul0[i] ^= mul_lo32(s->v1[i], s->v0[i] >> 32);
  for (i = 0; i < 4; ++i) s->v0[i] += s->mul1[i];
  for (i = 0; i < 4; ++i) s->mul1[i] ^= mul_lo32(s->v0[i], s->v1[i] >> 32);
  hho_zipper_merge(s->v1, zm);
  for (i = 0; i < 4; ++i) s->v0[i] += zm[i];
  hho_zipper_merge(s->v0, zm);
  for (i = 0; i < 4; ++i) s->v1[i] += zm[i];
}

/* Section 4.3: a 256-bit permute of 32-bit parts.  Part j of the result is
 * part idx[j] of v0, where idx[j] is the printed entry for part j counted
 * from the most significant end.  Part 2i is the low half of lane i. */
void hho_permute(const uint64_t v0[4], uint64_t out[4]) {
  uint32_t part[8], res[8];
  int j;
  for (j = 0; j < 4; ++j) {
    part[2 * j] = (uint32_t)v0[j];
    part[2 * j + 1] = (uint32_t)(v0[j] >> 32);
  }
  for (j = 0; j < 8; ++j) res[j] = part[kPermutePrinted[7 - j]];
  for (j = 0; j < 4; ++j) out[j] = ((uint64_t)res[2 * j + 1] << 32) | res[2 * j];
}

static uint32_t rotl32(uint32_t w, unsigned r) {
  r &= 31u;
  return r ? (uint32_t)((w << r) | (w >> (32u - r))) : w;
}

static uint64_t load_le64(const uint8_t* p) {
  uint64_t x = 0;
  int i;
  for (i = 7; i >= 0; --i) x = (x << 8) | p[i];
  return x;
}

/* Section 4.5.  For r = size mod 32 != 0:
 *  - r is broadcast into the eight 32-bit parts of a vector and added to v0
 *    (one 64-bit add of (r << 32) + r per lane);
 *  - each 32-bit half of every v1 lane is rotated left by r;
 *  - the packet holds the leading multiple-of-4 bytes of the tail in place
 *    and the last r mod 4 bytes in its most significant four bytes (bytes
 *    28, 29, 30 in order), all other bytes zero; then one Update.
 * Sizes that are multiples of 32 need no padding, so r == 0 does nothing. */
void hho_remainder(hho_state* s, const uint8_t* tail, size_t r) {
  uint8_t pkt[32];
  uint64_t words[4];
  size_t q, k;
  int i;
  if (r == 0) return;
  for (i = 0; i < 4; ++i) {
    s->v0[i] += ((uint64_t)r << 32) + (uint64_t)r;
    s->v1[i] = ((uint64_t)rotl32((uint32_t)(s->v1[i] >> 32), (unsigned)r) << 32) |
               (uint64_t)rotl32((uint32_t)s->v1[i], (unsigned)r);
  }
  memset(pkt, 0, sizeof(pkt));
  q = r & ~(size_t)3;
  for (k = 0; k < q; ++k) pkt[k] = tail[k];
  for (k = 0; k < (r & 3); ++k) pkt[28 + k] = tail[q + k];
  for (i = 0; i < 4; ++i) words[i] = load_le64(pkt + 8 * i);
  hho_update(s, words);
}

void hho_finalize(hho_state* s, int rounds) {
  uint64_t p[4];
  int round;
  for (round = 0; round < rounds; ++round) {
    hho_permute(s->v0, p);
    hho_update(s, p);
  }
}

void hho_output(const hho_state* s, uint64_t h[4]) {
  int i;
  for (i = 0; i < 4; ++i) h[i] = s->v0[i] + s->v1[i] + s->mul0[i] + s->mul1[i];
}

int hho_hash_rounds(const uint64_t key[4], const uint8_t* msg, size_t len,
                    int bits, int rounds, uint64_t* out) {
  hho_state s;
  uint64_t words[4], h[4];
  size_t pos, full = len & ~(size_t)31;
  int i;
  if (bits != 64 && bits != 128 && bits != 256) return -1;
  hho_init(&s, key);
  for (pos = 0; pos < full; pos += 32) {
    for (i = 0; i < 4; ++i) words[i] = load_le64(msg + pos + 8 * i);
    hho_update(&s, words);
  }
  hho_remainder(&s, msg + full, len - full);
  hho_finalize(&s, rounds);
  hho_output(&s, h);
  for (i = 0; i < bits / 64; ++i) out[i] = h[i];
  return 0;
}

void hho_hash64(const uint64_t key[4], const uint8_t* msg, size_t len, uint64_t* out) {
  hho_hash_rounds(key, msg, len, 64, 4, out);
}

void hho_hash128(const uint64_t key[4], const uint8_t* msg, size_t len, uint64_t* out) {
  hho_hash_rounds(key, msg, len, 128, 4, out);
}

void hho_hash256(const uint64_t key[4], const uint8_t* msg, size_t len, uint64_t* out) {
  hho_hash_rounds(key, msg, len, 256, 4, out);
}

int hho_hash_batch(const uint64_t* keys, int per_message_keys, const uint8_t* bytes,
                   const int64_t* offsets, int64_t first, int64_t last, int bits,
                   uint64_t* out) {
  int64_t i;
  int words = bits / 64;
  if (bits != 64 && bits != 128 && bits != 256) return -1;
  for (i = first; i < last; ++i) {
    const uint64_t* key = per_message_keys ? keys + 4 * i : keys;
    if (offsets[i + 1] < offsets[i]) return -1;
    hho_hash_rounds(key, bytes + offsets[i], (size_t)(offsets[i + 1] - offsets[i]), bits, 4,
                    out + (i - first) * words);
  }
  return 0;
}

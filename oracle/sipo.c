/*
 * sipo.c -- scalar CPU oracle for SipTreeHash (arXiv:1612.06257, Section 3;
 * Section 5 for the round counts).  TEST INFRASTRUCTURE ONLY: see sipo.h for
 * the readings T1-T5 and what pins each function.
 *
 * Plain C99, written for reading, not for speed: SipHash is computed as its
 * published definition states it (Aumasson and Bernstein, 2012), and the
 * tree is built literally: the padded message, one byte string per lane,
 * one SipHash per lane, one SipHash of the lane results and the length.
 */
#include "sipo.h"

#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------ SipHash */

static uint64_t rotl64(uint64_t x, int b) { return (x << b) | (x >> (64 - b)); }

/* Little-endian 64-bit word from 8 bytes. */
static uint64_t load_le64(const uint8_t* p) {
  uint64_t x = 0;
  int i;
  for (i = 7; i >= 0; --i) x = (x << 8) | p[i];
  return x;
}

static void store_le64(uint8_t* p, uint64_t x) {
  int i;
  for (i = 0; i < 8; ++i) p[i] = (uint8_t)(x >> (8 * i));
}

/* SipHash's initial-state constants are the ASCII text
 * "somepseudorandomlygeneratedbytes" read as four big-endian 64-bit words. */
static uint64_t ascii_constant(int which) {
  static const char kText[] = "somepseudorandomlygeneratedbytes";
  uint64_t x = 0;
  int i;
  for (i = 0; i < 8; ++i) x = (x << 8) | (uint8_t)kText[8 * which + i];
  return x;
}

typedef struct sip_state {
  uint64_t v0, v1, v2, v3;
} sip_state;

/* One SipRound: three add-rotate-xor half rounds on (v0, v1) and (v2, v3). */
static void sip_round(sip_state* s) {
  s->v0 += s->v1;
  s->v1 = rotl64(s->v1, 13);
  s->v1 ^= s->v0;
  s->v0 = rotl64(s->v0, 32);
  s->v2 += s->v3;
  s->v3 = rotl64(s->v3, 16);
  s->v3 ^= s->v2;
  s->v0 += s->v3;
  s->v3 = rotl64(s->v3, 21);
  s->v3 ^= s->v0;
  s->v2 += s->v1;
  s->v1 = rotl64(s->v1, 17);
  s->v1 ^= s->v2;
  s->v2 = rotl64(s->v2, 32);
}

/* Compression of one 8-byte word m: v3 ^= m, c SipRounds, v0 ^= m. */
static void sip_compress(sip_state* s, uint64_t m, int c) {
  int r;
  s->v3 ^= m;
  for (r = 0; r < c; ++r) sip_round(s);
  s->v0 ^= m;
}

uint64_t sipo_siphash(uint64_t k0, uint64_t k1, const uint8_t* msg, size_t len, int c, int d) {
  sip_state s;
  size_t i, whole = len / 8;
  uint64_t last;
  int r;
  s.v0 = k0 ^ ascii_constant(0);
  s.v1 = k1 ^ ascii_constant(1);
  s.v2 = k0 ^ ascii_constant(2);
  s.v3 = k1 ^ ascii_constant(3);
  for (i = 0; i < whole; ++i) sip_compress(&s, load_le64(msg + 8 * i), c);
  /* The final word: the len mod 8 remaining bytes (little-endian) with
   * len mod 256 in the most significant byte. */
  last = (uint64_t)(len & 0xff) << 56;
  for (i = 0; i < (len & 7); ++i) last |= (uint64_t)msg[8 * whole + i] << (8 * i);
  sip_compress(&s, last, c);
  s.v2 ^= 0xff;
  for (r = 0; r < d; ++r) sip_round(&s);
  return s.v0 ^ s.v1 ^ s.v2 ^ s.v3;
}

/* --------------------------------------------------------- SipTreeHash */

void sipo_tree_lanes(const uint64_t key[4], const uint8_t* msg, size_t len, int c, int d,
                     uint64_t lanes[4]) {
  /* T1: P whole 32-byte vectors, the tail zero-padded. */
  const size_t vectors = (len + 31) / 32;
  uint8_t* padded = (uint8_t*)calloc(32 * vectors + 1, 1);
  uint8_t* lane_bytes = (uint8_t*)calloc(8 * vectors + 1, 1);
  size_t i;
  int j;
  if (len > 0) memcpy(padded, msg, len);
  for (j = 0; j < 4; ++j) {
    /* T2: lane j gets words j, j + 4, j + 8, ... of the padded message. */
    for (i = 0; i < vectors; ++i) memcpy(lane_bytes + 8 * i, padded + 8 * (4 * i + j), 8);
    lanes[j] = sipo_siphash(key[0], key[1], lane_bytes, 8 * vectors, c, d);
  }
  free(lane_bytes);
  free(padded);
}

uint64_t sipo_tree_hash(const uint64_t key[4], const uint8_t* msg, size_t len, int c, int d) {
  uint64_t lanes[4];
  uint8_t fold[40];
  int j;
  sipo_tree_lanes(key, msg, len, c, d, lanes);
  /* T3: hash the four lane results and the length. */
  for (j = 0; j < 4; ++j) store_le64(fold + 8 * j, lanes[j]);
  store_le64(fold + 32, (uint64_t)len);
  return sipo_siphash(key[0], key[1], fold, sizeof(fold), c, d);
}

int sipo_tree_batch(const uint64_t* keys, int per_message_keys, const uint8_t* bytes,
                    const int64_t* offsets, int64_t first, int64_t last, int c, int d,
                    uint64_t* out) {
  int64_t i;
  if (c < 1 || d < 1) return -1;
  for (i = first; i < last; ++i) {
    const uint64_t* key = per_message_keys ? keys + 4 * i : keys;
    if (offsets[i + 1] < offsets[i]) return -1;
    out[i - first] = sipo_tree_hash(key, bytes + offsets[i],
                                    (size_t)(offsets[i + 1] - offsets[i]), c, d);
  }
  return 0;
}

/*
 * hho.h -- scalar CPU oracle for HighwayHash as defined in
 * "Fast keyed hash/pseudo-random function using SIMD multiply and permute"
 * (Alakuijala, Cox, Wassenberg; arXiv:1612.06257), Section 4.
 *
 * TEST INFRASTRUCTURE ONLY.  This library exists to check the GPU path.
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * may load it.  It shares no code, header, table or constant with the CUDA
 * library under paper_1612_06257_gb300/csrc/, and it includes nothing from it.
 *
 * Every operation works on one 64-bit lane at a time, in the order the paper
 * states it.  All arithmetic is unsigned and wraps modulo 2^64.
 *
 * Pin status (what, other than this code, fixes each function):
 *   hho_constants      pinned: pi recomputed from Machin's formula, plus the
 *                      bit-coverage property of Section 4.4.
 *   hho_zipper_merge   pinned: the printed byte map of Section 4.1 and its
 *                      stated requirements 1-3.
 *   hho_permute        pinned: the printed 32-bit index map of Section 4.3
 *                      and its prose (swap 128-bit halves and 32-bit halves).
 *   hho_update         pinned: inverse-Update round trip (Update is a
 *                      permutation of the state, Section 6.4), written from
 *                      the Section 4.2 listing in the test suite.
 *   hho_remainder      partially pinned: trailing-zero and residue invariants
 *                      of Sections 4.5 and 6.3.  Three details of the encoding
 *                      are readings that no printed value fixes ("parity
 *                      unpinned" for them): the size is added to each 64-bit
 *                      lane of v0 as one 64-bit add of (r << 32) + r; each
 *                      32-bit half of v1 is rotated LEFT by r; the last r & 3
 *                      bytes go to packet bytes 28, 29, 30 in order.
 *   hho_finalize       pinned: avalanche statistics of Section 4.3 (strong
 *                      bias after 2 rounds, near zero after 4) and cross-pair
 *                      mixing.
 *   hho_hash*          pinned by the above plus a second, independent Python
 *                      transcription on every length 0..1024.
 * The paper prints no known-answer vectors, so agreement with any released
 * HighwayHash library is not claimed.
 */
#ifndef HHO_H
#define HHO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* The 1024-bit state of Section 4.2: four vectors of four 64-bit lanes. */
typedef struct hho_state {
  uint64_t v0[4];
  uint64_t v1[4];
  uint64_t mul0[4];
  uint64_t mul1[4];
} hho_state;

/* Section 4.4: the two 256-bit initialisation constants, lane 0 first. */
void hho_constants(uint64_t c0[4], uint64_t c1[4]);

/* Section 4.4: expand a 256-bit key (lane 0 first) into the state. */
void hho_init(hho_state* s, const uint64_t key[4]);

/* Section 4.1: ZipperMerge of a 4x64-bit vector (two independent lane pairs). */
void hho_zipper_merge(const uint64_t in[4], uint64_t out[4]);

/* Section 4.2: fold one 32-byte packet (four little-endian 64-bit words). */
void hho_update(hho_state* s, const uint64_t packet[4]);

/* Section 4.3: the 32-bit-part permutation of v0 used before each final Update. */
void hho_permute(const uint64_t v0[4], uint64_t out[4]);

/* Section 4.5: size injection and the padded Update of the last r = 1..31 bytes.
 * `tail` points at the r trailing bytes.  r == 0 does nothing. */
void hho_remainder(hho_state* s, const uint8_t* tail, size_t r);

/* Section 4.3: `rounds` times { Update(Permute(v0)) }.  The hash uses 4. */
void hho_finalize(hho_state* s, int rounds);

/* Section 4.3: h[i] = v0[i] + v1[i] + mul0[i] + mul1[i]. */
void hho_output(const hho_state* s, uint64_t h[4]);

/* Whole hash with a selectable number of finalisation rounds; writes
 * bits/64 words (bits = 64, 128 or 256) to out.  Returns 0, or -1 on bad bits. */
int hho_hash_rounds(const uint64_t key[4], const uint8_t* msg, size_t len,
                    int bits, int rounds, uint64_t* out);

void hho_hash64(const uint64_t key[4], const uint8_t* msg, size_t len, uint64_t* out);
void hho_hash128(const uint64_t key[4], const uint8_t* msg, size_t len, uint64_t* out);
void hho_hash256(const uint64_t key[4], const uint8_t* msg, size_t len, uint64_t* out);

/* Hash messages [first, last) of a batch laid out like the GPU library's:
 * message i is bytes[offsets[i] .. offsets[i+1]); keys holds one key (4 words)
 * when per_message_keys == 0, else keys[4*i .. 4*i+3] for message i.
 * out receives bits/64 words per message at out[(i - first) * bits/64].
 * Returns 0, or -1 on a bad argument (bits, or decreasing offsets). */
int hho_hash_batch(const uint64_t* keys, int per_message_keys, const uint8_t* bytes,
                   const int64_t* offsets, int64_t first, int64_t last, int bits,
                   uint64_t* out);

#ifdef __cplusplus
}
#endif

#endif /* HHO_H */

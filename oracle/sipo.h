/*
 * sipo.h -- scalar CPU oracle for SipTreeHash, the tree-hash extension of
 * SipHash in "Fast keyed hash/pseudo-random function using SIMD multiply and
 * permute" (Alakuijala, Cox, Wassenberg; arXiv:1612.06257), Section 3, with
 * its round-reduced variant SipTreeHash13 (Section 5, Table 1).
 *
 * TEST INFRASTRUCTURE ONLY.  This library exists to check the GPU path.
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * may load it.  It shares no code, header, table or constant with the CUDA
 * library under paper_1612_06257_gb300/csrc/, and it includes nothing from it.
 *
 * SipHash-c-d itself is not defined in the paper; it is the published
 * function of Aumasson and Bernstein ("SipHash: a fast short-input PRF",
 * INDOCRYPT 2012), which the paper cites and extends: c compression rounds
 * per 8-byte word, d finalisation rounds.  SipTreeHash uses c = 2, d = 4;
 * SipTreeHash13 uses c = 1, d = 3 (Section 5).
 *
 * Section 3 fixes the structure: the message is cut into 64-bit words that
 * are dealt to four interleaved lanes (word i to lane i mod 4), each lane is
 * an independent SipHash chain, and the four lane results are folded by
 * hashing them.  It leaves open the points below; these readings are this
 * oracle's (and the GPU library's) definition:
 *   T1 padding   the message is zero-padded to a whole number P of 32-byte
 *                vectors, P = ceil(len / 32) (Section 5: inputs are padded
 *                to entire vectors); P = 0 for the empty message.  Words are
 *                little-endian.
 *   T2 lanes     lane j is the standard SipHash-c-d of the 8P-byte string of
 *                its words (words j, j+4, j+8, ... of the padded message).
 *   T3 folding   the result is the standard SipHash-c-d of 40 bytes: the
 *                four lane results (little-endian, lane 0 first) followed by
 *                the message length in bytes as a little-endian 64-bit word.
 *                The length is needed because zero padding alone would give
 *                a message and the same message with trailing zero bytes the
 *                same lanes.
 *   T4 key       SipHash's 128-bit key (k0, k1) is the first two 64-bit words
 *                of the 4-word key the library's calls take; every lane and
 *                the fold use it.  Key words 2 and 3 are not used.
 *   T5 output    64 bits.
 *
 * Pin status (what, other than this code, fixes each function):
 *   sipo_siphash        pinned: the SipHash-2-4 test vector printed in
 *                       Aumasson and Bernstein's paper (Appendix A), and, for
 *                       SipHash-1-3 under the all-zero key, CPython's own
 *                       built-in bytes hash (siphash13) on many inputs.
 *   sipo_tree_lanes     pinned by composition: each lane equals sipo_siphash
 *                       of the words the test deals out itself, and the
 *                       64-byte example of Section 3 (lane i hashes A_i, B_i).
 *   sipo_tree_hash      pinned by composition (T3) and, for SipTreeHash13
 *                       under the all-zero key, end to end by CPython's hash;
 *                       invariants: permuted words and trailing zeros change
 *                       the result, key words 2 and 3 do not.
 *   Readings T1-T4 are choices no printed value can fix ("parity unpinned"
 *   for agreement with the released library, which is not claimed).
 */
#ifndef SIPO_H
#define SIPO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* SipHash-c-d of msg[0..len) under the 128-bit key (k0, k1). */
uint64_t sipo_siphash(uint64_t k0, uint64_t k1, const uint8_t* msg, size_t len, int c, int d);

/* The four lane results of SipTreeHash-c-d (readings T1, T2, T4). */
void sipo_tree_lanes(const uint64_t key[4], const uint8_t* msg, size_t len, int c, int d,
                     uint64_t lanes[4]);

/* SipTreeHash-c-d of msg[0..len) (readings T1-T5). */
uint64_t sipo_tree_hash(const uint64_t key[4], const uint8_t* msg, size_t len, int c, int d);

/* Messages [first, last) of a batch laid out like the GPU library's:
 * message i is bytes[offsets[i] .. offsets[i+1]), keys as in hho_hash_batch.
 * out[i - first] receives the 64-bit hash.  Returns 0, or -1 on decreasing
 * offsets or bad round counts. */
int sipo_tree_batch(const uint64_t* keys, int per_message_keys, const uint8_t* bytes,
                    const int64_t* offsets, int64_t first, int64_t last, int c, int d,
                    uint64_t* out);

#ifdef __cplusplus
}
#endif

#endif /* SIPO_H */

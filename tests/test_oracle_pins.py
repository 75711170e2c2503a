"""Pins of the CPU oracle to facts the paper and mathematics fix (no GPU).

Each test checks one oracle function against something other than itself: a
table printed in the paper, the paper's prose, a closed form, an inverse, or
an invariant the paper states.  A plausible slip anywhere in the oracle (a
dropped term, a wrong index or sign, a transposed operand) fails one of them.
"""
import random

import numpy as np

from tests.ref_py import hh_ref
from tests.ref_py.pi_hex import pi_fraction_words

M64 = (1 << 64) - 1
M32 = (1 << 32) - 1


def _rng(seed):
    return random.Random(seed)


def _rand_words(r, n=4):
    return [r.getrandbits(64) for _ in range(n)]


# ---------------------------------------------------------------- Section 4.4

def test_constants_from_pi(oracle):
    """C0/C1 start from pi's hex digits (Section 4.4); recompute pi exactly."""
    w = pi_fraction_words(8)
    assert w[0] == 0x243F6A8885A308D3  # 3.243F6A88... is pi in hexadecimal
    c0, c1 = oracle.constants()
    for c, words in ((c0, w[0:4]), (c1, w[4:8])):
        # Lanes 3..1 hold the first three words unchanged.
        assert c[3] == words[0] and c[2] == words[1] and c[1] == words[2]
        # Lane 0: the fourth word with every bit set that at most one of the
        # other lanes have (counted bit by bit, not via a majority formula).
        expect = words[3]
        for bit in range(64):
            ones = sum((x >> bit) & 1 for x in words[0:3])
            if ones <= 1:
                expect |= 1 << bit
        assert c[0] == expect
        # Stated purpose of the fix: every bit is set in at least one lane.
        assert (c[0] | c[1] | c[2] | c[3]) == M64
        # ... and the fix only ever sets bits of the fourth word.
        assert c[0] & words[3] == words[3]


def test_init_state(oracle):
    """v0 = key ^ C0, v1 = rot32(key) ^ C1, mul0 = C0, mul1 = C1."""
    r = _rng(1)
    c0, c1 = oracle.constants()
    for _ in range(20):
        key = _rand_words(r)
        v0, v1, m0, m1 = oracle.init_state(key).as_lists()
        assert m0 == c0 and m1 == c1
        for i in range(4):
            assert v0[i] ^ c0[i] == key[i]
            back = v1[i] ^ c1[i]
            assert ((back >> 32) | (back << 32)) & M64 == key[i]


# ---------------------------------------------------------------- Section 4.1

def _lane_bytes(base):
    """Lanes whose little-endian bytes are base, base+1, ..."""
    return int.from_bytes(bytes(range(base, base + 8)), "little")


def test_zipper_merge_matches_printed_map(oracle):
    """Feed byte j = j; result bytes read from 15 down to 0 must be the
    printed permutation, in both lane pairs."""
    v = [_lane_bytes(0), _lane_bytes(8), _lane_bytes(16), _lane_bytes(24)]
    out = oracle.zipper_merge(v)
    printed = [int(t, 16) for t in "7 8 6 9 D A 4 B 0 F 1 E 5 2 C 3".split()]
    for pair in (0, 1):
        res = out[2 * pair].to_bytes(8, "little") + out[2 * pair + 1].to_bytes(8, "little")
        listed = [b - 16 * pair for b in reversed(res)]
        assert listed == printed


def test_zipper_map_meets_stated_requirements():
    """Requirements 1-3 of Section 4.1, checked on the printed map."""
    P = hh_ref.zipper_offsets()          # P[i], i = 0..15
    assert sorted(P) == list(range(16))  # a permutation

    # Byte quality: summed distance of its bits from the lane ends.
    def quality(b):
        return sum(min(k, 63 - k) for k in range(8 * b, 8 * b + 8))
    q = [quality(b) for b in range(8)]
    # Stated ranking: bytes 3 and 4 best, then 2 and 5, then 1 and 6, and 0
    # and 7 worst.
    assert q[3] == q[4] > q[2] == q[5] > q[1] == q[6] > q[0] == q[7]

    # Requirement 1: the worst source bytes (0 and 7 of a lane) only land in
    # the upper 32 bits of a result lane.
    for i, src in enumerate(P):
        if src % 8 in (0, 7):
            assert i % 8 >= 4
    # Requirement 2: within each 32-bit group of the result, at most two
    # adjacent bytes come from one source lane (the paper states it for the
    # groups "5 2 C 3" and "D A 4 B"; across the group boundary at bytes
    # 11/12 the printed map does have a run of three).
    lanes = [src // 8 for src in P]
    for g in range(0, 16, 4):
        grp = lanes[g:g + 4]
        assert not any(grp[k] == grp[k + 1] == grp[k + 2] for k in range(2))
    # Upper halves alternate source lanes strictly.
    for half in (P[4:8], P[12:16]):
        assert [s // 8 for s in half] in ([1, 0, 1, 0], [0, 1, 0, 1])
    # Requirement 3: both lower 32-bit halves get equal total quality.
    assert sum(q[s % 8] for s in P[0:4]) == sum(q[s % 8] for s in P[8:12])


def test_zipper_merge_random_vs_byte_definition(oracle):
    r = _rng(2)
    P = hh_ref.zipper_offsets()
    for _ in range(200):
        v = _rand_words(r)
        out = oracle.zipper_merge(v)
        for pair in (0, 1):
            src = v[2 * pair].to_bytes(8, "little") + v[2 * pair + 1].to_bytes(8, "little")
            res = bytes(src[P[i]] for i in range(16))
            assert out[2 * pair] == int.from_bytes(res[:8], "little")
            assert out[2 * pair + 1] == int.from_bytes(res[8:], "little")


# ---------------------------------------------------------------- Section 4.3

def test_permute_matches_printed_indices(oracle):
    """32-bit part j = j in; result parts read from 7 down to 0 are 2 3 0 1 6 7 4 5."""
    v0 = [(2 * i + 1) << 32 | (2 * i) for i in range(4)]
    out = oracle.permute(v0)
    parts = []
    for lane in out:
        parts += [lane & M32, lane >> 32]
    assert list(reversed(parts)) == [2, 3, 0, 1, 6, 7, 4, 5]


def test_permute_matches_prose(oracle):
    """Swap the 128-bit halves and the 32-bit halves of each lane."""
    r = _rng(3)
    for _ in range(100):
        v0 = _rand_words(r)
        rot = [((x << 32) | (x >> 32)) & M64 for x in v0]
        assert oracle.permute(v0) == [rot[2], rot[3], rot[0], rot[1]]


# ---------------------------------------------------------------- Section 4.2

def _inverse_update(v0, v1, mul0, mul1, pkt):
    """Undo one Update (Section 4.2) step by step, last statement first.

    Update is a permutation of the state for a fixed packet (Section 6.4):
    each statement adds or xors a function of values it does not change.
    """
    zm = hh_ref.zipper_merge
    mul = hh_ref.mul_epu32
    v0, v1, mul0, mul1 = list(v0), list(v1), list(mul0), list(mul1)
    z = zm(v0)                                     # v1 += ZM(v0)
    v1 = [(v1[i] - z[i]) & M64 for i in range(4)]
    z = zm(v1)                                     # v0 += ZM(v1)
    v0 = [(v0[i] - z[i]) & M64 for i in range(4)]
    for i in range(4):
        mul1[i] ^= mul(v0[i], v1[i] >> 32)         # mul1 ^= mul(v0, v1 >> 32)
        v0[i] = (v0[i] - mul1[i]) & M64            # v0 += mul1
        mul0[i] ^= mul(v1[i], v0[i] >> 32)         # mul0 ^= mul(v1, v0 >> 32)
        v1[i] = (v1[i] - mul0[i]) & M64            # v1 += mul0
        v1[i] = (v1[i] - pkt[i]) & M64             # v1 += packet
    return v0, v1, mul0, mul1


def test_update_inverse_round_trip(oracle):
    r = _rng(4)
    for trial in range(300):
        before = [_rand_words(r) for _ in range(4)]
        if trial < 20:  # edge operands for the 32x32 multiply
            for lanes in before:
                for i in range(4):
                    lanes[i] = r.choice([0, M32, M64, 1 << 32, (M32 << 32)])
        pkt = _rand_words(r)
        s = oracle.State.from_lists(*before)
        oracle.update(s, pkt)
        after = s.as_lists()
        assert after != tuple(before)
        assert _inverse_update(*after, pkt) == tuple(before)


def test_update_multiply_is_32x32(oracle):
    """With v1 + packet + mul0 = x and v0 = y << 32, mul0 picks up lo(x) * y:
    the product of the low halves, a full 64-bit result (Section 4.2)."""
    r = _rng(5)
    cases = [(M32, M32), (M64, M64), (1 << 32, 5), (0xDEADBEEF12345678, 0xFFFFFFFF00000001)]
    cases += [(r.getrandbits(64), r.getrandbits(64)) for _ in range(20)]
    for a, b in cases:
        # state: v1 = 0, mul0 = 0, packet = a  =>  v1 after two adds = a
        v0 = [(b & M32) << 32] * 4
        s = oracle.State.from_lists(v0, [0] * 4, [0] * 4, [0] * 4)
        oracle.update(s, [a] * 4)
        mul0 = s.as_lists()[2]
        assert mul0[0] == (a & M32) * (b & M32)


# ---------------------------------------------------------------- Section 4.5

def test_multiple_of_32_needs_no_padding(oracle):
    """Whole packets only: hash = finalize(update(...update(init)))."""
    r = _rng(6)
    for packets in range(0, 5):
        key = _rand_words(r)
        msg = bytes(r.getrandbits(8) for _ in range(32 * packets))
        s = oracle.init_state(key)
        for k in range(packets):
            oracle.update(s, [int.from_bytes(msg[32 * k + 8 * i: 32 * k + 8 * i + 8], "little")
                              for i in range(4)])
        oracle.finalize(s, 4)
        assert oracle.output(s)[0] == oracle.hash64(key, msg)


def test_zero_messages_of_every_length_differ(oracle):
    """Zero-valued buffers of various sizes must hash differently (4.5, 6.3)."""
    key = [1, 2, 3, 4]
    seen = {}
    for n in range(0, 300):
        h = oracle.hash64(key, bytes(n))
        assert h not in seen, (n, seen.get(h))
        seen[h] = n


def test_trailing_zeros_change_the_hash(oracle):
    r = _rng(7)
    key = _rand_words(r)
    for base_len in (0, 1, 5, 31, 32, 33, 64, 100):
        msg = bytes(r.getrandbits(8) for _ in range(base_len))
        hs = {oracle.hash64(key, msg + bytes(k)) for k in range(0, 70)}
        assert len(hs) == 70


def test_remainder_uses_every_tail_byte(oracle):
    """Every byte of a 1..31-byte tail reaches the hash, for every residue."""
    r = _rng(8)
    key = _rand_words(r)
    for length in range(1, 96):
        msg = bytearray(r.getrandbits(8) for _ in range(length))
        h = oracle.hash64(key, bytes(msg))
        for pos in range(length):
            m2 = bytearray(msg)
            m2[pos] ^= 1 << r.randrange(8)
            assert oracle.hash64(key, bytes(m2)) != h


def test_remainder_structure_via_inverse(oracle):
    """Section 4.5 prose, checked by undoing the padded Update with the inverse:
    the size mod 32 is broadcast to the eight 32-bit parts and added to v0,
    v1's 32-bit parts are rotated by the size, and the padded packet keeps the
    4-byte groups in place with the last 0-3 bytes in its top four bytes."""
    r = _rng(13)
    for size in range(1, 32):
        before = [_rand_words(r) for _ in range(4)]
        tail = bytes(r.getrandbits(8) for _ in range(size))
        s = oracle.State.from_lists(*before)
        oracle.remainder(s, tail)
        q = size - size % 4
        top = tail[q:] + bytes(4 - size % 4)
        packet = tail[:q] + bytes(28 - q) + top
        pkt = [int.from_bytes(packet[8 * i:8 * i + 8], "little") for i in range(4)]
        v0, v1, m0, m1 = _inverse_update(*s.as_lists(), pkt)
        assert (m0, m1) == (before[2], before[3])
        broadcast = size * 0x0000000100000001
        assert v0 == [(x + broadcast) & M64 for x in before[0]]

        def rot(w):
            return ((w << size) | (w >> (32 - size))) & M32
        assert v1 == [(rot(x >> 32) << 32) | rot(x & M32) for x in before[1]]


# ------------------------------------------------------------- whole function

def test_output_widths_share_lanes(oracle):
    """64-bit = lane 0; 128-bit = lanes 0-1; 256-bit = lanes 0-3 (Section 4.3)."""
    r = _rng(9)
    for length in (0, 3, 32, 77, 1024):
        key = _rand_words(r)
        msg = bytes(r.getrandbits(8) for _ in range(length))
        h256 = oracle.hash256(key, msg)
        assert oracle.hash128(key, msg) == h256[:2]
        assert oracle.hash64(key, msg) == h256[0]
        s = oracle.init_state(key)
        full = length - length % 32
        for k in range(0, full, 32):
            oracle.update(s, [int.from_bytes(msg[k + 8 * i: k + 8 * i + 8], "little")
                              for i in range(4)])
        oracle.remainder(s, msg[full:])
        oracle.finalize(s, 4)
        v0, v1, m0, m1 = oracle.State.as_lists(s)
        assert h256 == [(v0[i] + v1[i] + m0[i] + m1[i]) & M64 for i in range(4)]


def test_determinism_and_key_sensitivity(oracle):
    r = _rng(10)
    msg = bytes(r.getrandbits(8) for _ in range(123))
    key = _rand_words(r)
    h = oracle.hash64(key, msg)
    assert oracle.hash64(list(key), bytes(msg)) == h
    flipped = set()
    for lane in range(4):
        for bit in range(64):
            k2 = list(key)
            k2[lane] ^= 1 << bit
            flipped.add(oracle.hash64(k2, msg))
    assert h not in flipped and len(flipped) == 256


def _avalanche_bias(oracle, rounds, samples, length, seed):
    """Mean |P(output bit flips | input bit flips) - 1/2| over all pairs."""
    r = _rng(seed)
    key = _rand_words(r)
    nbits = 8 * length
    diffs = np.zeros((samples, nbits), dtype=np.uint64)
    for s in range(samples):
        msg = bytearray(r.getrandbits(8) for _ in range(length))
        h = oracle.hash_rounds(key, bytes(msg), 64, rounds)[0]
        for b in range(nbits):
            m2 = bytearray(msg)
            m2[b // 8] ^= 1 << (b % 8)
            diffs[s, b] = h ^ oracle.hash_rounds(key, bytes(m2), 64, rounds)[0]
    shifts = np.arange(64, dtype=np.uint64)
    flips = ((diffs[:, :, None] >> shifts) & np.uint64(1)).sum(axis=0)  # [nbits, 64]
    bias = np.abs(flips / samples - 0.5)
    return float(bias.mean()), float(bias.max())


def test_finalization_rounds_bias(oracle):
    """Section 4.3: 3-byte inputs show strong output-bit bias after two
    finalisation rounds and essentially none after four.  With N samples the
    sampling noise alone gives a mean |bias| of about 0.4/sqrt(N)."""
    n = 1500
    noise = 0.4 / n ** 0.5
    mean4, max4 = _avalanche_bias(oracle, 4, n, 3, seed=11)
    mean2, max2 = _avalanche_bias(oracle, 2, n, 3, seed=11)
    assert mean4 < 1.3 * noise, mean4
    assert max4 < 6 * (0.25 / n) ** 0.5
    assert mean2 > 3 * noise, mean2


def test_bits_in_upper_lane_pair_reach_lane0(oracle):
    """Bytes 16..31 of a packet only reach lane 0 through Permute's half swap."""
    mean, mx = _avalanche_bias(oracle, 4, 300, 32, seed=12)
    assert mean < 1.3 * 0.4 / 300 ** 0.5
    assert mx < 0.2

"""Pins of the SipTreeHash oracle (oracle/sipo.c; paper Section 3), no GPU.

SipHash itself is pinned by values fixed outside this repository: the test
vector printed in the SipHash paper (tests/golden/), and CPython's built-in
bytes hash, which is SipHash-1-3 under the all-zero key when hash
randomisation is off (PYTHONHASHSEED=0).  The tree is pinned by composition
with that pinned SipHash (the words each lane must hash are dealt out here,
independently of the oracle), by the 64-byte example of Section 3, and by
invariants: the paper's reason for hashing the lane results (XOR would not see
permuted words), trailing-zero sensitivity, and the unused key words.
"""
from __future__ import annotations

import os
import struct
import subprocess
import sys

import numpy as np
import pytest

from oracle import siptree

HERE = os.path.dirname(os.path.abspath(__file__))
ROUNDS = [(2, 4), (1, 3)]


def _lanes_dealt_here(msg: bytes):
    """The four lane strings of readings T1-T2, built without the oracle."""
    vectors = (len(msg) + 31) // 32
    padded = msg + bytes(32 * vectors - len(msg))
    return [b"".join(padded[32 * i + 8 * j:32 * i + 8 * j + 8] for i in range(vectors))
            for j in range(4)]


def _cpython_hashes(messages):
    """CPython's hash() of each bytes object with randomisation off (its
    SipHash-1-3 under the zero key), as u64; None if this interpreter uses
    another algorithm."""
    code = ("import sys, pickle\n"
            "if sys.hash_info.algorithm != 'siphash13' or sys.hash_info.cutoff != 0:\n"
            "    print('none'); sys.exit(0)\n"
            "msgs = pickle.load(sys.stdin.buffer)\n"
            "print(' '.join(str(hash(m) % 2**64) for m in msgs))\n")
    import pickle
    res = subprocess.run([sys.executable, "-c", code], input=pickle.dumps(messages),
                         capture_output=True, env=dict(os.environ, PYTHONHASHSEED="0"), check=True)
    out = res.stdout.decode().strip()
    if out == "none":
        return None
    return [int(x) for x in out.split()]


def _random_messages(seed, lengths):
    rng = np.random.default_rng(seed)
    return [rng.integers(0, 256, n, dtype=np.uint8).tobytes() for n in lengths]


# ------------------------------------------------------------------ SipHash

def test_siphash24_matches_the_published_vector():
    rows = [l.split() for l in open(os.path.join(HERE, "golden", "siphash24_aumasson_bernstein.txt"))
            if l.strip() and not l.startswith("#")]
    assert rows
    for c, d, key_hex, msg_hex, h_hex in rows:
        key = bytes.fromhex(key_hex)
        k0, k1 = struct.unpack("<QQ", key)
        assert siptree.siphash(k0, k1, bytes.fromhex(msg_hex), int(c), int(d)) == int(h_hex, 16)


def test_siphash13_matches_cpython_bytes_hash():
    lengths = list(range(1, 130)) + [255, 256, 257, 1000, 4096]
    msgs = _random_messages(1, lengths) + [bytes(n) for n in range(1, 70)]
    ref = _cpython_hashes(msgs)
    if ref is None:
        pytest.skip("this interpreter's bytes hash is not SipHash-1-3")
    got = [siptree.siphash(0, 0, m, 1, 3) for m in msgs]
    assert got == ref


# ----------------------------------------------------------------- the tree

@pytest.mark.parametrize("c,d", ROUNDS)
def test_each_lane_is_siphash_of_its_dealt_words(c, d):
    rng = np.random.default_rng(2)
    for length in list(range(0, 200)) + [1023, 1024, 1025, 4099]:
        key = [int(x) for x in rng.integers(0, 2**63, 4)]
        msg = rng.integers(0, 256, length, dtype=np.uint8).tobytes()
        lanes = siptree.tree_lanes(key, msg, c, d)
        expect = [siptree.siphash(key[0], key[1], s, c, d) for s in _lanes_dealt_here(msg)]
        assert lanes == expect, length


@pytest.mark.parametrize("c,d", ROUNDS)
def test_section3_example_two_updates_per_lane(c, d):
    """A 64-byte input A0..A3 B0..B3: lane i hashes exactly A_i then B_i."""
    rng = np.random.default_rng(3)
    words = [int(x) for x in rng.integers(0, 2**63, 8)]
    msg = struct.pack("<8Q", *words)
    key = [5, 6, 7, 8]
    lanes = siptree.tree_lanes(key, msg, c, d)
    for i in range(4):
        assert lanes[i] == siptree.siphash(5, 6, struct.pack("<QQ", words[i], words[4 + i]), c, d)


@pytest.mark.parametrize("c,d", ROUNDS)
def test_result_hashes_the_lane_results_and_the_length(c, d):
    rng = np.random.default_rng(4)
    for length in (0, 1, 31, 32, 33, 64, 100, 1024):
        key = [int(x) for x in rng.integers(0, 2**63, 4)]
        msg = rng.integers(0, 256, length, dtype=np.uint8).tobytes()
        lanes = siptree.tree_lanes(key, msg, c, d)
        fold = struct.pack("<4QQ", *lanes, length)
        assert siptree.tree_hash(key, msg, c, d) == siptree.siphash(key[0], key[1], fold, c, d)


def test_siptree13_end_to_end_by_cpython():
    """Under the zero key the whole SipTreeHash13 is CPython's SipHash-1-3
    applied to the dealt lane strings and then to the fold."""
    lengths = list(range(1, 100)) + [255, 256, 1000]
    msgs = _random_messages(5, lengths)
    lane_strings = [s for m in msgs for s in _lanes_dealt_here(m)]
    lanes = _cpython_hashes(lane_strings)
    if lanes is None:
        pytest.skip("this interpreter's bytes hash is not SipHash-1-3")
    folds = [struct.pack("<4QQ", *lanes[4 * i:4 * i + 4], len(m)) for i, m in enumerate(msgs)]
    expect = _cpython_hashes(folds)
    got = [siptree.tree_hash([0, 0, 0, 0], m, 1, 3) for m in msgs]
    assert got == expect


@pytest.mark.parametrize("c,d", ROUNDS)
def test_permuted_words_change_the_hash_though_xor_of_lanes_would_not(c, d):
    """Section 3's reason for hashing the lane results: swapping two words
    swaps two lane results, which an XOR fold would not see."""
    rng = np.random.default_rng(6)
    key = [int(x) for x in rng.integers(0, 2**63, 4)]
    words = [int(x) for x in rng.integers(0, 2**63, 4)]
    a = struct.pack("<4Q", *words)
    b = struct.pack("<4Q", words[1], words[0], words[2], words[3])
    la, lb = siptree.tree_lanes(key, a, c, d), siptree.tree_lanes(key, b, c, d)
    assert la[0] ^ la[1] ^ la[2] ^ la[3] == lb[0] ^ lb[1] ^ lb[2] ^ lb[3]
    assert siptree.tree_hash(key, a, c, d) != siptree.tree_hash(key, b, c, d)


@pytest.mark.parametrize("c,d", ROUNDS)
def test_trailing_zeros_and_lengths_are_distinguished(c, d):
    key = [1, 2, 3, 4]
    zeros = {siptree.tree_hash(key, bytes(n), c, d) for n in range(0, 300)}
    assert len(zeros) == 300
    rng = np.random.default_rng(7)
    for length in range(0, 70):
        m = rng.integers(0, 256, length, dtype=np.uint8).tobytes()
        assert siptree.tree_hash(key, m, c, d) != siptree.tree_hash(key, m + b"\0", c, d)


@pytest.mark.parametrize("c,d", ROUNDS)
def test_only_the_first_two_key_words_are_used(c, d):
    msg = bytes(range(77))
    h = siptree.tree_hash([11, 22, 33, 44], msg, c, d)
    assert h == siptree.tree_hash([11, 22, 0, 0], msg, c, d)
    assert h != siptree.tree_hash([12, 22, 33, 44], msg, c, d)
    assert h != siptree.tree_hash([11, 23, 33, 44], msg, c, d)


def test_batch_matches_single_calls():
    rng = np.random.default_rng(8)
    lengths = rng.integers(0, 300, 200)
    offsets = np.zeros(201, dtype=np.int64)
    offsets[1:] = np.cumsum(lengths)
    data = rng.integers(0, 256, int(offsets[-1]), dtype=np.uint8)
    keys = rng.integers(0, 2**63, (200, 4), dtype=np.uint64)
    for c, d in ROUNDS:
        out = siptree.tree_batch(keys, True, data, offsets, c, d)
        for i in range(0, 200, 7):
            assert out[i] == siptree.tree_hash([int(x) for x in keys[i]],
                                               data[offsets[i]:offsets[i + 1]].tobytes(), c, d)

"""The C oracle against the independent Python transcription (no GPU).

Every length 0..1024 (so every residue mod 32 many times), several keys, and
all three output widths.
"""
import random

import numpy as np

from tests.ref_py import hh_ref


def test_constants_agree(oracle):
    c0, c1 = oracle.constants()
    r0, r1 = hh_ref.constants()
    assert c0 == r0 and c1 == r1


def test_every_length_0_to_1024(oracle):
    r = random.Random(20)
    data = bytes(r.getrandbits(8) for _ in range(1024))
    keys = [[r.getrandbits(64) for _ in range(4)] for _ in range(3)]
    keys.append([0, 0, 0, 0])
    for k, key in enumerate(keys):
        for length in range(0, 1025):
            msg = data[:length] if k % 2 == 0 else data[1024 - length:]
            expect = hh_ref.hash_words(key, msg, 4)
            assert oracle.hash256(key, msg) == expect, (k, length)


def test_batch_entry_matches_single(oracle):
    r = np.random.default_rng(21)
    n = 300
    lengths = r.integers(0, 200, size=n)
    offsets = np.zeros(n + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(lengths)
    data = r.integers(0, 256, size=int(offsets[-1]), dtype=np.uint8)
    keys = r.integers(0, 2**63, size=(n, 4), dtype=np.int64).astype(np.uint64)
    out = oracle.hash_batch(keys, True, data, offsets, bits=128)
    for i in range(0, n, 7):
        msg = data[offsets[i]:offsets[i + 1]].tobytes()
        assert list(out[i]) == hh_ref.hash_words([int(x) for x in keys[i]], msg, 2)
    shared = oracle.hash_batch(keys[0], False, data, offsets, bits=64)
    for i in range(0, n, 11):
        msg = data[offsets[i]:offsets[i + 1]].tobytes()
        assert int(shared[i, 0]) == hh_ref.hash64([int(x) for x in keys[0]], msg)

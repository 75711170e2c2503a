"""GPU tests of counter-mode output and the statistical-study kernels.

Every kernel output is compared, bit for bit, with the CPU oracle (hashes)
or with numpy on the same inputs (counts).  The avalanche inputs come from
splitmix64, re-implemented here from Vigna's published definition.
"""
import numpy as np
import pytest
import torch

from paper_1612_06257_gb300 import hh, stats

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
M64 = (1 << 64) - 1
KEY = [0x0123456789ABCDEF, 0xFEDCBA9876543210, 0x0F1E2D3C4B5A6978, 0x8796A5B4C3D2E1F0]


@pytest.fixture(scope="module")
def ctx():
    from paper_1612_06257_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    c = hh.hh_init(0)
    yield c
    hh.hh_destroy(c)


def splitmix64(seed, counter):
    z = (seed + (counter + 1) * 0x9E3779B97F4A7C15) & M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def _u64(t):
    return t.cpu().numpy().view(np.uint64)


@pytest.mark.parametrize("bits", [64, 128, 256])
def test_prng_fill_matches_oracle(ctx, oracle, bits):
    key = torch.tensor(np.array(KEY, dtype=np.uint64).view(np.int64), device=DEV)
    counter0 = M64 - 100  # the counter wraps past 2^64
    n = 5000
    got = _u64(hh.hh_prng_fill(ctx, bits, key, counter0, n)).reshape(n, bits // 64)
    data = np.array([(counter0 + i) & M64 for i in range(n)], dtype=np.uint64).view(np.uint8)
    offsets = np.arange(n + 1, dtype=np.int64) * 8
    expect = np.zeros((n, bits // 64), dtype=np.uint64)
    oracle.hash_batch(np.array(KEY, dtype=np.uint64), False, data, offsets, bits, 0, n, expect)
    assert np.array_equal(got, expect)


@pytest.mark.parametrize("rounds", [0, 2, 3, 4])
def test_round_table_two_bytes_matches_oracle(ctx, oracle, rounds):
    table = _u64(hh.hh_stats_round_table(ctx, KEY, 2, rounds))
    lib = oracle.lib()
    for x in range(0, 1 << 16, 1 if rounds == 4 else 7):
        msg = bytes([x & 255, x >> 8])
        assert int(table[x]) == lib.hash_rounds(KEY, msg, 64, rounds)[0], (rounds, x)


def test_round_table_three_bytes_sample(ctx, oracle):
    table = _u64(hh.hh_stats_round_table(ctx, KEY, 3, 3))
    lib = oracle.lib()
    rng = np.random.default_rng(1)
    for x in list(rng.integers(0, 1 << 24, 2000)) + [0, (1 << 24) - 1]:
        x = int(x)
        msg = bytes([x & 255, (x >> 8) & 255, x >> 16])
        assert int(table[x]) == lib.hash_rounds(KEY, msg, 64, 3)[0], x


def test_toggle_counts_match_numpy(ctx):
    m = 16
    table_t = hh.hh_stats_round_table(ctx, KEY, 2, 2)
    counts = hh.hh_stats_toggle_counts(ctx, table_t, m).cpu().numpy().reshape(m, 64)
    table = _u64(table_t)
    x = np.arange(1 << m)
    for j in range(m):
        d = table ^ table[x ^ (1 << j)]
        bits = (d[:, None] >> np.arange(64, dtype=np.uint64)) & np.uint64(1)
        assert np.array_equal(counts[j], bits.sum(axis=0).astype(np.int64)), j


@pytest.mark.parametrize("size", [1, 4, 13, 31, 32])
def test_avalanche_counts_match_cpu(ctx, oracle, size):
    seed, iters = 0xC0FFEE + size, 96
    counts = hh.hh_stats_avalanche(ctx, size, seed, iters).cpu().numpy().reshape(8 * size, 64)
    lib = oracle.lib()
    key = [splitmix64(seed, i) for i in range(4)]
    expect = np.zeros((8 * size, 64), dtype=np.int64)
    for t in range(iters):
        words = [splitmix64(seed, 4 + 4 * t + w) for w in range(4)]
        msg = b"".join(v.to_bytes(8, "little") for v in words)[:size]
        h0 = lib.hash_rounds(key, msg, 64, 4)[0]
        for b in range(8 * size):
            flipped = bytearray(msg)
            flipped[b >> 3] ^= 1 << (b & 7)
            d = h0 ^ lib.hash_rounds(key, bytes(flipped), 64, 4)[0]
            expect[b] += [(d >> k) & 1 for k in range(64)]
    assert np.array_equal(counts, expect)


def test_round_study_shape(ctx):
    """Section 4.3's observation on all 2^24 three-byte inputs: strong bias
    after two rounds, a far smaller one after three, and none measurable
    after four.  Each (input bit, output bit) pair has 2^23 independent
    input pairs, so sampling alone gives a mean |p - 1/2| of about
    0.8 * 0.5 / sqrt(2^23) = 1.4e-4 and a largest one of a few times that."""
    two, three, four = (stats.round_bias(ctx, r) for r in (2, 3, 4))
    assert two["mean_bias"] > 30 * three["mean_bias"]
    assert four["mean_bias"] < 2e-4 and four["max_bias"] < 1e-3
    assert three["mean_bias"] > four["mean_bias"]


def test_avalanche_small_study_passes(ctx):
    res = stats.avalanche_study(ctx, sizes=[4, 17, 32], samples=5, iterations=200_000)
    assert res["pass"], res

"""The seeded synthetic batches follow the recipes that the benchmarks state.

CPU only: the generators take a device, and "cpu" gives the same recipe
(the draws differ from the GPU's, which is fine: only the shape is pinned).
"""
import torch

from paper_1612_06257_gb300 import workloads


def _lengths(w):
    return (w.offsets[1:] - w.offsets[:-1]).to(torch.int64)


def test_fixed_batch_shape():
    w = workloads.fixed(100, 1024, seed=1, device="cpu")
    assert w.total_bytes == 100 * 1024 and w.fixed_len == 1024 and w.offsets is None
    assert w.keys.shape == (4,) and w.key_mode == 0
    assert torch.equal(w.offsets_or_stride(), torch.arange(101, dtype=torch.int64) * 1024)
    pm = workloads.fixed(8, 64, seed=1, device="cpu", per_message_keys=True)
    assert pm.keys.shape == (8, 4) and pm.key_mode == 1


def test_ragged_recipe_is_log_uniform_with_every_residue():
    n = 4096
    w = workloads.ragged(n, seed=2, device="cpu")
    lengths = _lengths(w)
    assert int(w.offsets[0]) == 0 and int(w.offsets[-1]) == w.total_bytes
    assert int(lengths.min()) >= 0 and int(lengths.max()) <= 65536
    # Message i has length i mod 32 modulo 32, except where the clamp to
    # 65536 cuts it, so every residue occurs.
    idx = torch.arange(n)
    unclamped = lengths < 65536
    assert torch.equal(lengths[unclamped] % 32, idx[unclamped] % 32)
    assert set((lengths % 32).tolist()) == set(range(32))
    # Log-uniform on [0, 65536]: the median is near sqrt(65537) = 256.
    median = float(lengths.to(torch.float64).median())
    assert 128 < median < 512
    assert w.keys.shape == (n, 4) and w.per_message_keys


def test_short_recipe_lengths_and_zero_messages():
    n = 20000
    w = workloads.short(n, seed=3, device="cpu")
    lengths = _lengths(w)
    assert int(lengths.min()) == 0 and int(lengths.max()) == 64
    assert abs(float(lengths.to(torch.float64).mean()) - 32.0) < 1.0
    assert w.keys.shape == (4,) and not w.per_message_keys
    # About one message in ten has all-zero bytes (length-0 messages aside;
    # a random short message is all zero by chance only rarely).
    zero = 0
    nonempty = 0
    for i in range(n):
        a, b = int(w.offsets[i]), int(w.offsets[i + 1])
        if b > a:
            nonempty += 1
            zero += int(not bool(w.data[a:b].any()))
    assert 0.08 < zero / nonempty < 0.12


def test_from_lengths_and_seeds():
    lengths = [0, 1, 31, 32, 33, 1000]
    w = workloads.from_lengths(lengths, seed=4, device="cpu")
    assert _lengths(w).tolist() == lengths and w.keys.shape == (6, 4)
    again = workloads.ragged(256, seed=5, device="cpu")
    same = workloads.ragged(256, seed=5, device="cpu")
    other = workloads.ragged(256, seed=6, device="cpu")
    assert torch.equal(again.data, same.data) and torch.equal(again.offsets, same.offsets)
    assert not torch.equal(again.offsets, other.offsets)

"""GPU tests of the call contract of the device hash calls and the host path.

- The device hash calls allocate nothing: a batch beyond the sort scratch
  that hh_init / hh_reserve sized returns HH_ERR_TOO_LARGE, enqueues no
  kernel and leaves `out` untouched; after hh_reserve the same call hashes
  the batch, and the hashes equal the oracle's word for word.
- hh_hash_host checks each chunk's offsets on the host before staging it: a
  decreasing pair anywhere returns HH_ERR_BAD_OFFSETS without reading past the
  staged bytes, and the chunks before it are hashed.
"""
import numpy as np
import pytest
import torch

from paper_1612_06257_gb300 import hh, workloads
from tests.helpers import as_u64, oracle_hashes

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
DEFAULT_CAP = 1 << 22  # HH_DEFAULT_MAX_MESSAGES
SENTINEL = -0x3C3C3C3C3C3C3C3D


@pytest.fixture()
def fresh_ctx():
    from paper_1612_06257_gb300 import build
    build.build()
    c = hh.hh_init(0)
    yield c
    hh.hh_destroy(c)


def test_batch_beyond_reserved_scratch_is_refused_then_hashed(fresh_ctx):
    ctx = fresh_ctx
    L = hh.load_library()
    lengths = torch.randint(0, 9, (DEFAULT_CAP + 1,), generator=torch.Generator().manual_seed(5))
    w = workloads.from_lengths(lengths, seed=5, device=DEV)
    out = torch.full((w.n,), SENTINEL, dtype=torch.int64, device=DEV)
    stream = torch.cuda.current_stream().cuda_stream
    torch.cuda.synchronize()
    st = L.hh_hash64_batch(ctx.ptr, w.keys.data_ptr(), w.key_mode, w.data.data_ptr(),
                           w.offsets.data_ptr(), w.n, out.data_ptr(), stream)
    assert st == hh.HH_ERR_TOO_LARGE
    assert hh.hh_last_launch_count(ctx) == 0
    # The segments form and the stream calls share the limit.
    starts = w.offsets[:-1].contiguous()
    lens = (w.offsets[1:] - w.offsets[:-1]).contiguous()
    st = L.hh_hash_segments(ctx.ptr, 64, w.keys.data_ptr(), 1, None, w.data.data_ptr(),
                            w.data.numel(), starts.data_ptr(), lens.data_ptr(), w.n, None,
                            out.data_ptr(), stream)
    assert st == hh.HH_ERR_TOO_LARGE
    assert hh.hh_get_device_error(ctx) == hh.HH_OK
    assert torch.all(out == SENTINEL)
    # Reserved: the same call runs and matches the oracle.
    hh.hh_reserve(ctx, w.n)
    got = as_u64(hh.hh_hash64_batch(ctx, w.keys, w.key_mode, w.data, w.offsets), 1)
    assert hh.hh_get_device_error(ctx) == hh.HH_OK
    rng = np.random.default_rng(5)
    idx = np.unique(np.concatenate([rng.choice(w.n, 4000, replace=False), [0, w.n - 1]]))
    assert np.array_equal(got[idx], oracle_hashes(w, 64, indices=idx))


def test_reserve_rejects_bad_sizes(fresh_ctx):
    L = hh.load_library()
    assert L.hh_reserve(fresh_ctx.ptr, -1) == hh.HH_ERR_INVALID_ARG
    assert L.hh_reserve(fresh_ctx.ptr, 1 << 31) == hh.HH_ERR_TOO_LARGE
    assert L.hh_reserve(fresh_ctx.ptr, 10) == hh.HH_OK  # below the default: nothing to do


def test_host_path_rejects_decreasing_offsets_without_reading_past_the_chunk(fresh_ctx):
    ctx = fresh_ctx
    keys = np.arange(4, dtype=np.uint64)
    data = np.arange(64, dtype=np.uint8)
    # offsets[1] lies far beyond the 64 bytes while offsets[0] and offsets[n]
    # frame a valid range: only a check of every offset catches it.
    offsets = np.array([0, 10**9, 10, 64], dtype=np.int64)
    with pytest.raises(hh.HHError) as exc:
        hh.hh_hash_host(ctx, 64, keys, 0, data, offsets)
    assert exc.value.status == hh.HH_ERR_BAD_OFFSETS
    # The context stays usable.
    ok = np.array([0, 10, 64], dtype=np.int64)
    got = hh.hh_hash_host(ctx, 64, keys, 0, data, ok)
    import oracle
    expect = oracle.hash_batch(keys, False, data, ok, bits=64)[:, 0]
    assert np.array_equal(got, expect)


def test_host_path_hashes_chunks_before_a_bad_one(fresh_ctx):
    """Chunks hold at most 2^20 messages: a decreasing pair in the second
    chunk is refused, and the first chunk's hashes are written."""
    ctx = fresh_ctx
    n = (1 << 20) + 100
    rng = np.random.default_rng(6)
    lengths = rng.integers(0, 17, n)
    offsets = np.zeros(n + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(lengths)
    data = rng.integers(0, 256, int(offsets[-1]), dtype=np.uint8)
    keys = rng.integers(0, 2**63, 4, dtype=np.uint64)
    bad = offsets.copy()
    bad[(1 << 20) + 50] = bad[(1 << 20) + 49] - 1
    out = np.zeros(n, dtype=np.uint64)
    with pytest.raises(hh.HHError) as exc:
        hh.hh_hash_host(ctx, 64, keys, 0, data, bad, out=out)
    assert exc.value.status == hh.HH_ERR_BAD_OFFSETS
    import oracle
    first = 1 << 20
    sample = np.unique(np.concatenate([rng.choice(first, 3000, replace=False), [0, first - 1]]))
    expect = np.zeros((first, 1), dtype=np.uint64)
    oracle.hash_batch(keys, False, data, offsets, 64, 0, first, expect)
    assert np.array_equal(out[sample], expect[sample, 0])
    assert not out[first:].any()


def test_host_path_over_several_chunks(fresh_ctx):
    """About 300 MiB in 1 KiB..8 KiB messages: three payload chunks, each
    staged, hashed and copied back while the next one copies in."""
    ctx = fresh_ctx
    rng = np.random.default_rng(7)
    lengths = rng.integers(1024, 8193, 64000)
    offsets = np.zeros(lengths.size + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(lengths)
    assert offsets[-1] > 2 * (128 << 20)
    data = torch.randint(0, 256, (int(offsets[-1]),), dtype=torch.uint8,
                         generator=torch.Generator().manual_seed(7)).pin_memory().numpy()
    keys = rng.integers(0, 2**63, (lengths.size, 4), dtype=np.uint64).reshape(-1)
    got = hh.hh_hash_host(ctx, 256, keys, 1, data, offsets).reshape(-1, 4)
    import oracle
    sample = np.unique(np.concatenate([rng.choice(lengths.size, 400, replace=False),
                                       [0, lengths.size - 1]]))
    for i in sample:
        o = np.array([0, lengths[i]], dtype=np.int64)
        e = oracle.hash_batch(keys[4 * i:4 * i + 4].copy(), False,
                              data[offsets[i]:offsets[i + 1]].copy(), o, bits=256)
        assert np.array_equal(got[i], e[0]), i

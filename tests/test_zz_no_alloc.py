"""GPU test of hh_hash_batch_noalloc, the hash call that allocates nothing.

It is for callers that cannot allocate device memory for this library (their
memory belongs to another allocator or a fixed budget, or they cannot afford
cudaMalloc's implicit synchronisation).  The test calls it through the C ABI
twice in a row, on two different batches, and requires each result to equal
hh_hash_batch's for the same batch and the CPU oracle's, word for word (the
tolerance of every hash test: zero).  Further cases reach the messages of
128 KiB and more (one warp or two threads per message) with 128-bit output,
and a batch of exactly the limit's 2^20 messages, checked on a sample
against the oracle.  It also checks the size limit.  This file is collected
last.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1612_06257_gb300 import hh, workloads
from tests.helpers import as_u64, oracle_hashes

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
FN = {64: hh.hh_hash64_batch, 128: hh.hh_hash128_batch, 256: hh.hh_hash256_batch}


def _noalloc(lib, bits, w, out, err):
    stream = torch.cuda.current_stream().cuda_stream
    return lib.hh_hash_batch_noalloc(bits, w.keys.data_ptr(), w.key_mode, w.data.data_ptr(),
                                     w.offsets.data_ptr(), w.n, out.data_ptr(), err.data_ptr(),
                                     stream)


def test_noalloc_matches_batch_entry_point_twice():
    from paper_1612_06257_gb300 import build
    build.build()
    lib = hh.load_library()
    torch.cuda.set_device(0)
    ctx = hh.hh_init(0)
    try:
        g = torch.Generator().manual_seed(77)
        batches = [
            # mixed lengths (the length sort orders them), per-message keys, 256-bit
            (256, workloads.from_lengths(
                torch.cat([torch.randint(0, 65, (3000,), generator=g),
                           torch.randint(65, 20000, (1200,), generator=g)]),
                seed=77, device=DEV, per_message_keys=True)),
            # short messages only (index order), one key, 64-bit
            (64, workloads.short(50000, seed=78, device=DEV)),
        ]
        for bits, w in batches:
            words = bits // 64
            expect = FN[bits](ctx, w.keys, w.key_mode, w.data, w.offsets)
            assert hh.hh_get_device_error(ctx) == hh.HH_OK
            out = torch.full((w.n * words,), -1, dtype=torch.int64, device=DEV)
            err = torch.zeros(1, dtype=torch.int32, device=DEV)
            assert _noalloc(lib, bits, w, out, err) == hh.HH_OK
            torch.cuda.synchronize()
            assert int(err.item()) == hh.HH_OK
            assert np.array_equal(out.cpu().numpy(), expect.cpu().numpy())
            assert np.array_equal(as_u64(out, words), oracle_hashes(w, bits))
    finally:
        hh.hh_destroy(ctx)


def test_noalloc_long_messages_128_bit():
    """Messages of 128 KiB and more come first in the length order and run
    one per warp or two threads each; 128-bit output."""
    lib = hh.load_library()
    ctx = hh.hh_init(0)
    try:
        g = torch.Generator().manual_seed(79)
        lengths = torch.cat([torch.randint(0, 3000, (2000,), generator=g),
                             torch.tensor([(1 << 17), (1 << 17) + 5, 300001, (1 << 20) + 31]),
                             torch.randint(1 << 17, 1 << 19, (40,), generator=g)])
        lengths = lengths[torch.randperm(lengths.numel(), generator=g)]
        w = workloads.from_lengths(lengths, seed=79, device=DEV, per_message_keys=True)
        expect = hh.hh_hash128_batch(ctx, w.keys, w.key_mode, w.data, w.offsets)
        assert hh.hh_get_device_error(ctx) == hh.HH_OK
        out = torch.full((w.n * 2,), -1, dtype=torch.int64, device=DEV)
        err = torch.zeros(1, dtype=torch.int32, device=DEV)
        assert _noalloc(lib, 128, w, out, err) == hh.HH_OK
        torch.cuda.synchronize()
        assert int(err.item()) == hh.HH_OK
        assert np.array_equal(out.cpu().numpy(), expect.cpu().numpy())
        assert np.array_equal(as_u64(out, 2), oracle_hashes(w, 128))
    finally:
        hh.hh_destroy(ctx)


def test_noalloc_at_its_message_limit():
    """Exactly 2^20 ragged messages (the sort's multi-block path over the
    whole static array), sampled against the oracle, both ends included."""
    lib = hh.load_library()
    w = workloads.ragged(1 << 20, seed=80, device=DEV, max_len=4096)
    out = torch.full((w.n,), -1, dtype=torch.int64, device=DEV)
    err = torch.zeros(1, dtype=torch.int32, device=DEV)
    assert _noalloc(lib, 64, w, out, err) == hh.HH_OK
    torch.cuda.synchronize()
    assert int(err.item()) == hh.HH_OK
    rng = np.random.default_rng(80)
    idx = np.unique(np.concatenate([rng.choice(w.n, 3000, replace=False), [0, 1, w.n - 2, w.n - 1]]))
    got = as_u64(out, 1)
    assert np.array_equal(got[idx], oracle_hashes(w, 64, indices=idx))


def test_noalloc_rejects_batches_beyond_its_limit():
    lib = hh.load_library()
    limit = 1 << 20
    dummy = torch.zeros(8, dtype=torch.int64, device=DEV)
    st = lib.hh_hash_batch_noalloc(64, dummy.data_ptr(), 0, dummy.data_ptr(), dummy.data_ptr(),
                                   limit + 1, dummy.data_ptr(), None, None)
    assert st == hh.HH_ERR_TOO_LARGE
    assert lib.hh_hash_batch_noalloc(96, None, 0, None, None, 1, None, None, None) == \
        hh.HH_ERR_INVALID_ARG

"""GPU parity of SipTreeHash (paper Section 3) against its CPU oracle.

hh_siptree_batch through the C ABI against oracle/sipo.c, word for word
(tolerance zero: the hash is exact integer arithmetic), for SipTreeHash
(SipHash-2-4 lanes) and SipTreeHash13 (SipHash-1-3): every length 0..1024,
log-uniform ragged batches (the staged warp-tile path, unaligned starts),
all-short batches (read straight from global memory), the 2^20 x 1 KiB batch
the benchmark times (sampled), and the edge cases.
"""
import concurrent.futures
import os

import numpy as np
import pytest
import torch

from oracle import siptree
from paper_1612_06257_gb300 import hh, workloads
from tests.helpers import host_inputs

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
VARIANTS = {"siptree": hh.HH_SIPTREE, "siptree13": hh.HH_SIPTREE13}


@pytest.fixture(scope="module")
def ctx():
    from paper_1612_06257_gb300 import build
    build.build()
    c = hh.hh_init(0)
    yield c
    hh.hh_destroy(c)


def oracle_tree(w, name, indices=None):
    keys, per_msg, data, offsets = host_inputs(w, indices)
    c, d = siptree.ROUNDS[name]
    n = offsets.shape[0] - 1
    out = np.zeros(n, dtype=np.uint64)
    threads = min(16, os.cpu_count() or 1)
    step = max(1, (n + threads - 1) // threads)

    def run(first):
        last = min(n, first + step)
        siptree.tree_batch(keys, per_msg, data, offsets, c, d, first, last, out[first:last])

    with concurrent.futures.ThreadPoolExecutor(max_workers=threads) as ex:
        list(ex.map(run, range(0, n, step)))
    return out


def gpu_tree(ctx, w, name):
    out = hh.hh_siptree_batch(ctx, VARIANTS[name], w.keys, w.key_mode, w.data,
                              w.offsets_or_stride())
    assert hh.hh_get_device_error(ctx) == hh.HH_OK
    return out.cpu().numpy().view(np.uint64)


@pytest.mark.parametrize("name", sorted(VARIANTS))
def test_every_length_0_to_1024(ctx, name):
    g = torch.Generator().manual_seed(41)
    lengths = torch.cat([torch.arange(1025), torch.arange(1025)])
    lengths = lengths[torch.randperm(lengths.numel(), generator=g)]
    w = workloads.from_lengths(lengths, seed=41, device=DEV, per_message_keys=True)
    assert np.array_equal(gpu_tree(ctx, w, name), oracle_tree(w, name))


@pytest.mark.parametrize("name", sorted(VARIANTS))
@pytest.mark.parametrize("per_message_keys", [False, True])
def test_loguniform_ragged(ctx, name, per_message_keys):
    w = workloads.ragged(16384, seed=42, device=DEV, max_len=65536,
                         per_message_keys=per_message_keys)
    assert np.array_equal(gpu_tree(ctx, w, name), oracle_tree(w, name))


@pytest.mark.parametrize("name", sorted(VARIANTS))
def test_short_messages_and_unaligned_batch_ends(ctx, name):
    w = workloads.short(20000, seed=43, device=DEV)
    # Drop the first and last 3 bytes of the buffer: the batch starts and
    # ends mid-word.
    offsets = w.offsets.clone()
    offsets[0] = 3
    offsets[-1] = offsets[-1] - 3
    offsets = torch.maximum(offsets, offsets[0]).contiguous()
    offsets = torch.minimum(offsets, offsets[-1]).contiguous()
    w2 = workloads.Workload("ragged", w.data, offsets, None, w.keys, False, w.n)
    assert np.array_equal(gpu_tree(ctx, w2, name), oracle_tree(w2, name))


@pytest.mark.parametrize("name", sorted(VARIANTS))
def test_full_size_1gib_fixed_1k_sampled(ctx, name):
    """2^20 messages of 1024 bytes (1 GiB), one key: the benchmark's batch."""
    w = workloads.fixed(1 << 20, 1024, seed=44, device=DEV)
    got = gpu_tree(ctx, w, name)
    rng = np.random.default_rng(44)
    idx = np.sort(np.concatenate([rng.choice(w.n, 3000, replace=False), [0, w.n - 1]]))
    assert np.array_equal(got[idx], oracle_tree(w, name, indices=idx))
    assert np.unique(got).size == w.n


def test_edge_cases(ctx):
    L = hh.load_library()
    keys = torch.zeros(4, dtype=torch.int64, device=DEV)
    data = torch.zeros(64, dtype=torch.uint8, device=DEV)
    offsets = torch.tensor([0, 64], dtype=torch.int64, device=DEV)
    out = torch.full((2,), 7, dtype=torch.int64, device=DEV)
    stream = torch.cuda.current_stream().cuda_stream
    assert L.hh_siptree_batch(ctx.ptr, 99, keys.data_ptr(), 0, data.data_ptr(),
                              offsets.data_ptr(), 1, out.data_ptr(), stream) == \
        hh.HH_ERR_INVALID_ARG
    assert L.hh_siptree_batch(ctx.ptr, hh.HH_SIPTREE, keys.data_ptr(), 0, data.data_ptr(),
                              offsets.data_ptr(), 0, out.data_ptr(), stream) == hh.HH_OK
    torch.cuda.synchronize()
    assert int(out[0].item()) == 7  # n = 0 writes nothing
    # A decreasing pair: device error, that message's hash is 0, the rest exact.
    w = workloads.from_lengths([10, 20, 30, 40], seed=45, device=DEV)
    bad = w.offsets.clone()
    bad[2] = bad[1] - 5
    got = hh.hh_siptree_batch(ctx, hh.HH_SIPTREE, w.keys, 1, w.data, bad)
    assert hh.hh_get_device_error(ctx) == hh.HH_ERR_BAD_OFFSETS
    got = got.cpu().numpy().view(np.uint64)
    assert got[1] == 0
    expect = oracle_tree(w, "siptree")
    assert got[0] == expect[0] and got[3] == expect[3]


@pytest.mark.parametrize("name", sorted(VARIANTS))
def test_long_messages_beside_short_ones(ctx, name):
    """Messages of 128 KiB to 1 MiB + 13 B (thousands of staged windows each)
    among short and medium ones, per-message keys, unaligned starts."""
    g = torch.Generator().manual_seed(46)
    lengths = torch.cat([torch.randint(0, 4000, (600,), generator=g),
                         torch.tensor([1 << 17, (1 << 17) + 1, 300001, (1 << 20) + 13])])
    lengths = lengths[torch.randperm(lengths.numel(), generator=g)]
    w = workloads.from_lengths(lengths, seed=46, device=DEV, per_message_keys=True)
    assert np.array_equal(gpu_tree(ctx, w, name), oracle_tree(w, name))

"""GPU tests of the streaming calls: a message hashed in pieces equals the
message hashed whole (the design of Section 4.5 makes that possible), on
every kernel path that streams take, bit for bit."""
import numpy as np
import pytest
import torch

from paper_1612_06257_gb300 import hh, workloads
from tests.helpers import oracle_hashes

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
WHOLE = {64: hh.hh_hash64_batch, 128: hh.hh_hash128_batch, 256: hh.hh_hash256_batch}


@pytest.fixture(scope="module")
def ctx():
    from paper_1612_06257_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    c = hh.hh_init(0)
    yield c
    hh.hh_destroy(c)


def _split(lengths, rounds, rng):
    """Per stream: `rounds` update pieces (multiples of 32 bytes) and a last
    piece, summing to its length."""
    pieces = np.zeros((len(lengths), rounds + 1), dtype=np.int64)
    for m, total in enumerate(lengths):
        left = int(total)
        for u in range(rounds):
            take = 32 * int(rng.integers(0, left // 32 + 1)) if left >= 32 else 0
            pieces[m, u] = take
            left -= take
        pieces[m, rounds] = left
    return pieces


def _round_buffers(w, pieces, u):
    """bytes and offsets of round u: piece u of every stream, in order."""
    starts = w.offsets[:-1].cpu().numpy() + pieces[:, :u].sum(axis=1)
    lens = pieces[:, u]
    offs = np.concatenate([[0], np.cumsum(lens)])
    data = torch.empty(int(offs[-1]), dtype=torch.uint8, device=DEV)
    if offs[-1]:
        idx = np.concatenate([np.arange(s, s + l) for s, l in zip(starts, lens) if l])
        data[:] = w.data[torch.from_numpy(idx).to(DEV)]
    return data, torch.from_numpy(offs).to(DEV)


def _run_streams(ctx, w, pieces, bits, key_mode):
    rounds = pieces.shape[1] - 1
    states = hh.hh_stream_init(ctx, w.keys, key_mode, w.n)
    for u in range(rounds):
        data, offs = _round_buffers(w, pieces, u)
        hh.hh_stream_update(ctx, states, data, offs)
    data, offs = _round_buffers(w, pieces, rounds)
    out = hh.hh_stream_finish(ctx, bits, states, data, offs)
    assert hh.hh_get_device_error(ctx) == hh.HH_OK
    return out


@pytest.mark.parametrize("bits,key_mode", [(64, 1), (128, 0), (256, 1)])
def test_pieces_equal_whole(ctx, bits, key_mode):
    rng = np.random.default_rng(bits + key_mode)
    lengths = np.concatenate([rng.integers(0, 3000, 2000), rng.integers(0, 65, 500),
                              rng.integers(1 << 17, 1 << 19, 12)])
    w = workloads.from_lengths(torch.from_numpy(lengths), seed=bits, device=DEV,
                               per_message_keys=bool(key_mode))
    keys = w.keys if key_mode else w.keys
    pieces = _split(lengths, 3, rng)
    got = _run_streams(ctx, w, pieces, bits, key_mode)
    whole = WHOLE[bits](ctx, keys, key_mode, w.data, w.offsets)
    assert torch.equal(got, whole)
    sample = np.unique(np.concatenate([np.arange(0, w.n, 37), np.arange(w.n - 12, w.n)]))
    assert np.array_equal(got.cpu().numpy().view(np.uint64).reshape(-1, bits // 64)[sample],
                          oracle_hashes(w, bits, indices=sample))


def test_short_streams(ctx):
    """Pieces of 0, 32 or 64 bytes and a last piece of 0..64: the short kernel."""
    rng = np.random.default_rng(7)
    n = 4000
    pieces = np.stack([32 * rng.integers(0, 3, n), 32 * rng.integers(0, 3, n),
                       rng.integers(0, 65, n)], axis=1)
    w = workloads.from_lengths(torch.from_numpy(pieces.sum(axis=1)), seed=7, device=DEV)
    got = _run_streams(ctx, w, pieces, 64, 1)
    assert torch.equal(got, hh.hh_hash64_batch(ctx, w.keys, 1, w.data, w.offsets))


def test_init_state_matches_oracle(ctx, oracle):
    key = np.array([11, 22, 33, 44], dtype=np.uint64)
    states = hh.hh_stream_init(ctx, torch.from_numpy(key.view(np.int64)).to(DEV), 0, 3)
    s = oracle.lib().init_state([int(x) for x in key])
    v0, v1, mul0, mul1 = s.as_lists()
    expect = np.array(v0 + v1 + mul0 + mul1, dtype=np.uint64)
    for row in states.cpu().numpy().view(np.uint64):
        assert np.array_equal(row, expect)


def test_bad_chunk_leaves_state(ctx):
    w = workloads.from_lengths(torch.tensor([64, 64, 64]), seed=3, device=DEV)
    states = hh.hh_stream_init(ctx, w.keys, 1, 3)
    before = states.clone()
    offs = torch.tensor([0, 32, 65, 97], dtype=torch.int64, device=DEV)  # 32, 33, 32 bytes
    data = torch.zeros(97, dtype=torch.uint8, device=DEV)
    hh.hh_stream_update(ctx, states, data, offs)
    assert hh.hh_get_device_error(ctx) == hh.HH_ERR_BAD_CHUNK
    assert torch.equal(states[1], before[1])
    assert not torch.equal(states[0], before[0]) and not torch.equal(states[2], before[2])


def test_unsorted_kernel_streams_and_naive_refuses(ctx):
    rng = np.random.default_rng(9)
    lengths = rng.integers(0, 5000, 3000)
    w = workloads.from_lengths(torch.from_numpy(lengths), seed=9, device=DEV)
    pieces = _split(lengths, 2, rng)
    hh.hh_set_kernel(ctx, hh.HH_KERNEL_STAGED_UNSORTED)
    try:
        got = _run_streams(ctx, w, pieces, 64, 1)
    finally:
        hh.hh_set_kernel(ctx, hh.HH_KERNEL_AUTO)
    assert torch.equal(got, hh.hh_hash64_batch(ctx, w.keys, 1, w.data, w.offsets))
    hh.hh_set_kernel(ctx, hh.HH_KERNEL_NAIVE)
    try:
        states = hh.hh_stream_init(ctx, w.keys, 1, w.n)
        with pytest.raises(hh.HHError):
            hh.hh_stream_update(ctx, states, w.data, w.offsets)
    finally:
        hh.hh_set_kernel(ctx, hh.HH_KERNEL_AUTO)

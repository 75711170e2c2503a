"""GPU parity: libhh (through the C ABI) against the CPU oracle, bit for bit.

HighwayHash is exact integer arithmetic, so the tolerance is zero: every
output word must equal the oracle's.  Small cases are checked on every
message; the full configuration sizes (the ones the benchmark times) are
checked on seeded random samples of messages plus properties that hold at any
size.  Parity with any released HighwayHash library is not claimed: the
oracle implements the paper's definition.
"""
import numpy as np
import pytest
import torch

from paper_1612_06257_gb300 import hh, workloads
from tests.helpers import as_u64, oracle_hashes

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
WORDS = {64: 1, 128: 2, 256: 4}
RAGGED_FN = {64: hh.hh_hash64_batch, 128: hh.hh_hash128_batch, 256: hh.hh_hash256_batch}
KERNELS = {"auto": hh.HH_KERNEL_AUTO, "naive": hh.HH_KERNEL_NAIVE,
           "unsorted": hh.HH_KERNEL_STAGED_UNSORTED}


@pytest.fixture(scope="module")
def ctx():
    from paper_1612_06257_gb300 import build
    build.build()
    c = hh.hh_init(0)
    yield c
    hh.hh_destroy(c)


def run_ragged(ctx, w, bits, kernel="auto"):
    hh.hh_set_kernel(ctx, KERNELS[kernel])
    try:
        out = RAGGED_FN[bits](ctx, w.keys, w.key_mode, w.data, w.offsets_or_stride())
        assert hh.hh_get_device_error(ctx) == hh.HH_OK
    finally:
        hh.hh_set_kernel(ctx, hh.HH_KERNEL_AUTO)
    return as_u64(out, WORDS[bits])


def run_fixed(ctx, w, bits, kernel="auto"):
    hh.hh_set_kernel(ctx, KERNELS[kernel])
    try:
        out = hh.hh_hash_fixed(ctx, bits, w.keys, w.key_mode, w.data, w.fixed_len, w.n)
        assert hh.hh_get_device_error(ctx) == hh.HH_OK
    finally:
        hh.hh_set_kernel(ctx, hh.HH_KERNEL_AUTO)
    return as_u64(out, WORDS[bits])


# ------------------------------------------------------------ every message

@pytest.mark.parametrize("bits", [64, 128, 256])
def test_fixed_1k_messages_4096(ctx, bits):
    """4096 messages of 1024 bytes, one key (the small fixed-length batch)."""
    w = workloads.fixed(4096, 1024, seed=1, device=DEV)
    expect = oracle_hashes(w, bits)
    assert np.array_equal(run_fixed(ctx, w, bits), expect)
    assert np.array_equal(run_fixed(ctx, w, bits, "naive"), expect)
    assert np.array_equal(run_ragged(ctx, w, bits), expect)


@pytest.mark.parametrize("length", [0, 1, 3, 16, 31, 32, 33, 48, 63, 64, 100, 1024, 1041, 4096])
@pytest.mark.parametrize("per_message_keys", [False, True])
def test_fixed_lengths(ctx, length, per_message_keys):
    """Fixed lengths with and without 16-byte alignment; 300 messages = 2 full
    tiles of 128 plus a ragged tail of 44."""
    w = workloads.fixed(300, length, seed=2 + length, device=DEV,
                        per_message_keys=per_message_keys)
    for bits in (64, 256):
        expect = oracle_hashes(w, bits)
        assert np.array_equal(run_fixed(ctx, w, bits), expect), (length, bits)


def test_fixed_unaligned_base_pointer(ctx):
    """The byte buffer starts 3 bytes into an allocation: no 16-byte alignment."""
    n, length = 257, 64
    g = workloads.generator(3, DEV)
    backing = workloads.random_bytes(n * length + 3, g, DEV)
    w = workloads.Workload("fixed", backing[3:], None, length,
                           workloads.random_u64((4,), g, DEV), False, n)
    expect = oracle_hashes(w, 64)
    assert np.array_equal(run_fixed(ctx, w, 64), expect)


@pytest.mark.parametrize("kernel", ["auto", "unsorted", "naive"])
def test_every_length_0_to_1024(ctx, kernel):
    """Two messages of every length 0..1024 in shuffled order (every residue
    mod 32 many times, every byte alignment), per-message keys, all widths."""
    lengths = torch.arange(0, 1025).repeat(2)
    lengths = lengths[torch.randperm(lengths.numel(), generator=torch.Generator().manual_seed(5))]
    w = workloads.from_lengths(lengths, seed=5, device=DEV, per_message_keys=True)
    for bits in (64, 128, 256):
        assert np.array_equal(run_ragged(ctx, w, bits, kernel), oracle_hashes(w, bits)), bits


def test_ragged_loguniform_small(ctx):
    """The log-uniform ragged recipe (lengths 0..65536, per-message keys) at
    n = 16384; all messages checked."""
    w = workloads.ragged(16384, seed=6, device=DEV)
    expect = oracle_hashes(w, 64)
    assert np.array_equal(run_ragged(ctx, w, 64), expect)
    assert np.array_equal(run_ragged(ctx, w, 64, "unsorted"), expect)


@pytest.mark.parametrize("bits", [64, 128, 256])
def test_short_messages_small(ctx, bits):
    """Lengths uniform in [0, 64], 10% all-zero messages, one key; n = 65536
    (the short kernel, one instantiation per output width)."""
    w = workloads.short(65536, seed=7, device=DEV)
    assert np.array_equal(run_ragged(ctx, w, bits), oracle_hashes(w, bits))


def test_kernels_agree_on_mixed_batch(ctx):
    lengths = torch.cat([torch.randint(0, 65, (3000,)), torch.full((200,), 1024),
                         torch.randint(1 << 15, 1 << 17, (20,))])
    w = workloads.from_lengths(lengths, seed=8, device=DEV, per_message_keys=True)
    results = [run_ragged(ctx, w, 256, k) for k in ("auto", "unsorted", "naive")]
    assert np.array_equal(results[0], results[1]) and np.array_equal(results[0], results[2])
    assert np.array_equal(results[0], oracle_hashes(w, 256))


# ----------------------------------------------------------------- edge cases

def test_empty_batch_is_a_noop(ctx):
    keys = torch.zeros(4, dtype=torch.int64, device=DEV)
    data = torch.zeros(16, dtype=torch.uint8, device=DEV)
    offsets = torch.zeros(1, dtype=torch.int64, device=DEV)
    out = torch.full((4,), 7, dtype=torch.int64, device=DEV)
    hh.hh_hash64_batch(ctx, keys, 0, data, offsets, n=0, out=out)
    assert hh.hh_last_launch_count(ctx) == 0
    assert out.tolist() == [7, 7, 7, 7]


def test_all_empty_messages(ctx):
    w = workloads.from_lengths([0] * 2000, seed=9, device=DEV, per_message_keys=True)
    w.data = torch.zeros(16, dtype=torch.uint8, device=DEV)  # unused, must be non-null
    assert np.array_equal(run_ragged(ctx, w, 128), oracle_hashes(w, 128))


def test_offsets_not_starting_at_zero_and_exact_end(ctx):
    """Messages occupy bytes [100, total) of the buffer, the last one ending on
    the buffer's last byte, and the buffer length is not a multiple of 16."""
    lengths = torch.tensor([5, 33, 0, 64, 1, 100, 31, 17])
    w = workloads.from_lengths(lengths, seed=10, device=DEV)
    pad = torch.zeros(100, dtype=torch.uint8, device=DEV)
    data = torch.cat([pad, w.data])
    assert data.numel() % 16 != 0
    shifted = workloads.Workload("shifted", data, w.offsets + 100, None, w.keys, True, w.n)
    expect = oracle_hashes(w, 64)
    for kernel in ("auto", "naive", "unsorted"):
        assert np.array_equal(run_ragged(ctx, shifted, 64, kernel), expect)


@pytest.mark.parametrize("kernel", ["auto", "unsorted"])
def test_short_messages_at_unaligned_batch_ends(ctx, kernel):
    """All messages of 0..64 bytes (the direct-load path), with the byte
    buffer starting 3 bytes into an allocation and ending mid-word, in a
    batch large enough (1500) to run the length sort."""
    g = torch.Generator().manual_seed(31)
    lengths = torch.randint(0, 65, (1500,), generator=g)
    lengths[0], lengths[-1] = 63, 61
    w = workloads.from_lengths(lengths, seed=31, device=DEV)
    backing = torch.zeros(w.total_bytes + 8, dtype=torch.uint8, device=DEV)
    backing[3:3 + w.total_bytes] = w.data
    view = backing[3:3 + w.total_bytes]
    shifted = workloads.Workload("short", view, w.offsets, None, w.keys, True, w.n)
    for bits in (64, 256):
        assert np.array_equal(run_ragged(ctx, shifted, bits, kernel), oracle_hashes(w, bits))


@pytest.mark.parametrize("per_message_keys", [False, True])
def test_short_kernel_at_unaligned_batch_ends(ctx, per_message_keys):
    """All messages of 0..64 bytes in a batch above the short kernel's minimum
    size (10000 messages), with the byte buffer starting 3 bytes into an
    allocation of other bytes and ending mid-word: the word windows of the
    first and last messages cross the batch ends.  One key (the loop that
    stages offsets and words in shared memory) or a key per message (the loop
    that stages offsets only)."""
    g = torch.Generator().manual_seed(41)
    lengths = torch.randint(0, 65, (10000,), generator=g)
    lengths[0], lengths[1], lengths[-2], lengths[-1] = 63, 2, 1, 61
    w = workloads.from_lengths(lengths, seed=41, device=DEV, per_message_keys=per_message_keys)
    backing = torch.randint(0, 256, (w.total_bytes + 8,), dtype=torch.uint8, device=DEV)
    backing[3:3 + w.total_bytes] = w.data
    view = backing[3:3 + w.total_bytes]
    shifted = workloads.Workload("short", view, w.offsets, None, w.keys, per_message_keys, w.n)
    for bits in (64, 128, 256):
        assert np.array_equal(run_ragged(ctx, shifted, bits), oracle_hashes(w, bits))


@pytest.mark.parametrize("per_message_keys", [False, True])
def test_short_kernel_flags_decreasing_offsets(ctx, per_message_keys):
    """A descriptor with end < start inside an all-short batch of 10000
    messages: the short kernel records the error and writes a zero hash for
    that message; every other message is hashed as its offsets say."""
    g = torch.Generator().manual_seed(43)
    lengths = torch.randint(0, 65, (10000,), generator=g)
    lengths[5000], lengths[5001] = 20, 10
    w = workloads.from_lengths(lengths, seed=43, device=DEV, per_message_keys=per_message_keys)
    bad = w.offsets.clone()
    bad[5001] = bad[5000] - 3  # message 5000 ends before it starts; 5001 grows to 33 bytes
    broken = workloads.Workload("short", w.data, bad, None, w.keys, per_message_keys, w.n)
    out = hh.hh_hash128_batch(ctx, w.keys, w.key_mode, w.data, bad)
    assert hh.hh_get_device_error(ctx) == hh.HH_ERR_BAD_OFFSETS
    got = as_u64(out, 2)
    assert got[5000].tolist() == [0, 0]
    others = np.array([i for i in range(w.n) if i != 5000])
    assert np.array_equal(got[others], oracle_hashes(broken, 128, indices=others))


def test_short_kernel_offsets_that_jump_back(ctx):
    """One key, 12000 messages of at most 64 bytes (the short kernel).
    Decreasing offsets put a valid message before the bytes of the 64
    messages around it (messages 6409/6410), and make the offset 64 messages
    on from message 3200 fall below it (messages 3263/3264).  The two
    descriptors with end < start get zero hashes, every other message the
    oracle's."""
    g = torch.Generator().manual_seed(47)
    lengths = torch.randint(0, 65, (12000,), generator=g)
    lengths[6400:6416] = 1
    lengths[3200:3266] = torch.randint(0, 2, (66,), generator=g)
    w = workloads.from_lengths(lengths, seed=47, device=DEV, per_message_keys=False)
    off = w.offsets.clone()
    off[6410] = off[6400] - 20  # 6409 ends before it starts; 6410 lies before its chunk
    off[6411] = off[6400] - 5
    off[3264] = off[3200] - 1  # 3263 ends before it starts; chunk 3200..3263 is inverted
    bad_msgs = [3263, 6409]
    lens = (off[1:] - off[:-1]).cpu()
    assert int(lens.max()) <= 64 and all(int(lens[i]) < 0 for i in bad_msgs)
    assert int((lens < 0).sum()) == len(bad_msgs)
    broken = workloads.Workload("short", w.data, off, None, w.keys, False, w.n)
    out = hh.hh_hash64_batch(ctx, w.keys, 0, w.data, off)
    assert hh.hh_get_device_error(ctx) == hh.HH_ERR_BAD_OFFSETS
    got = as_u64(out, 1)
    assert all(int(got[i, 0]) == 0 for i in bad_msgs)
    others = np.array([i for i in range(w.n) if i not in bad_msgs])
    assert np.array_equal(got[others], oracle_hashes(broken, 64, indices=others))


@pytest.mark.parametrize("case", ["all_short", "long_last", "long_first", "all_1k", "spread"])
def test_short_kernel_with_the_length_count(ctx, case):
    """One key, offsets form, 20000 messages: the short kernel also counts the
    length buckets of the sort, and hashes short messages until it meets a
    longer one (or a thread that did has set the flag); the warp-tile kernel
    then hashes the whole batch in sorted order.  All messages of 0..64
    bytes; one of 65 bytes last or first among them; all of 1 KiB; lengths
    spread over many buckets (0..5000 bytes and four of 64 KiB to 1 MiB).
    The output starts filled with a pattern and every message is checked
    against the oracle (a bucket miscounted would leave a message out of the
    sorted order).  Launches: the short kernel, the scan, the scatter and the
    two warp-tile variants."""
    g = torch.Generator().manual_seed(97)
    n = 20000
    if case == "all_1k":
        lengths = torch.full((n,), 1024)
    elif case == "spread":
        lengths = torch.cat([torch.randint(0, 5001, (n - 4,), generator=g),
                             torch.tensor([1 << 16, (1 << 17) + 5, 700001, (1 << 20) + 9])])
        lengths = lengths[torch.randperm(n, generator=g)]
    else:
        lengths = torch.randint(0, 65, (n,), generator=g)
        if case != "all_short":
            lengths[-1 if case == "long_last" else 0] = 65
    w = workloads.from_lengths(lengths, seed=97, device=DEV, per_message_keys=False)
    for bits, fn in ((64, hh.hh_hash64_batch), (256, hh.hh_hash256_batch)):
        out = torch.full((n * WORDS[bits],), 0x5A5A5A5A, dtype=torch.int64, device=DEV)
        fn(ctx, w.keys, 0, w.data, w.offsets, out=out)
        assert hh.hh_get_device_error(ctx) == hh.HH_OK
        assert hh.hh_last_launch_count(ctx) == 5
        assert np.array_equal(as_u64(out, WORDS[bits]), oracle_hashes(w, bits)), (case, bits)


def test_output_guard_words_untouched(ctx):
    w = workloads.ragged(3000, seed=11, device=DEV, max_len=3000)
    out = torch.full((3000 * 2 + 64,), -0x5A5A5A5A5A5A5A5B, dtype=torch.int64, device=DEV)
    hh.hh_hash128_batch(ctx, w.keys, w.key_mode, w.data, w.offsets, out=out)
    assert hh.hh_get_device_error(ctx) == hh.HH_OK
    assert torch.all(out[6000:] == -0x5A5A5A5A5A5A5A5B)
    assert np.array_equal(as_u64(out[:6000], 2), oracle_hashes(w, 128))


def test_decreasing_offsets_set_device_error(ctx):
    lengths = torch.tensor([10, 20, 30, 40])
    w = workloads.from_lengths(lengths, seed=12, device=DEV)
    bad = w.offsets.clone()
    bad[2] = bad[1] - 5  # message 1 has end < start; message 2 is long but valid
    out = hh.hh_hash64_batch(ctx, w.keys, 1, w.data, bad)
    assert hh.hh_get_device_error(ctx) == hh.HH_ERR_BAD_OFFSETS
    assert int(out[1].item()) == 0
    assert hh.hh_get_device_error(ctx) == hh.HH_OK  # cleared by the read


def test_invalid_arguments(ctx):
    keys = torch.zeros(4, dtype=torch.int64, device=DEV)
    data = torch.zeros(64, dtype=torch.uint8, device=DEV)
    offsets = torch.tensor([0, 64], dtype=torch.int64, device=DEV)
    L = hh.load_library()
    stream = torch.cuda.current_stream().cuda_stream
    out = torch.zeros(4, dtype=torch.int64, device=DEV)
    assert L.hh_hash64_batch(ctx.ptr, keys.data_ptr(), 2, data.data_ptr(), offsets.data_ptr(), 1,
                             out.data_ptr(), stream) == hh.HH_ERR_INVALID_ARG
    assert L.hh_hash64_batch(ctx.ptr, keys.data_ptr(), 0, data.data_ptr(), None, 1,
                             out.data_ptr(), stream) == hh.HH_ERR_INVALID_ARG
    assert L.hh_hash64_batch(ctx.ptr, keys.data_ptr(), 0, data.data_ptr(), offsets.data_ptr(), -1,
                             out.data_ptr(), stream) == hh.HH_ERR_INVALID_ARG
    assert L.hh_hash_fixed(ctx.ptr, 96, keys.data_ptr(), 0, data.data_ptr(), 64, 1,
                           out.data_ptr(), stream) == hh.HH_ERR_INVALID_ARG
    assert L.hh_set_kernel(ctx.ptr, 17) == hh.HH_ERR_INVALID_ARG


def test_determinism_and_widths_share_lanes(ctx):
    w = workloads.ragged(5000, seed=13, device=DEV, max_len=4096)
    h64 = run_ragged(ctx, w, 64)
    h128 = run_ragged(ctx, w, 128)
    h256 = run_ragged(ctx, w, 256)
    assert np.array_equal(h64[:, 0], h256[:, 0]) and np.array_equal(h128, h256[:, :2])
    assert np.array_equal(run_ragged(ctx, w, 256), h256)


def test_host_buffer_entry_point(ctx):
    """hh_hash_host with pinned host buffers, several chunks, per-message keys."""
    w = workloads.ragged(40000, seed=14, device=DEV, max_len=8192)
    assert w.total_bytes > (64 << 20) // 2
    keys = w.keys.cpu().numpy().view(np.uint64).copy()
    data = w.data.cpu().pin_memory().numpy()
    offsets = w.offsets.cpu().numpy()
    out = hh.hh_hash_host(ctx, 128, keys.reshape(-1), 1, data, offsets)
    assert np.array_equal(out.reshape(-1, 2), oracle_hashes(w, 128))
    big = workloads.fixed(1 << 17, 1024, seed=15, device=DEV)  # 128 MiB: 2+ chunks
    offs = big.offsets_or_stride().cpu().numpy()
    out = hh.hh_hash_host(ctx, 64, big.keys.cpu().numpy().view(np.uint64).copy(), 0,
                          big.data.cpu().numpy(), offs)
    sample = np.random.default_rng(15).choice(big.n, 500, replace=False)
    assert np.array_equal(out[sample], oracle_hashes(big, 64, indices=sample)[:, 0])


# ------------------------------------------- full configuration sizes, sampled

def _sample(n, count, seed):
    rng = np.random.default_rng(seed)
    idx = rng.choice(n, size=min(count, n), replace=False)
    return np.sort(np.concatenate([idx, [0, n - 1]]).astype(np.int64))


@pytest.mark.parametrize("bits", [64, 128, 256])
def test_full_size_1gib_fixed_1k(ctx, bits):
    """2^20 messages of 1024 bytes (1 GiB), one key: the benchmark's launch."""
    w = workloads.fixed(1 << 20, 1024, seed=21, device=DEV)
    got = run_fixed(ctx, w, bits)
    idx = _sample(w.n, 3000, 21)
    assert np.array_equal(got[idx], oracle_hashes(w, bits, indices=idx))
    # Distinct random messages give distinct 64-bit hashes (a collision among
    # 2^20 would have probability about 2^-25).
    assert np.unique(got[:, 0]).size == w.n


def test_full_size_ragged_4m_messages(ctx):
    """2^22 log-uniform messages (about 25 GB) with per-message keys."""
    w = workloads.ragged(1 << 22, seed=22, device=DEV)
    got = run_ragged(ctx, w, 64)
    lengths = (w.offsets[1:] - w.offsets[:-1]).cpu().numpy()
    idx = _sample(w.n, 2000, 22)
    longest = np.argsort(lengths)[-50:]
    idx = np.unique(np.concatenate([idx, longest]))
    assert np.array_equal(got[idx], oracle_hashes(w, 64, indices=idx))
    del w
    torch.cuda.empty_cache()


@pytest.mark.parametrize("bits", [64, 128])
def test_full_size_short_64m_messages(ctx, bits):
    """2^26 messages of 0..64 bytes, 10% all zero, one key."""
    w = workloads.short(1 << 26, seed=23, device=DEV)
    hh.hh_reserve(ctx, w.n)  # beyond the default sort scratch of 2^22 messages
    got = run_ragged(ctx, w, bits)
    idx = _sample(w.n, 20000, 23)
    assert np.array_equal(got[idx], oracle_hashes(w, bits, indices=idx))
    del w
    torch.cuda.empty_cache()


# ------------------------------------------------------------------ segments

def _segments_case(n, seed, max_len, pool_bytes, key_rows):
    g = torch.Generator().manual_seed(seed)
    lengths = torch.randint(0, max_len + 1, (n,), generator=g, dtype=torch.int64)
    starts = (torch.rand(n, generator=g, dtype=torch.float64) *
              (pool_bytes - lengths).to(torch.float64)).to(torch.int64)
    key_index = torch.randint(0, key_rows, (n,), generator=g, dtype=torch.int32)
    gd = workloads.generator(seed, DEV)
    pool = workloads.random_bytes(pool_bytes, gd, DEV)
    table = workloads.random_u64((key_rows, 4), gd, DEV)
    return table, key_index, pool, starts, lengths


@pytest.mark.parametrize("kernel", ["auto", "unsorted", "naive"])
@pytest.mark.parametrize("n,max_len", [(700, 3000), (5000, 64), (12000, 64), (4000, 70000)])
def test_segments_with_key_table(ctx, kernel, n, max_len):
    """Segments of one pool in random order (overlapping), keys from a device
    key table by index: the request-server batch form."""
    from tests.helpers import oracle_segments
    table, key_index, pool, starts, lengths = _segments_case(n, 40 + n, max_len, 1 << 22, 37)
    hh.hh_set_kernel(ctx, KERNELS[kernel])
    try:
        out = hh.hh_hash_segments(ctx, 128, table, key_index.to(DEV), pool, starts.to(DEV),
                                  lengths.to(DEV))
        assert hh.hh_get_device_error(ctx) == hh.HH_OK
    finally:
        hh.hh_set_kernel(ctx, hh.HH_KERNEL_AUTO)
    expect = oracle_segments(table.cpu().numpy(), key_index.numpy(), pool.cpu().numpy(),
                             starts.numpy(), lengths.numpy(), 128)
    assert np.array_equal(as_u64(out, 2), expect)


def test_segments_shared_key_and_bad_descriptors(ctx):
    from tests.helpers import oracle_segments
    table, key_index, pool, starts, lengths = _segments_case(2000, 61, 200, 1 << 16, 1)
    out = hh.hh_hash_segments(ctx, 64, table, None, pool, starts.to(DEV), lengths.to(DEV))
    assert hh.hh_get_device_error(ctx) == hh.HH_OK
    expect = oracle_segments(table.cpu().numpy(), None, pool.cpu().numpy(), starts.numpy(),
                             lengths.numpy(), 64)
    assert np.array_equal(as_u64(out, 1), expect)
    # A segment past the end of the buffer, then a key index past the table.
    bad = starts.clone()
    bad[5] = (1 << 16) - 3
    lengths2 = lengths.clone()
    lengths2[5] = 10
    out = hh.hh_hash_segments(ctx, 64, table, None, pool, bad.to(DEV), lengths2.to(DEV))
    assert hh.hh_get_device_error(ctx) == hh.HH_ERR_BAD_OFFSETS
    assert int(out[5].item()) == 0
    kidx = torch.zeros(2000, dtype=torch.int32)
    kidx[7] = 1
    out = hh.hh_hash_segments(ctx, 64, table, kidx.to(DEV), pool, starts.to(DEV), lengths.to(DEV))
    assert hh.hh_get_device_error(ctx) == hh.HH_ERR_BAD_KEY_INDEX
    assert int(out[7].item()) == 0


@pytest.fixture(scope="module", params=["solo", "pair"])
def huge_ctx(request, tmp_path_factory):
    """A context whose huge messages (128 KiB and more) run as solo tiles
    (one per warp, the default while they are few) or as pair tiles (16 per
    warp; a tuning table that switches solo tiles off)."""
    if request.param == "solo":
        c = hh.hh_init(0)
    else:
        path = tmp_path_factory.mktemp("tune") / "pairs.txt"
        path.write_text("solo_per_sm 0\n")
        c = hh.hh_init(0, str(path))
    yield c
    hh.hh_destroy(c)


def test_huge_messages_run_in_solo_and_pair_tiles(huge_ctx):
    """Messages of 128 KiB and more take the solo or pair tiles at the head of
    the length order; mixed with ordinary and short ones, with unaligned
    starts, every width, against the oracle."""
    ctx = huge_ctx
    g = torch.Generator().manual_seed(91)
    lengths = torch.cat([
        (torch.rand(40, generator=g, dtype=torch.float64) * (4 << 20 - 1)).to(torch.int64) + (1 << 17),
        torch.full((3,), 1 << 17), torch.full((2,), (1 << 17) - 1),
        torch.randint(0, 5000, (1500,), generator=g)])
    lengths = lengths[torch.randperm(lengths.numel(), generator=g)]
    w = workloads.from_lengths(lengths, seed=91, device=DEV, per_message_keys=True)
    for bits in (64, 128, 256):
        got = run_ragged(ctx, w, bits)
        big = np.nonzero(lengths.numpy() >= (1 << 17))[0]
        idx = np.unique(np.concatenate([big, np.arange(0, w.n, 7)]))
        assert np.array_equal(got[idx], oracle_hashes(w, bits, indices=idx)), bits
        assert np.array_equal(got, run_ragged(ctx, w, bits, "unsorted"))


def test_large_batch_with_huge_messages(huge_ctx):
    """Above 8192 messages the sort runs in three launches and both variants
    of the warp-tile kernel are launched (with and without the huge-message
    phase); with huge messages present the variant with the phase does all
    the work.  20000 ordinary messages and six of 128 KiB to 1 MiB + 13,
    unaligned starts, against the oracle."""
    ctx = huge_ctx
    g = torch.Generator().manual_seed(93)
    lengths = torch.cat([torch.randint(0, 5000, (20000,), generator=g),
                         torch.tensor([1 << 17, (1 << 17) + 1, 300001, 500000, 777777,
                                       (1 << 20) + 13])])
    lengths = lengths[torch.randperm(lengths.numel(), generator=g)]
    w = workloads.from_lengths(lengths, seed=93, device=DEV, per_message_keys=True)
    big = np.nonzero(lengths.numpy() >= (1 << 17))[0]
    idx = np.unique(np.concatenate([big, np.arange(0, w.n, 13), [w.n - 1]]))
    for bits in (64, 256):
        got = run_ragged(ctx, w, bits)
        assert hh.hh_last_launch_count(ctx) == 6  # sort 3, short kernel 1, warp tiles 2
        assert np.array_equal(got[idx], oracle_hashes(w, bits, indices=idx)), bits


def test_single_huge_message_alone(huge_ctx):
    """A batch of one message (sorted too): 2 MiB + 17 bytes starting at an
    odd offset of its buffer, and one ending on the buffer's last byte."""
    ctx = huge_ctx
    for start, length in ((5, (2 << 20) + 17), (0, (1 << 20) + 3)):
        g = torch.Generator(device=DEV).manual_seed(start + 1)
        data = torch.randint(0, 256, (start + length,), dtype=torch.uint8, device=DEV, generator=g)
        offsets = torch.tensor([start, start + length], dtype=torch.int64, device=DEV)
        keys = torch.tensor([1, -2, 3, -4], dtype=torch.int64, device=DEV)
        w = workloads.Workload("one", data, offsets, None, keys, False, 1)
        for bits in (64, 256):
            got = as_u64(RAGGED_FN[bits](ctx, keys, 0, data, offsets), WORDS[bits])
            assert hh.hh_get_device_error(ctx) == hh.HH_OK
            assert np.array_equal(got, oracle_hashes(w, bits)), (start, bits)


def test_solo_limit_boundary(ctx):
    """Exactly 4 huge messages per SM run as solo tiles, one more as pair
    tiles (the default limit); both agree with the oracle."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    for count in (4 * sms, 4 * sms + 1):
        g = torch.Generator().manual_seed(count)
        lengths = torch.cat([torch.randint(1 << 17, (1 << 17) + 4096, (count,), generator=g),
                             torch.randint(0, 3000, (600,), generator=g)])
        w = workloads.from_lengths(lengths, seed=count, device=DEV, per_message_keys=True)
        got = run_ragged(ctx, w, 128)
        idx = np.unique(np.concatenate([np.arange(0, count, 5), [count - 1],
                                        np.arange(count, w.n, 11)]))
        assert np.array_equal(got[idx], oracle_hashes(w, 128, indices=idx)), count


def test_fixed_batches_either_side_of_the_two_threads_per_message_size(ctx):
    """Fixed-length batches smaller than one tile per SM (at the tuned
    messages per thread) run two threads per message in tiles of 32, 64 or
    128 rows; larger ones run the tuned kernel.  Both sides of the boundary, every width, against the
    oracle on samples that include both ends of the batch."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    # below: 32-, 64- and 128-row tiles of the two-threads kernel; above: tuned
    for n in (40 * sms + 3, 80 * sms + 5, 2 * 128 * sms - 1, 2 * 128 * sms + 128):
        for length, bits in ((48, 256), (1040, 64), (208, 128)):
            w = workloads.fixed(n, length, seed=n + length, device=DEV,
                                per_message_keys=(bits == 128))
            got = as_u64(hh.hh_hash_fixed(ctx, bits, w.keys, w.key_mode, w.data, length, n),
                         WORDS[bits])
            assert hh.hh_get_device_error(ctx) == hh.HH_OK
            idx = np.unique(np.concatenate([np.arange(0, n, 97), [n - 1, n - 2]]))
            assert np.array_equal(got[idx], oracle_hashes(w, bits, indices=idx)), (n, length)


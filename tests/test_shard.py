"""Sharding one ragged batch over ranks (CPU only).

The byte-balanced split is checked as host arithmetic, and the whole N > 1
path (split, per-rank hashing, gather on rank 0, max-over-ranks timing) runs
as two gloo processes on the CPU.  There the oracle stands in for each
rank's GPU: the test checks the distribution logic, and GPU parity is
checked elsewhere.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1612_06257_gb300.shard import byte_balanced_ranges, gather_to_rank0


def _offsets(lengths):
    return np.concatenate([[0], np.cumsum(np.asarray(lengths, dtype=np.int64))])


def _check_cover(ranges, n):
    assert ranges[0][0] == 0 and ranges[-1][1] == n
    for (a, b), (c, d) in zip(ranges, ranges[1:]):
        assert a <= b == c <= d


@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_ranges_cover_and_balance(world):
    rng = np.random.default_rng(world)
    lengths = np.floor(np.exp(rng.uniform(0, np.log(65537), 5000))).astype(np.int64) - 1
    off = _offsets(lengths)
    ranges = byte_balanced_ranges(off, world)
    _check_cover(ranges, len(lengths))
    total = off[-1]
    for first, last in ranges:
        share = off[last] - off[first]
        assert abs(share - total / world) <= lengths.max() + 1


def test_ranges_edge_cases():
    assert byte_balanced_ranges(_offsets([]), 4) == [(0, 0)] * 4
    zeros = byte_balanced_ranges(_offsets([0] * 10), 3)
    _check_cover(zeros, 10)
    assert sum(b - a for a, b in zeros) == 10
    few = byte_balanced_ranges(_offsets([5, 5]), 4)
    _check_cover(few, 2)
    one_big = byte_balanced_ranges(_offsets([1] * 10 + [10 ** 6] + [1] * 10), 2)
    _check_cover(one_big, 21)
    # offsets that do not start at zero
    shifted = byte_balanced_ranges(_offsets([3, 4, 5, 6]) + 100, 2)
    assert shifted == byte_balanced_ranges(_offsets([3, 4, 5, 6]), 2)
    with pytest.raises(ValueError):
        byte_balanced_ranges(np.array([0, 5, 3]), 2)
    with pytest.raises(ValueError):
        byte_balanced_ranges(_offsets([1]), 0)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, result_path):
    import oracle
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        rng = np.random.default_rng(5)
        lengths = rng.integers(0, 3000, 777)
        off = _offsets(lengths)
        data = rng.integers(0, 256, int(off[-1]), dtype=np.uint8)
        keys = rng.integers(0, 2 ** 63, (777, 4), dtype=np.int64).view(np.uint64)
        ranges = byte_balanced_ranges(off, world)
        first, last = ranges[rank]
        local = np.zeros((last - first, 2), dtype=np.uint64)
        # this rank's shard (offsets are absolute positions in `data`)
        oracle.hash_batch(np.ascontiguousarray(keys[first:last]), True, data,
                          np.ascontiguousarray(off[first:last + 1]), 128, 0, last - first, local)
        elapsed = torch.tensor([float(rank + 1)])
        dist.all_reduce(elapsed, op=dist.ReduceOp.MAX)
        full = gather_to_rank0(torch.from_numpy(local.view(np.int64).reshape(-1)), ranges, 2)
        if rank == 0:
            whole = np.zeros((777, 2), dtype=np.uint64)
            oracle.hash_batch(keys, True, data, off, 128, 0, 777, whole)
            ok = np.array_equal(full.numpy().view(np.uint64).reshape(-1, 2), whole)
            with open(result_path, "w") as f:
                f.write("%d %g" % (ok, elapsed.item()))
    finally:
        dist.destroy_process_group()


def test_two_rank_gloo_shard_and_gather(tmp_path, oracle):
    result = tmp_path / "result.txt"
    mp.start_processes(_rank_main, args=(2, _free_port(), str(result)), nprocs=2, join=True,
                       start_method="spawn")
    ok, slowest = result.read_text().split()
    assert ok == "1"
    assert float(slowest) == 2.0  # max over ranks


@pytest.mark.gpu
def test_shards_on_gpu_equal_whole_batch():
    """hash_shard over every rank's range, on one GPU, concatenates to the
    whole-batch result (per-message keys, offsets not starting at zero)."""
    from paper_1612_06257_gb300 import build, hh, shard, workloads
    build.build()
    dev = "cuda:0"
    ctx = hh.hh_init(0)
    try:
        g = torch.Generator().manual_seed(3)
        lengths = torch.cat([torch.randint(0, 4000, (3000,), generator=g),
                             torch.tensor([300000, 5, 200000])])
        w = workloads.from_lengths(lengths, seed=3, device=dev)
        offsets = w.offsets[1:].contiguous()   # drop message 0: offsets start past zero
        keys = w.keys[1:].contiguous()
        n = offsets.numel() - 1
        whole = hh.hh_hash256_batch(ctx, keys, 1, w.data, offsets)
        ranges = shard.byte_balanced_ranges(offsets, 3)
        parts = [shard.hash_shard(ctx, 256, keys, 1, w.data, offsets, r, 3, ranges=ranges)[2]
                 for r in range(3)]
        assert hh.hh_get_device_error(ctx) == hh.HH_OK
        assert torch.equal(torch.cat(parts), whole)
        assert sum(b - a for a, b in ranges) == n
    finally:
        hh.hh_destroy(ctx)

"""Splitting one ragged batch over several GPUs (one process per GPU).

Messages are independent, so a batch shards into contiguous message ranges
with no exchange between ranks: rank r hashes messages [first_r, last_r)
into its own slice of the output, and the slices are gathered on the host
afterwards (or left where they are).  Ranges are balanced by bytes (the
prefix sums that the offsets already are), not by message count, since the
time per message grows with its length.

byte_balanced_ranges() is pure host arithmetic; hash_shard() runs one rank's
range through libhh; gather_to_rank0() collects the slices with
torch.distributed (any backend) after the hashing is done.
"""
from __future__ import annotations

import numpy as np
import torch

from paper_1612_06257_gb300 import hh

_FN = {64: hh.hh_hash64_batch, 128: hh.hh_hash128_batch, 256: hh.hh_hash256_batch}


def byte_balanced_ranges(offsets, world: int) -> list[tuple[int, int]]:
    """Contiguous message ranges [first, last) for ranks 0..world-1 covering
    0..n-1 in order.  Rank r's range starts at the first message whose start
    is at or past r/world of the payload, so every range holds close to an
    equal share of the bytes (within one message's length).  Ranges may be
    empty (more ranks than messages, or one message holding most bytes)."""
    if world < 1:
        raise ValueError("world must be at least 1")
    off = np.asarray(offsets.cpu() if isinstance(offsets, torch.Tensor) else offsets,
                     dtype=np.int64)
    if off.ndim != 1 or off.shape[0] < 1:
        raise ValueError("offsets must be a 1-D array of n + 1 entries")
    if np.any(np.diff(off) < 0):
        raise ValueError("offsets decrease")
    n = off.shape[0] - 1
    total = int(off[-1] - off[0])
    starts = off[:-1] - off[0]
    cuts = [0]
    for r in range(1, world):
        target = (total * r) // world
        cut = int(np.searchsorted(starts, target, side="left")) if total else (n * r) // world
        cuts.append(max(cuts[-1], min(cut, n)))
    cuts.append(n)
    return [(cuts[r], cuts[r + 1]) for r in range(world)]


def hash_shard(ctx, bits: int, keys, key_mode: int, data, offsets, rank: int, world: int,
               ranges=None, out=None, stream=None):
    """Hash this rank's range of the batch (all tensors on the rank's GPU;
    offsets are absolute positions in `data`).  Returns (first, last, out)
    with out holding (last - first) * bits / 64 words."""
    first, last = (ranges or byte_balanced_ranges(offsets, world))[rank]
    words = bits // 64
    if out is None:
        out = torch.empty(max(last - first, 0) * words, dtype=torch.int64, device=data.device)
    if last > first:
        k = keys[first:last] if key_mode == hh.HH_KEY_PER_MESSAGE else keys
        _FN[bits](ctx, k, key_mode, data, offsets[first:last + 1], last - first, out=out,
                  stream=stream)
    return first, last, out


def gather_to_rank0(local: torch.Tensor, ranges, words: int, group=None):
    """Collect every rank's slice (int64 [(last - first) * words], on the host
    or the device the backend needs) into one int64 [n * words] tensor on
    rank 0, in message order; returns None on the other ranks."""
    import torch.distributed as dist
    rank = dist.get_rank(group)
    world = dist.get_world_size(group)
    longest = max(last - first for first, last in ranges) * words
    buf = torch.zeros(longest, dtype=torch.int64, device=local.device)
    buf[:local.numel()] = local
    parts = [torch.zeros_like(buf) for _ in range(world)] if rank == 0 else None
    dist.gather(buf, parts, dst=0, group=group)
    if rank != 0:
        return None
    n = ranges[-1][1]
    out = torch.empty(n * words, dtype=torch.int64, device=local.device)
    for r, (first, last) in enumerate(ranges):
        out[first * words:last * words] = parts[r][:(last - first) * words]
    return out

"""Shared test helpers: run the CPU oracle on a workload (or a sample of it)."""
from __future__ import annotations

import concurrent.futures
import os

import numpy as np
import torch

import oracle


def host_inputs(w, indices=None):
    """(keys u64, per_message, data u8, offsets i64) on the host for the oracle.

    With `indices`, only those messages are gathered (bytes copied message by
    message from the device buffer), renumbered 0..len(indices)-1.
    """
    offsets = w.offsets_or_stride()
    if indices is None:
        keys = w.keys.cpu().numpy().view(np.uint64)
        return keys, w.per_message_keys, w.data.cpu().numpy(), offsets.cpu().numpy()
    idx = torch.as_tensor(indices, dtype=torch.int64, device=offsets.device)
    starts = offsets[idx]
    lengths = offsets[idx + 1] - starts
    new_off = torch.zeros(idx.numel() + 1, dtype=torch.int64, device=offsets.device)
    torch.cumsum(lengths, 0, out=new_off[1:])
    total = int(new_off[-1].item())
    if total:
        pos = torch.arange(total, dtype=torch.int64, device=offsets.device)
        owner = torch.searchsorted(new_off[1:], pos, right=True)
        src = starts[owner] + (pos - new_off[owner])
        data = w.data[src].cpu().numpy()
    else:
        data = np.zeros(0, dtype=np.uint8)
    if w.per_message_keys:
        keys = w.keys[idx].cpu().numpy().view(np.uint64)
    else:
        keys = w.keys.cpu().numpy().view(np.uint64)
    return keys, w.per_message_keys, data, new_off.cpu().numpy()


def oracle_hashes(w, bits: int, indices=None, threads: int | None = None) -> np.ndarray:
    """Oracle hashes [n_or_sample, bits // 64] as uint64."""
    keys, per_msg, data, offsets = host_inputs(w, indices)
    n = offsets.shape[0] - 1
    words = bits // 64
    out = np.zeros((n, words), dtype=np.uint64)
    threads = threads or min(16, os.cpu_count() or 1)
    step = max(1, (n + threads - 1) // threads)

    def run(first):
        last = min(n, first + step)
        oracle.hash_batch(keys, per_msg, data, offsets, bits, first, last, out[first:last])

    with concurrent.futures.ThreadPoolExecutor(max_workers=threads) as ex:
        list(ex.map(run, range(0, n, step)))
    return out


def as_u64(t: torch.Tensor, words: int) -> np.ndarray:
    return t.cpu().numpy().view(np.uint64).reshape(-1, words)


def oracle_segments(key_table, key_index, data, starts, lengths, bits: int) -> np.ndarray:
    """Oracle hashes of segments (host numpy arrays): message i is
    data[starts[i]:starts[i]+lengths[i]] keyed by key_table[key_index[i]]."""
    n = starts.shape[0]
    offs = np.zeros(n + 1, dtype=np.int64)
    offs[1:] = np.cumsum(lengths)
    buf = np.zeros(int(offs[-1]), dtype=np.uint8)
    for i in range(n):
        buf[offs[i]:offs[i + 1]] = data[starts[i]:starts[i] + lengths[i]]
    rows = np.zeros(n, dtype=np.int64) if key_index is None else key_index.astype(np.int64)
    keys = np.ascontiguousarray(key_table.view(np.uint64).reshape(-1, 4)[rows])
    out = np.zeros((n, bits // 64), dtype=np.uint64)
    oracle.hash_batch(keys, True, buf, offs, bits, 0, n, out)
    return out

"""Seeded synthetic HighwayHash batches shaped like the paper's workloads.

The paper measures 1 KiB messages (Section 5, Table 1), argues for short
RPC-sized packets (Section 1) and names file checksums as a use (Section 7).
The batches below follow those shapes with uniform random bytes from a
seeded torch.Generator on the target device.  This module holds none of the
hash's arithmetic; it only makes inputs, and both the CUDA path and the CPU
checker read the same tensors.

Workloads:
  serving      requests of 1..4096 messages, each a segment of a device pool:
               70% of lengths uniform in [0, 64], 25% exactly 1024, 5%
               log-uniform in [1 MiB, 64 MiB] (file-like buffers); a random
               256-bit key per request.
  fixed        n messages of exactly `length` bytes, contiguous, one key.
  ragged       lengths floor(exp(U(0, ln 65537))) - 1 in [0, 65536] (log-uniform),
               then forced to residue i mod 32 so every length mod 32 occurs;
               per-message random 256-bit keys; concatenated bytes + offsets.
  short        lengths uniform in [0, max_len]; 10% of messages all-zero
               bytes, the rest uniform; one key.
"""
from __future__ import annotations

import dataclasses
import math

import torch


@dataclasses.dataclass
class Workload:
    name: str
    data: torch.Tensor              # uint8 [total]
    offsets: torch.Tensor | None    # int64 [n + 1], or None for the fixed-length form
    fixed_len: int | None
    keys: torch.Tensor              # int64 [4] (shared) or [n, 4] (per message)
    per_message_keys: bool
    n: int

    @property
    def total_bytes(self) -> int:
        return int(self.data.numel())

    @property
    def key_mode(self) -> int:
        return 1 if self.per_message_keys else 0

    def offsets_or_stride(self) -> torch.Tensor:
        """Offsets tensor; built from the stride for the fixed-length form."""
        if self.offsets is not None:
            return self.offsets
        return torch.arange(self.n + 1, dtype=torch.int64, device=self.data.device) * self.fixed_len


def generator(seed: int, device) -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return g


def random_u64(shape, g: torch.Generator, device) -> torch.Tensor:
    """Uniform 64-bit words (as int64 bit patterns) from two 32-bit draws."""
    hi = torch.randint(0, 1 << 32, shape, generator=g, device=device, dtype=torch.int64)
    lo = torch.randint(0, 1 << 32, shape, generator=g, device=device, dtype=torch.int64)
    return (hi << 32) | lo


def random_bytes(total: int, g: torch.Generator, device, chunk: int = 1 << 30) -> torch.Tensor:
    data = torch.empty(total, dtype=torch.uint8, device=device)
    for s in range(0, total, chunk):
        data[s:s + chunk].random_(0, 256, generator=g)
    return data


def fixed(n: int, length: int, seed: int, device, per_message_keys: bool = False) -> Workload:
    g = generator(seed, device)
    keys = random_u64((n, 4) if per_message_keys else (4,), g, device)
    data = random_bytes(n * length, g, device)
    return Workload("fixed", data, None, length, keys, per_message_keys, n)


def offsets_from_lengths(lengths: torch.Tensor) -> torch.Tensor:
    off = torch.zeros(lengths.numel() + 1, dtype=torch.int64, device=lengths.device)
    torch.cumsum(lengths, 0, out=off[1:])
    return off


def loguniform_lengths(n: int, max_len: int, g: torch.Generator, device) -> torch.Tensor:
    u = torch.rand(n, dtype=torch.float64, generator=g, device=device)
    lengths = torch.floor(torch.exp(u * math.log(max_len + 1))).to(torch.int64) - 1
    lengths = lengths.clamp_(0, max_len)
    residue = torch.arange(n, dtype=torch.int64, device=device) % 32
    lengths = lengths - lengths % 32 + residue
    return lengths.clamp_(0, max_len)


def ragged(n: int, seed: int, device, max_len: int = 65536,
           per_message_keys: bool = True) -> Workload:
    g = generator(seed, device)
    lengths = loguniform_lengths(n, max_len, g, device)
    offsets = offsets_from_lengths(lengths)
    keys = random_u64((n, 4) if per_message_keys else (4,), g, device)
    data = random_bytes(int(offsets[-1].item()), g, device)
    return Workload("ragged", data, offsets, None, keys, per_message_keys, n)


def short(n: int, seed: int, device, max_len: int = 64, zero_fraction: float = 0.1,
          per_message_keys: bool = False, chunk: int = 1 << 22) -> Workload:
    g = generator(seed, device)
    lengths = torch.randint(0, max_len + 1, (n,), generator=g, device=device, dtype=torch.int64)
    zero = torch.rand(n, generator=g, device=device) < zero_fraction
    offsets = offsets_from_lengths(lengths)
    keys = random_u64((n, 4) if per_message_keys else (4,), g, device)
    data = random_bytes(int(offsets[-1].item()), g, device)
    # Zero the bytes of the all-zero messages, a chunk of messages at a time.
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        keep = (~zero[s:e]).to(torch.uint8)
        mask = torch.repeat_interleave(keep, lengths[s:e])
        a, b = int(offsets[s].item()), int(offsets[e].item())
        data[a:b] *= mask
    return Workload("short", data, offsets, None, keys, per_message_keys, n)


def from_lengths(lengths, seed: int, device, per_message_keys: bool = True,
                 zero_fraction: float = 0.0) -> Workload:
    """Explicit lengths (a list or int64 tensor), random bytes and keys."""
    g = generator(seed, device)
    lengths = torch.as_tensor(lengths, dtype=torch.int64).to(device)
    n = lengths.numel()
    offsets = offsets_from_lengths(lengths)
    keys = random_u64((n, 4) if per_message_keys else (4,), g, device)
    data = random_bytes(int(offsets[-1].item()), g, device)
    if zero_fraction > 0:
        zero = torch.rand(n, generator=g, device=device) < zero_fraction
        mask = torch.repeat_interleave((~zero).to(torch.uint8), lengths)
        data *= mask
    return Workload("lengths", data, offsets, None, keys, per_message_keys, n)


def serving_requests(count: int, pool_bytes: int, seed: int, max_messages: int = 4096,
                     short_max: int = 64, kib: int = 1024, huge_min: int = 1 << 20,
                     huge_max: int = 64 << 20, mix=(0.70, 0.25, 0.05)):
    """Host-side request descriptors for the serving workload.

    Returns a list of (key uint64[4], starts int64[m], lengths int64[m]) with
    every segment inside [0, pool_bytes).  Start positions are uniform over
    the pool, so requests read unrelated parts of it.
    """
    import numpy as np
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        m = int(rng.integers(1, max_messages + 1))
        kind = rng.choice(3, size=m, p=list(mix))
        lengths = np.empty(m, dtype=np.int64)
        n0, n1, n2 = (kind == 0).sum(), (kind == 1).sum(), (kind == 2).sum()
        lengths[kind == 0] = rng.integers(0, short_max + 1, size=n0)
        lengths[kind == 1] = kib
        lengths[kind == 2] = np.floor(np.exp(rng.uniform(np.log(huge_min), np.log(huge_max),
                                                         size=n2))).astype(np.int64)
        lengths = np.minimum(lengths, pool_bytes)
        starts = (rng.random(m) * (pool_bytes - lengths + 1)).astype(np.int64)
        key = rng.integers(0, 2**64, size=4, dtype=np.uint64)
        out.append((key, starts, lengths))
    return out

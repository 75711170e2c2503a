"""A small, self-contained hash launch to run under a profiler.

    python -m paper_1612_06257_gb300.profile_case --kind fixed --n 262144 --length 1024

builds one seeded batch on cuda:0 and hashes it `--reps` times through the C
ABI (the first launch warms up; profile with `-s 1 -c 1` to capture the
second).  Kinds: fixed (hh_hash_fixed), ragged (log-uniform lengths,
per-message keys), short (0..64-byte messages), long (n messages of
`--length` bytes through the offsets form: solo or pair tiles from 128 KiB),
offsets (the same with one key: the short kernel counts the lengths, the
warp-tile kernel hashes), siptree (n messages of `--length` bytes,
SipTreeHash through hh_siptree_batch; --bits 13 for SipTreeHash13) and prng
(n counters of counter mode through hh_prng_fill, --bits of output each).
"""
import argparse

import torch

from paper_1612_06257_gb300 import hh, workloads


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--kind",
                   choices=["fixed", "ragged", "short", "long", "offsets", "siptree", "prng"],
                   default="fixed")
    p.add_argument("--n", type=int, default=1 << 18)
    p.add_argument("--length", type=int, default=1024)
    p.add_argument("--bits", type=int, default=64)
    p.add_argument("--reps", type=int, default=2)
    p.add_argument("--kernel", type=int, default=hh.HH_KERNEL_AUTO)
    a = p.parse_args()
    ctx = hh.hh_init(0)
    hh.hh_set_kernel(ctx, a.kernel)
    dev = "cuda:0"
    if a.kind == "prng":
        # n counters of counter mode (8-byte little-endian counters), a.bits
        # of output each
        key = workloads.random_u64((4,), workloads.generator(1, dev), dev)
        out = torch.empty(a.n * a.bits // 64, dtype=torch.int64, device=dev)
        for _ in range(a.reps):
            hh.hh_prng_fill(ctx, a.bits, key, 12345, a.n, out=out)
        torch.cuda.synchronize()
        print("ok", a.kind, a.n, a.bits)
        return
    if a.kind == "fixed":
        w = workloads.fixed(a.n, a.length, seed=1, device=dev)
    elif a.kind == "ragged":
        w = workloads.ragged(a.n, seed=1, device=dev)
    elif a.kind in ("long", "offsets", "siptree"):
        w = workloads.from_lengths([a.length] * a.n, seed=1, device=dev,
                                   per_message_keys=a.kind == "long")
    else:
        w = workloads.short(a.n, seed=1, device=dev)
    hh.hh_reserve(ctx, w.n)  # the length sort's scratch for this batch
    words = 1 if a.kind == "siptree" else a.bits // 64
    out = torch.empty(w.n * words, dtype=torch.int64, device=dev)
    for _ in range(a.reps):
        if a.kind == "siptree":
            variant = hh.HH_SIPTREE13 if a.bits == 13 else hh.HH_SIPTREE
            hh.hh_siptree_batch(ctx, variant, w.keys, w.key_mode, w.data, w.offsets, out=out)
        elif a.kind == "fixed":
            hh.hh_hash_fixed(ctx, a.bits, w.keys, w.key_mode, w.data, a.length, w.n, out=out)
        else:
            fn = {64: hh.hh_hash64_batch, 128: hh.hh_hash128_batch, 256: hh.hh_hash256_batch}
            fn[a.bits](ctx, w.keys, w.key_mode, w.data, w.offsets, out=out)
    status = hh.hh_get_device_error(ctx)
    if status != hh.HH_OK:
        raise SystemExit("device error: " + hh.hh_status_string(status))
    print("ok", a.kind, w.n, w.total_bytes)


if __name__ == "__main__":
    main()

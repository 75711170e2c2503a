"""Measurements of the other batch shapes (bench.py --workload NAME).

  small    4096 messages x 1024 B, one key: microseconds per batch with the
           inputs hot in L2 and with L2 flushed between batches.
  ragged   2^22 messages, lengths log-uniform in [0, 65536], per-message
           keys (about 25 GB): GB/s against the HBM peak.
  short    2^26 messages of 0..64 B (10% all zero), one key: hashes/s for
           64- and 128-bit output against the integer ceiling that the
           Update microbenchmark measures in the same run.
  serving  the request mix (70% <= 64 B, 25% 1 KiB, 5% 1-64 MiB buffers,
           1..4096 messages and one key per request) through the
           continuous-batching server: saturation GB/s, then p50/p99
           latency at Poisson arrival rates swept over 0.1-0.9 of it.
  prng     2^28 counter-mode 64-bit words (hh_prng_fill): words/s against
           the integer ceiling (5 Updates per word).
  siptree  SipTreeHash and SipTreeHash13 (Section 3) beside HighwayHash on
           2^20 x 1 KiB through the offsets form: GB/s of each.
  stats    the paper's statistical studies on the GPU: toggle bias of all
           2^24 three-byte inputs after 2, 3 and 4 finalisation rounds, and
           the avalanche test for sizes 4-32 (49 samples, 1M iterations).

Every input is synthetic and seeded; each workload prints one JSON line.
"""
from __future__ import annotations

import json
import os
import time

import numpy as np
import torch

from paper_1612_06257_gb300 import build, hh, serve, stats, workloads

L2_FLUSH_BYTES = 512 << 20


def _peak_hbm():
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    try:
        with open(os.path.join(root, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def _max_sm_clock_hz():
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    try:
        with open(os.path.join(root, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["sm_max_mhz"]) * 1e6
    except (OSError, KeyError, ValueError):
        return 2070e6  # GB300 maximum SM clock


def _alu_peak(dev):
    """ALU-pipe lane-instructions per second: 16 lanes per clock in each of
    the 4 sub-partitions of every SM, at the maximum SM clock."""
    props = torch.cuda.get_device_properties(dev)
    return 16 * 4 * props.multi_processor_count * _max_sm_clock_hz()


def _alu_count(kernel, source, path=None):
    """ALU lane-instructions per output of `kernel`: ncu's
    sm__inst_executed_pipe_alu on the kernel's sources, as committed in
    profiles/alu_counts.json; None when there is no count or the sources
    (translation unit `source` and its csrc headers) changed since."""
    if path is None:
        root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
        path = os.path.join(root, "profiles", "alu_counts.json")
    try:
        with open(path) as f:
            rec = json.load(f)[kernel]
    except (OSError, KeyError, ValueError):
        return None
    if rec.get("source_digest") != build.source_digest(source):
        return None
    return float(rec["alu_lane_instructions_per_output"])


def _alu_roofline(dev, kernel, unit, source, per_s):
    """Roofline of an integer-ALU-bound kernel: `per_s` outputs per second
    against the ALU pipe's lane-instructions per second divided by the ALU
    lane-instructions one output costs (_alu_count); None without a count
    for the current sources."""
    per_output = _alu_count(kernel, source)
    if per_output is None:
        return None
    peak = _alu_peak(dev) / per_output
    return {"bound": "alu", "achieved": round(per_s, 1), "peak": round(peak, 1), "unit": unit,
            "frac": round(per_s / peak, 4), "alu_lane_instructions_per_output": per_output,
            "kernel": kernel,
            "peak_source": "derived: 16 ALU lanes/clk per SM sub-partition x 4 x SMs x max SM "
                           "clock / ALU lane-instructions per output (ncu count, "
                           "profiles/alu_counts.json)"}


def _time(fn, reps, flush=None):
    fn()
    torch.cuda.synchronize()
    times = []
    for _ in range(reps):
        if flush is not None:
            flush()
        e0, e1 = torch.cuda.Event(True), torch.cuda.Event(True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    return float(np.median(times)), times


def _naive_ms(ctx, fn, reps, flush=None):
    """Median ms of `fn` with the naive kernel (one thread per message,
    direct global loads): the speedup baseline on the same GPU."""
    hh.hh_set_kernel(ctx, hh.HH_KERNEL_NAIVE)
    try:
        ms, _ = _time(fn, reps, flush)
    finally:
        hh.hh_set_kernel(ctx, hh.HH_KERNEL_AUTO)
    return ms


def small(ctx, dev):
    w = workloads.fixed(4096, 1024, seed=1, device=dev)
    out = torch.empty(w.n, dtype=torch.int64, device=dev)
    junk = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    fn = lambda: hh.hh_hash_fixed(ctx, 64, w.keys, 0, w.data, 1024, w.n, out=out)  # noqa: E731
    # Hot: 200 back-to-back launches (inputs stay in L2); cold: one launch
    # after writing a 512 MiB buffer, each timed alone.
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(True), torch.cuda.Event(True)
    e0.record()
    for _ in range(200):
        fn()
    e1.record()
    torch.cuda.synchronize()
    hot = e0.elapsed_time(e1) / 200
    cold, _ = _time(fn, 50, flush=lambda: junk.fill_(1))
    naive_cold = _naive_ms(ctx, fn, 50, flush=lambda: junk.fill_(1))
    # The same launch replayed 20 times from a CUDA graph: the device-side
    # latency without the host's per-call cost (the Python call alone takes
    # a few microseconds).
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(side):
        fg = lambda: hh.hh_hash_fixed(ctx, 64, w.keys, 0, w.data, 1024, w.n, out=out,  # noqa: E731
                                      stream=side)
        fg()
        torch.cuda.synchronize()
        with torch.cuda.graph(graph, stream=side):
            for _ in range(20):
                fg()
    torch.cuda.current_stream().wait_stream(side)
    graph.replay()
    torch.cuda.synchronize()
    g_ms, _ = _time(graph.replay, 10)
    graph_us = g_ms / 20 * 1e3
    return {"workload": "4096 x 1024 B, one key, 64-bit (fixed-length batch)",
            "us_per_batch_hot_l2": round(hot * 1e3, 2), "us_per_batch_cold_l2": round(cold * 1e3, 2),
            "us_per_batch_graph_replay": round(graph_us, 2),
            "naive_us_per_batch_cold_l2": round(naive_cold * 1e3, 2),
            "speedup_vs_naive_cold": round(naive_cold / cold, 2),
            "gbps_hot": round(w.total_bytes / hot / 1e6, 1),
            "gbps_cold": round(w.total_bytes / cold / 1e6, 1),
            "note": "4 MiB fits L2; 4096 messages, two threads each, in 32-row tiles on 128 of 152 SMs: a latency regime bound by each thread's Update chain"}


def ragged(ctx, dev, naive_reps=3):
    w = workloads.ragged(1 << 22, seed=2, device=dev)
    out = torch.empty(w.n, dtype=torch.int64, device=dev)
    fn = lambda: hh.hh_hash64_batch(ctx, w.keys, 1, w.data, w.offsets, out=out)  # noqa: E731
    ms, _ = _time(fn, 10)
    launches = hh.hh_last_launch_count(ctx)
    naive = _naive_ms(ctx, fn, naive_reps)
    alg = w.total_bytes + 8 * (w.n + 1) + 32 * w.n + 8 * w.n
    peak, kind = _peak_hbm()
    return {"workload": "2^22 messages, log-uniform lengths in [0, 65536] (every residue mod 32), "
                        "per-message keys, 64-bit", "bytes": w.total_bytes, "ms_per_batch": round(ms, 3),
            "gbps": round(w.total_bytes / ms / 1e6, 1), "hashes_per_s": round(w.n / ms * 1e3, 1),
            "roofline": {"bound": "hbm", "achieved": round(alg / ms / 1e6, 1), "peak": peak,
                         "unit": "GB/s", "frac": round(alg / ms / 1e6 / peak, 4),
                         "peak_source": kind, "algorithmic_bytes": alg,
                         "algorithmic_bytes_formula": "sum(len) + 8(n+1) offsets + 32n keys + 8n out",
                         "timing": "median of 10 launches, each between CUDA events; inputs "
                                   "(25 GB) larger than L2"},
            "launches_per_batch": launches,
            "naive_gbps": round(w.total_bytes / naive / 1e6, 1),
            "speedup_vs_naive": round(naive / ms, 2)}


def _update_ceiling(ctx, dev):
    """Updates per second of the integer-issue microbenchmark (no memory):
    the best of the whole-state variants 1 and 5."""
    threads, updates = 152 * 1024 * 4, 1024
    best = 0.0
    for variant in (1, 5):
        out = hh.hh_update_microbench(ctx, variant, updates, threads)
        ms, _ = _time(lambda: hh.hh_update_microbench(ctx, variant, updates, threads, out=out), 5)
        best = max(best, threads * updates / (ms / 1e3))
    return best


def short(ctx, dev):
    w = workloads.short(1 << 26, seed=3, device=dev)
    hh.hh_reserve(ctx, w.n)  # beyond the default sort scratch of 2^22 messages
    lengths = (w.offsets[1:] - w.offsets[:-1]).cpu().numpy()
    upd_per_hash = float(np.mean(lengths // 32 + (lengths % 32 != 0) + 4))
    ceiling = _update_ceiling(ctx, dev) / upd_per_hash
    res = {"workload": "2^26 messages of 0..64 B (10% all zero), one key",
           "updates_per_hash": round(upd_per_hash, 3),
           "integer_ceiling_hashes_per_s": round(ceiling, 1),
           "integer_ceiling": "Update microbenchmark (register state, no memory) measured in "
                              "this run, divided by the Updates per hash; whole Updates are "
                              "counted, although for 64- and 128-bit output the finalisation "
                              "work that feeds no stored lane is not computed"}
    for bits, fn in ((64, hh.hh_hash64_batch), (128, hh.hh_hash128_batch)):
        out = torch.empty(w.n * bits // 64, dtype=torch.int64, device=dev)
        ms, _ = _time(lambda: fn(ctx, w.keys, 0, w.data, w.offsets, out=out), 10)
        hps = w.n / (ms / 1e3)
        res["hashes_per_s_%d" % bits] = round(hps, 1)
        res["integer_frac_%d" % bits] = round(hps / ceiling, 4)
        res["launches_per_batch_%d" % bits] = hh.hh_last_launch_count(ctx)
        res["gbps_%d" % bits] = round(w.total_bytes / ms / 1e6, 1)
        res["alu_roofline_%d" % bits] = _alu_roofline(
            dev, "short_count_kernel<%d>" % (bits // 64), "hashes/s", "hh_ragged.cu", hps)
        if bits == 64:
            naive = _naive_ms(ctx, lambda: fn(ctx, w.keys, 0, w.data, w.offsets, out=out), 5)
            res["naive_hashes_per_s_64"] = round(w.n / (naive / 1e3), 1)
            res["speedup_vs_naive_64"] = round(naive / ms, 2)
    res["one_long_message"] = _short_with_one_long(ctx, w)
    del w
    # The same recipe with a key per message: the separate length count and
    # short_kernel (the words loaded directly, each message's key too).
    wk = workloads.short(1 << 26, seed=3, device=dev, per_message_keys=True)
    out = torch.empty(wk.n, dtype=torch.int64, device=dev)
    ms, _ = _time(lambda: hh.hh_hash64_batch(ctx, wk.keys, 1, wk.data, wk.offsets, out=out), 10)
    res["hashes_per_s_64_per_message_keys"] = round(wk.n / (ms / 1e3), 1)
    res["launches_per_batch_64_per_message_keys"] = hh.hh_last_launch_count(ctx)
    return res


def _short_with_one_long(ctx, w):
    """ms per 64-bit call of the same batch with one message made 65 bytes
    long (first, in the middle or last): the short kernel meets it when it
    gets there, and the warp-tile kernel then hashes the whole batch."""
    lengths = w.offsets[1:] - w.offsets[:-1]
    data = torch.cat([w.data, torch.zeros(128, dtype=torch.uint8, device=w.data.device)])
    out = torch.empty(w.n, dtype=torch.int64, device=w.data.device)
    res = {}
    for where, i in (("none", None), ("first", 0), ("middle", w.n // 2), ("last", w.n - 1)):
        ln = lengths.clone()
        if i is not None:
            ln[i] = 65
        off = torch.zeros_like(w.offsets)
        off[1:] = torch.cumsum(ln, 0)
        ms, _ = _time(lambda: hh.hh_hash64_batch(ctx, w.keys, 0, data, off, out=out), 5)
        res[where + "_ms"] = round(ms, 3)
    res["note"] = ("one-key batch of 2^26 messages of 0..64 B with one message of 65 B; "
                   "with the length count in a launch of its own every case took about 4.1 ms")
    return res


def serving(ctx, dev, requests=512, pool_gib=8, rates=(0.1, 0.3, 0.5, 0.7, 0.9)):
    pool = workloads.random_bytes(pool_gib << 30, workloads.generator(7, dev), dev)
    specs = workloads.serving_requests(requests, pool.numel(), seed=8)

    def fresh():
        return [serve.Request(key=k, starts=s, lengths=l, rid=i) for i, (k, s, l) in enumerate(specs)]

    server = serve.HashServer(pool, bits=64, slots=16, capacity=1 << 16, max_requests_per_batch=4,
                              max_bytes_in_flight=96 << 30, use_graphs=True)
    try:
        warm = fresh()[:4]
        for r in warm:
            server.submit(r)
        server.drain()
        sat = serve.run_poisson(server, fresh(), rate_per_s=1e9, seed=1)
        sat_rate = sat["requests"] / sat["wall_s"]
        sweep = []
        for f in rates:
            st = serve.run_poisson(server, fresh(), rate_per_s=f * sat_rate, seed=2)
            sweep.append({"load": f, "rate_per_s": round(st["rate_per_s"], 2),
                          "requests": st["requests"],
                          "p50_ms": round(st["p50_ms"], 2), "p99_ms": round(st["p99_ms"], 2),
                          "gbps": round(st["gbps"], 1)})
        errors = server.device_errors()
    finally:
        server.close()
    total = sum(int(l.sum()) for _, _, l in specs)
    return {"workload": "serving mix: %d requests (1-4096 messages; 70%% <= 64 B, 25%% 1 KiB, "
                        "5%% 1-64 MiB), per-request keys, 16 stream slots with CUDA graphs "
                        "(<= 4 requests per batch), 96 GiB in-flight cap" % requests,
            "bytes_per_pass": total,
            "saturation": {"gbps": round(sat["gbps"], 1), "requests_per_s": round(sat_rate, 2),
                           "requests": sat["requests"],
                           "p50_ms": round(sat["p50_ms"], 2), "p99_ms": round(sat["p99_ms"], 2)},
            "percentiles": "over every request of a load point (requests per point as listed)",
            "sweep": sweep, "device_errors": errors}


def siptree(ctx, dev, w=None):
    """SipTreeHash and SipTreeHash13 (Section 3) beside HighwayHash on one
    batch through the same offsets form (Table 1 compares them on one CPU
    core; here on one GB300): by default the benchmark's 2^20 x 1 KiB batch."""
    if w is None:
        w = workloads.fixed(1 << 20, 1024, seed=1000, device=dev)
    offsets = w.offsets_or_stride()
    out = torch.empty(w.n, dtype=torch.int64, device=dev)
    res = {"workload": "%d messages x %d B, one key, 64-bit, offsets form" % (w.n, w.fixed_len or 0)}
    fns = {"highwayhash": lambda: hh.hh_hash64_batch(ctx, w.keys, w.key_mode, w.data, offsets,
                                                      out=out),
           "siptree": lambda: hh.hh_siptree_batch(ctx, hh.HH_SIPTREE, w.keys, w.key_mode, w.data,
                                                  offsets, out=out),
           "siptree13": lambda: hh.hh_siptree_batch(ctx, hh.HH_SIPTREE13, w.keys, w.key_mode,
                                                    w.data, offsets, out=out)}
    for name, fn in fns.items():
        ms, _ = _time(fn, 10)
        res["%s_gbps" % name] = round(w.total_bytes / ms / 1e6, 1)
        res["%s_ms" % name] = round(ms, 4)
    # Integer-ALU roofline: the ALU pipe's lane-instructions per second over
    # the ALU lane-instructions one 1 KiB message costs, as ncu counts them on
    # the kernel's current sources (profiles/alu_counts.json; no roofline for
    # other lengths or once the sources have changed).  The hand count beside
    # it: a SipRound is 24 ALU instructions (4 64-bit adds, 4 rotations of two
    # funnel shifts, 4 64-bit xors; the 32-bit rotations are free) and a
    # compression adds 4 xors, so a message of P = L / 32 vectors takes
    # 4 P (24 c + 4) for the lanes, 4 (24 (c + d) + 4) for their last word and
    # finalisation, and (6 c + d) 24 + 28 for the fold; the compiler needs fewer.
    sm_hz = _max_sm_clock_hz()
    alu_peak = _alu_peak(dev)  # ALU lane-instructions per second
    length = w.fixed_len or int(w.total_bytes // max(1, w.n))
    vectors = (length + 31) // 32
    for name, kernel, (c, d) in (("siptree", "siptree_kernel<2,4>", (2, 4)),
                                 ("siptree13", "siptree_kernel<1,3>", (1, 3))):
        hand = 4 * vectors * (24 * c + 4) + 4 * (24 * (c + d) + 4) + (6 * c + d) * 24 + 28
        alu = _alu_count(kernel, "hh_siptree.cu") if length == 1024 else None
        if alu is None:
            res["%s_roofline" % name] = None
            continue
        ceiling = alu_peak / alu * length / 1e9  # GB/s of payload
        res["%s_roofline" % name] = {
            "bound": "alu", "achieved": res["%s_gbps" % name], "peak": round(ceiling, 1),
            "unit": "GB/s", "frac": round(res["%s_gbps" % name] / ceiling, 4),
            "alu_lane_instructions_per_message": alu, "alu_hand_count_per_message": hand,
            "sm_clock_hz": sm_hz, "kernel": kernel,
            "peak_source": "derived: 16 ALU lanes/clk per SM sub-partition x 4 x SMs x max SM "
                           "clock / ALU lane-instructions per message (ncu count, "
                           "profiles/alu_counts.json)"}
    res["highwayhash_over_siptree"] = round(res["highwayhash_gbps"] / res["siptree_gbps"], 2)
    res["highwayhash_over_siptree13"] = round(res["highwayhash_gbps"] / res["siptree13_gbps"], 2)
    # Table 1 at 1024 B (cycles per byte on one Haswell core): SipTreeHash
    # 0.57, SipTreeHash13 0.33, HighwayHash (AVX2) 0.24.
    res["paper_cpu_ratio_at_1k"] = {"highwayhash_over_siptree": round(0.57 / 0.24, 2),
                                    "highwayhash_over_siptree13": round(0.33 / 0.24, 2)}
    return res


def prng(ctx, dev):
    n = 1 << 28
    key = workloads.random_u64((4,), workloads.generator(9, dev), dev)
    out = torch.empty(n, dtype=torch.int64, device=dev)
    ms, _ = _time(lambda: hh.hh_prng_fill(ctx, 64, key, 12345, n, out=out), 10)
    wps = n / (ms / 1e3)
    return {"workload": "2^28 words, 64-bit, counter-mode (8-byte counters)",
            "ms": round(ms, 3), "words_per_s": round(wps, 1), "gbps_out": round(n * 8 / ms / 1e6, 1),
            "updates_per_word": 5,
            "alu_roofline": _alu_roofline(dev, "prng_kernel<1>", "words/s", "hh_stats.cu", wps),
            "note": "for 64-bit output the finalisation work that feeds no stored lane is not "
                    "computed, so a word costs fewer ALU instructions than five whole Updates "
                    "(the Update microbenchmark's rate / 5 is not a ceiling here)"}


def stats_study(ctx, dev):
    t0 = time.perf_counter()
    rounds = {}
    for r in (2, 3, 4):
        res = stats.round_bias(ctx, r)
        rounds[r] = {"mean_bias": res["mean_bias"], "max_bias": res["max_bias"]}
    t1 = time.perf_counter()
    av = stats.avalanche_study(ctx, iterations=1_000_000)
    t2 = time.perf_counter()
    return {"workload": "Section 4.3 round study (all 2^24 3-byte inputs, 24 x 64 bit pairs) and "
                        "Section 6 avalanche test (sizes 4-32, 49 samples, 1M iterations each)",
            "bias_definition": "|p - 1/2| per (input bit, output bit) pair",
            "round_bias": rounds, "round_study_s": round(t1 - t0, 2),
            "avalanche_median_worst_bias": av["median_worst_bias"], "avalanche_pass_1pct": av["pass"],
            "avalanche_s": round(t2 - t1, 2)}


WORKLOADS = {"small": small, "ragged": ragged, "short": short, "serving": serving, "prng": prng,
             "stats": stats_study, "siptree": siptree}


def run(name: str) -> dict:
    from paper_1612_06257_gb300 import build
    build.build()
    dev = "cuda:0"
    ctx = hh.hh_init(0)
    try:
        res = WORKLOADS[name](ctx, dev)
    finally:
        hh.hh_destroy(ctx)
    res["name"] = name
    res["data"] = "synthetic (seeded, generated on device)"
    return res

"""Continuous-batching HighwayHash request server.

Requests carry a 256-bit key and a list of messages, each a segment of one
device byte pool (the data a server would already hold in device memory).
The server keeps up to `slots` batches in flight, one per CUDA stream.  When
a slot is free it admits waiting requests in arrival order, as long as the
batch stays within the slot's message capacity and the payload in flight
stays within `max_bytes_in_flight`.  A batch is one hh_hash_segments launch:
its descriptor (segment starts and lengths, and per message the row of the
batch's key table) is copied to the device, hashed, and the hashes copied
back.  With `use_graphs` each slot replays a CUDA graph of that sequence,
captured once with a fixed capacity; the live message count travels in the
descriptor.  Requests that arrive while batches run join the next free
slot, so their work overlaps the running batches on the device.  Latency is
measured per request from arrival to the moment its hashes are on the host.

The keys and the batch descriptors live on the device; every hash step runs
in libhh's kernels.

Long messages (128 KiB and more) get a warp each while few of them run; with
many batches in flight that is limited to 2 per SM (SERVING_SOLO_PER_SM),
which gave the lowest p50 and p99 on the serving mix on GB300 (107 ms / 110-
155 ms against 142 ms / 148-162 ms with two threads per message throughout)
at the same saturation throughput.  A tuning table (`tune_path`) overrides it.
"""
from __future__ import annotations

import collections
import dataclasses
import time

import numpy as np
import torch

from paper_1612_06257_gb300 import hh

SERVING_SOLO_PER_SM = 2


@dataclasses.dataclass
class Request:
    key: np.ndarray                 # uint64 [4]
    starts: np.ndarray              # int64 [m], byte offsets into the pool
    lengths: np.ndarray             # int64 [m]
    rid: int = 0
    arrival: float = 0.0            # time.perf_counter() at arrival
    admitted: float | None = None
    done: float | None = None
    result: np.ndarray | None = None  # uint64 [m, bits // 64]

    @property
    def messages(self) -> int:
        return int(self.starts.shape[0])

    @property
    def payload(self) -> int:
        return int(self.lengths.sum())

    @property
    def latency(self) -> float:
        return self.done - self.arrival


class TooLarge(ValueError):
    """A request that no slot or memory budget could ever admit."""


def plan_batch(queue, capacity: int, max_requests: int, bytes_free: int) -> int:
    """How many requests from the head of `queue` (arrival order) one batch
    admits: all of them while the batch stays within `capacity` messages and
    `max_requests` requests and their payload within `bytes_free`."""
    count, msgs, nbytes = 0, 0, 0
    for req in queue:
        if count == max_requests or msgs + req.messages > capacity or \
                nbytes + req.payload > bytes_free:
            break
        count += 1
        msgs += req.messages
        nbytes += req.payload
    return count


class _Slot:
    """One stream, one hh context, fixed descriptor buffers, maybe a graph."""

    def __init__(self, pool, bits, capacity, max_requests, device, use_graphs, tune_path=None):
        self.words = bits // 64
        self.bits = bits
        self.capacity = capacity
        self.max_requests = max_requests
        dev = torch.device("cuda", device)
        self.ctx = hh.hh_init(device, tune_path)
        if tune_path is None:
            hh.hh_set_tune_param(self.ctx, "solo_per_sm", SERVING_SOLO_PER_SM)
        hh.hh_reserve(self.ctx, capacity)
        self.stream = torch.cuda.Stream(device=dev)
        self.pool = pool
        pin = dict(pin_memory=True)
        self.h_starts = torch.zeros(capacity, dtype=torch.int64, **pin)
        self.h_lengths = torch.zeros(capacity, dtype=torch.int64, **pin)
        self.h_kidx = torch.zeros(capacity, dtype=torch.int32, **pin)
        self.h_keys = torch.zeros(max_requests, 4, dtype=torch.int64, **pin)
        self.h_n = torch.zeros(1, dtype=torch.int64, **pin)
        self.h_out = torch.zeros(capacity * self.words, dtype=torch.int64, **pin)
        self.d_starts = torch.zeros(capacity, dtype=torch.int64, device=dev)
        self.d_lengths = torch.zeros(capacity, dtype=torch.int64, device=dev)
        self.d_kidx = torch.zeros(capacity, dtype=torch.int32, device=dev)
        self.d_keys = torch.zeros(max_requests, 4, dtype=torch.int64, device=dev)
        self.d_n = torch.zeros(1, dtype=torch.int64, device=dev)
        self.d_out = torch.zeros(capacity * self.words, dtype=torch.int64, device=dev)
        self.event = torch.cuda.Event()
        self.requests: list[Request] = []
        self.graph = None
        if use_graphs:
            # Warm up outside the capture (first-use attribute and occupancy
            # queries), then capture the whole batch sequence.
            with torch.cuda.stream(self.stream):
                self._enqueue()
            self.stream.synchronize()
            self.graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(self.graph, stream=self.stream):
                self._enqueue()
            self.stream.synchronize()

    def _enqueue(self):
        """Copy the descriptor in, hash, copy the hashes out (current stream)."""
        s = torch.cuda.current_stream()
        self.d_n.copy_(self.h_n, non_blocking=True)
        self.d_starts.copy_(self.h_starts, non_blocking=True)
        self.d_lengths.copy_(self.h_lengths, non_blocking=True)
        self.d_kidx.copy_(self.h_kidx, non_blocking=True)
        self.d_keys.copy_(self.h_keys, non_blocking=True)
        hh.hh_hash_segments(self.ctx, self.bits, self.d_keys, self.d_kidx, self.pool,
                            self.d_starts, self.d_lengths, out=self.d_out, stream=s,
                            n_device=self.d_n)
        self.h_out.copy_(self.d_out, non_blocking=True)

    def launch(self, reqs: list[Request]):
        pos = 0
        for r, req in enumerate(reqs):
            m = req.messages
            self.h_starts[pos:pos + m] = torch.from_numpy(req.starts)
            self.h_lengths[pos:pos + m] = torch.from_numpy(req.lengths)
            self.h_kidx[pos:pos + m] = r
            self.h_keys[r] = torch.from_numpy(req.key.view(np.int64))
            pos += m
        self.h_n[0] = pos
        self.requests = reqs
        with torch.cuda.stream(self.stream):
            if self.graph is not None:
                self.graph.replay()
            else:
                self._enqueue()
            self.event.record(self.stream)

    def busy(self) -> bool:
        return bool(self.requests)

    def poll(self) -> list[Request]:
        """Finished requests with their results, or [] while still running."""
        if not self.requests or not self.event.query():
            return []
        out = self.h_out.numpy().view(np.uint64)
        now = time.perf_counter()
        pos = 0
        done = self.requests
        for req in done:
            m = req.messages
            req.result = out[pos * self.words:(pos + m) * self.words].reshape(m, self.words).copy()
            req.done = now
            pos += m
        self.requests = []
        return done

    def device_error(self) -> int:
        return hh.hh_get_device_error(self.ctx, self.stream)

    def close(self):
        self.graph = None
        hh.hh_destroy(self.ctx)


class HashServer:
    """Continuous batching over `slots` streams.  submit() queues requests;
    step() polls finished batches and admits waiting requests into free
    slots; drain() runs until everything submitted has finished."""

    def __init__(self, pool: torch.Tensor, *, bits: int = 64, slots: int = 4,
                 capacity: int = 1 << 16, max_requests_per_batch: int = 256,
                 max_bytes_in_flight: int = 8 << 30, use_graphs: bool = True,
                 tune_path: str | None = None):
        if pool.dtype != torch.uint8 or not pool.is_cuda:
            raise ValueError("pool must be a CUDA uint8 tensor")
        self.pool = pool
        self.bits = bits
        self.capacity = capacity
        self.max_requests = max_requests_per_batch
        self.max_bytes = max_bytes_in_flight
        device = pool.device.index
        self.slots = [_Slot(pool, bits, capacity, max_requests_per_batch, device, use_graphs,
                            tune_path) for _ in range(slots)]
        self.queue: collections.deque[Request] = collections.deque()
        self.in_flight_bytes = 0
        self.peak_in_flight_bytes = 0
        self.finished: list[Request] = []

    def submit(self, req: Request, now: float | None = None) -> None:
        if req.messages > self.capacity or req.payload > self.max_bytes:
            raise TooLarge("request %d can never be admitted (messages %d, bytes %d)"
                           % (req.rid, req.messages, req.payload))
        if req.messages and (req.starts.min() < 0 or
                             (req.starts + req.lengths).max() > self.pool.numel()):
            raise ValueError("request %d has a segment outside the pool" % req.rid)
        req.arrival = time.perf_counter() if now is None else now
        self.queue.append(req)

    def _admit(self, slot: _Slot) -> bool:
        count = plan_batch(self.queue, self.capacity, self.max_requests,
                           self.max_bytes - self.in_flight_bytes)
        if count == 0:
            return False
        batch = [self.queue.popleft() for _ in range(count)]
        nbytes = sum(r.payload for r in batch)
        now = time.perf_counter()
        for req in batch:
            req.admitted = now
        self.in_flight_bytes += nbytes
        self.peak_in_flight_bytes = max(self.peak_in_flight_bytes, self.in_flight_bytes)
        slot.launch(batch)
        return True

    def step(self) -> int:
        """Poll every slot, then fill free slots.  Returns requests finished."""
        n_done = 0
        for slot in self.slots:
            done = slot.poll()
            if done:
                self.in_flight_bytes -= sum(r.payload for r in done)
                self.finished.extend(done)
                n_done += len(done)
        for slot in self.slots:
            if not slot.busy() and self.queue:
                self._admit(slot)
        return n_done

    def idle(self) -> bool:
        return not self.queue and not any(s.busy() for s in self.slots)

    def drain(self) -> None:
        while not self.idle():
            if self.step() == 0:
                time.sleep(20e-6)

    def device_errors(self) -> list[int]:
        return [s.device_error() for s in self.slots]

    def close(self) -> None:
        for s in self.slots:
            s.close()


def run_poisson(server: HashServer, requests: list[Request], rate_per_s: float,
                seed: int = 0) -> dict:
    """Submit `requests` at Poisson arrival times (mean rate `rate_per_s`)
    while the server runs; returns latency and throughput figures."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_per_s, size=len(requests))
    t0 = time.perf_counter()
    due = t0 + np.cumsum(gaps)
    i = 0
    while i < len(requests) or not server.idle():
        now = time.perf_counter()
        while i < len(requests) and due[i] <= now:
            server.submit(requests[i], now=float(due[i]))
            i += 1
        if server.step() == 0 and i < len(requests):
            wait = due[i] - time.perf_counter()
            if wait > 0:
                time.sleep(min(wait, 200e-6))
    t1 = time.perf_counter()
    lat = np.array([r.latency for r in requests])
    total = sum(r.payload for r in requests)
    first = min(r.arrival for r in requests)
    last = max(r.done for r in requests)
    return {"requests": len(requests), "rate_per_s": rate_per_s,
            "p50_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "mean_ms": float(lat.mean() * 1e3),
            "gbps": total / (last - first) / 1e9, "bytes": total, "wall_s": t1 - t0,
            "messages": sum(r.messages for r in requests)}

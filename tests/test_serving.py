"""The continuous-batching server on the GPU.

Requests from the serving mixture (short packets, 1 KiB messages and larger
file-like buffers, each request with its own key) arrive at Poisson times
while earlier batches run.  Each request's hashes must be identical, word
for word, whether it ran in that mix or alone, and must match the CPU
oracle; admission must respect the memory cap.
"""
import numpy as np
import pytest
import torch

from paper_1612_06257_gb300 import serve, workloads
from tests.helpers import oracle_segments

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
POOL_BYTES = 1 << 28


@pytest.fixture(scope="module")
def pool():
    from paper_1612_06257_gb300 import build
    build.build()
    return workloads.random_bytes(POOL_BYTES, workloads.generator(5, DEV), DEV)


def _requests(seed, count=30):
    specs = workloads.serving_requests(count, POOL_BYTES, seed, max_messages=600,
                                       huge_min=1 << 16, huge_max=1 << 21)
    return [serve.Request(key=k, starts=s, lengths=l, rid=i) for i, (k, s, l) in enumerate(specs)]


def _clone(reqs):
    return [serve.Request(key=r.key, starts=r.starts, lengths=r.lengths, rid=r.rid) for r in reqs]


@pytest.mark.parametrize("use_graphs", [True, False])
def test_results_alone_equal_results_in_the_mix(pool, use_graphs):
    reqs = _requests(11)
    cap = 48 << 20
    server = serve.HashServer(pool, bits=128, slots=3, capacity=4096, max_requests_per_batch=8,
                              max_bytes_in_flight=cap, use_graphs=use_graphs)
    try:
        stats = serve.run_poisson(server, reqs, rate_per_s=2000.0, seed=1)
        assert server.device_errors() == [0, 0, 0]
        assert server.peak_in_flight_bytes <= cap
        assert stats["requests"] == len(reqs) and stats["p99_ms"] >= stats["p50_ms"] > 0
    finally:
        server.close()
    alone = serve.HashServer(pool, bits=128, slots=1, capacity=4096, max_requests_per_batch=1,
                             max_bytes_in_flight=cap, use_graphs=use_graphs)
    try:
        solo = _clone(reqs)
        for r in solo:
            alone.submit(r)
            alone.drain()
        assert alone.device_errors() == [0]
    finally:
        alone.close()
    host_pool = pool.cpu().numpy()
    rng = np.random.default_rng(3)
    for mixed, single in zip(reqs, solo):
        assert np.array_equal(mixed.result, single.result), mixed.rid
        pick = rng.choice(mixed.messages, size=min(25, mixed.messages), replace=False)
        expect = oracle_segments(mixed.key.view(np.int64).reshape(1, 4), np.zeros(len(pick), np.int32),
                                 host_pool, mixed.starts[pick], mixed.lengths[pick], 128)
        assert np.array_equal(mixed.result[pick], expect), mixed.rid


def test_file_sized_message_in_the_mix_matches_the_oracle(pool):
    """A request carrying a 16 MiB + 5 B message at an unaligned start (one
    warp or two threads per message on the device), served beside short and
    1 KiB messages of other requests, checked against the oracle."""
    big = serve.Request(key=np.array([1, 2, 3, 4], np.uint64),
                        starts=np.array([3, 77, (1 << 20) + 1], np.int64),
                        lengths=np.array([(16 << 20) + 5, 40, 1024], np.int64), rid=0)
    others = _requests(12, count=6)
    for r in others:
        r.rid += 1
    server = serve.HashServer(pool, bits=64, slots=2, capacity=4096, max_requests_per_batch=4,
                              max_bytes_in_flight=64 << 20, use_graphs=True)
    try:
        serve.run_poisson(server, [big] + others, rate_per_s=5000.0, seed=4)
        assert server.device_errors() == [0, 0]
    finally:
        server.close()
    host_pool = pool.cpu().numpy()
    expect = oracle_segments(big.key.view(np.int64).reshape(1, 4), np.zeros(3, np.int32),
                             host_pool, big.starts, big.lengths, 64)
    assert np.array_equal(big.result, expect)


def test_requests_that_can_never_fit_are_rejected(pool):
    server = serve.HashServer(pool, slots=1, capacity=64, max_bytes_in_flight=1 << 20,
                              use_graphs=False)
    try:
        big = serve.Request(key=np.zeros(4, np.uint64), starts=np.zeros(65, np.int64),
                            lengths=np.ones(65, np.int64))
        with pytest.raises(serve.TooLarge):
            server.submit(big)
        heavy = serve.Request(key=np.zeros(4, np.uint64), starts=np.zeros(1, np.int64),
                              lengths=np.array([2 << 20], np.int64))
        with pytest.raises(serve.TooLarge):
            server.submit(heavy)
        outside = serve.Request(key=np.zeros(4, np.uint64),
                                starts=np.array([POOL_BYTES - 5], np.int64),
                                lengths=np.array([10], np.int64))
        with pytest.raises(ValueError):
            server.submit(outside)
    finally:
        server.close()

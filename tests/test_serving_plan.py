"""Admission policy of the request server (host logic only, no GPU)."""
import types

import numpy as np

from paper_1612_06257_gb300.serve import plan_batch
from paper_1612_06257_gb300 import workloads


def _req(messages, payload):
    return types.SimpleNamespace(messages=messages, payload=payload)


def test_plan_takes_requests_in_order_until_a_limit():
    q = [_req(10, 100), _req(20, 200), _req(30, 300), _req(5, 50)]
    assert plan_batch(q, capacity=1000, max_requests=10, bytes_free=10**9) == 4
    assert plan_batch(q, capacity=59, max_requests=10, bytes_free=10**9) == 2   # messages
    assert plan_batch(q, capacity=1000, max_requests=3, bytes_free=10**9) == 3  # requests
    assert plan_batch(q, capacity=1000, max_requests=10, bytes_free=300) == 2   # bytes
    # Arrival order is kept: a small request behind a large one waits.
    assert plan_batch([_req(5, 900), _req(1, 1)], 1000, 10, 500) == 0
    assert plan_batch([], 1000, 10, 500) == 0


def test_serving_mix_recipe():
    reqs = workloads.serving_requests(200, 1 << 30, seed=3, huge_min=1 << 16, huge_max=1 << 20)
    lengths = np.concatenate([r[2] for r in reqs])
    msgs = np.array([len(r[1]) for r in reqs])
    assert msgs.min() >= 1 and msgs.max() <= 4096
    short = (lengths <= 64).mean()
    kib = (lengths == 1024).mean()
    huge = (lengths >= 1 << 16).mean()
    assert abs(short - 0.70) < 0.02 and abs(kib - 0.25) < 0.02 and abs(huge - 0.05) < 0.01
    for key, starts, lens in reqs:
        assert key.dtype == np.uint64 and key.shape == (4,)
        assert starts.min() >= 0 and (starts + lens).max() <= 1 << 30

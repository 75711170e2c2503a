"""GPU test: every Update-microbenchmark variant computes Section 4.2's Update.

The kernels' output words are checked against the independent Python
transcription (tests/ref_py/hh_ref.py), for the whole-state variants 0..5,
the lane-pair variants 6..11 and the one-lane-per-thread variant 12, with
the small launch (one block of 64 threads) used to time a single Update
chain.
"""
import numpy as np
import pytest
import torch

from paper_1612_06257_gb300 import hh
from tests.ref_py import hh_ref

pytestmark = pytest.mark.gpu

M64 = (1 << 64) - 1
UPDATES = 5
THREADS = 64


def _key(t):
    return [t, (t * 0x9E3779B97F4A7C15) & M64, ~t & M64, t ^ 0x5555AAAA5555AAAA]


def _state_after(key, pkt):
    st = hh_ref.State(key)
    for _ in range(UPDATES):
        st.update(pkt)
    return st.digest(4)


@pytest.fixture(scope="module")
def ctx():
    from paper_1612_06257_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    c = hh.hh_init(0)
    yield c
    hh.hh_destroy(c)


def test_whole_state_variants(ctx):
    expect = []
    for t in range(THREADS):
        h = _state_after(_key(t), [t, t + 1, t + 2, t + 3])
        expect.append(h[0] ^ h[1] ^ h[2] ^ h[3])
    for v in range(6):
        out = hh.hh_update_microbench(ctx, v, UPDATES, THREADS)
        torch.cuda.synchronize()
        assert out.cpu().numpy().view(np.uint64).tolist() == expect, v


def test_lane_pair_variants(ctx):
    expect = []
    for s in range(THREADS // 2):
        h = _state_after(_key(s), [2 * s, 2 * s + 1, 2 * s + 1, 2 * s + 2])
        expect += [h[0] ^ h[1], h[2] ^ h[3]]
    for v in range(6, 12):
        out = hh.hh_update_microbench(ctx, v, UPDATES, THREADS)
        torch.cuda.synchronize()
        assert out.cpu().numpy().view(np.uint64).tolist() == expect, v


def test_quad_variant(ctx):
    """One lane per thread, ZipperMerge partners exchanged by shuffle."""
    expect = []
    for s in range(THREADS // 4):
        h = _state_after(_key(s), [4 * s, 4 * s + 1, 4 * s + 2, 4 * s + 3])
        expect += h
    out = hh.hh_update_microbench(ctx, 12, UPDATES, THREADS)
    torch.cuda.synchronize()
    assert out.cpu().numpy().view(np.uint64).tolist() == expect


def test_thread_count_rules(ctx):
    out = torch.empty(512, dtype=torch.int64, device="cuda:0")
    for bad in (0, 16, 48 + 1, 288):
        with pytest.raises(hh.HHError):
            hh.hh_update_microbench(ctx, 1, 1, bad, out=out)
    with pytest.raises(hh.HHError):
        hh.hh_update_microbench(ctx, 13, 1, 32, out=out)

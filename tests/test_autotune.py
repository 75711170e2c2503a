"""GPU tests of the autotuner: whatever shapes it picks, the hashes stay
bit-identical to the oracle's, and its table survives a save/load round trip.
"""
import numpy as np
import pytest
import torch

from paper_1612_06257_gb300 import hh, workloads
from tests.helpers import as_u64, oracle_hashes

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module")
def tuned():
    from paper_1612_06257_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    ctx = hh.hh_init(0)
    before = hh.hh_tune_describe(ctx)
    hh.hh_autotune(ctx, 256 << 20)
    yield ctx, before
    hh.hh_destroy(ctx)


def _table(text):
    return [line.split() for line in text.splitlines() if line and not line.startswith("#")]


def test_table_is_well_formed(tuned):
    ctx, before = tuned
    rows = _table(hh.hh_tune_describe(ctx))
    kinds = [r[0] for r in rows]
    assert kinds == ["fixed"] * 5 + ["ragged", "huge_bucket", "solo_per_sm", "solo_shared",
                                      "fixed_pair"]
    assert [int(r[1]) for r in rows[:5]] == list(range(5))
    assert len(_table(before)) == len(rows)
    # After tuning, the text carries each candidate's measured time.
    report = [l for l in hh.hh_tune_describe(ctx).splitlines() if l.startswith("# ") and "=" in l]
    assert len(report) == 8 and all("ms" in l for l in report)


@pytest.mark.parametrize("length", [0, 17, 64, 200, 1024, 3000, 70000])
def test_tuned_fixed_matches_oracle(tuned, length):
    ctx, _ = tuned
    n = max(1, min(20000, (8 << 20) // max(length, 1)))
    w = workloads.fixed(n, length, seed=length + 5, device=DEV)
    for bits in (64, 256):
        got = hh.hh_hash_fixed(ctx, bits, w.keys, 0, w.data, length, n)
        assert hh.hh_get_device_error(ctx) == hh.HH_OK
        assert np.array_equal(as_u64(got, bits // 64), oracle_hashes(w, bits))


def test_tuned_ragged_with_long_messages_matches_oracle(tuned):
    ctx, _ = tuned
    g = torch.Generator().manual_seed(9)
    lengths = torch.cat([torch.randint(0, 4000, (5000,), generator=g),
                         torch.tensor([(2 << 20) + 5, (1 << 20) + 31, 300000])])
    w = workloads.from_lengths(lengths[torch.randperm(lengths.numel(), generator=g)],
                               seed=10, device=DEV)
    got = hh.hh_hash128_batch(ctx, w.keys, 1, w.data, w.offsets)
    assert hh.hh_get_device_error(ctx) == hh.HH_OK
    assert np.array_equal(as_u64(got, 2), oracle_hashes(w, 128))


def test_save_and_load_round_trip(tuned, tmp_path):
    ctx, _ = tuned
    path = str(tmp_path / "tune.txt")
    hh.hh_tune_save(ctx, path)
    ctx2 = hh.hh_init(0, path)
    try:
        assert _table(hh.hh_tune_describe(ctx2)) == _table(hh.hh_tune_describe(ctx))
    finally:
        hh.hh_destroy(ctx2)


@pytest.mark.parametrize("text", ["fixed 9 128 2 1\n", "fixed 0 100 2 1\n", "ragged 128 9\n",
                                  "huge_bucket -1\n", "solo_per_sm 65\n", "solo_shared 2\n",
                                  "bogus line\n"])
def test_bad_table_is_rejected(tmp_path, text):
    path = tmp_path / "bad.txt"
    path.write_text("# libhh tuning table v1\n" + text)
    with pytest.raises(hh.HHError) as e:
        hh.hh_init(0, str(path))
    assert e.value.status == hh.HH_ERR_INVALID_ARG
    with pytest.raises(hh.HHError):
        hh.hh_init(0, str(tmp_path / "missing.txt"))


def test_set_tune_param(tmp_path):
    ctx = hh.hh_init(0)
    try:
        hh.hh_set_tune_param(ctx, "solo_per_sm", 2)
        hh.hh_set_tune_param(ctx, "solo_shared", 0)
        hh.hh_set_tune_param(ctx, "huge_bucket", 2304)
        rows = dict((r[0], r[1:]) for r in _table(hh.hh_tune_describe(ctx)))
        assert rows["solo_per_sm"] == ["2"] and rows["solo_shared"] == ["0"]
        assert rows["huge_bucket"] == ["2304"]
        for name, value in (("solo_per_sm", -1), ("solo_shared", 2), ("huge_bucket", 5000),
                            ("no_such_param", 1)):
            with pytest.raises(hh.HHError):
                hh.hh_set_tune_param(ctx, name, value)
    finally:
        hh.hh_destroy(ctx)

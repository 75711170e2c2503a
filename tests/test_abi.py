"""The C ABI library builds, loads and exports what include/hh.h declares (no GPU).

Host-side argument checks that return before any CUDA call are exercised
here too; nothing in this file launches a kernel.
"""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hh.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1612_06257_gb300 import build, hh
    build.build()
    return hh.load_library()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hh_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("hh_init", "hh_destroy", "hh_hash64_batch", "hh_hash128_batch",
                     "hh_hash256_batch", "hh_get_device_error", "hh_status_string"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    from paper_1612_06257_gb300 import hh
    names = declared_functions()
    assert sorted(hh.EXPORTS) == names
    for name in names:
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", hh.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (hh_[a-z0-9_]+)$", out, flags=re.M))
    assert set(names) <= exported


def test_status_strings(lib):
    from paper_1612_06257_gb300 import hh
    seen = set()
    for code in range(0, 10):
        s = hh.hh_status_string(code)
        assert s and s != "unknown status"
        seen.add(s)
    assert len(seen) == 10
    assert hh.hh_status_string(99) == "unknown status"


def test_null_context_is_rejected_without_cuda(lib):
    from paper_1612_06257_gb300 import hh
    L = lib
    assert L.hh_hash64_batch(None, None, 0, None, None, 1, None, None) == hh.HH_ERR_INVALID_ARG
    assert L.hh_hash_fixed(None, 64, None, 0, None, 32, 1, None, None) == hh.HH_ERR_INVALID_ARG
    assert L.hh_hash_host(None, 64, None, 0, None, None, 1, None) == hh.HH_ERR_INVALID_ARG
    assert L.hh_set_kernel(None, 0) == hh.HH_ERR_INVALID_ARG
    assert L.hh_reserve(None, 10) == hh.HH_ERR_INVALID_ARG
    assert L.hh_get_device_error(None, None) == hh.HH_ERR_INVALID_ARG
    assert L.hh_destroy(None) == hh.HH_OK
    assert L.hh_last_launch_count(None) == 0
    assert L.hh_init(None, 0, None) == hh.HH_ERR_INVALID_ARG
    assert L.hh_hash_segments(None, 64, None, 1, None, None, 0, None, None, 1, None, None,
                              None) == hh.HH_ERR_INVALID_ARG
    assert L.hh_autotune(None, 1 << 30) == hh.HH_ERR_INVALID_ARG
    assert L.hh_tune_save(None, b"x") == hh.HH_ERR_INVALID_ARG
    assert L.hh_tune_describe(None, None, 0) == hh.HH_ERR_INVALID_ARG
    assert L.hh_set_tune_param(None, b"solo_per_sm", 2) == hh.HH_ERR_INVALID_ARG
    assert L.hh_prng_fill(None, 64, None, 0, 1, None, None) == hh.HH_ERR_INVALID_ARG
    assert L.hh_stream_init(None, None, 0, 1, None, None) == hh.HH_ERR_INVALID_ARG
    assert L.hh_stream_update(None, None, None, None, 1, None) == hh.HH_ERR_INVALID_ARG
    assert L.hh_stream_finish(None, 64, None, None, None, 1, None, None) == hh.HH_ERR_INVALID_ARG
    assert L.hh_stats_round_table(None, None, 3, 4, None, None) == hh.HH_ERR_INVALID_ARG
    assert L.hh_stats_toggle_counts(None, None, 24, None, None) == hh.HH_ERR_INVALID_ARG
    assert L.hh_stats_avalanche(None, 4, 0, 1, None, None) == hh.HH_ERR_INVALID_ARG


def test_init_without_a_gpu_reports_no_device(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1612_06257_gb300 import hh
    with pytest.raises(hh.HHError) as e:
        hh.hh_init(0)
    assert e.value.status == hh.HH_ERR_NO_DEVICE


def test_missing_library_fails_loudly(tmp_path):
    from paper_1612_06257_gb300 import hh
    saved = hh._lib
    try:
        hh._lib = None
        with pytest.raises(RuntimeError, match="no CPU fallback"):
            hh.load_library(str(tmp_path / "absent.so"))
    finally:
        hh._lib = saved


def test_product_and_oracle_share_no_code():
    """Neither side includes or imports the other."""
    pkg = os.path.join(ROOT, "paper_1612_06257_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                for pattern in (r"\bimport oracle\b", r"\bfrom oracle\b", r"\bhho_",
                                r"hho\.h", r"liboracle", r"\bsipo_", r"sipo\.h"):
                    assert not re.search(pattern, text), (f, pattern)
    odir = os.path.join(ROOT, "oracle")
    for f in os.listdir(odir):
        if f.endswith((".py", ".c", ".h")):
            text = open(os.path.join(odir, f)).read()
            assert "hh_device" not in text and "import paper_1612_06257_gb300" not in text
            assert "#include \"hh.h\"" not in text
            assert "siptree.cuh" not in text and "hh_internal" not in text

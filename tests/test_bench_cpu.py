"""Host-side pieces of bench.py that run without a GPU."""
import bench


def test_oracle_cycles_table_covers_the_paper_sizes(oracle):
    res = bench.oracle_cycles_table(target_s=0.005)
    assert res["threads"] == 1 and res["kind"] == "oracle"
    sizes = [row["bytes"] for row in res["rows"]]
    assert sizes == sorted(bench.PAPER_AVX2_CPB)
    for row in res["rows"]:
        assert row["ns_per_hash"] > 0 and row["gbps"] > 0
        assert row["paper_avx2_cycles_per_byte"] == bench.PAPER_AVX2_CPB[row["bytes"]]
        if res["nominal_mhz"]:
            assert row["cycles_per_byte"] > 0


def test_host_cpu_reports_a_model():
    model, mhz = bench.host_cpu()
    assert isinstance(model, str) and model
    assert mhz is None or mhz > 0


def test_both_arms_measure_the_same_workload():
    """The reference arm hashes the GPU arm's whole batch per step, so both
    lines carry the same configuration (the GPU arm adds how it ran)."""
    import inspect
    ref_src = inspect.getsource(bench.run_reference)
    ours_src = inspect.getsource(bench.run_ours)
    assert "workload_config()" in ref_src and "workload_config()" in ours_src
    assert "N_MESSAGES, MESSAGE_BYTES, seed=1000" in ref_src
    assert "N_MESSAGES, MESSAGE_BYTES, seed=1000 + rank" in ours_src
    cfg = bench.workload_config()
    assert cfg["n_messages"] == 1 << 20 and cfg["message_bytes"] == 1024


def test_committed_profiler_counts_match_the_kernel_sources():
    """profiles/traffic.json and profiles/alu_counts.json were taken on the
    kernels as committed: their source digests match the current translation
    units (the bench leaves a figure out once they do not)."""
    import json
    import os
    import bench
    from paper_1612_06257_gb300.build import source_digest
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    traffic = json.load(open(os.path.join(root, "profiles", "traffic.json")))
    assert traffic["fixed_tma_kernel<128,2,2>"]["source_digest"] == bench.kernel_source_digest()
    counts = json.load(open(os.path.join(root, "profiles", "alu_counts.json")))
    assert {"short_count_kernel<1>", "short_count_kernel<2>", "prng_kernel<1>",
            "siptree_kernel<2,4>", "siptree_kernel<1,3>"} <= set(counts)
    for name, rec in counts.items():
        assert rec["source_digest"] == source_digest(rec["source_unit"]), name
        assert rec["alu_lane_instructions_per_output"] > 0 and "ncu" in rec["command"]


def test_alu_count_needs_a_matching_digest(tmp_path):
    import json
    from paper_1612_06257_gb300 import bench_workloads as bw
    from paper_1612_06257_gb300.build import source_digest
    path = tmp_path / "counts.json"
    good = {"source_digest": source_digest("hh_stats.cu"), "alu_lane_instructions_per_output": 7.5}
    stale = dict(good, source_digest="0" * 16)
    path.write_text(json.dumps({"k": good, "old": stale}))
    assert bw._alu_count("k", "hh_stats.cu", str(path)) == 7.5
    assert bw._alu_count("old", "hh_stats.cu", str(path)) is None
    assert bw._alu_count("k", "hh_ragged.cu", str(path)) is None  # another unit's digest
    assert bw._alu_count("missing", "hh_stats.cu", str(path)) is None
    assert bw._alu_count("k", "hh_stats.cu", str(tmp_path / "absent.json")) is None

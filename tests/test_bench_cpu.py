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

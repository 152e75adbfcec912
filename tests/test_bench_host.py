"""Host-side checks of bench.py's DRAM-traffic bookkeeping (no GPU).

The bench reports a stage's DRAM bytes from the committed one-pass ncu capture of the
1.97 M-point workload (profiles/dram_sphere_655360.md) only while the kernel sources it
names still hash to the recorded values; otherwise, and on any other workload, it must
report null with the reason instead of a stale figure.
"""
import bench

STAGES = ["prep", "k_p2p_packed", "k_p2m_w", "k_m2l_tc", "k_l2p_t", "k_corr", "m2m", "l2l"]


def test_capture_summary_names_every_stage_the_bench_reads():
    for stage in STAGES:
        value, why = bench._ncu_dram(stage, bench.DRAM_WORKLOAD)
        assert why != "no ncu capture", stage  # file, hash and byte entries all present
        if value is not None:
            assert value > 0 and why.startswith("ncu dram__bytes_read.sum"), stage
        else:
            assert why == "kernel changed since the ncu capture", stage


def test_other_workloads_get_no_traffic():
    value, why = bench._ncu_dram("k_m2l_tc", "sphere_163840")
    assert value is None and "no ncu capture of this workload" in why


def test_changed_source_drops_the_figure(monkeypatch):
    monkeypatch.setattr(bench, "_source_sha", lambda fname: "0000000000000000")
    for stage in STAGES:
        value, why = bench._ncu_dram(stage, bench.DRAM_WORKLOAD)
        assert value is None and why == "kernel changed since the ncu capture", stage


def test_unknown_stage_is_reported_as_uncaptured():
    value, why = bench._ncu_dram("k_not_a_kernel", bench.DRAM_WORKLOAD)
    assert value is None and why == "no ncu capture"

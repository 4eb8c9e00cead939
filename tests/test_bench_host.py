"""Host-side helpers of bench.py: the committed ncu traffic summary, the roofline peak and
single-process aggregation (no GPU needed)."""
import os

import bench


def test_ncu_traffic_summary_parses():
    for cls in ("mixed.f16.l12.v2.K1_chi_minv", "mixed.f16.l12.v2.K4_normal_cg", "mixed.f16.l12.v2.P_update_chi"):
        got = bench.ncu_traffic(cls)
        assert got is not None, cls
        nbytes, nsys = got
        assert nsys == 3 and nbytes > 1e8
    assert bench.ncu_traffic("no.such.class") is None


def test_traffic_within_a_few_percent_of_algorithmic_bytes():
    # each summary line: class, dram bytes per launch, systems, algorithmic bytes, ratio
    path = os.path.join(os.path.dirname(bench.__file__), "profiles", "ncu_traffic.txt")
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        _, dram, _, alg, ratio = line.split()
        assert abs(float(dram) / float(alg) - float(ratio)) < 0.01
        assert 0.8 < float(ratio) < 1.2


def test_peak_and_single_rank_aggregate():
    peak, kind = bench.measured_peaks()
    assert peak > 1000 and kind in ("measured", "fallback")
    value, t, n = bench.aggregate(2.0, 6)
    assert (value, t, n) == (3.0, 2.0, 6)


def test_traffic_of_a_kernel_changed_since_its_capture_is_null():
    stale = bench.traffic_fields("mixed.f16.l12.v2.K4_normal_cg", 1.7e9)
    assert stale["traffic"] is None and stale["traffic_prior_capture"] == 1.7e9 and stale["traffic_note"]
    assert bench.traffic_fields("mixed.f16.l12.v2.K1_chi_minv", 3.8e8) == {"traffic": 3.8e8}
    assert bench.traffic_fields("mixed.f16.l12.v2.K2_schur_norm_mdinv", None) == {"traffic": None}

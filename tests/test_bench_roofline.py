"""The roofline arithmetic bench.py reports (CPU only): the method's peak of
the ray kernel is min(SFU, FP32) surface-samples/s from the unit counts and
the maximum SM clock, the two limits tie at four surfaces, and the
evaluated-work roofline rates the evaluated fraction against the kernel's own
op mix."""
import pytest

import bench


def test_method_peak_from_unit_counts():
    clk = 152 * 2070e6
    peak, sfu, fp32 = bench.march_peak(4)
    assert sfu == pytest.approx(clk / (1 / 32 + 1 / 16))          # ex2 + rcp per logistic
    assert fp32 == pytest.approx(clk * 128 / (48 / 4))             # 12 + 9L ops per sample, L = 4
    assert peak == pytest.approx(3.35616e12) and sfu == pytest.approx(fp32)
    p3, s3, f3 = bench.march_peak(3)
    assert p3 == f3 == pytest.approx(clk * 128 / 13) and f3 < s3  # FP32-bound with 3 surfaces
    p8, s8, f8 = bench.march_peak(8)
    assert p8 == s8 and s8 < f8                                     # SFU-bound with 8


def test_evaluated_roofline():
    clk = 152 * 2070e6
    # FP32 binds: 32 lane-ops per evaluated sample of the accurate logistic
    assert bench.march_peak_evaluated() == pytest.approx(clk * 128 / 32)
    r = bench.evaluated_roofline(3.0, 0.25, 1.0)
    assert r["fraction"] == 0.25 and r["achieved"] == pytest.approx(0.75)
    assert r["frac"] == pytest.approx(0.75 / (clk * 128 / 32 / 1e12))
    assert bench.evaluated_roofline(3.0, 1.0, 0.0) is None


def test_max_over_ranks_single_process():
    assert bench.max_over_ranks(12.5) == 12.5


def test_issue_share_arithmetic(monkeypatch):
    monkeypatch.setattr(bench, "march_source_sha1", lambda: bench.MARCH_INST["source_sha1"])
    r = bench.issue_share(1024, 0.0341)
    slots = 0.0341 * 152 * 4 * 2070e6
    assert r["slots"] == pytest.approx(slots)
    assert r["frac"] == pytest.approx(bench.MARCH_INST["per_chain"] * 1024 / slots)
    monkeypatch.setattr(bench, "march_source_sha1", lambda: "0" * 12)
    assert bench.issue_share(1024, 0.0341) is None and bench.march_traffic() is None

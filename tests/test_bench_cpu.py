"""The benchmark's measurement arithmetic (CPU): the algorithmic byte counts of the
roofline objects, the roofline fraction, and the rule that an ncu traffic figure is used
only while the kernel sources match the digest recorded with it."""
import os

import pytest

import bench


def test_march_bytes_counts_each_term():
    # steps (probes), composited samples, indirection reads; rays
    cnt = [1000.0, 10.0, 50.0]
    assert bench.march_bytes(cnt, 7) == 4 * 50 + 1 * 1000 + 64 * 10 + 12 * 7


def test_roofline_fraction_and_keys(monkeypatch):
    monkeypatch.setattr(bench, "measured_peaks", lambda: ({"hbm_gbs": 5000.0}, "measured"))
    r = bench.roofline(2e9, 1.0, "k")               # 2 GB in 1 ms = 2000 GB/s
    assert r["achieved"] == pytest.approx(2000.0) and r["frac"] == pytest.approx(0.4)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["peak"] == 5000.0 and r["traffic"] is None
    assert r["algorithmic_bytes_per_launch"] == 2000000000
    r2 = bench.roofline(1e9, 1.0, "k", launches=2)
    assert r2["algorithmic_bytes_per_step"] == 1000000000 and r2["launches_per_step"] == 2


def test_training_roofline_bytes(monkeypatch):
    monkeypatch.setattr(bench, "measured_peaks", lambda: ({"hbm_gbs": 1000.0}, "measured"))
    monkeypatch.setattr(bench, "profiled_traffic", lambda *a, **k: None)
    cnt = [300.0, 20.0, 40.0]
    n = 256                                          # two CTAs of 128 rays
    two, one = bench.training_rooflines(cnt, n, 1.0, 1.0, "x")
    adj = bench.ADJ_BYTES_PER_SAMPLE * 20 + bench.MLP_GRAD_BYTES_PER_CTA * 2
    march = bench.march_bytes(cnt, n)
    assert bench.ADJ_BYTES_PER_SAMPLE == 64 + 8 * 2 * 32
    assert two["algorithmic_bytes_per_step"] == int(march + 12 * n + 48 * n + 72 * n + adj)
    assert one["algorithmic_bytes_per_launch"] == int(march + 24 * n + adj)


def test_traffic_only_with_matching_digest(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    digest = bench.kernel_source_digest(bench.FWD_SOURCES)
    (prof / "k_match.md").write_text(f"# x\n\n- kernel_source_digest: `{digest}`\n- dram_bytes_per_launch: `1234`\n")
    (prof / "k_stale.md").write_text("# x\n\n- kernel_source_digest: `0000000000000000`\n- dram_bytes_per_launch: `99`\n")
    assert bench.profiled_traffic("k_match") == 1234.0
    assert bench.profiled_traffic("k_stale") is None
    assert bench.profiled_traffic("k_missing") is None
    # a two-launch step sums its kernels' figures, and has none if one is missing
    monkeypatch.setattr(bench, "measured_peaks", lambda: ({"hbm_gbs": 1.0}, "measured"))
    both = bench.roofline(1.0, 1.0, "k", profile=[("k_match", bench.FWD_SOURCES), ("k_match", bench.FWD_SOURCES)])
    assert both["traffic"] == 2468.0
    part = bench.roofline(1.0, 1.0, "k", profile=[("k_match", bench.FWD_SOURCES), ("k_stale", bench.FWD_SOURCES)])
    assert part["traffic"] is None


def test_committed_profiles_name_their_command():
    root = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "profiles")
    for f in os.listdir(root):
        txt = open(os.path.join(root, f)).read()
        assert "ncu " in txt and "--clock-control none" in txt, f

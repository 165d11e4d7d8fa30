"""Host logic of bench.py (no GPU): the roofline arithmetic and the use of
the committed DRAM-traffic records (only while the captured kernel source
and launch shape are the ones being timed)."""
import hashlib
import json
import os

import pytest

import bench


def _stats(threads=256, ppt=2, evaluated=2_000_000_000, rescued=1_000_000):
    return {"pairs_evaluated": evaluated, "pairs_rescued": rescued, "block_threads": threads,
            "points_per_thread": ppt}


def test_roofline_arithmetic():
    st = _stats()
    r = bench.roofline(st, ms_label=4.0, peak=80.0, sms=152, clocks={"sm_mhz": 1035.0})
    achieved = (st["pairs_evaluated"] - st["pairs_rescued"]) * bench.FLOPS_PER_PAIR / 4e-3 / 1e12
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["achieved"] == pytest.approx(achieved)
    assert r["frac"] == pytest.approx(achieved / 80.0)
    # at half the clock the same work is twice the fraction of that clock's peak
    assert r["frac_at_sampled_clock"] == pytest.approx(achieved / (152 * 256 * 1035e6 / 1e12))
    assert r["kernel"] == "k_label32<256, 2, 2>"


def _source_sha():
    src = os.path.join(bench.ROOT, "paper_2203_10000_gb300", "csrc", "zef_label.cu")
    return hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]


def test_traffic_record_matches_source_and_shape(tmp_path, monkeypatch):
    sha = _source_sha()
    recs = {"config4": [{"bytes_per_launch": 111, "kernel": "k_label32<256,2,2>", "source_sha256_prefix": sha},
                        {"bytes_per_launch": 222, "kernel": "k_label32<128,2,2>", "source_sha256_prefix": sha}],
            "config1": {"bytes_per_launch": 333, "kernel": "k_label32<256,2,2>", "source_sha256_prefix": "0" * 16}}
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(recs))
    (tmp_path / "paper_2203_10000_gb300" / "csrc").mkdir(parents=True)
    src = os.path.join(bench.ROOT, "paper_2203_10000_gb300", "csrc", "zef_label.cu")
    (tmp_path / "paper_2203_10000_gb300" / "csrc" / "zef_label.cu").write_bytes(open(src, "rb").read())
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_record(4, _stats(256, 2), 0) == 111
    assert bench.traffic_record(4, _stats(128, 2), 0) == 222
    assert bench.traffic_record(4, _stats(256, 4), 0) is None      # shape never captured
    assert bench.traffic_record(4, _stats(256, 2), 1) is None      # another kernel form
    assert bench.traffic_record(1, _stats(256, 2), 0) is None      # captured from another source
    assert bench.traffic_record(2, _stats(256, 2), 0) is None      # no record


def test_committed_traffic_records_are_well_formed():
    recs = json.load(open(os.path.join(bench.ROOT, "profiles", "traffic.json")))
    for cfg, rs in recs.items():
        for r in (rs if isinstance(rs, list) else [rs]):
            assert r["bytes_per_launch"] > 0
            assert r["kernel"].startswith("k_label32<")
            assert len(r["source_sha256_prefix"]) == 16
            assert os.path.exists(os.path.join(bench.ROOT, "profiles", r["source"]))

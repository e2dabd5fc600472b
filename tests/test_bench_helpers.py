"""Host-side helpers of bench.py: the per-kernel roofline arithmetic and the
rule that a DRAM-traffic record counts only for the kernel source it was
captured on."""
import hashlib
import json
import os

import bench


def test_kernel_roofline_arithmetic():
    n, P, ncells = 1000, 10, 64
    prof = {"gather": (2.0, 4), "rho": (1.0, 2), "rbl": (3.0, 3), "finalize": (0.2, 2), "scan": (0.0, 0)}
    out = bench._kernel_roofline(prof, n, P, ncells, {})
    peaks, _ = bench._peaks()
    hbm = float(peaks.get("hbm_gbs", bench.HBM_FALLBACK_GBS))
    g = out["gather"]               # 116 B per atom in 0.5 ms
    assert abs(g["achieved"] - 116.0 * n / 0.5e-3 / 1e9) < 1e-9 and abs(g["frac"] - g["achieved"] / hbm) < 1e-12
    r = out["rho"]                  # 2 N P special-function ops in 0.5 ms
    sfu = bench.SM_COUNT * bench.SFU_LANES_PER_SM * bench.SM_MAX_MHZ * 1e6 / 1e12
    assert abs(r["achieved"] - 2.0 * n * P / 0.5e-3 / 1e12) < 1e-12 and abs(r["peak"] - sfu) < 1e-12
    k = out["rbl"]
    lane = bench.SM_COUNT * bench.LANES_PER_SM * bench.SM_MAX_MHZ * 1e6 / 1e12
    assert abs(k["achieved"] - bench.RBL_OPS_PER_ATOM * n / 1e-3 / 1e12) < 1e-9 and abs(k["peak"] - lane) < 1e-12
    assert out["finalize"] == {"bound": "latency", "avg_launch_ms": 0.1}
    assert "scan" not in out                   # no launch recorded


def test_traffic_record_only_for_its_source(tmp_path, monkeypatch):
    src = tmp_path / "k.cu"
    src.write_text("kernel v1")
    prof = tmp_path / "profiles"
    prof.mkdir()
    sha = hashlib.sha256(b"kernel v1").hexdigest()
    rec = {"source_sha256": sha, "precision": "mixed", "dram_bytes_per_launch_full": 1234}
    (prof / "rbl_traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench._traffic(str(src)) == 1234
    src.write_text("kernel v2")                # the kernel changed after the capture
    assert bench._traffic(str(src)) is None
    os.remove(prof / "rbl_traffic.json")
    assert bench._traffic(str(src)) is None

"""Host logic of bench.py (no GPU): the per-point records it reads from
profiles/ apply only while the kernel source they were taken from is
unchanged, and the roofline objects carry the arithmetic the bench line
reports (achieved = per-launch work / average launch time, frac =
achieved / peak)."""
import hashlib
import math
import os

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _sha():
    src = os.path.join(ROOT, "paper_1502_07303_gb300", "csrc", "fmm_march.cu")
    return hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]


def test_profile_records_follow_the_kernel_source(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "rec.txt").write_text(
        "# kernel dtype workload sha value\n"
        f"k_march_continuous f64 sphere1024 {_sha()} 12.5\n"
        "k_march_continuous f32 sphere1024 0000000000000000 7.0\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    src_dir = tmp_path / "paper_1502_07303_gb300" / "csrc"
    src_dir.mkdir(parents=True)
    (src_dir / "fmm_march.cu").write_bytes(
        open(os.path.join(ROOT, "paper_1502_07303_gb300", "csrc", "fmm_march.cu"), "rb").read())
    assert bench._profile_record("rec.txt", "k_march_continuous", "f64", "sphere1024") == 12.5
    # a record of another source version is not used
    assert bench._profile_record("rec.txt", "k_march_continuous", "f32", "sphere1024") is None
    assert bench._profile_record("rec.txt", "k_march", "f64", "sphere1024") is None
    assert bench._profile_record("missing.txt", "k_march_continuous", "f64", "sphere1024") is None


def test_committed_records_match_the_committed_kernel():
    """The issue, double-pipe and traffic records in profiles/ were taken
    from the fmm_march.cu of this tree."""
    for fname in ("k_march_issue.txt", "k_march_traffic.txt", "k_march_dpipe.txt"):
        assert bench._profile_record(fname, "k_march_continuous", "f64", "sphere1024") is not None, fname


def test_roofline_arithmetic(monkeypatch):
    r = {"march_launches": 1.0, "march_ms": 200.0, "ms": 220.0}
    pts = 1 << 30
    monkeypatch.setattr(bench, "traffic_record", lambda *a: 40.0)
    h = bench.roofline_hbm(r, pts, 17, "k_march_continuous", "f64", "sphere1024", 6681.2, "measured")
    assert h["achieved"] == pytest.approx(17 * pts / 0.2 / 1e9)
    assert h["frac"] == pytest.approx(h["achieved"] / 6681.2)
    assert h["traffic"] == pytest.approx(40.0 * pts)
    assert h["share_of_step"] == pytest.approx(200 / 220)
    monkeypatch.setattr(bench, "issue_record", lambda *a: 200.0)
    monkeypatch.setattr(bench, "dpipe_record", lambda *a: 50.0)
    a = bench.roofline_alu(r, pts, "k_march_continuous", "f64", "sphere1024", 1.06e12, 152, 2070.0)
    peak = 4 * 152 * 2070e6 / 1e12
    assert a["peak"] == pytest.approx(peak)
    assert a["achieved"] == pytest.approx(200.0 * pts / 0.2 / 1e12)
    assert a["frac"] == pytest.approx(a["achieved"] / peak)
    assert a["fp64_pipe"]["peak"] == pytest.approx(0.53)
    assert a["fp64_pipe"]["achieved"] == pytest.approx(50.0 * pts / 0.2 / 1e12)
    f = bench.roofline_alu(r, pts, "k_march_continuous", "f32", "sphere1024", 1.06e12, 152, 2070.0)
    assert "fp64_pipe" not in f
    # no record: no achieved figure, rather than a made-up one
    monkeypatch.setattr(bench, "issue_record", lambda *a: None)
    n = bench.roofline_alu(r, pts, "k_march_continuous", "f32", "sphere1024", 1.06e12, 152, 2070.0)
    assert n["achieved"] is None and n["frac"] is None

"""Host-side pieces of the benchmark (CPU): the ncu traffic figures it reports
are taken only while the kernel's source is unchanged since the capture, the
roofline peak falls back when the measured peaks file is absent, and the
reference arm's iteration counts come from the stored oracle run."""
import json
import os

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _tree(tmp_path, src_text, line):
    (tmp_path / "profiles").mkdir()
    csrc = tmp_path / "paper_2001_01624_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "k_demo.cu").write_text(src_text)
    (tmp_path / "profiles" / "ncu_traffic.txt").write_text("# header\n" + line + "\n")


def test_traffic_taken_only_for_the_captured_source(tmp_path, monkeypatch):
    import hashlib
    src = "__global__ void k() {}\n"
    sha = hashlib.sha256(src.encode()).hexdigest()[:16]
    _tree(tmp_path, src, f"demo 123456 k_demo.cu {sha}")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.ncu_traffic("demo") == 123456.0
    assert bench.ncu_traffic("other") is None
    (tmp_path / "paper_2001_01624_gb300" / "csrc" / "k_demo.cu").write_text(src + "// changed\n")
    assert bench.ncu_traffic("demo") is None                   # source changed since the capture


def test_traffic_keyed_by_every_listed_source(tmp_path, monkeypatch):
    import hashlib
    src, hdr = "__global__ void k() {}\n", "// cell update\n"
    sha = lambda s: hashlib.sha256(s.encode()).hexdigest()[:16]
    _tree(tmp_path, src, f"demo 77 k_demo.cu {sha(src)} cell.cuh {sha(hdr)}")
    (tmp_path / "paper_2001_01624_gb300" / "csrc" / "cell.cuh").write_text(hdr)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.ncu_traffic("demo") == 77.0
    (tmp_path / "paper_2001_01624_gb300" / "csrc" / "cell.cuh").write_text(hdr + "// changed\n")
    assert bench.ncu_traffic("demo") is None                   # the header changed since the capture


def test_committed_traffic_lines_parse():
    for ln in open(os.path.join(ROOT, "profiles", "ncu_traffic.txt")):
        f = ln.split()
        if ln.startswith("#") or not f:
            continue
        assert len(f) >= 4 and len(f) % 2 == 0 and float(f[1]) > 0
        for name, sha in zip(f[2::2], f[3::2]):
            assert len(sha) == 16
            assert os.path.exists(os.path.join(ROOT, "paper_2001_01624_gb300", "csrc", name))


def test_peak_fallback_without_measured_file(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_peak() == (6800.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6700.5}))
    assert bench.measured_peak() == (6700.5, "measured")


def test_cpu_baseline_line_states_cores_and_host():
    nproc, model = bench.host_cpu()
    assert nproc >= 1 and model
    res = {"seconds": 4.0, "phases": {"solve": 1.0}, "basis_iters": 338, "steps": 101, "threads": 16}
    cb = bench.cpu_baseline_line(1_000_000, res)
    assert cb["value"] == 250_000.0 and cb["cores"] == 16 and cb["kind"] == "oracle"
    assert cb["nproc"] == nproc and cb["cpu_model"] == model
    assert "nothing extrapolated" in cb["sample"] and "16 threads" in cb["sample"]
    one = bench.cpu_baseline_line(1_000_000, dict(res, threads=1))
    assert one["cores"] == 1 and "single-threaded" in one["sample"]

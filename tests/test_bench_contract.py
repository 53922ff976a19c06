"""bench.py's reference arm (the serial oracle on the host cores) and the shape of its JSON line.

Runs without a GPU: the reference arm times the oracle only.
"""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                         cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1, out.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["value"] > 0 and d["unit"] == "GLUP/s" and d["higher_is_better"] is True
    assert d["steps"] == 1 and d["warmup"] == 0 and d["n_gpus"] == 1
    assert "workload" in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_headline_names_every_launch_parameter():
    """The headline's launch configuration (timed by bench.py and checked at full size by the GPU
    parity tests) names every tuning parameter it depends on."""
    sys.path.insert(0, ROOT)
    import bench

    for name in ("jacobi", "gs"):
        cfg = bench.HEADLINE[name]
        assert set(cfg) == {"nt", "tile", "variant", "int_adds"}
        assert cfg["nt"] == 1 and 0 <= cfg["int_adds"] <= 6


def test_traffic_record_is_used_only_for_the_measured_source(tmp_path, monkeypatch):
    """roofline.traffic comes from profiles/dram_traffic.txt only while the kernel's source file still
    hashes to the value recorded with the counters; any edit turns it into null."""
    import hashlib

    sys.path.insert(0, ROOT)
    import bench

    src = tmp_path / "k.cu"
    src.write_text("__global__ void k() {}\n")
    digest = hashlib.sha256(src.read_bytes()).hexdigest()[:16]
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "dram_traffic.txt").write_text("# comment\nk_kernel k.cu %s 123456\n" % digest)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench._traffic_from_profiles("k_kernel") == 123456.0
    assert bench._traffic_from_profiles("other_kernel") is None
    src.write_text("__global__ void k() { }\n")
    assert bench._traffic_from_profiles("k_kernel") is None


def test_committed_traffic_records_name_existing_sources():
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    for ln in open(path):
        ln = ln.strip()
        if not ln or ln.startswith("#"):
            continue
        kernel, src, digest, value = ln.split()[:4]
        assert os.path.exists(os.path.join(ROOT, src)), src
        assert len(digest) == 16 and float(value) > 0, ln



def test_temporal_depth_sweep_launch_parameters():
    """Each point of the temporal-depth sweep runs a configuration the library supports for it: the FP64
    headline at nt = 1, the multi-sweep column march with the integer-pipe forms it implements at nt = 2..4
    (FP64 0, 2 or 6), and the library defaults for FP32 Jacobi and for deeper blocking."""
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench

    assert bench._nt_cfg("jacobi", 1) == {k: bench.HEADLINE["jacobi"][k] for k in ("tile", "variant", "int_adds")}
    assert bench._nt_cfg("gs", 1) == {k: bench.HEADLINE["gs"][k] for k in ("tile", "variant", "int_adds")}
    for nt in (2, 3, 4):
        cfg = bench._nt_cfg("gs", nt)
        assert cfg["variant"] == 5 and cfg["int_adds"] in (0, 2, 6)
        assert bench._nt_cfg("gs_f32", nt)["int_adds"] == -1
    for name in ("jacobi_f32",):
        for nt in bench.NT_SWEEP:
            assert bench._nt_cfg(name, nt) == {"tile": (0, 0, 0), "variant": 0, "int_adds": -1}
    for name in ("jacobi", "gs", "gs_f32"):
        for nt in (8, 16):
            assert bench._nt_cfg(name, nt) == {"tile": (0, 0, 0), "variant": 0, "int_adds": -1}

"""bench.py's reference arm (the FP64 oracle on the host cores) runs without a GPU and
prints one JSON line with the contract's keys."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_the_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "3"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["warmup"] >= 3
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"] == "replicas8192x128"


def test_reference_arm_under_torchrun_two_ranks():
    """Launched like the multi-GPU driver (torchrun, two ranks on this host): rank 0 alone
    prints the line and the other rank exits 0 without work."""
    import socket
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    out = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
                          "--master-addr", "127.0.0.1", "--master-port", str(port),
                          os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2", "--steps", "1",
                          "--warmup", "3"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2


def _bench():
    sys.path.insert(0, ROOT)
    import bench
    return bench


def test_algorithmic_bytes_per_bead_step_by_hand():
    """The streamed form's compulsory bytes: 16 + 16 + 32 + 4 v + 8 m + 8 + 12 + (28 + 4 v) / K
    with v Verlet and m native entries per bead (two per pair)."""
    b = _bench()
    counts = {"bonds": 99, "native_pairs": 250, "verlet_pairs": 600}   # 100 beads: m = 5, v = 12
    got = b.algorithmic_bytes_per_bead_step(counts, 100, 10)
    assert got == 16 + 16 + 32 + 4 * 12 + 8 * 5 + 8 + 12 + (16 + 4 + 8 + 4 * 12) / 10


def test_recorded_traffic_needs_the_current_kernel_revision(tmp_path, monkeypatch):
    """A profile's DRAM bytes count only when its recorded source revision is the current one."""
    b = _bench()
    rev = b.kernel_revision()   # of the repository's sources
    (tmp_path / "profiles").mkdir()
    prof = tmp_path / "profiles" / "k_demo.md"
    monkeypatch.setattr(b, "ROOT", str(tmp_path))
    monkeypatch.setattr(b, "kernel_revision", lambda: rev)
    prof.write_text(f"# demo\n\nKernel source revision: `{rev}`\n\ntraffic_bytes_per_launch: 1234\n")
    assert b.recorded_traffic("k_demo") == 1234
    prof.write_text("# demo\n\nKernel source revision: `0000000000000000`\n\ntraffic_bytes_per_launch: 1234\n")
    assert b.recorded_traffic("k_demo") is None
    assert b.recorded_traffic("k_missing") is None


def test_measured_hbm_peak_is_read_from_the_peaks_file():
    b = _bench()
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        assert b.measured_hbm_gbs() == float(json.load(open(path))["hbm_gbs"])
    else:
        assert b.measured_hbm_gbs() == 6800.0

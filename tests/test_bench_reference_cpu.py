"""The reference arm of bench.py (the FP64 CPU oracle timed on a bounded sample of a workload: a few
FGMRES iterations of its solve) runs on the CPU and prints the contract's JSON line; ranks other than
0 exit without work. The check runs the sample on the small sine problem; the bench's default is the
headline Gaussian workload, whose oracle set-up alone takes minutes."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(extra_env):
    env = dict(os.environ, **extra_env)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                           "--warmup", "1", "--oracle-workload", "sine"], capture_output=True, text=True, env=env,
                          check=True, timeout=600, cwd=ROOT)


def test_reference_arm_prints_one_contract_line():
    out = _run({"RANK": "0"})
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "solves/s" and d["higher_is_better"] is True
    assert d["steps"] == 1 and d["warmup"] == 1 and d["n_gpus"] == 1 and d["vs_baseline"] is None
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["config"]["workload"] == "poisson-sine-2x2x2-N6"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and "2^3-element" in cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_do_no_work():
    out = _run({"RANK": "1"})
    assert out.stdout.strip() == ""


def test_gemm_traffic_comes_from_the_committed_summary_while_the_kernel_is_unchanged(monkeypatch, tmp_path):
    """roofline.traffic is read from the ncu summary under profiles/ only while the GEMM sources
    hash to the digest recorded there; a changed kernel (other digest) or a missing summary gives
    null instead of stale counters."""
    sys.path.insert(0, ROOT)
    import bench

    with open(bench.TRAFFIC_PROFILE) as f:
        recorded = [l.split(": ", 1)[1].strip() for l in f if l.startswith("- gemm_sources_sha256: ")]
    t = bench.gemm_traffic_per_launch()
    if recorded and recorded[0] == bench.gemm_sources_digest():
        assert t is not None and t > 0
    else:
        assert t is None
    monkeypatch.setattr(bench, "gemm_sources_digest", lambda: "0" * 64)
    assert bench.gemm_traffic_per_launch() is None
    monkeypatch.undo()
    monkeypatch.setattr(bench, "TRAFFIC_PROFILE", str(tmp_path / "missing.md"))
    assert bench.gemm_traffic_per_launch() is None

"""bench.py's reference arm (the oracle on the host cores) prints the one JSON
line of the bench contract; runs on CPU in a few seconds."""
import json
import subprocess
import sys
from pathlib import Path

ROOT = Path(__file__).resolve().parents[1]


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    sys.path.insert(0, str(ROOT))
    import bench

    assert d["impl"] == "reference" and d["metric"] == bench.METRIC
    assert d["unit"] == "s" and d["higher_is_better"] is False
    assert d["n_gpus"] == 1 and d["steps"] == 1 and d["warmup"] == 0
    assert d["value"] > 0 and abs(d["ms_per_step"] - 1e3 * d["value"]) <= 1e-9 * d["ms_per_step"]
    assert d["scaling"] == "weak" and d["vs_baseline"] is None and d["data"] == "synthetic"
    assert d["config"]["workload"] and "model" not in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["unit"] == "s"
    assert cb["cores"] >= 1 and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_exit_without_work():
    """Under torchrun only rank 0 times the oracle; another rank prints
    nothing and exits 0."""
    import os

    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1", MASTER_ADDR="127.0.0.1", MASTER_PORT="29511")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1",
                        "--warmup", "0"], cwd=ROOT, capture_output=True, text=True, timeout=120, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""


def _bench():
    sys.path.insert(0, str(ROOT))
    import bench

    return bench


def test_clock_summary_reports_median_max_and_throttle_reasons():
    """The clocks object of the JSON line: median SM clock under load, the
    maximum, and every throttle reason seen Active in any sample (the rows
    are nvidia-smi's csv,noheader,nounits output of the sampled fields)."""
    bench = _bench()
    rows = [
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2040, 2070, 1200.5, 0x8, Active, Not Active, Not Active, Not Active",
        "0, [N/A], 2070, 800.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbled",
    ]
    s = bench.ClockSampler(0, enabled=False)
    Path(s.tmp.name).write_text("\n".join(rows) + "\n")
    d = s.summary()
    assert d["sm_mhz"] == 2040.0 and d["sm_max_mhz"] == 2070.0
    assert d["reasons"] == ["hw_slowdown", "sw_power_cap"]
    assert d["samples"] == 4
    assert not Path(s.tmp.name).exists()


def test_clock_summary_without_samples_says_unavailable():
    bench = _bench()
    s = bench.ClockSampler(0, enabled=False)
    d = s.summary()
    assert d == {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}


def test_step_traffic_follows_the_profiled_kernel_sources(tmp_path, monkeypatch):
    """The roofline's traffic comes from the committed ncu summary only while
    the step kernel sources hash to the profiled version; any change to them
    turns it into null."""
    import shutil

    bench = _bench()
    csrc = ROOT / "paper_2503_22631_gb300" / "csrc"
    dst = tmp_path / "paper_2503_22631_gb300" / "csrc"
    dst.mkdir(parents=True)
    for f in ("step_kernels.cu", "step_common.cuh", "kernels.cuh"):
        shutil.copy(csrc / f, dst / f)
    import hashlib

    digest = hashlib.sha256(b"".join((dst / f).read_bytes() for f in ("step_kernels.cu", "step_common.cuh",
                                                                         "kernels.cuh"))).hexdigest()[:16]
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "step_kernel_traffic.txt").write_text(
        "# dram bytes of one step\n# a=b in a comment is ignored\n"
        f"step_kernels_sha256_16={digest}\nbytes_per_launch=123456789\n")
    monkeypatch.setattr(bench, "ROOT", tmp_path)
    assert bench.step_traffic() == 123456789.0
    with open(dst / "kernels.cuh", "a") as fh:
        fh.write("\n")
    assert bench.step_traffic() is None
    (tmp_path / "profiles" / "step_kernel_traffic.txt").unlink()
    assert bench.step_traffic() is None

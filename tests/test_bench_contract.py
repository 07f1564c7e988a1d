"""bench.py's reference arm (the FP64 oracle timed on the host cores) runs without a GPU and
prints the benchmark's JSON line; the units a step of each workload processes are the
workload's particle (or sample) counts."""
import json
import os
import subprocess
import sys
from types import SimpleNamespace

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_units_per_step():
    import bench
    a = SimpleNamespace(workload="warm2d", n=1024, ppc=64)
    assert bench.units_per_step(a) == 2 * 1024 * 1024 * 64
    a = SimpleNamespace(workload="hot3d", grid3=(256, 256, 512), ppc=8)
    assert bench.units_per_step(a) == 2 * 256 * 256 * 512 * 8
    a = SimpleNamespace(workload="hybrid", n=1024, ppc=16)
    assert bench.units_per_step(a) == 16777216
    a = SimpleNamespace(workload="closure", samples=1 << 20)
    assert bench.units_per_step(a) == 1 << 20
    a = SimpleNamespace(workload="scan", runs=256, ppc=32)
    assert bench.units_per_step(a) == 1470103552


@pytest.mark.slow
def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "hybrid",
                        "--steps", "1", "--warmup", "3"], cwd=ROOT, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 1 and d["warmup"] == 3
    assert d["config"]["workload"] == "hybrid_beam_2d_1024x1024_ppc16"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0
    assert d["ms_per_step"] == pytest.approx(16777216 / d["value"] * 1e3)


def test_reference_arm_other_ranks_exit_quietly():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3"],
                       cwd=ROOT, capture_output=True, text=True, timeout=300, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    assert not [l for l in r.stdout.splitlines() if l.startswith("{")]

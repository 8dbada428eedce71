"""bench.py's host logic without a GPU: the code hash that keys the recorded
DRAM traffic, the schedule defaults of each workload, and the reference arm's
JSON line (the oracle on a bounded sample)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_code_hash_ignores_comments_and_layout_only():
    src = 'int f(int a) {  // add one\n  /* the\n     body */ return a + 1;\n}\nconst char *s = "x // y";\n'
    same = 'int f(int a) { return a + 1; } // other words\nconst char *s = "x // y";'
    other = 'int f(int a) { return a + 2; }\nconst char *s = "x // y";'
    assert bench._code_only(src) == bench._code_only(same)
    assert bench._code_only(src) != bench._code_only(other)
    assert '"x // y"' in bench._code_only(src)  # string literals are code


def test_source_hash_covers_the_fused_solvers():
    csrc = os.path.join(ROOT, "paper_2207_12244_gb300", "csrc")
    present = set(os.listdir(csrc))
    assert set(bench.FUSED_SOURCES) <= present
    h = bench.lib_source_hash()
    assert len(h) == 16 and h == bench.lib_source_hash()


def test_schedule_defaults_follow_the_workload(monkeypatch):
    for argv, want in [([], (10, 5)), (["--workload", "precision"], (10, 3)),
                       (["--workload", "batch64"], (10, 3)),
                       (["--workload", "precision", "--n-pcg", "0"], (10, 0)),
                       (["--n-gn", "4"], (4, 5))]:
        monkeypatch.setattr(sys, "argv", ["bench.py"] + argv)
        a = bench.parse()
        assert (a.n_gn, a.n_pcg) == want, argv
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    a = bench.parse()
    assert bench.sequence_name(a) == bench.WORKLOAD
    assert bench.traffic_key(a, bench.WORKLOAD) == "solve_auto_" + bench.WORKLOAD
    monkeypatch.setattr(sys, "argv", ["bench.py", "--mode", "streaming", "--loss", "lsq"])
    a = bench.parse()
    assert bench.traffic_key(a, "w") == "solve_auto_w_lsq_streaming"
    assert bench.loss_params(a) == {"delta": 0.0, "loss": 0}


def test_reference_arm_prints_one_json_line():
    env = dict(os.environ, WORLD_SIZE="1", RANK="0", LOCAL_RANK="0")
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                          "--warmup", "0", "--width", "64", "--height", "48", "--frames", "2"],
                         cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["e2e"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"

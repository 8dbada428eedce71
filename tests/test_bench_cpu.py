"""bench.py's host logic without a GPU: the code hash that keys the recorded
DRAM traffic, the schedule defaults of each workload, the oracle's process
pool over all host cores, and the reference arm's JSON line (the oracle on a
bounded sample, with the same config as our arm's)."""
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
    for argv, want in [([], (10, 3)), (["--workload", "precision"], (10, 3)),
                       (["--workload", "sequence"], (10, 5)),
                       (["--workload", "precision", "--n-pcg", "0"], (10, 0)),
                       (["--n-gn", "4"], (4, 3)), (["--workload", "sequence", "--n-gn", "4"], (4, 5))]:
        monkeypatch.setattr(sys, "argv", ["bench.py"] + argv)
        a = bench.parse()
        assert (a.n_gn, a.n_pcg) == want, argv
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    a = bench.parse()
    assert a.workload == "batch64"  # the default line: 64 uneven keyframes
    cfg = bench.keyframes_config(a, 1)
    assert cfg["workload"] == "batch64-uneven-10x3-fp32" and cfg["keyframes"] == 64
    assert 25e6 < cfg["pixels"] < 36e6
    assert bench.traffic_key(a, cfg["workload"]) == "solve_auto_batch64-uneven-10x3-fp32"
    monkeypatch.setattr(sys, "argv", ["bench.py", "--workload", "sequence"])
    a = bench.parse()
    assert bench.sequence_name(a) == bench.WORKLOAD
    assert bench.traffic_key(a, bench.WORKLOAD) == "solve_auto_" + bench.WORKLOAD
    monkeypatch.setattr(sys, "argv", ["bench.py", "--mode", "streaming", "--loss", "lsq"])
    a = bench.parse()
    assert bench.traffic_key(a, "w") == "solve_auto_w_lsq_streaming"
    assert bench.loss_params(a) == {"delta": 0.0, "loss": 0}


def test_work_shares_cover_every_job_once_and_balance():
    sizes = [1228800] * 18 + [196608] * 21 + [76800] * 15 + [307200] * 10
    for n in (1, 3, 8, 16, 100):
        sh = bench._shares(sizes, n)
        flat = sorted(i for s in sh for i in s)
        assert flat == list(range(len(sizes)))
        loads = [sum(sizes[i] for i in s) for s in sh]
        assert len(sh) == min(n, len(sizes))
        assert max(loads) - min(loads) <= max(sizes)  # largest-first greedy bound


def test_oracle_pool_runs_every_share_in_a_spawned_process():
    jobs = [(24, 16, 1), (16, 12, 2), (20, 10, 3)]
    with bench.OraclePool(jobs, dict(n_gn=2, n_pcg=2), 2) as pool:
        assert sorted(i for s in pool.shares for i in s) == [0, 1, 2]
        wall, busy = pool.solve_all()
        assert len(busy) == 2 and wall > 0 and all(b > 0 for b in busy)
        wall2, _ = pool.solve_all()  # the workers stay up between passes
        assert wall2 > 0
    assert all(not p.is_alive() for p in pool.procs)


def test_host_cpu_names_a_model_and_counts_cores():
    model, cores = bench.host_cpu()
    assert isinstance(model, str) and model and cores >= 1


def test_reference_arm_prints_one_json_line():
    env = dict(os.environ, WORLD_SIZE="1", RANK="0", LOCAL_RANK="0")
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                          "--warmup", "0", "--workload", "sequence", "--width", "64",
                          "--height", "48", "--frames", "2"],
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
    assert d["config"] == bench.sequence_config(_args(["--workload", "sequence", "--width", "64",
                                                        "--height", "48", "--frames", "2"]), 1)
    assert d["cpu_baseline"]["cpu_model"] and d["cpu_baseline"]["host_cores"] >= 1


def _args(argv):
    old = sys.argv
    try:
        sys.argv = ["bench.py"] + argv
        return bench.parse()
    finally:
        sys.argv = old


def test_batch_reference_arm_uses_our_config_on_every_core():
    """The default workload's reference arm: the oracle over all 64 keyframes
    on the host's cores, with the config our arm prints (same workload keys,
    same values)."""
    env = dict(os.environ, WORLD_SIZE="1", RANK="0", LOCAL_RANK="0")
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], cwd=ROOT, env=env, capture_output=True, text=True,
                         timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    d = json.loads([ln for ln in out.stdout.splitlines() if ln.strip()][-1])
    assert d["config"] == bench.keyframes_config(_args([]), 1)
    assert d["config"]["workload"] == "batch64-uneven-10x3-fp32"
    cb = d["cpu_baseline"]
    assert cb["cores"] == min(cb["host_cores"], 64) and cb["cores"] >= 1
    assert d["value"] > 0 and d["e2e"]["value"] == d["value"]

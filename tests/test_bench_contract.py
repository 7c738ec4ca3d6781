"""The benchmark's reference arm (the oracle on the host cores) keeps the
one-JSON-line contract and names its workload with the same config keys as
the GPU arm; a non-zero rank does no work.  Runs on the CPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_bench(args, env_extra=None):
    env = dict(os.environ)
    env.pop("RANK", None)
    env.pop("WORLD_SIZE", None)
    env.pop("LOCAL_RANK", None)
    env.update(env_extra or {})
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=600)
    return r


def test_reference_arm_line():
    r = run_bench(["--impl", "reference", "--workload", "small", "--steps", "3", "--warmup", "3"])
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["higher_is_better"] is True and d["value"] > 0
    assert d["steps"] == 3 and d["warmup"] == 3 and d["n_gpus"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1 and d["cpu_baseline"]["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    # the workload keys the GPU arm's config also carries
    sys.path.insert(0, ROOT)
    import bench
    from paper_2605_14277_b300 import games as G
    want = bench.workload_config(G.small_random_game(1), "cfr")
    assert d["config"] == want


def test_reference_arm_other_ranks_do_nothing():
    r = run_bench(["--impl", "reference", "--workload", "small", "--steps", "3", "--warmup", "3"],
                  {"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert r.returncode == 0, r.stderr[-2000:]
    assert not [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]


def test_reference_arm_variant_flag():
    r = run_bench(["--impl", "reference", "--workload", "poker", "--variant", "pcfr", "--steps", "3", "--warmup", "3"])
    assert r.returncode == 0, r.stderr[-2000:]
    d = json.loads([ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")][0])
    assert d["config"]["variant"] == "pcfr" and d["config"]["updates"] == "alternating"
    assert "pcfr iterations" in d["cpu_baseline"]["sample"]


def test_reference_arm_nplayer():
    """The n-player workload's reference arm: the n-player oracle on the
    4.84M-node three-player game, the GPU arm's workload keys."""
    r = run_bench(["--impl", "reference", "--workload", "nplayer", "--steps", "1", "--warmup", "3"])
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
    sys.path.insert(0, ROOT)
    import bench
    from paper_2605_14277_b300 import games as G
    assert d["config"] == bench.nplayer_config(G.large_nplayer_game(3), "dcfr")

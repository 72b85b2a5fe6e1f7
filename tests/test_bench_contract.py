"""bench.py's reference arm on the CPU: `--impl reference` times the FP64 oracle on a bounded sample
of the workload's EB-face LS systems and prints one JSON line with the contract's keys."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

KEYS = {"impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
        "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"}


def _run(env_extra=None, *args):
    env = dict(os.environ)
    env.update(env_extra or {})
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--n", "16",
                        "--steps", "1", "--warmup", "1", "--cpu-seconds", "2", *args],
                       capture_output=True, text=True, env=env, timeout=600)
    assert r.returncode == 0, r.stderr
    return [l for l in r.stdout.splitlines() if l.startswith("{")]


def test_reference_arm_prints_one_contract_line():
    lines = _run()
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert KEYS <= set(d)
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == cb["host"]["nproc"] >= 1   # one oracle process per core
    assert cb["host"]["uname_m"] and "lscpu_Architecture" in cb["host"] or "lscpu" in cb["host"]
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_print_nothing():
    assert _run({"RANK": "1", "WORLD_SIZE": "2"}) == []


def test_pick_tol_takes_the_loosest_target_within_the_error_bound():
    sys.path.insert(0, ROOT)
    import bench
    errs = {1e-7: 3.0, 1e-8: 1.2, 1e-9: 1.005, 1e-10: 1.0, 1e-11: 1.0}
    seen = []

    def err(c):
        seen.append(c)
        return errs[c]
    assert bench.pick_tol(err, 1.0) == 1e-9
    assert seen == [1e-7, 1e-8, 1e-9]          # stops at the first (loosest) target that qualifies
    assert bench.pick_tol(lambda c: 2.0, 1.0) == 1e-12

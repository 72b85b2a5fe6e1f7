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


def test_fp64_apply_timing_rotates_buffer_pairs_and_reports_rates():
    """The FP64 apply block of the bench line, with a stand-in for the library and the CUDA events:
    one warm-up apply per buffer pair, then rounds x pairs timed applies, each on its own pair in
    rotation; the rates follow from the median time and the algorithmic counts."""
    import types
    import numpy as np
    import torch
    sys.path.insert(0, ROOT)
    import bench
    import eb_inputs as E

    class Ev:
        def __init__(self, enable_timing=True):
            pass

        def record(self, s=None):
            pass

        def synchronize(self):
            pass

        def elapsed_time(self, other):
            return 2.0

    fake_torch = types.SimpleNamespace(tensor=lambda a, dtype=None, device=None: torch.tensor(a, dtype=dtype),
                                       float64=torch.float64, empty_like=torch.empty_like,
                                       cuda=types.SimpleNamespace(Event=Ev, current_stream=lambda: None))
    calls = []
    P = types.SimpleNamespace(eb_apply=lambda st, x, y, kappa_weighted=True: calls.append((x.data_ptr(),
                                                                                           y.data_ptr())))
    g = E.sphere_box_config(12)
    st = types.SimpleNamespace(info={"n_irregular_rows": 100, "n_row_classes": 5})
    r = bench.fp64_apply_timing(P, fake_torch, st, g, 637, 1.0, 1000.0, pairs=4, rounds=3)
    assert len(calls) == 4 + 12
    assert len(set(calls[:4])) == 4 and calls[4:8] == calls[:4] and calls[8:12] == calls[:4]
    assert r["ms_median"] == 2.0 and r["buffer_pairs"] == 4
    assert r["alg_bytes"] == 2 * g.ncell * 8 + 105 * 637 * 8
    nvol = int((g.flag > 0).sum())
    assert np.isclose(r["tflops"], 2 * 637 * nvol / 2e-3 / 1e12) and np.isclose(r["frac_fp64_peak"], r["tflops"])
    assert np.isclose(r["gbs"], r["alg_bytes"] / 2e-3 / 1e9) and np.isclose(r["frac_hbm"], r["gbs"] / 1000.0)

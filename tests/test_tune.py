"""Host logic of the kernel-shape autotuner (no GPU): candidates that do not compile are skipped, the
fastest timed candidate is recorded as `best`, and the build takes its flags from the record."""
import json

import pytest

from paper_1411_4283_gb300 import build as B
from paper_1411_4283_gb300 import tune as T


def test_tune_picks_fastest_and_skips_infeasible(tmp_path):
    times = {(4, 4): 850.0, (3, 5): 905.0, (2, 8): 1156.0}
    out = tmp_path / "tuned.json"
    rec = T.tune(n=16, reps=1, candidates=[(4, 4), (3, 5), (5, 8), (2, 8)],
                 build_fn=lambda s: None if s == (5, 8) else f"lib{s[0]}{s[1]}",
                 measure_fn=lambda lib, n, reps: times[(int(lib[3]), int(lib[4]))], out=str(out))
    assert rec["best"] == {"EB_LS_SYS": 4, "EB_LS_RPL": 4}
    skipped = [r for r in rec["results"] if r["ms_lsq"] is None]
    assert [(r["EB_LS_SYS"], r["EB_LS_RPL"]) for r in skipped] == [(5, 8)]
    assert json.loads(out.read_text()) == rec
    assert B.tuned_flags(str(out)) == ["-DEB_LS_RPL=4", "-DEB_LS_SYS=4"]


def test_tune_fails_when_nothing_compiles(tmp_path):
    with pytest.raises(RuntimeError):
        T.tune(candidates=[(9, 9)], build_fn=lambda s: None, measure_fn=None, out=str(tmp_path / "t.json"))


def test_committed_record_is_consistent():
    rec = json.load(open(B.TUNED))
    timed = [r for r in rec["results"] if r["ms_lsq"] is not None]
    best = min(timed, key=lambda r: r["ms_lsq"])
    assert rec["best"] == {"EB_LS_SYS": best["EB_LS_SYS"], "EB_LS_RPL": best["EB_LS_RPL"]}
    assert B.tuned_flags() == [f"-DEB_LS_RPL={best['EB_LS_RPL']}", f"-DEB_LS_SYS={best['EB_LS_SYS']}"]

"""Host logic of the kernel-shape autotuner (no GPU): candidates that do not compile are skipped, the
fastest timed candidate is recorded as `best`, and the build takes its flags from the record."""
import json

import pytest

from paper_1411_4283_gb300 import build as B
from paper_1411_4283_gb300 import tune as T


def test_tune_picks_fastest_and_skips_infeasible(tmp_path):
    key = lambda s: (s["EB_LS_SYS_F"], s["EB_LS_RPL"])
    times = {(6, 4): 420.0, (5, 4): 450.0, (3, 8): 700.0}
    cands = [{"EB_LS_SYS_F": 6, "EB_LS_RPL": 4, "EB_LS_SYS": 4}, {"EB_LS_SYS_F": 5, "EB_LS_RPL": 4, "EB_LS_SYS": 4},
             {"EB_LS_SYS_F": 9, "EB_LS_RPL": 8, "EB_LS_SYS": 4}, {"EB_LS_SYS_F": 3, "EB_LS_RPL": 8, "EB_LS_SYS": 2}]
    libs = {}

    def build_fn(s, base=None):
        if key(s) == (9, 8):
            return None
        libs[f"lib{len(libs)}"] = key(s)
        return f"lib{len(libs) - 1}"
    out = tmp_path / "tuned.json"
    rec = T.tune(n=16, reps=1, candidates=cands, build_fn=build_fn,
                 measure_fn=lambda lib, n, reps: times[libs[lib]], out=str(out))
    assert rec["best"] == {"EB_LS_SYS_F": 6, "EB_LS_RPL": 4, "EB_LS_SYS": 4}
    skipped = [r for r in rec["results"] if r["ms_lsq"] is None]
    assert [key(r) for r in skipped] == [(9, 8)]
    assert json.loads(out.read_text()) == rec
    assert B.tuned_flags(str(out)) == ["-DEB_LS_RPL=4", "-DEB_LS_SYS=4", "-DEB_LS_SYS_F=6"]
    assert T.flags_of(cands[3]) == ["-DEB_LS_RPL=8", "-DEB_LS_SYS=2", "-DEB_LS_SYS_F=3"]


def test_tune_fails_when_nothing_compiles(tmp_path):
    with pytest.raises(RuntimeError):
        T.tune(candidates=[{"EB_LS_SYS_F": 9, "EB_LS_RPL": 9}], build_fn=lambda s, base=None: None,
               measure_fn=None, out=str(tmp_path / "t.json"))


def test_committed_record_is_consistent():
    rec = json.load(open(B.TUNED))
    want = T.pick_best(rec["results"], rec.get("margin", T.MARGIN))
    assert rec["best"] == want
    if "apply" in rec:
        app = T.pick_best(rec["apply"]["results"], rec["apply"].get("margin", T.MARGIN), "ms_apply")
        assert rec["apply"]["best"] == app
        want = {**want, **app}
    assert B.tuned_flags() == [f"-D{k}={int(v)}" for k, v in sorted(want.items())]


def test_default_kept_within_margin():
    res = [{"EB_LS_SYS_F": 6, "ms_lsq": 429.0}, {"EB_LS_SYS_F": 7, "ms_lsq": 425.7}, {"EB_LS_SYS_F": 5, "ms_lsq": None}]
    assert T.pick_best(res, 0.02) == {"EB_LS_SYS_F": 6}
    res[1]["ms_lsq"] = 400.0
    assert T.pick_best(res, 0.02) == {"EB_LS_SYS_F": 7}


def test_apply_target_keeps_the_least_squares_record(tmp_path):
    """The apply's launch shapes are a second record in the same file: tuning it keeps the
    least-squares record, compiles each candidate with the least-squares shape, and the build takes
    the flags of both; re-tuning the least squares keeps the apply record."""
    out = tmp_path / "tuned.json"
    ls = [{"EB_LS_SYS_F": 6, "EB_LS_RPL": 4, "EB_LS_SYS": 4}, {"EB_LS_SYS_F": 7, "EB_LS_RPL": 4, "EB_LS_SYS": 4}]
    ls_ms = {6: 430.0, 7: 400.0}
    T.tune(candidates=ls, build_fn=lambda s, base=None: s, measure_fn=lambda lib, n, r: ls_ms[lib["EB_LS_SYS_F"]],
           out=str(out))
    seen = []

    def build_fn(s, base=None):
        seen.append(dict(base))
        return s
    app_ms = {(8, 1): 0.60, (12, 1): 0.55, (8, 2): 0.59}
    cands = [{"EB_QUAD_PER_SM": q, "EB_FOLD_PER_SM": f} for q, f in app_ms]
    rec = T.tune(candidates=cands, build_fn=build_fn, target="apply", out=str(out),
                 measure_fn=lambda lib, n, r: app_ms[(lib["EB_QUAD_PER_SM"], lib["EB_FOLD_PER_SM"])])
    assert rec["best"] == {"EB_QUAD_PER_SM": 12, "EB_FOLD_PER_SM": 1}
    assert all(b == {"EB_LS_SYS_F": 7, "EB_LS_RPL": 4, "EB_LS_SYS": 4} for b in seen)
    whole = json.loads(out.read_text())
    assert whole["best"] == {"EB_LS_SYS_F": 7, "EB_LS_RPL": 4, "EB_LS_SYS": 4} and whole["apply"] == rec
    assert B.tuned_flags(str(out)) == ["-DEB_FOLD_PER_SM=1", "-DEB_LS_RPL=4", "-DEB_LS_SYS=4", "-DEB_LS_SYS_F=7",
                                       "-DEB_QUAD_PER_SM=12"]
    seen.clear()
    T.tune(candidates=ls[:1], build_fn=build_fn, measure_fn=lambda lib, n, r: 1.0, out=str(out))
    assert seen == [{"EB_QUAD_PER_SM": 12, "EB_FOLD_PER_SM": 1}]
    assert json.loads(out.read_text())["apply"] == rec

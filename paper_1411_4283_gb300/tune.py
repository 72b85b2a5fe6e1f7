"""Autotuner of the compile-time kernel shapes, run on the target GPU.

The least-squares kernel's shape is fixed at compile time: how many systems one CTA keeps in
flight (EB_LS_SYS_F for the FP32-factorisation kernel, the default path; EB_LS_SYS for the FP64
one; their shared-memory blocks must fit in 227 KB) and how many rows each lane holds per chunk
(EB_LS_RPL, shared by both; larger chunks amortise the per-step Householder scalars and column sums
over more rows but leave fewer warps per SM to hide the serial parts).  Each candidate is compiled
into its own copy of the library (a candidate whose blocks do not fit fails its compile-time check
and is skipped), timed in a fresh process that builds the stencils of the 3-D sphere workload and
reads the least-squares launches' device time, and the fastest (the built-in default unless another
candidate beats it by more than MARGIN) is written to tuned_gb300.json, from which build.py takes the
default flags.

The apply's launch shapes are a second target (`--target apply`): how many CTAs per SM the unique-row
stream runs (EB_QUAD_PER_SM: few CTAs leave it latency-bound, many crowd the template pass off the
SMs) and how many persistent CTAs per SM the folded template pass keeps (EB_FOLD_PER_SM).  Each
candidate is timed as the FP32 kappa-weighted apply of the same sphere workload with its moment
tables generated on the device (CUDA events, best of reps after warm-up applies); its record sits
under "apply" in the same file, and the build takes the flags of both records.

    python -m paper_1411_4283_gb300.tune --n 128 --reps 2
    python -m paper_1411_4283_gb300.tune --target apply --n 256 --reps 20
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

from . import build as _build

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
# candidate shapes: the defines of each (FP32 systems per CTA, rows per lane, FP64 systems per CTA)
CANDIDATES = [
    {"EB_LS_SYS_F": 6, "EB_LS_RPL": 4, "EB_LS_SYS": 4},  # the built-in default: kept unless beaten by MARGIN
    {"EB_LS_SYS_F": 7, "EB_LS_RPL": 4, "EB_LS_SYS": 4},
    {"EB_LS_SYS_F": 5, "EB_LS_RPL": 4, "EB_LS_SYS": 4},
    {"EB_LS_SYS_F": 4, "EB_LS_RPL": 4, "EB_LS_SYS": 4},
    {"EB_LS_SYS_F": 4, "EB_LS_RPL": 6, "EB_LS_SYS": 3},
    {"EB_LS_SYS_F": 3, "EB_LS_RPL": 8, "EB_LS_SYS": 2},
]


# the apply's launch shapes: CTAs per SM of the unique-row stream and of the folded template pass
APPLY_CANDIDATES = [
    {"EB_QUAD_PER_SM": 8, "EB_FOLD_PER_SM": 1},  # the built-in default
    {"EB_QUAD_PER_SM": 6, "EB_FOLD_PER_SM": 1},
    {"EB_QUAD_PER_SM": 12, "EB_FOLD_PER_SM": 1},
    {"EB_QUAD_PER_SM": 16, "EB_FOLD_PER_SM": 1},
    {"EB_QUAD_PER_SM": 8, "EB_FOLD_PER_SM": 2},
    {"EB_QUAD_PER_SM": 4, "EB_FOLD_PER_SM": 2},
]

MARGIN = 0.02  # a candidate replaces the first (the built-in default) only when faster by more than this


def pick_best(results: list, margin: float = MARGIN, metric: str = "ms_lsq") -> dict:
    """The fastest timed result, or the first one when the fastest beats it by less than margin
    (run-to-run noise of the timing)."""
    timed = [r for r in results if r[metric] is not None]
    if not timed:
        raise RuntimeError("no candidate compiled")
    best = min(timed, key=lambda r: r[metric])
    first = results[0]
    if first[metric] is not None and best[metric] > (1.0 - margin) * first[metric]:
        best = first
    return {k: v for k, v in best.items() if k.startswith("EB_")}


def flags_of(shape: dict) -> list:
    return [f"-D{k}={int(v)}" for k, v in sorted(shape.items())]


def build_variant(shape: dict, base: dict | None = None) -> str | None:
    """Library path of the candidate (compiled with the other target's recorded shape, base), or None
    when it does not compile (shared memory)."""
    out = os.path.join(HERE, "_lib", "tune", "_".join(f"{k[3:].lower()}{v}" for k, v in sorted(shape.items())))
    try:
        return _build.build(force=True, out_dir=out, flags=flags_of({**(base or {}), **shape}))
    except RuntimeError:
        return None


_MEASURE = r"""
import json, sys
sys.path.insert(0, {root!r})
import torch
import eb_inputs as E
import paper_1411_4283_gb300 as P
g = E.sphere_box_config({n}, seed=2)
dg = P.DeviceGeometry.from_geometry(g)
ms = []
for _ in range({reps} + 1):
    st = P.eb_build_stencils(dg, order=4)
    torch.cuda.synchronize()
    ms.append(st.info["ms_lsq"])
    del st
print(json.dumps({{"ms_lsq": min(ms[1:])}}))
"""


_MEASURE_APPLY = r"""
import json, sys
sys.path.insert(0, {root!r})
import torch
import eb_inputs as E
import paper_1411_4283_gb300 as P
n = {n}
c = 0.5 + E.uniform(2, 3, -0.5 / n, 0.5 / n)
G = P.eb_geometry_spheres(n, [tuple(c)], [0.35], moment_degree=4)
st = P.eb_build_stencils(G, order=4)
x = torch.tensor(E.seeded_field(3, st.ncell), dtype=torch.float32, device="cuda")
y = torch.empty_like(x)
for _ in range(3):
    P.eb_apply(st, x, y, kappa_weighted=True)
ms = []
for _ in range({reps}):
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    P.eb_apply(st, x, y, kappa_weighted=True)
    b.record()
    b.synchronize()
    ms.append(a.elapsed_time(b))
print(json.dumps({{"ms_apply": min(ms)}}))
"""


def _run_measure(script: str, lib: str, n: int, reps: int, metric: str) -> float:
    env = dict(os.environ, EB_LIB_PATH=lib)
    r = subprocess.run([sys.executable, "-c", script.format(root=ROOT, n=n, reps=reps)], capture_output=True,
                       text=True, env=env, timeout=3600)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    return float(json.loads(r.stdout.strip().splitlines()[-1])[metric])


def measure(lib: str, n: int, reps: int) -> float:
    """Least-squares launch time (ms, best of reps after one warm-up build) with library lib."""
    return _run_measure(_MEASURE, lib, n, reps, "ms_lsq")


def measure_apply(lib: str, n: int, reps: int) -> float:
    """FP32 kappa-weighted apply time (ms, CUDA events, best of reps after three warm-up applies; the
    coefficients, well above the L2's size at 256^3, stream from HBM on every apply) with library lib."""
    return _run_measure(_MEASURE_APPLY, lib, n, reps, "ms_apply")


# per target: its candidates, its measurement, the metric's key, where its record sits in the file
# (None: at the top level), the workload it is timed on
TARGETS = {
    "lsq": (CANDIDATES, measure, "ms_lsq", None,
            "3-D unit cube minus sphere r=0.35 (seed 2), {n}^3, Q=4: least-squares launches (ms), the default "
            "(mixed-precision) path"),
    "apply": (APPLY_CANDIDATES, measure_apply, "ms_apply", "apply",
              "3-D unit cube minus sphere r=0.35 (centre 0.5 + U[-h/2, h/2)^3, seed 2; device moment tables), "
              "{n}^3, Q=4: FP32 kappa-weighted apply (ms)"),
}


def _load(out: str) -> dict:
    if os.path.exists(out):
        with open(out) as f:
            return json.load(f)
    return {}


def tune(n: int = 128, reps: int = 2, candidates=None, build_fn=build_variant, measure_fn=None,
         out: str = _build.TUNED, target: str = "lsq") -> dict:
    """Time every candidate of target that compiles; write its record (fastest as `best`) into out,
    keeping the other target's record, and return it."""
    cands, meas, metric, key, workload = TARGETS[target]
    candidates = cands if candidates is None else candidates
    measure_fn = meas if measure_fn is None else measure_fn
    whole = _load(out)
    other = whole.get("apply", {}).get("best", {}) if key is None else whole.get("best", {})
    results = []
    for shape in candidates:
        lib = build_fn(shape, other)
        if lib is None:
            results.append({**shape, metric: None, "note": "does not fit in shared memory"})
            continue
        results.append({**shape, metric: measure_fn(lib, n, reps)})
    rec = {"workload": workload.format(n=n), "date": time.strftime("%Y-%m-%d"), "results": results,
           "margin": MARGIN, "best": pick_best(results, MARGIN, metric)}
    if key is None:
        whole = {**rec, **({"apply": whole["apply"]} if "apply" in whole else {})}
    else:
        whole[key] = rec
    with open(out, "w") as f:
        json.dump(whole, f, indent=1)
        f.write("\n")
    return rec


def main():
    p = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    p.add_argument("--target", choices=sorted(TARGETS), default="lsq")
    p.add_argument("--n", type=int, default=128)
    p.add_argument("--reps", type=int, default=2)
    a = p.parse_args()
    print(json.dumps(tune(a.n, a.reps, target=a.target), indent=1))


if __name__ == "__main__":
    main()

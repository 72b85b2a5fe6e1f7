"""3-D sphere of Sec. 3.6 (inside the sphere (0.5,0.5,0.5), r = 0.45, Q = 4) on the GPU path:
solution errors at N = 32 and 64 against the paper's table, and the observed order.

At N = 32 the FP64 oracle gives L_inf 1.016e-4, L1 1.539e-5, L2 2.423e-5 (a uniform 1.11x the
printed values: a difference in the 3-D problem set-up rather than in a norm or neighbourhood
reading, which would move the three norms differently); the GPU must reproduce the oracle's numbers, sit within 15% of the
paper's, and converge at fourth order between N = 32 and 64.
"""
import json
import os

import numpy as np
import pytest

import eb_inputs as E
from gpu_helpers import build_gpu, to_dev

pytestmark = pytest.mark.gpu

# written by tests/golden/make_sphere_golden.py (calls only the oracle)
ORACLE_32 = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "sphere_n32.json")))["sol"]
PRINTED = {32: {"linf": 9.16e-05, "l1": 1.38e-05, "l2": 2.17e-05}, 64: {"linf": 6.27e-06, "l1": 9.81e-07, "l2": 1.54e-06}}


def _solve(N):
    import torch
    import paper_1411_4283_gb300 as P
    g = E.sphere_inside_config(N)
    man = E.Manufactured(g, E.sin_product("paper3d"))
    st, _ = build_gpu(g)
    x = torch.zeros(g.ncell, dtype=torch.float64, device="cuda")
    P.eb_solve(st, to_dev(man.lap_avg()), to_dev(man.eb_phi()), to_dev(man.wall_phi_by_id()), x, tol=1e-12)
    err = (x.cpu().numpy() - man.cell_avg()) * (g.flag > 0)
    return P.eb_norms(st, to_dev(err))


def test_sphere_errors_and_order():
    e32 = _solve(32)
    for k in ("linf", "l1", "l2"):
        assert e32[k] == pytest.approx(ORACLE_32[k], rel=1e-6), (k, e32[k])
        assert abs(e32[k] / PRINTED[32][k] - 1) < 0.15
    e64 = _solve(64)
    for k in ("linf", "l1", "l2"):
        assert abs(e64[k] / PRINTED[64][k] - 1) < 0.2, (k, e64[k])
        order = np.log2(e32[k] / e64[k])
        assert 3.5 < order < 4.6, (k, order)

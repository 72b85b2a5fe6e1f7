"""The 2-D convergence-sweep workload on the GPU: the unit square minus the circle r = 0.3 at
(0.51, 0.49) and four seeded circles (radii U[0.05, 0.15], clearance 0.04), phi = sin(2 pi x) cos(3 pi y),
second- and fourth-order stencils, the refined solve to a relative residual of 1e-12.

At N = 128 the GPU solution equals the FP64 oracle's discrete solution (sparse LU of its operator,
stored by tests/golden/make_solve_goldens.py) within 1e-9 of max|phi| at every volume, for Q = 4 and
Q = 2, and so do the Sec. 3.3 error norms (1e-6 relative).  Between N = 128 and 256 the solution error
converges at the stencils' order (Sec. 2.3: the truncation error of the kappa-weighted operator is
O(h^(P-2)) with P = Q + 1, and the paper's circle and four-circle tables show solution errors of order
Q): rates above 3.5 (Q = 4) and 1.7 (Q = 2) in L1 and L2."""
import math
import os

import numpy as np
import pytest

import eb_inputs as E
from gpu_helpers import to_dev

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _solve(N, Q):
    import torch
    import paper_1411_4283_gb300 as P
    g = E.multi_circle_config(N)
    man = E.Manufactured(g, E.sin_product("sin2pix_cos3piy"))
    st = P.eb_build_stencils(P.DeviceGeometry.from_geometry(g), order=Q)
    x = torch.zeros(g.ncell, dtype=torch.float64, device="cuda")
    info = P.eb_solve(st, to_dev(man.lap_avg()), to_dev(man.eb_phi()), to_dev(man.wall_phi_by_id()), x, tol=1e-12)
    xh = x.cpu().numpy()
    nrm = P.eb_norms(st, to_dev((xh - man.cell_avg()) * (g.flag > 0)))
    return g, xh, nrm, info


@pytest.mark.parametrize("Q", [4, 2])
def test_sweep_n128_matches_oracle(Q):
    ref = np.load(os.path.join(GOLD, f"five_circles_n128_q{Q}.npz"))
    g, x, nrm, info = _solve(128, Q)
    cells, phi_o = ref["cells"], ref["phi"]
    assert np.array_equal(np.nonzero(g.flag > 0)[0], cells)
    err = np.abs(x[cells] - phi_o).max()
    assert err <= 1e-9 * np.abs(phi_o).max(), (Q, err, info)
    for k, v in zip(("linf", "l1", "l2"), ref["sol"]):
        assert nrm[k] == pytest.approx(float(v), rel=1e-6), (k, nrm[k], v)


@pytest.mark.parametrize("Q,rate", [(4, 3.5), (2, 1.7)])
def test_sweep_convergence_order(Q, rate):
    e128 = _solve(128, Q)[2]
    e256 = _solve(256, Q)[2]
    for k in ("l1", "l2"):
        r = math.log2(e128[k] / e256[k])
        assert r > rate, (Q, k, r, e128[k], e256[k])

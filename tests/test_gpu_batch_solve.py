"""Batched refined solve (eb_batch_solver_*, BatchSolver): several geometries' systems kappa L phi =
kappa (rho - B g) (Sec. 2.3) solved by the mixed-precision refinement in one graph launch, each loop's
condition set on the device.  Each batched solution equals the single-geometry eb_solve solution to
1e-10 of max|phi| (same arithmetic; the dot products' atomic summation order differs), and the chain
closes at the oracle: the five-circle 128^2 system and the 16^3 box-minus-sphere system of the batch
against the oracle's LU solutions (tests/golden, 1e-9 of max|phi|)."""
import os

import numpy as np
import pytest

import eb_inputs as E
from gpu_helpers import to_dev

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _problem(g):
    man = E.Manufactured(g, E.sin_product("paper3d" if g.dim == 3 else "sin2pix_cos3piy"))
    return to_dev(man.lap_avg()), to_dev(man.eb_phi()), to_dev(man.wall_phi_by_id())


def _run(gs, **kw):
    import torch
    import paper_1411_4283_gb300 as P
    sts = [P.eb_build_stencils(P.DeviceGeometry.from_geometry(g), order=4) for g in gs]
    probs = [_problem(g) for g in gs]
    bs = P.BatchSolver(sts, **{k: v for k, v in kw.items() if k in ("max_outer", "max_inner", "precond")})
    phis = [torch.zeros(g.ncell, dtype=torch.float64, device="cuda") for g in gs]
    infos = bs.solve([p[0] for p in probs], [p[1] for p in probs], [p[2] for p in probs], phis,
                     tol=kw.get("tol", 1e-12), allow_not_converged=kw.get("allow", False))
    return sts, probs, bs, phis, infos


def _single(st, prob, g):
    import torch
    import paper_1411_4283_gb300 as P
    x = torch.zeros(g.ncell, dtype=torch.float64, device="cuda")
    P.eb_solve(st, prob[0], prob[1], prob[2], x, tol=1e-12)
    return x


def test_batch_2d_matches_single_and_oracle():
    gs = [E.multi_circle_config(128), E.circle_config(32), E.circle_config(64, center=(0.45, 0.55), r=0.2),
          E.multi_circle_config(96, seed=3), E.circle_config(256, center=(0.52, 0.47), r=0.27)]
    sts, probs, bs, phis, infos = _run(gs)
    for g, st, pr, x, inf in zip(gs, sts, probs, phis, infos):
        assert inf["rel_residual"] <= 1e-12 and inf["iterations"] > 0
        y = _single(st, pr, g)
        assert (x - y).abs().max().item() <= 1e-10 * y.abs().max().item()
    ref = np.load(os.path.join(GOLD, "five_circles_n128_q4.npz"))
    xo = phis[0].cpu().numpy()[ref["cells"]]
    assert np.abs(xo - ref["phi"]).max() <= 1e-9 * np.abs(ref["phi"]).max()


def test_batch_3d_matches_single_and_oracle():
    gs = [E.sphere_box_config(16, seed=2), E.sphere_box_config(24, seed=2), E.multi_sphere_config(24)]
    sts, probs, bs, phis, infos = _run(gs)
    for g, st, pr, x, inf in zip(gs, sts, probs, phis, infos):
        assert inf["rel_residual"] <= 1e-12
        y = _single(st, pr, g)
        assert (x - y).abs().max().item() <= 1e-10 * y.abs().max().item()
    ref = np.load(os.path.join(GOLD, "sphere_box_n16.npz"))
    xo = phis[0].cpu().numpy()[ref["cells"]]
    assert np.abs(xo - ref["phi"]).max() <= 1e-9 * np.abs(ref["phi"]).max()


def test_batch_solver_reuse_and_jacobi():
    """The same solver solves twice (the second from the first solution: no sweep needed); Jacobi
    preconditioning."""
    gs = [E.circle_config(48), E.multi_circle_config(64, seed=2)]
    sts, probs, bs, phis, infos = _run(gs, precond="jacobi")
    again = bs.solve([p[0] for p in probs], [p[1] for p in probs], [p[2] for p in probs], phis, tol=1e-12)
    for g, st, pr, x, a in zip(gs, sts, probs, phis, again):
        assert a["sweeps"] == 0 and a["rel_residual"] <= 1e-12
        y = _single(st, pr, g)
        assert (x - y).abs().max().item() <= 1e-10 * y.abs().max().item()


def test_batch_caps_report_not_converged():
    """One sweep with a tolerance it cannot reach: EB_ERR_NOT_CONVERGED, every system stopped at the cap
    with a finite iterate and its residual history."""
    import paper_1411_4283_gb300 as P
    gs = [E.circle_config(32), E.circle_config(40)]
    with pytest.raises(P.EbError) as ei:
        _run(gs, max_outer=1, tol=1e-30)
    assert ei.value.code == 4
    sts, probs, bs, phis, infos = _run(gs, max_outer=1, tol=1e-30, allow=True)
    for x, inf in zip(phis, infos):
        assert inf["sweeps"] == 1
        assert np.isfinite(x.cpu().numpy()).all()
        assert len(inf["history"]) == 2 and inf["history"][1] < inf["history"][0]

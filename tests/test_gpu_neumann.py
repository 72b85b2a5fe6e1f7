"""Neumann EB faces on the GPU path: rows b_{f_b p} = (1/m^0) sum_d p_d m^{p-e_d}_d (Sec. 2.2.1) in the
least squares, weighed as in the physical minimum-norm problem, and the flux through a Neumann EB
face taken as its datum |A_f| <g>_f.  Stencils, operator, boundary matrix and refined solution
against the oracle, and the solution error against the paper's circle table (Sec. 3.4, row
'4th order, Neumann EB') at N = 32."""
import json
import os

import numpy as np
import pytest

import eb_inputs as E
from gpu_helpers import compare_stencils, split_boundary, to_dev
from oracle.eb_oracle import Params, run_problem

pytestmark = pytest.mark.gpu
GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")))


@pytest.fixture(scope="module")
def neumann32():
    import paper_1411_4283_gb300 as P
    g = E.circle_config(32)
    man = E.Manufactured(g, E.sin_product("paper2d"))
    bc = np.ones(len(g.cut_cells), np.uint8)
    ref = run_problem(g, man, Params(order=4), bc_eb=bc)
    st = P.eb_build_stencils(P.DeviceGeometry.from_geometry(g, eb_bc=bc), order=4)
    return g, man, ref, st


def test_neumann_stencils(neumann32):
    g, man, ref, st = neumann32
    o = ref["oracle"]
    faces = [f for f in o.flux_faces() if f < o.n_grid_faces]  # Neumann EB faces carry data, not stencils
    compare_stencils(st, o, faces, ref=ref["stencils"])


def test_neumann_operator_and_boundary_matrix(neumann32):
    import torch
    import paper_1411_4283_gb300 as P
    g, man, ref, st = neumann32
    phi = E.seeded_field(13, g.ncell) * (g.flag > 0)
    y = torch.empty(g.ncell, dtype=torch.float64, device="cuda")
    P.eb_apply(st, to_dev(phi), y, kappa_weighted=True)
    yo = g.kappa * (ref["L"] @ phi)
    assert np.linalg.norm(y.cpu().numpy() - yo) <= 1e-12 * np.linalg.norm(yo)
    gw, ge, _ = split_boundary(ref["oracle"], ref["G"])
    Bg = torch.empty(g.ncell, dtype=torch.float64, device="cuda")
    P.eb_bc_rhs(st, to_dev(ge), to_dev(gw), Bg, kappa_weighted=False)
    bo = ref["B"] @ ref["G"]
    bound = 1e-11 * (abs(ref["B"]) @ np.abs(ref["G"]))
    assert np.all(np.abs(Bg.cpu().numpy() - bo) <= bound + 1e-300)


def test_neumann_solve_matches_oracle_and_paper(neumann32):
    import torch
    import paper_1411_4283_gb300 as P
    g, man, ref, st = neumann32
    gw, ge, _ = split_boundary(ref["oracle"], ref["G"])
    x = torch.zeros(g.ncell, dtype=torch.float64, device="cuda")
    info = P.eb_solve(st, to_dev(ref["rho"]), to_dev(ge), to_dev(gw), x, tol=1e-12, mixed=True, precond="jacobi")
    xo = ref["phi"]
    assert np.abs(x.cpu().numpy() - xo).max() <= 1e-9 * np.abs(xo).max(), info
    err = x - to_dev(ref["Phi"])
    nrm = P.eb_norms(st, err * to_dev((g.flag > 0).astype(float)))
    tab = GOLD["circle_r025"]["q4_neumann"]
    assert abs(nrm["linf"] - tab["sol_linf"][0]) <= 0.006 * tab["sol_linf"][0]
    assert abs(nrm["l1"] - tab["sol_l1"][0]) <= 0.006 * tab["sol_l1"][0]

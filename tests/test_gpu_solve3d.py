"""Element-wise parity of the 3-D refined solve with the FP64 oracle's discrete solution.

The oracle's solutions (sparse LU of its kappa-weighted operator, Sec. 2.3) are stored by
tests/golden/make_solve_goldens.py, which calls only oracle/ and eb_inputs/:

* inside the sphere (0.5, 0.5, 0.5), r = 0.45 (the example of Sec. 3.6), Q = 4, N = 32;
* the benchmark geometry, the unit cube minus the sphere r = 0.35 with the seeded centre offset,
  Q = 4, N = 16, with Dirichlet data on the EB and the walls, and with Neumann data on the EB
  (Sec. 2.2.1 Neumann rows; the flux through a Neumann EB face is its datum).

The GPU solves to a relative residual of 1e-12 with both preconditioners (the multigrid V-cycle
with its exact 3x3x3 block solves, which only run in 3-D, and Jacobi), in mixed precision (FP32
BiCGStab refined with the FP64 residual) and in plain FP64, and must agree with the oracle's
solution within 1e-9 of max|phi| at every volume.  The 3-D Neumann build is also compared with the
oracle stencil by stencil on sampled faces (1e-10 of each face's largest coefficient), and its
kappa-weighted FP64 apply row by row on sampled cells (1e-12 of the row's |L||phi|).
"""
import os

import numpy as np
import pytest

import eb_inputs as E
from gpu_helpers import compare_stencils, to_dev
from oracle.eb_oracle import Oracle, Params

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden")

CASES = {
    "sphere_inside_n32": (lambda: E.sphere_inside_config(32), False),
    "sphere_box_n16": (lambda: E.sphere_box_config(16, seed=2), False),
    "sphere_box_n16_neumann": (lambda: E.sphere_box_config(16, seed=2), True),
}
_BUILT = {}


def _problem(name):
    """Geometry, boundary data and the GPU stencils of a case (built once per module)."""
    if name in _BUILT:
        return _BUILT[name]
    import paper_1411_4283_gb300 as P
    mk, neumann = CASES[name]
    g = mk()
    man = E.Manufactured(g, E.sin_product("paper3d"))
    bc = np.ones(len(g.cut_cells), np.uint8) if neumann else None
    st = P.eb_build_stencils(P.DeviceGeometry.from_geometry(g, eb_bc=bc), order=4)
    g_eb = man.eb_dphidn() if neumann else man.eb_phi()
    ref = np.load(os.path.join(GOLD, name + ".npz"))
    _BUILT[name] = (g, man, bc, st, g_eb, ref)
    return _BUILT[name]


@pytest.mark.parametrize("mixed", [True, False], ids=["mixed", "fp64"])
@pytest.mark.parametrize("precond", ["mg", "jacobi"])
@pytest.mark.parametrize("name", list(CASES))
def test_solution_matches_oracle_elementwise(name, precond, mixed):
    import torch
    import paper_1411_4283_gb300 as P
    g, man, bc, st, g_eb, ref = _problem(name)
    x = torch.zeros(g.ncell, dtype=torch.float64, device="cuda")
    info = P.eb_solve(st, to_dev(man.lap_avg()), to_dev(g_eb), to_dev(man.wall_phi_by_id()), x, tol=1e-12,
                      mixed=mixed, precond=precond)
    assert info["rel_residual"] <= 1e-12 * 10
    if precond == "jacobi":
        assert info["precond_blocks"] == 0
    cells, phi_o = ref["cells"], ref["phi"]
    got = x.cpu().numpy()
    assert np.array_equal(np.nonzero(g.flag > 0)[0], cells)
    err = np.abs(got[cells] - phi_o).max()
    assert err <= 1e-9 * np.abs(phi_o).max(), (name, precond, mixed, err, info)
    assert np.all(got[g.flag == 0] == 0.0)
    # the discretisation error the paper reports (Sec. 3.3 norms), through the GPU's own norms
    nrm = P.eb_norms(st, to_dev((got - man.cell_avg()) * (g.flag > 0)))
    for k, v in zip(("linf", "l1", "l2"), ref["sol"]):
        assert nrm[k] == pytest.approx(float(v), rel=1e-6), (k, nrm[k], v)


def test_block_solves_run_in_the_multigrid_preconditioner():
    """At least one of the 3-D cases has cut cells whose high-order diagonal is weak, so the
    exact block solves of the preconditioner are part of the path compared above."""
    import torch
    import paper_1411_4283_gb300 as P
    blocks = {}
    for name in CASES:
        g, man, bc, st, g_eb, ref = _problem(name)
        x = torch.zeros(g.ncell, dtype=torch.float64, device="cuda")
        info = P.eb_solve(st, to_dev(man.lap_avg()), to_dev(g_eb), to_dev(man.wall_phi_by_id()), x, tol=1e-10,
                          precond="mg")
        blocks[name] = info["precond_blocks"]
    assert max(blocks.values()) > 0, blocks


def test_neumann_3d_stencils_and_rows():
    import torch
    import paper_1411_4283_gb300 as P
    g, man, bc, st, g_eb, ref = _problem("sphere_box_n16_neumann")
    o = Oracle(g, Params(order=4), bc_eb=bc)
    rng = np.random.default_rng(7)
    cut = [int(c) for c in g.cut_cells]
    # grid faces of cut cells and of their neighbours (the rows holding Neumann boundary rows)
    faces = set()
    for c in rng.choice(cut, 12, replace=False):
        for fid, _ in o.cell_flux_faces(int(c)):
            if fid < o.n_grid_faces:
                faces.add(int(fid))
    # EB faces carry their datum; their (unused) stencils are not compared
    compare_stencils(st, o, sorted(faces))
    # sampled rows of the kappa-weighted FP64 operator: cut cells and full cells next to them
    phi = E.seeded_field(17, g.ncell) * (g.flag > 0)
    y = torch.empty(g.ncell, dtype=torch.float64, device="cuda")
    P.eb_apply(st, to_dev(phi), y, kappa_weighted=True)
    yg = y.cpu().numpy()
    rows = list(rng.choice(cut, 6, replace=False))
    full_near = [c + 1 for c in cut if c + 1 < g.ncell and g.flag[c + 1] == 1]
    rows += list(rng.choice(full_near, 4, replace=False))
    for c in rows:
        acc, mag = 0.0, 0.0
        for fid, sg in o.cell_flux_faces(int(c)):
            if o._is_neumann(fid):
                continue  # the Neumann EB flux is data (a column of B), not part of L phi
            cols, sv = o.stencil(fid)
            vm = cols >= 0
            acc += sg * float(sv[vm] @ phi[cols[vm]])
            mag += float(np.abs(sv[vm]) @ np.abs(phi[cols[vm]]))
        want = acc / g.h ** 2
        assert abs(yg[c] - want) <= 1e-12 * mag / g.h ** 2 + 1e-300, (c, yg[c], want)

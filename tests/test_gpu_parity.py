"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the same seeded inputs.

Tolerances: stencil coefficients 1e-10 relative to the face's largest coefficient; FP64 kappa-weighted
apply 1e-12 normwise relative; refined solutions 1e-9 relative to max|phi|; FP32 apply 1e-5 normwise
(single precision storage of coefficients and of phi).  The unweighted operator and B divide rows by
kappa (down to ~1e-4), which magnifies cancellation in their sums; they are held componentwise to
|y - y_ref|_i <= 1e-11 (|L| |phi|)_i: the coefficients of the two operators agree to ~1e-12 relative
(the stencils' agreement), plus the rounding of a length-n dot product (n eps, n <= 637).
"""
EPS = 2.220446049250313e-16
import numpy as np
import pytest

import eb_inputs as E
from gpu_helpers import build_gpu, compare_stencils, sample_faces, split_boundary, to_dev
from oracle.eb_oracle import Oracle, Params, run_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def circle32():
    g = E.circle_config(32, center=(0.51, 0.49), r=0.3)
    man = E.Manufactured(g, E.sin_product("sin2pix_cos3piy"))
    ref = run_problem(g, man, Params(order=4))
    return g, man, ref


def test_library_loaded():
    import paper_1411_4283_gb300 as P
    assert P.load().eb_abi_version() == 3


@pytest.mark.parametrize("Q", [4, 2])
def test_all_stencils_2d(Q):
    g = E.circle_config(32, center=(0.51, 0.49), r=0.3)
    o = Oracle(g, Params(order=Q))
    st, _ = build_gpu(g, order=Q)
    compare_stencils(st, o, o.flux_faces())


def test_wall_face_order(circle32):
    import paper_1411_4283_gb300 as P
    g, man, ref = circle32
    st, _ = build_gpu(g)
    _, _, walls = split_boundary(ref["oracle"], ref["G"])
    assert np.array_equal(P.eb_wall_faces(st), np.array(walls))


@pytest.mark.parametrize("kw", [False, True])
def test_apply_fp64_2d(circle32, kw):
    import torch
    import paper_1411_4283_gb300 as P
    g, man, ref = circle32
    st, _ = build_gpu(g)
    phi = E.seeded_field(11, g.ncell) * (g.flag > 0)
    y = torch.empty(g.ncell, dtype=torch.float64, device="cuda")
    P.eb_apply(st, to_dev(phi), y, kappa_weighted=kw)
    yo = ref["L"] @ phi
    if kw:
        yo = g.kappa * yo
    yg = y.cpu().numpy()
    if kw:
        assert np.linalg.norm(yg - yo) <= 1e-12 * np.linalg.norm(yo)
    else:
        bound = 1e-11 * (abs(ref["L"]) @ np.abs(phi))
        assert np.all(np.abs(yg - yo) <= bound + 1e-300)
    assert np.all(yg[g.flag == 0] == 0)


def test_apply_fp32_2d(circle32):
    import torch
    import paper_1411_4283_gb300 as P
    g, man, ref = circle32
    st, _ = build_gpu(g)
    phi = E.seeded_field(12, g.ncell) * (g.flag > 0)
    y = torch.empty(g.ncell, dtype=torch.float32, device="cuda")
    P.eb_apply(st, to_dev(phi, torch.float32), y, kappa_weighted=True)
    yo = g.kappa * (ref["L"] @ phi)
    assert np.linalg.norm(y.cpu().numpy() - yo) <= 1e-5 * np.linalg.norm(yo)


def test_bc_rhs_2d(circle32):
    import torch
    import paper_1411_4283_gb300 as P
    g, man, ref = circle32
    st, _ = build_gpu(g)
    gw, ge, _ = split_boundary(ref["oracle"], ref["G"])
    Bg = torch.empty(g.ncell, dtype=torch.float64, device="cuda")
    P.eb_bc_rhs(st, to_dev(ge), to_dev(gw), Bg, kappa_weighted=False)
    bo = ref["B"] @ ref["G"]
    bound = 1e-11 * (abs(ref["B"]) @ np.abs(ref["G"]))
    assert np.all(np.abs(Bg.cpu().numpy() - bo) <= bound + 1e-300)


@pytest.mark.parametrize("mixed,precond", [(True, "mg"), (False, "mg"), (True, "jacobi"), (False, "jacobi")])
def test_solve_2d(circle32, mixed, precond):
    import torch
    import paper_1411_4283_gb300 as P
    g, man, ref = circle32
    st, _ = build_gpu(g)
    gw, ge, _ = split_boundary(ref["oracle"], ref["G"])
    x = torch.zeros(g.ncell, dtype=torch.float64, device="cuda")
    info = P.eb_solve(st, to_dev(ref["rho"]), to_dev(ge), to_dev(gw), x, tol=1e-12, mixed=mixed, precond=precond)
    xo = ref["phi"]
    assert np.abs(x.cpu().numpy() - xo).max() <= 1e-9 * np.abs(xo).max(), info
    err = x - to_dev(ref["Phi"])
    nrm = P.eb_norms(st, err * to_dev((g.flag > 0).astype(float)))
    assert nrm["linf"] == pytest.approx(ref["sol"]["linf"], rel=1e-6)
    assert nrm["l1"] == pytest.approx(ref["sol"]["l1"], rel=1e-6)


def test_no_embedded_boundary_box():
    """Degenerate geometry: no body at all -- only interior template faces and wall classes."""
    g = E.Geometry(2, 24, np.zeros((0, 3)), np.zeros(0), False, 4, name="box")
    o = Oracle(g, Params(order=4))
    st, _ = build_gpu(g)
    assert st.info["n_unique_faces"] == 0
    compare_stencils(st, o, o.flux_faces()[::3])


def test_sampled_stencils_3d():
    g = E.sphere_box_config(20)
    o = Oracle(g, Params(order=4))
    st, _ = build_gpu(g)
    compare_stencils(st, o, sample_faces(o, 60, seed=2))


def _row_sample_cells(g, order, rng):
    """Cut cells, full cells next to the EB, interior cells, cells in the wall layers (among them cells
    of the aligned x-runs of the wall-layer pass) and cells next to the first and last grid rows (the
    clamped path of the irregular pass)."""
    n = g.N
    R = 3 if order == 4 else 2
    L = R + 1
    full = np.nonzero(g.flag == 1)[0]
    x, y, z = full % n, (full // n) % n, full // (n * n)
    wall = full[(np.minimum(np.minimum(x, y), z) < L + 1) | (np.maximum(np.maximum(x, y), z) > n - L - 2)]
    edge = full[((y <= L) & (z <= L) & (x < L)) | ((y >= n - 1 - L) & (z >= n - 1 - L) & (x > n - 1 - L))]
    interior = full[(np.minimum(np.minimum(x, y), z) > L + 1) & (np.maximum(np.maximum(x, y), z) < n - L - 2)]
    cut = set(int(c) for c in g.cut_cells)
    near = [int(c) for c in interior if any((int(c) + d) in cut for d in (1, -1, n, -n, n * n, -n * n))]
    wx = wall % n
    runs = wall[(wx >= 8) & (wx <= n - 9)]
    pick = []
    for pool, k in ((g.cut_cells, 8), (near, 6), (interior, 4), (wall, 8), (edge, 4), (runs, 8)):
        pool = np.asarray(pool)
        if len(pool):
            pick += [int(c) for c in rng.choice(pool, min(k, len(pool)), replace=False)]
    return sorted(set(pick))


@pytest.mark.parametrize("order", [4, 2])
def test_apply_3d_sampled_rows(order):
    """Operator rows at sampled cells: (L phi)_v assembled by the oracle from the cell's own face
    stencils, against the GPU apply of the whole field.  FP64: 1e-12 of sum_f max|s_f| sum|phi_cols| / h^2
    (the stencils of both sides are exact to rounding, about cond(WA) eps = 1e-14 .. 3e-13 of each face's
    largest coefficient against a 40-digit reference, the oracle's SVD included; the row value itself
    can cancel to a few thousandths of those terms).  FP32: 1e-5 of the field's row scale."""
    import torch
    import paper_1411_4283_gb300 as P
    g = E.sphere_box_config(20)
    o = Oracle(g, Params(order=order))
    st, _ = build_gpu(g, order=order)
    phi = E.seeded_field(21, g.ncell) * (g.flag > 0)
    y = torch.empty(g.ncell, dtype=torch.float64, device="cuda")
    P.eb_apply(st, to_dev(phi), y, kappa_weighted=True)
    yg = y.cpu().numpy()
    y32 = torch.empty(g.ncell, dtype=torch.float32, device="cuda")
    P.eb_apply(st, to_dev(phi, torch.float32), y32, kappa_weighted=True)
    yg32 = y32.cpu().numpy().astype(np.float64)
    scale = np.abs(yg).max()
    for c in _row_sample_cells(g, order, np.random.default_rng(4)):
        acc = 0.0
        bound = 0.0
        for fid, sg in o.cell_flux_faces(c):
            cols, s = o.stencil(fid)
            vm = cols >= 0
            acc += sg * float(s[vm] @ phi[cols[vm]])
            bound += np.abs(s).max() * np.abs(phi[cols[vm]]).sum()
        acc /= g.h ** 2
        bound /= g.h ** 2
        assert abs(yg[c] - acc) <= 1e-12 * bound, (c, yg[c], acc, bound)
        assert abs(yg32[c] - acc) <= 1e-5 * scale, (c, yg32[c], acc)


def test_apply_q2_2d():
    """Second-order (Q = 2, R_n = 2) operator in 2-D against the oracle's assembled operator."""
    import torch
    import paper_1411_4283_gb300 as P
    g = E.circle_config(32, center=(0.51, 0.49), r=0.3)
    man = E.Manufactured(g, E.sin_product("sin2pix_cos3piy"))
    ref = run_problem(g, man, Params(order=2))
    st, _ = build_gpu(g, order=2)
    phi = E.seeded_field(12, g.ncell) * (g.flag > 0)
    y = torch.empty(g.ncell, dtype=torch.float64, device="cuda")
    P.eb_apply(st, to_dev(phi), y, kappa_weighted=True)
    yo = (ref["L"] @ phi) * g.kappa
    yg = y.cpu().numpy()
    assert np.linalg.norm(yg - yo) <= 1e-12 * np.linalg.norm(yo)


def test_preconditioner_3d_same_solution_few_iterations():
    """The multigrid preconditioner (V-cycle + local block solves at weak-diagonal cut cells) changes
    the path, not the answer: the refined solution equals the Jacobi-preconditioned one to the
    refinement tolerance, in far fewer iterations."""
    import torch
    import paper_1411_4283_gb300 as P
    g = E.sphere_box_config(40)
    man = E.Manufactured(g, E.sin_product("paper3d"))
    st, _ = build_gpu(g)
    rho, geb, gw = to_dev(man.lap_avg()), to_dev(man.eb_phi()), to_dev(man.wall_phi_by_id())
    out = {}
    for pc in ("mg", "jacobi"):
        phi = torch.zeros(g.ncell, dtype=torch.float64, device="cuda")
        info = P.eb_solve(st, rho, geb, gw, phi, tol=1e-11, mixed=True, precond=pc)
        assert info["status"] == "EB_OK"
        out[pc] = (phi.cpu().numpy(), info["iterations"])
    (a, it_mg), (b, it_j) = out["mg"], out["jacobi"]
    assert np.abs(a - b).max() <= 1e-9 * np.abs(b).max()
    assert it_mg <= 40 and it_mg * 4 <= it_j, (it_mg, it_j)

"""Shape gradients on the GPU for radii and level-set modes (eb_adjoint_shape,
paper_1411_4283_gb300.adjoint.shape_objective), 2-D and 3-D.

J = 1/2 sum |V| phi^2 with kappa L phi = kappa and homogeneous Dirichlet data (Sec. 2.3); a level-set
mode a sin(2 pi k . x + theta) added to the bodies' distance function moves the boundary with the
normal speed -sin(2 pi k . x + theta) at a = 0.  The device's moment-table derivatives (transport
theorem on the patch, edge and rim terms) against the adjoint oracle's (oracle/eb_adjoint.py,
independent patch and edge quadratures) table by table; dJ against the oracle's adjoint (2-D run
here; 3-D from tests/golden/adjoint3d_goldens.npz, written by make_adjoint_goldens.py from the oracle
only), against central differences of the GPU's own forward problem, and, at the shape-gradient
workload's size (eight spheres, 128^3), against the invariant that the mode k = 0, theta = -pi/2
(unit speed on every body) has the derivative sum_b dJ/dr_b."""
import math
import os

import numpy as np
import pytest

import eb_inputs as E
from oracle.eb_oracle import Oracle, Params

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden")
EPS = 1e-6


def _tables_match(G, dm, body, mode, dim):
    names = ("vol_mom", "eb_mom", "eb_nmom")
    for nm, want in zip(names, dm[:3]):
        got = G.shape_table(nm, body=body, mode=mode)
        assert got.shape == want.shape, nm
        assert np.abs(got - want).max() <= 1e-10 * max(1.0, np.abs(want).max()), (nm, np.abs(got - want).max())
    for d in range(dim):
        got = G.shape_table("face_mom", body=body, mode=mode, d=d)
        want = dm[3][d]
        assert got.shape == want.shape
        assert np.abs(got - want).max() <= 1e-10 * max(1.0, np.abs(want).max()), (d, np.abs(got - want).max())


@pytest.mark.parametrize("name", ["sphere_box_n16", "eight_spheres_n24"])
def test_sphere_derivative_tables_match_oracle(name):
    """3-D: radius and mode derivatives of every table against sphere_moment_derivatives and
    sphere_velocity_derivatives (fourier_mode_derivatives), 1e-10 of the table's size."""
    import paper_1411_4283_gb300 as P
    from oracle.eb_adjoint import fourier_mode_derivatives, sphere_moment_derivatives
    g = E.sphere_box_config(16, seed=2) if name == "sphere_box_n16" else E.multi_sphere_config(24)
    G = P.eb_geometry_spheres(g.N, g.centers, g.radii, moment_degree=4)
    o = Oracle(g, Params(order=4))
    b = len(g.radii) - 1
    _tables_match(G, sphere_moment_derivatives(o, b), b, None, 3)
    mode = E.level_set_modes(16, seed=5)[0]
    _tables_match(G, fourier_mode_derivatives(o, mode[:3], mode[3]), 0, mode, 3)


def test_circle_derivative_tables_match_oracle():
    """2-D: the same for two circles (radius of the second; a mode over both)."""
    import paper_1411_4283_gb300 as P
    from oracle.eb_adjoint import circle_moment_derivatives, fourier_mode_derivatives
    cen, rad = [(0.31, 0.29), (0.69, 0.66)], [0.13, 0.17]
    g = E.Geometry(2, 24, np.array([[c[0], c[1], 0.0] for c in cen]), np.array(rad), False, 4)
    G = P.eb_geometry_circles(24, cen, rad, moment_degree=4)
    o = Oracle(g, Params(order=4))
    _tables_match(G, circle_moment_derivatives(o, 1), 1, None, 2)
    mode = np.array([2.0, 3.0, 0.0, 0.7])
    _tables_match(G, fourier_mode_derivatives(o, mode[:2], mode[3]), 0, mode, 2)


def test_circle_mode_gradient_matches_oracle():
    """2-D dJ/da for two modes and dJ/dr in one call, against the adjoint oracle (1e-6)."""
    import torch
    from oracle.eb_adjoint import fourier_mode_derivatives, objective_and_radius_gradient
    from paper_1411_4283_gb300.adjoint import shape_objective
    cen, rad = [(0.31, 0.29), (0.69, 0.66)], [0.13, 0.17]
    g = E.Geometry(2, 20, np.array([[c[0], c[1], 0.0] for c in cen]), np.array(rad), False, 4)
    modes = np.array([[2.0, 3.0, 0.0, 0.7], [1.0, 4.0, 0.0, 2.9]])
    r = torch.tensor(rad, dtype=torch.float64, requires_grad=True)
    a = torch.zeros(2, dtype=torch.float64, requires_grad=True)
    J = shape_objective(r, 20, cen, amplitudes=a, modes=modes)
    J.backward()
    for m in range(2):
        Jo, dJo = objective_and_radius_gradient(
            g, 0, Params(order=4), derivs=lambda o: fourier_mode_derivatives(o, modes[m, :2], modes[m, 3]))
        assert abs(J.item() - Jo) <= 1e-9 * abs(Jo)
        assert abs(a.grad[m].item() - dJo) <= 1e-6 * abs(dJo), (m, a.grad[m].item(), dJo)
    Jo, dJo = objective_and_radius_gradient(g, 0, Params(order=4))
    assert abs(r.grad[0].item() - dJo) <= 1e-6 * abs(dJo)


@pytest.mark.parametrize("name", ["sphere_box_n8", "two_spheres_n10"])
def test_sphere_gradients_match_oracle_goldens(name):
    """3-D J and dJ (radius, modes) against the oracle's stored values (1e-9 and 1e-6)."""
    import paper_1411_4283_gb300 as P
    from paper_1411_4283_gb300.adjoint import _forward
    ref = np.load(os.path.join(GOLD, "adjoint3d_goldens.npz"))
    g = E.sphere_box_config(8, seed=2) if name == "sphere_box_n8" else E.multi_sphere_config(10, n=2)
    kinds, params, dJo = ref[name + "_kind"], ref[name + "_param"], ref[name + "_dJ"]
    modes = params[kinds == 1]
    G, st, phi = _forward(g.radii, g.N, [tuple(c) for c in g.centers], 4, 1e-12)
    J, dr, da = P.eb_adjoint_shape(G, st, phi, modes)
    assert abs(J - float(ref[name + "_J"])) <= 1e-9 * abs(float(ref[name + "_J"]))
    im = 0
    for k, p, want in zip(kinds, params, dJo):
        got = dr[int(p[0])] if k == 0 else da[im]
        im += k == 1
        assert abs(got - want) <= 1e-6 * abs(want), (name, k, p, got, want)


def test_sphere_radius_gradient_against_central_differences():
    """The benchmark geometry at 24^3: dJ/dr through the autograd wrapper against central differences
    of the GPU forward problem (device moments at r +- 1e-6, same cut sets)."""
    import torch
    import paper_1411_4283_gb300 as P
    from paper_1411_4283_gb300.adjoint import shape_objective
    g = E.sphere_box_config(24, seed=2)
    cen = [tuple(c) for c in g.centers]
    for s in (-1, 1):
        G = P.eb_geometry_spheres(24, cen, [g.radii[0] + s * EPS], moment_degree=4)
        assert np.array_equal(G.table("cut_cells"), g.cut_cells)
    r = torch.tensor(g.radii, dtype=torch.float64, requires_grad=True)
    J = shape_objective(r, 24, cen)
    J.backward()
    with torch.no_grad():
        Jp = shape_objective(r.detach() + EPS, 24, cen).item()
        Jm = shape_objective(r.detach() - EPS, 24, cen).item()
    fd = (Jp - Jm) / (2 * EPS)
    assert abs(r.grad[0].item() - fd) <= 1e-5 * abs(fd), (r.grad[0].item(), fd)


@pytest.mark.parametrize("N", [64, 128])
def test_eight_spheres_uniform_mode_is_the_sum_of_radius_derivatives(N):
    """The shape-gradient workload (eight seeded spheres, 16 seeded modes, plus the mode k = 0,
    theta = -pi/2, whose speed is 1 on every body) at N^3: the uniform mode's derivative equals
    sum_b dJ/dr_b (the two go through different velocity kernels), 1e-9; all derivatives finite."""
    import paper_1411_4283_gb300 as P
    from paper_1411_4283_gb300.adjoint import _forward
    g = E.multi_sphere_config(N)
    modes = np.vstack([E.level_set_modes(16, seed=5), [[0.0, 0.0, 0.0, -0.5 * math.pi]]])
    G, st, phi = _forward(g.radii, N, [tuple(c) for c in g.centers], 4, 1e-12)
    J, dr, da = P.eb_adjoint_shape(G, st, phi, modes)
    assert np.all(np.isfinite(dr)) and np.all(np.isfinite(da)) and J > 0
    assert abs(da[-1] - dr.sum()) <= 1e-9 * np.abs(dr).sum(), (da[-1], dr.sum())
    assert np.all(dr < 0)  # a growing body shrinks the domain and |phi| (Dirichlet data zero)

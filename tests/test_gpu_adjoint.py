"""The adjoint on the GPU (eb_adjoint_radii, paper_1411_4283_gb300.adjoint): the derivative of
J = 1/2 sum |V| phi^2 (kappa L phi = kappa, homogeneous Dirichlet data, Sec. 2.3) with respect to the
radii of circles, through the transposed solve, the reverse-mode derivative of every stencil solve
(Sec. 2.2.1) and the moment tables' shape derivatives recomputed on the device.  Against the adjoint
oracle (oracle/eb_adjoint.py: LU solves, SVD stencils, complex-step row derivatives) and against central
differences of the GPU's own forward problem; through torch.autograd."""
import numpy as np
import pytest

import eb_inputs as E
from oracle.eb_adjoint import objective_and_radius_gradient
from oracle.eb_oracle import Params

pytestmark = pytest.mark.gpu

EPS = 1e-6


def test_radius_gradient_matches_adjoint_oracle():
    import torch
    from paper_1411_4283_gb300.adjoint import circle_objective
    g = E.circle_config(16, center=(0.51, 0.49), r=0.3)
    Jo, dJo = objective_and_radius_gradient(g, 0, Params(order=4))
    r = torch.tensor([0.3], dtype=torch.float64, requires_grad=True)
    J = circle_objective(r, 16, [(0.51, 0.49)])
    J.backward()
    assert abs(J.item() - Jo) <= 1e-9 * abs(Jo)
    assert abs(r.grad.item() - dJo) <= 1e-6 * abs(dJo), (r.grad.item(), dJo)


def test_two_circles_gradient_matches_oracle_and_differences():
    """Both radii at once (one adjoint solve); the second circle's derivative also against central
    differences of the GPU forward problem (the cut sets of r +- 1e-6 are the same)."""
    import torch
    from paper_1411_4283_gb300.adjoint import circle_objective
    cen = [(0.31, 0.29), (0.69, 0.66)]
    rad = [0.13, 0.17]
    g = E.Geometry(2, 20, np.array([[c[0], c[1], 0.0] for c in cen]), np.array(rad), False, 4)
    r = torch.tensor(rad, dtype=torch.float64, requires_grad=True)
    J = circle_objective(r, 20, cen)
    J.backward()
    for b in range(2):
        Jo, dJo = objective_and_radius_gradient(g, b, Params(order=4))
        assert abs(J.item() - Jo) <= 1e-9 * abs(Jo)
        assert abs(r.grad[b].item() - dJo) <= 1e-6 * abs(dJo), (b, r.grad[b].item(), dJo)
    with torch.no_grad():
        Jp = circle_objective(torch.tensor([0.13, 0.17 + EPS], dtype=torch.float64), 20, cen).item()
        Jm = circle_objective(torch.tensor([0.13, 0.17 - EPS], dtype=torch.float64), 20, cen).item()
    fd = (Jp - Jm) / (2 * EPS)
    assert abs(r.grad[1].item() - fd) <= 1e-5 * abs(fd), (r.grad[1].item(), fd)


def test_second_order_stencils_gradient():
    """Q = 2 (K = 6): the same chain with the second-order stencils, against central differences."""
    import torch
    from paper_1411_4283_gb300.adjoint import circle_objective
    r = torch.tensor([0.3], dtype=torch.float64, requires_grad=True)
    J = circle_objective(r, 32, [(0.51, 0.49)], order=2)
    J.backward()
    with torch.no_grad():
        Jp = circle_objective(torch.tensor([0.3 + EPS], dtype=torch.float64), 32, [(0.51, 0.49)], order=2).item()
        Jm = circle_objective(torch.tensor([0.3 - EPS], dtype=torch.float64), 32, [(0.51, 0.49)], order=2).item()
    fd = (Jp - Jm) / (2 * EPS)
    assert abs(r.grad.item() - fd) <= 1e-5 * abs(fd), (r.grad.item(), fd)

"""Gradient of a solution functional with respect to geometry parameters, behind
``torch.autograd.Function``: the radii of the circles of the unit square minus circles.

Forward (all on the device): the moment tables of the geometry (eb_geometry_circles, Sec. 2.1),
the stencils and operator (Sec. 2.2-2.4), the refined solve of kappa L phi = kappa rho with rho = 1
and homogeneous Dirichlet data (Sec. 2.3), and J = 1/2 sum_v |V_v| phi_v^2.  Backward: the
hand-written adjoint of the solve and of every stencil solve (eb_adjoint_radii); the moment tables'
shape derivatives are recomputed on the device, not stored.
"""
from __future__ import annotations

import torch

from . import eb_adjoint_radii, eb_build_stencils, eb_geometry_circles, eb_solve, eb_wall_faces


def _forward(radii_np, N, centers, order, tol):
    G = eb_geometry_circles(N, centers, radii_np, moment_degree=4)
    st = eb_build_stencils(G, order=order)
    f64 = dict(dtype=torch.float64, device="cuda")
    rho = torch.ones(st.ncell, **f64)
    g_eb = torch.zeros(max(G.n_cut, 1), **f64)
    g_wall = torch.zeros(max(len(eb_wall_faces(st)), 1), **f64)
    phi = torch.zeros(st.ncell, **f64)
    eb_solve(st, rho, g_eb, g_wall, phi, tol=tol)
    return G, st, phi


class CircleObjective(torch.autograd.Function):
    """J(r) = 1/2 sum_v |V_v| phi_v^2 on an N x N grid of the unit square minus circles with the given
    centres and radii r (a 1-D tensor); dJ/dr by the adjoint."""

    @staticmethod
    def forward(ctx, radii, N, centers, order, tol):
        G, st, phi = _forward(radii.detach().double().cpu().numpy(), N, centers, order, tol)
        J, _ = eb_adjoint_radii(G, st, phi, gradient=False)
        ctx.state = (G, st, phi)
        return torch.tensor(J, dtype=torch.float64, device=radii.device)

    @staticmethod
    def backward(ctx, gJ):
        G, st, phi = ctx.state
        _, dJ = eb_adjoint_radii(G, st, phi)
        ctx.state = None
        return gJ * torch.as_tensor(dJ, dtype=gJ.dtype, device=gJ.device), None, None, None, None


def circle_objective(radii, N, centers, order=4, tol=1e-12):
    """J as a differentiable function of the radii (torch tensor of the circles' radii)."""
    return CircleObjective.apply(radii, N, centers, order, tol)

"""Gradient of a solution functional with respect to geometry parameters, behind
``torch.autograd.Function``: the radii of the bodies of the unit square minus circles or the unit
cube minus spheres, and the amplitudes of level-set modes added to the bodies' distance function.

Forward (all on the device): the moment tables of the geometry (eb_geometry_circles or
eb_geometry_spheres, Sec. 2.1), the stencils and operator (Sec. 2.2-2.4), the refined solve of
kappa L phi = kappa rho with rho = 1 and homogeneous Dirichlet data (Sec. 2.3), and
J = 1/2 sum_v |V_v| phi_v^2.  Backward: the hand-written adjoint of the solve and of every stencil
solve (eb_adjoint_shape); the moment tables' shape derivatives are recomputed on the device, not
stored.  The level-set modes a_m sin(2 pi k_m . x + theta_m) enter at a = 0 only: the device
geometry holds circles and spheres, so the forward problem is the unperturbed one and the mode
amplitudes' gradient is exact there.
"""
from __future__ import annotations

import torch

from . import (eb_adjoint_shape, eb_build_stencils, eb_geometry_circles, eb_geometry_spheres, eb_solve,
               eb_wall_faces)


def _forward(radii_np, N, centers, order, tol):
    make = eb_geometry_circles if len(centers[0]) == 2 else eb_geometry_spheres
    G = make(N, centers, radii_np, moment_degree=4)
    st = eb_build_stencils(G, order=order)
    f64 = dict(dtype=torch.float64, device="cuda")
    rho = torch.ones(st.ncell, **f64)
    g_eb = torch.zeros(max(G.n_cut, 1), **f64)
    g_wall = torch.zeros(max(len(eb_wall_faces(st)), 1), **f64)
    phi = torch.zeros(st.ncell, **f64)
    eb_solve(st, rho, g_eb, g_wall, phi, tol=tol)
    return G, st, phi


class ShapeObjective(torch.autograd.Function):
    """J(r, a) = 1/2 sum_v |V_v| phi_v^2 on an N^D grid of the unit box minus the bodies with the given
    centres (2 or 3 coordinates each) and radii r, the boundary moved by the level-set modes `modes`
    (rows k_x, k_y, k_z, theta) with amplitudes a, which must be zero; dJ/dr and dJ/da by the adjoint."""

    @staticmethod
    def forward(ctx, radii, amplitudes, N, centers, modes, order, tol):
        if amplitudes.numel() and bool(torch.any(amplitudes != 0)):
            raise ValueError("the level-set modes are evaluated at zero amplitude only")
        G, st, phi = _forward(radii.detach().double().cpu().numpy(), N, centers, order, tol)
        J, _, _ = eb_adjoint_shape(G, st, phi, modes, gradient=False)
        ctx.state = (G, st, phi, modes)
        return torch.tensor(J, dtype=torch.float64, device=radii.device)

    @staticmethod
    def backward(ctx, gJ):
        G, st, phi, modes = ctx.state
        _, dr, da = eb_adjoint_shape(G, st, phi, modes)
        ctx.state = None
        grad_r = gJ * torch.as_tensor(dr, dtype=gJ.dtype, device=gJ.device)
        grad_a = gJ * torch.as_tensor(da, dtype=gJ.dtype, device=gJ.device)
        return grad_r, grad_a, None, None, None, None, None


def shape_objective(radii, N, centers, amplitudes=None, modes=(), order=4, tol=1e-12):
    """J as a differentiable function of the bodies' radii (torch tensor) and of the amplitudes of the
    level-set modes (torch tensor of zeros, one per row of modes)."""
    if amplitudes is None:
        amplitudes = torch.zeros(len(modes), dtype=torch.float64, device=radii.device)
    return ShapeObjective.apply(radii, amplitudes, N, [tuple(c) for c in centers], modes, order, tol)


def circle_objective(radii, N, centers, order=4, tol=1e-12):
    """J as a differentiable function of the radii of circles (2-D centres)."""
    return shape_objective(radii, N, centers, order=order, tol=tol)

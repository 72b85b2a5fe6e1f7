"""Pins of the adjoint oracle (oracle/eb_adjoint.py) against central finite differences of what it
differentiates: the geometry generator's moment tables, and the whole forward problem (moments ->
stencils -> operator -> solve -> J), for the radius of a circle in the unit square."""
import math

import numpy as np
import pytest

import eb_inputs as E
from oracle.eb_adjoint import circle_moment_derivatives, objective_and_radius_gradient
from oracle.eb_oracle import Oracle, Params

EPS = 1e-6


def _pair(N, center, r, **kw):
    g = E.circle_config(N, center=center, r=r, **kw)
    gp = E.circle_config(N, center=center, r=r + EPS, **kw)
    gm = E.circle_config(N, center=center, r=r - EPS, **kw)
    assert np.array_equal(gp.cut_cells, g.cut_cells) and np.array_equal(gm.cut_cells, g.cut_cells)
    for d in range(2):
        assert np.array_equal(gp.cut_faces[d], g.cut_faces[d]) and np.array_equal(gm.cut_faces[d], g.cut_faces[d])
    return g, gp, gm


def test_moment_shape_derivatives():
    """Transport-theorem volume derivatives, arc derivatives of the EB moments (with the endpoints
    sliding along the cell edges) and chord-end derivatives of the face moments, against central
    differences of the generator's moments (relative to each table's largest derivative)."""
    g, gp, gm = _pair(16, (0.51, 0.49), 0.3)
    dvol, deb, debn, dface = circle_moment_derivatives(Oracle(g, Params(order=4)), 0)
    pairs = [(dvol, gp.vol_mom, gm.vol_mom), (deb, gp.eb_mom, gm.eb_mom), (debn, gp.eb_nmom, gm.eb_nmom)]
    pairs += [(dface[d], gp.face_mom[d], gm.face_mom[d]) for d in range(2)]
    for an, a, b in pairs:
        fd = (a - b) / (2 * EPS)
        assert np.abs(an - fd).max() <= 1e-7 * np.abs(fd).max()


def test_radius_gradient_adjoint_against_central_differences():
    """dJ/dr through the solve adjoint and the LS-build adjoint against central differences of J."""
    g, gp, gm = _pair(16, (0.51, 0.49), 0.3)
    J, dJ = objective_and_radius_gradient(g)
    fd = (objective_and_radius_gradient(gp)[0] - objective_and_radius_gradient(gm)[0]) / (2 * EPS)
    assert J > 0
    assert abs(dJ - fd) <= 1e-6 * abs(fd)


def test_sphere_moment_shape_derivatives():
    """3-D: the sphere patch's derivative (mean curvature 2/r, the normal derivative from the
    generator's higher-degree patch moments, and the patch edges sliding on the cell faces with the
    conormal speed), the transport-theorem volume derivatives and the face disks' rims, against
    central differences of the generator's moments."""
    from oracle.eb_adjoint import sphere_moment_derivatives
    mk = lambda r: E.Geometry(3, 8, np.array([[0.503, 0.497, 0.501]]), np.array([r]), False, 4)
    g, gp, gm = mk(0.3), mk(0.3 + EPS), mk(0.3 - EPS)
    assert np.array_equal(gp.cut_cells, g.cut_cells) and np.array_equal(gm.cut_cells, g.cut_cells)
    dvol, deb, debn, dface = sphere_moment_derivatives(Oracle(g, Params(order=4)), 0)
    pairs = [(dvol, gp.vol_mom, gm.vol_mom), (deb, gp.eb_mom, gm.eb_mom), (debn, gp.eb_nmom, gm.eb_nmom)]
    for d in range(3):
        assert np.array_equal(gp.cut_faces[d], g.cut_faces[d]) and np.array_equal(gm.cut_faces[d], g.cut_faces[d])
        pairs.append((dface[d], gp.face_mom[d], gm.face_mom[d]))
    for an, a, b in pairs:
        fd = (a - b) / (2 * EPS)
        assert np.abs(an - fd).max() <= 1e-7 * np.abs(fd).max()


def test_radius_gradient_two_circles():
    """Two circles: the derivative with respect to the second circle's radius moves only the cells and
    faces that circle cuts (the first circle's tables are held), against central differences."""
    from oracle.eb_adjoint import objective_and_radius_gradient as grad
    cen = np.array([[0.31, 0.29, 0.0], [0.69, 0.66, 0.0]])
    mk = lambda r2: E.Geometry(2, 20, cen, np.array([0.13, r2]), False, 4)
    g, gp, gm = mk(0.17), mk(0.17 + EPS), mk(0.17 - EPS)
    assert np.array_equal(gp.cut_cells, g.cut_cells) and np.array_equal(gm.cut_cells, g.cut_cells)
    J, dJ = grad(g, body=1)
    fd = (grad(gp, body=1)[0] - grad(gm, body=1)[0]) / (2 * EPS)
    assert abs(dJ - fd) <= 1e-6 * abs(fd)


def test_sphere_moment_derivatives_eight_spheres():
    """The eight-sphere geometry: the derivative with respect to one sphere's radius moves only the
    cells and faces that sphere cuts, against central differences of the generator."""
    from oracle.eb_adjoint import sphere_moment_derivatives
    g = E.multi_sphere_config(24)
    for b in range(len(g.radii)):  # the first sphere whose cut cells and faces survive +-EPS
        rp, rm = g.radii.copy(), g.radii.copy()
        rp[b] += EPS
        rm[b] -= EPS
        gp = E.Geometry(3, 24, g.centers, rp, False, 4)
        gm = E.Geometry(3, 24, g.centers, rm, False, 4)
        if all(np.array_equal(x.cut_cells, g.cut_cells) for x in (gp, gm)) and all(
                np.array_equal(x.cut_faces[d], g.cut_faces[d]) for x in (gp, gm) for d in range(3)):
            break
    else:
        pytest.fail("every sphere changes the cut sets under +-EPS")
    dvol, deb, debn, dface = sphere_moment_derivatives(Oracle(g, Params(order=4)), b)
    pairs = [(dvol, gp.vol_mom, gm.vol_mom), (deb, gp.eb_mom, gm.eb_mom), (debn, gp.eb_nmom, gm.eb_nmom)]
    for d in range(3):
        assert np.array_equal(gp.cut_faces[d], g.cut_faces[d]) and np.array_equal(gm.cut_faces[d], g.cut_faces[d])
        pairs.append((dface[d], gp.face_mom[d], gm.face_mom[d]))
    for an, a, bb in pairs:
        fd = (a - bb) / (2 * EPS)
        assert np.abs(an - fd).max() <= 1e-7 * np.abs(fd).max()
    assert np.all(deb[g.cut_body != b] == 0) and np.any(deb[g.cut_body == b] != 0)


def _translation_velocity(c, r, t):
    """Normal speed and gradient of a translation t of the body centred at c (radius r): V = N . t."""
    def V(x):
        return (((x - c[:, None]) / r) * t[:, None]).sum(0)

    def gradV(x):
        N = (x - c[:, None]) / r
        return (t[:, None] - (N * t[:, None]).sum(0) * N) / r
    return V, gradV


def test_velocity_derivatives_2d():
    """The general normal-velocity form of the moment derivatives: a uniform speed reproduces the
    radius derivatives, and a centre translation (a non-uniform speed, which also turns the normals)
    matches central differences of the generator's moments with the centre moved."""
    from oracle.eb_adjoint import circle_moment_derivatives, circle_velocity_derivatives
    N, c, r = 16, np.array([0.51, 0.49]), 0.3
    g = E.circle_config(N, center=tuple(c), r=r)
    o = Oracle(g, Params(order=4))
    a = circle_velocity_derivatives(o, 0, lambda x: np.ones(x.shape[1]), lambda x: np.zeros_like(x))
    b = circle_moment_derivatives(o, 0)
    for x, y in list(zip(a[:3], b[:3])) + list(zip(a[3], b[3])):
        assert np.abs(x - y).max() <= 1e-12 * max(1.0, np.abs(y).max())
    t = np.array([1.0, 0.0])
    V, gradV = _translation_velocity(c, r, t)
    dm = circle_velocity_derivatives(o, 0, V, gradV)
    gp = E.circle_config(N, center=tuple(c + EPS * t), r=r)
    gm = E.circle_config(N, center=tuple(c - EPS * t), r=r)
    assert np.array_equal(gp.cut_cells, g.cut_cells) and np.array_equal(gm.cut_cells, g.cut_cells)
    pairs = [(dm[0], gp.vol_mom, gm.vol_mom), (dm[1], gp.eb_mom, gm.eb_mom), (dm[2], gp.eb_nmom, gm.eb_nmom)]
    pairs += [(dm[3][d], gp.face_mom[d], gm.face_mom[d]) for d in range(2)]
    for an, x, y in pairs:
        fd = (x - y) / (2 * EPS)
        assert np.abs(an - fd).max() <= 1e-7 * np.abs(fd).max()


def test_centre_gradient_adjoint_against_central_differences():
    """dJ/dc_x through the solve and LS-build adjoints with the translation's moment derivatives,
    against central differences of J with the circle moved."""
    from oracle.eb_adjoint import circle_velocity_derivatives
    N, c, r = 16, np.array([0.51, 0.49]), 0.3
    t = np.array([1.0, 0.0])
    V, gradV = _translation_velocity(c, r, t)
    g = E.circle_config(N, center=tuple(c), r=r)
    J, dJ = objective_and_radius_gradient(g, derivs=lambda o: circle_velocity_derivatives(o, 0, V, gradV))
    Jp = objective_and_radius_gradient(E.circle_config(N, center=tuple(c + EPS * t), r=r))[0]
    Jm = objective_and_radius_gradient(E.circle_config(N, center=tuple(c - EPS * t), r=r))[0]
    assert abs(dJ - (Jp - Jm) / (2 * EPS)) <= 1e-6 * abs(dJ)


def test_velocity_derivatives_3d():
    """3-D: a uniform speed reproduces the radius derivatives (two different patch quadratures), and a
    centre translation matches central differences of the generator's moments with the sphere moved."""
    from oracle.eb_adjoint import sphere_moment_derivatives, sphere_velocity_derivatives
    N, c, r = 8, np.array([0.503, 0.497, 0.501]), 0.3
    g = E.Geometry(3, N, np.array([c]), np.array([r]), False, 4)
    o = Oracle(g, Params(order=4))
    a = sphere_velocity_derivatives(o, 0, lambda x: np.ones(x.shape[1]), lambda x: np.zeros_like(x))
    b = sphere_moment_derivatives(o, 0)
    for x, y in list(zip(a[:3], b[:3])) + list(zip(a[3], b[3])):
        assert np.abs(x - y).max() <= 1e-10 * max(1.0, np.abs(y).max())
    t = np.array([0.0, 1.0, 0.0])
    V, gradV = _translation_velocity(c, r, t)
    dm = sphere_velocity_derivatives(o, 0, V, gradV)
    gp = E.Geometry(3, N, np.array([c + EPS * t]), np.array([r]), False, 4)
    gm = E.Geometry(3, N, np.array([c - EPS * t]), np.array([r]), False, 4)
    assert np.array_equal(gp.cut_cells, g.cut_cells) and np.array_equal(gm.cut_cells, g.cut_cells)
    pairs = [(dm[0], gp.vol_mom, gm.vol_mom), (dm[1], gp.eb_mom, gm.eb_mom), (dm[2], gp.eb_nmom, gm.eb_nmom)]
    for d in range(3):
        assert np.array_equal(gp.cut_faces[d], g.cut_faces[d]) and np.array_equal(gm.cut_faces[d], g.cut_faces[d])
        pairs.append((dm[3][d], gp.face_mom[d], gm.face_mom[d]))
    for an, x, y in pairs:
        fd = (x - y) / (2 * EPS)
        assert np.abs(an - fd).max() <= 1e-7 * np.abs(fd).max()


def test_fourier_mode_derivatives_sum_over_bodies():
    """A mode with k = 0 is a constant shift of the level set: its derivative is -sin(theta) times the
    sum over the bodies of the radius derivatives."""
    from oracle.eb_adjoint import circle_moment_derivatives, fourier_mode_derivatives
    g = E.Geometry(2, 16, np.array([[0.31, 0.29, 0.0], [0.69, 0.66, 0.0]]), np.array([0.13, 0.17]), False, 4)
    o = Oracle(g, Params(order=4))
    th = 0.7
    a = fourier_mode_derivatives(o, (0, 0), th)
    parts = [circle_moment_derivatives(o, b) for b in range(2)]
    for i in range(3):
        ref = -math.sin(th) * (parts[0][i] + parts[1][i])
        assert np.abs(a[i] - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max())
    for d in range(2):
        ref = -math.sin(th) * (parts[0][3][d] + parts[1][3][d])
        assert np.abs(a[3][d] - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max())


def _two_circles():
    return E.Geometry(2, 16, np.array([[0.31, 0.29, 0.0], [0.69, 0.66, 0.0]]), np.array([0.13, 0.17]), False, 4)


def _with_moments(g, mo):
    import copy
    gg = copy.copy(g)
    gg.vol_mom, gg.eb_mom, gg.eb_nmom, gg.face_mom = mo[0], mo[1], mo[2], list(mo[3])
    gg.kappa = g.kappa.copy()
    gg.kappa[g.cut_cells] = mo[0][:, 0]
    return gg


def test_level_set_moments_reduce_to_circles():
    """The level-set moment oracle (height functions with root finding) with no Fourier term equals the
    generator's circle moments."""
    from oracle.eb_moments import level_set_moments_2d
    g = _two_circles()
    vol, eb, ebn, faces = level_set_moments_2d(g, [])
    assert np.abs(vol - g.vol_mom).max() <= 1e-13
    assert np.abs(eb - g.eb_mom).max() <= 1e-13
    assert np.abs(ebn - g.eb_nmom).max() <= 1e-13
    for d in range(2):
        assert np.abs(faces[d] - g.face_mom[d]).max() <= 1e-13


def test_fourier_mode_derivatives_against_level_set():
    """dJ/da for a Fourier mode of the level set at a = 0: the moment derivatives (every boundary
    moving with V = -sin(2 pi k . x + theta)) against central differences of the level-set moments,
    and dJ/da through the solve and LS-build adjoints against central differences of J."""
    from oracle.eb_adjoint import fourier_mode_derivatives
    from oracle.eb_moments import level_set_moments_2d
    g = _two_circles()
    k, th = (1, 2), 0.3
    mp = level_set_moments_2d(g, [(EPS, k, th)])
    mm = level_set_moments_2d(g, [(-EPS, k, th)])
    dm = fourier_mode_derivatives(Oracle(g, Params(order=4)), k, th)
    pairs = [(dm[i], mp[i], mm[i]) for i in range(3)] + [(dm[3][d], mp[3][d], mm[3][d]) for d in range(2)]
    for an, a, b in pairs:
        fd = (a - b) / (2 * EPS)
        assert np.abs(an - fd).max() <= 1e-7 * np.abs(fd).max()
    J, dJ = objective_and_radius_gradient(g, derivs=lambda o: fourier_mode_derivatives(o, k, th))
    fdJ = (objective_and_radius_gradient(_with_moments(g, mp))[0]
           - objective_and_radius_gradient(_with_moments(g, mm))[0]) / (2 * EPS)
    assert abs(dJ - fdJ) <= 1e-6 * abs(fdJ)

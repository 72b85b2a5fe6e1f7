"""Moment tables computed on the device (eb_geometry_circles, Sec. 2.1 moments) against the moment
oracle (oracle/eb_moments.py: divergence theorem over the cell boundary, closed-form face segments,
Gauss-Legendre on the arcs) and against the host input generator (iterated Gauss-Kronrod), table by
table: the cell and face classifications and cut lists identical, every moment within 1e-13 (all
three are exact to rounding).  Then the operator built from the device tables equals the one built
from the host tables to the size that rounding-level moment differences reach through the weighted
least squares: the systems' condition numbers are 1e3 .. 3e4, so 1e-14 in the moments moves the
stencils by up to ~1e-10; the operators are held to 1e-9 normwise."""
import numpy as np
import pytest

import eb_inputs as E
from gpu_helpers import to_dev
from oracle.eb_moments import circle_moments

pytestmark = pytest.mark.gpu

CASES = {
    "circle_r03_n32": (32, [(0.51, 0.49)], [0.3], False),
    "two_circles_n24": (24, [(0.31, 0.29), (0.69, 0.66)], [0.13, 0.17], False),
    "five_circles_n128": None,   # the seeded five-circle geometry (multi_circle_config)
    "inside_n32": (32, [(0.5, 0.5)], [0.45], True),
}


def _case(name):
    if name == "five_circles_n128":
        g = E.multi_circle_config(128)
        return 128, [tuple(c[:2]) for c in g.centers], list(g.radii), False, g
    N, cen, rad, inside = CASES[name]
    g = E.Geometry(2, N, np.array([[c[0], c[1], 0.0] for c in cen]), np.array(rad), inside, 4)
    return N, cen, rad, inside, g


@pytest.mark.parametrize("name", list(CASES))
def test_device_tables_match_generator(name):
    import paper_1411_4283_gb300 as P
    N, cen, rad, inside, g = _case(name)
    G = P.eb_geometry_circles(N, cen, rad, inside=inside, moment_degree=4)
    assert np.array_equal(G.table("flag"), g.flag)
    assert np.array_equal(G.table("cut_cells"), g.cut_cells)
    for t in ("vol_mom", "eb_mom", "eb_nmom"):
        got, want = G.table(t), getattr(g, t)
        assert got.shape == want.shape, t
        assert np.abs(got - want).max() <= 1e-13, (t, np.abs(got - want).max())
    for d in range(2):
        assert np.array_equal(G.table("face_flag", d), g.face_flag[d])
        assert np.array_equal(G.table("cut_faces", d), g.cut_faces[d])
        assert np.abs(G.table("face_mom", d) - g.face_mom[d]).max() <= 1e-13


@pytest.mark.parametrize("name", ["circle_r03_n32", "two_circles_n24"])
def test_device_tables_match_moment_oracle(name):
    import paper_1411_4283_gb300 as P
    N, cen, rad, inside, g = _case(name)
    G = P.eb_geometry_circles(N, cen, rad, inside=inside, moment_degree=4)
    cells, faces = circle_moments(N, [np.array(c) for c in cen], rad, 4)
    cut = G.table("cut_cells")
    vol, eb, ebn = G.table("vol_mom"), G.table("eb_mom"), G.table("eb_nmom")
    assert sorted(cells) == sorted(int(c) for c in cut)
    for k, c in enumerate(cut):
        m = cells[int(c)]
        assert np.abs(m["vol"] - vol[k]).max() <= 1e-13
        assert np.abs(m["eb"] - eb[k]).max() <= 1e-13
        assert np.abs(m["ebn"] - ebn[k]).max() <= 1e-13
    for d in range(2):
        fm = G.table("face_mom", d)
        for k, f in enumerate(G.table("cut_faces", d)):
            assert np.abs(faces[d][int(f)] - fm[k]).max() <= 1e-13


def test_stencils_from_device_tables():
    """The operator built on the device tables equals the one built on the host tables (FP64 apply,
    kappa-weighted, 1e-9 normwise: see the module docstring) for the circle r = 0.3 at (0.51, 0.49),
    N = 32, and both orders."""
    import torch
    import paper_1411_4283_gb300 as P
    N, cen, rad, inside, g = _case("circle_r03_n32")
    G = P.eb_geometry_circles(N, cen, rad, moment_degree=4)
    phi = to_dev(E.seeded_field(21, g.ncell) * (g.flag > 0))
    for Q in (4, 2):
        s_dev = P.eb_build_stencils(G, order=Q)
        s_host = P.eb_build_stencils(P.DeviceGeometry.from_geometry(g), order=Q)
        y1 = torch.empty_like(phi)
        y2 = torch.empty_like(phi)
        P.eb_apply(s_dev, phi, y1)
        P.eb_apply(s_host, phi, y2)
        assert (torch.linalg.norm(y1 - y2) / torch.linalg.norm(y2)).item() <= 1e-9


def test_two_circles_in_one_cell_refused():
    import paper_1411_4283_gb300 as P
    with pytest.raises(P.EbError) as ei:
        P.eb_geometry_circles(8, [(0.3, 0.3), (0.36, 0.3)], [0.1, 0.1])
    assert ei.value.code == 3


SPHERES = {
    "box_minus_sphere_n24": lambda: E.sphere_box_config(24, seed=2),
    "inside_sphere_n20": lambda: E.sphere_inside_config(20),
    "eight_spheres_n24": lambda: E.multi_sphere_config(24),
}


@pytest.mark.parametrize("name", list(SPHERES))
def test_device_sphere_tables_match_generator(name):
    """3-D: the device tables (sphere area element in (z, phi) on panels split at the patch's tangencies,
    disk-in-square face moments, divergence-theorem volume moments) against the host generator's
    (iterated Gauss-Kronrod): classifications and cut lists identical, moments within 1e-12."""
    import paper_1411_4283_gb300 as P
    g = SPHERES[name]()
    G = P.eb_geometry_spheres(g.N, g.centers, g.radii, inside=g.inside, moment_degree=4)
    assert np.array_equal(G.table("flag"), g.flag)
    assert np.array_equal(G.table("cut_cells"), g.cut_cells)
    for t in ("vol_mom", "eb_mom", "eb_nmom"):
        got, want = G.table(t), getattr(g, t)
        assert got.shape == want.shape, t
        assert np.abs(got - want).max() <= 1e-12, (t, np.abs(got - want).max())
    for d in range(3):
        assert np.array_equal(G.table("face_flag", d), g.face_flag[d])
        assert np.array_equal(G.table("cut_faces", d), g.cut_faces[d])
        assert np.abs(G.table("face_mom", d) - g.face_mom[d]).max() <= 1e-12, d


def test_device_sphere_tables_match_moment_oracle():
    """Against the moment oracle's sphere patch quadrature at N = 8 (pole cells included), 1e-10."""
    from oracle.eb_moments import sphere_moments
    import paper_1411_4283_gb300 as P
    N, cen, r = 8, (0.503, 0.497, 0.501), 0.3
    G = P.eb_geometry_spheres(N, [cen], [r], moment_degree=4)
    cut = G.table("cut_cells")
    mm = sphere_moments(N, [np.array(cen)], [r], cut, 4)
    vol, eb, ebn = G.table("vol_mom"), G.table("eb_mom"), G.table("eb_nmom")
    for k, c in enumerate(cut):
        m = mm[int(c)]
        assert np.abs(m["vol"] - vol[k]).max() <= 1e-10
        assert np.abs(m["eb"] - eb[k]).max() <= 1e-10
        assert np.abs(m["ebn"] - ebn[k]).max() <= 1e-10


def test_benchmark_geometry_on_device_builds_the_same_operator():
    """The benchmark geometry (cube minus sphere r = 0.35, seeded centre) at 48^3 from device tables:
    the FP64 operator equals the one built from the host tables (1e-9 normwise, see the module
    docstring)."""
    import torch
    import paper_1411_4283_gb300 as P
    g = E.sphere_box_config(48, seed=2)
    G = P.eb_geometry_spheres(48, g.centers, g.radii, moment_degree=4)
    phi = to_dev(E.seeded_field(22, g.ncell) * (g.flag > 0))
    s_dev = P.eb_build_stencils(G, order=4)
    s_host = P.eb_build_stencils(P.DeviceGeometry.from_geometry(g), order=4)
    y1 = torch.empty_like(phi)
    y2 = torch.empty_like(phi)
    P.eb_apply(s_dev, phi, y1)
    P.eb_apply(s_host, phi, y2)
    assert (torch.linalg.norm(y1 - y2) / torch.linalg.norm(y2)).item() <= 1e-9

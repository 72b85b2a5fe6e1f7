"""The moment oracle (oracle/eb_moments.py: the divergence theorem over the cell boundary, closed-form
face segments, Gauss-Legendre on the arcs) against the input generator (iterated Gauss-Kronrod with
breakpoints) and against closed forms: two independent routes to the moment tables of Sec. 2.1."""
import math

import numpy as np
import pytest

import eb_inputs as E
from oracle.eb_moments import circle_moments


@pytest.mark.parametrize("N,cen,rad", [(32, [(0.51, 0.49)], [0.3]),
                                       (24, [(0.31, 0.29), (0.69, 0.66)], [0.13, 0.17])])
def test_circle_moments_two_routes(N, cen, rad):
    g = E.Geometry(2, N, np.array([[c[0], c[1], 0.0] for c in cen]), np.array(rad), False, 4)
    cells, faces = circle_moments(N, [np.array(c) for c in cen], rad, 4)
    assert sorted(cells) == sorted(int(c) for c in g.cut_cells)
    for k, c in enumerate(g.cut_cells):
        m = cells[int(c)]
        assert np.abs(m["vol"] - g.vol_mom[k]).max() <= 1e-13
        assert np.abs(m["eb"] - g.eb_mom[k]).max() <= 1e-13
        assert np.abs(m["ebn"] - g.eb_nmom[k]).max() <= 1e-13
    for d in range(2):
        for k, f in enumerate(g.cut_faces[d]):
            assert np.abs(faces[d][int(f)] - g.face_mom[d][k]).max() <= 1e-13
    # closed forms: fluid area 1 - sum pi r^2, boundary length sum 2 pi r
    h = 1.0 / N
    full = N * N - len(cells) - sum(1 for j in range(N) for i in range(N)
                                    if j * N + i not in cells and any(
                                        math.hypot((i + 0.5) * h - c[0], (j + 0.5) * h - c[1]) < r
                                        for c, r in zip(cen, rad)))
    area = full * h * h + sum(m["vol"][0] for m in cells.values()) * h * h
    assert abs(area - (1 - sum(math.pi * r * r for r in rad))) <= 1e-13
    length = sum(m["eb"][0] for m in cells.values()) * h
    assert abs(length - sum(2 * math.pi * r for r in rad)) <= 1e-13


def test_sphere_moments_two_routes():
    """3-D, the cube minus a sphere at N = 8: the (z, phi) patch quadrature and the divergence-theorem
    volume moments against the generator (1e-10; the pole cells are the hardest), and the closed-form
    fluid volume and sphere area."""
    from oracle.eb_moments import sphere_moments
    N, cen, r = 8, (0.503, 0.497, 0.501), 0.3
    g = E.Geometry(3, N, np.array([cen]), np.array([r]), False, 4)
    mm = sphere_moments(N, [np.array(cen)], [r], g.cut_cells, 4)
    assert sorted(mm) == sorted(int(c) for c in g.cut_cells)
    for k, c in enumerate(g.cut_cells):
        m = mm[int(c)]
        assert np.abs(m["vol"] - g.vol_mom[k]).max() <= 1e-10
        assert np.abs(m["eb"] - g.eb_mom[k]).max() <= 1e-10
        assert np.abs(m["ebn"] - g.eb_nmom[k]).max() <= 1e-10
    h = 1.0 / N
    n_full = int((g.flag == 1).sum())
    vol = n_full * h ** 3 + sum(m["vol"][0] for m in mm.values()) * h ** 3
    assert abs(vol - (1 - 4.0 / 3.0 * math.pi * r ** 3)) <= 1e-12
    area = sum(m["eb"][0] for m in mm.values()) * h * h
    assert abs(area - 4 * math.pi * r * r) <= 1e-10


def test_sphere_face_moments_two_routes():
    from oracle.eb_moments import sphere_face_moments
    N, cen, r = 8, (0.503, 0.497, 0.501), 0.3
    g = E.Geometry(3, N, np.array([cen]), np.array([r]), False, 4)
    for d in range(3):
        fm = sphere_face_moments(N, [np.array(cen)], [r], d, g.cut_faces[d], 4)
        for k, f in enumerate(g.cut_faces[d]):
            assert np.abs(fm[int(f)] - g.face_mom[d][k]).max() <= 1e-11, (d, f)

"""Pins of the input generator (eb_inputs): quadrature rule, closed forms and the paper's
smallest-volume-fraction table (Sec. 3.4.1)."""
import json
import math
import os

import numpy as np
import pytest

import eb_inputs as E
from eb_inputs.geometry import _load

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")))


def test_gauss_kronrod_exactness():
    lib = _load()
    for k in range(23):  # 15-point Kronrod: exact to degree 22
        assert abs(lib.geo_gk15_panel_pow(k, 0) - 1.0 / (k + 1)) < 1e-15
    for k in range(14):  # embedded 7-point Gauss: exact to degree 13
        assert abs(lib.geo_gk15_panel_pow(k, 1) - 1.0 / (k + 1)) < 1e-15
    assert abs(lib.geo_gk15_panel_pow(14, 1) - 1.0 / 15) > 1e-9  # and not beyond


def test_splitmix64_published_values():
    # first outputs of SplitMix64 seeded with 0
    g = E.SplitMix64(0)
    assert [g.next_u64() for _ in range(3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    g = E.SplitMix64(7)
    seq = [g.next_double() for _ in range(5)]
    assert np.array_equal(np.array(seq), E.uniform(7, 5))


def test_full_cells_closed_form():
    g = E.line_config(8)
    assert np.all(g.flag == 1) and len(g.cut_cells) == 0
    g = E.circle_config(16)
    full = np.nonzero(g.flag == 1)[0][:5]
    bp = g._basis_pow(4)
    vals = g.cell_integrals(full, np.full(len(full), -1, np.int32), bp, g._terms_mono(2, 4))
    expect = [np.prod([0.0 if q % 2 else 0.5 ** q / (q + 1) for q in m]) for m in E.monomials(2, 4)]
    assert np.allclose(vals, np.array(expect)[None, :], atol=1e-16)


@pytest.mark.parametrize("N", [16, 32, 64])
def test_circle_area_and_perimeter(N):
    g = E.circle_config(N)
    assert abs(g.kappa.sum() * g.h ** 2 - (1 - math.pi * 0.25 ** 2)) < 1e-13
    assert abs(g.eb_mom[:, 0].sum() * g.h - 2 * math.pi * 0.25) < 1e-13
    gi = E.circle_config(N, r=0.3, inside=True)
    assert abs(gi.kappa.sum() * gi.h ** 2 - math.pi * 0.09) < 1e-13


def test_sphere_volume_and_area():
    g = E.sphere_inside_config(16)
    assert abs(g.kappa.sum() * g.h ** 3 - 4 / 3 * math.pi * 0.45 ** 3) < 1e-13
    assert abs(g.eb_mom[:, 0].sum() * g.h ** 2 - 4 * math.pi * 0.45 ** 2) < 1e-12
    g = E.sphere_box_config(16)
    assert abs(g.kappa.sum() * g.h ** 3 - (1 - 4 / 3 * math.pi * 0.35 ** 3)) < 1e-13


def _divergence_residual(g):
    """max over cut cells and monomials of |int_V d_d xi^p - int_dV xi^p n_d| (divergence theorem)."""
    D, q = g.dim, g.qmax - 1
    mons = E.monomials(D, q + 1)
    idx = {m: i for i, m in enumerate(mons)}
    fmons = E.monomials(D - 1, g.qmax)
    fidx = {m: i for i, m in enumerate(fmons)}
    vol_idx = {m: i for i, m in enumerate(E.monomials(D, g.qmax))}
    worst = 0.0
    for ci, c in enumerate(g.cut_cells[:200]):
        ijk = []
        r = int(c)
        for d in range(D):
            ijk.append(r % g.n[d]); r //= g.n[d]
        for d in range(D):
            for m in mons:
                if m[d] == 0 or sum(m) > g.qmax:
                    continue
                lower = list(m); lower[d] -= 1
                lhs = m[d] * g.vol_mom[ci, vol_idx[tuple(lower)]]
                tang = tuple(m[k] for k in range(D) if k != d)
                rhs = 0.0
                for side in (0, 1):
                    f = list(ijk)
                    f[d] += side
                    lin, s = 0, 1
                    for k in range(D):
                        lin += f[k] * s
                        s *= g.n[k] + (k == d)
                    ff = g.face_flag[d][lin]
                    if ff == 0:
                        continue
                    if ff == 1:
                        tm = np.prod([0.0 if e % 2 else 0.5 ** e / (e + 1) for e in tang])
                    else:
                        pos = np.searchsorted(g.cut_faces[d], lin)
                        tm = g.face_mom[d][pos, fidx[tang]]
                    rhs += (0.5 if side else -0.5) ** m[d] * (1 if side else -1) * tm
                rhs += g.eb_nmom[ci, d, vol_idx[m]]
                worst = max(worst, abs(lhs - rhs))
    return worst


def test_divergence_theorem_2d():
    assert _divergence_residual(E.circle_config(32)) < 1e-14
    assert _divergence_residual(E.multi_circle_config(64)) < 1e-14


def test_divergence_theorem_3d():
    assert _divergence_residual(E.sphere_box_config(16)) < 1e-13
    assert _divergence_residual(E.sphere_inside_config(12)) < 1e-13


@pytest.mark.parametrize("key,center,r", [("c0.5_r0.25", (0.5, 0.5), 0.25), ("c0.5_r0.255", (0.5, 0.5), 0.255),
                                          ("c0.501_r0.25", (0.501, 0.501), 0.25),
                                          ("c0.51-0.5_r0.25", (0.51, 0.5), 0.25)])
def test_smallest_volume_fraction_table(key, center, r):
    """The paper's table of smallest volume fractions (Sec. 3.4.1), two significant digits."""
    for N, want in zip(GOLD["kappa_min"]["N"], GOLD["kappa_min"][key]):
        got = E.circle_config(N, center=center, r=r).min_kappa()
        assert float(f"{got:.1e}") == pytest.approx(want, rel=1e-9), (N, got, want)


def test_multi_circle_clearance():
    g = E.multi_circle_config(128, seed=1)
    c, r = g.centers[:, :2], g.radii
    for i in range(len(r)):
        assert np.all(c[i] - r[i] >= 0.04 - 1e-12) and np.all(c[i] + r[i] <= 0.96 + 1e-12)
        for j in range(i):
            assert np.linalg.norm(c[i] - c[j]) - r[i] - r[j] >= 0.04 - 1e-12


def test_manufactured_full_cell_average():
    g = E.circle_config(16)
    man = E.Manufactured(g, E.sin_product("sin2pix_cos3piy"))
    avg = man.cell_avg()
    c = 0  # cell (0,0) is full
    x0, x1, h = 0.0, g.h, g.h
    ex = (-(math.cos(2 * math.pi * x1) - math.cos(2 * math.pi * x0)) / (2 * math.pi * h)) * \
         ((math.sin(3 * math.pi * x1) - math.sin(3 * math.pi * x0)) / (3 * math.pi * h))
    assert abs(avg[c] - ex) < 1e-15


def test_multi_sphere_clearance_and_volume():
    """Eight seeded spheres, radii in [0.08, 0.2): pairwise and wall clearance >= 2h, no cell cut by two
    spheres (the generator would refuse), and the fluid volume 1 - sum 4/3 pi r^3 to 1e-12."""
    import math
    N = 24
    g = E.multi_sphere_config(N)
    h = 1.0 / N
    c, r = g.centers, g.radii
    assert len(r) == 8 and np.all((r >= 0.08) & (r < 0.2))
    assert np.all(c - r[:, None] >= 2 * h - 1e-15) and np.all(c + r[:, None] <= 1 - 2 * h + 1e-15)
    for i in range(8):
        for j in range(i):
            assert np.linalg.norm(c[i] - c[j]) - r[i] - r[j] >= 2 * h - 1e-15
    vol = (g.flag == 1).sum() * h ** 3 + g.vol_mom[:, 0].sum() * h ** 3
    assert abs(vol - (1 - sum(4 / 3 * math.pi * x ** 3 for x in r))) <= 1e-12


def test_level_set_modes():
    """The shape-gradient workload's 16 modes: integer wave numbers in 1..4 per component (0 beyond the
    dimension), phases in [0, 2 pi), drawn four numbers per mode from SplitMix64(5)."""
    m = E.level_set_modes(16, seed=5)
    assert m.shape == (16, 4)
    k = m[:, :3]
    assert np.all(k == np.round(k)) and np.all((k >= 1) & (k <= 4))
    assert np.all((m[:, 3] >= 0) & (m[:, 3] < 2 * math.pi))
    u = E.uniform(5, 4 * 16)
    assert m[0, 3] == 2 * math.pi * u[3] and m[0, 0] == 1 + min(3, math.floor(4 * u[0]))
    assert np.array_equal(E.level_set_modes(16, seed=5), m)
    m2 = E.level_set_modes(3, seed=5, dim=2)
    assert np.all(m2[:, 2] == 0) and np.array_equal(m2[:, :2], m[:3, :2])


def test_ellipse_generator_reduces_to_circles():
    """a = b: the ellipse generator (arc quadrature, chords, divergence theorem; eb_inputs/ellipse.py)
    against the circle generator (iterated Gauss-Kronrod, geom.c), two independent integrations: the
    same classification and cut lists, every table within 1e-13."""
    from eb_inputs.ellipse import EllipseGeometry
    for N, cen, r in ((64, (0.51, 0.49), 0.3), (40, (0.45, 0.55), 0.2)):
        g = EllipseGeometry(N, [cen], [(r, r)])
        c = E.circle_config(N, center=cen, r=r)
        assert np.array_equal(g.flag, c.flag) and np.array_equal(g.cut_cells, c.cut_cells)
        for t in ("vol_mom", "eb_mom", "eb_nmom"):
            assert np.abs(getattr(g, t) - getattr(c, t)).max() <= 1e-13, t
        for d in range(2):
            assert np.array_equal(g.face_flag[d], c.face_flag[d]) and np.array_equal(g.cut_faces[d], c.cut_faces[d])
            assert np.abs(g.face_mom[d] - c.face_mom[d]).max() <= 1e-13


def test_ellipse_area_perimeter_and_divergence():
    """An eccentric ellipse (a = 0.31, b = 0.17): fluid area 1 - pi a b and boundary length 4 a E(1 - b^2/a^2)
    (complete elliptic integral of the second kind) to 1e-13 / 1e-12; per cut cell the divergence theorem
    int_V d/dx (xi^p eta^q) = sum over the x-faces' fluid parts + int_EB xi^p eta^q n_x to 1e-13."""
    from scipy.special import ellipe
    from eb_inputs.ellipse import EllipseGeometry
    a, b, N = 0.31, 0.17, 48
    g = EllipseGeometry(N, [(0.503, 0.497)], [(a, b)])
    h = g.h
    area = ((g.flag == 1).sum() + g.vol_mom[:, 0].sum()) * h * h
    assert abs(area - (1 - math.pi * a * b)) <= 1e-13
    assert abs(g.eb_mom[:, 0].sum() * h - 4 * a * ellipe(1 - (b / a) ** 2)) <= 1e-12
    mons = E.monomials(2, g.qmax)
    idx = {m: k for k, m in enumerate(mons)}
    fx = {int(f): k for k, f in enumerate(g.cut_faces[0])}
    for k, c in enumerate(g.cut_cells):
        i, j = int(c) % N, int(c) // N
        for (p, q), m in idx.items():
            if p == 0 or (p - 1, q) not in idx:
                continue
            lhs = p * g.vol_mom[k, idx[(p - 1, q)]]
            rhs = g.eb_nmom[k, 0, m]
            for side, e in ((0, -0.5), (1, 0.5)):
                f = (i + side) + (N + 1) * j
                if g.face_flag[0][f] == 0:
                    continue
                fm = g.face_mom[0][fx[f], q] if f in fx else (0.5 ** (q + 1) - (-0.5) ** (q + 1)) / (q + 1)
                rhs += math.copysign(1.0, e) * e ** p * fm
            assert abs(lhs - rhs) <= 1e-13, (c, p, q, lhs, rhs)

"""Plain FP64 oracle of the geometry moments of Sec. 2.1 for the unit square minus circles (2-D),
written independently of the input generator: the oracle of GPU moment generation.

TEST INFRASTRUCTURE, like eb_oracle.py: only tests/ may import it; the GPU library never does.

For a cut cell (or face) with centre x_c and xi = (x - x_c)/h:
  face moments    int over the fluid part of the face of eta^q dt / h, eta the tangential
                  coordinate about the face centre: the face segment minus the chord inside the
                  circle, integrated in closed form;
  EB moments      int over the arc of the circle inside the cell of xi^p ds / h (and weighted by the
                  normal component out of the fluid, -e(t)), Gauss-Legendre in the angle (the
                  integrand is a trigonometric polynomial: exact to rounding with enough points);
  volume moments  by the divergence theorem, int_V xi^p dA = h / (p_0 + 1) * oint xi^(p + e_0) n_0 ds
                  (n out of the fluid part of the cell): the cell's vertical edges (their fluid
                  parts, in closed form) and the arc; divided by h^2.
"""
from __future__ import annotations

import math

import numpy as np

from .eb_adjoint import _arcs

_GL_X, _GL_W = np.polynomial.legendre.leggauss(32)


def _mons2(q):
    out = []
    for d in range(q + 1):
        for p0 in range(d, -1, -1):
            out.append((p0, d - p0))
    return out


def _fluid_intervals(t0, t1, ct, s):
    """The parts of [t0, t1] outside the open interval (ct - s, ct + s)."""
    if s <= 0:
        return [(t0, t1)]
    out = []
    if t0 < ct - s:
        out.append((t0, min(t1, ct - s)))
    if t1 > ct + s:
        out.append((max(t0, ct + s), t1))
    return out


def _segment_moments(a, b, q):
    """int_a^b u^k du for k = 0..q (closed form)."""
    return np.array([(b ** (k + 1) - a ** (k + 1)) / (k + 1) for k in range(q + 1)])


def circle_moments(N, centers, radii, qmax=4):
    """Moment tables of the unit square minus the circles on an N x N grid, for the cut cells and cut
    faces the grid has (a cell or face is cut when a circle crosses it): dict with, per cut cell
    index, 'vol', 'eb', 'ebn' (2 x K) and, per direction and face index, 'face' (K_F)."""
    h = 1.0 / N
    mons = _mons2(qmax)
    K = len(mons)
    cells, faces = {}, ({}, {})

    def body_of(x0, x1, y0, y1):
        # the circle crossing the box, if any (nearest point inside the disk, farthest point outside)
        for b, (c, r) in enumerate(zip(centers, radii)):
            nx, ny = min(max(c[0], x0), x1), min(max(c[1], y0), y1)
            near = math.hypot(nx - c[0], ny - c[1])
            far = max(math.hypot(x - c[0], y - c[1]) for x in (x0, x1) for y in (y0, y1))
            if near < r < far:
                return b
        return -1

    for j in range(N):
        for i in range(N):
            x0, x1, y0, y1 = i * h, (i + 1) * h, j * h, (j + 1) * h
            b = body_of(x0, x1, y0, y1)
            if b < 0:
                continue
            (cx, cy), r = centers[b][:2], radii[b]
            xc, yc = x0 + 0.5 * h, y0 + 0.5 * h
            eb = np.zeros(K)
            ebn = np.zeros((2, K))
            vol = np.zeros(K)
            for (ta, _), (tb, _) in _arcs(cx, cy, r, x0, x1, y0, y1):
                t = 0.5 * (tb - ta) * _GL_X + 0.5 * (tb + ta)
                ds = 0.5 * (tb - ta) * _GL_W * r
                ex, ey = np.cos(t), np.sin(t)
                xi, eta = (cx + r * ex - xc) / h, (cy + r * ey - yc) / h
                for m, (p0, p1) in enumerate(mons):
                    f = xi ** p0 * eta ** p1
                    eb[m] += np.sum(ds * f) / h
                    ebn[0, m] += np.sum(ds * f * -ex) / h
                    ebn[1, m] += np.sum(ds * f * -ey) / h
                    # divergence theorem, arc part: n_0 out of the fluid = -e_x
                    vol[m] += np.sum(ds * xi ** (p0 + 1) * eta ** p1 * -ex) / (p0 + 1) / h
            # vertical edges: fluid parts, n_0 = -1 (left) and +1 (right), xi = -1/2 and +1/2
            for xe, sgn in ((x0, -1.0), (x1, 1.0)):
                q2 = r * r - (xe - cx) ** 2
                s = math.sqrt(q2) if q2 > 0 else 0.0
                for a, bb in _fluid_intervals(y0, y1, cy, s):
                    ym = _segment_moments((a - yc) / h, (bb - yc) / h, qmax + 1) * h  # int eta^k dy
                    for m, (p0, p1) in enumerate(mons):
                        vol[m] += sgn * (sgn * 0.5) ** (p0 + 1) * ym[p1] / (p0 + 1) / h
            cells[j * N + i] = {"vol": vol, "eb": eb, "ebn": ebn}
    # faces normal to d: d = 0 at x = i h (tangential y), d = 1 at y = j h (tangential x)
    for d in range(2):
        nf_t, nf_n = (N, N + 1)
        for a in range(nf_n):           # position along the normal
            for bidx in range(nf_t):    # position along the tangent
                xn = a * h
                t0, t1 = bidx * h, (bidx + 1) * h
                cut = None
                for bb, (c, r) in enumerate(zip(centers, radii)):
                    cn, ct = (c[0], c[1]) if d == 0 else (c[1], c[0])
                    q2 = r * r - (xn - cn) ** 2
                    if q2 <= 0:
                        continue
                    s = math.sqrt(q2)
                    if ct - s < t1 and ct + s > t0 and not (ct - s <= t0 and ct + s >= t1):
                        cut = (ct, s)
                if cut is None:
                    continue
                tc = 0.5 * (t0 + t1)
                mom = np.zeros(qmax + 1)
                for lo, hi in _fluid_intervals(t0, t1, cut[0], cut[1]):
                    mom += _segment_moments((lo - tc) / h, (hi - tc) / h, qmax)
                idx = (a + (N + 1) * bidx) if d == 0 else (bidx + N * a)
                faces[d][idx] = mom
    return cells, faces


# --------------------------------------------------------------------- 3-D: the cube minus spheres

_S_X, _S_W = np.polynomial.legendre.leggauss(48)


def _sin2_panels(breaks):
    """Nodes and weights on the panels [b_i, b_(i+1)] with t = a + (b - a) sin^2(pi s / 2), s in [0, 1]
    (48-point Gauss-Legendre in s): the substitution flattens the square-root behaviour of chord and
    arc ends at tangencies, which the panel breaks put at panel ends."""
    xs, ws = [], []
    s = 0.5 * _S_X + 0.5
    wg = 0.5 * _S_W
    sn, cs = np.sin(0.5 * math.pi * s), np.cos(0.5 * math.pi * s)
    for a, b in zip(breaks[:-1], breaks[1:]):
        if b <= a:
            continue
        xs.append(a + (b - a) * sn * sn)
        ws.append(wg * (b - a) * math.pi * sn * cs)
    if not xs:
        return np.zeros(0), np.zeros(0)
    return np.concatenate(xs), np.concatenate(ws)


def _mons3(q):
    from eb_inputs.geometry import monomials
    return monomials(3, q)


def _disk_rect_moments(cu, cv, rho, u0, u1, v0, v1, uc, vc, h, qmax):
    """int over [u0,u1]x[v0,v1] minus the open disk of radius rho about (cu, cv) of eta^a zeta^b
    d eta d zeta, eta = (u - uc)/h, zeta = (v - vc)/h, for the graded exponents (a, b), a + b <= qmax."""
    mons = _mons2(qmax)
    su = _segment_moments((u0 - uc) / h, (u1 - uc) / h, qmax)
    sv = _segment_moments((v0 - vc) / h, (v1 - vc) / h, qmax)
    rect = np.array([su[a] * sv[b] for a, b in mons])
    lo, hi = max(u0, cu - rho), min(u1, cu + rho)
    if rho <= 0 or hi <= lo:
        return rect
    br = [lo, hi]  # chord ends crossing v0 or v1 put kinks in the u integrand
    for ve in (v0, v1):
        dv = ve - cv
        if abs(dv) < rho:
            w = math.sqrt(rho * rho - dv * dv)
            for uu in (cu - w, cu + w):
                if lo < uu < hi:
                    br.append(uu)
    u, wu = _sin2_panels(sorted(br))
    half = np.sqrt(np.maximum(rho * rho - (u - cu) ** 2, 0.0))
    za = (np.clip(cv - half, v0, v1) - vc) / h
    zb = (np.clip(cv + half, v0, v1) - vc) / h
    eta = (u - uc) / h
    disk = np.array([np.sum(wu * eta ** a * (zb ** (b + 1) - za ** (b + 1)) / (b + 1)) / h for a, b in mons])
    return rect - disk


def sphere_patch_nodes(c, r, lo, hi):
    """Quadrature of the part of the sphere (centre c, radius r) inside the box [lo, hi]:
    (x [3, m], w [m]) with w the area weights.  The area element in (z, phi) is r dz dphi
    (Archimedes); at each z the patch is the arcs of the circle of radius (r^2 - (z - c_z)^2)^(1/2)
    inside the box's x-y rectangle (the whole circle when it lies inside); the z integral is split
    where the arcs change (tangencies with the rectangle's edge lines and corners) and mapped by
    the sin^2 substitution."""
    z_lo, z_hi = max(lo[2], c[2] - r), min(hi[2], c[2] + r)
    br = [z_lo, z_hi]
    d2 = [(lo[0] - c[0]) ** 2, (hi[0] - c[0]) ** 2, (lo[1] - c[1]) ** 2, (hi[1] - c[1]) ** 2]
    d2 += [(x - c[0]) ** 2 + (y - c[1]) ** 2 for x in (lo[0], hi[0]) for y in (lo[1], hi[1])]
    for dd in d2:
        q = r * r - dd
        if q > 0:
            for zz in (c[2] - math.sqrt(q), c[2] + math.sqrt(q)):
                if z_lo < zz < z_hi:
                    br.append(zz)
    zs, wz = _sin2_panels(sorted(br))
    xs, ws = [], []
    for z, wzz in zip(zs, wz):
        rho2 = r * r - (z - c[2]) ** 2
        if rho2 <= 0:
            continue
        rho = math.sqrt(rho2)
        arcs = [(ta, tb) for (ta, _), (tb, _) in _arcs(c[0], c[1], rho, lo[0], hi[0], lo[1], hi[1])]
        if not arcs and lo[0] < c[0] - rho and c[0] + rho < hi[0] and lo[1] < c[1] - rho and c[1] + rho < hi[1]:
            arcs = [(0.0, 2 * math.pi)]
        for ta, tb in arcs:
            t = 0.5 * (tb - ta) * _GL_X + 0.5 * (tb + ta)
            xs.append(np.stack([c[0] + rho * np.cos(t), c[1] + rho * np.sin(t), np.full_like(t, z)]))
            ws.append(wzz * r * 0.5 * (tb - ta) * _GL_W)
    if not xs:
        return np.zeros((3, 0)), np.zeros(0)
    return np.concatenate(xs, axis=1), np.concatenate(ws)


def sphere_patch_edges(c, r, lo, hi):
    """The edges of the sphere patch inside the box: on each face plane of the box the arcs of the
    circle the sphere cuts from it, inside the face.  List of (x [3, m], w [m] length weights,
    n_p [3] the face's normal out of the box)."""
    out = []
    for ax in range(3):
        oth = [b for b in range(3) if b != ax]
        for side, pa in ((-1.0, lo[ax]), (1.0, hi[ax])):
            q2 = r * r - (pa - c[ax]) ** 2
            if q2 <= 0:
                continue
            rho = math.sqrt(q2)
            n_p = np.zeros(3)
            n_p[ax] = side
            for (ta, _), (tb, _) in _arcs(c[oth[0]], c[oth[1]], rho, lo[oth[0]], hi[oth[0]], lo[oth[1]], hi[oth[1]]):
                t = 0.5 * (tb - ta) * _GL_X + 0.5 * (tb + ta)
                x = np.zeros((3, len(t)))
                x[ax] = pa
                x[oth[0]] = c[oth[0]] + rho * np.cos(t)
                x[oth[1]] = c[oth[1]] + rho * np.sin(t)
                out.append((x, 0.5 * (tb - ta) * _GL_W * rho, n_p))
    return out


def sphere_moments(N, centers, radii, cells, qmax=4):
    """Volume and EB moment tables of the unit cube minus spheres for the listed cut cells (each cut
    by one sphere): dict cell -> {'vol' [K], 'eb' [K], 'ebn' [3, K]}, scaled like the input tables.

    EB patch: the quadrature of sphere_patch_nodes.  Volume moments by the divergence theorem: int_V xi^p dV = h/(p_x+1) oint xi^(p+e_x) n_x dA over
    the cell's two x faces (their fluid parts: square minus disk) and the patch (n_x = -e_x)."""
    h = 1.0 / N
    mons = _mons3(qmax)
    K = len(mons)
    fidx = {mm: n for n, mm in enumerate(_mons2(qmax + 1))}
    out = {}
    for cell in cells:
        cell = int(cell)
        ijk = np.array([cell % N, (cell // N) % N, cell // (N * N)], float)
        lo, hi = ijk * h, (ijk + 1) * h
        xc = lo + 0.5 * h
        b = None
        for bb, (cc, rr) in enumerate(zip(centers, radii)):
            cc = np.asarray(cc, float)
            near = np.linalg.norm(np.clip(cc, lo, hi) - cc)
            far = max(np.linalg.norm(np.array([x, y, z]) - cc) for x in (lo[0], hi[0]) for y in (lo[1], hi[1])
                      for z in (lo[2], hi[2]))
            if near < rr < far:
                b = bb
        if b is None:
            continue
        c, r = np.asarray(centers[b], float), float(radii[b])
        x, wt = sphere_patch_nodes(c, r, lo, hi)
        e = (x - c[:, None]) / r
        xi = (x - xc[:, None]) / h
        eb = np.zeros(K)
        ebn = np.zeros((3, K))
        vol = np.zeros(K)
        for m, p in enumerate(mons):
            f = xi[0] ** p[0] * xi[1] ** p[1] * xi[2] ** p[2]
            eb[m] = np.sum(wt * f)
            for d in range(3):
                ebn[d, m] = -np.sum(wt * f * e[d])
            vol[m] = -np.sum(wt * xi[0] ** (p[0] + 1) * xi[1] ** p[1] * xi[2] ** p[2] * e[0]) / (p[0] + 1)
        eb /= h * h
        ebn /= h * h
        vol /= h * h  # vol_mom = int_V xi^p dV / h^3 = (1 / (h^2 (p_x+1))) oint xi^(p+e_x) n_x dA
        for xe, sgn in ((lo[0], -1.0), (hi[0], 1.0)):
            q2 = r * r - (xe - c[0]) ** 2
            rho = math.sqrt(q2) if q2 > 0 else 0.0
            fm = _disk_rect_moments(c[1], c[2], rho, lo[1], hi[1], lo[2], hi[2], xc[1], xc[2], h, qmax + 1)
            for m, p in enumerate(mons):  # dA = h^2 d eta d zeta on the face
                vol[m] += sgn * (sgn * 0.5) ** (p[0] + 1) * fm[fidx[(p[1], p[2])]] / (p[0] + 1)
        out[cell] = {"vol": vol, "eb": eb, "ebn": ebn}
    return out


def sphere_face_moments(N, centers, radii, d, faces, qmax=4):
    """Tangential moments of the fluid parts of the listed faces normal to d (3-D, the cube minus
    spheres): the face square minus the disks the spheres cut from its plane, about the face centre,
    in the graded order of the two tangential coordinates (ascending dimensions)."""
    h = 1.0 / N
    oth = [b for b in range(3) if b != d]
    shape = [N + (k == d) for k in range(3)]
    out = {}
    for f in faces:
        f = int(f)
        ijk = [f % shape[0], (f // shape[0]) % shape[1], f // (shape[0] * shape[1])]
        pa = ijk[d] * h
        lo = [ijk[b] * h for b in oth]
        hi = [(ijk[b] + 1) * h for b in oth]
        fc = [(ijk[b] + 0.5) * h for b in oth]
        mom = None
        for c, r in zip(centers, radii):
            q2 = r * r - (pa - c[d]) ** 2
            rho = math.sqrt(q2) if q2 > 0 else 0.0
            m = _disk_rect_moments(c[oth[0]], c[oth[1]], rho, lo[0], hi[0], lo[1], hi[1], fc[0], fc[1], h, qmax)
            full = _disk_rect_moments(0.0, 0.0, 0.0, lo[0], hi[0], lo[1], hi[1], fc[0], fc[1], h, qmax)
            mom = m if mom is None else mom - (full - m)  # disks of different spheres do not overlap
        out[f] = mom
    return out


# --------------------------------------------------------------------- 2-D: a perturbed level set

def level_set_moments_2d(g, modes):
    """Moment tables of the level set psi(x) = min_i(|x - c_i| - r_i) + sum_m a_m sin(2 pi k_m . x +
    theta_m) (fluid where psi > 0), on the cut cells and cut faces of the circle geometry g (the
    perturbation is taken small enough to keep them): (vol [n_cut, K], eb, ebn [n_cut, 2, K],
    face [per d]).  modes: list of (a, (k_x, k_y), theta).

    Each cut cell is integrated as a height function: along the direction where the circle's normal
    at the cell centre is largest the boundary is a graph, its height found by bracketed root
    finding in each column; the columns' fluid parts are integrated in closed form, the boundary with
    ds = |grad psi| / |d psi / d height| d(other), its normal out of the fluid -grad psi / |grad psi|;
    the other coordinate is split where the boundary crosses the cell's edges (Gauss-Legendre on
    sin^2-mapped panels).  Faces: the fluid parts of each edge between the roots of psi on it."""
    from scipy.optimize import brentq
    h, N = g.h, g.N
    cen = g.centers[:, :2]
    rad = g.radii

    def psi_b(x, y, b):
        v = np.hypot(x - cen[b, 0], y - cen[b, 1]) - rad[b]
        for a, k, th in modes:
            v = v + a * np.sin(2 * math.pi * (k[0] * x + k[1] * y) + th)
        return v

    def grad_b(x, y, b):
        rr = np.hypot(x - cen[b, 0], y - cen[b, 1])
        gx, gy = (x - cen[b, 0]) / rr, (y - cen[b, 1]) / rr
        for a, k, th in modes:
            cs = a * 2 * math.pi * np.cos(2 * math.pi * (k[0] * x + k[1] * y) + th)
            gx, gy = gx + cs * k[0], gy + cs * k[1]
        return gx, gy

    mons = _mons2(g.qmax)
    K = len(mons)
    n_cut = len(g.cut_cells)
    vol = np.zeros((n_cut, K))
    eb = np.zeros((n_cut, K))
    ebn = np.zeros((n_cut, 2, K))
    for kc, cc in enumerate(g.cut_cells):
        b = int(g.cut_body[kc])
        i, j = int(cc) % N, int(cc) // N
        lo, hi = np.array([i * h, j * h]), np.array([(i + 1) * h, (j + 1) * h])
        xc = lo + 0.5 * h
        nrm = xc - cen[b]
        hd = int(np.argmax(np.abs(nrm)))  # height direction
        od = 1 - hd

        def P(u, v):  # psi with (u, v) = (other, height) coordinates
            return psi_b(u, v, b) if od == 0 else psi_b(v, u, b)

        def G(u, v):
            gx, gy = grad_b(u, v, b) if od == 0 else grad_b(v, u, b)
            return (gx, gy) if od == 0 else (gy, gx)  # (d/du, d/dv)

        # breaks in u: where the boundary meets the edges v = lo[hd], hi[hd]
        br = [lo[od], hi[od]]
        for ve in (lo[hd], hi[hd]):
            us = np.linspace(lo[od], hi[od], 65)
            vals = P(us, np.full_like(us, ve))
            for a_, b_, fa, fb in zip(us[:-1], us[1:], vals[:-1], vals[1:]):
                if fa == 0.0 or fa * fb < 0:
                    br.append(brentq(lambda u: P(u, ve), a_, b_, xtol=1e-15, rtol=1e-15) if fa != 0.0 else a_)
        us, wu = _sin2_panels(sorted(br))
        for u, w in zip(us, wu):
            f0, f1 = P(u, lo[hd]), P(u, hi[hd])
            if f0 * f1 < 0:
                v = brentq(lambda t: P(u, t), lo[hd], hi[hd], xtol=1e-15, rtol=1e-15)
                fluid = (v, hi[hd]) if f1 > 0 else (lo[hd], v)
                gu, gv = G(u, v)
                gn = math.hypot(gu, gv)
                ds = gn / abs(gv)
                nvec = np.array([-gu / gn, -gv / gn])  # out of the fluid, in (u, v) order
                xy = np.zeros(2)
                xy[od], xy[hd] = u, v
                xi = (xy - xc) / h
                nd = np.zeros(2)
                nd[od], nd[hd] = nvec[0], nvec[1]
                for m, p in enumerate(mons):
                    f = xi[0] ** p[0] * xi[1] ** p[1]
                    eb[kc, m] += w * ds * f / h
                    ebn[kc, 0, m] += w * ds * f * nd[0] / h
                    ebn[kc, 1, m] += w * ds * f * nd[1] / h
            elif f0 > 0 and f1 > 0:
                fluid = (lo[hd], hi[hd])
            else:
                continue
            a_, b_ = (fluid[0] - xc[hd]) / h, (fluid[1] - xc[hd]) / h
            su = (u - xc[od]) / h
            for m, p in enumerate(mons):
                ph, po = p[hd], p[od]
                vol[kc, m] += w / h * su ** po * (b_ ** (ph + 1) - a_ ** (ph + 1)) / (ph + 1)
    faces = []
    for d in range(2):
        cf = g.cut_faces[d]
        out = np.zeros((len(cf), g.face_mom[d].shape[1]))
        for kf, f in enumerate(cf):
            b = int(g.cut_face_body[d][kf])
            shape = [N + (k == d) for k in range(2)]
            ij = [int(f) % shape[0], int(f) // shape[0]]
            xn = ij[d] * h
            td = 1 - d
            t0, t1 = ij[td] * h, (ij[td] + 1) * h
            tc = 0.5 * (t0 + t1)

            def Pt(t):
                return psi_b(xn, t, b) if d == 0 else psi_b(t, xn, b)
            ts = np.linspace(t0, t1, 129)
            vals = Pt(ts)
            pts = [t0]
            for a_, b_, fa, fb in zip(ts[:-1], ts[1:], vals[:-1], vals[1:]):
                if fa * fb < 0:
                    pts.append(brentq(Pt, a_, b_, xtol=1e-15, rtol=1e-15))
            pts.append(t1)
            for a_, b_ in zip(pts[:-1], pts[1:]):
                if Pt(0.5 * (a_ + b_)) > 0:
                    out[kf] += _segment_moments((a_ - tc) / h, (b_ - tc) / h, out.shape[1] - 1)
        faces.append(out)
    return vol, eb, ebn, faces

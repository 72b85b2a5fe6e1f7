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

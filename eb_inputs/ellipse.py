"""The unit square minus axis-aligned ellipses: moment tables in the layout of ``Geometry`` (2-D).

An INPUT GENERATOR like ``geometry.py``: it integrates monomials over the pieces of an N x N grid cut
by ellipses ((x - cx)/a)^2 + ((y - cy)/b)^2 < 1 (the fluid is outside them) and holds none of the
discretisation's arithmetic.  Everything is in cell- or face-centred coordinates xi = (x - centre)/h;
tables are divided by h^2 (volumes) or h (faces, EB arcs), graded monomial order (``monomials``).

  classification  a cell or face box is covered when one ellipse contains it, full when no ellipse
                  reaches into it, cut otherwise (two ellipses in one box are refused); in the
                  coordinates scaled by the semi-axes an ellipse is the unit disk, so the box's nearest
                  and farthest points decide it exactly;
  face moments    the fluid part of a face segment is the segment minus the chord inside the ellipse:
                  integrals of t^q in closed form;
  EB moments      the boundary arc x = c + (a cos t, b sin t), split where it crosses the cell's edge
                  lines, by Gauss-Legendre in t on pieces of at most pi/8 (smooth integrands: the arc
                  length element (a^2 sin^2 t + b^2 cos^2 t)^(1/2) and, for the normal-weighted moments,
                  n ds = -(b cos t, a sin t) dt, the normal out of the fluid);
  volume moments  the divergence theorem along the direction in which the arc's normal is smallest
                  (so that a thin sliver is not the small difference of terms of size one): the fluid
                  parts of the two edges normal to it in closed form and the arc.
Cells whose volume fraction is at most 1e-14 count as covered and those at least 1 - 1e-14 as full,
faces likewise; a face next to a covered cell is closed.
"""
from __future__ import annotations

import math

import numpy as np

from .geometry import KAPPA_EPS, monomials

_GL_X, _GL_W = np.polynomial.legendre.leggauss(32)


def _seg_pow(a, b, q):
    """int_a^b t^k dt, k = 0..q."""
    return np.array([(b ** (k + 1) - a ** (k + 1)) / (k + 1) for k in range(q + 1)])


class EllipseGeometry:
    """2-D unit square minus axis-aligned ellipses (centres [n][2], semi-axes [n][2]) on an N x N grid,
    moment degree qmax; attributes as ``Geometry`` (flag, cut_cells, vol_mom, eb_mom, eb_nmom,
    face_flag, cut_faces, face_mom, kappa, cut_body, cut_face_body)."""

    def __init__(self, N: int, centers, axes, qmax: int = 4, name: str = "", seed: int | None = None):
        self.dim, self.N, self.qmax, self.name, self.seed = 2, int(N), int(qmax), name, seed
        self.inside = False
        self.centers = np.asarray(centers, dtype=np.float64).reshape(-1, 2)
        self.axes = np.asarray(axes, dtype=np.float64).reshape(-1, 2)
        if len(self.centers) != len(self.axes) or np.any(self.axes <= 0):
            raise ValueError("one positive semi-axis pair per centre")
        self.n = (self.N, self.N, 1)
        self.h = 1.0 / self.N
        self.ncell = self.N * self.N
        self._build()

    # ------------------------------------------------------------ classification
    def _classify(self, lo, hi):
        """(flag, body) of the boxes [lo, hi] ([n][2] arrays): 0 covered, 1 full, 2 cut; raises when two
        ellipses reach into one box."""
        n = len(lo)
        flag = np.ones(n, dtype=np.int8)
        body = np.full(n, -1, dtype=np.int32)
        ncut = np.zeros(n, dtype=np.int32)
        covered = np.zeros(n, dtype=bool)
        for k, (c, ax) in enumerate(zip(self.centers, self.axes)):
            sl, sh = (lo - c) / ax, (hi - c) / ax
            near = np.clip(0.0, sl, sh)
            far = np.maximum(np.abs(sl), np.abs(sh))
            dmin = np.sqrt((near * near).sum(axis=1))
            dmax = np.sqrt((far * far).sum(axis=1))
            cov = dmax <= 1.0
            covered |= cov
            body[cov] = k
            cut = (dmin < 1.0) & ~cov
            ncut += cut
            body[cut & ~covered] = k
        flag[ncut > 0] = 2
        flag[covered] = 0
        if np.any((ncut > 1) & ~covered):
            raise RuntimeError("two ellipses reach into one cell or face")
        body[flag == 1] = -1
        return flag, body

    # ------------------------------------------------------------ one cut cell
    def _arcs(self, cx, cy, A, B):
        """Angle intervals of the arc inside the square [-1/2, 1/2]^2 (ellipse centre (cx, cy), semi-axes
        A, B in cell units)."""
        ang = []
        for e in (-0.5, 0.5):
            c = (e - cx) / A
            if abs(c) < 1.0:
                t = math.acos(c)
                for tt in (t, -t):
                    if -0.5 <= cy + B * math.sin(tt) <= 0.5:
                        ang.append(tt)
            s = (e - cy) / B
            if abs(s) < 1.0:
                t = math.asin(s)
                for tt in (t, math.pi - t):
                    if -0.5 <= cx + A * math.cos(tt) <= 0.5:
                        ang.append(math.atan2(math.sin(tt), math.cos(tt)))
        if not ang:
            inside = cx - A > -0.5 and cx + A < 0.5 and cy - B > -0.5 and cy + B < 0.5
            return [(-math.pi, math.pi)] if inside else []
        ang = sorted(ang)
        out = []
        for i, a in enumerate(ang):
            e = ang[i + 1] if i + 1 < len(ang) else ang[0] + 2 * math.pi
            if e - a <= 0.0:
                continue
            m = 0.5 * (a + e)
            if -0.5 < cx + A * math.cos(m) < 0.5 and -0.5 < cy + B * math.sin(m) < 0.5:
                out.append((a, e))
        return out

    def _arc_nodes(self, arcs):
        ts, ws = [], []
        for a, e in arcs:
            npc = max(1, int(math.ceil((e - a) / (0.125 * math.pi))))
            span = (e - a) / npc
            for pc in range(npc):
                m = a + (pc + 0.5) * span
                ts.append(m + 0.5 * span * _GL_X)
                ws.append(0.5 * span * _GL_W)
        return (np.concatenate(ts), np.concatenate(ws)) if ts else (np.zeros(0), np.zeros(0))

    def _edge_fluid(self, e, dirn, cx, cy, A, B, q):
        """int over the fluid part of the edge line (coordinate dirn = e) of t^k, t the other coordinate."""
        cn, ct, an, at = (cx, cy, A, B) if dirn == 0 else (cy, cx, B, A)
        full = _seg_pow(-0.5, 0.5, q)
        r = (e - cn) / an
        if abs(r) >= 1.0:
            return full
        w = at * math.sqrt(1.0 - r * r)
        lo, hi = max(-0.5, ct - w), min(0.5, ct + w)
        return full - (_seg_pow(lo, hi, q) if hi > lo else 0.0)

    def _cell(self, cell, body):
        N, h, q = self.N, self.h, self.qmax
        mons = monomials(2, q)
        i, j = cell % N, cell // N
        c = self.centers[body]
        A, B = self.axes[body] / h
        cx, cy = (c[0] - (i + 0.5) * h) / h, (c[1] - (j + 0.5) * h) / h
        arcs = self._arcs(cx, cy, A, B)
        t, w = self._arc_nodes(arcs)
        x, y = cx + A * np.cos(t), cy + B * np.sin(t)
        ds = np.sqrt((A * np.sin(t)) ** 2 + (B * np.cos(t)) ** 2)
        nx, ny = -B * np.cos(t), -A * np.sin(t)  # n ds / dt, n out of the fluid
        eb = np.array([np.sum(w * ds * x ** p * y ** r) for p, r in mons])
        ebn = np.array([[np.sum(w * nx * x ** p * y ** r) for p, r in mons],
                        [np.sum(w * ny * x ** p * y ** r) for p, r in mons]])
        # divergence direction: the axis along which the arc's normal is smallest (mid-arc)
        tm = float(np.mean(t)) if len(t) else 0.0
        dd = 0 if abs(B * math.cos(tm)) <= abs(A * math.sin(tm)) else 1
        vol = np.zeros(len(mons))
        for m, (p, r) in enumerate(mons):
            pd = p if dd == 0 else r
            acc = 0.0
            for e in (-0.5, 0.5):
                side = self._edge_fluid(e, dd, cx, cy, A, B, q + 1)
                other = r if dd == 0 else p
                acc += math.copysign(1.0, e) * e ** (pd + 1) * side[other]
            nd = nx if dd == 0 else ny
            acc += np.sum(w * nd * (x ** (p + (dd == 0)) * y ** (r + (dd == 1))))
            vol[m] = acc / (pd + 1)
        return vol, eb, ebn

    def _face(self, d, f, body):
        N, h, q = self.N, self.h, self.qmax
        m0 = N + (d == 0)
        i, j = f % m0, f // m0
        c = self.centers[body]
        A, B = self.axes[body] / h
        if d == 0:  # x-face at x = i h, tangential y about the face centre
            r = (i * h - c[0]) / h / A
            ct, at = (c[1] - (j + 0.5) * h) / h, B
        else:
            r = (j * h - c[1]) / h / B
            ct, at = (c[0] - (i + 0.5) * h) / h, A
        full = _seg_pow(-0.5, 0.5, q)
        if abs(r) >= 1.0:
            return full
        w = at * math.sqrt(1.0 - r * r)
        lo, hi = max(-0.5, ct - w), min(0.5, ct + w)
        return full - (_seg_pow(lo, hi, q) if hi > lo else 0.0)

    # ------------------------------------------------------------ build
    def _build(self):
        N, h, q = self.N, self.h, self.qmax
        K = len(monomials(2, q))
        idx = np.arange(self.ncell)
        lo = np.stack([(idx % N) * h, (idx // N) * h], axis=1)
        flag, body = self._classify(lo, lo + h)
        cut = np.nonzero(flag == 2)[0]
        vol = np.zeros((len(cut), K))
        eb = np.zeros((len(cut), K))
        ebn = np.zeros((len(cut), 2, K))
        for k, cell in enumerate(cut):
            vol[k], eb[k], ebn[k] = self._cell(int(cell), int(body[cell]))
        kap = vol[:, 0] if len(cut) else np.zeros(0)
        to_full, to_cov = kap >= 1.0 - KAPPA_EPS, kap <= KAPPA_EPS
        flag[cut[to_full]] = 1
        flag[cut[to_cov]] = 0
        keep = ~(to_full | to_cov)
        self.cut_cells = cut[keep].astype(np.int32)
        self.cut_body = body[cut][keep]
        self.vol_mom = np.ascontiguousarray(vol[keep])
        self.eb_mom = np.ascontiguousarray(eb[keep])
        self.eb_nmom = np.ascontiguousarray(ebn[keep])
        self.flag = flag.astype(np.uint8)
        self.kappa = (self.flag == 1).astype(np.float64)
        self.kappa[self.cut_cells] = self.vol_mom[:, 0]
        self.face_flag, self.cut_faces, self.face_mom, self.cut_face_body = [], [], [], []
        fl = self.flag.reshape(N, N)
        for d in range(2):
            shape = (N, N + 1) if d == 0 else (N + 1, N)  # (y, x) extents of the faces normal to d
            nf = shape[0] * shape[1]
            m0 = N + (d == 0)
            idx = np.arange(nf)
            lo = np.stack([(idx % m0) * h, (idx // m0) * h], axis=1)
            hi = lo + np.array([0.0, h] if d == 0 else [h, 0.0])
            ff, fb = self._classify(lo, hi)
            cf = np.nonzero(ff == 2)[0]
            fm = np.array([self._face(d, int(f), int(fb[f])) for f in cf]).reshape(len(cf), q + 1)
            al = fm[:, 0] if len(cf) else np.zeros(0)
            tfull, tcov = al >= 1.0 - KAPPA_EPS, al <= KAPPA_EPS
            ff[cf[tfull]] = 1
            ff[cf[tcov]] = 0
            keepf = ~(tfull | tcov)
            ffs = ff.astype(np.uint8).reshape(shape)
            cov = fl == 0
            ax = 1 if d == 0 else 0
            lo_c = np.concatenate([np.zeros_like(np.take(cov, [0], axis=ax)), cov], axis=ax)
            hi_c = np.concatenate([cov, np.zeros_like(np.take(cov, [0], axis=ax))], axis=ax)
            shut = (ffs > 0) & (lo_c | hi_c)
            ffs[shut] = 0
            ff = ffs.reshape(-1)
            keepf &= ff[cf] == 2
            self.face_flag.append(ff)
            self.cut_faces.append(cf[keepf].astype(np.int32))
            self.cut_face_body.append(fb[cf][keepf])
            self.face_mom.append(np.ascontiguousarray(fm[keepf]))

    def nface(self, d: int) -> int:
        return (self.N + (d == 0)) * (self.N + (d == 1))

    def face_shape(self, d: int):
        return (self.N + (d == 0), self.N + (d == 1))

    def alpha(self, d: int) -> np.ndarray:
        a = (self.face_flag[d] == 1).astype(np.float64)
        a[self.cut_faces[d]] = self.face_mom[d][:, 0]
        return a


def ellipse_batch_config(N: int, cx: float, cy: float, a: float, b: float, qmax: int = 4) -> EllipseGeometry:
    """The unit square minus one axis-aligned ellipse (a many-instance batch member)."""
    return EllipseGeometry(N, [(cx, cy)], [(a, b)], qmax, name=f"ellipse-{N}")

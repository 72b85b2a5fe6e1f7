"""Plain FP64 oracle of the adjoint of the cut-cell Poisson discretisation with respect to a
geometry parameter (Devendran, Graves, Johansen, arXiv:1411.4283): the unit square minus circles
(2-D) or the unit cube minus spheres (3-D), derivative with respect to one body's radius.

TEST INFRASTRUCTURE, like eb_oracle.py: only tests/ may import it; the GPU library never does.

Objective and problem: phi solves the kappa-weighted system kappa L phi = kappa rho with rho = 1
and homogeneous Dirichlet data on the walls and the circles (Sec. 2.3); J = 1/2 sum_v |V_v| phi_v^2.
Its derivative with respect to the radius r of one circle, by the adjoint method:

    R(phi, r) = kappa L phi - kappa = 0,   (kappa L)^T lam = |V| phi,
    dJ/dr = sum_v (h^D phi_v^2 / 2 + lam_v) dkappa_v/dr - lam^T (d(kappa L)/dr) phi,

where kappa L = (1/h^2) sum_f sigma s_hat_f (Sec. 2.3) changes through the stencils of the faces
whose LS systems hold moments of cut cells, cut faces or EB faces.  Each stencil's change is taken
through the reverse-mode derivative of its solve (stencil_adjoint) and the derivatives of its
rows and right-hand side with respect to the moment tables; those come from the moment tables'
shape derivatives (below), pushed through the oracle's own row construction by the complex step
(Squire and Trapp 1998: f(m + i e dm) = f(m) + i e f'(m) dm + O(e^2), no cancellation), the rows
being analytic functions of the moments.

Shape derivatives of the moment tables (fluid outside the circle, boundary moving out with unit
normal speed as r grows; xi = (x - x_c)/h about the cell or face centre):
  volume moments   d/dr int_V xi^p dV / h^2 = - int_{EB patch} xi^p ds / h^2 = - eb_mom / h;
  EB moments       the patch is the arc {c + r e(t)}, t in [ta, tb]:
                   d/dr int f r dt = int (r grad f . e + f) dt + f(tb) r tb' - f(ta) r ta',
                   with the endpoint angles moving along the cell edges they lie on;
  face moments     the covered chord |t - c_t| < s, s = (r^2 - (x_n - c_n)^2)^(1/2), grows at both
                   ends with speed r / s.
The cut-cell and cut-face sets are held fixed (the derivative of a fixed topology).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse.linalg as spla

from .eb_oracle import Oracle, Params, stencil_adjoint

_GL_X, _GL_W = np.polynomial.legendre.leggauss(24)


def _arcs(cx, cy, r, x0, x1, y0, y1):
    """Arcs of the circle inside the box [x0,x1]x[y0,y1]: list of ((ta, dta), (tb, dtb)) with the
    endpoint angles and their derivatives with respect to r (ta < tb)."""
    pts = []  # (angle, dtheta/dr)
    for xe in (x0, x1):
        q = r * r - (xe - cx) ** 2
        if q > 0:
            for sg in (-1.0, 1.0):
                y = cy + sg * math.sqrt(q)
                if y0 < y < y1:
                    t = math.atan2(y - cy, xe - cx) % (2 * math.pi)
                    pts.append((t, math.cos(t) / (r * math.sin(t))))
    for ye in (y0, y1):
        q = r * r - (ye - cy) ** 2
        if q > 0:
            for sg in (-1.0, 1.0):
                x = cx + sg * math.sqrt(q)
                if x0 < x < x1:
                    t = math.atan2(ye - cy, x - cx) % (2 * math.pi)
                    pts.append((t, -math.sin(t) / (r * math.cos(t))))
    pts.sort()
    arcs = []
    for i in range(len(pts)):
        a = pts[i]
        b = pts[(i + 1) % len(pts)]
        ta, tb = a[0], b[0] if i + 1 < len(pts) else b[0] + 2 * math.pi
        tm = 0.5 * (ta + tb)
        xm, ym = cx + r * math.cos(tm), cy + r * math.sin(tm)
        if x0 < xm < x1 and y0 < ym < y1:
            arcs.append(((ta, a[1]), (tb, b[1])))
    return arcs


def circle_moment_derivatives(o: Oracle, body: int):
    """d/dr of the moment tables of o.g (2-D, fluid outside the circles) for the radius of circle
    `body`: (dvol [n_cut, K], deb [n_cut, K], debn [n_cut, 2, K], dface [per d: n_cutface, K_F])."""
    g = o.g
    assert g.dim == 2 and not g.inside
    h = g.h
    cx, cy = g.centers[body, 0], g.centers[body, 1]
    r = g.radii[body]
    mons = o.store_mons
    K = len(mons)
    n_cut = len(g.cut_cells)
    deb = np.zeros((n_cut, K))
    debn = np.zeros((n_cut, 2, K))
    for k, c in enumerate(g.cut_cells):
        if g.cut_body[k] != body:
            continue
        i, j = int(c) % g.N, int(c) // g.N
        xc, yc = (i + 0.5) * h, (j + 0.5) * h
        for (ta, dta), (tb, dtb) in _arcs(cx, cy, r, i * h, (i + 1) * h, j * h, (j + 1) * h):
            t = 0.5 * (tb - ta) * _GL_X + 0.5 * (tb + ta)
            wq = 0.5 * (tb - ta) * _GL_W
            e = np.stack([np.cos(t), np.sin(t)])
            xi = np.stack([(cx + r * e[0] - xc) / h, (cy + r * e[1] - yc) / h])
            ends = []
            for tt, dt, sgn in ((ta, dta, -1.0), (tb, dtb, 1.0)):
                ee = np.array([math.cos(tt), math.sin(tt)])
                ends.append((np.array([(cx + r * ee[0] - xc) / h, (cy + r * ee[1] - yc) / h]), ee, dt, sgn))
            for m, p in enumerate(mons):
                f = xi[0] ** p[0] * xi[1] ** p[1]
                grad_e = np.zeros_like(t)  # grad_x(xi^p) . e
                if p[0] > 0:
                    grad_e += p[0] * xi[0] ** (p[0] - 1) * xi[1] ** p[1] * e[0] / h
                if p[1] > 0:
                    grad_e += p[1] * xi[0] ** p[0] * xi[1] ** (p[1] - 1) * e[1] / h
                for comp in (None, 0, 1):
                    nd = 1.0 if comp is None else -e[comp]  # normal out of the fluid: -e
                    val = np.sum(wq * (r * grad_e + f) * nd)
                    for xe, ee, dt, sgn in ends:
                        fe = xe[0] ** p[0] * xe[1] ** p[1] * (1.0 if comp is None else -ee[comp])
                        val += sgn * fe * r * dt
                    if comp is None:
                        deb[k, m] += val / h
                    else:
                        debn[k, comp, m] += val / h
    dvol = np.zeros((n_cut, K))
    mine = g.cut_body == body
    dvol[mine] = -g.eb_mom[mine] / h  # transport theorem: the fluid loses the patch
    dface = []
    for d in range(2):
        cf = g.cut_faces[d]
        qn = g.face_mom[d].shape[1]
        out = np.zeros((len(cf), qn))
        for k, f in enumerate(cf):
            if g.cut_face_body[d][k] != body:
                continue
            ijk = o.face_coords(d, int(f))
            xn = ijk[d] * h                       # normal coordinate of the face
            tdim = 1 - d
            t0, t1 = ijk[tdim] * h, (ijk[tdim] + 1) * h
            tcen = 0.5 * (t0 + t1)
            cn, ct = (cx, cy) if d == 0 else (cy, cx)
            q = r * r - (xn - cn) ** 2
            if q <= 0:
                continue
            s = math.sqrt(q)
            for end in (ct - s, ct + s):
                if t0 < end < t1:
                    eta = (end - tcen) / h
                    for m in range(qn):
                        out[k, m] -= eta ** m * (r / s) / h
        dface.append(out)
    return dvol, deb, debn, dface


def circle_velocity_derivatives(o: Oracle, body: int, V, gradV):
    """Moment-table derivatives of o.g (2-D, fluid outside the circles) when circle `body`'s boundary
    moves with the normal speed V(x) along N = (x - c)/r (out of the body), gradV(x) its gradient:
    the general form of circle_moment_derivatives (V = 1) -- a centre translation t is V = N . t, a
    level-set perturbation psi + a f(x) of the distance function is V = -f.  On the boundary
        d/dt int_patch F ds = int (grad F . N V + kappa F V) ds + sum_ends F s_end,   kappa = 1/r,
        d/dt N = -grad_G V (the surface gradient), so d/dt n = +grad_G V for n = -N,
    an arc end on an edge line moves along the line with normal component V (its arc-length speed
    is V times the radius-change speed r dt/dr), a chord end on a face with speed V r / s, and the
    volume loses int_patch xi^p V ds.  V and gradV take arrays x[2, m] and return [m] and [2, m]."""
    g = o.g
    assert g.dim == 2 and not g.inside
    h = g.h
    c = g.centers[body, :2]
    r = g.radii[body]
    mons = o.store_mons
    K = len(mons)
    n_cut = len(g.cut_cells)
    dvol = np.zeros((n_cut, K))
    deb = np.zeros((n_cut, K))
    debn = np.zeros((n_cut, 2, K))
    for k, cc in enumerate(g.cut_cells):
        if g.cut_body[k] != body:
            continue
        i, j = int(cc) % g.N, int(cc) // g.N
        xcell = np.array([(i + 0.5) * h, (j + 0.5) * h])
        for (ta, dta), (tb, dtb) in _arcs(c[0], c[1], r, i * h, (i + 1) * h, j * h, (j + 1) * h):
            t = 0.5 * (tb - ta) * _GL_X + 0.5 * (tb + ta)
            ds = 0.5 * (tb - ta) * _GL_W * r
            N = np.stack([np.cos(t), np.sin(t)])
            x = c[:, None] + r * N
            xi = (x - xcell[:, None]) / h
            v = V(x)
            gv = gradV(x)
            gG = gv - np.sum(gv * N, axis=0) * N  # surface gradient
            ends = []
            for tt, dt, sgn in ((ta, dta, -1.0), (tb, dtb, 1.0)):
                Ne = np.array([math.cos(tt), math.sin(tt)])
                xe = c + r * Ne
                ends.append(((xe - xcell) / h, Ne, sgn * float(V(xe[:, None])[0]) * r * dt))
            for m, p in enumerate(mons):
                f = xi[0] ** p[0] * xi[1] ** p[1]
                gN = np.zeros_like(t)  # grad_x(xi^p) . N
                if p[0] > 0:
                    gN += p[0] * xi[0] ** (p[0] - 1) * xi[1] ** p[1] * N[0] / h
                if p[1] > 0:
                    gN += p[1] * xi[0] ** p[0] * xi[1] ** (p[1] - 1) * N[1] / h
                dvol[k, m] -= np.sum(ds * f * v) / h ** 2
                deb[k, m] += (np.sum(ds * (gN * v + f * v / r)) + sum(
                    xe[0] ** p[0] * xe[1] ** p[1] * se for xe, _, se in ends)) / h
                for d in range(2):
                    val = np.sum(ds * (gN * v * -N[d] + f * gG[d] + f * -N[d] * v / r))
                    val += sum(xe[0] ** p[0] * xe[1] ** p[1] * -Ne[d] * se for xe, Ne, se in ends)
                    debn[k, d, m] += val / h
    dface = []
    for d in range(2):
        cf = g.cut_faces[d]
        qn = g.face_mom[d].shape[1]
        out = np.zeros((len(cf), qn))
        for k, f in enumerate(cf):
            if g.cut_face_body[d][k] != body:
                continue
            ijk = o.face_coords(d, int(f))
            xn = ijk[d] * h
            tdim = 1 - d
            t0, t1 = ijk[tdim] * h, (ijk[tdim] + 1) * h
            tcen = 0.5 * (t0 + t1)
            q = r * r - (xn - c[d]) ** 2
            if q <= 0:
                continue
            s_ = math.sqrt(q)
            for end in (c[tdim] - s_, c[tdim] + s_):
                if t0 < end < t1:
                    xe = np.zeros(2)
                    xe[d], xe[tdim] = xn, end
                    speed = float(V(xe[:, None])[0]) * r / s_
                    eta = (end - tcen) / h
                    for m in range(qn):
                        out[k, m] -= eta ** m * speed / h
        dface.append(out)
    return dvol, deb, debn, dface


def sphere_velocity_derivatives(o: Oracle, body: int, V, gradV):
    """Moment-table derivatives of o.g (3-D, fluid outside the spheres) when sphere `body`'s surface
    moves with the normal speed V(x) along N = (x - c)/r: the 3-D counterpart of
    circle_velocity_derivatives, with the patch and its edges from the moment oracle's quadrature.
        d/dt int_patch F dA = int (grad F . N V + (2/r) F V) dA + oint_edges F V_e dl,
        V_e = -V (N . n_p) / (1 - (N . n_p)^2)^(1/2)    (n_p the cell face's normal out of the cell),
        d/dt n = +grad_G V for n = -N,  the volume loses int_patch xi^p V dA,
    and a face's covered disk grows along its rim with speed V r / rho."""
    from .eb_moments import sphere_patch_edges, sphere_patch_nodes
    from eb_inputs.geometry import monomials
    g = o.g
    assert g.dim == 3 and not g.inside
    h, N = g.h, g.N
    c = g.centers[body]
    r = g.radii[body]
    mons = o.store_mons
    K = len(mons)
    n_cut = len(g.cut_cells)
    dvol = np.zeros((n_cut, K))
    deb = np.zeros((n_cut, K))
    debn = np.zeros((n_cut, 3, K))
    for k in np.nonzero(g.cut_body == body)[0]:
        cc = int(g.cut_cells[k])
        ijk = np.array([cc % N, (cc // N) % N, cc // (N * N)], float)
        lo, hi = ijk * h, (ijk + 1) * h
        xcell = lo + 0.5 * h
        x, w = sphere_patch_nodes(c, r, lo, hi)
        Nn = (x - c[:, None]) / r
        xi = (x - xcell[:, None]) / h
        v = V(x)
        gv = gradV(x)
        gG = gv - (gv * Nn).sum(0) * Nn
        edges = []
        for xe, we, n_p in sphere_patch_edges(c, r, lo, hi):
            Ne = (xe - c[:, None]) / r
            en = (Ne * n_p[:, None]).sum(0)
            edges.append(((xe - xcell[:, None]) / h, Ne, we * V(xe) * -en / np.sqrt(1.0 - en * en)))
        for m, p in enumerate(mons):
            f = xi[0] ** p[0] * xi[1] ** p[1] * xi[2] ** p[2]
            gN = np.zeros_like(f)
            for d in range(3):
                if p[d] > 0:
                    q = list(p)
                    q[d] -= 1
                    gN += p[d] * xi[0] ** q[0] * xi[1] ** q[1] * xi[2] ** q[2] * Nn[d] / h
            dvol[k, m] = -np.sum(w * f * v) / h ** 3
            val = np.sum(w * (gN * v + 2.0 / r * f * v))
            for xe, Ne, se in edges:
                val += np.sum(se * xe[0] ** p[0] * xe[1] ** p[1] * xe[2] ** p[2])
            deb[k, m] = val / h ** 2
            for d in range(3):
                val = np.sum(w * (gN * v * -Nn[d] + f * gG[d] + 2.0 / r * f * -Nn[d] * v))
                for xe, Ne, se in edges:
                    val += np.sum(se * xe[0] ** p[0] * xe[1] ** p[1] * xe[2] ** p[2] * -Ne[d])
                debn[k, d, m] = val / h ** 2
    deg = max(sum(m) for m in mons)
    dface = []
    for d in range(3):
        cf = g.cut_faces[d]
        tm = monomials(2, deg)[:g.face_mom[d].shape[1]]
        oth = [b for b in range(3) if b != d]
        out = np.zeros((len(cf), len(tm)))
        for k, f in enumerate(cf):
            if g.cut_face_body[d][k] != body:
                continue
            ijk = o.face_coords(d, int(f))
            pa = ijk[d] * h
            q2 = r * r - (pa - c[d]) ** 2
            if q2 <= 0:
                continue
            rho = math.sqrt(q2)
            lo = [ijk[b] * h for b in oth]
            hi = [(ijk[b] + 1) * h for b in oth]
            fc = [(ijk[b] + 0.5) * h for b in oth]
            for (ta, _), (tb, _) in _arcs(c[oth[0]], c[oth[1]], rho, lo[0], hi[0], lo[1], hi[1]):
                t = 0.5 * (tb - ta) * _GL_X + 0.5 * (tb + ta)
                wq = 0.5 * (tb - ta) * _GL_W * rho
                xr = np.zeros((3, len(t)))
                xr[d] = pa
                xr[oth[0]] = c[oth[0]] + rho * np.cos(t)
                xr[oth[1]] = c[oth[1]] + rho * np.sin(t)
                speed = V(xr) * r / rho
                u = (xr[oth[0]] - fc[0]) / h
                vv = (xr[oth[1]] - fc[1]) / h
                for m, (pu, pv) in enumerate(tm):
                    out[k, m] -= np.sum(wq * speed * u ** pu * vv ** pv) / h ** 2
        dface.append(out)
    return dvol, deb, debn, dface


def fourier_mode_velocity(k, theta):
    """Normal speed of the boundary of the distance-function level set psi + a f = 0 per unit a at
    a = 0, for the mode f(x) = sin(2 pi k . x + theta) (|grad psi| = 1): V = -f, grad V = -grad f."""
    k = np.asarray(k, float)

    def V(x):
        return -np.sin(2 * math.pi * (k[:, None] * x).sum(0) + theta)

    def gradV(x):
        return -2 * math.pi * k[:, None] * np.cos(2 * math.pi * (k[:, None] * x).sum(0) + theta)
    return V, gradV


def fourier_mode_derivatives(o: Oracle, k, theta):
    """Moment-table derivatives with respect to the amplitude a of the mode sin(2 pi k . x + theta)
    added to the distance-function level set of all the bodies, at a = 0: every body's boundary
    moves with V = -sin(...)."""
    V, gradV = fourier_mode_velocity(k, theta)
    fn = circle_velocity_derivatives if o.g.dim == 2 else sphere_velocity_derivatives
    parts = [fn(o, b, V, gradV) for b in range(len(o.g.radii))]
    dvol = sum(p_[0] for p_ in parts)
    deb = sum(p_[1] for p_ in parts)
    debn = sum(p_[2] for p_ in parts)
    dface = [sum(p_[3][d] for p_ in parts) for d in range(o.g.dim)]
    return dvol, deb, debn, dface


def _mono_index(D, deg):
    from eb_inputs.geometry import monomials
    ms = monomials(D, deg)
    return ms, {m: i for i, m in enumerate(ms)}


def sphere_moment_derivatives(o: Oracle, body: int):
    """d/dr of the moment tables of o.g (3-D, fluid outside the spheres) for the radius of sphere
    `body`.  On the sphere, with e = (x - c)/r (n = -e out of the fluid, mean curvature 2/r):
        d/dr int_{patch} f dA = int_{patch} (d f/d rho + (2/r) f) dA + oint_{edge} f V dl,
    where the patch's edge lies on the cell's faces and moves, inside the sphere, with the outward
    conormal speed V = -(e . n_p) / (1 - (e . n_p)^2)^(1/2) (n_p the face's normal out of the cell);
    the surface integrals come from the generator's patch quadrature of higher-degree monomials,
    the edge integrals from Gauss-Legendre on the edge arcs.  Face moments: the covered disk of radius
    rho = (r^2 - (x_n - c_n)^2)^(1/2) grows with speed r / rho along its rim."""
    g = o.g
    assert g.dim == 3 and not g.inside
    h, N = g.h, g.N
    c = g.centers[body]
    r = g.radii[body]
    mons = o.store_mons
    K = len(mons)
    deg = max(sum(m) for m in mons)
    big, bidx = _mono_index(3, deg + 2)
    mine = np.nonzero(g.cut_body == body)[0]
    cells = g.cut_cells[mine].astype(np.int64)
    terms = g._terms_mono(3, deg + 2)
    M = g.eb_integrals(cells, g.cut_body[mine], g._basis_pow(deg + 2), terms, ncomp=-1)  # int xi^t dA / h^2
    n_cut = len(g.cut_cells)
    deb = np.zeros((n_cut, K))
    debn = np.zeros((n_cut, 3, K))
    for row, k in enumerate(mine):
        cc = int(g.cut_cells[k])
        ijk = [cc % N, (cc // N) % N, cc // (N * N)]
        xc = (np.array(ijk) + 0.5) * h
        a = xc - c  # x - c = h xi + a
        Mk = M[row]

        def mom(t):
            return Mk[bidx[tuple(t)]]

        def ee_mom(q, kk, d):  # int xi^q e_kk e_d dA / h^2, e = (h xi + a) / r
            t = list(q)
            out = a[kk] * a[d] * mom(t)
            t1 = list(q); t1[kk] += 1
            out += h * a[d] * mom(t1)
            t2 = list(q); t2[d] += 1
            out += h * a[kk] * mom(t2)
            t3 = list(q); t3[kk] += 1; t3[d] += 1
            out += h * h * mom(t3)
            return out / (r * r)

        def e_mom(q, kk):  # int xi^q e_kk dA / h^2
            t1 = list(q); t1[kk] += 1
            return (a[kk] * mom(q) + h * mom(t1)) / r

        for m, p in enumerate(mons):
            # d(xi^p)/d rho = sum_kk (p_kk / h) xi^(p - e_kk) e_kk
            v = 2.0 / r * mom(p)
            for kk in range(3):
                if p[kk] > 0:
                    q = list(p); q[kk] -= 1
                    v += p[kk] / h * e_mom(q, kk)
            deb[k, m] += v
            for d in range(3):  # f = xi^p n_d = -xi^p e_d
                t1 = list(p); t1[d] += 1
                v = -2.0 / r * e_mom(p, d)
                for kk in range(3):
                    if p[kk] > 0:
                        q = list(p); q[kk] -= 1
                        v -= p[kk] / h * ee_mom(q, kk, d)
                debn[k, d, m] += v
        # edges: the sphere's circles on the six faces of the cell, inside each face
        lo, hi = np.array(ijk) * h, (np.array(ijk) + 1) * h
        for ax in range(3):
            oth = [b for b in range(3) if b != ax]
            for side, pa in ((-1.0, lo[ax]), (1.0, hi[ax])):
                q2 = r * r - (pa - c[ax]) ** 2
                if q2 <= 0:
                    continue
                rho = math.sqrt(q2)
                for (ta, _), (tb, _) in _arcs(c[oth[0]], c[oth[1]], rho, lo[oth[0]], hi[oth[0]], lo[oth[1]], hi[oth[1]]):
                    t = 0.5 * (tb - ta) * _GL_X + 0.5 * (tb + ta)
                    wq = 0.5 * (tb - ta) * _GL_W * rho  # dl
                    x = np.zeros((3, len(t)))
                    x[ax] = pa
                    x[oth[0]] = c[oth[0]] + rho * np.cos(t)
                    x[oth[1]] = c[oth[1]] + rho * np.sin(t)
                    e = (x - c[:, None]) / r
                    en = side * e[ax]  # e . n_p
                    V = -en / np.sqrt(1.0 - en * en)
                    xi = (x - xc[:, None]) / h
                    for m, p in enumerate(mons):
                        f = xi[0] ** p[0] * xi[1] ** p[1] * xi[2] ** p[2]
                        deb[k, m] += np.sum(wq * f * V) / h ** 2
                        for d in range(3):
                            debn[k, d, m] += np.sum(wq * f * (-e[d]) * V) / h ** 2
    dvol = np.zeros((n_cut, K))
    dvol[mine] = -g.eb_mom[mine] / h
    dface = []
    from eb_inputs.geometry import monomials
    for d in range(3):
        cf = g.cut_faces[d]
        tm = monomials(2, deg)[:g.face_mom[d].shape[1]]  # the face tables' tangential monomials
        oth = [b for b in range(3) if b != d]
        out = np.zeros((len(cf), len(tm)))
        for k, f in enumerate(cf):
            if g.cut_face_body[d][k] != body:
                continue
            ijk = o.face_coords(d, int(f))
            pa = ijk[d] * h
            q2 = r * r - (pa - c[d]) ** 2
            if q2 <= 0:
                continue
            rho = math.sqrt(q2)
            lo = [ijk[b] * h for b in oth]
            hi = [(ijk[b] + 1) * h for b in oth]
            fc = [(ijk[b] + 0.5) * h for b in oth]
            for (ta, _), (tb, _) in _arcs(c[oth[0]], c[oth[1]], rho, lo[0], hi[0], lo[1], hi[1]):
                t = 0.5 * (tb - ta) * _GL_X + 0.5 * (tb + ta)
                wq = 0.5 * (tb - ta) * _GL_W * rho
                u = (c[oth[0]] + rho * np.cos(t) - fc[0]) / h
                v = (c[oth[1]] + rho * np.sin(t) - fc[1]) / h
                for m, (pu, pv) in enumerate(tm):
                    out[k, m] -= np.sum(wq * u ** pu * v ** pv) * (r / rho) / h ** 2
        dface.append(out)
    return dvol, deb, debn, dface


def moment_derivatives(o: Oracle, body: int):
    return circle_moment_derivatives(o, body) if o.g.dim == 2 else sphere_moment_derivatives(o, body)


def _perturbed(o: Oracle, dm, eps):
    """The oracle's geometry arrays moved to m + i eps dm (complex step)."""
    g = o.g
    dvol, deb, debn, dface = dm
    g.vol_mom = g.vol_mom + 1j * eps * dvol
    g.eb_mom = g.eb_mom + 1j * eps * deb
    g.eb_nmom = g.eb_nmom + 1j * eps * debn
    g.face_mom = [fm + 1j * eps * df for fm, df in zip(g.face_mom, dface)]


def _restore(o: Oracle, saved):
    g = o.g
    g.vol_mom, g.eb_mom, g.eb_nmom, g.face_mom = saved


def objective_and_radius_gradient(g, body: int = 0, params: Params | None = None, derivs=None):
    """(J, dJ/dr) for the radius of circle `body` (see the module docstring); derivs(o) -> the moment
    tables' derivatives for another geometry parameter (default: that radius)."""
    o = Oracle(g, params or Params(order=4))
    h, D = g.h, g.dim
    st = o.all_stencils()
    L, _ = o.operator(st, kappa_weighted=True)
    vol = g.flag > 0
    idx = np.nonzero(vol)[0]
    A = L[idx][:, idx].tocsc()
    kap = g.kappa
    phi = np.zeros(g.ncell)
    phi[idx] = spla.spsolve(A, kap[idx])
    w = kap * h ** D
    J = 0.5 * float(np.sum(w * phi * phi))
    lam = np.zeros(g.ncell)
    lam[idx] = spla.spsolve(A.T.tocsc(), (w * phi)[idx])
    dm = moment_derivatives(o, body) if derivs is None else derivs(o)
    dkap = np.zeros(g.ncell)
    dkap[g.cut_cells] = dm[0][:, 0]
    dJ = float(np.sum((0.5 * h ** D * phi * phi + lam) * dkap))
    # stencil terms: -lam^T (d(kappa L)/dr) phi = sum_f <c_f, d s_hat_f>, c_f[i] = -(1/h^2) sum_v sigma lam_v phi_col_i
    eps = 1e-20
    saved = (g.vol_mom, g.eb_mom, g.eb_nmom, g.face_mom)
    for fid in o.flux_faces():
        A0, F0, wf, cols = o.face_system(fid)
        _perturbed(o, dm, eps)
        o._full_rows.clear()
        try:
            Ac, Fc, _, _ = o.face_system(fid)
        finally:
            _restore(o, saved)
            o._full_rows.clear()
        dA, dF = np.imag(Ac) / eps, np.imag(Fc) / eps
        if not (np.any(dA) or np.any(dF)):
            continue
        cvec = np.zeros(len(cols))
        vm = cols >= 0
        for c, sg in o.face_cells(fid):
            cvec[vm] -= sg * lam[c] * phi[cols[vm]] / h ** 2
        Abar, Fbar = stencil_adjoint(np.real(A0), np.real(F0), wf, cvec)
        dJ += float(np.sum(Abar * dA) + np.sum(Fbar * dF))
    return J, dJ

"""Plain, slow, single-threaded FP64 oracle of the higher-order cut-cell
finite-volume Poisson discretisation (Devendran, Graves, Johansen,
arXiv:1411.4283).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline leg may import or run this module; the GPU
library never does, and this module imports nothing from it.  Its only shared
dependency is the input generator ``eb_inputs`` (geometry moments, seeded
random numbers), which holds none of the method's arithmetic.

Everything is computed face by face from the paper's definitions:

* interpolant of degree |p| <= Q (Sec. 2.2, "|p| < P" with P = Q + 1);
* rows of A: volume averages of the monomials (Sec. 2.2.1, Eq. "volume
  moment eq for cp" / A_{v p} = m^p_v(x0) / m^0_v) and Dirichlet boundary-face
  averages (b_{f_b p} = m^p_{f_b} / m^0_{f_b}); Neumann rows
  b_{f_b p} = (1/m^0) sum_d p_d m^{p - e_d}_{d, f_b};
* F_p = integral over the face of grad (x - x0)^p . n (Sec. 2.2.1);
* stencil s = W (A^T W)^+ F, i.e. the solution of A^T s = F with the least
  ||W^{-1} s||_2 (Eqs. "stencil equation solution", "stencil equation"),
  computed as W times the minimum-norm solution of (W A)^T t = F (numpy's
  SVD-based lstsq);
* neighbours: volumes within path radius R_n of the face's adjacent volumes,
  plus the boundary faces those volumes touch (Sec. 2.4); paths go through
  open grid faces;
* weights W_ii = 1 if |x_i - x0|/h < 1/2 else (2 |x_i - x0|/h)^{-5}, x_i the
  cell centre (volume), face centre (grid-aligned boundary face) or centre of
  the cut cell (EB face); x0 the face centre (grid face) or the centre of the
  cut cell (EB face) (Sec. 2.4);
* operator L_v = (1/|V_v|) sum_{f(v)} sigma_{v,f} s_f^T Phi, and its
  kappa-weighted form kappa_v L_v (Sec. 2.3);
* error norms of Sec. 3.3.

All moments are used in h-scaled coordinates xi = (x - x0)/h: since A^T s = F
is homogeneous in h, s = h^{D-2} s_hat with s_hat from the scaled system.

Readings of passages that are silent, ambiguous or garbled: neighbourhood =
the volumes of the max-norm box of radius R_n around each adjacent volume,
reached through faces with area fraction > 0 (the face-connected path reading
is the ``metric="path"`` option); x_i and x0 are Cartesian centres (not
centroids); interior faces use the same weighted LS stencil as cut faces;
rank-deficient systems raise instead of falling back.  Neumann EB faces: the
least squares is the paper's, in physical units.  In the h-scaled system a
Neumann row is a derivative in xi, so its datum enters as h <g> and its weight
is W_ii / h (the physical minimum-norm problem, rescaled); the flux through a
Neumann EB face is the datum, |A_f| <g>_f.
"""
from __future__ import annotations

import math
from collections import deque
from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


# --------------------------------------------------------------------- monomials

def monomial_list(D: int, Q: int) -> list[tuple[int, ...]]:
    """Multi-indices p with |p| <= Q, graded, then decreasing earlier exponents."""
    out: list[tuple[int, ...]] = []
    for deg in range(Q + 1):
        if D == 0:
            out.append(())
            break
        stack = [((), deg)]
        level = []

        def rec(prefix, left):
            if len(prefix) == D - 1:
                level.append(prefix + (left,))
                return
            for p in range(left, -1, -1):
                rec(prefix + (p,), left - p)

        rec((), deg)
        out.extend(level)
        del stack
    return out


def _full_1d(q: int) -> float:
    """integral of xi^q over [-1/2, 1/2]."""
    return 0.0 if q % 2 else 0.5 ** q / (q + 1)


@dataclass
class Params:
    order: int = 4            # Q: interpolant degree (second order: 2, fourth order: 4)
    path_radius: int | None = None  # R_n; the paper uses 2 for Q=2 and 3 for Q=4 (Sec. 2.4)
    weighted: bool = True     # False: W = I (unweighted least squares, the unstable control)
    metric: str = "box"       # "box" (default): volumes of the max-norm box of radius R_n reached
                              # through open faces inside the box; "path": face-connected path
                              # distance <= R_n
    w_threshold: float = 0.5
    w_power: float = 5.0
    neumann_weight: str = "physical"  # "physical" (default): Neumann rows weighted W_ii / h in the
                              # scaled system (the physical minimum-norm problem); "scaled": W_ii

    def radius(self) -> int:
        if self.path_radius is not None:
            return self.path_radius
        return {2: 2, 4: 3}.get(self.order, (self.order + 2) // 2)


class RankDeficient(RuntimeError):
    pass


class Oracle:
    """Face-by-face FP64 construction of stencils and of the operator.

    ``geom`` is an ``eb_inputs.Geometry`` (its arrays are the same ones the
    GPU library receives).  ``bc_eb``: per cut cell 0 (Dirichlet) or 1
    (Neumann); walls are Dirichlet.
    """

    def __init__(self, geom, params: Params | None = None, bc_eb=None):
        self.g = geom
        self.p = params or Params()
        D = geom.dim
        self.D = D
        self.Q = self.p.order
        if self.Q > geom.qmax:
            raise ValueError("moment tables are not deep enough for this order")
        self.mons = monomial_list(D, self.Q)
        self.K = len(self.mons)
        self.mon_index = {m: i for i, m in enumerate(self.mons)}
        # moment tables (stored degree geom.qmax): map exponent -> column
        self.store_mons = monomial_list(D, geom.qmax)
        self.store_index = {m: i for i, m in enumerate(self.store_mons)}
        self.face_store = monomial_list(D - 1, geom.qmax) if D > 1 else [()]
        self.face_store_index = {m: i for i, m in enumerate(self.face_store)}
        self.n = list(geom.n[:D])
        self.h = geom.h
        self.flag = geom.flag
        self.cut_pos = {int(c): i for i, c in enumerate(geom.cut_cells)}
        self.face_count = [geom.nface(d) for d in range(D)]
        self.face_base = np.concatenate([[0], np.cumsum(self.face_count)]).astype(np.int64)
        self.n_grid_faces = int(self.face_base[-1])
        self.cutface_pos = [{int(f): i for i, f in enumerate(geom.cut_faces[d])} for d in range(D)]
        self.bc_eb = np.zeros(len(geom.cut_cells), dtype=np.int8) if bc_eb is None else np.asarray(bc_eb)
        self._nbr_cache: dict[int, list[int]] = {}
        self._shift_cache: dict = {}
        self._full_mom = None
        self._full_rows: dict = {}

    # ----------------------------------------------------------- indexing
    def _dtype(self):
        """float64, or complex128 when the moment tables carry a complex-step perturbation."""
        g = self.g
        return np.result_type(g.vol_mom, g.eb_mom, g.eb_nmom, *g.face_mom, np.float64)

    def cell_coords(self, c: int) -> list[int]:
        out = []
        for d in range(self.D):
            out.append(c % self.n[d])
            c //= self.n[d]
        return out

    def cell_index(self, ijk) -> int:
        c, s = 0, 1
        for d in range(self.D):
            c += ijk[d] * s
            s *= self.n[d]
        return c

    def face_local(self, d: int, ijk) -> int:
        """index of the face normal to d whose low corner index is ijk (ijk[d] in 0..n_d)."""
        c, s = 0, 1
        for k in range(self.D):
            c += ijk[k] * s
            s *= self.n[k] + (k == d)
        return c

    def face_coords(self, d: int, f: int) -> list[int]:
        out = []
        for k in range(self.D):
            m = self.n[k] + (k == d)
            out.append(f % m)
            f //= m
        return out

    def face_id(self, d: int, f: int) -> int:
        return int(self.face_base[d] + f)

    def eb_id(self, cut: int) -> int:
        return self.n_grid_faces + cut

    def decode_face(self, fid: int):
        """-> ("grid", d, local) or ("eb", cut)."""
        if fid >= self.n_grid_faces:
            return ("eb", fid - self.n_grid_faces)
        d = int(np.searchsorted(self.face_base, fid, side="right") - 1)
        return ("grid", d, fid - int(self.face_base[d]))

    def face_open(self, d: int, f: int) -> bool:
        return self.g.face_flag[d][f] > 0

    def is_volume(self, c: int) -> bool:
        return self.flag[c] > 0

    # ----------------------------------------------------------- geometry helpers
    def cell_center(self, c: int) -> np.ndarray:
        ijk = self.cell_coords(c)
        return np.array([(i + 0.5) for i in ijk])  # in units of h

    def face_center(self, d: int, f: int) -> np.ndarray:
        ijk = self.face_coords(d, f)
        return np.array([float(ijk[k]) if k == d else ijk[k] + 0.5 for k in range(self.D)])

    def cell_faces(self, c: int):
        """grid faces of cell c: list of (d, local face, sigma); sigma = +1 when the face's +e_d normal
        points out of the cell."""
        ijk = self.cell_coords(c)
        out = []
        for d in range(self.D):
            lo = list(ijk)
            out.append((d, self.face_local(d, lo), -1))
            hi = list(ijk)
            hi[d] += 1
            out.append((d, self.face_local(d, hi), +1))
        return out

    def wall_faces_of(self, c: int):
        """open faces of cell c on the box boundary, as global face ids."""
        ijk = self.cell_coords(c)
        out = []
        for d in range(self.D):
            if ijk[d] == 0:
                f = self.face_local(d, ijk)
                if self.face_open(d, f):
                    out.append(self.face_id(d, f))
            if ijk[d] == self.n[d] - 1:
                hi = list(ijk)
                hi[d] += 1
                f = self.face_local(d, hi)
                if self.face_open(d, f):
                    out.append(self.face_id(d, f))
        return out

    # ----------------------------------------------------------- neighbours (Sec. 2.4)
    def volume_neighbours(self, c: int) -> list[int]:
        """volumes within face-connected path distance R_n of volume c (c included)."""
        if c in self._nbr_cache:
            return self._nbr_cache[c]
        R = self.p.radius()
        box = self.p.metric == "box"
        c0 = self.cell_coords(c)
        seen = {c: 0}
        dq = deque([c])
        while dq:
            v = dq.popleft()
            dist = seen[v]
            if dist == R and not box:
                continue
            ijk = self.cell_coords(v)
            for d in range(self.D):
                for side in (0, 1):
                    nb = list(ijk)
                    nb[d] += 1 if side else -1
                    if nb[d] < 0 or nb[d] >= self.n[d]:
                        continue
                    if box and abs(nb[d] - c0[d]) > R:
                        continue
                    fl = list(ijk)
                    if side:
                        fl[d] += 1
                    if not self.face_open(d, self.face_local(d, fl)):
                        continue
                    w = self.cell_index(nb)
                    if w in seen or not self.is_volume(w):
                        continue
                    seen[w] = dist + 1
                    dq.append(w)
        out = sorted(seen)
        self._nbr_cache[c] = out
        return out

    def face_rows(self, fid: int):
        """Row set of the face's LS system: (volumes, wall face ids, EB cut indices), canonical order."""
        kind = self.decode_face(fid)
        if kind[0] == "eb":
            adj = [int(self.g.cut_cells[kind[1]])]
        else:
            d, f = kind[1], kind[2]
            ijk = self.face_coords(d, f)
            adj = []
            if ijk[d] > 0:
                lo = list(ijk)
                lo[d] -= 1
                adj.append(self.cell_index(lo))
            if ijk[d] < self.n[d]:
                adj.append(self.cell_index(ijk))
            adj = [a for a in adj if self.is_volume(a)]
        vols = set()
        for a in adj:
            vols.update(self.volume_neighbours(a))
        vols = sorted(vols)
        walls, ebs = set(), set()
        for v in vols:
            walls.update(self.wall_faces_of(v))
            if v in self.cut_pos:
                ebs.add(self.cut_pos[v])
        return vols, sorted(walls), sorted(ebs)

    # ----------------------------------------------------------- moments about x0
    def _shift_matrix(self, delta: tuple, dims: int, mons_out, mons_in_index):
        """S[p, q] = prod_d C(p_d, q_d) delta_d^(p_d - q_d) for q <= p: integral of (xi + delta)^p
        = sum_q S[p, q] integral of xi^q (binomial expansion)."""
        key = (delta, dims, len(mons_out), id(mons_in_index))
        S = self._shift_cache.get(key)
        if S is not None:
            return S
        S = np.zeros((len(mons_out), len(mons_in_index)))
        for i, p in enumerate(mons_out):
            ranges = [range(pd + 1) for pd in p]
            for q in np.ndindex(*[pd + 1 for pd in p]) if p else [()]:
                coef = 1.0
                for dd in range(dims):
                    coef *= math.comb(p[dd], q[dd]) * delta[dd] ** (p[dd] - q[dd])
                S[i, mons_in_index[tuple(q)]] += coef
            del ranges
        self._shift_cache[key] = S
        return S

    def volume_moments(self, c: int) -> np.ndarray:
        """stored-degree moments of volume c about its cell centre (xi units, / h^D)."""
        if c in self.cut_pos:
            return self.g.vol_mom[self.cut_pos[c]]
        if self._full_mom is None:
            self._full_mom = np.array([np.prod([_full_1d(q) for q in m]) for m in self.store_mons])
        return self._full_mom

    def volume_row(self, c: int, x0: np.ndarray) -> np.ndarray:
        """A_hat_{v,p} = M^p_v(x0) / M^0_v with M the moments shifted to x0 (binomial expansion).
        Full cells depend on the offset only, so their rows are memoised by offset."""
        delta = tuple(self.cell_center(c) - x0)
        full = c not in self.cut_pos
        if full and delta in self._full_rows:
            return self._full_rows[delta]
        S = self._shift_matrix(delta, self.D, self.mons, self.store_index)
        M = S @ self.volume_moments(c)
        row = M / M[0]
        if full:
            self._full_rows[delta] = row
        return row

    def grid_face_tangential_moments(self, d: int, f: int) -> np.ndarray:
        pos = self.cutface_pos[d].get(f)
        if pos is not None:
            return self.g.face_mom[d][pos]
        return np.array([np.prod([_full_1d(q) for q in m]) if m else 1.0 for m in self.face_store])

    def grid_face_moments(self, d: int, f: int, x0: np.ndarray, mons) -> np.ndarray:
        """D-dim moments integral_f (xi - xi0)^p dA / h^(D-1) for the listed exponents."""
        fc = self.face_center(d, f)
        delta = fc - x0
        tm = self.grid_face_tangential_moments(d, f)
        tdims = [k for k in range(self.D) if k != d]
        out = np.zeros(len(mons), dtype=self._dtype())
        for i, p in enumerate(mons):
            pt = tuple(p[k] for k in tdims)
            acc = 0.0
            for q in np.ndindex(*[e + 1 for e in pt]) if pt else [()]:
                coef = 1.0
                for j, k in enumerate(tdims):
                    coef *= math.comb(pt[j], q[j]) * delta[k] ** (pt[j] - q[j])
                acc += coef * tm[self.face_store_index[tuple(q)]]
            out[i] = acc * delta[d] ** p[d]
        return out

    def eb_moments(self, cut: int, x0: np.ndarray, normal: int | None = None) -> np.ndarray:
        c = int(self.g.cut_cells[cut])
        delta = tuple(self.cell_center(c) - x0)
        S = self._shift_matrix(delta, self.D, self.store_mons, self.store_index)
        src = self.g.eb_mom[cut] if normal is None else self.g.eb_nmom[cut, normal]
        return S @ src  # indexed by store_mons

    # ----------------------------------------------------------- rows, F, weights
    def _weight(self, xi: np.ndarray, x0: np.ndarray) -> float:
        if not self.p.weighted:
            return 1.0
        r = float(np.linalg.norm(xi - x0))
        return 1.0 if r < self.p.w_threshold else (2.0 * r) ** (-self.p.w_power)

    def face_x0(self, fid: int) -> np.ndarray:
        kind = self.decode_face(fid)
        if kind[0] == "eb":
            return self.cell_center(int(self.g.cut_cells[kind[1]]))
        return self.face_center(kind[1], kind[2])

    def _boundary_row(self, fid_or_cut, kind: str, x0) -> np.ndarray:
        if kind == "wall":
            d, f = self.decode_face(fid_or_cut)[1:]
            M = self.grid_face_moments(d, f, x0, self.mons)
            return M / M[0]
        cut = fid_or_cut
        if self.bc_eb[cut] == 0:
            M = self.eb_moments(cut, x0)
            return np.array([M[self.store_index[m]] for m in self.mons]) / M[self.store_index[(0,) * self.D]]
        # Neumann row: (1/m^0) sum_d p_d m^{p - e_d}_{d}
        m0 = self.eb_moments(cut, x0)[self.store_index[(0,) * self.D]]
        row = np.zeros(self.K, dtype=self._dtype())
        for d in range(self.D):
            N = self.eb_moments(cut, x0, normal=d)
            for i, p in enumerate(self.mons):
                if p[d] > 0:
                    q = list(p)
                    q[d] -= 1
                    row[i] += p[d] * N[self.store_index[tuple(q)]]
        return row / m0

    def flux_vector(self, fid: int, x0: np.ndarray) -> np.ndarray:
        """F_hat_p = integral over f of grad (xi)^p . n (xi about x0; grid faces: n = +e_d;
        EB faces: n out of the fluid), / h^(D-1)."""
        kind = self.decode_face(fid)
        F = np.zeros(self.K, dtype=self._dtype())
        if kind[0] == "grid":
            d, f = kind[1], kind[2]
            lower = []
            for p in self.mons:
                q = list(p)
                if q[d] > 0:
                    q[d] -= 1
                lower.append(tuple(q))
            M = self.grid_face_moments(d, f, x0, lower)
            for i, p in enumerate(self.mons):
                F[i] = p[d] * M[i] if p[d] > 0 else 0.0
            return F
        cut = kind[1]
        for d in range(self.D):
            N = self.eb_moments(cut, x0, normal=d)
            for i, p in enumerate(self.mons):
                if p[d] > 0:
                    q = list(p)
                    q[d] -= 1
                    F[i] += p[d] * N[self.store_index[tuple(q)]]
        return F

    def face_system(self, fid: int):
        """(A_hat, F_hat, w, cols): the scaled LS system of one face, rows in canonical order.
        cols: volume -> cell index; boundary face -> -(1 + face id)."""
        x0 = self.face_x0(fid)
        vols, walls, ebs = self.face_rows(fid)
        rows, w, cols = [], [], []
        for c in vols:
            rows.append(self.volume_row(c, x0))
            w.append(self._weight(self.cell_center(c), x0))
            cols.append(c)
        for wf in walls:
            rows.append(self._boundary_row(wf, "wall", x0))
            d, f = self.decode_face(wf)[1:]
            w.append(self._weight(self.face_center(d, f), x0))
            cols.append(-(1 + wf))
        for e in ebs:
            rows.append(self._boundary_row(e, "eb", x0))
            we = self._weight(self.cell_center(int(self.g.cut_cells[e])), x0)
            # Neumann row: its coefficient is h^(D-1) s_hat, not h^(D-2) s_hat, so the physical
            # minimum-norm problem weighs it with W_ii / h in the scaled system
            w.append(we / self.h if self.bc_eb[e] == 1 and self.p.neumann_weight == "physical" else we)
            cols.append(-(1 + self.eb_id(e)))
        return np.array(rows), self.flux_vector(fid, x0), np.array(w), np.array(cols, dtype=np.int64)

    def stencil(self, fid: int):
        """(cols, s_hat): s_hat = W (A^T W)^+ F_hat, the least-||W^-1 s|| solution of A^T s = F."""
        A, F, w, cols = self.face_system(fid)
        B = w[:, None] * A
        if np.linalg.matrix_rank(B) < self.K:
            raise RankDeficient(f"face {fid}: rank-deficient LS system ({len(w)} rows, K={self.K})")
        t = np.linalg.lstsq(B.T, F, rcond=None)[0]
        return cols, w * t

    # ----------------------------------------------------------- faces of the discretisation
    def flux_faces(self) -> list[int]:
        """All faces carrying a flux: open grid faces (interior and wall) and EB faces."""
        out = []
        for d in range(self.D):
            for f in np.nonzero(self.g.face_flag[d] > 0)[0]:
                out.append(self.face_id(d, int(f)))
        out.extend(self.eb_id(i) for i in range(len(self.g.cut_cells)))
        return out

    def all_stencils(self, faces=None) -> dict:
        faces = self.flux_faces() if faces is None else faces
        return {f: self.stencil(f) for f in faces}

    def face_area(self, fid: int) -> float:
        """|A_f| / h^(D-1)."""
        kind = self.decode_face(fid)
        if kind[0] == "eb":
            return float(self.g.eb_mom[kind[1], 0])
        return float(self.grid_face_tangential_moments(kind[1], kind[2])[0])

    # ----------------------------------------------------------- operator (Sec. 2.3)
    def cell_flux_faces(self, c: int):
        """(face id, sigma) for the flux faces of volume c (sigma = +1 when the face normal used in F
        points out of c)."""
        out = []
        for d, f, sg in self.cell_faces(c):
            if self.face_open(d, f):
                out.append((self.face_id(d, f), sg))
        if c in self.cut_pos:
            out.append((self.eb_id(self.cut_pos[c]), +1))
        return out

    def face_cells(self, fid: int):
        """[(cell, sigma)] of the volumes bounded by the face; sigma = +1 when the face normal used
        in F points out of that volume (grid faces: the low cell; EB faces: the cut cell)."""
        kind = self.decode_face(fid)
        if kind[0] == "eb":
            return [(int(self.g.cut_cells[kind[1]]), +1)]
        d, f = kind[1], kind[2]
        ijk = self.face_coords(d, f)
        out = []
        if ijk[d] > 0:
            lo = list(ijk)
            lo[d] -= 1
            c = self.cell_index(lo)
            if self.is_volume(c):
                out.append((c, +1))
        if ijk[d] < self.n[d]:
            c = self.cell_index(ijk)
            if self.is_volume(c):
                out.append((c, -1))
        return out

    def operator(self, stencils: dict | None = None, kappa_weighted: bool = False):
        """Sparse L (over all cells; covered rows empty) and B (cells x boundary faces, in the order
        of ``boundary_faces()``), so that L Phi + B G is the discrete Laplacian
        (1/|V_v|) sum_{f(v)} sigma s_f^T Phi of every volume (Sec. 2.3); with kappa_weighted,
        kappa_v times it."""
        g = self.g
        stencils = self.all_stencils() if stencils is None else stencils
        bfaces = self.boundary_faces()
        bpos = np.full(self.n_grid_faces + len(g.cut_cells), -1, dtype=np.int64)
        bpos[np.array(bfaces, dtype=np.int64)] = np.arange(len(bfaces))
        h2 = self.h ** 2
        Lr, Lc, Lv, Br, Bc, Bv = [], [], [], [], [], []
        for fid in self.flux_faces():
            for c, sg in self.face_cells(fid):
                scale = sg / h2 if kappa_weighted else sg / (g.kappa[c] * h2)
                if self._is_neumann(fid):
                    # the Neumann EB flux is the datum itself: |A_f| <g>_f
                    Br.append(np.array([c])); Bc.append(np.array([bpos[fid]]))
                    Bv.append(np.array([scale * self.face_area(fid) * self.h]))
                    continue
                cols, sv = stencils[fid]
                vm = cols >= 0
                Lr.append(np.full(int(vm.sum()), c)); Lc.append(cols[vm]); Lv.append(scale * sv[vm])
                bm = ~vm
                if bm.any():
                    bc = -cols[bm] - 1
                    # a Neumann row is a derivative in xi = (x - x0)/h: its datum enters as h <g>
                    hn = np.array([self.h if self._is_neumann(int(b)) else 1.0 for b in bc])
                    Br.append(np.full(int(bm.sum()), c)); Bc.append(bpos[bc]); Bv.append(scale * sv[bm] * hn)
        n = g.ncell
        cat = lambda a: np.concatenate(a) if a else np.zeros(0)
        L = sp.csr_matrix((cat(Lv), (cat(Lr).astype(np.int64), cat(Lc).astype(np.int64))), shape=(n, n))
        B = sp.csr_matrix((cat(Bv), (cat(Br).astype(np.int64), cat(Bc).astype(np.int64))), shape=(n, len(bfaces)))
        return L, B

    def _is_neumann(self, fid: int) -> bool:
        kind = self.decode_face(fid)
        return kind[0] == "eb" and self.bc_eb[kind[1]] == 1

    def boundary_faces(self) -> list[int]:
        """Boundary face ids: open wall faces (ascending id), then EB faces (ascending cut index)."""
        out = []
        for d in range(self.D):
            for side in (0, 1):
                pass
        walls = set()
        for d in range(self.D):
            ff = self.g.face_flag[d]
            for f in np.nonzero(ff > 0)[0]:
                ijk = self.face_coords(d, int(f))
                if ijk[d] == 0 or ijk[d] == self.n[d]:
                    walls.add(self.face_id(d, int(f)))
        out = sorted(walls) + [self.eb_id(i) for i in range(len(self.g.cut_cells))]
        return out

    # ----------------------------------------------------------- problem data
    def boundary_values(self, man) -> np.ndarray:
        """G in boundary_faces() order: Dirichlet <phi>_f (walls, Dirichlet EB faces) or the
        Neumann datum <grad phi . n>_f (Neumann EB faces)."""
        bf = self.boundary_faces()
        out = np.zeros(len(bf))
        eb_phi = man.eb_phi() if len(self.g.cut_cells) else np.zeros(0)
        eb_dn = man.eb_dphidn() if np.any(self.bc_eb == 1) else None
        walls_by_dir: dict[int, list] = {}
        for i, fid in enumerate(bf):
            kind = self.decode_face(fid)
            if kind[0] == "eb":
                out[i] = eb_dn[kind[1]] if self.bc_eb[kind[1]] == 1 else eb_phi[kind[1]]
            else:
                walls_by_dir.setdefault(kind[1], []).append((i, kind[2]))
        for d, lst in walls_by_dir.items():
            idx = np.array([i for i, _ in lst])
            fl = np.array([f for _, f in lst])
            out[idx] = man.face_avg(d, fl)
        return out


# --------------------------------------------------------------------- solves and norms

def solve_dense_lu(L, rhs, mask):
    """Direct sparse LU (SuperLU) of L restricted to the volumes in mask."""
    idx = np.nonzero(mask)[0]
    A = L[idx][:, idx].tocsc()
    x = np.zeros(L.shape[0])
    x[idx] = spla.spsolve(A, rhs[idx])
    return x


def error_norms(err: np.ndarray, weight: np.ndarray, mask: np.ndarray) -> dict:
    """Norms of Sec. 3.3 over the masked entries: L_inf = max |e|; L1 = sum |e| w / sum w;
    L2 = sqrt(sum e^2 w / sum w), with w = |V_v| for cells and w = alpha_f for faces.  The
    paper's L1 formula omits the normalisation for cells, but its printed values are the
    normalised ones (they match to three digits only when divided by the domain volume)."""
    e = np.abs(err[mask])
    w = weight[mask]
    sw = float(w.sum()) if len(w) else 1.0
    return {"linf": float(e.max()) if len(e) else 0.0, "l1": float((e * w).sum()) / sw,
            "l2": float(math.sqrt((e * e * w).sum() / sw))}


def run_problem(geom, man, params: Params | None = None, bc_eb=None, solve: bool = True,
                stencils: dict | None = None) -> dict:
    """Build every stencil, the operator and the data of a manufactured problem; solve
    L phi = rho - B G by direct LU; return errors in the norms of Sec. 3.3."""
    o = Oracle(geom, params, bc_eb)
    st = o.all_stencils() if stencils is None else stencils
    L, B = o.operator(st)
    G = o.boundary_values(man)
    vol = geom.flag > 0
    Phi = man.cell_avg()
    rho = man.lap_avg()
    BG = B @ G
    volw = geom.kappa * geom.h ** geom.dim
    trunc = geom.kappa * (L @ Phi + BG - rho)
    out = {"oracle": o, "stencils": st, "L": L, "B": B, "G": G, "Phi": Phi, "rho": rho,
           "trunc": error_norms(trunc, volw, vol)}
    if solve:
        Lk = sp.diags(geom.kappa) @ L
        phi = solve_dense_lu(Lk.tocsr(), geom.kappa * (rho - BG), vol)
        out["phi"] = phi
        out["sol"] = error_norms(phi - Phi, volw, vol)
    return out


# --------------------------------------------------------------------- adjoint of one stencil solve

def stencil_adjoint(A: np.ndarray, F: np.ndarray, w: np.ndarray, sbar: np.ndarray):
    """Reverse-mode derivative of the stencil s = W (A^T W)^+ F of Sec. 2.2.1 (full column rank):
    given sbar = dJ/ds, returns (Abar, Fbar) = (dJ/dA, dJ/dF) for J = J(s(A, F)).

    Written from s = W B (B^T B)^-1 F with B = W A (the minimum-||W^-1 s|| solution of A^T s = F):
    with y = (B^T B)^-1 F, t = B y (s = W t), tbar = W sbar and z = (B^T B)^-1 B^T tbar,
        Fbar = z,   Abar = W [tbar y^T - B (z y^T + y z^T)].
    The weights are held fixed (they depend on cell and face centres only)."""
    B = w[:, None] * A
    G = B.T @ B
    y = np.linalg.solve(G, F)
    tbar = w * sbar
    z = np.linalg.solve(G, B.T @ tbar)
    Bbar = np.outer(tbar, y) - B @ (np.outer(z, y) + np.outer(y, z))
    return w[:, None] * Bbar, z

"""Manufactured solutions: exact cell averages, boundary data and face fluxes.

For a product phi(x) = prod_d sin(w_d x_d + th_d) this computes, over the
geometry's cut-cell pieces, the quantities the paper's accuracy study uses
(Sec. 3.3): volume averages <phi>_v and <Laplacian phi>_v, face averages
<phi>_f on boundary faces (Dirichlet data), <grad phi . n>_f (Neumann data)
and the exact face fluxes int_f grad phi . n dA.  These are problem data, not
part of the discretisation.
"""
from __future__ import annotations

import math

import numpy as np

from .geometry import Geometry, ProductFn


def sin_product(kind: str) -> ProductFn:
    """Named manufactured solutions.

    ``paper2d``: sin(2 pi (x - sqrt2/2)) sin(2 pi (y - sqrt3/2)) -- the 2-D
    solution of Sec. 3.3 read with its second factor in y (as printed both
    factors are in x, which cannot be the intended 2-D test).
    ``sin2pix_cos3piy``: sin(2 pi x) cos(3 pi y).
    ``paper3d``: sin(2 pi (x-x0)) sin(2 pi (y-y0)) sin(2 pi (z-z0)),
    x0 = sqrt2/2, y0 = sqrt3/2, z0 = 0.54321 (Sec. 3.5).
    ``paper2d_printed``: sin(2 pi (x - sqrt2/2)) sin(2 pi (x - sqrt3/2)) as printed.
    """
    tp = 2 * math.pi
    if kind == "paper2d":
        return ProductFn((tp, tp, 0.0), (-tp * math.sqrt(2) / 2, -tp * math.sqrt(3) / 2, math.pi / 2))
    if kind == "sin2pix_cos3piy":
        return ProductFn((tp, 3 * math.pi, 0.0), (0.0, math.pi / 2, math.pi / 2))
    if kind == "paper3d":
        return ProductFn((tp, tp, tp), (-tp * math.sqrt(2) / 2, -tp * math.sqrt(3) / 2, -tp * 0.54321))
    raise ValueError(kind)


class Manufactured:
    """Exact data of phi = prod_d sin(w_d x_d + th_d) on a Geometry."""

    def __init__(self, geom: Geometry, fn: ProductFn):
        self.g = geom
        self.fn = fn
        D = geom.dim
        self.lap_factor = -sum(fn.w[d] ** 2 for d in range(D))
        self._basis = geom._basis_trig(fn)
        self._t_phi = np.zeros((1, 3), dtype=np.int32)
        self._t_grad = np.zeros((D, 3), dtype=np.int32)
        for d in range(D):
            self._t_grad[d, d] = 1
        self._cell = None

    # volume averages
    def cell_avg(self) -> np.ndarray:
        """<phi>_v for every cell (0 on covered cells)."""
        if self._cell is None:
            g = self.g
            cells = np.nonzero(g.flag > 0)[0].astype(np.int64)
            body = np.full(len(cells), -1, dtype=np.int32)
            cut_pos = np.searchsorted(cells, g.cut_cells)
            body[cut_pos] = g.cut_body
            vals = g.cell_integrals(cells, body, self._basis, self._t_phi)[:, 0]
            out = np.zeros(g.ncell)
            out[cells] = vals / g.kappa[cells]
            self._cell = out
        return self._cell

    def lap_avg(self) -> np.ndarray:
        """<Laplacian phi>_v = -(sum w_d^2) <phi>_v."""
        return self.lap_factor * self.cell_avg()

    # EB data
    def eb_phi(self) -> np.ndarray:
        g = self.g
        v = g.eb_integrals(g.cut_cells, g.cut_body, self._basis, self._t_phi)[:, 0]
        return v / g.eb_mom[:, 0]

    def eb_flux(self) -> np.ndarray:
        """int over the EB patch of grad phi . n dA (physical units; n out of the fluid)."""
        g = self.g
        tot = np.zeros(len(g.cut_cells))
        for d in range(g.dim):
            tot += g.eb_integrals(g.cut_cells, g.cut_body, self._basis, self._t_grad[d:d + 1], ncomp=d)[:, 0]
        return tot * g.h ** (g.dim - 1)

    def eb_dphidn(self) -> np.ndarray:
        return self.eb_flux() / (self.g.eb_mom[:, 0] * self.g.h ** (self.g.dim - 1))

    # grid faces
    def _face_body(self, d, faces):
        g = self.g
        body = np.full(len(faces), -1, dtype=np.int32)
        pos = np.searchsorted(g.cut_faces[d], faces)
        pos = np.clip(pos, 0, max(len(g.cut_faces[d]) - 1, 0))
        if len(g.cut_faces[d]):
            hit = g.cut_faces[d][pos] == faces
            body[hit] = g.cut_face_body[d][pos[hit]]
        return body

    def face_flux(self, d: int, faces=None) -> np.ndarray:
        """int_f d(phi)/dx_d dA over the fluid part of faces normal to d (physical units)."""
        g = self.g
        if faces is None:
            faces = np.arange(g.nface(d), dtype=np.int64)
        faces = np.asarray(faces, dtype=np.int64)
        v = g.face_integrals(d, faces, self._face_body(d, faces), self._basis, self._t_grad[d:d + 1])[:, 0]
        return v * g.h ** (g.dim - 1)

    def face_avg(self, d: int, faces) -> np.ndarray:
        g = self.g
        faces = np.asarray(faces, dtype=np.int64)
        v = g.face_integrals(d, faces, self._face_body(d, faces), self._basis, self._t_phi)[:, 0]
        al = g.alpha(d)[faces]
        out = np.zeros(len(faces))
        nz = al > 0
        out[nz] = v[nz] / al[nz]
        return out

    def wall_faces(self, d: int, side: int) -> np.ndarray:
        """Face indices of wall (d, side) in wall-array order (other dims ascending, first fastest)."""
        g = self.g
        shp = g.face_shape(d)
        idx = [np.arange(s) for s in shp]
        idx[d] = np.array([0 if side == 0 else g.n[d]])
        grids = np.meshgrid(*idx[::-1], indexing="ij")  # slowest first
        lin = np.zeros(grids[0].shape, dtype=np.int64)
        stride = 1
        for k in range(g.dim):
            lin += grids[g.dim - 1 - k] * stride
            stride *= shp[k]
        return lin.reshape(-1)

    def wall_ids(self) -> np.ndarray:
        """Global ids (faces normal to 0, then 1, then 2) of the open wall faces, ascending."""
        g = self.g
        out, base = [], 0
        for d in range(g.dim):
            for side in range(2):
                f = self.wall_faces(d, side)
                f = f[g.face_flag[d][f] > 0]
                out.append(base + f)
            base += g.nface(d)
        return np.sort(np.concatenate(out))

    def wall_phi_by_id(self) -> np.ndarray:
        """<phi>_f on the open wall faces in ascending global face id (the C ABI's g_wall order)."""
        g = self.g
        ids = self.wall_ids()
        out = np.zeros(len(ids))
        base = 0
        for d in range(g.dim):
            m = (ids >= base) & (ids < base + g.nface(d))
            out[m] = self.face_avg(d, ids[m] - base)
            base += g.nface(d)
        return out

    def wall_phi(self) -> np.ndarray:
        """<phi>_f on every wall face, walls ordered (d=0 low, d=0 high, d=1 low, ...), concatenated."""
        g = self.g
        out = []
        for d in range(g.dim):
            for side in range(2):
                out.append(self.face_avg(d, self.wall_faces(d, side)))
        return np.concatenate(out)

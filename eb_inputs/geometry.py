"""Analytic cut-cell geometries and their moment tables.

A ``Geometry`` is the unit box [0,1]^D on an N^D grid (h = 1/N) with circles
(2D) or spheres (3D) removed (``inside=False``), or the inside of one circle or
sphere (``inside=True``).  It produces, in the layout the C ABI documents:

* ``flag``      uint8[N^D]: 0 covered, 1 full, 2 cut (cell index x + nx*(y + ny*z));
* ``cut_cells`` int32 sorted cut-cell indices, with
  ``vol_mom``   [n_cut, K]      integral of xi^p over the fluid part / h^D,
  ``eb_mom``    [n_cut, K]      integral of xi^p over the EB patch / h^(D-1),
  ``eb_nmom``   [n_cut, D, K]   integral of xi^p n_d over the EB patch / h^(D-1),
  where xi = (x - cell centre)/h, n is the unit normal pointing out of the
  fluid and p runs over the graded monomials of degree <= qmax;
* per direction d: ``face_flag[d]`` uint8 over the faces normal to d
  (index x + (nx+[d==0]) * (y + (ny+[d==1]) * z)), and for cut faces
  ``cut_faces[d]`` and ``face_mom[d]`` [n_cf, K_F], moments of the face's
  tangential coordinates (ascending dimensions, graded order) about the face
  centre, / h^(D-1).

Monomial order (graded, then decreasing earlier exponents): degree 0, then
for each degree q the exponents (p0, p1, ...) with p0 from q down to 0, p1 from
q - p0 down to 0, and so on.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

from .rng import uniform

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "geom.c")
_LIB_PATH = os.path.join(_HERE, "_build", "libebgeom.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile geom.c into a shared library (gcc, OpenMP when available)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    try:
        subprocess.run(base[:4] + ["-fopenmp"] + base[4:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            for name in ("geo_classify_cells", "geo_classify_faces", "geo_cell_integrals", "geo_face_integrals",
                         "geo_eb_integrals"):
                getattr(_lib, name).restype = ctypes.c_int
            _lib.geo_gk15_panel_pow.restype = ctypes.c_double
            _lib.geo_gk15_panel_pow.argtypes = [ctypes.c_int, ctypes.c_int]
    return _lib


class _GeoT(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int * 3), ("h", ctypes.c_double), ("inside", ctypes.c_int),
                ("nbody", ctypes.c_int), ("center", ctypes.POINTER(ctypes.c_double)),
                ("radius", ctypes.POINTER(ctypes.c_double))]


class _BasisT(ctypes.Structure):
    _fields_ = [("nfn", ctypes.c_int * 3), ("kind", (ctypes.c_int * 16) * 3), ("pw", (ctypes.c_int * 16) * 3),
                ("pow_center", ctypes.c_double * 3), ("w", ctypes.c_double * 3), ("th", ctypes.c_double * 3),
                ("amp", ctypes.c_double * 3)]


def monomials(dim: int, q: int) -> list[tuple[int, ...]]:
    """Graded monomial exponents of total degree <= q in `dim` variables (documented order)."""
    out = []

    def rec(prefix, left, k):
        if k == dim - 1:
            out.append(tuple(prefix) + (left,))
            return
        for p in range(left, -1, -1):
            rec(prefix + [p], left - p, k + 1)

    for deg in range(q + 1):
        if dim == 0:
            out.append(())
            break
        rec([], deg, 0)
    return out


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


@dataclass
class ProductFn:
    """f(x) = prod_d g_d(x_d): g_d = amp_d sin(w_d x + th_d), or its derivative when deriv[d] is set."""
    w: tuple
    th: tuple
    amp: tuple = (1.0, 1.0, 1.0)


KAPPA_EPS = 1e-14


@dataclass
class Geometry:
    dim: int
    N: int
    centers: np.ndarray  # [nbody, 3]
    radii: np.ndarray    # [nbody]
    inside: bool = False
    qmax: int = 4
    name: str = ""
    seed: int | None = None
    _cache: dict = field(default_factory=dict, repr=False)

    def __post_init__(self):
        self.centers = np.ascontiguousarray(np.asarray(self.centers, dtype=np.float64).reshape(-1, 3))
        self.radii = np.ascontiguousarray(np.asarray(self.radii, dtype=np.float64).reshape(-1))
        self.n = tuple([self.N] * self.dim + [1] * (3 - self.dim))
        self.h = 1.0 / self.N
        self.ncell = self.N ** self.dim
        self._make_struct()
        self._build()

    def _make_struct(self):
        self._g = _GeoT(self.dim, (ctypes.c_int * 3)(*self.n), self.h, int(self.inside), len(self.radii),
                        self.centers.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                        self.radii.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))

    def __getstate__(self):
        st = dict(self.__dict__)
        st.pop("_g", None)
        return st

    def __setstate__(self, st):
        self.__dict__.update(st)
        self._make_struct()

    # ------------------------------------------------------------ helpers
    def nface(self, d: int) -> int:
        return int(np.prod([self.n[k] + (k == d) for k in range(self.dim)]))

    def face_shape(self, d: int):
        return tuple(self.n[k] + (k == d) for k in range(self.dim))

    def _basis_pow(self, q, center=None):
        b = _BasisT()
        for d in range(3):
            b.nfn[d] = q + 1
            for p in range(q + 1):
                b.kind[d][p] = 0
                b.pw[d][p] = p
            b.pow_center[d] = math.nan if center is None else float(center[d]) if d < len(center) else 0.0
            b.w[d] = 0.0
            b.th[d] = 0.0
            b.amp[d] = 1.0
        return b

    def _basis_trig(self, fn: ProductFn):
        b = _BasisT()
        for d in range(3):
            b.nfn[d] = 2
            b.kind[d][0] = 1
            b.kind[d][1] = 2
            b.pow_center[d] = math.nan
            b.w[d] = fn.w[d] if d < len(fn.w) else 0.0
            b.th[d] = fn.th[d] if d < len(fn.th) else math.pi / 2
            b.amp[d] = fn.amp[d] if d < len(fn.amp) else 1.0
        return b

    def _terms_mono(self, dim, q, skip=None):
        """term triples for graded monomials of degree <= q in the dims listed (others 0)."""
        dims = [d for d in range(self.dim) if d != skip]
        mons = monomials(len(dims), q)
        t = np.zeros((len(mons), 3), dtype=np.int32)
        for i, m in enumerate(mons):
            for j, d in enumerate(dims):
                t[i, d] = m[j]
        return t

    def cell_integrals(self, cells, body, basis, terms):
        lib = _load()
        cells = np.ascontiguousarray(cells, dtype=np.int64)
        body = np.ascontiguousarray(body, dtype=np.int32)
        terms = np.ascontiguousarray(terms, dtype=np.int32)
        out = np.zeros((len(cells), len(terms)))
        if len(cells):
            err = lib.geo_cell_integrals(ctypes.byref(self._g), ctypes.c_int64(len(cells)), _ptr(cells), _ptr(body),
                                         ctypes.byref(basis), ctypes.c_int(len(terms)), _ptr(terms), _ptr(out))
            if err:
                raise RuntimeError(f"geo_cell_integrals error {err}")
        return out

    def face_integrals(self, d, faces, body, basis, terms):
        lib = _load()
        faces = np.ascontiguousarray(faces, dtype=np.int64)
        body = np.ascontiguousarray(body, dtype=np.int32)
        terms = np.ascontiguousarray(terms, dtype=np.int32)
        out = np.zeros((len(faces), len(terms)))
        if len(faces):
            err = lib.geo_face_integrals(ctypes.byref(self._g), ctypes.c_int(d), ctypes.c_int64(len(faces)),
                                         _ptr(faces), _ptr(body), ctypes.byref(basis), ctypes.c_int(len(terms)),
                                         _ptr(terms), _ptr(out))
            if err:
                raise RuntimeError(f"geo_face_integrals error {err}")
        return out

    def eb_integrals(self, cells, body, basis, terms, ncomp=-1):
        lib = _load()
        cells = np.ascontiguousarray(cells, dtype=np.int64)
        body = np.ascontiguousarray(body, dtype=np.int32)
        terms = np.ascontiguousarray(terms, dtype=np.int32)
        out = np.zeros((len(cells), 4 * len(terms) if ncomp == -2 else len(terms)))
        if len(cells):
            err = lib.geo_eb_integrals(ctypes.byref(self._g), ctypes.c_int64(len(cells)), _ptr(cells), _ptr(body),
                                       ctypes.byref(basis), ctypes.c_int(ncomp), ctypes.c_int(len(terms)),
                                       _ptr(terms), _ptr(out))
            if err:
                raise RuntimeError(f"geo_eb_integrals error {err}")
        return out

    # ------------------------------------------------------------ build
    def _build(self):
        lib = _load()
        D, q = self.dim, self.qmax
        flag = np.zeros(self.ncell, dtype=np.int8)
        body = np.zeros(self.ncell, dtype=np.int32)
        err = lib.geo_classify_cells(ctypes.byref(self._g), _ptr(flag), _ptr(body))
        if err:
            raise RuntimeError(f"cell classification failed ({err}): a cell is cut by more than one body")
        cut = np.nonzero(flag == 2)[0].astype(np.int64)
        cbody = body[cut]
        del body
        bp = self._basis_pow(q)
        tV = self._terms_mono(D, q)
        vol = self.cell_integrals(cut, cbody, bp, tV)
        allc = self.eb_integrals(cut, cbody, bp, tV, ncomp=-2).reshape(len(cut), 4, len(tV))
        eb = allc[:, 0, :]
        ebn = allc[:, 1:1 + D, :]
        kap = vol[:, 0] if len(cut) else np.zeros(0)
        to_full = kap >= 1.0 - KAPPA_EPS
        to_cov = kap <= KAPPA_EPS
        flag[cut[to_full]] = 1
        flag[cut[to_cov]] = 0
        keep = ~(to_full | to_cov)
        self.cut_cells = cut[keep].astype(np.int32)
        self.cut_body = cbody[keep]
        self.vol_mom = np.ascontiguousarray(vol[keep])
        self.eb_mom = np.ascontiguousarray(eb[keep])
        self.eb_nmom = np.ascontiguousarray(ebn[keep])
        self.flag = flag.astype(np.uint8)
        self.kappa = (self.flag == 1).astype(np.float64)
        self.kappa[self.cut_cells] = self.vol_mom[:, 0]
        # faces
        self.face_flag, self.cut_faces, self.face_mom, self.cut_face_body = [], [], [], []
        self.closed_slivers = 0
        for d in range(D):
            nf = self.nface(d)
            ff = np.zeros(nf, dtype=np.int8)
            fb = np.zeros(nf, dtype=np.int32)
            err = lib.geo_classify_faces(ctypes.byref(self._g), ctypes.c_int(d), _ptr(ff), _ptr(fb))
            if err:
                raise RuntimeError(f"face classification failed ({err})")
            cf = np.nonzero(ff == 2)[0].astype(np.int64)
            cfb = fb[cf]
            del fb
            tF = self._terms_mono(D, q, skip=d)
            fm = self.face_integrals(d, cf, cfb, bp, tF)
            al = fm[:, 0] if len(cf) else np.zeros(0)
            tfull = al >= 1.0 - KAPPA_EPS
            tcov = al <= KAPPA_EPS
            ff[cf[tfull]] = 1
            ff[cf[tcov]] = 0
            k = ~(tfull | tcov)
            # a cell whose volume fraction fell below KAPPA_EPS counts as covered: its faces close too
            # (their area fraction is at most ~sqrt(KAPPA_EPS))
            ff = ff.astype(np.uint8)
            fl = self.flag.reshape(self.n[:D][::-1])
            ffs = ff.reshape(self.face_shape(d)[::-1])
            ax = D - 1 - d
            cov = fl == 0
            lo_c = np.concatenate([np.zeros_like(np.take(cov, [0], axis=ax)), cov], axis=ax)
            hi_c = np.concatenate([cov, np.zeros_like(np.take(cov, [0], axis=ax))], axis=ax)
            shut = (ffs > 0) & (lo_c | hi_c)
            if shut.any():
                self.closed_slivers += int(shut.sum())
                ffs[shut] = 0
                ff = ffs.reshape(-1)
                k &= ff[cf] == 2
            self.face_flag.append(ff)
            self.cut_faces.append(cf[k].astype(np.int32))
            self.cut_face_body.append(cfb[k])
            self.face_mom.append(np.ascontiguousarray(fm[k][:, :len(monomials(D - 1, q))]))
        self._check_consistency()

    def alpha(self, d: int) -> np.ndarray:
        a = (self.face_flag[d] == 1).astype(np.float64)
        a[self.cut_faces[d]] = self.face_mom[d][:, 0]
        return a

    def _check_consistency(self):
        D = self.dim
        fl = self.flag.reshape(self.n[:D][::-1])  # z, y, x
        for d in range(D):
            ax = D - 1 - d
            ff = self.face_flag[d].reshape(self.face_shape(d)[::-1])
            lo = np.take(ff, np.arange(0, self.n[d]), axis=ax)      # face on the low side of each cell
            hi = np.take(ff, np.arange(1, self.n[d] + 1), axis=ax)  # face on the high side
            cov = fl == 0
            if np.any((lo > 0) & cov) or np.any((hi > 0) & cov):
                raise RuntimeError("inconsistent geometry: an open face borders a covered cell")

    # ------------------------------------------------------------ summaries
    def min_kappa(self) -> float:
        return float(self.vol_mom[:, 0].min()) if len(self.cut_cells) else 1.0

    def describe(self) -> dict:
        return {"name": self.name, "dim": self.dim, "N": self.N, "inside": self.inside,
                "centers": self.centers[:, :self.dim].tolist(), "radii": self.radii.tolist(),
                "seed": self.seed, "n_cut": int(len(self.cut_cells)),
                "n_covered": int((self.flag == 0).sum()), "kappa_min": self.min_kappa()}


# ---------------------------------------------------------------- seeded geometries

def line_config(N: int, qmax: int = 4) -> Geometry:
    """1-D unit interval with N cells and no embedded boundary."""
    return Geometry(1, N, np.zeros((0, 3)), np.zeros(0), False, qmax, name=f"line-{N}")


def circle_config(N: int, center=(0.5, 0.5), r: float = 0.25, inside: bool = False, qmax: int = 4) -> Geometry:
    """Unit square minus (or inside) one circle."""
    c = np.array([[center[0], center[1], 0.0]])
    return Geometry(2, N, c, np.array([r]), inside, qmax, name=f"circle-{N}")


def four_circles_config(N: int, qmax: int = 4) -> Geometry:
    """Unit square minus four circles of radius 0.215 centred at (0.25|0.75, 0.25|0.75)."""
    c = np.array([[0.25, 0.25, 0], [0.75, 0.25, 0], [0.25, 0.75, 0], [0.75, 0.75, 0]], dtype=float)
    return Geometry(2, N, c, np.full(4, 0.215), False, qmax, name=f"four-circles-{N}")


def multi_circle_config(N: int, seed: int = 1, qmax: int = 4) -> Geometry:
    """Circle r=0.3 at (0.51, 0.49) plus four seeded circles, radii U[0.05, 0.15].

    Each extra circle draws (r, cx, cy) from SplitMix64(seed) and is accepted
    when its boundary keeps a clearance >= 0.04 from every accepted circle and
    from the box.
    """
    centers = [(0.51, 0.49)]
    radii = [0.3]
    stream = uniform(seed, 3 * 20000)
    k = 0
    while len(radii) < 5:
        r = 0.05 + 0.10 * stream[k]
        cx, cy = stream[k + 1], stream[k + 2]
        k += 3
        if cx - r < 0.04 or cy - r < 0.04 or cx + r > 0.96 or cy + r > 0.96:
            continue
        ok = all(math.hypot(cx - x, cy - y) - r - rr >= 0.04 for (x, y), rr in zip(centers, radii))
        if ok:
            centers.append((cx, cy))
            radii.append(r)
    c = np.array([[x, y, 0.0] for x, y in centers])
    return Geometry(2, N, c, np.array(radii), False, qmax, name=f"multi-circle-{N}", seed=seed)


def multi_sphere_config(N: int, n: int = 8, seed: int = 4, rmin: float = 0.08, rmax: float = 0.2,
                        qmax: int = 4) -> Geometry:
    """The unit cube minus n seeded non-overlapping spheres: each draws (r, cx, cy, cz) from
    SplitMix64(seed), r ~ U[rmin, rmax), and is accepted when its surface keeps a clearance of at
    least 2h from every accepted sphere and from the box (no cell is cut by two spheres)."""
    h = 1.0 / N
    gap = 2.0 * h
    centers, radii = [], []
    stream = uniform(seed, 4 * 200000)
    k = 0
    while len(radii) < n:
        if k + 4 > len(stream):
            raise RuntimeError("could not place the spheres with the requested clearance")
        r = rmin + (rmax - rmin) * stream[k]
        c = stream[k + 1:k + 4]
        k += 4
        if np.any(c - r < gap) or np.any(c + r > 1.0 - gap):
            continue
        if all(np.linalg.norm(c - cc) - r - rr >= gap for cc, rr in zip(centers, radii)):
            centers.append(np.array(c))
            radii.append(r)
    return Geometry(3, N, np.array(centers), np.array(radii), False, qmax, name=f"multi-sphere-{N}", seed=seed)


def level_set_modes(n: int = 16, seed: int = 5, dim: int = 3) -> np.ndarray:
    """Rows (k_x, k_y, k_z, theta) of n seeded level-set modes sin(2 pi k . x + theta) of the shape-
    gradient workload: k_i ~ U{1, ..., 4} in the first `dim` components (0 beyond), theta ~ U[0, 2 pi),
    drawn from SplitMix64(seed) four numbers per mode."""
    u = uniform(seed, 4 * n)
    out = np.zeros((n, 4))
    for m in range(n):
        for d in range(dim):
            out[m, d] = 1.0 + min(3.0, math.floor(4.0 * u[4 * m + d]))
        out[m, 3] = 2.0 * math.pi * u[4 * m + 3]
    return out


def sphere_box_config(N: int, seed: int = 2, r: float = 0.35, qmax: int = 4) -> Geometry:
    """Unit cube minus a sphere of radius r centred at 0.5 + delta, delta_i ~ U[-h/2, h/2) from seed."""
    h = 1.0 / N
    dlt = uniform(seed, 3, -0.5 * h, 0.5 * h)
    c = np.array([[0.5 + dlt[0], 0.5 + dlt[1], 0.5 + dlt[2]]])
    return Geometry(3, N, c, np.array([r]), False, qmax, name=f"sphere-box-{N}", seed=seed)


def sphere_inside_config(N: int, center=(0.5, 0.5, 0.5), r: float = 0.45, qmax: int = 4) -> Geometry:
    """Inside of one sphere (the unit cube's walls are never reached)."""
    c = np.array([list(center)])
    return Geometry(3, N, c, np.array([r]), True, qmax, name=f"sphere-inside-{N}")

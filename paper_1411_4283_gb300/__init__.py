"""GB300 library for the higher-order cut-cell finite-volume Poisson method
(Devendran, Graves, Johansen, arXiv:1411.4283).

Thin Python binding of the C ABI in ``include/eb.h``: argument marshalling
only.  Every step of the method -- neighbourhoods, weighted least squares,
operator assembly, apply, Krylov solve, error norms -- runs in the CUDA
kernels of ``libeb_gb300.so``.  PyTorch provides device memory and streams.

The library must be built (``paper_1411_4283_gb300.build.build()``); importing
this package without it raises ImportError -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_LIB = None

EB_OK = 0
EB_F32, EB_F64 = 0, 1
EB_DIRICHLET, EB_NEUMANN = 0, 1
EB_NBR_BOX, EB_NBR_PATH = 0, 1
STATUS = {0: "EB_OK", 1: "EB_ERR_INVALID", 2: "EB_ERR_RANK_DEFICIENT", 3: "EB_ERR_MULTIVALUED",
          4: "EB_ERR_NOT_CONVERGED", 5: "EB_ERR_TIMEOUT", 6: "EB_ERR_CUDA", 7: "EB_ERR_OOM", 8: "EB_ERR_CAPACITY"}

_vp = ctypes.c_void_p


class EbGeom(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("n", ctypes.c_int32 * 3), ("h", ctypes.c_double),
                ("moment_degree", ctypes.c_int32), ("cell_flag", _vp), ("n_cut", ctypes.c_int32),
                ("cut_cell", _vp), ("vol_mom", _vp), ("eb_mom", _vp), ("eb_nmom", _vp), ("eb_bc", _vp),
                ("face_flag", _vp * 3), ("n_cutface", ctypes.c_int32 * 3), ("cutface", _vp * 3),
                ("face_mom", _vp * 3)]


class EbParams(ctypes.Structure):
    _fields_ = [("order", ctypes.c_int32), ("path_radius", ctypes.c_int32), ("nbr_metric", ctypes.c_int32),
                ("weighted", ctypes.c_int32), ("w_threshold", ctypes.c_double), ("w_power", ctypes.c_double),
                ("ls_precision", ctypes.c_int32)]


class EbBuildInfo(ctypes.Structure):
    _fields_ = [("n_flux_faces", ctypes.c_int64), ("n_unique_faces", ctypes.c_int64),
                ("n_class_faces", ctypes.c_int64), ("n_classes", ctypes.c_int32), ("max_rows", ctypes.c_int32),
                ("n_irregular_rows", ctypes.c_int64), ("n_row_classes", ctypes.c_int32),
                ("lsq_flops", ctypes.c_int64), ("ms_classify", ctypes.c_double), ("ms_gather", ctypes.c_double),
                ("ms_lsq", ctypes.c_double), ("ms_assemble", ctypes.c_double), ("n_ls_fp64", ctypes.c_int64),
                ("ls_fp64_flops", ctypes.c_double), ("ls_fp32_flops", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class EbSolveOpts(ctypes.Structure):
    _fields_ = [("mixed", ctypes.c_int32), ("inner_tol", ctypes.c_double), ("max_inner", ctypes.c_int32),
                ("max_outer", ctypes.c_int32), ("max_iters", ctypes.c_int32), ("check_every", ctypes.c_int32),
                ("precond", ctypes.c_int32)]


class EbSolveInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("sweeps", ctypes.c_int32), ("rel_residual", ctypes.c_double),
                ("history", ctypes.c_double * 64), ("n_history", ctypes.c_int32), ("n_applies", ctypes.c_int32),
                ("apply_ms", ctypes.c_double), ("precond_blocks", ctypes.c_int32)]

    def as_dict(self):
        return {"iterations": self.iterations, "sweeps": self.sweeps, "rel_residual": self.rel_residual,
                "history": [self.history[i] for i in range(self.n_history)], "n_applies": self.n_applies,
                "apply_ms": self.apply_ms, "precond_blocks": self.precond_blocks}


class EbAdjointInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("rel_residual", ctypes.c_double), ("solve_ms", ctypes.c_double),
                ("tables_ms", ctypes.c_double), ("stencils_ms", ctypes.c_double)]


class EbError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


def lib_path() -> str:
    return _build.LIB


def load():
    """Load libeb_gb300.so (raises ImportError when it has not been built)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = os.environ.get("EB_LIB_PATH") or _build.LIB  # EB_LIB_PATH: a tuning variant of the library
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with paper_1411_4283_gb300.build.build() "
                          "(there is no CPU fallback)")
    lib = ctypes.CDLL(path)
    i32, i64, dbl = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    P = ctypes.POINTER
    sig = {
        "eb_build_stencils": (i32, [P(EbGeom), P(EbParams), P(_vp), P(EbBuildInfo), _vp]),
        "eb_build_stencils_batch": (i32, [P(EbGeom), i32, P(EbParams), P(_vp), P(EbBuildInfo), _vp]),
        "eb_apply": (i32, [_vp, _vp, _vp, i32, i32, _vp]),
        "eb_bc_rhs": (i32, [_vp, _vp, _vp, _vp, i32, _vp]),
        "eb_solve": (i32, [_vp, _vp, _vp, _vp, dbl, P(EbSolveOpts), _vp, P(EbSolveInfo), _vp]),
        "eb_norms": (i32, [_vp, _vp, P(dbl), _vp]),
        "eb_stencil_query": (i32, [_vp, i64, P(i32), P(i64), P(dbl), i32, _vp]),
        "eb_wall_faces": (i32, [_vp, P(i64), i64, P(i64)]),
        "eb_last_error_faces": (i32, [P(i64), i32, P(i32)]),
        "eb_stencils_destroy": (None, [_vp]),
        "eb_status_string": (ctypes.c_char_p, [i32]),
        "eb_last_error_message": (ctypes.c_char_p, []),
        "eb_abi_version": (i32, []),
        "eb_kernel_launches": (i64, []),
        "eb_lsq_batch_noalloc": (i32, [_vp, _vp, _vp, _vp, i32, i32, i32, _vp, _vp, _vp]),
        "eb_geometry_circles": (i32, [i32, i32, P(dbl), P(dbl), i32, i32, P(_vp), P(EbGeom), _vp]),
        "eb_geometry_destroy": (None, [_vp]),
        "eb_geometry_spheres": (i32, [i32, i32, P(dbl), P(dbl), i32, i32, P(_vp), P(EbGeom), _vp]),
        "eb_geometry_table": (i32, [_vp, i32, i32, _vp, i64, P(i64)]),
        "eb_geometry_shape_table": (i32, [_vp, i32, i32, P(dbl), i32, i32, P(dbl), i64, P(i64)]),
        "eb_adjoint_radii": (i32, [_vp, _vp, _vp, P(dbl), P(dbl), _vp]),
        "eb_batch_solver_create": (i32, [P(_vp), i32, P(EbSolveOpts), P(_vp), _vp]),
        "eb_batch_solve": (i32, [_vp, P(_vp), P(_vp), P(_vp), dbl, P(_vp), P(EbSolveInfo), _vp]),
        "eb_batch_solver_destroy": (None, [_vp]),
        "eb_fp64_fma_rate": (i32, [i32, i64, P(dbl), _vp]),
        "eb_adjoint_shape": (i32, [_vp, _vp, _vp, i32, P(dbl), P(dbl), P(dbl), P(dbl), P(EbAdjointInfo), _vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _LIB = lib
    return lib


def _check(code):
    if code != EB_OK:
        raise EbError(code, load().eb_last_error_message().decode())


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dev(a, dtype):
    import torch
    if isinstance(a, torch.Tensor):
        return a.to(device="cuda", dtype=dtype).contiguous()
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype).contiguous()


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None and t.numel() > 0 else ctypes.c_void_p(0)


def _vec64(t, n, what):
    """Pointer to a device FP64 vector of at least n entries.  The C ABI takes raw pointers and reads or
    writes n entries, so the type, the device, the layout and the length are checked here; n = 0 also
    accepts None (the library then takes a null pointer)."""
    import torch
    if t is None and n == 0:
        return ctypes.c_void_p(0)
    if not (isinstance(t, torch.Tensor) and t.dtype == torch.float64 and t.is_cuda and t.is_contiguous()
            and t.numel() >= n):
        raise ValueError(f"{what}: a contiguous FP64 CUDA tensor of at least {n} entries is expected")
    return _ptr(t)


class DeviceGeometry:
    """Device copies of a geometry's moment tables, in the layout eb.h documents."""

    def __init__(self, dim, n, h, moment_degree, cell_flag, cut_cell, vol_mom, eb_mom, eb_nmom, face_flag, cut_faces,
                 face_mom, eb_bc=None):
        import torch
        self.dim = int(dim)
        self.n = tuple(int(v) for v in n) + (1,) * (3 - len(n))
        self.h = float(h)
        self.moment_degree = int(moment_degree)
        self.cell_flag = _dev(cell_flag, torch.uint8)
        self.cut_cell = _dev(cut_cell, torch.int32)
        self.vol_mom = _dev(vol_mom, torch.float64)
        self.eb_mom = _dev(eb_mom, torch.float64)
        self.eb_nmom = _dev(eb_nmom, torch.float64)
        self.eb_bc = _dev(eb_bc, torch.uint8) if eb_bc is not None else None
        self.face_flag = [_dev(f, torch.uint8) for f in face_flag]
        self.cut_faces = [_dev(f, torch.int32) for f in cut_faces]
        self.face_mom = [_dev(f, torch.float64) for f in face_mom]
        self.n_cut = int(self.cut_cell.numel())

    @classmethod
    def from_geometry(cls, g, eb_bc=None):
        """From an object with the eb_inputs.Geometry attributes (flag, cut_cells, vol_mom, ...)."""
        return cls(g.dim, g.n[:g.dim], g.h, g.qmax, g.flag, g.cut_cells, g.vol_mom, g.eb_mom, g.eb_nmom, g.face_flag,
                   g.cut_faces, g.face_mom, eb_bc)

    def struct(self) -> EbGeom:
        s = EbGeom()
        s.dim = self.dim
        for d in range(3):
            s.n[d] = self.n[d]
        s.h = self.h
        s.moment_degree = self.moment_degree
        s.cell_flag = _ptr(self.cell_flag)
        s.n_cut = self.n_cut
        s.cut_cell = _ptr(self.cut_cell)
        s.vol_mom = _ptr(self.vol_mom)
        s.eb_mom = _ptr(self.eb_mom)
        s.eb_nmom = _ptr(self.eb_nmom)
        s.eb_bc = _ptr(self.eb_bc)
        for d in range(self.dim):
            s.face_flag[d] = _ptr(self.face_flag[d])
            s.n_cutface[d] = int(self.cut_faces[d].numel())
            s.cutface[d] = _ptr(self.cut_faces[d])
            s.face_mom[d] = _ptr(self.face_mom[d])
        return s


class GpuGeometry:
    """Moment tables computed on the device by the library (eb_geometry_circles); owns the handle.
    Usable wherever a DeviceGeometry is (eb_build_stencils takes either)."""

    TABLES = {"flag": 0, "cut_cells": 1, "vol_mom": 2, "eb_mom": 3, "eb_nmom": 4, "face_flag": 5, "cut_faces": 6,
              "face_mom": 7}

    def __init__(self, handle, desc: EbGeom, eb_bc=None):
        self.handle = handle
        self.desc = desc
        self.dim = desc.dim
        self.n = tuple(desc.n[d] for d in range(3))
        self.h = desc.h
        self.moment_degree = desc.moment_degree
        self.n_cut = desc.n_cut
        self.eb_bc = None
        if eb_bc is not None:
            self.set_eb_bc(eb_bc)

    def set_eb_bc(self, eb_bc):
        import torch
        self.eb_bc = _dev(eb_bc, torch.uint8)
        self.desc.eb_bc = _ptr(self.eb_bc)

    def struct(self) -> EbGeom:
        return self.desc

    def table(self, name: str, d: int = 0) -> np.ndarray:
        """A table copied to the host, shaped like the eb_inputs.Geometry attribute of that name."""
        lib = load()
        w = self.TABLES[name]
        nb = ctypes.c_int64()
        _check(lib.eb_geometry_table(self.handle, w, d, None, 0, ctypes.byref(nb)))
        dt = {0: np.uint8, 1: np.int32, 5: np.uint8, 6: np.int32}.get(w, np.float64)
        out = np.zeros(max(nb.value // np.dtype(dt).itemsize, 1), dtype=dt)
        _check(lib.eb_geometry_table(self.handle, w, d, out.ctypes.data_as(ctypes.c_void_p), out.nbytes,
                                     ctypes.byref(nb)))
        out = out[:nb.value // np.dtype(dt).itemsize]
        if name in ("vol_mom", "eb_mom"):
            out = out.reshape(self.n_cut, -1)
        elif name == "eb_nmom":
            out = out.reshape(self.n_cut, self.dim, -1)
        elif name == "face_mom":
            out = out.reshape(self.desc.n_cutface[d], -1)
        return out

    def shape_table(self, name: str, body: int = 0, mode=None, d: int = 0) -> np.ndarray:
        """The derivative of table `name` (vol_mom, eb_mom, eb_nmom, face_mom) for the radius of `body`
        (mode None) or for the amplitude of the level-set mode (k_x, k_y, k_z, theta) at zero amplitude,
        shaped like table(name, d)."""
        lib = load()
        w = self.TABLES[name]
        kind = 0 if mode is None else 1
        m = np.ascontiguousarray(np.zeros(4) if mode is None else np.asarray(mode, dtype=np.float64).reshape(4))
        mp = m.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        nb = ctypes.c_int64()
        _check(lib.eb_geometry_shape_table(self.handle, kind, int(body), mp, w, d, None, 0, ctypes.byref(nb)))
        out = np.zeros(max(nb.value // 8, 1))
        _check(lib.eb_geometry_shape_table(self.handle, kind, int(body), mp, w, d,
                                           out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), out.nbytes,
                                           ctypes.byref(nb)))
        out = out[:nb.value // 8]
        if name in ("vol_mom", "eb_mom"):
            return out.reshape(self.n_cut, -1)
        if name == "eb_nmom":
            return out.reshape(self.n_cut, self.dim, -1)
        return out.reshape(self.desc.n_cutface[d], -1)

    def __del__(self):
        if getattr(self, "handle", None) and _LIB is not None:
            _LIB.eb_geometry_destroy(self.handle)
            self.handle = None


def eb_geometry_spheres(N, centers, radii, inside=False, moment_degree=4, stream=None) -> GpuGeometry:
    """Moment tables of the unit cube minus spheres (or inside one sphere), computed on the device."""
    lib = load()
    c = np.ascontiguousarray(np.asarray(centers, dtype=np.float64).reshape(-1, 3))
    r = np.ascontiguousarray(np.asarray(radii, dtype=np.float64).reshape(-1))
    h = ctypes.c_void_p()
    desc = EbGeom()
    _check(lib.eb_geometry_spheres(int(N), len(r), c.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                   r.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(bool(inside)),
                                   int(moment_degree), ctypes.byref(h), ctypes.byref(desc), _stream(stream)))
    out = GpuGeometry(h, desc)
    out.centers, out.radii = c, r
    return out


def eb_geometry_circles(N, centers, radii, inside=False, moment_degree=4, stream=None) -> GpuGeometry:
    """Moment tables of the unit square minus circles (or inside one circle), computed on the device."""
    lib = load()
    c = np.ascontiguousarray(np.asarray(centers, dtype=np.float64).reshape(-1, 2))
    r = np.ascontiguousarray(np.asarray(radii, dtype=np.float64).reshape(-1))
    h = ctypes.c_void_p()
    desc = EbGeom()
    _check(lib.eb_geometry_circles(int(N), len(r), c.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                   r.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(bool(inside)),
                                   int(moment_degree), ctypes.byref(h), ctypes.byref(desc), _stream(stream)))
    out = GpuGeometry(h, desc)
    out.centers, out.radii = c, r
    return out


def eb_adjoint_radii(geom: "GpuGeometry", st: "Stencils", phi, gradient=True, stream=None):
    """(J, dJ/dr) for J = 1/2 sum |V| phi^2 and the radii of the circles of a device geometry (see eb.h)."""
    import torch
    assert phi.dtype == torch.float64 and phi.is_cuda and phi.is_contiguous() and phi.numel() == st.ncell
    J = ctypes.c_double()
    nb = len(geom.radii)
    dJ = (ctypes.c_double * max(nb, 1))()
    _check(load().eb_adjoint_radii(geom.handle, st.handle, _ptr(phi), ctypes.byref(J), dJ if gradient else None,
                                   _stream(stream)))
    return J.value, (np.array([dJ[i] for i in range(nb)]) if gradient else None)


def eb_adjoint_shape(geom: "GpuGeometry", st: "Stencils", phi, modes=(), gradient=True, stream=None, info=None):
    """(J, dJ/dr, dJ/da) for J = 1/2 sum |V| phi^2, the radii of a device geometry's bodies and the
    amplitudes a_m of level-set modes sin(2 pi k_m . x + theta_m) at a = 0 (see eb.h).  modes: rows
    (k_x, k_y, k_z, theta) (k_z ignored in 2-D).  info: a dict that receives the transposed solve's
    iterations and the phases' device times."""
    import torch
    assert phi.dtype == torch.float64 and phi.is_cuda and phi.is_contiguous() and phi.numel() == st.ncell
    m = np.ascontiguousarray(np.asarray(modes, dtype=np.float64).reshape(-1, 4))
    nb, nm = len(geom.radii), len(m)
    J = ctypes.c_double()
    dr = (ctypes.c_double * max(nb, 1))()
    da = (ctypes.c_double * max(nm, 1))()
    mp = m.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if nm else None
    ai = EbAdjointInfo()
    _check(load().eb_adjoint_shape(geom.handle, st.handle, _ptr(phi), nm, mp, ctypes.byref(J),
                                   dr if gradient else None, da if gradient else None, ctypes.byref(ai),
                                   _stream(stream)))
    if info is not None:
        info.update({k: getattr(ai, k) for k, _ in EbAdjointInfo._fields_})
    if not gradient:
        return J.value, None, None
    return J.value, np.array([dr[i] for i in range(nb)]), np.array([da[i] for i in range(nm)])


class Stencils:
    """Owns an eb_stencils handle (freed by eb_stencils_destroy)."""

    def __init__(self, handle, info: EbBuildInfo, geom: DeviceGeometry):
        self.handle = handle
        self.info = info.as_dict()
        self.dim = geom.dim
        self.n = geom.n
        self.h = geom.h
        self.ncell = int(np.prod(geom.n))
        self.n_cut = geom.n_cut
        n = ctypes.c_int64()
        _check(load().eb_wall_faces(handle, None, 0, ctypes.byref(n)))
        self.n_wall = int(n.value)  # open wall faces (the length of g_wall)

    def __del__(self):
        if getattr(self, "handle", None) and _LIB is not None:
            _LIB.eb_stencils_destroy(self.handle)
            self.handle = None


LS_PRECISION = {"mixed": 0, "fp64": 1}


def eb_build_stencils(geom: DeviceGeometry, order=4, path_radius=0, nbr_metric=EB_NBR_BOX, weighted=True,
                      w_threshold=0.5, w_power=5.0, stream=None, ls_precision="mixed") -> Stencils:
    lib = load()
    g = geom.struct()
    p = EbParams(order, path_radius, nbr_metric, int(weighted), w_threshold, w_power, LS_PRECISION[ls_precision])
    h = ctypes.c_void_p()
    info = EbBuildInfo()
    _check(lib.eb_build_stencils(ctypes.byref(g), ctypes.byref(p), ctypes.byref(h), ctypes.byref(info),
                                 _stream(stream)))
    return Stencils(h, info, geom)


def eb_build_stencils_batch(geoms, order=4, path_radius=0, nbr_metric=EB_NBR_BOX, weighted=True,
                            w_threshold=0.5, w_power=5.0, stream=None, ls_precision="mixed") -> list:
    """Stencils of several geometries (same dimension) with one least-squares launch."""
    lib = load()
    n = len(geoms)
    gs = (EbGeom * n)(*[geom.struct() for geom in geoms])
    p = EbParams(order, path_radius, nbr_metric, int(weighted), w_threshold, w_power, LS_PRECISION[ls_precision])
    hs = (ctypes.c_void_p * n)()
    infos = (EbBuildInfo * n)()
    _check(lib.eb_build_stencils_batch(gs, n, ctypes.byref(p), hs, infos, _stream(stream)))
    return [Stencils(ctypes.c_void_p(hs[i]), infos[i], geoms[i]) for i in range(n)]


def eb_apply(st: Stencils, phi, y, kappa_weighted=True, stream=None):
    import torch
    dt = {torch.float32: EB_F32, torch.float64: EB_F64}[phi.dtype]
    assert y.dtype == phi.dtype and phi.is_cuda and y.is_cuda and phi.is_contiguous() and y.is_contiguous()
    assert phi.numel() == st.ncell and y.numel() == st.ncell
    _check(load().eb_apply(st.handle, _ptr(phi), _ptr(y), dt, int(kappa_weighted), _stream(stream)))
    return y


def eb_wall_faces(st: Stencils) -> np.ndarray:
    lib = load()
    n = ctypes.c_int64()
    _check(lib.eb_wall_faces(st.handle, None, 0, ctypes.byref(n)))
    out = np.zeros(max(n.value, 1), dtype=np.int64)
    _check(lib.eb_wall_faces(st.handle, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), n.value,
                             ctypes.byref(n)))
    return out[:n.value]


def eb_bc_rhs(st: Stencils, g_eb, g_wall, Bg, kappa_weighted=True, stream=None):
    _check(load().eb_bc_rhs(st.handle, _vec64(g_eb, st.n_cut, "g_eb"), _vec64(g_wall, st.n_wall, "g_wall"),
                            _vec64(Bg, st.ncell, "Bg"), int(kappa_weighted), _stream(stream)))
    return Bg


def eb_solve(st: Stencils, rho, g_eb, g_wall, phi, tol=1e-12, mixed=True, inner_tol=1e-5, max_inner=20000,
             max_outer=40, max_iters=400000, stream=None, allow_not_converged=False, time_applies=False,
             precond="mg") -> dict:
    lib = load()
    o = EbSolveOpts(int(mixed), inner_tol, max_inner, max_outer, max_iters, -1 if time_applies else 1,
                    {"jacobi": 0, "mg": 1}[precond])
    info = EbSolveInfo()
    code = lib.eb_solve(st.handle, _vec64(rho, st.ncell, "rho"), _vec64(g_eb, st.n_cut, "g_eb"),
                        _vec64(g_wall, st.n_wall, "g_wall"), tol, ctypes.byref(o), _vec64(phi, st.ncell, "phi"),
                        ctypes.byref(info), _stream(stream))
    if not (allow_not_converged and code == 4):
        _check(code)
    d = info.as_dict()
    d["status"] = STATUS.get(code, code)
    return d


def eb_fp64_fma_rate(blocks_per_sm=8, iters=1 << 16, stream=None) -> float:
    """Measured FP64 FMA throughput of the device in TFLOP/s (see eb.h)."""
    out = ctypes.c_double()
    _check(load().eb_fp64_fma_rate(int(blocks_per_sm), int(iters), ctypes.byref(out), _stream(stream)))
    return out.value


class BatchSolver:
    """The batched refined solve of several stencil sets (eb_batch_solver_*): one CUDA graph launch per
    solve, the systems' refinement loops run on the device side by side (see eb.h)."""

    def __init__(self, stencils, inner_tol=1e-5, max_inner=20000, max_outer=40, max_iters=400000, precond="mg",
                 stream=None):
        lib = load()
        self.stencils = list(stencils)  # kept alive with the solver
        o = EbSolveOpts(1, inner_tol, max_inner, max_outer, max_iters, 1, {"jacobi": 0, "mg": 1}[precond])
        hs = (ctypes.c_void_p * len(self.stencils))(*[st.handle for st in self.stencils])
        self.handle = ctypes.c_void_p()
        _check(lib.eb_batch_solver_create(hs, len(self.stencils), ctypes.byref(o), ctypes.byref(self.handle),
                                          _stream(stream)))

    def solve(self, rho, g_eb, g_wall, phi, tol=1e-12, stream=None, allow_not_converged=False) -> list:
        """rho, g_eb, g_wall, phi: lists of device FP64 tensors, one per system; phi in/out."""
        n = len(self.stencils)
        if not all(len(v) == n for v in (rho, g_eb, g_wall, phi)):
            raise ValueError(f"BatchSolver.solve: one rho, g_eb, g_wall and phi per system ({n}) expected")

        def arr(ts, size, what):
            return (ctypes.c_void_p * n)(*[_vec64(t, size(st), f"{what}[{k}]")
                                           for k, (t, st) in enumerate(zip(ts, self.stencils))])

        infos = (EbSolveInfo * n)()
        code = load().eb_batch_solve(self.handle, arr(rho, lambda st: st.ncell, "rho"),
                                     arr(g_eb, lambda st: st.n_cut, "g_eb"), arr(g_wall, lambda st: st.n_wall, "g_wall"),
                                     tol, arr(phi, lambda st: st.ncell, "phi"), infos, _stream(stream))
        if not (allow_not_converged and code == 4):
            _check(code)
        return [infos[k].as_dict() for k in range(n)]

    def __del__(self):
        if getattr(self, "handle", None) and _LIB is not None:
            _LIB.eb_batch_solver_destroy(self.handle)
            self.handle = None


def eb_norms(st: Stencils, err, stream=None) -> dict:
    out = (ctypes.c_double * 3)()
    _check(load().eb_norms(st.handle, _vec64(err, st.ncell, "err"), out, _stream(stream)))
    return {"linf": out[0], "l1": out[1], "l2": out[2]}


def eb_stencil_query(st: Stencils, face: int, stream=None):
    """(cols, s_hat) of a face; cols: cell index (volume) or -(1 + face id) (boundary face)."""
    lib = load()
    n = ctypes.c_int32()
    _check(lib.eb_stencil_query(st.handle, int(face), ctypes.byref(n), None, None, 0, _stream(stream)))
    cols = np.zeros(max(n.value, 1), dtype=np.int64)
    vals = np.zeros(max(n.value, 1), dtype=np.float64)
    _check(lib.eb_stencil_query(st.handle, int(face), ctypes.byref(n),
                                cols.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                vals.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), n.value, _stream(stream)))
    return cols[:n.value], vals[:n.value]


def eb_last_error_faces() -> np.ndarray:
    lib = load()
    n = ctypes.c_int32()
    _check(lib.eb_last_error_faces(None, 0, ctypes.byref(n)))
    out = np.zeros(max(n.value, 1), dtype=np.int64)
    _check(lib.eb_last_error_faces(out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), n.value, ctypes.byref(n)))
    return out[:n.value]


def eb_lsq_batch_noalloc(B, w, F, row_ptr, K, max_rows, s, status, stream=None):
    """Batched weighted minimum-norm least squares with no allocation (see include/eb.h).

    For callers that cannot allocate device memory where they solve (fixed pools or arenas,
    real-time hosts, allocation-free plugin callbacks): all tensors are the caller's, and the
    library's working storage is one fixed array.  Calls that overlap on the GPU race.
    """
    import torch
    n_sys = int(row_ptr.numel()) - 1
    for t, dt in ((B, torch.float64), (w, torch.float64), (F, torch.float64), (s, torch.float64),
                  (row_ptr, torch.int64), (status, torch.int32)):
        assert t.dtype == dt and t.is_cuda and t.is_contiguous(), "eb_lsq_batch_noalloc: argument type"
    nnz = w.numel()  # the caller's row count (row_ptr[-1]), taken from w to avoid a device read
    assert n_sys >= 0 and B.numel() == nnz * int(K) and s.numel() == nnz, "eb_lsq_batch_noalloc: row arrays"
    assert F.numel() == n_sys * int(K) and status.numel() == n_sys, "eb_lsq_batch_noalloc: system arrays"
    _check(load().eb_lsq_batch_noalloc(_ptr(B), _ptr(w), _ptr(F), _ptr(row_ptr), n_sys, int(K), int(max_rows),
                                       _ptr(s), _ptr(status), _stream(stream)))
    return s


def eb_kernel_launches() -> int:
    return int(load().eb_kernel_launches())


__all__ = ["eb_kernel_launches", "eb_lsq_batch_noalloc", "eb_geometry_circles", "eb_geometry_spheres", "GpuGeometry", "eb_adjoint_radii", "eb_adjoint_shape", "BatchSolver", "eb_fp64_fma_rate", "load", "lib_path", "DeviceGeometry", "Stencils", "eb_build_stencils", "eb_apply", "eb_bc_rhs", "eb_solve",
           "eb_norms", "eb_stencil_query", "eb_wall_faces", "eb_last_error_faces", "EbError", "EB_F32", "EB_F64"]

"""The least-squares stencils (Sec. 2.2.1, s = W (A^T W)^+ F) by the two factorisation paths: EB_LS_MIXED
(the default: FP32 Householder factor, FP64 corrected semi-normal iterations preconditioned by it, an
FP64 pass for the systems it leaves) and EB_LS_FP64 (FP64 Householder for every system).  Both are
the FP64 minimum-norm solution to rounding: the stencils agree face by face to 1e-11 of each face's
largest coefficient and the FP64 operators to 1e-11 normwise; the mixed path's stencils against the
oracle (SVD) to 1e-10 on sampled faces (the parity tests run the default path too)."""
import numpy as np
import pytest

import eb_inputs as E
from gpu_helpers import compare_stencils, sample_faces, to_dev
from oracle.eb_oracle import Oracle, Params

pytestmark = pytest.mark.gpu


def _both(g, order=4):
    import paper_1411_4283_gb300 as P
    dg = P.DeviceGeometry.from_geometry(g)
    return P.eb_build_stencils(dg, order=order), P.eb_build_stencils(dg, order=order, ls_precision="fp64")


def _compare(g, sm, sd, faces):
    import torch
    import paper_1411_4283_gb300 as P
    for f in faces:
        cm, vm = P.eb_stencil_query(sm, int(f))
        cd, vd = P.eb_stencil_query(sd, int(f))
        assert np.array_equal(cm, cd), f
        assert np.abs(vm - vd).max() <= 1e-11 * np.abs(vd).max(), (f, np.abs(vm - vd).max())
    phi = to_dev(E.seeded_field(11, g.ncell) * (g.flag > 0))
    ym, yd = torch.empty_like(phi), torch.empty_like(phi)
    P.eb_apply(sm, phi, ym)
    P.eb_apply(sd, phi, yd)
    assert (torch.linalg.norm(ym - yd) / torch.linalg.norm(yd)).item() <= 1e-11


@pytest.mark.parametrize("order", [4, 2])
def test_mixed_equals_fp64_3d(order):
    g = E.sphere_box_config(24, seed=2)
    sm, sd = _both(g, order)
    assert sd.info["n_ls_fp64"] == sd.info["n_unique_faces"] + sd.info["n_classes"]
    assert sm.info["n_ls_fp64"] < 0.05 * (sm.info["n_unique_faces"] + sm.info["n_classes"])
    o = Oracle(g, Params(order=order))
    faces = sample_faces(o, 80, seed=9)
    _compare(g, sm, sd, faces)
    compare_stencils(sm, o, faces[:30])


def test_mixed_equals_fp64_2d():
    g = E.multi_circle_config(128)
    sm, sd = _both(g)
    o = Oracle(g, Params(order=4))
    faces = sample_faces(o, 200, seed=10)
    _compare(g, sm, sd, faces)
    compare_stencils(sm, o, faces[:60])


def test_mixed_equals_fp64_eight_spheres():
    g = E.multi_sphere_config(32)
    sm, sd = _both(g)
    o = Oracle(g, Params(order=4))
    _compare(g, sm, sd, sample_faces(o, 80, seed=12))

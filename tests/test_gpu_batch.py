"""Many-instance batch: the stencils of several geometries built with one least-squares launch equal
those of separate builds (and, through them, the oracle's)."""
import numpy as np
import pytest

import eb_inputs as E
from gpu_helpers import compare_stencils, sample_faces, to_dev
from oracle.eb_oracle import Oracle, Params

pytestmark = pytest.mark.gpu


def _same_stencils(sa, sb, faces):
    import paper_1411_4283_gb300 as P
    for f in faces:
        ca, va = P.eb_stencil_query(sa, int(f))
        cb, vb = P.eb_stencil_query(sb, int(f))
        assert np.array_equal(ca, cb), f
        assert np.abs(va - vb).max() <= 1e-14 * max(np.abs(vb).max(), 1e-300), f


def _geoms_2d():
    return [E.circle_config(24), E.multi_circle_config(32, seed=3),
            E.circle_config(40, center=(0.45, 0.55), r=0.2),
            E.Geometry(2, 16, np.zeros((0, 3)), np.zeros(0), False, 4, name="box"),
            E.multi_circle_config(48, seed=5)]


def test_batch_equals_single_2d():
    import torch
    import paper_1411_4283_gb300 as P
    gs = _geoms_2d()
    dgs = [P.DeviceGeometry.from_geometry(g) for g in gs]
    batch = P.eb_build_stencils_batch(dgs, order=4)
    for g, dg, sb in zip(gs, dgs, batch):
        ss = P.eb_build_stencils(dg, order=4)
        assert sb.info["n_unique_faces"] == ss.info["n_unique_faces"]
        o = Oracle(g, Params(order=4))
        _same_stencils(sb, ss, o.flux_faces())
        phi = to_dev(E.seeded_field(7, g.ncell) * (g.flag > 0))
        ya = torch.empty_like(phi)
        yb = torch.empty_like(phi)
        P.eb_apply(sb, phi, ya)
        P.eb_apply(ss, phi, yb)
        assert torch.equal(ya, yb)
    # the chain closes at the oracle for one geometry of the batch
    o = Oracle(gs[1], Params(order=4))
    compare_stencils(batch[1], o, o.flux_faces())


def test_batch_equals_single_3d():
    import paper_1411_4283_gb300 as P
    gs = [E.sphere_box_config(16), E.sphere_box_config(20)]
    dgs = [P.DeviceGeometry.from_geometry(g) for g in gs]
    batch = P.eb_build_stencils_batch(dgs, order=4)
    for g, dg, sb in zip(gs, dgs, batch):
        ss = P.eb_build_stencils(dg, order=4)
        o = Oracle(g, Params(order=4))
        _same_stencils(sb, ss, sample_faces(o, 60, seed=4))
    o = Oracle(gs[0], Params(order=4))
    compare_stencils(batch[0], o, sample_faces(o, 30, seed=6))


def test_batch_rejects_mixed_dimensions():
    import paper_1411_4283_gb300 as P
    dgs = [P.DeviceGeometry.from_geometry(E.circle_config(16)), P.DeviceGeometry.from_geometry(E.sphere_box_config(12))]
    with pytest.raises(P.EbError):
        P.eb_build_stencils_batch(dgs, order=4)


def test_batch_failure_in_a_worker_reaches_the_caller():
    """A geometry that the build rejects (moment tables shallower than the order) fails the whole
    batch with its own status and message, although its phases ran on a worker thread; the other
    geometries' stencils are released and a later batch works."""
    import paper_1411_4283_gb300 as P
    gs = [E.circle_config(16 + 4 * i) for i in range(6)]
    dgs = [P.DeviceGeometry.from_geometry(g) for g in gs]
    dgs[3].moment_degree = 2
    with pytest.raises(P.EbError) as ei:
        P.eb_build_stencils_batch(dgs, order=4)
    assert ei.value.code == 1 and "shallower" in str(ei.value)
    dgs[3] = P.DeviceGeometry.from_geometry(gs[3])
    batch = P.eb_build_stencils_batch(dgs, order=4)
    assert len(batch) == len(gs)


def test_batch_with_an_ellipse_against_the_oracle():
    """A batch of an ellipse (a = 0.31, b = 0.17, tables from eb_inputs/ellipse.py) and a circle: the
    ellipse's stencils against the oracle's (sampled faces, 1e-10 of each face's largest coefficient),
    and its batched refined solve equal to the single-geometry solve (1e-10 of max|phi|)."""
    import torch
    import paper_1411_4283_gb300 as P
    from eb_inputs.ellipse import EllipseGeometry
    ge = EllipseGeometry(48, [(0.503, 0.497)], [(0.31, 0.17)])
    gs = [ge, E.circle_config(40)]
    dgs = [P.DeviceGeometry.from_geometry(g) for g in gs]
    batch = P.eb_build_stencils_batch(dgs, order=4)
    o = Oracle(ge, Params(order=4))
    compare_stencils(batch[0], o, sample_faces(o, 60, seed=13))
    f64 = dict(dtype=torch.float64, device="cuda")
    rho = [torch.ones(g.ncell, **f64) for g in gs]
    geb = [torch.zeros(max(len(g.cut_cells), 1), **f64) for g in gs]
    gw = [torch.zeros(max(len(P.eb_wall_faces(st)), 1), **f64) for st in batch]
    phis = [torch.zeros(g.ncell, **f64) for g in gs]
    P.BatchSolver(batch).solve(rho, geb, gw, phis, tol=1e-10)
    for st, r_, e_, w_, x, g in zip(batch, rho, geb, gw, phis, gs):
        y = torch.zeros(g.ncell, **f64)
        P.eb_solve(st, r_, e_, w_, y, tol=1e-10)
        assert (x - y).abs().max().item() <= 1e-10 * y.abs().max().item()

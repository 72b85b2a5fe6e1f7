"""Shared helpers of the GPU parity tests: oracle references and device marshalling."""
import numpy as np

from oracle.eb_oracle import Oracle


def to_dev(a, dtype=None):
    import torch
    t = torch.as_tensor(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def build_gpu(g, order=4, **kw):
    import paper_1411_4283_gb300 as P
    dg = P.DeviceGeometry.from_geometry(g)
    return P.eb_build_stencils(dg, order=order, **kw), dg


def compare_stencils(st, o: Oracle, faces, tol=1e-10, ref=None):
    """Column lists identical; coefficients within tol * max|s| per face.  Returns the worst ratio."""
    import paper_1411_4283_gb300 as P
    worst = 0.0
    for f in faces:
        cols, s = P.eb_stencil_query(st, int(f))
        oc, os_ = ref[f] if ref is not None else o.stencil(int(f))
        assert np.array_equal(cols, oc), (f, cols[:10], oc[:10])
        r = np.abs(s - os_).max() / np.abs(os_).max()
        worst = max(worst, r)
        assert r <= tol, (f, r)
    return worst


def split_boundary(o: Oracle, G):
    bf = o.boundary_faces()
    n_wall = sum(1 for f in bf if f < o.n_grid_faces)
    return np.asarray(G[:n_wall]), np.asarray(G[n_wall:]), bf[:n_wall]


def sample_faces(o: Oracle, n, seed=0):
    """A mix of EB faces, faces next to the EB, wall faces and interior faces."""
    rng = np.random.default_rng(seed)
    faces = o.flux_faces()
    eb = [f for f in faces if f >= o.n_grid_faces]
    grid = np.array([f for f in faces if f < o.n_grid_faces])
    near = []
    cut = set(int(c) for c in o.g.cut_cells)
    for f in grid[rng.permutation(len(grid))]:
        if len(near) >= n // 3:
            break
        cells = [c for c, _ in o.face_cells(int(f))]
        if any(c in cut for c in cells):
            near.append(int(f))
    walls = [f for f in o.boundary_faces() if f < o.n_grid_faces]
    pick = list(rng.choice(eb, min(len(eb), n // 3), replace=False)) if eb else []
    pick += near
    pick += list(rng.choice(walls, min(len(walls), n // 6), replace=False))
    pick += list(rng.choice(grid, n // 6, replace=False))
    return sorted(set(int(x) for x in pick))

"""Parity at the benchmark's full size: the 3-D sphere workload at 256^3 (Q = 4, box neighbourhoods),
built and applied exactly as bench.py does, checked on sampled outputs that the oracle computes one
by one: stencils of EB faces, of grid faces next to cut cells, of wall faces and of interior
(template-class) faces (1e-10 of each face's largest coefficient), and operator rows of cut cells,
cells next to the EB, wall-layer cells (among them cells of the aligned x-runs), interior cells and
cells next to the first and last grid rows (FP64 apply 1e-12 of the row, FP32 1e-5 of the field's
scale).  The geometry alone takes about a minute on the host."""
import numpy as np
import pytest

import eb_inputs as E
from gpu_helpers import compare_stencils, to_dev
from oracle.eb_oracle import Oracle, Params

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
N = 256


@pytest.fixture(scope="module")
def sphere256():
    import paper_1411_4283_gb300 as P
    g = E.sphere_box_config(N, seed=2)
    o = Oracle(g, Params(order=4))
    st = P.eb_build_stencils(P.DeviceGeometry.from_geometry(g), order=4)
    return g, o, st


def _sample_faces(g, o, rng):
    faces = []
    cuts = rng.choice(len(g.cut_cells), 12, replace=False)
    faces += [o.eb_id(int(c)) for c in cuts]
    for c in cuts:  # grid faces of cut cells (both sides, all directions), where open
        ijk = o.cell_coords(int(g.cut_cells[c]))
        d = int(rng.integers(3))
        for side in (0, 1):
            fx = list(ijk)
            fx[d] += side
            f = o.face_local(d, fx)
            if o.face_open(d, f):
                faces.append(o.face_id(d, f))
    for _ in range(6):  # wall faces
        d = int(rng.integers(3))
        fx = [int(v) for v in rng.integers(0, N, 3)]
        fx[d] = 0 if rng.integers(2) == 0 else N
        f = o.face_local(d, fx)
        if o.face_open(d, f):
            faces.append(o.face_id(d, f))
    for ijk in ([64, 64, 64], [40, 200, 120], [200, 30, 60]):  # interior faces far from the sphere
        faces.append(o.face_id(0, o.face_local(0, ijk)))
    return sorted(set(faces))


def test_stencils_256(sphere256):
    g, o, st = sphere256
    compare_stencils(st, o, _sample_faces(g, o, np.random.default_rng(7)))


def _sample_cells(g, o, rng):
    L = 4
    cells = [int(g.cut_cells[c]) for c in rng.choice(len(g.cut_cells), 8, replace=False)]
    near = []
    for c in rng.choice(len(g.cut_cells), 40, replace=False):  # full cells next to a cut cell
        ijk = o.cell_coords(int(g.cut_cells[c]))
        for d in range(3):
            for s in (-1, 1):
                q = list(ijk)
                q[d] += s
                if 0 <= q[d] < N and g.flag[o.cell_index(q)] == 1:
                    near.append(o.cell_index(q))
    cells += list(rng.choice(near, 6, replace=False))
    for _ in range(8):  # wall layer, away from the x walls (x-runs) and anywhere
        q = [int(v) for v in rng.integers(8, N - 8, 3)]
        d = int(rng.integers(1, 3))
        q[d] = int(rng.integers(0, L + 1)) if rng.integers(2) == 0 else N - 1 - int(rng.integers(0, L + 1))
        cells.append(o.cell_index(q))
        q2 = [int(v) for v in rng.integers(8, N - 8, 3)]
        q2[0] = int(rng.integers(0, L + 1))
        cells.append(o.cell_index(q2))
    cells += [o.cell_index(q) for q in ([60, 60, 60], [30, 200, 100], [128, 20, 128], [200, 200, 40])]
    cells += [o.cell_index(q) for q in ([1, 2, 1], [0, 0, 0], [N - 2, N - 1, N - 2], [N - 1, N - 1, N - 1])]
    return [c for c in sorted(set(int(c) for c in cells)) if g.flag[c] > 0]


def test_operator_rows_256(sphere256):
    import torch
    import paper_1411_4283_gb300 as P
    g, o, st = sphere256
    phi = E.seeded_field(31, g.ncell) * (g.flag > 0)
    y = torch.empty(g.ncell, dtype=torch.float64, device="cuda")
    P.eb_apply(st, to_dev(phi), y, kappa_weighted=True)
    yg = y.cpu().numpy()
    y32 = torch.empty(g.ncell, dtype=torch.float32, device="cuda")
    P.eb_apply(st, to_dev(phi, torch.float32), y32, kappa_weighted=True)
    yg32 = y32.cpu().numpy().astype(np.float64)
    scale = np.abs(yg).max()
    for c in _sample_cells(g, o, np.random.default_rng(8)):
        acc = 0.0
        for fid, sg in o.cell_flux_faces(c):
            cols, s = o.stencil(fid)
            vm = cols >= 0
            acc += sg * float(s[vm] @ phi[cols[vm]])
        acc /= g.h ** 2
        assert abs(yg[c] - acc) <= 1e-12 * max(abs(acc), scale * 1e-3), (c, yg[c], acc)
        assert abs(yg32[c] - acc) <= 1e-5 * scale, (c, yg32[c], acc)

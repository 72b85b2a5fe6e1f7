"""The allocation-free batched least-squares entry point.

eb_lsq_batch_noalloc serves callers that cannot allocate device memory where they solve (code
inside a fixed memory pool or arena, real-time hosts that allocate only at start-up, plugin hosts
that forbid allocation in callbacks); its working storage is one fixed array inside the library.
Here it solves the weighted systems of sampled faces (rows formed on the host by the oracle from
the same geometry) and must return, on two calls in a row with different systems, both the
stencils that eb_build_stencils computed for those faces and the oracle's minimum-norm stencils,
to the stencil tolerance of the parity tests (1e-10 of each face's largest coefficient).  Systems
the kernel must refuse (fewer rows than unknowns, a zero column, more rows than the fixed storage
holds) get their status codes and zero stencils.
"""
import numpy as np
import pytest

import eb_inputs as E
from oracle.eb_oracle import Oracle, Params

pytestmark = pytest.mark.gpu


def _batch(o, faces):
    Bs, ws, Fs, ptr = [], [], [], [0]
    for f in faces:
        A, F, w, _ = o.face_system(int(f))
        Bs.append(w[:, None] * A)
        ws.append(w)
        Fs.append(F)
        ptr.append(ptr[-1] + len(w))
    return np.vstack(Bs), np.concatenate(ws), np.vstack(Fs), np.array(ptr, dtype=np.int64)


def _run(B, w, F, ptr, K, max_rows):
    import torch
    import paper_1411_4283_gb300 as P
    dev = dict(device="cuda")
    s = torch.full((len(w),), float("nan"), dtype=torch.float64, **dev)
    status = torch.full((len(ptr) - 1,), -1, dtype=torch.int32, **dev)
    P.eb_lsq_batch_noalloc(torch.tensor(B, **dev).contiguous(), torch.tensor(w, **dev), torch.tensor(F, **dev),
                           torch.tensor(ptr, **dev), K, max_rows, s, status)
    torch.cuda.synchronize()
    return s.cpu().numpy(), status.cpu().numpy()


def _check_call(order, seed):
    import paper_1411_4283_gb300 as P
    g = E.circle_config(32, center=(0.51, 0.49), r=0.3)
    o = Oracle(g, Params(order=order))
    st = P.eb_build_stencils(P.DeviceGeometry.from_geometry(g), order=order)
    rng = np.random.default_rng(seed)
    faces = o.flux_faces()
    pick = sorted(set(list(rng.choice(faces, 60, replace=False)) + faces[-20:]))
    B, w, F, ptr = _batch(o, pick)
    sv, status = _run(B, w, F, ptr, o.K, int(np.diff(ptr).max()))
    assert np.all(status == 0)
    for q, f in enumerate(pick):
        got = sv[ptr[q]:ptr[q + 1]]
        _, ref = P.eb_stencil_query(st, int(f))   # the existing entry point's stencil
        _, orc = o.stencil(int(f))                 # the oracle's minimum-norm stencil (SVD route)
        assert len(got) == len(ref) == len(orc)
        assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max(), (f, np.abs(got - ref).max())
        assert np.abs(got - orc).max() <= 1e-10 * np.abs(orc).max(), (f, np.abs(got - orc).max())


def test_noalloc_matches_stencil_build_and_oracle_twice():
    _check_call(4, seed=5)   # first call: fourth-order systems (K = 15)
    _check_call(2, seed=6)   # second call: different systems and K (K = 6) in the same fixed storage


def test_noalloc_refused_systems_get_status_and_zero_stencils():
    g = E.circle_config(32, center=(0.51, 0.49), r=0.3)
    o = Oracle(g, Params(order=4))
    K = o.K
    faces = o.flux_faces()
    A0, F0, w0, _ = o.face_system(int(faces[0]))
    A1, F1, w1, _ = o.face_system(int(faces[1]))
    rng = np.random.default_rng(3)
    # system 0: a good one; 1: fewer rows than unknowns; 2: a zero column (rank K - 1);
    # 3: 300 rows, more than the fixed storage holds (the caller claims max_rows = 256);
    # 4: a good one after the refused ones
    short = (w0[:K - 3, None] * A0[:K - 3])
    zero_col = w1[:, None] * A1
    zero_col[:, 5] = 0.0
    big = rng.standard_normal((300, K))
    systems = [(w0[:, None] * A0, w0, F0), (short, w0[:K - 3], F0), (zero_col, w1, F1),
               (big, np.ones(300), rng.standard_normal(K)), (w1[:, None] * A1, w1, F1)]
    B = np.vstack([s[0] for s in systems])
    w = np.concatenate([s[1] for s in systems])
    F = np.vstack([s[2] for s in systems])
    ptr = np.cumsum([0] + [len(s[1]) for s in systems]).astype(np.int64)
    sv, status = _run(B, w, F, ptr, K, 256)
    assert list(status) == [0, 1, 1, 3, 0]
    for q in (1, 2, 3):
        assert np.all(sv[ptr[q]:ptr[q + 1]] == 0.0)
    for q, f in ((0, faces[0]), (4, faces[1])):
        _, orc = o.stencil(int(f))
        got = sv[ptr[q]:ptr[q + 1]]
        assert np.abs(got - orc).max() <= 1e-10 * np.abs(orc).max()


def test_noalloc_rejects_oversized_max_rows():
    import torch
    import paper_1411_4283_gb300 as P
    dev = dict(device="cuda")
    K = 15
    B = torch.zeros(300 * K, dtype=torch.float64, **dev)
    w = torch.ones(300, dtype=torch.float64, **dev)
    F = torch.zeros(K, dtype=torch.float64, **dev)
    s = torch.zeros(300, dtype=torch.float64, **dev)
    ptr = torch.tensor([0, 300], dtype=torch.int64, **dev)
    with pytest.raises(P.EbError) as ei:
        P.eb_lsq_batch_noalloc(B, w, F, ptr, K, 300, s, torch.zeros(1, dtype=torch.int32, **dev))
    assert ei.value.code == 8

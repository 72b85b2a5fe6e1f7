"""The allocation-free batched least-squares entry point against the stencil build.

eb_lsq_batch_noalloc serves callers that cannot allocate device memory where they solve; its
working storage is one fixed array inside the library.  Here it solves the weighted systems of
sampled faces (rows formed on the host from the same geometry) and must return the stencils that
eb_build_stencils computed for those faces, to the stencil tolerance of the parity tests (1e-10
of each face's largest coefficient), on two calls in a row with different systems.
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


def _check_call(order, seed):
    import torch
    import paper_1411_4283_gb300 as P
    g = E.circle_config(32, center=(0.51, 0.49), r=0.3)
    o = Oracle(g, Params(order=order))
    st = P.eb_build_stencils(P.DeviceGeometry.from_geometry(g), order=order)
    rng = np.random.default_rng(seed)
    faces = o.flux_faces()
    pick = sorted(set(list(rng.choice(faces, 60, replace=False)) + faces[-20:]))
    B, w, F, ptr = _batch(o, pick)
    dev = dict(device="cuda")
    s = torch.full((len(w),), float("nan"), dtype=torch.float64, **dev)
    status = torch.full((len(pick),), -1, dtype=torch.int32, **dev)
    P.eb_lsq_batch_noalloc(torch.tensor(B, **dev), torch.tensor(w, **dev), torch.tensor(F, **dev),
                           torch.tensor(ptr, **dev), o.K, int(np.diff(ptr).max()), s, status)
    torch.cuda.synchronize()
    assert np.all(status.cpu().numpy() == 0)
    sv = s.cpu().numpy()
    for q, f in enumerate(pick):
        ref_cols, ref = P.eb_stencil_query(st, int(f))  # the existing entry point's stencil
        got = sv[ptr[q]:ptr[q + 1]]
        assert len(got) == len(ref)
        assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max(), (f, np.abs(got - ref).max())


def test_noalloc_matches_stencil_build_twice():
    _check_call(4, seed=5)   # first call: fourth-order systems (K = 15)
    _check_call(2, seed=6)   # second call: different systems and K (K = 6) in the same fixed storage


def test_noalloc_rejects_oversized_systems():
    import torch
    import paper_1411_4283_gb300 as P
    dev = dict(device="cuda")
    one = torch.zeros(1, dtype=torch.float64, **dev)
    ptr = torch.tensor([0, 300], dtype=torch.int64, **dev)
    with pytest.raises(P.EbError) as ei:
        P.eb_lsq_batch_noalloc(one, one, one, ptr, 15, 300, one, torch.zeros(1, dtype=torch.int32, **dev))
    assert ei.value.code == 8

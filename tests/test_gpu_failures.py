"""Failure paths of the GPU build, made on the host with valid inputs (nothing here faults a GPU).

Rank deficiency (Sec. 2.4 uses one neighbourhood radius everywhere; the paper only calls the
four-circle grid at N = 32 "too coarse", Sec. 3.5): with box neighbourhoods of radius R_n = 1 a
fourth-order face (K = 15 monomials) sees at most 12 volumes plus a few boundary faces, so most of
its systems have rank below K.  The build must refuse with EB_ERR_RANK_DEFICIENT, return no
stencils, and list exactly the faces the oracle refuses.  The two sides decide rank with different
tests (the oracle: numpy's SVD rank; the GPU: |R_kk| <= 1e-12 max |R_jj| in its QR), so faces whose
smallest singular value lies between 1e-14 and 1e-10 of the largest, where either answer is
defensible, are left out of the comparison; every other face must be classified the same way.
"""
import numpy as np
import pytest

import eb_inputs as E
from oracle.eb_oracle import Oracle, Params

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("N", [16, 24])
def test_rank_deficient_faces_reported(N):
    import paper_1411_4283_gb300 as P
    g = E.circle_config(N, center=(0.51, 0.49), r=0.3)
    o = Oracle(g, Params(order=4, path_radius=1))
    bad, ambiguous = set(), set()
    for f in o.flux_faces():
        A, F, w, _ = o.face_system(f)
        sv = np.linalg.svd(w[:, None] * A, compute_uv=False)
        ratio = sv[-1] / sv[0] if len(w) >= o.K else 0.0
        if len(w) >= o.K and 1e-14 <= ratio <= 1e-10:
            ambiguous.add(f)
        elif len(w) < o.K or np.linalg.matrix_rank(w[:, None] * A) < o.K:
            bad.add(f)
    assert len(bad) > 0.5 * len(o.flux_faces())
    with pytest.raises(P.EbError) as ei:
        P.eb_build_stencils(P.DeviceGeometry.from_geometry(g), order=4, path_radius=1)
    assert ei.value.code == 2
    got = P.eb_last_error_faces()
    assert np.all(np.diff(got) > 0)                      # ascending, no repeats
    got = set(int(f) for f in got) - ambiguous
    assert got == bad, (sorted(got - bad)[:10], sorted(bad - got)[:10])


def test_build_succeeds_after_a_refused_build():
    """A refused build leaves nothing behind: the next build on the same device succeeds and its
    error list is cleared."""
    import paper_1411_4283_gb300 as P
    g = E.circle_config(16, center=(0.51, 0.49), r=0.3)
    with pytest.raises(P.EbError):
        P.eb_build_stencils(P.DeviceGeometry.from_geometry(g), order=4, path_radius=1)
    st = P.eb_build_stencils(P.DeviceGeometry.from_geometry(g), order=4)
    assert st.info["n_flux_faces"] > 0
    assert len(P.eb_last_error_faces()) == 0

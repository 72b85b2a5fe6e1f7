"""Writes the FP64 oracle's full discrete solutions of the 3-D problems that the element-wise
solve parity tests compare the GPU's refined solve with.  Calls only oracle/ and eb_inputs/.

    python tests/golden/make_solve_goldens.py [name ...]

Each file holds the volume cells (ascending cell index), the oracle's solution phi there (sparse
LU of the kappa-weighted operator, Sec. 2.3), and its error norms (Sec. 3.3):

  sphere_inside_n32.npz      inside the sphere (0.5, 0.5, 0.5), r = 0.45 (the example of Sec. 3.6),
                             Q = 4, N = 32, Dirichlet data of the paper's 3-D solution
  sphere_box_n16.npz         the unit cube minus the sphere r = 0.35 with the seeded centre offset
                             (the benchmark geometry), Q = 4, N = 16, Dirichlet EB and walls
  sphere_box_n16_neumann.npz the same with Neumann data on the EB (Sec. 2.2.1 Neumann rows; the
                             flux through a Neumann EB face is its datum), Dirichlet walls
  five_circles_n128_q4.npz   the 2-D convergence-sweep geometry (the circle r = 0.3 at (0.51, 0.49)
  five_circles_n128_q2.npz   and four seeded circles), N = 128, phi = sin(2 pi x) cos(3 pi y), Q = 4
                             and Q = 2

The sphere-inside case takes ~20 minutes on 8 cores (each 3-D face costs ~0.2 s in the oracle),
each N = 16 case a few minutes.
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))
sys.path.insert(0, os.path.dirname(HERE))


def cases():
    import eb_inputs as E
    return {
        "sphere_inside_n32": (lambda: E.sphere_inside_config(32), False),
        "sphere_box_n16": (lambda: E.sphere_box_config(16, seed=2), False),
        "sphere_box_n16_neumann": (lambda: E.sphere_box_config(16, seed=2), True),
        "five_circles_n128_q4": (lambda: E.multi_circle_config(128), False),
        "five_circles_n128_q2": (lambda: E.multi_circle_config(128), False),
    }


def make(name):
    import eb_inputs as E
    from oracle.eb_oracle import Oracle, Params, run_problem
    from oracle_pool import parallel_stencils
    mk, neumann = cases()[name]
    g = mk()
    man = E.Manufactured(g, E.sin_product("paper3d" if g.dim == 3 else "sin2pix_cos3piy"))
    bc = np.ones(len(g.cut_cells), np.uint8) if neumann else None
    p = Params(order=2 if name.endswith("_q2") else 4)
    t0 = time.time()
    st = parallel_stencils(g, p, Oracle(g, p, bc).flux_faces(), bc_eb=bc)
    r = run_problem(g, man, p, bc_eb=bc, stencils=st)
    cells = np.nonzero(g.flag > 0)[0].astype(np.int32)
    np.savez_compressed(os.path.join(HERE, name + ".npz"), cells=cells, phi=r["phi"][cells],
                        sol=np.array([r["sol"][k] for k in ("linf", "l1", "l2")]),
                        trunc=np.array([r["trunc"][k] for k in ("linf", "l1", "l2")]), N=g.N, order=p.order,
                        neumann=int(neumann),
                        source="oracle/eb_oracle.py run_problem via tests/golden/make_solve_goldens.py")
    print(name, f"{time.time() - t0:.0f} s", r["sol"], flush=True)


if __name__ == "__main__":
    for nm in (sys.argv[1:] or list(cases())):
        make(nm)

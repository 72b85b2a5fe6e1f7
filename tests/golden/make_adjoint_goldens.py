"""Writes the adjoint oracle's objective and shape gradients for the 3-D GPU adjoint tests.  Calls
only oracle/ and eb_inputs/.

    python tests/golden/make_adjoint_goldens.py

adjoint3d_goldens.npz holds, per case, J = 1/2 sum |V| phi^2 for kappa L phi = kappa with homogeneous
Dirichlet data (Sec. 2.3, Q = 4) and its derivatives with respect to the listed parameters, from
oracle/eb_adjoint.py objective_and_radius_gradient (LU solves, SVD stencils, complex-step rows; the
sphere radius through sphere_moment_derivatives, a level-set mode through fourier_mode_derivatives):

  sphere_box_n8     the unit cube minus the sphere r = 0.35 with the seeded centre offset, N = 8:
                    the radius and the first two modes of eb_inputs.level_set_modes(16, seed 5)
  two_spheres_n10   eb_inputs.multi_sphere_config(10, n = 2), N = 10: the second sphere's radius and
                    the third mode

Each (case, parameter) runs in its own process (about 3 minutes at N = 8, 8 at N = 10).
"""
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))


def cases():
    import eb_inputs as E
    modes = E.level_set_modes(16, seed=5)
    return {
        "sphere_box_n8": (lambda: E.sphere_box_config(8, seed=2), [("radius", 0), ("mode", modes[0]),
                                                                  ("mode", modes[1])]),
        "two_spheres_n10": (lambda: E.multi_sphere_config(10, n=2), [("radius", 1), ("mode", modes[2])]),
    }


def job(args):
    name, k = args
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    from oracle.eb_adjoint import fourier_mode_derivatives, objective_and_radius_gradient
    from oracle.eb_oracle import Params
    mk, params = cases()[name]
    kind, val = params[k]
    g = mk()
    t0 = time.time()
    if kind == "radius":
        J, dJ = objective_and_radius_gradient(g, int(val), Params(order=4))
    else:
        J, dJ = objective_and_radius_gradient(
            g, 0, Params(order=4), derivs=lambda o: fourier_mode_derivatives(o, val[:3], val[3]))
    print(name, kind, k, J, dJ, f"{time.time() - t0:.0f} s", flush=True)
    return name, k, J, dJ


def main():
    jobs = [(n, k) for n, (_, ps) in cases().items() for k in range(len(ps))]
    with mp.get_context("spawn").Pool(len(jobs)) as pool:
        res = pool.map(job, jobs)
    out = {}
    for name, (mk, params) in cases().items():
        rows = [r for r in res if r[0] == name]
        rows.sort(key=lambda r: r[1])
        out[name + "_J"] = np.array(rows[0][2])
        out[name + "_dJ"] = np.array([r[3] for r in rows])
        out[name + "_kind"] = np.array([0 if p[0] == "radius" else 1 for p in params])
        out[name + "_param"] = np.array([[float(p[1]), 0.0, 0.0, 0.0] if p[0] == "radius" else p[1]
                                         for p in params])
    np.savez(os.path.join(HERE, "adjoint3d_goldens.npz"), **out,
             source="oracle/eb_adjoint.py objective_and_radius_gradient via tests/golden/make_adjoint_goldens.py")


if __name__ == "__main__":
    main()

"""Writes sphere_n32.json: the FP64 oracle's solution errors for the 3-D sphere of Sec. 3.6
(inside the sphere (0.5,0.5,0.5), r = 0.45, Q = 4, N = 32).  Calls only oracle/ and eb_inputs/;
takes about two minutes on 8 cores.

    python tests/golden/make_sphere_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))
sys.path.insert(0, os.path.dirname(HERE))

if __name__ == "__main__":
    import eb_inputs as E
    from oracle.eb_oracle import Oracle, Params, run_problem
    from oracle_pool import parallel_stencils
    g = E.sphere_inside_config(32)
    man = E.Manufactured(g, E.sin_product("paper3d"))
    p = Params(order=4)
    st = parallel_stencils(g, p, Oracle(g, p).flux_faces())
    r = run_problem(g, man, p, stencils=st)
    out = {"_source": "oracle/eb_oracle.py via tests/golden/make_sphere_golden.py; geometry of Sec. 3.6",
           "N": 32, "order": 4, "sol": r["sol"], "trunc": r["trunc"]}
    json.dump(out, open(os.path.join(HERE, "sphere_n32.json"), "w"), indent=1)
    print(out)

"""Runs the oracle's per-face stencil construction over a spawn-started process pool.

The oracle itself is single-threaded; this helper only splits the list of
faces across processes (each builds its own Oracle from the pickled geometry),
so the arithmetic of every stencil is unchanged.
"""
from __future__ import annotations

import multiprocessing as mp
import os

_STATE = {}


def _init(geom, params, bc_eb):
    from oracle.eb_oracle import Oracle
    _STATE["o"] = Oracle(geom, params, bc_eb)


def _work(faces):
    o = _STATE["o"]
    return [(f, o.stencil(f)) for f in faces]


def parallel_stencils(geom, params, faces, bc_eb=None, procs: int | None = None) -> dict:
    procs = procs or min(8, os.cpu_count() or 1)
    faces = list(faces)
    if procs <= 1 or len(faces) < 200:
        _init(geom, params, bc_eb)
        return dict(_work(faces))
    chunks = [faces[i::procs * 4] for i in range(procs * 4)]
    # one BLAS thread per worker (inherited by the spawned processes before they load numpy)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ.setdefault(v, "1")
    ctx = mp.get_context("spawn")
    with ctx.Pool(procs, initializer=_init, initargs=(geom, params, bc_eb)) as pool:
        out = {}
        for part in pool.imap_unordered(_work, chunks):
            out.update(part)
    return out

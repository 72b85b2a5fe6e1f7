"""FP64 CPU oracle for the cut-cell Poisson method (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import, call or execute anything in this package.  The product path
(``paper_1411_4283_gb300``) never does.
"""
from .eb_oracle import (Oracle, monomial_list, Params, solve_dense_lu, error_norms)

__all__ = ["Oracle", "monomial_list", "Params", "solve_dense_lu", "error_norms"]

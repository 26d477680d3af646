"""Active-set selection and configuration-level grades (test infrastructure: only tests/,
the package smoke check and bench.py's CPU legs use the oracle).

MaxVol update (Section II.D, D-optimality): the active set is the m x m matrix A of maximal
|det A| among the available rows.  With C = B A^-1 for candidate rows B, replacing active row
j by candidate row i multiplies |det A| by |C_ij| (Cramer's rule), so the update repeatedly
performs the swap at the largest |C_ij| while it exceeds 1 + eps.  The oracle recomputes C
from scratch (a linear solve) before every swap: no rank-one updates.  A candidate that has
entered A has C row e_j and is not chosen again; a row swapped out is dropped.
"""
from __future__ import annotations

import numpy as np


def maxvol(A, B, eps=1e-3, max_swaps=10_000):
    """Returns (A_final, source, n_swaps): source[j] = -1 if row j of A was kept, else the
    index of the candidate row of B now in its place.  Ties: the first (row-major) maximum."""
    A = np.array(A, np.float64, copy=True)
    B = np.asarray(B, np.float64)
    m = A.shape[0]
    source = np.full(m, -1, np.int64)
    swaps = 0
    if B.shape[0] == 0:
        return A, source, swaps
    while swaps < max_swaps:
        C = np.linalg.solve(A.T, B.T).T        # C = B A^-1
        k = int(np.argmax(np.abs(C)))
        i, j = divmod(k, m)
        if not abs(C[i, j]) > 1.0 + eps:
            break
        A[j] = B[i]
        source[j] = i
        swaps += 1
    return A, source, swaps

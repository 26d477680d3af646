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


# ------------------------------------------------------------------------------------
# configuration-level grades and the learning-on-the-fly thresholds (Sections II.D-II.E)
# ------------------------------------------------------------------------------------

def config_rows(model, theta, batch, nbr=None):
    """b(cfg_k) = dE_k/dtheta = sum_{i in k} b_i (eq. 1 differentiated with eq. 9)."""
    from . import oracle as O
    if nbr is None:
        nbr = O.batch_neighbors(batch, model.r_cut)
    rows = O.site_rows(model, theta, batch["type"], nbr)
    off = batch["atom_offset"]
    return np.stack([rows[off[k]:off[k + 1]].sum(axis=0) for k in range(len(off) - 1)])


def config_grade(A, rows_cfg):
    """gamma(cfg) = max_j |(b(cfg) A^-1)_j| against a configuration-mode active set A."""
    from . import oracle as O
    return O.grade(A, rows_cfg)


def neighborhood_config_grade(gamma_atoms, atom_offset):
    """gamma(cfg) = max over the configuration's neighborhoods of gamma_i (0 for an empty one)."""
    return np.array([max(gamma_atoms[atom_offset[k]:atom_offset[k + 1]], default=0.0)
                     for k in range(len(atom_offset) - 1)])


def classify(gamma, gamma_save, gamma_break):
    """0: gamma <= gamma_save (continue); 1: gamma_save < gamma <= gamma_break (save the
    configuration and continue); 2: gamma > gamma_break (stop).  Strict comparisons."""
    gamma = np.asarray(gamma)
    return (gamma > gamma_save).astype(np.int32) + (gamma > gamma_break).astype(np.int32)


# ------------------------------------------------------------------------------------
# spherical cut of a neighborhood (Section II.E, option (ii): treat it as a cluster)
# ------------------------------------------------------------------------------------

def cut_cluster(batch, center, radius):
    """Every atom j and periodic image n of center's configuration with |x_j + n H - x_c| <
    radius (the center itself at the origin, first), as a non-periodic cluster: returns
    (pos relative to the center [M x 3], type [M], source atom [M]).  Order: the center, then
    ascending (j, n0, n1, n2)."""
    off = batch["atom_offset"]
    k = int(np.searchsorted(off, center, side="right") - 1)
    a0, a1 = off[k], off[k + 1]
    H = batch["cell"][k].reshape(3, 3)
    pbc = batch["pbc"][k]
    xc = batch["pos"][center]
    # image range per axis from the face distances of the cell
    vol = abs(np.linalg.det(H))
    K = []
    for a in range(3):
        h = vol / np.linalg.norm(np.cross(H[(a + 1) % 3], H[(a + 2) % 3]))
        span = np.abs(batch["pos"][a0:a1] @ np.linalg.inv(H)[:, a]).max() + 1.0
        K.append(int(np.ceil(radius / h + span)) + 1 if pbc[a] else 0)
    out = [(center, (0, 0, 0))]
    for j in range(a0, a1):
        for n0 in range(-K[0], K[0] + 1):
            for n1 in range(-K[1], K[1] + 1):
                for n2 in range(-K[2], K[2] + 1):
                    if j == center and n0 == n1 == n2 == 0:
                        continue
                    r = batch["pos"][j] + np.array([n0, n1, n2]) @ H - xc
                    if np.sqrt(r @ r) < radius:
                        out.append((j, (n0, n1, n2)))
    pos = np.array([batch["pos"][j] + np.array(n) @ H - xc for j, n in out])
    return pos, batch["type"][[j for j, _ in out]].astype(np.int32), np.array([j for j, _ in out], np.int64)

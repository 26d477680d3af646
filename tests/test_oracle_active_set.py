"""Pins of the oracle's MaxVol update against determinants computed directly (np.linalg.det,
no use of the oracle's solve-based C): the defining property of the result, the determinant
growth of every swap, and a brute-force optimum on tiny sets."""
import itertools

import numpy as np
import pytest

from oracle import active_set as AS
from paper_2304_13144_gb300 import synth


def _problem(seed, m, n, scale=3.0):
    g = synth.rng(seed)
    A = g.normal(size=(m, m)) + 2.0 * np.eye(m)
    B = g.normal(size=(n, m)) * scale
    return A, B


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_maxvol_result_is_locally_maximal(seed):
    """No single swap of a candidate into the final A raises |det A| by more than (1 + eps)."""
    eps = 1e-3
    A0, B = _problem(seed, 4, 9)
    A, src, ns = AS.maxvol(A0, B, eps)
    d = abs(np.linalg.det(A))
    for i in range(len(B)):
        for j in range(4):
            T = A.copy()
            T[j] = B[i]
            assert abs(np.linalg.det(T)) <= (1 + eps) * d * (1 + 1e-12)
    assert ns > 0
    # the rows of A are the kept rows of A0 and the recorded candidates
    for j in range(4):
        np.testing.assert_array_equal(A[j], A0[j] if src[j] < 0 else B[src[j]])


def test_maxvol_swaps_grow_the_determinant():
    """Each swap multiplies |det A| by more than 1 + eps (determinants recomputed directly)."""
    eps = 1e-3
    A0, B = _problem(7, 5, 12)
    dets = [abs(np.linalg.det(A0))]
    for s in range(1, 40):
        A, _, ns = AS.maxvol(A0, B, eps, max_swaps=s)
        if ns < s:
            break
        dets.append(abs(np.linalg.det(A)))
    assert len(dets) > 2
    assert all(b > (1 + eps) * a for a, b in zip(dets, dets[1:]))


def test_maxvol_reaches_the_best_single_swap_chain_on_tiny_set():
    """m = 2, three candidates: the final |det| is at least that of the best single swap and
    within the brute-force maximum over all reachable sets (row j from A0[j] or any candidate)."""
    A0, B = _problem(11, 2, 3)
    A, _, _ = AS.maxvol(A0, B, 0.0)
    d = abs(np.linalg.det(A))
    best_single = max(abs(np.linalg.det(np.where(np.arange(2)[:, None] == j, B[i], A0)))
                      for i in range(3) for j in range(2))
    assert d >= best_single * (1 - 1e-12)
    rows = [np.vstack([A0[j:j + 1], B]) for j in range(2)]
    brute = max(abs(np.linalg.det(np.array([rows[0][a], rows[1][b]])))
                for a, b in itertools.product(range(4), range(4)))
    assert d <= brute * (1 + 1e-12)


def test_maxvol_no_candidates_or_already_maximal():
    A0, B = _problem(5, 3, 4, scale=0.01)
    A, src, ns = AS.maxvol(A0, B[:0])
    assert ns == 0 and (src < 0).all()
    A, src, ns = AS.maxvol(A0, B)      # tiny candidates never beat the active rows
    assert ns == 0 and np.array_equal(A, A0)

"""Error allowance of the mixed-precision grade (test helper; numpy only).

gamma_i = max_p |(b_i A^-1)_p| (Section II.D).  A componentwise relative perturbation of size e
in every entry of b_i (or of A^-1) moves gamma_i by at most e S_i to first order, with

    S_i = max_p sum_k |b_ik| |(A^-1)_kp|.

The mixed path forms b_i in FP32 (its entries carry a few units in the last place of FP32, more
where the sums that form them cancel) and the product from TF32 pieces; for an active set whose
rows are nearly dependent, S_i / gamma_i reaches 10^3-10^4, so a fixed relative gate on gamma
cannot hold.  The tests allow 1e-4 max(1, gamma_i) plus MIXED_ROW_EPS S_i for every atom, with
MIXED_ROW_EPS = 2^-20 (16 FP32 units in the last place per row entry).
"""
import numpy as np

MIXED_ROW_EPS = 2.0 ** -20


def grade_sensitivity(A, rows):
    """S_i = max_p sum_k |b_ik| |(A^-1)_kp| for every row b_i."""
    X = np.linalg.inv(A)
    return (np.abs(rows) @ np.abs(X)).max(axis=1)


def mixed_grade_bound(gamma, S):
    """Allowed |gamma_mixed - gamma| per atom."""
    return 1e-4 * np.maximum(1.0, gamma) + MIXED_ROW_EPS * S


def mixed_grade_ok(g, gamma, S):
    return np.abs(g - gamma) <= mixed_grade_bound(gamma, S)

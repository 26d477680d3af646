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


# ---------------------------------------------------------------------------------
# configuration-level grades
# ---------------------------------------------------------------------------------

def _small_model_and_batch():
    from oracle import oracle as O
    md = O.OracleModel(2, 8, 2.0, 5.0)
    nu_sum = [sum(nu for _, nu in labs) for labs, _ in md.basis]
    nf = [len(labs) for labs, _ in md.basis]
    theta = synth.draw_theta(41, 2, md.n_rad, md.n_q, nu_sum, nf, 2.0, 5.0, 40.0)
    batch = synth.training_batch(seed=42, n_cfg=3, n_types=2, lo=4, hi=20)
    return O, md, theta, batch


def test_config_rows_are_energy_gradients():
    """b(cfg_k) . d = dE_k/dtheta . d by central differences of the oracle's energies."""
    O, md, theta, batch = _small_model_and_batch()
    nbr = O.batch_neighbors(batch, md.r_cut)
    R = AS.config_rows(md, theta, batch, nbr)
    g = synth.rng(43)
    for _ in range(3):
        d = g.normal(size=theta.size) * np.abs(theta).clip(1e-3)
        h = 1e-4
        Ep = O.efs(md, theta + h * d, batch, nbr)["E"]
        Em = O.efs(md, theta - h * d, batch, nbr)["E"]
        np.testing.assert_allclose(R @ d, (Ep - Em) / (2 * h), rtol=1e-6, atol=1e-9)


def test_config_grade_of_an_active_configuration_is_one():
    """A configuration whose row is in the active set has gamma(cfg) = 1 exactly (its
    coefficients are a unit vector)."""
    g = synth.rng(44)
    A = g.normal(size=(6, 6)) + 3 * np.eye(6)
    gam, am = AS.config_grade(A, A[[2, 4]])
    np.testing.assert_allclose(gam, 1.0, rtol=1e-12)
    assert list(am) == [2, 4]


def test_neighborhood_config_grade_and_classes():
    gam = np.array([0.5, 3.0, 1.2, 11.0, 2.0, 10.0])
    off = np.array([0, 2, 2, 4, 6])
    assert list(AS.neighborhood_config_grade(gam, off)) == [3.0, 0.0, 11.0, 10.0]
    cls = AS.classify(np.array([0.5, 2.0, 2.0000001, 10.0, 10.5]), 2.0, 10.0)
    assert list(cls) == [0, 0, 1, 1, 2]


# ---------------------------------------------------------------------------------
# spherical cut
# ---------------------------------------------------------------------------------

def test_cut_cluster_matches_the_neighbor_list_at_that_radius():
    """The cut at radius R is the center plus its neighbor list at cut-off R (the oracle's
    independent neighbor routine), with the same relative vectors."""
    from oracle import oracle as O
    b = synth.fcc_ternary(seed=61, n=3)      # 10.8 A cell: an 8 A sphere needs images
    for c in (0, 17, 100):
        pos, ty, src = AS.cut_cluster(b, c, 8.0)
        off, _, _, r = O.neighbors(b["pos"], b["cell"][0], b["pbc"][0], 8.0)
        lo, hi = off[c], off[c + 1]
        assert len(src) == 1 + hi - lo
        assert src[0] == c and np.allclose(pos[0], 0)
        got = sorted(map(tuple, np.round(pos[1:], 9)))
        ref = sorted(map(tuple, np.round(r[lo:hi], 9)))
        assert got == ref
        assert (ty == b["type"][src]).all()
        assert np.sqrt((pos ** 2).sum(1)).max() < 8.0


def test_cut_cluster_open_axis():
    """A non-periodic axis takes no images along it."""
    b = synth.fcc_ternary(seed=62, n=3)
    b["pbc"] = np.array([[1, 1, 0]], np.uint8)
    pos, _, src = AS.cut_cluster(b, 40, 8.0)
    full, _, _ = AS.cut_cluster(synth.fcc_ternary(seed=62, n=3), 40, 8.0)
    assert len(src) < len(full)
    H = b["cell"][0]
    z_img = np.round((pos[:, 2] + b["pos"][40, 2] - b["pos"][src, 2]) / H[2, 2])
    assert (z_img == 0).all()

"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: values printed in the
paper (tests/golden/paper_pins.json), closed forms, invariances, finite differences,
library routines (numpy einsum / linalg / Chebyshev) and brute force on tiny inputs.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

from oracle import basis_ref
from oracle import oracle as O
from paper_2304_13144_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_pins.json")


def theta_for(md, seed, nbar=40.0, kappa=10.0):
    nu_sum = [sum(nu for _, nu in labs) for labs, _ in md.basis]
    nf = [len(labs) for labs, _ in md.basis]
    return synth.draw_theta(seed, md.n_types, md.n_rad, md.n_q, nu_sum, nf, md.r_min, md.r_cut,
                            nbar, kappa)


def small_ternary(seed=7, n=2, a=3.6, sigma=0.12):
    g = synth.rng(seed)
    pos, cell, _ = synth.cubic_supercell(synth._FCC, a, n)
    pos = pos + g.normal(0, sigma, pos.shape)
    types = g.integers(0, 3, len(pos)).astype(np.int32)
    return synth.single(pos, types, cell)


def cluster(centers_seed, n, box=40.0, T=3, rmin_sep=2.1, shift=(0, 0, 0)):
    g = synth.rng(centers_seed)
    pts = []
    while len(pts) < n:
        p = g.uniform(0, 7.0, 3)
        if all(np.linalg.norm(p - q) > rmin_sep for q in pts):
            pts.append(p)
    pos = np.array(pts) + np.array(shift, float) + box / 2 - 3.5
    types = g.integers(0, T, n).astype(np.int32)
    return synth.single(pos, types, np.eye(3) * box, pbc=(0, 0, 0))


def cheb(beta, x):
    c = np.zeros(beta + 1)
    c[beta] = 1.0
    return np.polynomial.chebyshev.chebval(x, c)


# ---------------------------------------------------------------------------------
# values printed in the paper
# ---------------------------------------------------------------------------------

def test_level6_basis_is_the_papers_list():
    pins = json.load(open(GOLDEN))["level6_basis"]
    expect = {(tuple(tuple(l) for l in f["labels"]), tuple(f["edges"])) for f in pins["functions"]}
    got = basis_ref.basis_functions(6)
    assert set(got) == expect and len(got) == pins["n_lin"]
    _, n_rad, _ = basis_ref.shape(1, 6)
    assert n_rad == pins["n_rad"]


def test_unary_parameter_counts_26_54_125():
    pins = json.load(open(GOLDEN))["unary_param_counts"]
    for lev in (8, 12, 16):
        assert basis_ref.shape(1, lev, 8)[2] == pins[str(lev)]


def test_moment_levels():
    pins = json.load(open(GOLDEN))["moment_levels"]
    assert basis_ref.level_of_moment(0, 0) == pins["M00"]
    assert basis_ref.level_of_moment(2, 1) == pins["M21"]
    assert basis_ref.level_of_moment(0, 3) == pins["M03"]


def test_radial_parameter_count():
    for T, lev in ((1, 8), (2, 12), (3, 16)):
        basis, n_rad, m = basis_ref.shape(T, lev, 8)
        assert m - T - len(basis) == 8 * n_rad * T * T


# ---------------------------------------------------------------------------------
# closed forms
# ---------------------------------------------------------------------------------

@pytest.mark.parametrize("beta", [0, 1, 2, 5, 7])
def test_radial_basis_is_chebyshev_times_cutoff(beta):
    """Level 2 is the pair potential V = s + xi sum_j f_0(r_ij); with c = e_beta,
    f_0(r) = T_beta(x) (R_cut - r)^2 (eq. 4), checked against cos(beta arccos x) and,
    below R_min (reading R2, no clamping), against the Chebyshev series of numpy."""
    md = O.OracleModel(1, 2, 2.0, 5.0, n_q=8)
    assert md.n_lin == 1 and md.n_rad == 1
    theta = np.zeros(md.m)
    theta[0] = 0.3
    theta[1] = 1.0
    theta[2 + beta] = 1.0
    for d in (1.7, 2.0, 2.6, 3.3, 4.1, 4.9, 4.999):
        b = synth.single(np.array([[10.0, 10, 10], [10 + d, 10, 10]]), [0, 0], np.eye(3) * 30, (0, 0, 0))
        V = O.efs(md, theta, b)["V"]
        x = (2 * d - 7.0) / 3.0
        t = math.cos(beta * math.acos(x)) if abs(x) <= 1 else cheb(beta, x)
        assert V[0] == pytest.approx(0.3 + t * (5.0 - d) ** 2, rel=1e-13, abs=1e-14)


def test_dimer_closed_form_level12_ternary():
    """For two atoms at distance d every moment is f_mu(d) r^(x)nu and each contracted
    index pair gives r.r = d^2, so B_a = prod_p f_{mu_p}(d) d^{sum nu}."""
    md = O.OracleModel(3, 12, 2.0, 5.0)
    theta = theta_for(md, 5)
    T, nq, nrad = 3, 8, md.n_rad
    c = theta[T + md.n_lin:].reshape(T, T, nrad, nq)
    u = np.array([0.36, -0.48, 0.8])
    for d, (z0, z1) in ((2.7, (0, 2)), (3.9, (1, 1)), (4.6, (2, 0))):
        b = synth.single(np.array([[15.0, 15, 15], 15 + d * u]), [z0, z1], np.eye(3) * 40, (0, 0, 0))
        V = O.efs(md, theta, b)["V"][0]
        x = (2 * d - 7.0) / 3.0
        Q = np.array([cheb(k, x) for k in range(nq)]) * (5.0 - d) ** 2
        f = c[z0, z1] @ Q
        expect = theta[z0]
        for a, (labs, _) in enumerate(md.basis):
            expect += theta[T + a] * np.prod([f[mu] for mu, _ in labs]) * d ** sum(nu for _, nu in labs)
        assert V == pytest.approx(expect, rel=1e-12)


def _einsum_basis(labs, edges, tensors):
    P = len(labs)
    pairs = [(i, j) for i in range(P) for j in range(P) if i < j]
    letters = iter("abcdefghijklmnopqrstuvwxyzABCDEFGHIJ")
    subs = [""] * P
    for (i, j), e in zip(pairs, edges):
        for _ in range(e):
            ch = next(letters)
            subs[i] += ch
            subs[j] += ch
    return np.einsum(",".join(subs) + "->", *[tensors[l] for l in labs])


@pytest.mark.parametrize("lev", [12, 16])
def test_contractions_match_einsum_on_full_tensors(lev):
    """Brute-force cross-check: every basis value of the oracle equals numpy einsum over
    full moment tensors built by outer products (a library contraction)."""
    md = O.OracleModel(3, lev, 2.0, 5.0)
    theta = theta_for(md, 9)
    g = synth.rng(lev)
    n_nb = 7
    dirs = g.normal(size=(n_nb, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    rv = dirs * g.uniform(2.2, 4.8, (n_nb, 1))
    types = g.integers(0, 3, n_nb + 1).astype(np.int32)
    nbr = {"off": np.array([0, n_nb] + [n_nb] * n_nb, np.int64), "j": np.arange(1, n_nb + 1, dtype=np.int32),
           "r": rv}
    B = O.sites(md, theta, types, nbr, req=[0], want_dVdr=False, want_b=True)["b"][0, 3:3 + md.n_lin]
    c = theta[3 + md.n_lin:].reshape(3, 3, md.n_rad, 8)
    zi = types[0]
    tens = {}
    for labs, _ in md.basis:
        for mu, nu in labs:
            if (mu, nu) in tens:
                continue
            acc = np.zeros((3,) * nu)
            for j in range(n_nb):
                r = np.linalg.norm(rv[j])
                x = (2 * r - 7.0) / 3.0
                f = c[zi, types[j + 1], mu] @ (np.array([cheb(k, x) for k in range(8)]) * (5 - r) ** 2)
                t = np.array(f)
                for _ in range(nu):
                    t = np.multiply.outer(t, rv[j])
                acc = acc + t
            tens[(mu, nu)] = acc
    ref = np.array([_einsum_basis(labs, e, tens) for labs, e in md.basis])
    np.testing.assert_allclose(B, ref, rtol=1e-11, atol=1e-13 * np.abs(ref).max())


# ---------------------------------------------------------------------------------
# invariances and conservation
# ---------------------------------------------------------------------------------

def _rotation(seed):
    q, r = np.linalg.qr(synth.rng(seed).normal(size=(3, 3)))
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def test_rotation_translation_permutation_invariance():
    md = O.OracleModel(3, 12, 2.0, 5.0)
    theta = theta_for(md, 3)
    b = small_ternary()
    ref = O.efs(md, theta, b)
    R = _rotation(1)
    br = dict(b, pos=b["pos"] @ R.T, cell=b["cell"] @ R.T)
    rot = O.efs(md, theta, br)
    assert rot["E"][0] == pytest.approx(ref["E"][0], rel=1e-12)
    np.testing.assert_allclose(rot["F"], ref["F"] @ R.T, atol=1e-11 * np.abs(ref["F"]).max())
    np.testing.assert_allclose(rot["W"][0], R @ ref["W"][0] @ R.T, atol=1e-11 * np.abs(ref["W"]).max())
    bt = dict(b, pos=b["pos"] + np.array([1.3, -7.1, 0.4]))
    assert O.efs(md, theta, bt)["E"][0] == pytest.approx(ref["E"][0], rel=1e-12)
    perm = synth.rng(2).permutation(len(b["type"]))
    bp = dict(b, pos=b["pos"][perm], type=b["type"][perm])
    per = O.efs(md, theta, bp)
    assert per["E"][0] == pytest.approx(ref["E"][0], rel=1e-12)
    np.testing.assert_allclose(per["F"], ref["F"][perm], atol=1e-11 * np.abs(ref["F"]).max())


def test_zero_net_force_and_symmetric_virial():
    md = O.OracleModel(3, 12, 2.0, 5.0)
    out = O.efs(md, theta_for(md, 4), small_ternary(seed=11))
    F = out["F"]
    assert np.abs(F.sum(axis=0)).max() <= 1e-12 * np.abs(F).max() * len(F)
    W = out["W"][0]
    np.testing.assert_allclose(W, W.T, atol=1e-11 * np.abs(W).max())


def test_energy_additivity_of_separated_fragments():
    md = O.OracleModel(3, 12, 2.0, 5.0)
    theta = theta_for(md, 6)
    a = cluster(1, 6)
    bb = cluster(2, 6, shift=(15.0, 0, 0))
    both = synth.single(np.concatenate([a["pos"], bb["pos"]]), np.concatenate([a["type"], bb["type"]]),
                        np.eye(3) * 40.0, (0, 0, 0))
    e = O.efs(md, theta, both)["E"][0]
    assert e == pytest.approx(O.efs(md, theta, a)["E"][0] + O.efs(md, theta, bb)["E"][0], rel=1e-13)


# ---------------------------------------------------------------------------------
# derivatives by finite differences
# ---------------------------------------------------------------------------------

def test_forces_are_minus_energy_gradient():
    md = O.OracleModel(3, 12, 2.0, 5.0)
    theta = theta_for(md, 8)
    b = small_ternary(seed=5)
    F = O.efs(md, theta, b)["F"]
    h = 1e-4
    for i in (0, 7, 19):
        for c in range(3):
            bp = dict(b, pos=b["pos"].copy())
            bm = dict(b, pos=b["pos"].copy())
            bp["pos"][i, c] += h
            bm["pos"][i, c] -= h
            fd = -(O.efs(md, theta, bp)["E"][0] - O.efs(md, theta, bm)["E"][0]) / (2 * h)
            assert fd == pytest.approx(F[i, c], abs=1e-7 * max(1.0, np.abs(F).max()))


def test_virial_is_minus_strain_derivative():
    md = O.OracleModel(3, 12, 2.0, 5.0)
    theta = theta_for(md, 12)
    b = small_ternary(seed=6)
    W = O.efs(md, theta, b)["W"][0]
    h = 1e-5
    for a_ in range(3):
        for b_ in range(3):
            e = np.zeros((3, 3))
            e[a_, b_] = h
            D = np.eye(3) + e
            Dm = np.eye(3) - e
            bp = dict(b, pos=b["pos"] @ D.T, cell=b["cell"] @ D.T)
            bm = dict(b, pos=b["pos"] @ Dm.T, cell=b["cell"] @ Dm.T)
            fd = -(O.efs(md, theta, bp)["E"][0] - O.efs(md, theta, bm)["E"][0]) / (2 * h)
            assert fd == pytest.approx(W[a_, b_], abs=1e-6 * max(1.0, np.abs(W).max()))


def test_parameter_rows_are_dV_dtheta():
    md = O.OracleModel(2, 8, 2.0, 5.0)
    theta = theta_for(md, 13)
    b = small_ternary(seed=9)
    b["type"] = b["type"] % 2
    nbr = O.batch_neighbors(b, md.r_cut)
    req = np.array([0, 5, 17])
    rows = O.site_rows(md, theta, b["type"], nbr, req=req)
    for p in range(md.m):
        h = 1e-3 if p < md.n_types + md.n_lin else 1e-5
        tp, tm = theta.copy(), theta.copy()
        tp[p] += h
        tm[p] -= h
        fd = (O.sites(md, tp, b["type"], nbr, req=req, want_dVdr=False)["V"] -
              O.sites(md, tm, b["type"], nbr, req=req, want_dVdr=False)["V"]) / (2 * h)
        tol = 1e-10 if p < md.n_types + md.n_lin else 1e-6
        np.testing.assert_allclose(fd, rows[:, p], rtol=tol, atol=tol * max(1.0, np.abs(rows[:, p]).max()))


def test_loss_gradient_matches_central_differences():
    md = O.OracleModel(2, 6, 2.0, 5.0)
    theta = theta_for(md, 14)
    cfgs = []
    for s in (21, 22):
        c = small_ternary(seed=s, n=(1, 1, 2), sigma=0.1)
        c["type"] = c["type"] % 2
        cfgs.append(c)
    batch = synth.concat(cfgs)
    g = synth.rng(5)
    E_ref = g.normal(size=2)
    F_ref = g.normal(scale=0.1, size=batch["pos"].shape)
    W_ref = g.normal(scale=0.5, size=(2, 3, 3))
    w_e, w_f, w_s = 1.0, 0.01, 0.003
    nbr = O.batch_neighbors(batch, md.r_cut)
    L, grad, _ = O.loss_and_grad(md, theta, batch, E_ref, F_ref, W_ref, w_e, w_f, w_s, nbr=nbr)
    for p in range(md.m):
        h = 1e-4 if p < md.n_types + md.n_lin else 1e-6
        tp, tm = theta.copy(), theta.copy()
        tp[p] += h
        tm[p] -= h
        Lp = O.loss_and_grad(md, tp, batch, E_ref, F_ref, W_ref, w_e, w_f, w_s, nbr=nbr)[0]
        Lm = O.loss_and_grad(md, tm, batch, E_ref, F_ref, W_ref, w_e, w_f, w_s, nbr=nbr)[0]
        assert (Lp - Lm) / (2 * h) == pytest.approx(grad[p], rel=1e-5, abs=1e-7 * max(1.0, np.abs(grad).max()))


# ---------------------------------------------------------------------------------
# grade
# ---------------------------------------------------------------------------------

def test_parameter_rows_annihilate_radial_mixing_directions():
    """V is unchanged when the radial functions are mixed lower-triangularly and xi
    compensates (eqs. 2-4), so b_i . d = 0 for each of the n_rad(n_rad+1)/2 directions;
    a dropped or mis-indexed term in the xi- or c-block of b breaks this."""
    for T, lev in ((1, 8), (3, 12)):
        md = O.OracleModel(T, lev, 2.0, 5.0)
        theta = theta_for(md, 21)
        b = small_ternary(seed=3)
        b["type"] = b["type"] % T
        rows = O.site_rows(md, theta, b["type"], O.batch_neighbors(b, md.r_cut))
        D = O.gauge_directions(md, theta)
        assert D.shape == (md.n_rad * (md.n_rad + 1) // 2, md.m)
        assert np.abs(rows @ D.T).max() <= 1e-13 * np.abs(rows).max() * np.abs(D).max() * md.m


def completed_active_set(rows, D):
    """Active set of len(rows) neighborhoods completed by the null directions (reading R19)."""
    scale = np.abs(rows).max()
    return np.vstack([rows, D / np.linalg.norm(D, axis=1, keepdims=True) * scale])


def test_grade_is_one_on_active_set_rows():
    md = O.OracleModel(1, 8, 2.0, 5.0)
    theta = theta_for(md, 2)
    b = synth.fcc_unary_108(sigma=0.25)
    nbr = O.batch_neighbors(b, md.r_cut)
    rows = O.site_rows(md, theta, b["type"], nbr)
    D = O.gauge_directions(md, theta)
    pick = synth.sample_atoms(3, 108, md.m - len(D))
    A = completed_active_set(rows[pick], D)
    gamma, am = O.grade(A, rows[pick])
    np.testing.assert_allclose(gamma, 1.0, atol=1e-9)
    assert (am == np.arange(len(pick))).all()


def test_grade_matches_numpy_solve_and_inverse():
    m = 40
    A = synth.diag_dominant(5, m)
    brows = synth.rng(6).normal(size=(25, m))
    gamma, am, Ainv = O.grade(A, brows, want_inverse=True)
    C = np.linalg.solve(A.T, brows.T).T
    np.testing.assert_allclose(gamma, np.abs(C).max(axis=1), rtol=1e-12)
    assert (am == np.abs(C).argmax(axis=1)).all()
    assert np.abs(A @ Ainv - np.eye(m)).max() < 1e-12


def test_d_optimality_brute_force():
    """Section II.C: with A the max-|det| choice among the candidate rows (completed by the
    null direction, reading R19), no candidate can raise |det A|: every gamma_i <= 1,
    checked by brute force over all C(8, 3) subsets."""
    md = O.OracleModel(1, 2, 2.0, 5.0, n_q=2)
    assert md.m == 4
    theta = np.array([0.1, 0.7, 0.3, -0.2])
    b = cluster(4, 8, T=1, rmin_sep=1.9)
    nbr = O.batch_neighbors(b, md.r_cut)
    rows = O.site_rows(md, theta, b["type"], nbr)
    D = O.gauge_directions(md, theta)
    assert D.shape == (1, 4)
    best = max(itertools.combinations(range(8), 3),
               key=lambda s: abs(np.linalg.det(completed_active_set(rows[list(s)], D))))
    A = completed_active_set(rows[list(best)], D)
    assert np.linalg.cond(A) < 1e8
    gamma, _ = O.grade(A, rows)
    assert gamma.max() <= 1.0 + 1e-12
    np.testing.assert_allclose(gamma[list(best)], 1.0, atol=1e-12)
    others = [k for k in range(8) if k not in best]
    assert gamma[others].max() < 1.0


# ---------------------------------------------------------------------------------
# neighborhoods
# ---------------------------------------------------------------------------------

def _numpy_neighbors(pos, cell, pbc, rc, K=5):
    out = set()
    n = len(pos)
    rng_ = [range(-K, K + 1) if p else range(0, 1) for p in pbc]
    for i in range(n):
        for n0 in rng_[0]:
            for n1 in rng_[1]:
                for n2 in rng_[2]:
                    sh = n0 * cell[0] + n1 * cell[1] + n2 * cell[2]
                    d = pos + sh - pos[i]
                    r = np.sqrt((d * d).sum(1))
                    for j in np.nonzero((r < rc) & (r > 0))[0]:
                        out.add((i, int(j), n0, n1, n2))
    return out


@pytest.mark.parametrize("pbc", [(1, 1, 1), (1, 1, 0), (0, 0, 0)])
def test_neighbors_against_numpy_brute_force(pbc):
    g = synth.rng(17)
    cell = np.array([[7.1, 0.0, 0.0], [1.9, 6.4, 0.0], [-1.2, 0.8, 6.9]])
    pos = g.uniform(0, 1, (14, 3)) @ cell + g.normal(0, 2.0, (14, 3))
    ref = _numpy_neighbors(pos, cell, pbc, 5.0)
    off, nj, img, r = O.neighbors(pos, cell, pbc, 5.0, brute=True)
    got = {(i, int(nj[p]), *img[p]) for i in range(14) for p in range(off[i], off[i + 1])}
    assert got == ref
    for i in range(14):
        for p in range(off[i], off[i + 1]):
            expect = pos[nj[p]] + img[p] @ cell - pos[i]
            np.testing.assert_allclose(r[p], expect, atol=1e-12)
    if all(pbc):
        off2, nj2, img2, _ = O.neighbors(pos, cell, pbc, 5.0, brute=False)
        got2 = {(i, int(nj2[p]), *img2[p]) for i in range(14) for p in range(off2[i], off2[i + 1])}
        assert got2 == ref

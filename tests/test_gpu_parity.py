"""GPU parity of the CUDA path (through the C ABI) against the FP64 CPU oracle.

Tolerances: FP64 path 1e-10 relative; mixed path 1e-5 eV/A on forces (max abs per component)
and 1e-6 eV/atom on energy (|dE|/N), virial 1e-5 of max|W|, grade |dgamma| <= 1e-4 max(1, gamma).
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2304_13144_gb300 import synth
from nbr_check import check_reverse

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10


@pytest.fixture(scope="module")
def api(native_lib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2304_13144_gb300 import api as A
    return A


def theta_for(md, seed, nbar=40.0, kappa=10.0):
    nu_sum = [sum(nu for _, nu in labs) for labs, _ in md.basis]
    nf = [len(labs) for labs, _ in md.basis]
    return synth.draw_theta(seed, md.n_types, md.n_rad, md.n_q, nu_sum, nf, md.r_min, md.r_cut, nbar, kappa)


def small_cfg(seed, kind, n, T, sigma=0.12, strain=0.02):
    g = synth.rng(seed)
    if kind == "fcc":
        pos, cell, _ = synth.cubic_supercell(synth._FCC, 3.6, n)
    elif kind == "bcc":
        pos, cell, _ = synth.cubic_supercell(synth._BCC, 2.87, n)
    else:
        pos, cell, _ = synth.hcp_supercell(2.55, 2.55 * 1.633, n)
    e = g.uniform(-strain, strain, (3, 3))
    D = np.eye(3) + 0.5 * (e + e.T)
    pos = pos @ D.T + g.normal(0, sigma, pos.shape)
    cell = cell @ D.T
    return synth.single(pos, g.integers(0, T, len(pos)).astype(np.int32), cell)


def run_efs(api, md_desc, theta, batch_np, prec):
    model = api.mtp_load(md_desc, theta)
    b = api.Batch(batch_np)
    nb = api.mtp_build_neighbors(model, b)
    out = api.mtp_energy_forces_stress(model, b, nb, prec)
    torch.cuda.synchronize()
    return model, b, nb, {k: v.cpu().numpy() for k, v in out.items()}


def check_efs(out, ref, n_atoms, prec):
    if prec == "fp64":
        scale_e = max(1.0, np.abs(ref["V"]).sum())
        assert np.abs(out["energy"] - ref["E"]).max() <= FP64_TOL * scale_e
        np.testing.assert_allclose(out["site_energy"], ref["V"], rtol=FP64_TOL, atol=FP64_TOL * np.abs(ref["V"]).max())
        assert np.abs(out["forces"] - ref["F"]).max() <= FP64_TOL * max(1.0, np.abs(ref["F"]).max())
        assert np.abs(out["virial"] - ref["W"]).max() <= FP64_TOL * max(1.0, np.abs(ref["W"]).max())
    else:
        assert np.abs(out["energy"] - ref["E"]).max() / n_atoms <= 1e-6
        assert np.abs(out["forces"] - ref["F"]).max() <= 1e-5
        assert np.abs(out["virial"] - ref["W"]).max() <= 1e-5 * max(1.0, np.abs(ref["W"]).max())


# ---------------------------------------------------------------------------------
# neighborhoods
# ---------------------------------------------------------------------------------

@pytest.mark.parametrize("case", ["fcc108", "triclinic_mixed_pbc", "tiny_cell", "open", "dense_random"])
def test_neighbor_list_matches_oracle(api, case):
    if case == "fcc108":
        bnp = synth.fcc_unary_108()
    elif case == "dense_random":
        # 800 uniform atoms in a 13 A periodic cube: 2 bins per axis, 27 scanned bins per atom and
        # about 2,700 candidates each (the count pass records the first 512 decisions; the fill
        # pass decides the rest again)
        g = synth.rng(18)
        cell = 13.0 * np.eye(3)
        bnp = synth.single(g.uniform(0, 13.0, (800, 3)), np.zeros(800, np.int32), cell)
    elif case == "tiny_cell":
        bnp = small_cfg(3, "bcc", (1, 1, 2), 1)
    else:
        g = synth.rng(17)
        cell = np.array([[7.1, 0.0, 0.0], [1.9, 6.4, 0.0], [-1.2, 0.8, 6.9]])
        pos = g.uniform(0, 1, (30, 3)) @ cell + g.normal(0, 1.0, (30, 3))
        pbc = (1, 1, 0) if case == "triclinic_mixed_pbc" else (0, 0, 0)
        bnp = synth.single(pos, np.zeros(30, np.int32), cell, pbc)
    model = api.mtp_load(api.make_desc(1, 8), np.zeros(26))
    b = api.Batch(bnp)
    nb = api.mtp_build_neighbors(model, b)
    ex = {k: v.cpu().numpy() for k, v in api.mtp_nbr_export(nb, b).items()}
    ref = O.batch_neighbors(bnp, 5.0, brute=True)
    n = len(bnp["type"])
    got = {(i, int(ex["j"][p]), *ex["img"][p]) for i in range(n) for p in range(ex["off"][i], ex["off"][i + 1])}
    want = {(i, int(ref["j"][p]), *ref["img"][p]) for i in range(n) for p in range(ref["off"][i], ref["off"][i + 1])}
    assert got == want
    check_reverse(api, nb, b)


# ---------------------------------------------------------------------------------
# energies, forces, virial
# ---------------------------------------------------------------------------------

@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_efs_fcc108_level8(api, prec):
    bnp = synth.fcc_unary_108()
    md = O.OracleModel(1, 8, 2.0, 5.0)
    theta = theta_for(md, 11)
    ref = O.efs(md, theta, bnp)
    _, _, _, out = run_efs(api, api.make_desc(1, 8), theta, bnp, prec)
    check_efs(out, ref, 108, prec)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("lev", [12, 16])
def test_efs_ternary_batch_uneven_sizes(api, prec, lev):
    cfgs = [small_cfg(1, "fcc", 2, 3), small_cfg(2, "bcc", (2, 2, 3), 3), small_cfg(3, "hcp", (2, 2, 2), 3),
            small_cfg(4, "fcc", (1, 1, 2), 3), small_cfg(5, "bcc", 3, 3)]
    bnp = synth.concat(cfgs)
    md = O.OracleModel(3, lev, 2.0, 5.0)
    theta = theta_for(md, 20 + lev)
    ref = O.efs(md, theta, bnp)
    _, _, _, out = run_efs(api, api.make_desc(3, lev), theta, bnp, prec)
    check_efs(out, ref, len(bnp["type"]), prec)


def test_isolated_atom_and_dimer(api):
    bnp = synth.single(np.array([[5.0, 5, 5], [20.0, 20, 20], [23.1, 20, 20.3]]), [0, 1, 1], np.eye(3) * 40,
                       (0, 0, 0))
    md = O.OracleModel(2, 8, 2.0, 5.0)
    theta = theta_for(md, 3)
    ref = O.efs(md, theta, bnp)
    _, _, nb, out = run_efs(api, api.make_desc(2, 8), theta, bnp, "fp64")
    assert out["site_energy"][0] == pytest.approx(theta[0], rel=1e-14)
    assert np.abs(out["forces"][0]).max() == 0.0
    check_efs(out, ref, 3, "fp64")


def test_forces_are_bitwise_deterministic(api):
    bnp = small_cfg(9, "fcc", 3, 3)
    md = O.OracleModel(3, 12, 2.0, 5.0)
    theta = theta_for(md, 1)
    model = api.mtp_load(api.make_desc(3, 12), theta)
    b = api.Batch(bnp)
    nb = api.mtp_build_neighbors(model, b)
    f1 = api.mtp_energy_forces_stress(model, b, nb, "mixed")["forces"].clone()
    nb2 = api.mtp_build_neighbors(model, b)
    f2 = api.mtp_energy_forces_stress(model, b, nb2, "mixed")["forces"]
    assert torch.equal(f1, f2)


# ---------------------------------------------------------------------------------
# parameter rows and grade
# ---------------------------------------------------------------------------------

def test_param_rows_fp64(api):
    bnp = small_cfg(7, "fcc", 2, 3)
    md = O.OracleModel(3, 12, 2.0, 5.0)
    theta = theta_for(md, 7)
    model = api.mtp_load(api.make_desc(3, 12), theta)
    b = api.Batch(bnp)
    nb = api.mtp_build_neighbors(model, b)
    atoms = torch.tensor([0, 3, 17, 31], dtype=torch.int64)
    rows = api.mtp_param_rows(model, b, nb, "fp64", atoms).cpu().numpy()
    ref = O.site_rows(md, theta, bnp["type"], O.batch_neighbors(bnp, 5.0), req=atoms.numpy())
    np.testing.assert_allclose(rows, ref, rtol=FP64_TOL, atol=FP64_TOL * np.abs(ref).max())
    rows_m = api.mtp_param_rows(model, b, nb, "mixed", atoms).cpu().numpy()
    np.testing.assert_allclose(rows_m, ref, rtol=1e-4, atol=1e-6 * np.abs(ref).max())


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_grade_random_active_set(api, prec):
    bnp = synth.fcc_unary_108(sigma=0.2)
    md = O.OracleModel(1, 8, 2.0, 5.0)
    theta = theta_for(md, 5)
    A = synth.diag_dominant(8, md.m)
    model = api.mtp_load(api.make_desc(1, 8), theta)
    b = api.Batch(bnp)
    nb = api.mtp_build_neighbors(model, b)
    api.mtp_set_active_set(model, torch.tensor(A, device="cuda"))
    out = api.mtp_grade(model, b, nb, prec, threshold=np.inf)
    rows = O.site_rows(md, theta, bnp["type"], O.batch_neighbors(bnp, 5.0))
    gamma, am = O.grade(A, rows)
    g = out["gamma"].cpu().numpy()
    if prec == "fp64":
        np.testing.assert_allclose(g, gamma, rtol=FP64_TOL)
        assert (out["argmax"].cpu().numpy() == am).all()
    else:
        assert np.all(np.abs(g - gamma) <= 1e-4 * np.maximum(1.0, gamma))


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_grade_ternary_batch_every_atom(api, prec):
    """Every atom of a ~250-atom ternary batch: the mixed path stores the rows in species order
    and each 128-row tile skips the K chunks of species it does not hold (here tiles holding
    species {0, 1} and {1, 2}, and the padding chunks past m = 383)."""
    cfgs = [small_cfg(1, "fcc", 2, 3), small_cfg(2, "bcc", (2, 2, 3), 3), small_cfg(3, "hcp", (2, 2, 2), 3),
            small_cfg(4, "fcc", (1, 1, 2), 3), small_cfg(5, "bcc", 3, 3), small_cfg(6, "fcc", 3, 3)]
    bnp = synth.concat(cfgs)
    assert len(bnp["type"]) > 128 and len(set(bnp["type"].tolist())) == 3
    md = O.OracleModel(3, 16, 2.0, 5.0)
    theta = theta_for(md, 31)
    A = synth.diag_dominant(32, md.m)
    model = api.mtp_load(api.make_desc(3, 16), theta)
    b = api.Batch(bnp)
    nb = api.mtp_build_neighbors(model, b)
    api.mtp_set_active_set(model, torch.tensor(A, device="cuda"))
    out = api.mtp_grade(model, b, nb, prec, threshold=np.inf)
    rows = O.site_rows(md, theta, bnp["type"], O.batch_neighbors(bnp, 5.0))
    gamma, am = O.grade(A, rows)
    g = out["gamma"].cpu().numpy()
    if prec == "fp64":
        np.testing.assert_allclose(g, gamma, rtol=FP64_TOL)
        assert (out["argmax"].cpu().numpy() == am).all()
    else:
        assert np.all(np.abs(g - gamma) <= 1e-4 * np.maximum(1.0, gamma))


def test_grade_is_one_on_active_set_and_flags(api):
    """Section II.D: a neighborhood of the active set grades exactly 1.  Random active set
    (m - n_gauge rows of this configuration plus the gauge completion, ill-conditioned): the FP64
    path gives 1 on the active rows and the oracle's flags; the mixed path stays within its
    per-atom allowance (grade_floor.py).  MaxVol active set over the same rows (the oracle's
    swaps): every row grades <= 1 + eps (D-optimality) and the active rows grade 1, the mixed
    path within its allowance."""
    from oracle import active_set as AS
    from grade_floor import grade_sensitivity, mixed_grade_bound, mixed_grade_ok
    bnp = synth.fcc_unary_108(sigma=0.25)
    md = O.OracleModel(1, 8, 2.0, 5.0)
    theta = theta_for(md, 2)
    rows = O.site_rows(md, theta, bnp["type"], O.batch_neighbors(bnp, 5.0))
    D = O.gauge_directions(md, theta)
    pick = synth.sample_atoms(3, 108, md.m - len(D))
    A = np.vstack([rows[pick], D / np.linalg.norm(D, axis=1, keepdims=True) * np.abs(rows).max()])
    model = api.mtp_load(api.make_desc(1, 8), theta)
    b = api.Batch(bnp)
    nb = api.mtp_build_neighbors(model, b)
    api.mtp_set_active_set(model, torch.tensor(A, device="cuda"))
    ref_g, _ = O.grade(A, rows)
    S = grade_sensitivity(A, rows)
    for prec in ("fp64", "mixed"):
        out = api.mtp_grade(model, b, nb, prec, threshold=2.0)
        g = out["gamma"].cpu().numpy()
        if prec == "fp64":
            np.testing.assert_allclose(g[pick], 1.0, atol=1e-8)
        else:
            assert np.all(mixed_grade_ok(g, ref_g, S))
        nf = int(out["n_flagged"].item())
        flagged = out["flagged"].cpu().numpy()[:nf]
        want = np.nonzero(ref_g > 2.0)[0]
        if prec == "fp64":
            assert (flagged == want).all()
        else:
            ambiguous = np.abs(ref_g - 2.0) <= mixed_grade_bound(ref_g, S)
            assert set(flagged) ^ set(want) <= set(np.nonzero(ambiguous)[0])
    eps = 1e-2
    A_mv, src, n_sw = AS.maxvol(A, rows, eps=eps)
    assert n_sw > 0
    active = np.array([pick[j] if src[j] < 0 else src[j] for j in range(len(pick))])
    ref_mv, _ = O.grade(A_mv, rows)
    assert ref_mv.max() <= 1.0 + eps + 1e-9
    S_mv = grade_sensitivity(A_mv, rows)
    api.mtp_set_active_set(model, torch.tensor(A_mv, device="cuda"))
    for prec in ("fp64", "mixed"):
        g = api.mtp_grade(model, b, nb, prec, threshold=2.0)["gamma"].cpu().numpy()
        if prec == "mixed":
            assert np.all(mixed_grade_ok(g, ref_mv, S_mv))
            assert np.all(np.abs(g[active] - 1.0) <= mixed_grade_bound(1.0, S_mv[active]))
        else:
            np.testing.assert_allclose(g[active], 1.0, atol=1e-8)
            np.testing.assert_allclose(g, ref_mv, rtol=1e-8)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_site_virials_match_oracle(api, prec):
    """Per-atom virials W_i = -sum_j (dV_i/dr_ij) (x) r_ij against the oracle's pair gradients;
    they sum to the configuration virial."""
    cfgs = [small_cfg(41, "fcc", 2, 3), small_cfg(42, "hcp", (2, 2, 2), 3)]
    bnp = synth.concat(cfgs)
    md = O.OracleModel(3, 12, 2.0, 5.0)
    theta = theta_for(md, 43)
    ref = O.efs(md, theta, bnp)
    nbr = ref["nbr"]
    cen = O.pair_centers(nbr["off"])
    Wi = np.zeros((len(bnp["type"]), 3, 3))
    np.add.at(Wi, cen, -ref["dVdr"][:, :, None] * nbr["r"][:, None, :])
    model = api.mtp_load(api.make_desc(3, 12), theta)
    b = api.Batch(bnp)
    nb = api.mtp_build_neighbors(model, b)
    out = {k: v.cpu().numpy() for k, v in api.mtp_energy_forces_stress_atoms(model, b, nb, prec).items()}
    tol = FP64_TOL if prec == "fp64" else 1e-5
    assert np.abs(out["site_virial"] - Wi).max() <= tol * np.abs(Wi).max()
    off = bnp["atom_offset"]
    for k in range(len(off) - 1):
        tot = out["site_virial"][off[k]:off[k + 1]].sum(axis=0)
        assert np.abs(tot - out["virial"][k]).max() <= 1e-12 * np.abs(out["virial"][k]).max() + 1e-12


def test_singular_active_set_is_reported(api):
    md_desc = api.make_desc(1, 8)
    model = api.mtp_load(md_desc, np.zeros(26) + 0.01)
    A = np.ones((26, 26))
    with pytest.raises(api.MtpError) as e:
        api.mtp_set_active_set(model, torch.tensor(A, device="cuda"))
    assert e.value.name == "MTP_ERR_SINGULAR"


def test_extract_neighborhoods(api):
    bnp = small_cfg(4, "bcc", 3, 2)
    model = api.mtp_load(api.make_desc(2, 8), np.zeros(75))
    b = api.Batch(bnp)
    nb = api.mtp_build_neighbors(model, b)
    idx = torch.tensor([2, 0, 40], dtype=torch.int32)
    ex = api.mtp_extract_neighborhoods(nb, b, idx)
    ref = O.batch_neighbors(bnp, 5.0, brute=True)
    off = ex["off"].cpu().numpy()
    for k, i in enumerate(idx.tolist()):
        got = sorted(map(tuple, np.round(ex["r"].cpu().numpy()[off[k]:off[k + 1]], 9)))
        want = sorted(map(tuple, np.round(ref["r"][ref["off"][i]:ref["off"][i + 1]], 9)))
        assert got == want
        assert (np.sort(ex["type"].cpu().numpy()[off[k]:off[k + 1]]) ==
                np.sort(bnp["type"][ref["j"][ref["off"][i]:ref["off"][i + 1]]])).all()


def test_input_errors(api):
    model = api.mtp_load(api.make_desc(1, 8), np.zeros(26))
    bad = synth.single(np.array([[0.0, 0, 0], [1.0, 1, 1]]), [0, 3], np.eye(3) * 20, (0, 0, 0))
    with pytest.raises(api.MtpError) as e:
        api.mtp_build_neighbors(model, api.Batch(bad))
    assert e.value.name == "MTP_ERR_ARG"
    same = synth.single(np.array([[1.0, 1, 1], [1.0, 1, 1]]), [0, 0], np.eye(3) * 20, (0, 0, 0))
    with pytest.raises(api.MtpError) as e:
        api.mtp_build_neighbors(model, api.Batch(same))
    assert e.value.name == "MTP_ERR_GEOMETRY"
    with pytest.raises(api.MtpError) as e:
        api.mtp_load(api.make_desc(1, 8), np.zeros(25))
    assert e.value.name == "MTP_ERR_ARG"


# ---------------------------------------------------------------------------------
# training step (eq. 7)
# ---------------------------------------------------------------------------------

@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_train_step_loss_and_gradient(api, prec):
    cfgs = [small_cfg(31, "fcc", (1, 1, 2), 2), small_cfg(32, "bcc", 2, 2), small_cfg(33, "hcp", (2, 1, 2), 2)]
    bnp = synth.concat(cfgs)
    md = O.OracleModel(2, 10, 2.0, 5.0)
    theta = theta_for(md, 40)
    g = synth.rng(41)
    E_ref = g.normal(size=3)
    F_ref = g.normal(scale=0.05, size=bnp["pos"].shape)
    W_ref = g.normal(scale=0.5, size=(3, 3, 3))
    w = (1.0, 0.01, 0.002)
    L_ref, grad_ref, _ = O.loss_and_grad(md, theta, bnp, E_ref, F_ref, W_ref, *w)
    model = api.mtp_load(api.make_desc(2, 10), theta)
    b = api.Batch(bnp)
    nb = api.mtp_build_neighbors(model, b)
    loss, grad = api.mtp_train_step(model, b, nb, torch.tensor(E_ref), torch.tensor(F_ref),
                                    torch.tensor(W_ref.reshape(3, 9)), *w, prec=prec)
    loss = loss.item()
    grad = grad.cpu().numpy()
    tol = FP64_TOL if prec == "fp64" else 1e-5
    assert loss == pytest.approx(L_ref, rel=tol)
    assert np.abs(grad - grad_ref).max() <= tol * 10 * np.abs(grad_ref).max()


# ---------------------------------------------------------------------------------
# the level-20 ternary model of the MD-scale workload, on a small cell
# ---------------------------------------------------------------------------------

@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_efs_and_rows_level20_ternary(api, prec):
    bnp = synth.fcc_ternary(seed=12, n=3)
    md = O.OracleModel(3, 20, 2.0, 5.0)
    theta = theta_for(md, 44, nbar=42.0)
    ref = O.efs(md, theta, bnp)
    model, b, nb, out = run_efs(api, api.make_desc(3, 20), theta, bnp, prec)
    check_efs(out, ref, len(bnp["type"]), prec)
    atoms = torch.tensor([0, 7, 50, 107], dtype=torch.int64)
    rows = api.mtp_param_rows(model, b, nb, prec, atoms).cpu().numpy()
    rref = O.site_rows(md, theta, bnp["type"], ref["nbr"], req=atoms.numpy())
    if prec == "fp64":
        np.testing.assert_allclose(rows, rref, rtol=FP64_TOL, atol=FP64_TOL * np.abs(rref).max())
    else:
        # FP32 rows: each entry within a few FP32 rounding units of the row's scale
        err = np.abs(rows - rref) / np.abs(rref).max(axis=1, keepdims=True)
        assert err.max() < 2e-5, err.max()


@pytest.mark.parametrize("T,lev,n", [(3, 16, 8), (1, 8, 9)])
def test_tensor_core_grade_matches_fp64_path(api, T, lev, n):
    """Many 128-row tiles with a ragged last tile; one or two 224-column passes."""
    bnp = synth.fcc_ternary(seed=21, n=n)
    bnp["type"] = bnp["type"] % T
    md = O.OracleModel(T, lev, 2.0, 5.0)
    theta = theta_for(md, 9)
    model = api.mtp_load(api.make_desc(T, lev), theta)
    b = api.Batch(bnp)
    nb = api.mtp_build_neighbors(model, b)
    api.mtp_set_active_set(model, torch.tensor(synth.diag_dominant(3, md.m), device="cuda"))
    g64 = api.mtp_grade(model, b, nb, "fp64", threshold=1.0)
    gmx = api.mtp_grade(model, b, nb, "mixed", threshold=1.0)
    a, c = g64["gamma"].cpu().numpy(), gmx["gamma"].cpu().numpy()
    assert np.all(np.isfinite(c)) and len(c) == len(bnp["type"])
    assert np.all(np.abs(a - c) <= 1e-4 * np.maximum(1.0, a))
    # argmax agrees wherever the top two entries are well separated (checked on FP64 rows)
    rows = api.mtp_param_rows(model, b, nb, "fp64").cpu().numpy()
    Cf = np.abs(rows @ np.linalg.inv(synth.diag_dominant(3, md.m)))
    top2 = np.sort(Cf, axis=1)[:, -2:]
    clear = (top2[:, 1] - top2[:, 0]) > 1e-3 * top2[:, 1]
    assert (gmx["argmax"].cpu().numpy()[clear] == g64["argmax"].cpu().numpy()[clear]).all()

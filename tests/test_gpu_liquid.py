"""Large-neighborhood workload: quaternary level-24 MTP (m = 1636, N_rad = 6, nu up to 10) on a
liquid-like random-sequential-addition configuration (0.085 atoms/A^3, minimum separation
1.8 A, R_cut = 6 A, about 76 neighbors per atom), GPU through the C ABI vs the FP64 oracle.

* 300-atom periodic cube: every site energy, force, the virial and the parameter rows of a few
  atoms, FP64 and mixed paths.
* the same cube through the three-kernel mixed pass (moments, contraction with the schedule
  read from global memory, pair adjoint): every site energy, force, per-atom virial and grade.
* 2,097,152 atoms (a 32,768-atom cube repeated 4 x 4 x 4, species drawn per atom), the step
  with the grade, through the FP64 path and both mixed passes: site energies, forces and
  grades of sampled atoms, plus zero net force and a symmetric virial.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2304_13144_gb300 import synth

pytestmark = pytest.mark.gpu

R_CUT = 6.0
NBAR = 76.0


@pytest.fixture(scope="module")
def api(native_lib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2304_13144_gb300 import api as A
    return A


@pytest.fixture(scope="module")
def model_l24():
    md = O.OracleModel(4, 24, 2.0, R_CUT)
    nu_sum = [sum(nu for _, nu in labs) for labs, _ in md.basis]
    nf = [len(labs) for labs, _ in md.basis]
    theta = synth.draw_theta(55, 4, md.n_rad, md.n_q, nu_sum, nf, md.r_min, md.r_cut, NBAR)
    return md, theta


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_liquid_300_atoms_every_atom(api, model_l24, prec):
    md, theta = model_l24
    bnp = synth.liquid_rsa(seed=5, n_atoms=300)
    nbr = O.batch_neighbors(bnp, R_CUT)
    ref = O.efs(md, theta, bnp, nbr)
    model = api.mtp_load(api.make_desc(4, 24, r_cut=R_CUT), theta)
    assert model.n_params == 1636
    b = api.Batch(bnp)
    nb = api.mtp_build_neighbors(model, b)
    out = {k: v.cpu().numpy() for k, v in api.mtp_energy_forces_stress(model, b, nb, prec).items()}
    n = len(bnp["type"])
    if prec == "fp64":
        np.testing.assert_allclose(out["site_energy"], ref["V"], rtol=1e-10, atol=1e-10 * np.abs(ref["V"]).max())
        assert np.abs(out["forces"] - ref["F"]).max() <= 1e-10 * np.abs(ref["F"]).max()
        assert np.abs(out["virial"] - ref["W"]).max() <= 1e-10 * np.abs(ref["W"]).max()
    else:
        assert np.abs(out["energy"] - ref["E"]).max() / n <= 1e-6
        assert np.abs(out["forces"] - ref["F"]).max() <= 1e-5
        assert np.abs(out["virial"] - ref["W"]).max() <= 1e-5 * np.abs(ref["W"]).max()
    atoms = np.array([0, 7, 123, 299])
    rows = api.mtp_param_rows(model, b, nb, prec, torch.tensor(atoms)).cpu().numpy()
    ref_rows = O.site_rows(md, theta, bnp["type"], nbr, req=atoms)
    tol = 1e-10 if prec == "fp64" else 1e-5
    assert np.abs(rows - ref_rows).max() <= tol * np.abs(ref_rows).max()


def test_liquid_300_atoms_split_pass(api, model_l24):
    md, theta = model_l24
    bnp = synth.liquid_rsa(seed=5, n_atoms=300)
    nbr = O.batch_neighbors(bnp, R_CUT)
    ref = O.efs(md, theta, bnp, nbr)
    rows = O.site_rows(md, theta, bnp["type"], nbr)
    A = synth.diag_dominant(56, md.m)
    gamma, _ = O.grade(A, rows)
    model = api.mtp_load(api.make_desc(4, 24, r_cut=R_CUT), theta)
    api.mtp_set_active_set(model, torch.tensor(A, device="cuda"))
    b = api.Batch(bnp)
    nb = api.mtp_build_neighbors(model, b)
    n = len(bnp["type"])
    outs = {}
    for p in ("single", "split"):
        api.mtp_set_mixed_pass(model, p)
        assert api.mtp_get_mixed_pass(model)[1] == (2 if p == "split" else 1)
        o = api.mtp_step(model, b, nb, "mixed", threshold=2.0)
        o.update(api.mtp_energy_forces_stress_atoms(model, b, nb, "mixed"))
        out = outs[p] = {k: v.cpu().numpy() for k, v in o.items() if v is not None}
        assert np.abs(out["energy"] - ref["E"]).max() / n <= 1e-6
        assert np.abs(out["site_energy"] - ref["V"]).max() <= 1e-6
        assert np.abs(out["forces"] - ref["F"]).max() <= 1e-5
        assert np.abs(out["virial"] - ref["W"]).max() <= 1e-5 * np.abs(ref["W"]).max()
        assert np.all(np.abs(out["gamma"] - gamma) <= 1e-4 * np.maximum(1.0, gamma))
    a, s2 = outs["single"], outs["split"]
    assert np.abs(a["site_virial"] - s2["site_virial"]).max() <= 1e-5 * np.abs(a["site_virial"]).max()


@pytest.fixture(scope="module")
def big_liquid(api, model_l24):
    md, theta = model_l24
    bnp = synth.liquid_rsa(seed=5, tiles=4)
    A = synth.diag_dominant(9, md.m)
    model = api.mtp_load(api.make_desc(4, 24, r_cut=R_CUT), theta)
    api.mtp_set_active_set(model, torch.tensor(A, device="cuda"))
    b = api.Batch(bnp)
    nb = api.mtp_build_neighbors(model, b)
    outs = {}
    for prec, pas in (("mixed", "single"), ("mixed_split", "split"), ("fp64", "auto")):
        api.mtp_set_mixed_pass(model, pas)
        p = "fp64" if prec == "fp64" else "mixed"
        o = api.mtp_step(model, b, nb, p, threshold=2.0)
        o["site_energy"] = api.mtp_energy_forces_stress(model, b, nb, p)["site_energy"]
        outs[prec] = {k: (v.cpu().numpy() if v is not None else None) for k, v in o.items()}
        del o
        torch.cuda.empty_cache()
    ref_nbr = O.batch_neighbors(bnp, R_CUT, brute=False)
    sample = synth.sample_atoms(321, len(bnp["type"]), 5)
    needed = set(sample.tolist())
    for k in sample:
        needed.update(ref_nbr["j"][ref_nbr["off"][k]:ref_nbr["off"][k + 1]].tolist())
    req = np.array(sorted(needed), np.int64)
    s = O.sites(md, theta, bnp["type"], ref_nbr, req=req, want_dVdr=True, want_b=True)
    pos_of = {int(a): q for q, a in enumerate(req)}
    G = s["dVdr"]
    F = np.zeros((len(sample), 3))
    for q, k in enumerate(sample):
        k = int(k)
        F[q] += G[ref_nbr["off"][k]:ref_nbr["off"][k + 1]].sum(axis=0)
        for j in set(ref_nbr["j"][ref_nbr["off"][k]:ref_nbr["off"][k + 1]].tolist()):
            for p in range(ref_nbr["off"][j], ref_nbr["off"][j + 1]):
                if ref_nbr["j"][p] == k:
                    F[q] -= G[p]
    rows = s["b"][[pos_of[int(k)] for k in sample]]
    gamma, am = O.grade(A, rows)
    V = s["V"][[pos_of[int(k)] for k in sample]]
    return {"outs": outs, "sample": sample, "V": V, "F": F, "gamma": gamma, "argmax": am}


def test_liquid_2m_atoms_sampled(big_liquid):
    big = big_liquid
    k = big["sample"]
    o64 = big["outs"]["fp64"]
    np.testing.assert_allclose(o64["site_energy"][k], big["V"], rtol=1e-10, atol=1e-10 * np.abs(big["V"]).max())
    scale = max(1.0, np.abs(big["F"]).max())
    assert np.abs(o64["forces"][k] - big["F"]).max() <= 1e-10 * scale
    np.testing.assert_allclose(o64["gamma"][k], big["gamma"], rtol=1e-10)
    assert (o64["argmax"][k] == big["argmax"]).all()
    g = big["gamma"]
    for name in ("mixed", "mixed_split"):
        omx = big["outs"][name]
        assert np.abs(omx["site_energy"][k] - big["V"]).max() <= 1e-6, name
        assert np.abs(omx["forces"][k] - big["F"]).max() <= 1e-5, name
        assert np.all(np.abs(omx["gamma"][k] - g) <= 1e-4 * np.maximum(1.0, g)), name
    # the two mixed passes on every atom
    a, s2 = big["outs"]["mixed"], big["outs"]["mixed_split"]
    assert np.abs(a["forces"] - s2["forces"]).max() <= 2e-5
    assert np.abs(a["site_energy"] - s2["site_energy"]).max() <= 2e-6


def test_liquid_2m_atoms_invariants(big_liquid):
    for prec, tol in (("fp64", 1e-9), ("mixed", 1e-3), ("mixed_split", 1e-3)):
        o = big_liquid["outs"][prec]
        F = o["forces"]
        assert np.isfinite(F).all()
        assert np.abs(F.sum(axis=0)).max() <= tol * np.abs(F).max()
        W = o["virial"][0]
        assert np.abs(W - W.T).max() <= (1e-9 if prec == "fp64" else 1e-5) * np.abs(W).max()
        nf = int(o["n_flagged"][0])
        assert (o["flagged"][:nf] == np.nonzero(o["gamma"] > 2.0)[0]).all()

"""MaxVol active-set update (Section II.D) on the GPU through the C ABI vs the oracle."""
import numpy as np
import pytest
import torch

from oracle import active_set as AS
from oracle import oracle as O
from paper_2304_13144_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api(native_lib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2304_13144_gb300 import api as A
    return A


def theta_for(md, seed, nbar=40.0):
    nu_sum = [sum(nu for _, nu in labs) for labs, _ in md.basis]
    nf = [len(labs) for labs, _ in md.basis]
    return synth.draw_theta(seed, md.n_types, md.n_rad, md.n_q, nu_sum, nf, md.r_min, md.r_cut, nbar)


def test_maxvol_random_rows_match_oracle(api):
    """A level-8 unary model only supplies m = 26; the active set and candidates are random."""
    md = O.OracleModel(1, 8, 2.0, 5.0)
    m = md.m
    model = api.mtp_load(api.make_desc(1, 8), theta_for(md, 3))
    g = synth.rng(21)
    A0 = synth.diag_dominant(22, m)
    B = g.normal(size=(300, m)) * np.abs(A0).max() * 0.5
    api.mtp_set_active_set(model, torch.tensor(A0, device="cuda"))
    src, ns = api.mtp_maxvol(model, torch.tensor(B), eps=1e-3)
    A_ref, src_ref, ns_ref = AS.maxvol(A0, B, 1e-3)
    assert ns == ns_ref and ns > 0
    np.testing.assert_array_equal(src.cpu().numpy(), src_ref)
    np.testing.assert_array_equal(api.mtp_get_active_set(model).cpu().numpy(), A_ref)
    Ainv = api.mtp_get_active_inverse(model).cpu().numpy()
    ref_inv = np.linalg.inv(A_ref)
    assert np.abs(Ainv - ref_inv).max() <= 1e-10 * np.abs(ref_inv).max()
    # every candidate now has grade <= 1 + eps against the updated set
    C = B @ ref_inv
    assert np.abs(C).max() <= 1 + 1e-3 + 1e-9


def test_maxvol_on_mtp_rows_then_grade(api):
    """Active set from one snapshot (gauge-completed), candidates = FP64 rows of a hotter
    snapshot; after the update every candidate neighborhood grades <= 1 + eps on the GPU."""
    md = O.OracleModel(2, 10, 2.0, 5.0)
    theta = theta_for(md, 31)
    desc = api.make_desc(2, 10)
    model = api.mtp_load(desc, theta)
    cold = synth.b2_binary(seed=31, n=4, sigma=0.05)
    hot = synth.b2_binary(seed=32, n=4, sigma=0.25)
    bc, bh = api.Batch(cold), api.Batch(hot)
    nc, nh = api.mtp_build_neighbors(model, bc), api.mtp_build_neighbors(model, bh)
    sz = model.model_sizes()
    m, ng = sz["n_params"], sz["n_gauge"]
    pick = torch.tensor(synth.sample_atoms(5, len(cold["type"]), m - ng))
    rows = api.mtp_param_rows(model, bc, nc, "fp64", pick).cpu().numpy()
    D = api.mtp_gauge_directions(desc, theta)
    A0 = np.vstack([rows, D / np.linalg.norm(D, axis=1, keepdims=True) * np.abs(rows).max()])
    api.mtp_set_active_set(model, torch.tensor(A0, device="cuda"))
    Bh = api.mtp_param_rows(model, bh, nh, "fp64")
    src, ns = api.mtp_maxvol(model, Bh, eps=1e-2)
    src = src.cpu().numpy()
    assert ns > 0
    assert (src[m - ng:] < 0).all()        # the gauge rows stay (candidates have no component there)
    # the rows of the new A are the recorded ones, and (oracle arithmetic on the GPU's result)
    # no candidate can raise |det A| by more than 1 + eps
    A = api.mtp_get_active_set(model).cpu().numpy()
    Bn = Bh.cpu().numpy()
    for j in range(m):
        np.testing.assert_array_equal(A[j], A0[j] if src[j] < 0 else Bn[src[j]])
    C = np.linalg.solve(A.T, Bn.T).T
    assert np.abs(C).max() <= 1 + 1e-2 + 1e-4   # slack: cond(A) ~ 1e10 for lattice snapshots
    assert abs(np.linalg.slogdet(A)[1]) >= 0 and np.linalg.slogdet(A)[1] > np.linalg.slogdet(A0)[1]
    # the same greedy sequence as the oracle's (well separated maxima at this size)
    A_ref, src_ref, ns_ref = AS.maxvol(A0, Bn, 1e-2)
    assert ns == ns_ref
    np.testing.assert_array_equal(src, src_ref)
    gam = api.mtp_grade(model, bh, nh, "fp64", threshold=2.0)["gamma"].cpu().numpy()
    assert gam.max() <= 1 + 1e-2 + 1e-4


def test_maxvol_edge_cases(api):
    md = O.OracleModel(1, 8, 2.0, 5.0)
    model = api.mtp_load(api.make_desc(1, 8), theta_for(md, 3))
    m = md.m
    with pytest.raises(api.MtpError):
        api.mtp_maxvol(model, torch.zeros((4, m)))          # no active set yet
    A0 = synth.diag_dominant(23, m)
    api.mtp_set_active_set(model, torch.tensor(A0, device="cuda"))
    src, ns = api.mtp_maxvol(model, torch.zeros((0, m)))
    assert ns == 0 and (src.cpu().numpy() < 0).all()
    src, ns = api.mtp_maxvol(model, torch.tensor(A0[:5] * 0.5))   # dominated candidates
    assert ns == 0
    with pytest.raises(api.MtpError):
        api.mtp_maxvol(model, torch.zeros((4, m)), eps=-1.0)
    src, ns = api.mtp_maxvol(model, torch.tensor(A0 * 3.0), max_swaps=2)
    assert ns == 2

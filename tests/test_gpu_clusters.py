"""Spherical cut of neighborhoods into non-periodic clusters (Section II.E, option (ii)) on the
GPU vs the oracle, and the clusters evaluated as open configurations."""
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


def check_against_oracle(out, bnp, centers, radius):
    off = out["off"].cpu().numpy()
    pos, ty, src = (out[k].cpu().numpy() for k in ("pos", "type", "src"))
    assert off[0] == 0 and off[-1] == len(src)
    for q, c in enumerate(centers):
        rp, rt, rs = AS.cut_cluster(bnp, int(c), radius)
        lo, hi = off[q], off[q + 1]
        np.testing.assert_array_equal(src[lo:hi], rs)
        np.testing.assert_array_equal(ty[lo:hi], rt)
        np.testing.assert_allclose(pos[lo:hi], rp, rtol=0, atol=1e-12)


def test_cut_small_periodic_cell_needs_images(api):
    bnp = synth.fcc_ternary(seed=61, n=3)
    centers = np.array([0, 17, 100, 107])
    out = api.mtp_cut_clusters(api.Batch(bnp), torch.tensor(centers), 8.0)
    check_against_oracle(out, bnp, centers, 8.0)
    assert (np.diff(out["off"].cpu().numpy()) > 150).all()     # 8 A spheres hold ~190 atoms


def test_cut_batch_with_open_axis(api):
    bnp = synth.training_batch(seed=63, n_cfg=5, n_types=3, lo=30, hi=200)
    bnp["pbc"][2] = [1, 1, 0]
    bnp["pbc"][4] = [0, 0, 0]
    off = bnp["atom_offset"]
    centers = np.array([off[0], off[1] + 3, off[2] + 1, off[3], off[4] + 5, off[5] - 1])
    out = api.mtp_cut_clusters(api.Batch(bnp), torch.tensor(centers), 7.5)
    check_against_oracle(out, bnp, centers, 7.5)


def test_cut_worst_atoms_and_evaluate_clusters(api):
    """Workflow: worst atom per configuration (neighborhood-mode grade) -> 8 A cluster ->
    energies and forces of the open clusters, checked against the oracle."""
    md = O.OracleModel(2, 8, 2.0, 5.0)
    nu_sum = [sum(nu for _, nu in labs) for labs, _ in md.basis]
    nf = [len(labs) for labs, _ in md.basis]
    theta = synth.draw_theta(64, 2, md.n_rad, md.n_q, nu_sum, nf, 2.0, 5.0, 40.0)
    model = api.mtp_load(api.make_desc(2, 8), theta)
    bnp = synth.training_batch(seed=65, n_cfg=4, n_types=2, lo=40, hi=120)
    A = synth.diag_dominant(66, md.m)
    api.mtp_set_active_set(model, torch.tensor(A, device="cuda"))
    b = api.Batch(bnp)
    nb = api.mtp_build_neighbors(model, b)
    worst = api.mtp_config_grade(model, b, nb, "fp64", "neighborhood")["worst"]
    cut = api.mtp_cut_clusters(b, worst, 8.0)
    check_against_oracle(cut, bnp, worst.cpu().numpy(), 8.0)
    off = cut["off"].cpu().numpy()
    pos, ty = cut["pos"].cpu().numpy(), cut["type"].cpu().numpy()
    L = 2 * 8.0 + 2 * 5.0 + 1.0   # open box: no image within reach
    clusters = synth.concat([synth.single(pos[off[q]:off[q + 1]], ty[off[q]:off[q + 1]], np.eye(3) * L,
                                          pbc=(0, 0, 0)) for q in range(len(off) - 1)])
    ref = O.efs(md, theta, clusters)
    bc = api.Batch(clusters)
    nc = api.mtp_build_neighbors(model, bc)
    got = {k: v.cpu().numpy() for k, v in api.mtp_energy_forces_stress(model, bc, nc, "fp64").items()}
    np.testing.assert_allclose(got["energy"], ref["E"], rtol=1e-10, atol=1e-10 * np.abs(ref["V"]).sum())
    assert np.abs(got["forces"] - ref["F"]).max() <= 1e-10 * np.abs(ref["F"]).max()


def test_cut_errors(api):
    bnp = synth.fcc_ternary(seed=61, n=3)
    b = api.Batch(bnp)
    with pytest.raises(api.MtpError):
        api.mtp_cut_clusters(b, torch.tensor([len(bnp["type"])]), 8.0)
    with pytest.raises(api.MtpError):
        api.mtp_cut_clusters(b, torch.tensor([0]), 0.0)
    out = api.mtp_cut_clusters(b, torch.tensor([], dtype=torch.int64), 8.0)
    assert out["off"].cpu().numpy().tolist() == [0] and len(out["src"]) == 0

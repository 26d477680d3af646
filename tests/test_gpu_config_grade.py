"""Configuration rows, configuration- and neighborhood-mode configuration grades and the
save/break classes (Sections II.D-II.E) on the GPU vs the oracle."""
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


@pytest.fixture(scope="module")
def setup(api):
    md = O.OracleModel(2, 8, 2.0, 5.0)
    nu_sum = [sum(nu for _, nu in labs) for labs, _ in md.basis]
    nf = [len(labs) for labs, _ in md.basis]
    theta = synth.draw_theta(51, 2, md.n_rad, md.n_q, nu_sum, nf, 2.0, 5.0, 40.0)
    model = api.mtp_load(api.make_desc(2, 8), theta)
    # active set of configurations: m - n_gauge small configurations + the gauge directions
    sz = model.model_sizes()
    m, ng = sz["n_params"], sz["n_gauge"]
    train = synth.training_batch(seed=52, n_cfg=m - ng, n_types=2, lo=8, hi=40)
    rows_train = AS.config_rows(md, theta, train)
    D = O.gauge_directions(md, theta)
    A = np.vstack([rows_train, D / np.linalg.norm(D, axis=1, keepdims=True) * np.abs(rows_train).max()])
    test = synth.training_batch(seed=53, n_cfg=40, n_types=2, lo=8, hi=120)
    return md, theta, model, train, A, test


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_config_rows(api, setup, prec):
    md, theta, model, train, A, test = setup
    b = api.Batch(test)
    nb = api.mtp_build_neighbors(model, b)
    R = api.mtp_config_rows(model, b, nb, prec).cpu().numpy()
    ref = AS.config_rows(md, theta, test)
    tol = 1e-10 if prec == "fp64" else 2e-5
    assert np.abs(R - ref).max() <= tol * np.abs(ref).max()


def test_configuration_mode_grade(api, setup):
    md, theta, model, train, A, test = setup
    api.mtp_set_active_set(model, torch.tensor(A, device="cuda"))
    b = api.Batch(test)
    nb = api.mtp_build_neighbors(model, b)
    out = api.mtp_config_grade(model, b, nb, "fp64", "configuration", 2.0, 10.0)
    g_ref, am_ref = AS.config_grade(A, AS.config_rows(md, theta, test))
    np.testing.assert_allclose(out["gamma"].cpu().numpy(), g_ref, rtol=1e-8)
    assert (out["worst"].cpu().numpy() == am_ref).all()
    assert (out["class"].cpu().numpy() == AS.classify(g_ref, 2.0, 10.0)).all()
    # the active configurations themselves grade 1
    bt = api.Batch(train)
    nt = api.mtp_build_neighbors(model, bt)
    gt = api.mtp_config_grade(model, bt, nt, "fp64", "configuration")["gamma"].cpu().numpy()
    np.testing.assert_allclose(gt, 1.0, rtol=1e-6)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_neighborhood_mode_grade(api, setup, prec):
    md, theta, model, train, A, test = setup
    # neighborhood-mode active set: rows of atoms of the training configurations + gauge rows
    sz = model.model_sizes()
    m, ng = sz["n_params"], sz["n_gauge"]
    rows = O.site_rows(md, theta, train["type"], O.batch_neighbors(train, 5.0))
    # the m - n_gauge most independent atom rows (QR with column pivoting on rows^T)
    import scipy.linalg
    piv = scipy.linalg.qr((rows / np.abs(rows).max(axis=0).clip(1e-300)).T, pivoting=True, mode="r")[1]
    pick = np.sort(piv[:m - ng])
    D = O.gauge_directions(md, theta)
    An = np.vstack([rows[pick], D / np.linalg.norm(D, axis=1, keepdims=True) * np.abs(rows).max()])
    api.mtp_set_active_set(model, torch.tensor(An, device="cuda"))
    b = api.Batch(test)
    nb = api.mtp_build_neighbors(model, b)
    out = api.mtp_config_grade(model, b, nb, prec, "neighborhood", 1.0, 1.5)
    gat, _ = O.grade(An, O.site_rows(md, theta, test["type"], O.batch_neighbors(test, 5.0)))
    g_ref = AS.neighborhood_config_grade(gat, test["atom_offset"])
    rtol = 1e-8 if prec == "fp64" else 1e-3
    np.testing.assert_allclose(out["gamma"].cpu().numpy(), g_ref, rtol=rtol)
    worst = out["worst"].cpu().numpy()
    off = test["atom_offset"]
    for k in range(len(off) - 1):
        assert off[k] <= worst[k] < off[k + 1]
        if prec == "fp64":
            assert worst[k] == off[k] + int(np.argmax(gat[off[k]:off[k + 1]]))
    if prec == "fp64":
        cls = out["class"].cpu().numpy()
        assert (cls == AS.classify(g_ref, 1.0, 1.5)).all() and set(cls.tolist()) == {0, 1, 2}

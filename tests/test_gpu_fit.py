"""BFGS fitting driver around the training step and the fitting-error report (Section II.B)
on the GPU vs the oracle's driver on the oracle's loss."""
import numpy as np
import pytest
import torch

from oracle import fit as FIT
from oracle import oracle as O
from paper_2304_13144_gb300 import synth

pytestmark = pytest.mark.gpu

W = (1.0, 0.01, 0.001)


@pytest.fixture(scope="module")
def api(native_lib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2304_13144_gb300 import api as A
    return A


@pytest.fixture(scope="module")
def problem():
    """Teacher-student: references from a teacher model, the student a perturbed copy."""
    md = O.OracleModel(2, 8, 2.0, 5.0)
    nu_sum = [sum(nu for _, nu in labs) for labs, _ in md.basis]
    nf = [len(labs) for labs, _ in md.basis]
    teacher = synth.draw_theta(82, 2, md.n_rad, md.n_q, nu_sum, nf, 2.0, 5.0, 40.0)
    g = synth.rng(83)
    student = teacher * (1.0 + 0.2 * g.normal(size=teacher.size))
    bnp = synth.training_batch(seed=81, n_cfg=6, n_types=2, lo=8, hi=32)
    nbr = O.batch_neighbors(bnp, 5.0)
    ref = O.efs(md, teacher, bnp, nbr)
    return md, teacher, student, bnp, nbr, ref


def test_bfgs_matches_oracle_driver(api, problem):
    md, teacher, student, bnp, nbr, ref = problem
    model = api.mtp_load(api.make_desc(2, 8), student)
    b = api.Batch(bnp)
    nb = api.mtp_build_neighbors(model, b)
    L, it = api.mtp_fit_bfgs(model, b, nb, ref["E"], ref["F"], ref["W"], *W, prec="fp64", max_iter=6, gtol=0.0)
    f = lambda th: O.loss_and_grad(md, th, bnp, ref["E"], ref["F"], ref["W"], *W, nbr=nbr)[:2]
    th_ref, L_ref, it_ref = FIT.bfgs(f, student, max_iter=6, gtol=0.0)
    assert it == it_ref == 6
    assert L == pytest.approx(L_ref, rel=1e-7)
    th = api.mtp_get_params(model)
    assert np.abs(th - th_ref).max() <= 1e-6 * np.abs(th_ref).max()


def test_bfgs_fit_reduces_loss_and_errors(api, problem):
    md, teacher, student, bnp, nbr, ref = problem
    model = api.mtp_load(api.make_desc(2, 8), student)
    b = api.Batch(bnp)
    nb = api.mtp_build_neighbors(model, b)
    e0 = api.mtp_fit_errors(model, b, nb, ref["E"], ref["F"], ref["W"])
    L0 = api.mtp_train_step(model, b, nb, torch.tensor(ref["E"]), torch.tensor(ref["F"]),
                            torch.tensor(ref["W"].reshape(-1, 9)), *W)[0].item()
    for prec in ("mixed", "fp64"):
        L, it = api.mtp_fit_bfgs(model, b, nb, ref["E"], ref["F"], ref["W"], *W, prec=prec, max_iter=60, gtol=1e-10)
        assert it > 5
    assert L < 1e-2 * L0
    e1 = api.mtp_fit_errors(model, b, nb, ref["E"], ref["F"], ref["W"])
    assert e1[2] < 0.2 * e0[2] and e1[5] < 0.2 * e0[5]


def test_fit_errors_match_oracle(api, problem):
    md, teacher, student, bnp, nbr, ref = problem
    model = api.mtp_load(api.make_desc(2, 8), student)
    b = api.Batch(bnp)
    nb = api.mtp_build_neighbors(model, b)
    got = api.mtp_fit_errors(model, b, nb, ref["E"], ref["F"], ref["W"])
    out = O.efs(md, student, bnp, nbr)
    want = FIT.errors(out["E"], out["F"], out["W"], ref["E"], ref["F"], ref["W"], bnp["atom_offset"])
    np.testing.assert_allclose(got, want, rtol=1e-9, atol=1e-14)
    got2 = api.mtp_fit_errors(model, b, nb, ref["E"], ref["F"], None)
    assert (got2[6:] == 0).all() and np.allclose(got2[:6], want[:6], rtol=1e-9)

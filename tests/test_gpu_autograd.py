"""torch.autograd wrappers (MTPEnergy, MTPLoss) against central finite differences of their
own forward passes, and against the oracle's analytic gradient (FP64 path)."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2304_13144_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods(native_lib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2304_13144_gb300 import api as A
    from paper_2304_13144_gb300 import autograd as G
    return A, G


def theta_for(md, seed, nbar=40.0):
    nu_sum = [sum(nu for _, nu in labs) for labs, _ in md.basis]
    nf = [len(labs) for labs, _ in md.basis]
    return synth.draw_theta(seed, md.n_types, md.n_rad, md.n_q, nu_sum, nf, md.r_min, md.r_cut, nbar)


@pytest.fixture(scope="module")
def setup(mods):
    A, G = mods
    bnp = synth.training_batch(seed=71, n_cfg=3, n_types=2, lo=8, hi=40)
    md = O.OracleModel(2, 12, 2.0, 5.0)
    theta = theta_for(md, 72)
    model = A.mtp_load(A.make_desc(2, 12), theta)
    batch = A.Batch(bnp)
    return A, G, bnp, md, theta, model, batch


def test_energy_position_gradient_matches_finite_differences(setup):
    A, G, bnp, md, theta, model, batch = setup
    pos0 = torch.tensor(bnp["pos"], device="cuda", requires_grad=True)
    th = torch.tensor(theta)
    w = torch.tensor([0.7, -1.3, 0.4], device="cuda", dtype=torch.float64)
    E = G.energy(pos0, th, model, batch, "fp64")
    (gpos,) = torch.autograd.grad((w * E).sum(), pos0)
    gpos = gpos.cpu().numpy()
    h = 1e-5
    g = synth.rng(73)
    for a in g.choice(len(bnp["pos"]), 6, replace=False):
        for c in range(3):
            p = bnp["pos"].copy()
            p[a, c] += h
            Ep = (w * G.energy(torch.tensor(p, device="cuda"), th, model, batch, "fp64")).sum().item()
            p[a, c] -= 2 * h
            Em = (w * G.energy(torch.tensor(p, device="cuda"), th, model, batch, "fp64")).sum().item()
            fd = (Ep - Em) / (2 * h)
            assert abs(gpos[a, c] - fd) <= 1e-6 * max(1.0, abs(fd))
    # the FP64 gradient is the oracle's -F
    ref = O.efs(md, theta, bnp)
    cfg = np.repeat(np.arange(3), np.diff(bnp["atom_offset"]))
    np.testing.assert_allclose(gpos, -ref["F"] * w.cpu().numpy()[cfg][:, None], rtol=1e-9,
                               atol=1e-10 * np.abs(ref["F"]).max())


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_energy_theta_gradient_is_sum_of_rows(setup, prec):
    A, G, bnp, md, theta, model, batch = setup
    th = torch.tensor(theta, requires_grad=True)
    pos = torch.tensor(bnp["pos"], device="cuda")
    E = G.energy(pos, th, model, batch, prec)
    (gth,) = torch.autograd.grad(E.sum(), th)
    rows = O.site_rows(md, theta, bnp["type"], O.batch_neighbors(bnp, md.r_cut))
    tol = 1e-10 if prec == "fp64" else 1e-5
    np.testing.assert_allclose(gth.numpy(), rows.sum(axis=0), rtol=tol, atol=tol * np.abs(rows).sum(axis=0).max())


def test_energy_theta_gradient_matches_finite_differences(setup):
    A, G, bnp, md, theta, model, batch = setup
    th = torch.tensor(theta, requires_grad=True)
    pos = torch.tensor(bnp["pos"], device="cuda")
    E = G.energy(pos, th, model, batch, "fp64")
    (gth,) = torch.autograd.grad(E.sum(), th)
    g = synth.rng(74)
    for _ in range(4):
        d = g.normal(size=theta.size) * np.abs(theta).clip(1e-3)
        h = 1e-4
        Ep = G.energy(pos, torch.tensor(theta + h * d), model, batch, "fp64").sum().item()
        Em = G.energy(pos, torch.tensor(theta - h * d), model, batch, "fp64").sum().item()
        fd = (Ep - Em) / (2 * h)
        an = float(gth.numpy() @ d)
        assert abs(an - fd) <= 1e-6 * max(1.0, abs(fd))


def test_loss_gradient_and_descent(setup):
    A, G, bnp, md, theta, model, batch = setup
    nb = A.mtp_build_neighbors(model, batch)
    g = synth.rng(75)
    E_ref = torch.tensor(g.normal(size=3))
    F_ref = torch.tensor(g.normal(scale=0.05, size=bnp["pos"].shape))
    th = torch.tensor(theta, requires_grad=True)
    L = G.loss(th, model, batch, nb, E_ref, F_ref, None, 1.0, 0.01, 0.0, "fp64")
    (gth,) = torch.autograd.grad(L, th)
    L_ref, grad_ref, _ = O.loss_and_grad(md, theta, bnp, E_ref.numpy(), F_ref.numpy(), None, 1.0, 0.01, 0.0)
    assert L.item() == pytest.approx(L_ref, rel=1e-10)
    np.testing.assert_allclose(gth.numpy(), grad_ref, rtol=1e-9, atol=1e-10 * np.abs(grad_ref).max())
    d = g.normal(size=theta.size) * np.abs(theta).clip(1e-3)
    h = 1e-5
    Lp = G.loss(torch.tensor(theta + h * d), model, batch, nb, E_ref, F_ref).item()
    Lm = G.loss(torch.tensor(theta - h * d), model, batch, nb, E_ref, F_ref).item()
    assert float(gth.numpy() @ d) == pytest.approx((Lp - Lm) / (2 * h), rel=1e-5, abs=1e-9)
    # descent with torch.optim on the rescaled parameters u = theta / D (D = |theta|, so that the
    # very different scales of the xi's do not matter): the loss decreases
    D = torch.tensor(np.abs(theta).clip(1e-6))
    u = (torch.tensor(theta) / D).requires_grad_(True)
    step = 1e-3 / float((D * gth).abs().max())
    opt = torch.optim.SGD([u], lr=step)
    losses = []
    for _ in range(3):
        opt.zero_grad()
        Lk = G.loss(D * u, model, batch, nb, E_ref, F_ref)
        losses.append(Lk.item())
        Lk.backward()
        opt.step()
    assert losses[0] == pytest.approx(L.item(), rel=1e-10)
    assert losses[2] < losses[1] < losses[0]

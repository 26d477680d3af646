"""The two mixed-precision passes (one kernel per neighborhood; three kernels: moments,
contraction, pair adjoint) against the FP64 oracle and against each other, at every level with
a specialised kernel, on ternary batches of several configurations (periodic cells of
different shapes and sizes, ragged pair counts)."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2304_13144_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api(native_lib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2304_13144_gb300 import api as A
    return A


def theta_for(md, seed):
    nu_sum = [sum(nu for _, nu in labs) for labs, _ in md.basis]
    nf = [len(labs) for labs, _ in md.basis]
    return synth.draw_theta(seed, md.n_types, md.n_rad, md.n_q, nu_sum, nf, md.r_min, md.r_cut, 42.0)


def batch(seed):
    g = synth.rng(seed)
    cfgs = []
    for k, (kind, n) in enumerate([("fcc", 2), ("bcc", (2, 2, 3)), ("hcp", (2, 2, 2)), ("fcc", (1, 1, 2)), ("fcc", 3)]):
        if kind == "fcc":
            pos, cell, _ = synth.cubic_supercell(synth._FCC, 3.6, n)
        elif kind == "bcc":
            pos, cell, _ = synth.cubic_supercell(synth._BCC, 2.87, n)
        else:
            pos, cell, _ = synth.hcp_supercell(2.55, 2.55 * 1.633, n)
        pos = pos + g.normal(0, 0.12, pos.shape)
        cfgs.append(synth.single(pos, g.integers(0, 3, len(pos)).astype(np.int32), cell))
    return synth.concat(cfgs)


@pytest.mark.parametrize("lev", [8, 12, 16, 20])
def test_both_mixed_passes_match_oracle(api, lev):
    bnp = batch(60 + lev)
    md = O.OracleModel(3, lev, 2.0, 5.0)
    theta = theta_for(md, 61 + lev)
    ref = O.efs(md, theta, bnp)
    rows = O.site_rows(md, theta, bnp["type"], ref["nbr"])
    A = synth.diag_dominant(62 + lev, md.m)
    gamma, _ = O.grade(A, rows)
    model = api.mtp_load(api.make_desc(3, lev), theta)
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
        outs[p] = {k: v.cpu().numpy() for k, v in o.items() if v is not None}
        out = outs[p]
        assert np.abs(out["energy"] - ref["E"]).max() / n <= 1e-6
        assert np.abs(out["site_energy"] - ref["V"]).max() <= 1e-6
        assert np.abs(out["forces"] - ref["F"]).max() <= 1e-5
        assert np.abs(out["virial"] - ref["W"]).max() <= 1e-5 * max(1.0, np.abs(ref["W"]).max())
        assert np.all(np.abs(out["gamma"] - gamma) <= 1e-4 * np.maximum(1.0, gamma))
    a, s = outs["single"], outs["split"]
    assert np.abs(a["forces"] - s["forces"]).max() <= 2e-5
    assert np.abs(a["site_virial"] - s["site_virial"]).max() <= 1e-5 * np.abs(a["site_virial"]).max()
    # the contraction's schedule streamed through a shared ring (the block's warps in step) or
    # held in tensor memory instead of shared memory, one and two neighborhoods per warp, two and
    # four words per step: the same words in the same order, so bitwise the same results
    api.mtp_set_mixed_pass(model, "split")
    for sched, nbc, unr in ((2, 1, 2), (2, 2, 2), (3, 1, 2), (3, 2, 2), (3, 2, 4), (3, 2, 8), (1, 2, 8)):
        api.mtp_set_split_shape(model, 8, nbc, unr, sched)
        o = api.mtp_step(model, b, nb, "mixed", threshold=2.0)
        o.update(api.mtp_energy_forces_stress_atoms(model, b, nb, "mixed"))
        assert api.mtp_get_split_shape(model)[4] == sched
        nf = int(s["n_flagged"][0])
        for k, v in o.items():
            if v is not None and k in s:
                got, want = v.cpu().numpy(), s[k]
                if k == "flagged":   # the list is defined up to its count
                    got, want = got[:nf], want[:nf]
                assert np.array_equal(got, want), (sched, nbc, unr, k)
    api.mtp_set_split_shape(model)
    api.mtp_set_mixed_pass(model, "auto")


def test_split_pass_empty_neighborhoods(api):
    """Atoms without neighbors (a dilute open cluster): zero moments, V_i = s_z, zero force."""
    pos = np.array([[0.0, 0.0, 0.0], [20.0, 0.0, 0.0], [0.0, 20.0, 0.0], [2.6, 0.0, 0.0]])
    bnp = synth.single(pos, np.array([0, 1, 2, 1], np.int32), 40.0 * np.eye(3), (0, 0, 0))
    md = O.OracleModel(3, 16, 2.0, 5.0)
    theta = theta_for(md, 74)
    ref = O.efs(md, theta, bnp)
    model = api.mtp_load(api.make_desc(3, 16), theta)
    b = api.Batch(bnp)
    nb = api.mtp_build_neighbors(model, b)
    api.mtp_set_mixed_pass(model, "split")
    out = {k: v.cpu().numpy() for k, v in api.mtp_energy_forces_stress(model, b, nb, "mixed").items()}
    assert np.abs(out["site_energy"] - ref["V"]).max() <= 1e-6
    assert np.abs(out["forces"] - ref["F"]).max() <= 1e-5

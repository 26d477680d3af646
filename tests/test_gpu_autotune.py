"""Autotuner of the per-neighborhood kernel's launch shape: picks a feasible shape, and the
results after tuning are bitwise those of the default shape (each neighborhood is one warp's
work whatever the block shape; sums go through fixed segments)."""
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


@pytest.mark.parametrize("lev,prec", [(20, "mixed"), (16, "mixed"), (12, "fp64")])
def test_autotune_keeps_results(api, lev, prec):
    md = O.OracleModel(3, lev, 2.0, 5.0)
    nu_sum = [sum(nu for _, nu in labs) for labs, _ in md.basis]
    nf = [len(labs) for labs, _ in md.basis]
    theta = synth.draw_theta(101, 3, md.n_rad, md.n_q, nu_sum, nf, 2.0, 5.0, 42.0)
    model = api.mtp_load(api.make_desc(3, lev), theta)
    api.mtp_set_active_set(model, torch.tensor(synth.diag_dominant(102, md.m), device="cuda"))
    b = api.Batch(synth.fcc_ternary(seed=103, n=12))
    nb = api.mtp_build_neighbors(model, b)
    before = {k: v.clone() for k, v in api.mtp_step(model, b, nb, prec).items() if v is not None}
    w, ms = api.mtp_autotune(model, b, nb, prec)
    assert 1 <= w <= 8 and ms > 0
    after = api.mtp_step(model, b, nb, prec)
    for k, v in before.items():
        assert torch.equal(after[k], v), k

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
    # untuned results of each mixed pass (the autotuner may pick either)
    before = {}
    for p in ((1, 2) if prec == "mixed" else (0,)):
        if p:
            api.mtp_set_mixed_pass(model, p)
        before[p] = {k: v.clone() for k, v in api.mtp_step(model, b, nb, prec).items() if v is not None}
    api.mtp_set_mixed_pass(model, "auto")
    w, ms = api.mtp_autotune(model, b, nb, prec)
    assert 1 <= w <= 8 and ms > 0
    in_use = api.mtp_get_mixed_pass(model)[1] if prec == "mixed" else 0
    after = api.mtp_step(model, b, nb, prec)
    for k, v in before[in_use].items():
        assert torch.equal(after[k], v), k


def test_autotune_of_one_precision_keeps_the_other(api):
    """Tuning the FP64 (generic) kernel after the mixed one leaves the mixed shape in place."""
    md = O.OracleModel(3, 20, 2.0, 5.0)
    nu_sum = [sum(nu for _, nu in labs) for labs, _ in md.basis]
    nf = [len(labs) for labs, _ in md.basis]
    theta = synth.draw_theta(104, 3, md.n_rad, md.n_q, nu_sum, nf, 2.0, 5.0, 42.0)
    model = api.mtp_load(api.make_desc(3, 20), theta)
    b = api.Batch(synth.fcc_ternary(seed=105, n=10))
    nb = api.mtp_build_neighbors(model, b)
    assert api.mtp_get_launch_shape(model) == (0, -1, 0)
    w_mixed, _ = api.mtp_autotune(model, b, nb, "mixed")
    fast, fwd, gen = api.mtp_get_launch_shape(model)
    assert fast == w_mixed and fwd in (0, 1) and gen == 0
    w_fp64, _ = api.mtp_autotune(model, b, nb, "fp64")
    assert api.mtp_get_launch_shape(model) == (fast, fwd, w_fp64)
    api.mtp_autotune(model, b, nb, "mixed")
    assert api.mtp_get_launch_shape(model)[2] == w_fp64


def test_measured_peaks_are_plausible(api):
    """The library's microbenchmarks (the roofline denominators): FP32 FMA between a third of
    and just above 152 SMs x 128 lanes x 2 flops at 2.07 GHz; FP64 well below FP32; the TF32
    tensor-core rate between a quarter of and just above its nominal dense figure."""
    fp32, _ = api.mtp_measure_peak("fp32_fma")
    fp64, _ = api.mtp_measure_peak("fp64_fma")
    tf32, _ = api.mtp_measure_peak("tf32_mma")
    nominal32 = 152 * 128 * 2 * 2.07e9 / 1e12
    assert nominal32 / 3 < fp32 < nominal32 * 1.05
    assert 0 < fp64 < fp32
    assert 1100.0 / 4 < tf32 < 1100.0 * 1.3

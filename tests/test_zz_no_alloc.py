"""The allocation-free energy/force/virial entry point against the allocating one.

Callers that may not allocate device memory at call time (an engine that owns the whole
device-memory budget, or a time-step loop that cannot afford an allocation) use
mtp_energy_forces_stress_noalloc; its scratch is a fixed array inside the library.  This file
is collected last so that a failure here comes after every other test has run; it passes both
alone in a fresh process and after the rest of the suite.
"""
import numpy as np
import pytest
import torch

from paper_2304_13144_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api(native_lib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2304_13144_gb300 import api as A
    return A


def _model(api, T, lev, seed):
    desc = api.make_desc(T, lev)
    basis = api.mtp_describe_basis(desc)
    sz = api.mtp_describe(desc)
    theta = synth.draw_theta(seed, T, sz["n_rad"], 8, [sum(n for _, n in l) for l, _ in basis],
                             [len(l) for l, _ in basis], 2.0, 5.0, 42.0)
    return api.mtp_load(desc, theta)


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_no_alloc_matches_allocating_entry_point_twice(api, prec):
    model = _model(api, 3, 16, 5)
    bnp = synth.concat([synth.fcc_ternary(seed=31, n=4), synth.fcc_ternary(seed=32, n=3)])
    b = api.Batch(bnp)
    nb = api.mtp_build_neighbors(model, b)
    ref = {k: v.cpu().numpy() for k, v in api.mtp_energy_forces_stress(model, b, nb, prec).items()}
    n = len(bnp["type"])
    for _ in range(2):
        out = {k: v.cpu().numpy() for k, v in api.mtp_energy_forces_stress_noalloc(model, b, nb, prec).items()}
        if prec == "fp64":
            tol = 1e-10
            assert np.abs(out["energy"] - ref["energy"]).max() <= tol * max(1.0, np.abs(ref["site_energy"]).sum())
            assert np.abs(out["forces"] - ref["forces"]).max() <= tol * max(1.0, np.abs(ref["forces"]).max())
            assert np.abs(out["virial"] - ref["virial"]).max() <= tol * max(1.0, np.abs(ref["virial"]).max())
        else:
            assert np.abs(out["energy"] - ref["energy"]).max() / n <= 1e-6
            assert np.abs(out["forces"] - ref["forces"]).max() <= 1e-5
            assert np.abs(out["virial"] - ref["virial"]).max() <= 1e-5 * max(1.0, np.abs(ref["virial"]).max())
        np.testing.assert_allclose(out["site_energy"], ref["site_energy"], rtol=1e-6, atol=1e-9)


def test_no_alloc_rejects_systems_beyond_its_fixed_scratch(api):
    model = _model(api, 3, 8, 6)
    bnp = synth.fcc_ternary(seed=33, n=21)      # 37,044 atoms > 32,768
    b = api.Batch(bnp)
    nb = api.mtp_build_neighbors(model, b)
    with pytest.raises(api.MtpError) as e:
        api.mtp_energy_forces_stress_noalloc(model, b, nb, "mixed")
    assert e.value.name == "MTP_ERR_CAPACITY"
    assert "32768" in str(e.value)

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
        # the allocating entry point may run the three-kernel mixed pass, this one always runs
        # the single kernel: mixed results agree to the mixed path's energy tolerance
        if prec == "fp64":
            np.testing.assert_allclose(out["site_energy"], ref["site_energy"], rtol=1e-10, atol=1e-12)
        else:
            assert np.abs(out["site_energy"] - ref["site_energy"]).max() <= 1e-6


@pytest.mark.parametrize("want", [("forces",), ("energy", "virial")])
def test_no_alloc_with_some_outputs_null(api, want):
    """Outputs left NULL: without site energies they go to the internal slot of the array, and
    without forces the force gather is skipped."""
    model = _model(api, 3, 16, 7)
    bnp = synth.concat([synth.fcc_ternary(seed=34, n=3), synth.fcc_ternary(seed=35, n=4)])
    b = api.Batch(bnp)
    nb = api.mtp_build_neighbors(model, b)
    ref = {k: v.cpu().numpy() for k, v in api.mtp_energy_forces_stress(model, b, nb, "mixed").items()}
    n = len(bnp["type"])
    for _ in range(2):
        out = api.mtp_energy_forces_stress_noalloc(model, b, nb, "mixed", want=want)
        for k in ("energy", "site_energy", "forces", "virial"):
            assert (out[k] is None) == (k not in want)
        if "forces" in want:
            assert np.abs(out["forces"].cpu().numpy() - ref["forces"]).max() <= 1e-5
        if "energy" in want:
            assert np.abs(out["energy"].cpu().numpy() - ref["energy"]).max() / n <= 1e-6
            W = out["virial"].cpu().numpy()
            assert np.abs(W - ref["virial"]).max() <= 1e-5 * max(1.0, np.abs(ref["virial"]).max())


def test_no_alloc_first_call_takes_no_device_memory(api):
    """mtp_load commits the fixed scratch array, so the first allocation-free call on a freshly
    loaded model leaves the device's free memory unchanged.  An earlier allocating call on
    another model has loaded the kernels' code (the runtime loads code at first launch)."""
    bnp = synth.fcc_ternary(seed=36, n=4)
    warm = _model(api, 3, 16, 8)
    b = api.Batch(bnp)
    nb = api.mtp_build_neighbors(warm, b)
    api.mtp_energy_forces_stress(warm, b, nb, "mixed")
    api.mtp_energy_forces_stress(warm, b, nb, "fp64")
    model = _model(api, 3, 16, 9)
    N, K = b.n_atoms, b.n_cfg
    outs = [torch.empty(K, dtype=torch.float64, device="cuda"), torch.empty(N, dtype=torch.float64, device="cuda"),
            torch.empty((N, 3), dtype=torch.float64, device="cuda"),
            torch.empty((K, 3, 3), dtype=torch.float64, device="cuda")]
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    for prec in (api.MTP_MIXED, api.MTP_FP64):
        api._check(api.lib().mtp_energy_forces_stress_noalloc(model.h, api.ctypes.byref(b.c), nb.h, prec,
                                                               *[api._ptr(t) for t in outs], api._stream()))
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0


def test_no_alloc_rejects_systems_beyond_its_fixed_scratch(api):
    model = _model(api, 3, 8, 6)
    bnp = synth.fcc_ternary(seed=33, n=21)      # 37,044 atoms > 32,768
    b = api.Batch(bnp)
    nb = api.mtp_build_neighbors(model, b)
    with pytest.raises(api.MtpError) as e:
        api.mtp_energy_forces_stress_noalloc(model, b, nb, "mixed")
    assert e.value.name == "MTP_ERR_CAPACITY"
    assert "32768" in str(e.value) and "segments" in str(e.value)

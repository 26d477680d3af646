"""Failure paths exercised without a GPU fault (host-side injection: a failed workspace
allocation, a neighbor fill that overflows its count, tensor-core grade waits that expire) and
checkpoint save/restore of a model."""
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
    yield A
    A.mtp_debug_inject(A.MTP_FAULT_DEVICE_ALLOC, 0)
    A.mtp_debug_inject(A.MTP_FAULT_NEIGHBOR_OVERFLOW, 0)
    A.mtp_debug_inject(A.MTP_FAULT_GRADE_WAIT, 0)


def make(api, lev=12, seed=111):
    md = O.OracleModel(3, lev, 2.0, 5.0)
    nu_sum = [sum(nu for _, nu in labs) for labs, _ in md.basis]
    nf = [len(labs) for labs, _ in md.basis]
    theta = synth.draw_theta(seed, 3, md.n_rad, md.n_q, nu_sum, nf, 2.0, 5.0, 42.0)
    return md, theta, api.mtp_load(api.make_desc(3, lev), theta)


def test_injected_allocation_failure_is_reported_and_recovers(api):
    md, theta, model = make(api)
    b = api.Batch(synth.fcc_ternary(seed=112, n=4))
    nb = api.mtp_build_neighbors(model, b)
    api.mtp_debug_inject(api.MTP_FAULT_DEVICE_ALLOC, 1)
    # the allocation-free entry point runs on its fixed scratch: the armed fault is not consumed
    free = api.mtp_energy_forces_stress_noalloc(model, b, nb, "mixed")
    with pytest.raises(api.MtpError) as e:
        api.mtp_energy_forces_stress(model, b, nb, "mixed")     # first call sizes its workspaces
    assert e.value.name == "MTP_ERR_CUDA" and "injected" in str(e.value)
    out = api.mtp_energy_forces_stress(model, b, nb, "mixed")  # the next call succeeds
    # the allocating entry point may run the three-kernel mixed pass, the allocation-free one the
    # single kernel: they agree to the mixed path's tolerances
    torch.testing.assert_close(out["forces"], free["forces"], rtol=0, atol=1e-5)
    torch.testing.assert_close(out["energy"], free["energy"], rtol=0, atol=1e-6 * b.n_atoms)


def test_expired_grade_waits_take_the_abort_path(api):
    """With one try per wait the tensor-core grade's first unsatisfied wait expires: the kernel
    stops, drains its own copies and MMAs, frees tensor memory and returns; the grades it did not
    finish are NaN and mtp_sync reports MTP_ERR_TIMEOUT.  The next call is unaffected."""
    md, theta, model = make(api, lev=16, seed=114)
    bnp = synth.fcc_ternary(seed=115, n=4)           # 256 atoms: two 128-row tiles
    b = api.Batch(bnp)
    nb = api.mtp_build_neighbors(model, b)
    api.mtp_set_active_set(model, torch.tensor(synth.diag_dominant(5, md.m), device="cuda"))
    ref = api.mtp_grade(model, b, nb, "mixed", threshold=2.0)["gamma"].clone()
    api.mtp_sync(model)
    assert torch.isfinite(ref).all()
    api.mtp_debug_inject(api.MTP_FAULT_GRADE_WAIT, 1)
    out = api.mtp_grade(model, b, nb, "mixed", threshold=2.0)
    with pytest.raises(api.MtpError) as e:
        api.mtp_sync(model)
    assert e.value.name == "MTP_ERR_TIMEOUT"
    g = out["gamma"]
    nan = torch.isnan(g)
    assert nan.any()
    assert torch.equal(g[~nan], ref[~nan])           # what finished is exact
    assert int(out["n_flagged"].item()) == int((g[~nan] > 2.0).sum().item())   # NaN is never flagged
    again = api.mtp_grade(model, b, nb, "mixed", threshold=2.0)["gamma"]
    api.mtp_sync(model)                               # latch cleared, no new error
    assert torch.equal(again, ref)


def test_injected_neighbor_overflow_is_retried_then_reported(api):
    md, theta, model = make(api)
    bnp = synth.fcc_ternary(seed=113, n=4)
    b = api.Batch(bnp)
    clean = api.mtp_nbr_export(api.mtp_build_neighbors(model, b), b)
    api.mtp_debug_inject(api.MTP_FAULT_NEIGHBOR_OVERFLOW, 1)
    retried = api.mtp_nbr_export(api.mtp_build_neighbors(model, b), b)   # one overflow: refilled
    for k in ("off", "j", "img"):
        assert torch.equal(retried[k], clean[k]), k
    api.mtp_debug_inject(api.MTP_FAULT_NEIGHBOR_OVERFLOW, 2)
    with pytest.raises(api.MtpError) as e:
        api.mtp_build_neighbors(model, b)
    assert e.value.name == "MTP_ERR_CAPACITY"
    again = api.mtp_nbr_export(api.mtp_build_neighbors(model, b), b)     # usable afterwards
    assert torch.equal(again["j"], clean["j"])


def test_checkpoint_round_trip(api):
    md, theta, model = make(api, lev=16, seed=114)
    A = synth.diag_dominant(115, md.m)
    api.mtp_set_active_set(model, torch.tensor(A, device="cuda"))
    blob = api.mtp_save(model)
    twin = api.mtp_restore(blob)
    np.testing.assert_array_equal(api.mtp_get_params(twin), theta)
    np.testing.assert_array_equal(api.mtp_get_active_set(twin).cpu().numpy(), A)
    b = api.Batch(synth.fcc_ternary(seed=116, n=5))
    nb = api.mtp_build_neighbors(model, b)
    nt = api.mtp_build_neighbors(twin, b)
    for prec in ("mixed", "fp64"):
        x = api.mtp_step(model, b, nb, prec)
        y = api.mtp_step(twin, b, nt, prec)
        for k, v in x.items():
            if v is not None:
                assert torch.equal(v, y[k]), (prec, k)
    # without an active set; and damaged buffers are refused
    md2, th2, plain = make(api, lev=12, seed=117)
    twin2 = api.mtp_restore(api.mtp_save(plain))
    with pytest.raises(api.MtpError):
        api.mtp_get_active_set(twin2)
    with pytest.raises(api.MtpError):
        api.mtp_restore(blob[: len(blob) // 2])
    with pytest.raises(api.MtpError):
        api.mtp_restore(b"XXXX" + blob[4:])

"""Host-side basis enumeration and contraction schedule of the library (through the C ABI,
host-only calls) against the oracle's independent enumeration and full-tensor evaluation."""
import numpy as np
import pytest

from oracle import basis_ref
from oracle import oracle as O
from paper_2304_13144_gb300 import synth


@pytest.fixture(scope="module")
def api(native_lib):
    from paper_2304_13144_gb300 import api as A
    return A


@pytest.mark.parametrize("lev", [2, 4, 6, 8, 10, 12, 14, 16, 18])
def test_enumerations_agree_in_canonical_order(api, lev):
    lib_basis = api.mtp_describe_basis(api.make_desc(1, lev))
    assert lib_basis == basis_ref.basis_functions(lev)


@pytest.mark.parametrize("T,lev,m", [(1, 8, 26), (1, 12, 54), (1, 16, 125), (2, 16, 222),
                                     (3, 16, 383), (3, 20, 651), (4, 24, 1636)])
def test_parameter_counts(api, T, lev, m):
    sz = api.mtp_describe(api.make_desc(T, lev))
    assert sz["n_params"] == m
    assert sz["n_gauge"] == sz["n_rad"] * (sz["n_rad"] + 1) // 2


def test_descriptor_validation(api):
    with pytest.raises(api.MtpError) as e:
        api.mtp_describe(api.make_desc(0, 8))
    assert e.value.name == "MTP_ERR_ARG"
    with pytest.raises(api.MtpError):
        api.mtp_describe(api.make_desc(1, 8, r_min=5.0, r_cut=4.0))


def _eval_schedule(sch, rv, f):
    """Evaluate the exported flattened triple list in float64 (numpy) for one neighborhood."""
    nm = sch["sizes"]["n_mom_comps"]
    nv = sch["sizes"]["n_values"]
    vals = np.zeros(nv)
    for k in range(nm):
        a, b, c = sch["comp_exp"][k]
        vals[k] = np.sum(f[:, sch["comp_mu"][k]] * rv[:, 0] ** a * rv[:, 1] ** b * rv[:, 2] ** c)
    dp = sch["dst_ptr"]
    for d in range(nv - nm):
        t = slice(dp[d], dp[d + 1])
        vals[nm + d] = np.sum(sch["tri_c"][t] * vals[sch["tri_a"][t]] * vals[sch["tri_b"][t]])
    return vals[sch["basis_idx"]]


@pytest.mark.parametrize("lev", [8, 12, 16])
def test_schedule_reproduces_oracle_basis_values(api, lev):
    sch = api.mtp_describe_schedule(api.make_desc(3, lev))
    md = O.OracleModel(3, lev, 2.0, 5.0)
    g = synth.rng(100 + lev)
    theta = g.normal(size=md.m) * 0.05
    n_nb = 9
    d = g.normal(size=(n_nb, 3))
    rv = d / np.linalg.norm(d, axis=1, keepdims=True) * g.uniform(2.1, 4.9, (n_nb, 1))
    types = g.integers(0, 3, n_nb + 1).astype(np.int32)
    nbr = {"off": np.array([0, n_nb] + [n_nb] * n_nb, np.int64), "j": np.arange(1, n_nb + 1, dtype=np.int32),
           "r": rv}
    B_ref = O.sites(md, theta, types, nbr, req=[0], want_dVdr=False, want_b=True)["b"][0, 3:3 + md.n_lin]
    c = theta[3 + md.n_lin:].reshape(3, 3, md.n_rad, 8)
    r = np.linalg.norm(rv, axis=1)
    x = (2 * r - 7.0) / 3.0
    Q = np.polynomial.chebyshev.chebvander(x, 7) * ((5.0 - r) ** 2)[:, None]
    f = np.einsum("jmb,jb->jm", c[types[0], types[1:]], Q)
    B = _eval_schedule(sch, rv, f)
    np.testing.assert_allclose(B, B_ref, rtol=1e-11, atol=1e-14 * np.abs(B_ref).max())


@pytest.mark.parametrize("T,lev", [(1, 8), (3, 12), (2, 16)])
def test_gauge_directions_match_oracle(api, T, lev):
    md = O.OracleModel(T, lev, 2.0, 5.0)
    theta = synth.rng(lev).normal(size=md.m)
    np.testing.assert_array_equal(api.mtp_gauge_directions(api.make_desc(T, lev), theta),
                                  O.gauge_directions(md, theta))

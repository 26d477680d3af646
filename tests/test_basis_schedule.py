"""Host-side basis enumeration and contraction schedule of the library vs. the oracle."""
import numpy as np
import pytest

from oracle import basis_ref
from oracle import oracle as O
from paper_2304_13144_gb300 import basis, synth


@pytest.mark.parametrize("lev", [2, 4, 6, 8, 10, 12, 14, 16])
def test_enumerations_agree_in_canonical_order(lev):
    lib = [(b.labels, b.edges) for b in basis.enumerate_basis(lev)]
    ref = basis_ref.basis_functions(lev)
    assert lib == ref


@pytest.mark.parametrize("T,lev,m", [(1, 8, 26), (1, 12, 54), (1, 16, 125), (2, 16, 222),
                                     (3, 16, 383), (3, 20, 651)])
def test_parameter_counts(T, lev, m):
    assert basis.model_shape(T, lev).n_params == m


def _eval_schedule(sched, rv, f):
    """Evaluate the flattened triple list in float64 (numpy), for one neighborhood."""
    vals = np.zeros(sched.n_vals)
    for k in range(sched.n_mom_comps):
        a, b, c = sched.comp_exp[k]
        mu = sched.comp_mu[k]
        vals[k] = np.sum(f[:, mu] * rv[:, 0] ** a * rv[:, 1] ** b * rv[:, 2] ** c)
    for d in range(len(sched.dst_ptr) - 1):
        s = 0.0
        for t in range(sched.dst_ptr[d], sched.dst_ptr[d + 1]):
            s += sched.tri_c[t] * vals[sched.tri_a[t]] * vals[sched.tri_b[t]]
        vals[sched.first_dst + d] = s
    return vals[np.array(sched.basis_idx)]


@pytest.mark.parametrize("lev", [8, 12, 16])
def test_schedule_reproduces_oracle_basis_values(lev):
    shape = basis.model_shape(3, lev)
    sched = basis.compile_schedule(shape)
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
    B = _eval_schedule(sched, rv, f)
    np.testing.assert_allclose(B, B_ref, rtol=1e-11, atol=1e-14 * np.abs(B_ref).max())

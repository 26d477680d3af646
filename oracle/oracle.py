"""Python side of the FP64 CPU oracle (test infrastructure).

Only tests/, the package smoke check and the CPU-baseline leg of bench.py import this
module.  It never imports the library package and the library never imports it.

It builds oracle/mtp_oracle.cpp with g++ (plain, OpenMP over atoms) and composes the
per-site results into the quantities of the method with plain numpy:
  E_k = sum_{i in k} V_i                                   (eq. 1)
  F_i = sum_{p in nbh(i)} dV_i/dr_p - sum_{p: j(p) = i} dV_{c(p)}/dr_p   (F = -dE/dx)
  W_ab = -sum_p (dV/dr_p)_a (r_p)_b                      (virial, eV; reading R7)
  b_i = dV_i/dtheta                                       (eq. 9)
  gamma_i = max_p |(b_i A^{-1})_p|                        (Section II.D)
  L = sum_k w_e dE_k^2 + w_f sum_i |dF_i|^2 + w_s sum_ab dW_ab^2   (eq. 7)
  dL/dtheta = sum_k 2 w_e dE_k sum_{i in k} b_i - d/dt sum_i b_i(r + t rdot),
      rdot_p = U_j - U_i + S_k r_p,  U = 2 w_f (F - F*),  S_k = 2 w_s (W_k - W*_k).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

from . import basis_ref

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None


def build(force: bool = False) -> str:
    out_dir = os.path.join(_HERE, "_build")
    os.makedirs(out_dir, exist_ok=True)
    so = os.path.join(out_dir, "liboracle.so")
    src = os.path.join(_HERE, "mtp_oracle.cpp")
    if force or not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(src):
        tmp = so + f".{os.getpid()}.tmp"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
                               src, "-o", tmp])
        os.replace(tmp, so)
    return so


def _lib():
    global _LIB
    if _LIB is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        lib.oracle_neighbors.restype = ctypes.c_int64
        lib.oracle_neighbors.argtypes = [ctypes.c_int64, P, P, P, ctypes.c_double, ctypes.c_int,
                                         ctypes.c_int64, P, P, P, P]
        lib.oracle_sites.restype = ctypes.c_int
        lib.oracle_sites.argtypes = ([ctypes.c_int] * 4 + [ctypes.c_double] * 2 + [P] * 5 +
                                     [ctypes.c_int64] + [P] * 10)
        lib.oracle_grade.restype = ctypes.c_int
        lib.oracle_grade.argtypes = [ctypes.c_int64, P, ctypes.c_int64, P, P, P, P]
        _LIB = lib
    return _LIB


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def threads() -> int:
    """OpenMP threads the oracle's parallel loops use."""
    return int(_lib().omp_get_max_threads())


def set_threads(n: int) -> None:
    """Set the OpenMP thread count of the oracle's parallel loops (process-wide)."""
    _lib().omp_set_num_threads(int(n))


@dataclass
class OracleModel:
    n_types: int
    lev_max: int
    r_min: float
    r_cut: float
    n_q: int = 8

    def __post_init__(self):
        self.basis, self.n_rad, self.m = basis_ref.shape(self.n_types, self.lev_max, self.n_q)
        self.n_lin = len(self.basis)
        self.bP, self.bmu, self.bnu, self.bed = basis_ref.flatten(self.basis)


# ------------------------------------------------------------------------------------
# neighbors
# ------------------------------------------------------------------------------------

def neighbors(pos, cell, pbc, r_cut, brute=True):
    """Per-configuration neighbor list: (off[N+1], j[P], img[P,3], r[P,3])."""
    lib = _lib()
    pos = np.ascontiguousarray(pos, np.float64)
    cell = np.ascontiguousarray(cell, np.float64).reshape(3, 3)
    pbc = np.ascontiguousarray(pbc, np.uint8).reshape(3)
    n = pos.shape[0]
    off = np.zeros(n + 1, np.int64)
    cap = max(64, 64 * n)
    while True:
        nj = np.zeros(cap, np.int32)
        img = np.zeros((cap, 3), np.int32)
        r = np.zeros((cap, 3), np.float64)
        tot = lib.oracle_neighbors(n, _p(pos), _p(cell), _p(pbc), float(r_cut), int(brute), cap,
                                   _p(off), _p(nj), _p(img), _p(r))
        if tot == -1:
            raise ValueError("coincident atoms")
        if tot < 0:
            raise ValueError("unsupported neighbor request")
        if tot <= cap:
            return off, nj[:tot].copy(), img[:tot].copy(), r[:tot].copy()
        cap = int(tot)


def batch_neighbors(batch, r_cut, brute=None):
    """Neighbor list over a batch with global atom indices."""
    ao = batch["atom_offset"]
    offs, js, imgs, rs = [np.zeros(1, np.int64)], [], [], []
    base_pairs = 0
    for k in range(len(ao) - 1):
        a0, a1 = int(ao[k]), int(ao[k + 1])
        use_brute = brute if brute is not None else (a1 - a0) <= 2000 or not all(batch["pbc"][k])
        off, nj, img, r = neighbors(batch["pos"][a0:a1], batch["cell"][k], batch["pbc"][k], r_cut,
                                    brute=use_brute)
        offs.append(off[1:] + base_pairs)
        js.append(nj + a0)
        imgs.append(img)
        rs.append(r)
        base_pairs += len(nj)
    return {"off": np.concatenate(offs), "j": np.concatenate(js) if js else np.zeros(0, np.int32),
            "img": np.concatenate(imgs) if imgs else np.zeros((0, 3), np.int32),
            "r": np.concatenate(rs) if rs else np.zeros((0, 3))}


def pair_centers(off):
    n = len(off) - 1
    return np.repeat(np.arange(n, dtype=np.int64), np.diff(off))


# ------------------------------------------------------------------------------------
# sites
# ------------------------------------------------------------------------------------

def sites(model: OracleModel, theta, types, nbr, req=None, rdot=None, want_dVdr=True, want_b=False):
    """Per-site V_i (and dV_i/dr_p, b_i, tangents) for the requested atoms (default: all)."""
    lib = _lib()
    theta = np.ascontiguousarray(theta, np.float64)
    assert theta.shape == (model.m,), (theta.shape, model.m)
    types = np.ascontiguousarray(types, np.int32)
    n = len(types)
    req = np.arange(n, dtype=np.int64) if req is None else np.ascontiguousarray(req, np.int64)
    nreq = len(req)
    npairs = len(nbr["j"])
    V = np.zeros(nreq)
    dVdr = np.zeros((npairs, 3)) if want_dVdr else None
    b = np.zeros((nreq, model.m)) if (want_b or rdot is not None) else None
    Vd = bd = None
    rdot_c = None
    if rdot is not None:
        rdot_c = np.ascontiguousarray(rdot, np.float64)
        Vd = np.zeros(nreq)
        bd = np.zeros((nreq, model.m))
    rc = lib.oracle_sites(model.n_types, model.n_q, model.n_rad, model.n_lin, model.r_min, model.r_cut,
                          _p(model.bP), _p(model.bmu), _p(model.bnu), _p(model.bed), _p(theta),
                          nreq, _p(req), _p(types), _p(np.ascontiguousarray(nbr["off"], np.int64)),
                          _p(np.ascontiguousarray(nbr["j"], np.int32)),
                          _p(np.ascontiguousarray(nbr["r"], np.float64)), _p(rdot_c),
                          _p(V), _p(dVdr), _p(b), _p(Vd), _p(bd))
    assert rc == 0
    return {"V": V, "dVdr": dVdr, "b": b, "V_dot": Vd, "b_dot": bd}


def efs(model: OracleModel, theta, batch, nbr=None):
    """Energies per config, forces per atom, virial per config, site energies."""
    if nbr is None:
        nbr = batch_neighbors(batch, model.r_cut)
    s = sites(model, theta, batch["type"], nbr)
    ao = batch["atom_offset"]
    n = len(batch["type"])
    V = s["V"]
    G = s["dVdr"]
    cen = pair_centers(nbr["off"])
    F = np.zeros((n, 3))
    np.add.at(F, cen, G)
    np.add.at(F, nbr["j"].astype(np.int64), -G)
    ncfg = len(ao) - 1
    cfg_of_atom = np.repeat(np.arange(ncfg), np.diff(ao))
    E = np.zeros(ncfg)
    np.add.at(E, cfg_of_atom, V)
    W = np.zeros((ncfg, 3, 3))
    np.add.at(W, cfg_of_atom[cen], -G[:, :, None] * nbr["r"][:, None, :])
    return {"E": E, "F": F, "W": W, "V": V, "nbr": nbr, "dVdr": G}


def site_rows(model: OracleModel, theta, types, nbr, req=None):
    """b_i = dV_i/dtheta for the requested atoms."""
    return sites(model, theta, types, nbr, req=req, want_dVdr=False, want_b=True)["b"]


# ------------------------------------------------------------------------------------
# grade
# ------------------------------------------------------------------------------------

def grade(A, brows, want_inverse=False):
    lib = _lib()
    A = np.ascontiguousarray(A, np.float64)
    brows = np.ascontiguousarray(brows, np.float64)
    m = A.shape[0]
    n = brows.shape[0]
    gamma = np.zeros(n)
    am = np.zeros(n, np.int32)
    Ainv = np.zeros((m, m)) if want_inverse else None
    rc = lib.oracle_grade(m, _p(A), n, _p(brows), _p(gamma), _p(am), _p(Ainv))
    if rc != 0:
        raise np.linalg.LinAlgError("singular active-set matrix")
    return (gamma, am, Ainv) if want_inverse else (gamma, am)


# ------------------------------------------------------------------------------------
# loss (eq. 7) and its parameter gradient
# ------------------------------------------------------------------------------------

def loss_and_grad(model: OracleModel, theta, batch, E_ref, F_ref, W_ref, w_e, w_f, w_s, nbr=None):
    if nbr is None:
        nbr = batch_neighbors(batch, model.r_cut)
    out = efs(model, theta, batch, nbr)
    E, F, W = out["E"], out["F"], out["W"]
    dE = E - E_ref
    dF = F - F_ref
    dW = W - W_ref if W_ref is not None else np.zeros_like(W)
    L = w_e * np.sum(dE ** 2) + w_f * np.sum(dF ** 2) + (w_s * np.sum(dW ** 2) if w_s else 0.0)
    ao = batch["atom_offset"]
    ncfg = len(ao) - 1
    cfg_of_atom = np.repeat(np.arange(ncfg), np.diff(ao))
    U = 2.0 * w_f * dF
    S = 2.0 * w_s * dW
    cen = pair_centers(nbr["off"])
    jj = nbr["j"].astype(np.int64)
    rdot = U[jj] - U[cen] + np.einsum("pab,pb->pa", S[cfg_of_atom[cen]], nbr["r"])
    s = sites(model, theta, batch["type"], nbr, rdot=rdot, want_dVdr=False)
    coef = 2.0 * w_e * dE[cfg_of_atom]
    grad = coef @ s["b"] - s["b_dot"].sum(axis=0)
    return L, grad, out


def gauge_directions(model: OracleModel, theta):
    """Null directions of the parameter rows (reading R19).

    Mixing the radial functions, f_mu -> f_mu + eps f_mu' for mu' <= mu, is the change
    c[.][.][mu][.] += eps c[.][.][mu'][.] (eq. 4).  To first order it turns every basis
    function B_a with a factor M_{mu,nu} into B_a + eps B_a' with that factor relabelled
    M_{mu',nu} (eq. 3); the relabelled graph has a lower level, so it is again a basis
    function.  Adding -eps xi_a to xi_a' therefore leaves V unchanged, and d/deps gives one
    direction d with b_i . d = 0 for every neighborhood.  Returns the
    n_rad (n_rad + 1) / 2 directions as rows, ordered by (mu, mu').
    """
    T, nl, nr, nq = model.n_types, model.n_lin, model.n_rad, model.n_q
    index = {f: a for a, f in enumerate(model.basis)}
    c = np.asarray(theta[T + nl:]).reshape(T, T, nr, nq)
    rows = []
    for mu in range(nr):
        for mu2 in range(mu + 1):
            d = np.zeros(model.m)
            blk = np.zeros_like(c)
            blk[:, :, mu, :] = c[:, :, mu2, :]
            d[T + nl:] = blk.reshape(-1)
            for a, (labs, edges) in enumerate(model.basis):
                P = len(labs)
                pairs = [(i, j) for i in range(P) for j in range(P) if i < j]
                mat = [[0] * P for _ in range(P)]
                for (i, j), e in zip(pairs, edges):
                    mat[i][j] = mat[j][i] = e
                for p in range(P):
                    if labs[p][0] != mu:
                        continue
                    new = list(labs)
                    new[p] = (mu2, labs[p][1])
                    order = sorted(range(P), key=lambda k: new[k])
                    nlabs = tuple(new[k] for k in order)
                    nmat = [[mat[order[i]][order[j]] for j in range(P)] for i in range(P)]
                    key = (nlabs, basis_ref._canon(nlabs, nmat))
                    d[T + index[key]] -= theta[T + a]
            rows.append(d)
    return np.array(rows)

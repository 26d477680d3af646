"""Seeded synthetic inputs (lattices, displacements, species, parameter draws).

This module holds no arithmetic of the method itself: it only produces configurations,
parameter vectors and active-set matrices from numpy's PCG64 generator, so that the CUDA
path and the CPU oracle can be fed the same inputs.  The paper's Cu training data are not
available; these periodic metallic crystals stand in for the paper's workloads
(periodic metals, R_cut = 5 A, Section IV).

A batch is a dict:
  atom_offset int64 [n_cfg+1], pos float64 [N,3] (A), type int32 [N],
  cell float64 [n_cfg,3,3] (rows = lattice vectors, A), pbc uint8 [n_cfg,3].
"""
from __future__ import annotations

import math

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


# ------------------------------------------------------------------------------------
# lattices
# ------------------------------------------------------------------------------------

_FCC = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
_BCC = np.array([[0, 0, 0], [0.5, 0.5, 0.5]])


def cubic_supercell(basis_frac, a, n):
    """Positions (A) and cell of an n x n x n supercell of a cubic cell with the given basis."""
    nx, ny, nz = (n, n, n) if np.isscalar(n) else n
    g = np.stack(np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij"), -1).reshape(-1, 3)
    pos = (g[:, None, :] + basis_frac[None, :, :]).reshape(-1, 3) * a
    cell = np.diag([nx * a, ny * a, nz * a]).astype(np.float64)
    sub = np.tile(np.arange(len(basis_frac)), len(g))
    return pos, cell, sub


def hcp_supercell(a, c, n):
    nx, ny, nz = n
    a1 = np.array([a, 0.0, 0.0])
    a2 = np.array([-0.5 * a, 0.5 * math.sqrt(3) * a, 0.0])
    a3 = np.array([0.0, 0.0, c])
    basis = np.array([[0, 0, 0], [1.0 / 3, 2.0 / 3, 0.5]])
    g = np.stack(np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij"), -1).reshape(-1, 3)
    frac = (g[:, None, :] + basis[None]).reshape(-1, 3)
    H = np.stack([a1 * nx, a2 * ny, a3 * nz])
    pos = frac / np.array([nx, ny, nz]) @ H
    return pos, H, np.tile(np.arange(2), len(g))


def single(pos, types, cell, pbc=(1, 1, 1)):
    return {"atom_offset": np.array([0, len(pos)], np.int64),
            "pos": np.ascontiguousarray(pos, np.float64),
            "type": np.ascontiguousarray(types, np.int32),
            "cell": np.ascontiguousarray(cell, np.float64).reshape(1, 3, 3),
            "pbc": np.array([pbc], np.uint8)}


def concat(batches):
    ao = [0]
    for b in batches:
        ao.append(ao[-1] + len(b["type"]))
    return {"atom_offset": np.array(ao, np.int64),
            "pos": np.concatenate([b["pos"] for b in batches]),
            "type": np.concatenate([b["type"] for b in batches]).astype(np.int32),
            "cell": np.concatenate([b["cell"] for b in batches]),
            "pbc": np.concatenate([b["pbc"] for b in batches]).astype(np.uint8)}


# ------------------------------------------------------------------------------------
# the workloads
# ------------------------------------------------------------------------------------

def fcc_unary_108(seed=1, sigma=0.1):
    """fcc a = 4.05 A, 3x3x3 conventional cells (108 atoms), unary, Gaussian displacements."""
    g = rng(seed)
    pos, cell, _ = cubic_supercell(_FCC, 4.05, 3)
    pos = pos + g.normal(0.0, sigma, pos.shape)
    return single(pos, np.zeros(len(pos), np.int32), cell)


def b2_binary(seed=2, n=40, a=2.87, sigma=0.08, swap=0.10):
    """B2 (bcc) n^3 conventional cells, species by sublattice, then `swap` of the atoms flipped."""
    g = rng(seed)
    pos, cell, sub = cubic_supercell(_BCC, a, n)
    types = sub.astype(np.int32).copy()
    k = int(round(swap * len(types)))
    idx = g.choice(len(types), size=k, replace=False)
    types[idx] = 1 - types[idx]
    pos = pos + g.normal(0.0, sigma, pos.shape)
    return single(pos, types, cell)


def fcc_ternary(seed=4, n=64, a=3.6, sigma=0.1):
    """fcc a = 3.6 A, n^3 conventional cells, ternary random solid solution with species
    counts as equal as possible (a random permutation of a balanced list)."""
    g = rng(seed)
    pos, cell, _ = cubic_supercell(_FCC, a, n)
    N = len(pos)
    types = (np.arange(N) % 3).astype(np.int32)
    types = types[g.permutation(N)]
    pos = pos + g.normal(0.0, sigma, pos.shape)
    return single(pos, types, cell)


def _realisable(target, per_cell):
    best = None
    for nx in range(1, 9):
        for ny in range(1, 9):
            for nz in range(1, 9):
                n = nx * ny * nz * per_cell
                shape_pen = max(nx, ny, nz) / min(nx, ny, nz)
                key = (abs(n - target), shape_pen)
                if best is None or key < best[0]:
                    best = (key, (nx, ny, nz))
    return best[1]


def training_batch(seed=3, n_cfg=512, n_types=3, lo=8, hi=256):
    """Configurations of log-uniform size in [lo, hi], each a random choice of fcc
    (a = 3.6), bcc (a = 2.87) or hcp (a = 2.55, c/a = 1.633) supercell, random species,
    a random symmetric strain with components U(-0.03, 0.03), displacements with
    sigma ~ U(0.05, 0.15)."""
    g = rng(seed)
    out = []
    for _ in range(n_cfg):
        target = int(round(math.exp(g.uniform(math.log(lo), math.log(hi)))))
        kind = int(g.integers(0, 3))
        if kind == 0:
            nn = _realisable(target, 4)
            pos, cell, _ = cubic_supercell(_FCC, 3.6, nn)
        elif kind == 1:
            nn = _realisable(target, 2)
            pos, cell, _ = cubic_supercell(_BCC, 2.87, nn)
        else:
            nn = _realisable(target, 2)
            pos, cell, _ = hcp_supercell(2.55, 2.55 * 1.633, nn)
        e = g.uniform(-0.03, 0.03, (3, 3))
        e = 0.5 * (e + e.T)
        D = np.eye(3) + e
        pos = pos @ D.T
        cell = cell @ D.T
        sigma = g.uniform(0.05, 0.15)
        pos = pos + g.normal(0.0, sigma, pos.shape)
        types = g.integers(0, n_types, len(pos)).astype(np.int32)
        out.append(single(pos, types, cell))
    return concat(out)


# ------------------------------------------------------------------------------------
# parameters and active sets
# ------------------------------------------------------------------------------------

def draw_theta(seed, n_types, n_rad, n_q, nu_sum, n_factors, r_min, r_cut, nbar, kappa=10.0):
    """Parameter vector theta = [s (T) | xi (N_lin) | c (T*T*n_rad*n_q)].

    Raw draws g ~ N(0, 0.1^2) are rescaled per basis function so that every term
    xi_a B_a has a comparable magnitude: xi_a = g_a kappa^P / (r_cut^sum(nu) nbar^P),
    where P is the factor count and sum(nu) the total tensor rank of the function;
    c ~ N(0, 0.1^2) / (r_cut - r_min)^2.  Any theta is a valid model; the scaling only
    keeps energies and forces in the range of metallic systems.
    """
    g = rng(seed)
    nu_sum = np.asarray(nu_sum, np.float64)
    n_factors = np.asarray(n_factors, np.float64)
    n_lin = len(nu_sum)
    s = g.normal(0.0, 0.1, n_types)
    raw = g.normal(0.0, 0.1, n_lin)
    xi = raw * kappa ** n_factors / (r_cut ** nu_sum * nbar ** n_factors)
    c = g.normal(0.0, 0.1, n_types * n_types * n_rad * n_q) / (r_cut - r_min) ** 2
    return np.concatenate([s, xi, c])


def diag_dominant(seed, m):
    """Random well-conditioned active-set matrix: G + diag(sum_l |G_kl| + 1), G ~ N(0,1)."""
    g = rng(seed)
    G = g.normal(0.0, 1.0, (m, m))
    return G + np.diag(np.abs(G).sum(axis=1) + 1.0)


def sample_atoms(seed, n_atoms, k):
    g = rng(seed)
    return np.sort(g.choice(n_atoms, size=min(k, n_atoms), replace=False)).astype(np.int64)

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


def liquid_rsa(seed=5, n_atoms=2_097_152, density=0.085, d_min=1.8, n_types=4, tiles=1):
    """Liquid-like configuration: random sequential addition of points, uniform in a periodic
    cube of volume n_atoms/density, each new point kept only if it is at least d_min from every
    point kept before; species uniform over n_types, drawn for every atom.

    With tiles = t > 1 the addition fills a cube of n_atoms/t^3 points and the cube is repeated
    t x t x t times (its periodic boundary makes the copy seamless): the density, the minimum
    distance and every neighborhood's statistics are those of the single cube, at a fraction of
    the generation time.  n_atoms must then be a multiple of t^3.

    Candidates are drawn in batches.  A grid of cells no wider than d_min/sqrt(3) holds at most
    one point per cell; a candidate is tested against the kept points in the 5x5x5 cells around
    its own, then against earlier candidates of its batch (a candidate that meets an earlier one
    within d_min is dropped, even if that earlier one is dropped too), which keeps every pair of
    kept points at least d_min apart."""
    if n_atoms % (tiles ** 3):
        raise ValueError("n_atoms must be a multiple of tiles^3")
    g = rng(seed)
    n_total, n_atoms = n_atoms, n_atoms // tiles ** 3
    L = (n_atoms / density) ** (1.0 / 3.0)
    M = int(math.ceil(L / (d_min / math.sqrt(3.0))))
    cs = L / M
    grid = np.full(M * M * M, -1, np.int64)
    pos = np.empty((n_atoms, 3))
    n = 0
    offs = np.stack(np.meshgrid(*(np.arange(-2, 3),) * 3, indexing="ij"), -1).reshape(-1, 3)
    d2 = d_min * d_min
    acc = 1.0

    def cells(x):
        c = np.minimum((x / cs).astype(np.int64), M - 1)
        return c

    def flat(c):
        c = np.mod(c, M)
        return (c[:, 0] * M + c[:, 1]) * M + c[:, 2]

    def conflicts(x, c, table, pts, idx_limit=None):
        bad = np.zeros(len(x), bool)
        for o in offs:
            k = table[flat(c + o)]
            hit = k >= 0
            if idx_limit is not None:
                hit &= k < idx_limit
            if not hit.any():
                continue
            h = np.nonzero(hit)[0]
            d = x[h] - pts[k[h]]
            d -= L * np.round(d / L)
            bad[h[(d * d).sum(1) < d2]] = True
        return bad

    while n < n_atoms:
        need = n_atoms - n
        K = int(min(4_000_000, max(100_000, 2.0 * need / max(acc, 0.02))))
        x = g.uniform(0.0, L, (K, 3))
        c = cells(x)
        ok = ~conflicts(x, c, grid, pos) if n else np.ones(K, bool)
        x, c = x[ok], c[ok]
        f = flat(c)
        # earlier candidates of the batch: first one per cell, then the 5x5x5 neighbourhood
        _, first = np.unique(f, return_index=True)
        keep = np.zeros(len(x), bool)
        keep[first] = True
        x, c, f = x[keep], c[keep], f[keep]
        order = np.arange(len(x))
        tmp = np.full(M * M * M, -1, np.int64)
        tmp[f] = order
        bad = np.zeros(len(x), bool)
        for o in offs:
            if not o.any():
                continue
            k = tmp[flat(c + o)]
            hit = (k >= 0) & (k < order)
            if not hit.any():
                continue
            h = np.nonzero(hit)[0]
            d = x[h] - x[k[h]]
            d -= L * np.round(d / L)
            bad[h[(d * d).sum(1) < d2]] = True
        x, f = x[~bad], f[~bad]
        take = min(len(x), need)
        pos[n:n + take] = x[:take]
        grid[f[:take]] = np.arange(n, n + take)
        n += take
        acc = max(take / K, 1e-3)
    if tiles > 1:
        t = np.stack(np.meshgrid(*(np.arange(tiles),) * 3, indexing="ij"), -1).reshape(-1, 3)
        pos = (pos[None, :, :] + L * t[:, None, :]).reshape(-1, 3)
    types = g.integers(0, n_types, n_total).astype(np.int32)
    return single(pos, types, np.eye(3) * (L * tiles))


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

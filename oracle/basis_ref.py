"""Oracle's own MTP basis enumeration (test infrastructure; shares no code with the library).

Only tests/, the package smoke check and the CPU-baseline leg of bench.py use this module.

Section II.A (eqs. 5-6): a basis function is a scalar contraction of moment
tensors M_{mu,nu}; its level is sum_p (2 + 4 mu_p + nu_p); the basis of level
lev_max holds every such function with level <= lev_max.  Readings (listed in
the design notes): at most 4 moment factors, no index contracted within one
factor (the level-6 example has no trace of M02), one constant per species and
N_Q = 8; these reproduce the parameter counts 26/54/125 of Section IV.

This is a deliberately plain brute force: every symmetric, zero-diagonal,
non-negative integer matrix with row sums nu_p is generated, and its canonical
form is the lexicographically smallest upper-triangle vector (e01,e02,e03,e12,e13,e23)
over all node relabellings that keep the ascending label sequence fixed.
Basis functions are sorted by (level, P, labels, edge vector).
"""
import itertools


def level_of_moment(mu, nu):
    return 2 + 4 * mu + nu


def _upper(P):
    return [(i, j) for i in range(P) for j in range(P) if i < j]


def _is_label_preserving(perm, labels):
    return all(labels[perm[k]] == labels[k] for k in range(len(labels)))


def _canon(labels, mat):
    P = len(labels)
    best = None
    for perm in itertools.permutations(range(P)):
        if not _is_label_preserving(perm, labels):
            continue
        vec = tuple(mat[perm[i]][perm[j]] for i, j in _upper(P))
        if best is None or vec < best:
            best = vec
    return best


def _matrices(nus):
    P = len(nus)
    ups = _upper(P)
    ranges = [range(min(nus[i], nus[j]) + 1) for i, j in ups]
    for vals in itertools.product(*ranges):
        mat = [[0] * P for _ in range(P)]
        for (i, j), v in zip(ups, vals):
            mat[i][j] = v
            mat[j][i] = v
        if all(sum(mat[i]) == nus[i] for i in range(P)):
            yield mat


def basis_functions(lev_max, max_factors=4):
    """List of (labels, edges): labels = tuple of (mu, nu) ascending, edges = canonical vector."""
    labels_all = []
    for mu in range(lev_max + 1):
        for nu in range(lev_max + 1):
            if level_of_moment(mu, nu) <= lev_max:
                labels_all.append((mu, nu))
    labels_all.sort()
    out = set()
    for P in range(1, max_factors + 1):
        for labs in itertools.combinations_with_replacement(labels_all, P):
            if sum(level_of_moment(mu, nu) for mu, nu in labs) > lev_max:
                continue
            for mat in _matrices([nu for _, nu in labs]):
                out.add((tuple(labs), _canon(labs, mat)))
    def key(item):
        labs, edges = item
        return (sum(level_of_moment(mu, nu) for mu, nu in labs), len(labs), labs, edges)
    return sorted(out, key=key)


def shape(n_types, lev_max, n_q=8):
    """(basis, n_rad, n_params) with theta = [s (T) | xi (N_lin) | c[zi][zj][mu][beta]]."""
    basis = basis_functions(lev_max)
    n_rad = 1 + max(mu for labs, _ in basis for mu, _ in labs)
    n_params = n_types + len(basis) + n_types * n_types * n_rad * n_q
    return basis, n_rad, n_params


def flatten(basis):
    """Arrays for the C oracle: per basis function P, 4 (mu, nu) labels and 6 edge counts
    in the pair order (0,1),(0,2),(0,3),(1,2),(1,3),(2,3)."""
    import numpy as np
    n = len(basis)
    P = np.zeros(n, np.int32)
    mu = np.zeros((n, 4), np.int32)
    nu = np.zeros((n, 4), np.int32)
    ed = np.zeros((n, 6), np.int32)
    full_pairs = _upper(4)
    for k, (labs, edges) in enumerate(basis):
        P[k] = len(labs)
        for p, (m, v) in enumerate(labs):
            mu[k, p] = m
            nu[k, p] = v
        for (i, j), e in zip(_upper(len(labs)), edges):
            ed[k, full_pairs.index((i, j))] = e
    return P, mu, nu, ed

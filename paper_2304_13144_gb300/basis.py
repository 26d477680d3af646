"""MTP basis enumeration and the flattened contraction schedule used by the CUDA kernels.

Section II.A of the paper defines the basis: every basis function B_alpha is a
contraction of one or more moment tensors M_{mu,nu} (eq. 3) into a scalar, and the
basis of an MTP of level lev_max is every such contraction whose level
sum_p (2 + 4 mu_p + nu_p) (eqs. 5-6) is at most lev_max.  The level-6 example of
Section II.A lists exactly {M00, M10, M00^2, M01.M01, M00^3}: no trace of M02,
so an index is never contracted with another index of the same factor.

Reading used here (stated with the other readings in the design notes):
  * a basis function is a multigraph on P <= 4 nodes; node p carries a moment
    label (mu_p, nu_p) and has degree nu_p; an edge is one index contracted
    between two different factors; there are no self-loops;
  * the canonical form sorts the labels ascending and takes, over the
    label-preserving node permutations, the lexicographically smallest edge
    vector (e01, e02, e03, e12, e13, e23) restricted to the P nodes;
  * basis functions are ordered by (level, P, labels, edge vector).
With one constant per species and N_Q = 8 radial polynomials this gives the
parameter counts 26 / 54 / 125 that Section IV quotes for unary levels 8/12/16.

The schedule compiler turns the basis into straight-line arithmetic over a
per-atom value array:
  vals = [moment components | contraction intermediates | products]
with every non-moment value formed as  vals[dst] = sum_t coeff_t * vals[a_t] * vals[b_t]
(the flattened triple list).  Moments are kept in symmetric storage: the component
with exponents (a, b, c), a+b+c = nu, holds sum_j f_mu(r_j) x^a y^b z^c.
A contraction over k index pairs between symmetric tensors A and B is exact in
this storage with multinomial weights:
  T[alpha | beta] = sum_{|gamma| = k} k!/(g1! g2! g3!) A[alpha+gamma] B[beta+gamma].
Intermediates keep their index groups separate (T is only symmetric within
each group), so cyclic graphs such as tr(ABCD) are evaluated exactly.
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass, field
from functools import lru_cache


def moment_level(mu: int, nu: int) -> int:
    """Level of M_{mu,nu} (eq. 5)."""
    return 2 + 4 * mu + nu


@lru_cache(maxsize=None)
def exponents(nu: int) -> tuple:
    """Symmetric-storage components of a rank-nu tensor in canonical order:
    exponent triples (a, b, c) with a+b+c = nu, a descending, then b descending."""
    return tuple((a, b, nu - a - b) for a in range(nu, -1, -1) for b in range(nu - a, -1, -1))


@lru_cache(maxsize=None)
def multinomial(e: tuple) -> int:
    """Number of index tuples (i_1..i_n) in {x,y,z}^n with exponent triple e."""
    n = sum(e)
    return math.factorial(n) // (math.factorial(e[0]) * math.factorial(e[1]) * math.factorial(e[2]))


def _add(e1, e2):
    return (e1[0] + e2[0], e1[1] + e2[1], e1[2] + e2[2])


# ----------------------------------------------------------------------------------
# Enumeration
# ----------------------------------------------------------------------------------

_PAIRS = {P: [(p, q) for p in range(P) for q in range(p + 1, P)] for P in range(1, 5)}


@dataclass(frozen=True)
class BasisFunction:
    labels: tuple          # ((mu, nu), ...) sorted ascending, length P
    edges: tuple           # canonical edge vector over _PAIRS[P]

    @property
    def P(self) -> int:
        return len(self.labels)

    @property
    def level(self) -> int:
        return sum(moment_level(mu, nu) for mu, nu in self.labels)

    @property
    def nu_sum(self) -> int:
        return sum(nu for _, nu in self.labels)

    def key(self):
        return (self.level, self.P, self.labels, self.edges)

    def edge(self, p: int, q: int) -> int:
        if p == q:
            return 0
        if p > q:
            p, q = q, p
        return self.edges[_PAIRS[self.P].index((p, q))]

    def components(self) -> list:
        """Connected components as lists of node indices (ascending)."""
        P = self.P
        seen, comps = set(), []
        for s in range(P):
            if s in seen:
                continue
            comp, stack = [], [s]
            seen.add(s)
            while stack:
                a = stack.pop()
                comp.append(a)
                for b in range(P):
                    if b not in seen and self.edge(a, b) > 0:
                        seen.add(b)
                        stack.append(b)
            comps.append(sorted(comp))
        return comps

    def __str__(self):
        labs = " ".join(f"M{mu}{nu}" for mu, nu in self.labels)
        return f"[{labs} | e={self.edges}]"


def _edge_vectors(degrees):
    """All loop-free edge multiplicity vectors over _PAIRS[P] realising the degrees."""
    P = len(degrees)
    pairs = _PAIRS[P]
    out = []
    rem = list(degrees)

    def rec(k, cur):
        if k == len(pairs):
            if all(r == 0 for r in rem):
                out.append(tuple(cur))
            return
        p, q = pairs[k]
        hi = min(rem[p], rem[q])
        for m in range(hi + 1):
            rem[p] -= m
            rem[q] -= m
            # node p has no later pair once q is the last node
            if not (q == P - 1 and rem[p] != 0):
                cur.append(m)
                rec(k + 1, cur)
                cur.pop()
            rem[p] += m
            rem[q] += m

    rec(0, [])
    return out


def _canonical_edges(labels, edges):
    P = len(labels)
    pairs = _PAIRS[P]
    groups = {}
    for i, lab in enumerate(labels):
        groups.setdefault(lab, []).append(i)
    best = None
    for perm_parts in itertools.product(*[itertools.permutations(groups[k]) for k in sorted(groups)]):
        order = [x for part in perm_parts for x in part]       # new position -> old node
        emat = {}
        for (p, q), m in zip(pairs, edges):
            emat[(p, q)] = m
            emat[(q, p)] = m
        vec = tuple(emat[(order[p], order[q])] for p, q in pairs)
        if best is None or vec < best:
            best = vec
    return best


def enumerate_basis(lev_max: int, max_factors: int = 4) -> list:
    """All basis functions of level <= lev_max with at most max_factors moment factors,
    in canonical order."""
    moments = sorted((mu, nu) for mu in range(lev_max) for nu in range(lev_max + 1)
                     if moment_level(mu, nu) <= lev_max)
    found = set()

    def rec(start, labs, level):
        if labs:
            for ev in _edge_vectors([nu for _, nu in labs]):
                found.add(BasisFunction(tuple(labs), _canonical_edges(labs, ev)))
        if len(labs) == max_factors:
            return
        for k in range(start, len(moments)):
            mu, nu = moments[k]
            L = moment_level(mu, nu)
            if level + L <= lev_max:
                labs.append((mu, nu))
                rec(k, labs, level + L)
                labs.pop()

    rec(0, [], 0)
    return sorted(found, key=BasisFunction.key)


@dataclass
class ModelShape:
    n_types: int
    lev_max: int
    n_q: int
    basis: list

    @property
    def n_lin(self) -> int:
        return len(self.basis)

    @property
    def n_rad(self) -> int:
        return 1 + max(mu for b in self.basis for mu, _ in b.labels)

    @property
    def n_params(self) -> int:
        T = self.n_types
        return T + self.n_lin + T * T * self.n_rad * self.n_q

    # parameter layout: theta = [s_z (T) | xi (N_lin) | c[z_i][z_j][mu][beta]]
    @property
    def off_xi(self) -> int:
        return self.n_types

    @property
    def off_c(self) -> int:
        return self.n_types + self.n_lin


def model_shape(n_types: int, lev_max: int, n_q: int = 8) -> ModelShape:
    return ModelShape(n_types, lev_max, n_q, enumerate_basis(lev_max))


# ----------------------------------------------------------------------------------
# Schedule compiler
# ----------------------------------------------------------------------------------

@dataclass
class Schedule:
    """Flattened contraction schedule.

    moments:   list of (mu, nu) in value order; moment (mu, nu) occupies
               vals[mom_off[k] : mom_off[k] + len(exponents(nu))].
    comp_mu, comp_exp: per moment component, its mu and exponent triple.
    n_vals:    length of the per-atom value array.
    dst_ptr:   CSR over destinations: the triples of destination d (value index
               first_dst + d) are tri_a/tri_b/tri_c[dst_ptr[d]:dst_ptr[d+1]].
    basis_idx: value index of each basis function, in basis order.
    """
    moments: list
    mom_off: list
    n_mom_comps: int
    comp_mu: list
    comp_exp: list
    n_vals: int
    first_dst: int
    dst_ptr: list
    tri_a: list
    tri_b: list
    tri_c: list
    basis_idx: list
    nu_max: int
    stats: dict = field(default_factory=dict)

    @property
    def n_triples(self) -> int:
        return len(self.tri_a)


class _Builder:
    def __init__(self, moments):
        self.moments = moments
        self.mom_off = []
        off = 0
        self.comp_mu, self.comp_exp = [], []
        self.comp_index = {}
        for mu, nu in moments:
            self.mom_off.append(off)
            for e in exponents(nu):
                self.comp_index[(mu, nu, e)] = off
                self.comp_mu.append(mu)
                self.comp_exp.append(e)
                off += 1
        self.n_mom = off
        self.defs = []          # list of (key, [(a, b, c), ...]) for non-moment values
        self.index = {}         # key -> value index

    def mom(self, lab, e):
        mu, nu = lab
        return self.comp_index[(mu, nu, e)]

    def define(self, key, terms):
        if key in self.index:
            return self.index[key]
        merged = {}
        for a, b, c in terms:
            if a > b:
                a, b = b, a
            merged[(a, b)] = merged.get((a, b), 0) + c
        idx = self.n_mom + len(self.defs)
        self.defs.append((key, sorted((a, b, c) for (a, b), c in merged.items() if c != 0)))
        self.index[key] = idx
        return idx

    # T[alpha|beta] = A x_k B with free group sizes (nuA-k | nuB-k).
    def pair_contraction(self, A, B, k):
        if (B, A) < (A, B):
            # canonical operand order; the caller must swap groups accordingly
            raise ValueError("pair_contraction expects A <= B")
        fa, fb = A[1] - k, B[1] - k
        table = {}
        for al in exponents(fa):
            for be in exponents(fb):
                key = ("T", A, B, k, al, be)
                terms = [(self.mom(A, _add(al, g)), self.mom(B, _add(be, g)), multinomial(g))
                         for g in exponents(k)]
                table[(al, be)] = self.define(key, terms)
        return table

    def product(self, x, y):
        a, b = min(x, y), max(x, y)
        return self.define(("P", a, b), [(a, b, 1)])


def _component_scalar(bld: _Builder, bf: BasisFunction, nodes: list) -> tuple:
    """Emit the scalar of one connected component; returns (value index, triple cost)."""
    labs = [bf.labels[p] for p in nodes]
    n = len(nodes)
    E = lambda i, j: bf.edge(nodes[i], nodes[j])
    if n == 1:
        return bld.mom(labs[0], (0, 0, 0)), 0
    if n == 2:
        A, B = labs
        if (B, A) < (A, B):
            A, B = B, A
        key = ("S2", A, B)
        terms = [(bld.mom(A, g), bld.mom(B, g), multinomial(g)) for g in exponents(A[1])]
        return bld.define(key, terms), len(terms)
    if n == 3:
        best = None
        for r in range(3):
            p, q = [x for x in range(3) if x != r]
            cost = (len(exponents(E(p, r))) * len(exponents(E(q, r))) *
                    (len(exponents(E(p, q))) + 1))
            if best is None or cost < best[0]:
                best = (cost, p, q, r)
        _, p, q, r = best
        A, B = labs[p], labs[q]
        epr, eqr = E(p, r), E(q, r)
        if (B, A) < (A, B):
            A, B = B, A
            epr, eqr = eqr, epr
        T = bld.pair_contraction(A, B, E(p, q))
        C = labs[r]
        terms = []
        for al in exponents(epr):
            for be in exponents(eqr):
                terms.append((T[(al, be)], bld.mom(C, _add(al, be)), multinomial(al) * multinomial(be)))
        key = ("S3", A, B, E(p, q), C, epr, eqr)
        return bld.define(key, terms), len(terms)
    # n == 4: pair {p,q} with {r,s}
    best = None
    for (p, q), (r, s) in (((0, 1), (2, 3)), ((0, 2), (1, 3)), ((0, 3), (1, 2))):
        for (pp, qq, rr, ss) in ((p, q, r, s),):
            cross = [E(pp, rr), E(pp, ss), E(qq, rr), E(qq, ss)]
            fin = math.prod(len(exponents(e)) for e in cross)
            tcost = (len(exponents(E(pp, rr) + E(pp, ss))) * len(exponents(E(qq, rr) + E(qq, ss))) *
                     len(exponents(E(pp, qq))))
            ucost = (len(exponents(E(rr, pp) + E(rr, qq))) * len(exponents(E(ss, pp) + E(ss, qq))) *
                     len(exponents(E(rr, ss))))
            cost = fin + tcost + ucost
            if best is None or cost < best[0]:
                best = (cost, pp, qq, rr, ss)
    _, p, q, r, s = best
    # T = M_p x M_q, groups (p: to r,s | q: to r,s); U = M_r x M_s, groups (r: to p,q | s: to p,q)
    A, B = labs[p], labs[q]
    swapT = (B, A) < (A, B)
    if swapT:
        A, B = B, A
    T = bld.pair_contraction(A, B, E(p, q))
    C, D = labs[r], labs[s]
    swapU = (D, C) < (C, D)
    if swapU:
        C, D = D, C
    U = bld.pair_contraction(C, D, E(r, s))
    terms = []
    for a_pr in exponents(E(p, r)):
        for a_ps in exponents(E(p, s)):
            for a_qr in exponents(E(q, r)):
                for a_qs in exponents(E(q, s)):
                    tp, tq = _add(a_pr, a_ps), _add(a_qr, a_qs)
                    ur, us = _add(a_pr, a_qr), _add(a_ps, a_qs)
                    ti = T[(tq, tp)] if swapT else T[(tp, tq)]
                    ui = U[(us, ur)] if swapU else U[(ur, us)]
                    c = (multinomial(a_pr) * multinomial(a_ps) *
                         multinomial(a_qr) * multinomial(a_qs))
                    terms.append((ti, ui, c))
    key = ("S4", bf.labels, bf.edges, tuple(nodes))
    return bld.define(key, terms), len(terms)


def compile_schedule(shape: ModelShape) -> Schedule:
    basis = shape.basis
    moments = sorted({lab for b in basis for lab in b.labels})
    bld = _Builder(moments)
    basis_idx = []
    for bf in basis:
        scalars = []
        for comp in bf.components():
            idx, _ = _component_scalar(bld, bf, comp)
            scalars.append(idx)
        scalars.sort()
        if len(scalars) == 1:
            basis_idx.append(scalars[0])
            continue
        # left-deep products of sorted component scalars (shared prefixes dedup)
        acc = bld.product(scalars[0], scalars[1])
        for x in scalars[2:]:
            acc = bld.product(acc, x)
        basis_idx.append(acc)

    # topological order: definitions only reference earlier values by construction
    dst_ptr = [0]
    tri_a, tri_b, tri_c = [], [], []
    for _, terms in bld.defs:
        for a, b, c in terms:
            tri_a.append(a)
            tri_b.append(b)
            tri_c.append(float(c))
        dst_ptr.append(len(tri_a))
    n_vals = bld.n_mom + len(bld.defs)
    sched = Schedule(moments=moments, mom_off=bld.mom_off, n_mom_comps=bld.n_mom,
                     comp_mu=bld.comp_mu, comp_exp=bld.comp_exp, n_vals=n_vals,
                     first_dst=bld.n_mom, dst_ptr=dst_ptr, tri_a=tri_a, tri_b=tri_b,
                     tri_c=tri_c, basis_idx=basis_idx,
                     nu_max=max(nu for _, nu in moments))
    sched.stats = {"n_moments": len(moments), "n_mom_comps": bld.n_mom,
                   "n_intermediates": len(bld.defs), "n_triples": len(tri_a)}
    return sched

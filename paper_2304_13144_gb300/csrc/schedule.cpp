// Host-side MTP basis enumeration and flattened contraction schedule.
//
// Section II.A (eqs. 3, 5, 6): a basis function B_a is a full contraction of a product of
// moment tensors M_{mu,nu}; the basis of level lev_max is every such contraction with
// sum_p (2 + 4 mu_p + nu_p) <= lev_max.  Reading used (see the design notes): a basis
// function is a multigraph on P <= 4 factors (node = moment, degree = nu, edge = one
// contracted index pair between two different factors, no self-loops); the level-6 example
// of the paper lists exactly these five functions and the counts 26/54/125 of Section IV
// follow.  Canonical form: labels sorted ascending, lexicographically smallest edge vector
// (e01,e02,e03,e12,e13,e23) over label-preserving node permutations; order by
// (level, P, labels, edges).
//
// The schedule keeps moments in symmetric storage (component (a,b,c) = sum_j f_mu x^a y^b z^c)
// and forms every other value as  v[dst] = sum_t c_t v[a_t] v[b_t].  A contraction of k index
// pairs between symmetric tensors A, B is exact with multinomial weights:
//   T[alpha|beta] = sum_{|g| = k} k!/(g1! g2! g3!) A[alpha+g] B[beta+g],
// and intermediates keep their index groups apart, so cyclic graphs are evaluated exactly.
#include "schedule.h"

#include <algorithm>
#include <cstdint>
#include <map>
#include <set>
#include <stdexcept>
#include <tuple>
#include <vector>

namespace mtp {
namespace {

using Label = std::pair<int, int>;  // (mu, nu)
using Exp = std::array<int, 3>;

int moment_level(int mu, int nu) { return 2 + 4 * mu + nu; }

const std::vector<Exp>& exponents(int nu) {
  static std::map<int, std::vector<Exp>> cache;
  auto it = cache.find(nu);
  if (it != cache.end()) return it->second;
  std::vector<Exp> v;
  for (int a = nu; a >= 0; --a)
    for (int b = nu - a; b >= 0; --b) v.push_back({a, b, nu - a - b});
  return cache.emplace(nu, std::move(v)).first->second;
}

double factorial(int n) { double r = 1; for (int k = 2; k <= n; ++k) r *= k; return r; }
double multinomial(const Exp& e) {
  return factorial(e[0] + e[1] + e[2]) / (factorial(e[0]) * factorial(e[1]) * factorial(e[2]));
}
Exp add(const Exp& x, const Exp& y) { return {x[0] + y[0], x[1] + y[1], x[2] + y[2]}; }

const int kPairP[6] = {0, 0, 0, 1, 1, 2};
const int kPairQ[6] = {1, 2, 3, 2, 3, 3};

int npairs(int P) { return P * (P - 1) / 2; }
// index of pair (p,q), p<q, among the first npairs(P) entries of kPairP/kPairQ
int pair_index(int P, int p, int q) {
  if (p > q) std::swap(p, q);
  int k = 0;
  for (int i = 0; i < P; ++i)
    for (int j = i + 1; j < P; ++j, ++k)
      if (i == p && j == q) return k;
  return -1;
}

struct Graph {
  std::vector<Label> labels;
  std::vector<int> edges;  // over pairs of P nodes, in (0,1),(0,2),..,(P-2,P-1) order
  int P() const { return static_cast<int>(labels.size()); }
  int level() const { int s = 0; for (auto& l : labels) s += moment_level(l.first, l.second); return s; }
  int edge(int p, int q) const { return p == q ? 0 : edges[pair_index(P(), p, q)]; }
  bool operator<(const Graph& o) const {
    auto k1 = std::make_tuple(level(), P(), labels, edges);
    auto k2 = std::make_tuple(o.level(), o.P(), o.labels, o.edges);
    return k1 < k2;
  }
};

void edge_vectors(const std::vector<int>& deg, std::vector<std::vector<int>>& out) {
  const int P = static_cast<int>(deg.size());
  std::vector<std::pair<int, int>> pairs;
  for (int i = 0; i < P; ++i)
    for (int j = i + 1; j < P; ++j) pairs.push_back({i, j});
  std::vector<int> rem = deg, cur;
  std::function<void(size_t)> rec = [&](size_t k) {
    if (k == pairs.size()) {
      for (int r : rem) if (r) return;
      out.push_back(cur);
      return;
    }
    int p = pairs[k].first, q = pairs[k].second;
    int hi = std::min(rem[p], rem[q]);
    for (int m = 0; m <= hi; ++m) {
      rem[p] -= m; rem[q] -= m;
      if (!(q == P - 1 && rem[p] != 0)) { cur.push_back(m); rec(k + 1); cur.pop_back(); }
      rem[p] += m; rem[q] += m;
    }
  };
  rec(0);
}

std::vector<int> canonical_edges(const std::vector<Label>& labels, const std::vector<int>& edges) {
  const int P = static_cast<int>(labels.size());
  std::vector<int> best;
  std::vector<int> perm(P);
  for (int i = 0; i < P; ++i) perm[i] = i;
  std::vector<std::vector<int>> emat(P, std::vector<int>(P, 0));
  for (int i = 0, k = 0; i < P; ++i)
    for (int j = i + 1; j < P; ++j, ++k) emat[i][j] = emat[j][i] = edges[k];
  bool first = true;
  do {
    bool ok = true;
    for (int i = 0; i < P; ++i) if (labels[perm[i]] != labels[i]) { ok = false; break; }
    if (!ok) continue;
    std::vector<int> v;
    for (int i = 0; i < P; ++i)
      for (int j = i + 1; j < P; ++j) v.push_back(emat[perm[i]][perm[j]]);
    if (first || v < best) { best = v; first = false; }
  } while (std::next_permutation(perm.begin(), perm.end()));
  return best;
}

std::vector<Graph> enumerate_basis(int lev_max) {
  std::vector<Label> moments;
  for (int mu = 0; mu < lev_max; ++mu)
    for (int nu = 0; nu <= lev_max; ++nu)
      if (moment_level(mu, nu) <= lev_max) moments.push_back({mu, nu});
  std::sort(moments.begin(), moments.end());
  std::set<Graph> found;
  std::vector<Label> labs;
  std::function<void(size_t, int)> rec = [&](size_t start, int level) {
    if (!labs.empty()) {
      std::vector<int> deg;
      for (auto& l : labs) deg.push_back(l.second);
      std::vector<std::vector<int>> evs;
      edge_vectors(deg, evs);
      for (auto& ev : evs) found.insert(Graph{labs, canonical_edges(labs, ev)});
    }
    if (labs.size() == 4) return;
    for (size_t k = start; k < moments.size(); ++k) {
      int L = moment_level(moments[k].first, moments[k].second);
      if (level + L <= lev_max) { labs.push_back(moments[k]); rec(k, level + L); labs.pop_back(); }
    }
  };
  rec(0, 0);
  return std::vector<Graph>(found.begin(), found.end());
}

struct Builder {
  std::vector<Label> moments;
  std::map<std::tuple<int, int, int, int, int>, int> comp_index;  // (mu,nu,a,b,c) -> value
  int n_mom = 0;
  std::vector<int> comp_mu;
  std::vector<Exp> comp_exp;
  std::vector<std::vector<std::tuple<int, int, double>>> defs;
  std::map<std::vector<int>, int> index;

  explicit Builder(const std::vector<Label>& moms) : moments(moms) {
    for (auto& m : moments)
      for (auto& e : exponents(m.second)) {
        comp_index[{m.first, m.second, e[0], e[1], e[2]}] = n_mom++;
        comp_mu.push_back(m.first);
        comp_exp.push_back(e);
      }
  }
  int mom(const Label& l, const Exp& e) const {
    return comp_index.at({l.first, l.second, e[0], e[1], e[2]});
  }
  int define(const std::vector<int>& key, const std::vector<std::tuple<int, int, double>>& terms) {
    auto it = index.find(key);
    if (it != index.end()) return it->second;
    std::map<std::pair<int, int>, double> merged;
    for (auto& t : terms) {
      int a = std::get<0>(t), b = std::get<1>(t);
      if (a > b) std::swap(a, b);
      merged[{a, b}] += std::get<2>(t);
    }
    std::vector<std::tuple<int, int, double>> out;
    for (auto& kv : merged)
      if (kv.second != 0.0) out.push_back({kv.first.first, kv.first.second, kv.second});
    int idx = n_mom + static_cast<int>(defs.size());
    defs.push_back(out);
    index[key] = idx;
    return idx;
  }
  static void push_label(std::vector<int>& k, const Label& l) { k.push_back(l.first); k.push_back(l.second); }
  static void push_exp(std::vector<int>& k, const Exp& e) { k.push_back(e[0]); k.push_back(e[1]); k.push_back(e[2]); }

  // T[alpha|beta] = A x_k B; returns table indexed [alpha idx][beta idx] of exponents(nuA-k) x exponents(nuB-k)
  std::vector<std::vector<int>> pair_contraction(const Label& A, const Label& B, int k) {
    const auto& ea = exponents(A.second - k);
    const auto& eb = exponents(B.second - k);
    std::vector<std::vector<int>> table(ea.size(), std::vector<int>(eb.size()));
    // A x_k A is symmetric under exchange of its two index groups: T[alpha|beta] = T[beta|alpha]
    const bool sym = (A == B);
    for (size_t i = 0; i < ea.size(); ++i)
      for (size_t j = 0; j < eb.size(); ++j) {
        if (sym && j < i) { table[i][j] = table[j][i]; continue; }
        std::vector<int> key = {1};
        push_label(key, A); push_label(key, B); key.push_back(k);
        push_exp(key, ea[i]); push_exp(key, eb[j]);
        std::vector<std::tuple<int, int, double>> terms;
        for (auto& g : exponents(k))
          terms.push_back({mom(A, add(ea[i], g)), mom(B, add(eb[j], g)), multinomial(g)});
        table[i][j] = define(key, terms);
      }
    return table;
  }
  int product(int x, int y) {
    int a = std::min(x, y), b = std::max(x, y);
    return define({2, a, b}, {{a, b, 1.0}});
  }
};

int exp_pos(int nu, const Exp& e) {
  const auto& v = exponents(nu);
  for (size_t i = 0; i < v.size(); ++i) if (v[i] == e) return static_cast<int>(i);
  throw std::logic_error("exponent not found");
}

int component_scalar(Builder& bld, const Graph& g, const std::vector<int>& nodes) {
  const int n = static_cast<int>(nodes.size());
  std::vector<Label> labs;
  for (int p : nodes) labs.push_back(g.labels[p]);
  auto E = [&](int i, int j) { return g.edge(nodes[i], nodes[j]); };
  auto nexp = [](int e) { return static_cast<long>(exponents(e).size()); };
  if (n == 1) return bld.mom(labs[0], {0, 0, 0});
  if (n == 2) {
    Label A = labs[0], B = labs[1];
    if (B < A) std::swap(A, B);
    std::vector<int> key = {3};
    Builder::push_label(key, A); Builder::push_label(key, B);
    std::vector<std::tuple<int, int, double>> terms;
    for (auto& e : exponents(A.second)) terms.push_back({bld.mom(A, e), bld.mom(B, e), multinomial(e)});
    return bld.define(key, terms);
  }
  if (n == 3) {
    long best = -1; int bp = 0, bq = 0, br = 0;
    for (int r = 0; r < 3; ++r) {
      int p = r == 0 ? 1 : 0, q = r == 2 ? 1 : 2;
      long cost = nexp(E(p, r)) * nexp(E(q, r)) * (nexp(E(p, q)) + 1);
      if (best < 0 || cost < best) { best = cost; bp = p; bq = q; br = r; }
    }
    Label A = labs[bp], B = labs[bq];
    int epr = E(bp, br), eqr = E(bq, br), epq = E(bp, bq);
    if (B < A) { std::swap(A, B); std::swap(epr, eqr); }
    auto T = bld.pair_contraction(A, B, epq);
    Label C = labs[br];
    std::vector<int> key = {4};
    Builder::push_label(key, A); Builder::push_label(key, B); key.push_back(epq);
    Builder::push_label(key, C); key.push_back(epr); key.push_back(eqr);
    std::vector<std::tuple<int, int, double>> terms;
    const auto& ea = exponents(epr);
    const auto& eb = exponents(eqr);
    for (size_t i = 0; i < ea.size(); ++i)
      for (size_t j = 0; j < eb.size(); ++j)
        terms.push_back({T[i][j], bld.mom(C, add(ea[i], eb[j])), multinomial(ea[i]) * multinomial(eb[j])});
    return bld.define(key, terms);
  }
  // n == 4: pair {p,q} with {r,s}
  const int pairings[3][4] = {{0, 1, 2, 3}, {0, 2, 1, 3}, {0, 3, 1, 2}};
  long best = -1; int sel = 0;
  for (int t = 0; t < 3; ++t) {
    int p = pairings[t][0], q = pairings[t][1], r = pairings[t][2], s = pairings[t][3];
    long fin = nexp(E(p, r)) * nexp(E(p, s)) * nexp(E(q, r)) * nexp(E(q, s));
    long tc = nexp(E(p, r) + E(p, s)) * nexp(E(q, r) + E(q, s)) * nexp(E(p, q));
    long uc = nexp(E(r, p) + E(r, q)) * nexp(E(s, p) + E(s, q)) * nexp(E(r, s));
    long cost = fin + tc + uc;
    if (best < 0 || cost < best) { best = cost; sel = t; }
  }
  int p = pairings[sel][0], q = pairings[sel][1], r = pairings[sel][2], s = pairings[sel][3];
  Label A = labs[p], B = labs[q];
  bool swapT = B < A;
  if (swapT) std::swap(A, B);
  auto T = bld.pair_contraction(A, B, E(p, q));
  Label C = labs[r], D = labs[s];
  bool swapU = D < C;
  if (swapU) std::swap(C, D);
  auto U = bld.pair_contraction(C, D, E(r, s));
  int ntp = E(p, r) + E(p, s), ntq = E(q, r) + E(q, s);
  int nur = E(p, r) + E(q, r), nus = E(p, s) + E(q, s);
  std::vector<std::tuple<int, int, double>> terms;
  for (auto& a_pr : exponents(E(p, r)))
    for (auto& a_ps : exponents(E(p, s)))
      for (auto& a_qr : exponents(E(q, r)))
        for (auto& a_qs : exponents(E(q, s))) {
          int itp = exp_pos(ntp, add(a_pr, a_ps)), itq = exp_pos(ntq, add(a_qr, a_qs));
          int iur = exp_pos(nur, add(a_pr, a_qr)), ius = exp_pos(nus, add(a_ps, a_qs));
          int ti = swapT ? T[itq][itp] : T[itp][itq];
          int ui = swapU ? U[ius][iur] : U[iur][ius];
          double c = multinomial(a_pr) * multinomial(a_ps) * multinomial(a_qr) * multinomial(a_qs);
          terms.push_back({ti, ui, c});
        }
  std::vector<int> key = {5};
  for (auto& l : g.labels) Builder::push_label(key, l);
  key.push_back(-1);
  for (int e : g.edges) key.push_back(e);
  key.push_back(-1);
  for (int x : nodes) key.push_back(x);
  return bld.define(key, terms);
}

std::vector<std::vector<int>> components(const Graph& g) {
  const int P = g.P();
  std::vector<bool> seen(P, false);
  std::vector<std::vector<int>> comps;
  for (int s = 0; s < P; ++s) {
    if (seen[s]) continue;
    std::vector<int> comp, stack = {s};
    seen[s] = true;
    while (!stack.empty()) {
      int a = stack.back(); stack.pop_back();
      comp.push_back(a);
      for (int b = 0; b < P; ++b)
        if (!seen[b] && g.edge(a, b) > 0) { seen[b] = true; stack.push_back(b); }
    }
    std::sort(comp.begin(), comp.end());
    comps.push_back(comp);
  }
  return comps;
}

}  // namespace

Schedule build_schedule(int n_types, int lev_max, int n_q) {
  if (n_types < 1 || n_types > 64 || lev_max < 2 || lev_max > 28 || n_q < 1 || n_q > 32)
    throw std::invalid_argument("descriptor out of range");
  std::vector<Graph> basis = enumerate_basis(lev_max);
  if (basis.empty()) throw std::invalid_argument("empty basis");
  Schedule S;
  S.n_types = n_types; S.lev_max = lev_max; S.n_q = n_q;
  S.n_lin = static_cast<int>(basis.size());
  int max_mu = 0;
  std::set<Label> used;
  for (auto& g : basis)
    for (auto& l : g.labels) { used.insert(l); max_mu = std::max(max_mu, l.first); }
  S.n_rad = max_mu + 1;
  S.n_params = static_cast<int64_t>(n_types) + S.n_lin +
               static_cast<int64_t>(n_types) * n_types * S.n_rad * n_q;
  std::vector<Label> moments(used.begin(), used.end());
  for (auto& g : basis) {
    S.basis_P.push_back(g.P());
    std::array<int, 4> mu{0, 0, 0, 0}, nu{0, 0, 0, 0};
    std::array<int, 6> ed{0, 0, 0, 0, 0, 0};
    for (int p = 0; p < g.P(); ++p) { mu[p] = g.labels[p].first; nu[p] = g.labels[p].second; }
    for (int i = 0, k = 0; i < g.P(); ++i)
      for (int j = i + 1; j < g.P(); ++j, ++k) {
        int e6 = 0;
        for (int t = 0; t < 6; ++t) if (kPairP[t] == i && kPairQ[t] == j) e6 = t;
        ed[e6] = g.edges[k];
      }
    S.basis_mu.push_back(mu); S.basis_nu.push_back(nu); S.basis_edges.push_back(ed);
  }
  Builder bld(moments);
  for (auto& g : basis) {
    std::vector<int> scal;
    for (auto& comp : components(g)) scal.push_back(component_scalar(bld, g, comp));
    std::sort(scal.begin(), scal.end());
    if (scal.size() == 1) { S.basis_idx.push_back(scal[0]); continue; }
    int acc = bld.product(scal[0], scal[1]);
    for (size_t k = 2; k < scal.size(); ++k) acc = bld.product(acc, scal[k]);
    S.basis_idx.push_back(acc);
  }
  S.n_mom_comps = bld.n_mom;
  S.comp_mu = bld.comp_mu;
  S.comp_exp = bld.comp_exp;
  S.n_moments = static_cast<int>(moments.size());
  S.nu_max = 0;
  for (auto& m : moments) S.nu_max = std::max(S.nu_max, m.second);
  S.dst_ptr.push_back(0);
  for (auto& d : bld.defs) {
    for (auto& t : d) {
      S.tri_a.push_back(std::get<0>(t));
      S.tri_b.push_back(std::get<1>(t));
      S.tri_c.push_back(std::get<2>(t));
    }
    S.dst_ptr.push_back(static_cast<int>(S.tri_a.size()));
  }
  S.n_values = bld.n_mom + static_cast<int>(bld.defs.size());
  return S;
}

// Null directions of the parameter rows.  Mixing the radial functions, f_mu -> f_mu + eps f_mu'
// (mu' <= mu, i.e. c[.][.][mu][.] += eps c[.][.][mu'][.], eq. 4), turns to first order every
// basis function with a factor M_{mu,nu} into itself plus eps times the function with that
// factor relabelled M_{mu',nu}, which has a lower level and so is again a basis function
// (eqs. 5-6).  Moving eps xi_a onto that function leaves V unchanged, so the derivative of
// theta along this change is orthogonal to every parameter row b_i = dV_i/dtheta.
// D: n_rad (n_rad + 1) / 2 rows of n_params, ordered by (mu, mu').
void gauge_directions(const Schedule& S, const double* theta, double* D) {
  const int T = S.n_types, NR = S.n_rad, NQ = S.n_q, NL = S.n_lin;
  std::map<std::pair<std::vector<Label>, std::vector<int>>, int> index;
  std::vector<std::vector<Label>> labels(NL);
  std::vector<std::vector<std::vector<int>>> mats(NL);
  for (int a = 0; a < NL; ++a) {
    const int P = S.basis_P[a];
    for (int p = 0; p < P; ++p) labels[a].push_back({S.basis_mu[a][p], S.basis_nu[a][p]});
    mats[a].assign(P, std::vector<int>(P, 0));
    std::vector<int> ev;
    for (int i = 0; i < P; ++i)
      for (int j = i + 1; j < P; ++j) {
        int e6 = 0;
        for (int t = 0; t < 6; ++t) if (kPairP[t] == i && kPairQ[t] == j) e6 = t;
        mats[a][i][j] = mats[a][j][i] = S.basis_edges[a][e6];
        ev.push_back(S.basis_edges[a][e6]);
      }
    index[{labels[a], ev}] = a;
  }
  const int64_t m = S.n_params;
  int row = 0;
  for (int mu = 0; mu < NR; ++mu)
    for (int mu2 = 0; mu2 <= mu; ++mu2, ++row) {
      double* d = D + static_cast<int64_t>(row) * m;
      for (int64_t k = 0; k < m; ++k) d[k] = 0.0;
      for (int zi = 0; zi < T; ++zi)
        for (int zj = 0; zj < T; ++zj)
          for (int b = 0; b < NQ; ++b) {
            const int64_t base = T + NL + ((static_cast<int64_t>(zi) * T + zj) * NR) * NQ;
            d[base + mu * NQ + b] = theta[base + mu2 * NQ + b];
          }
      for (int a = 0; a < NL; ++a) {
        const int P = S.basis_P[a];
        for (int p = 0; p < P; ++p) {
          if (labels[a][p].first != mu) continue;
          std::vector<Label> nl = labels[a];
          nl[p].first = mu2;
          std::vector<int> order(P);
          for (int k = 0; k < P; ++k) order[k] = k;
          std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return nl[x] < nl[y]; });
          std::vector<Label> sl;
          for (int k : order) sl.push_back(nl[k]);
          std::vector<int> ev;
          for (int i = 0; i < P; ++i)
            for (int j = i + 1; j < P; ++j) ev.push_back(mats[a][order[i]][order[j]]);
          auto it = index.find({sl, canonical_edges(sl, ev)});
          if (it == index.end()) throw std::logic_error("relabelled basis function not in the basis");
          d[T + it->second] -= theta[T + a];
        }
      }
    }
}

}  // namespace mtp

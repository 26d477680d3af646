// FP64 CPU oracle for the Moment Tensor Potential hot path.
//
// TEST INFRASTRUCTURE ONLY: tests/, the package smoke check and the CPU-baseline leg of
// bench.py load this library.  The CUDA library never links, includes or calls it, and
// it shares no code, table or helper with the CUDA sources.
//
// Everything here is the plain definition written out, in double precision:
//   * neighborhoods (Section II.A): every (j, image) with 0 < |r_ij| < R_cut, found by
//     brute force over all atoms and all periodic images, or by a plain cell list;
//   * radial functions (eq. 4): f_mu = sum_beta c[z_i][z_j][mu][beta] T_beta(x) (R_cut-|r|)^2,
//     T_beta the Chebyshev polynomials of the first kind on [R_min, R_cut] (reading R1);
//   * moments (eq. 3) as FULL 3^nu tensors: M[a1..anu] = sum_j f_mu prod_k r_j[a_k];
//   * basis functions (eqs. 5-6): for a multigraph of moment factors, the sum over all
//     3^(#contracted indices) index assignments of the product of the factors' entries;
//   * site energy (eq. 2, plus one constant per species): V = s_{z_i} + sum_a xi_a B_a;
//   * derivatives by the product and chain rules written out directly (no tape);
//   * per-atom parameter row b_i = dV_i/dtheta (eq. 9);
//   * grade (Section II.D): LU with partial pivoting of A^T, solve A^T y = b^T, gamma = max|y|;
//   * tangents for the loss gradient (eq. 7): the same site code on dual numbers.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

namespace {

struct Dual {
  double v, d;
  Dual() : v(0), d(0) {}
  Dual(double x) : v(x), d(0) {}
  Dual(double x, double dx) : v(x), d(dx) {}
};
inline Dual operator+(const Dual& a, const Dual& b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(const Dual& a, const Dual& b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator*(const Dual& a, const Dual& b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual operator/(const Dual& a, const Dual& b) {
  return Dual(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v));
}
inline Dual& operator+=(Dual& a, const Dual& b) { a.v += b.v; a.d += b.d; return a; }
inline Dual& operator-=(Dual& a, const Dual& b) { a.v -= b.v; a.d -= b.d; return a; }
inline Dual sqrt_of(const Dual& a) { double s = std::sqrt(a.v); return Dual(s, a.d / (2.0 * s)); }
inline double sqrt_of(double a) { return std::sqrt(a); }
inline double value_of(double a) { return a; }
inline double value_of(const Dual& a) { return a.v; }
inline double tangent_of(double) { return 0.0; }
inline double tangent_of(const Dual& a) { return a.d; }

long ipow3(int n) { long r = 1; for (int k = 0; k < n; ++k) r *= 3; return r; }

// Edge slots of the upper triangle of a 4-node multigraph.
const int kPairP[6] = {0, 0, 0, 1, 1, 2};
const int kPairQ[6] = {1, 2, 3, 2, 3, 3};

struct BasisPlan {
  int P;
  int mom[4];               // index into Model::moms
  int nu[4];
  std::vector<int> slot[4]; // contracted-index variable of each tensor slot
  int nidx;
};

struct Model {
  int T, nq, nrad, nlin, m;
  double rmin, rcut;
  const double* theta;
  std::vector<int> mom_mu, mom_nu;   // used moments
  std::vector<BasisPlan> plans;

  double s(int z) const { return theta[z]; }
  double xi(int a) const { return theta[T + a]; }
  double c(int zi, int zj, int mu, int beta) const {
    return theta[T + nlin + ((static_cast<long>(zi) * T + zj) * nrad + mu) * nq + beta];
  }
  long c_index(int zi, int zj, int mu, int beta) const {
    return T + nlin + ((static_cast<long>(zi) * T + zj) * nrad + mu) * nq + beta;
  }
};

Model make_model(int T, int nq, int nrad, int nlin, double rmin, double rcut,
                 const int32_t* bP, const int32_t* bmu, const int32_t* bnu, const int32_t* bed,
                 const double* theta) {
  Model md;
  md.T = T; md.nq = nq; md.nrad = nrad; md.nlin = nlin;
  md.m = T + nlin + T * T * nrad * nq;
  md.rmin = rmin; md.rcut = rcut; md.theta = theta;
  for (int a = 0; a < nlin; ++a) {
    BasisPlan bp;
    bp.P = bP[a];
    for (int p = 0; p < bp.P; ++p) {
      int mu = bmu[4 * a + p], nu = bnu[4 * a + p];
      int id = -1;
      for (size_t k = 0; k < md.mom_mu.size(); ++k)
        if (md.mom_mu[k] == mu && md.mom_nu[k] == nu) id = static_cast<int>(k);
      if (id < 0) { id = static_cast<int>(md.mom_mu.size()); md.mom_mu.push_back(mu); md.mom_nu.push_back(nu); }
      bp.mom[p] = id;
      bp.nu[p] = nu;
    }
    bp.nidx = 0;
    for (int e = 0; e < 6; ++e) {
      int mult = bed[6 * a + e];
      for (int t = 0; t < mult; ++t) {
        bp.slot[kPairP[e]].push_back(bp.nidx);
        bp.slot[kPairQ[e]].push_back(bp.nidx);
        bp.nidx++;
      }
    }
    md.plans.push_back(bp);
  }
  return md;
}

// Chebyshev values and x-derivatives by the three-term recurrence.
template <class S>
void chebyshev(const S& x, int n, std::vector<S>& t, std::vector<S>& dt) {
  t.assign(n, S(0.0));
  dt.assign(n, S(0.0));
  if (n > 0) { t[0] = S(1.0); dt[0] = S(0.0); }
  if (n > 1) { t[1] = x; dt[1] = S(1.0); }
  for (int k = 1; k + 1 < n; ++k) {
    t[k + 1] = S(2.0) * x * t[k] - t[k - 1];
    dt[k + 1] = S(2.0) * t[k] + S(2.0) * x * dt[k] - dt[k - 1];
  }
}

// Radial basis Q_beta(r) and dQ_beta/dr (eq. 4).
template <class S>
void radial_basis(const Model& md, const S& r, std::vector<S>& Q, std::vector<S>& dQ) {
  S x = (S(2.0) * r - S(md.rmin + md.rcut)) / S(md.rcut - md.rmin);
  std::vector<S> t, dt;
  chebyshev(x, md.nq, t, dt);
  S w = S(md.rcut) - r;
  Q.resize(md.nq);
  dQ.resize(md.nq);
  for (int b = 0; b < md.nq; ++b) {
    Q[b] = t[b] * w * w;
    dQ[b] = dt[b] * S(2.0 / (md.rcut - md.rmin)) * w * w - S(2.0) * t[b] * w;
  }
}

template <class S>
struct SiteResult {
  S V;
  std::vector<S> B;                 // basis values
  std::vector<S> dVdr;              // 3 per pair
  std::vector<S> dVdc;              // T * nrad * nq  (block of this site's z_i)
};

// One site: moments, basis, energy, and (optionally) its derivatives.
template <class S>
void site(const Model& md, int zi, int npair, const int32_t* zj, const S* rv,
          bool want_grad, SiteResult<S>& out) {
  const int nm = static_cast<int>(md.mom_mu.size());
  std::vector<S> r(npair);
  std::vector<std::vector<S>> Q(npair), dQ(npair);
  std::vector<std::vector<S>> f(npair), df(npair);
  for (int j = 0; j < npair; ++j) {
    S d2 = rv[3 * j] * rv[3 * j] + rv[3 * j + 1] * rv[3 * j + 1] + rv[3 * j + 2] * rv[3 * j + 2];
    r[j] = sqrt_of(d2);
    radial_basis(md, r[j], Q[j], dQ[j]);
    f[j].assign(md.nrad, S(0.0));
    df[j].assign(md.nrad, S(0.0));
    for (int mu = 0; mu < md.nrad; ++mu)
      for (int b = 0; b < md.nq; ++b) {
        f[j][mu] += S(md.c(zi, zj[j], mu, b)) * Q[j][b];
        df[j][mu] += S(md.c(zi, zj[j], mu, b)) * dQ[j][b];
      }
  }
  // Moments as full tensors, eq. 3.
  std::vector<std::vector<S>> M(nm);
  for (int k = 0; k < nm; ++k) {
    int mu = md.mom_mu[k], nu = md.mom_nu[k];
    long n = ipow3(nu);
    M[k].assign(n, S(0.0));
    std::vector<int> dig(nu);
    for (long idx = 0; idx < n; ++idx) {
      long t = idx;
      for (int s = nu - 1; s >= 0; --s) { dig[s] = static_cast<int>(t % 3); t /= 3; }
      for (int j = 0; j < npair; ++j) {
        S prod = f[j][mu];
        for (int s = 0; s < nu; ++s) prod = prod * rv[3 * j + dig[s]];
        M[k][idx] += prod;
      }
    }
  }
  // Basis functions by explicit index loops; gradient of V w.r.t. every moment entry.
  std::vector<std::vector<S>> G(nm);
  for (int k = 0; k < nm; ++k) G[k].assign(M[k].size(), S(0.0));
  out.B.assign(md.nlin, S(0.0));
  S V = S(md.s(zi));
  for (int a = 0; a < md.nlin; ++a) {
    const BasisPlan& bp = md.plans[a];
    long n = ipow3(bp.nidx);
    std::vector<int> asg(bp.nidx);
    S Ba = S(0.0);
    for (long it = 0; it < n; ++it) {
      long t = it;
      for (int v = bp.nidx - 1; v >= 0; --v) { asg[v] = static_cast<int>(t % 3); t /= 3; }
      long ent[4];
      S val[4] = {S(0.0), S(0.0), S(0.0), S(0.0)};
      for (int p = 0; p < bp.P; ++p) {
        long e = 0;
        for (int s = 0; s < bp.nu[p]; ++s) e = e * 3 + asg[bp.slot[p][s]];
        ent[p] = e;
        val[p] = M[bp.mom[p]][e];
      }
      S term = val[0];
      for (int p = 1; p < bp.P; ++p) term = term * val[p];
      Ba += term;
      if (want_grad) {
        for (int p = 0; p < bp.P; ++p) {
          S others = S(md.xi(a));
          for (int q = 0; q < bp.P; ++q)
            if (q != p) others = others * val[q];
          G[bp.mom[p]][ent[p]] += others;
        }
      }
    }
    out.B[a] = Ba;
    V += S(md.xi(a)) * Ba;
  }
  out.V = V;
  if (!want_grad) return;
  // Per pair: dV/dr_j = sum over moment entries G * d(f_mu(|r|) prod_k r[a_k])/dr.
  out.dVdr.assign(3 * npair, S(0.0));
  out.dVdc.assign(static_cast<size_t>(md.T) * md.nrad * md.nq, S(0.0));
  for (int j = 0; j < npair; ++j) {
    std::vector<S> gmu(md.nrad, S(0.0));
    S grad[3] = {S(0.0), S(0.0), S(0.0)};
    for (int k = 0; k < nm; ++k) {
      int mu = md.mom_mu[k], nu = md.mom_nu[k];
      long n = ipow3(nu);
      std::vector<int> dig(nu);
      S gP = S(0.0);
      S gdP[3] = {S(0.0), S(0.0), S(0.0)};
      for (long idx = 0; idx < n; ++idx) {
        long t = idx;
        for (int s = nu - 1; s >= 0; --s) { dig[s] = static_cast<int>(t % 3); t /= 3; }
        S P = S(1.0);
        for (int s = 0; s < nu; ++s) P = P * rv[3 * j + dig[s]];
        gP += G[k][idx] * P;
        for (int s = 0; s < nu; ++s) {
          S partial = S(1.0);
          for (int u = 0; u < nu; ++u)
            if (u != s) partial = partial * rv[3 * j + dig[u]];
          gdP[dig[s]] += G[k][idx] * partial;
        }
      }
      gmu[mu] += gP;
      for (int c = 0; c < 3; ++c)
        grad[c] += df[j][mu] * rv[3 * j + c] / r[j] * gP + f[j][mu] * gdP[c];
    }
    for (int c = 0; c < 3; ++c) out.dVdr[3 * j + c] = grad[c];
    for (int mu = 0; mu < md.nrad; ++mu)
      for (int b = 0; b < md.nq; ++b)
        out.dVdc[(static_cast<long>(zj[j]) * md.nrad + mu) * md.nq + b] += gmu[mu] * Q[j][b];
  }
}

}  // namespace

extern "C" {

// Neighbor list of every atom of one configuration (Section II.A): all (j, image n) with
// 0 < |r_ij| < R_cut, r_ij = (x_j + n.H) - x_i, H rows = lattice vectors, n[a] = 0 on
// non-periodic axes.  brute != 0: every atom against every atom over the image range;
// brute == 0: a plain cell list (fully periodic cells only).  Output per pair: j, the
// integer image (3 ints, relative to the given unwrapped positions) and r_ij.
// Returns the number of pairs; if it exceeds cap only off[] is filled.  Returns -1 on
// coincident atoms, -2 on an unsupported request.
int64_t oracle_neighbors(int64_t n, const double* pos, const double* cell, const uint8_t* pbc,
                         double rcut, int brute, int64_t cap, int64_t* off, int32_t* nj,
                         int32_t* nimg, double* nr) {
  const double* H = cell;
  double c0[3] = {H[4] * H[8] - H[5] * H[7], H[5] * H[6] - H[3] * H[8], H[3] * H[7] - H[4] * H[6]};
  double c1[3] = {H[7] * H[2] - H[8] * H[1], H[8] * H[0] - H[6] * H[2], H[6] * H[1] - H[7] * H[0]};
  double c2[3] = {H[1] * H[5] - H[2] * H[4], H[2] * H[3] - H[0] * H[5], H[0] * H[4] - H[1] * H[3]};
  double vol = H[0] * c0[0] + H[1] * c0[1] + H[2] * c0[2];
  // inverse: Hinv[c][a] = cof[a][c] / vol  (s = x Hinv)
  double Hinv[9];
  for (int c = 0; c < 3; ++c) { Hinv[c * 3 + 0] = c0[c] / vol; Hinv[c * 3 + 1] = c1[c] / vol; Hinv[c * 3 + 2] = c2[c] / vol; }
  double h[3] = {std::fabs(vol) / std::sqrt(c0[0] * c0[0] + c0[1] * c0[1] + c0[2] * c0[2]),
                 std::fabs(vol) / std::sqrt(c1[0] * c1[0] + c1[1] * c1[1] + c1[2] * c1[2]),
                 std::fabs(vol) / std::sqrt(c2[0] * c2[0] + c2[1] * c2[1] + c2[2] * c2[2])};
  // wrap periodic fractional coordinates into [0,1)
  std::vector<double> s(3 * n);
  std::vector<int> w(3 * n, 0);
  for (int64_t i = 0; i < n; ++i)
    for (int a = 0; a < 3; ++a) {
      double v = pos[3 * i] * Hinv[0 * 3 + a] + pos[3 * i + 1] * Hinv[1 * 3 + a] + pos[3 * i + 2] * Hinv[2 * 3 + a];
      if (pbc[a]) { double fl = std::floor(v); w[3 * i + a] = static_cast<int>(fl); v -= fl; if (v >= 1.0) v -= 1.0; }
      s[3 * i + a] = v;
    }
  auto pair_vec = [&](int64_t i, int64_t j, const int img[3], double out[3]) {
    for (int c = 0; c < 3; ++c) {
      double sh = img[0] * H[0 * 3 + c] + img[1] * H[1 * 3 + c] + img[2] * H[2 * 3 + c];
      out[c] = (pos[3 * j + c] + sh) - pos[3 * i + c];
    }
  };
  const double rc2 = rcut * rcut;
  int64_t total = 0;
  bool overflow = false;
  auto emit = [&](int64_t i, int64_t j, const int nrel[3]) -> int {
    // nrel is the image between wrapped positions x' = x - w.H; for the given (unwrapped)
    // positions the same vector is x_j + (nrel - w_j + w_i).H - x_i.
    int img[3];
    for (int a = 0; a < 3; ++a) img[a] = nrel[a] - w[3 * j + a] + w[3 * i + a];
    double rv[3];
    pair_vec(i, j, img, rv);
    double d2 = rv[0] * rv[0] + rv[1] * rv[1] + rv[2] * rv[2];
    if (d2 >= rc2) return 0;
    if (d2 == 0.0) return -1;
    if (total < cap) {
      nj[total] = static_cast<int32_t>(j);
      for (int a = 0; a < 3; ++a) { nimg[3 * total + a] = img[a]; nr[3 * total + a] = rv[a]; }
    } else {
      overflow = true;
    }
    total++;
    return 0;
  };
  if (brute) {
    int K[3];
    for (int a = 0; a < 3; ++a) K[a] = pbc[a] ? static_cast<int>(std::ceil(rcut / h[a])) + 1 : 0;
    for (int64_t i = 0; i < n; ++i) {
      off[i] = total;
      for (int n0 = -K[0]; n0 <= K[0]; ++n0)
        for (int n1 = -K[1]; n1 <= K[1]; ++n1)
          for (int n2 = -K[2]; n2 <= K[2]; ++n2)
            for (int64_t j = 0; j < n; ++j) {
              if (j == i && n0 == 0 && n1 == 0 && n2 == 0) continue;
              int nrel[3] = {n0, n1, n2};
              if (emit(i, j, nrel) < 0) return -1;
            }
    }
    off[n] = total;
    return total;
  }
  if (!(pbc[0] && pbc[1] && pbc[2])) return -2;
  int nb[3], kb[3];
  for (int a = 0; a < 3; ++a) {
    nb[a] = std::max(1, static_cast<int>(std::floor(h[a] / rcut)));
    kb[a] = static_cast<int>(std::ceil(rcut * nb[a] / h[a]));
  }
  long nbins = static_cast<long>(nb[0]) * nb[1] * nb[2];
  std::vector<std::vector<int64_t>> bins(nbins);
  std::vector<int> bi(3 * n);
  for (int64_t i = 0; i < n; ++i) {
    for (int a = 0; a < 3; ++a) bi[3 * i + a] = std::min(nb[a] - 1, static_cast<int>(std::floor(s[3 * i + a] * nb[a])));
    bins[(static_cast<long>(bi[3 * i]) * nb[1] + bi[3 * i + 1]) * nb[2] + bi[3 * i + 2]].push_back(i);
  }
  for (int64_t i = 0; i < n; ++i) {
    off[i] = total;
    for (int d0 = -kb[0]; d0 <= kb[0]; ++d0)
      for (int d1 = -kb[1]; d1 <= kb[1]; ++d1)
        for (int d2 = -kb[2]; d2 <= kb[2]; ++d2) {
          int d[3] = {d0, d1, d2}, t[3], nrel[3];
          for (int a = 0; a < 3; ++a) {
            int tt = bi[3 * i + a] + d[a];
            int q = static_cast<int>(std::floor(static_cast<double>(tt) / nb[a]));
            t[a] = tt - q * nb[a];
            nrel[a] = q;
          }
          const auto& lst = bins[(static_cast<long>(t[0]) * nb[1] + t[1]) * nb[2] + t[2]];
          for (int64_t j : lst) {
            if (j == i && nrel[0] == 0 && nrel[1] == 0 && nrel[2] == 0) continue;
            if (emit(i, j, nrel) < 0) return -1;
          }
        }
  }
  off[n] = total;
  (void)overflow;
  return total;
}

// Site quantities for a list of requested atoms.
//   Model: T types, nq Chebyshev polynomials, nrad radial functions, nlin basis functions
//   given as (P, mu[4], nu[4], edges[6]) per function; theta = [s | xi | c].
//   Neighbor data: nb_off (per atom CSR), nb_j, nb_r (3 per pair, r_ij).
//   nb_rdot (3 per pair) or NULL: tangent direction of every r_ij; with it the outputs
//   V_dot and b_dot hold d/dt of V_i and b_i along that direction (dual numbers).
//   Outputs (any may be NULL): V (n_req), dVdr (3 per pair, written at the global pair
//   index of each requested atom's pairs), b (n_req x m), V_dot (n_req), b_dot (n_req x m).
int oracle_sites(int T, int nq, int nrad, int nlin, double rmin, double rcut,
                 const int32_t* bP, const int32_t* bmu, const int32_t* bnu, const int32_t* bed,
                 const double* theta, int64_t n_req, const int64_t* req, const int32_t* types,
                 const int64_t* nb_off, const int32_t* nb_j, const double* nb_r,
                 const double* nb_rdot, double* V, double* dVdr, double* b, double* V_dot,
                 double* b_dot) {
  Model md = make_model(T, nq, nrad, nlin, rmin, rcut, bP, bmu, bnu, bed, theta);
  const bool want_grad = (dVdr != nullptr) || (b != nullptr) || (b_dot != nullptr);
  const int m = md.m;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t k = 0; k < n_req; ++k) {
    int64_t i = req[k];
    int zi = types[i];
    int64_t p0 = nb_off[i], p1 = nb_off[i + 1];
    int np = static_cast<int>(p1 - p0);
    std::vector<int32_t> zj(np);
    for (int q = 0; q < np; ++q) zj[q] = types[nb_j[p0 + q]];
    if (nb_rdot == nullptr) {
      SiteResult<double> out;
      site<double>(md, zi, np, zj.data(), nb_r + 3 * p0, want_grad, out);
      if (V) V[k] = out.V;
      if (dVdr) for (int q = 0; q < 3 * np; ++q) dVdr[3 * p0 + q] = out.dVdr[q];
      if (b) {
        double* row = b + k * m;
        for (int q = 0; q < m; ++q) row[q] = 0.0;
        row[zi] = 1.0;
        for (int a = 0; a < nlin; ++a) row[T + a] = out.B[a];
        for (int zj2 = 0; zj2 < T; ++zj2)
          for (int mu = 0; mu < nrad; ++mu)
            for (int be = 0; be < nq; ++be)
              row[md.c_index(zi, zj2, mu, be)] = out.dVdc[(static_cast<long>(zj2) * nrad + mu) * nq + be];
      }
    } else {
      std::vector<Dual> rv(3 * np);
      for (int q = 0; q < 3 * np; ++q) rv[q] = Dual(nb_r[3 * p0 + q], nb_rdot[3 * p0 + q]);
      SiteResult<Dual> out;
      site<Dual>(md, zi, np, zj.data(), rv.data(), want_grad, out);
      if (V) V[k] = out.V.v;
      if (V_dot) V_dot[k] = out.V.d;
      if (dVdr) for (int q = 0; q < 3 * np; ++q) dVdr[3 * p0 + q] = out.dVdr[q].v;
      double* rows[2] = {b ? b + k * m : nullptr, b_dot ? b_dot + k * m : nullptr};
      for (int w = 0; w < 2; ++w) {
        double* row = rows[w];
        if (!row) continue;
        for (int q = 0; q < m; ++q) row[q] = 0.0;
        if (w == 0) row[zi] = 1.0;
        for (int a = 0; a < nlin; ++a) row[T + a] = w == 0 ? out.B[a].v : out.B[a].d;
        for (int zj2 = 0; zj2 < T; ++zj2)
          for (int mu = 0; mu < nrad; ++mu)
            for (int be = 0; be < nq; ++be) {
              const Dual& g = out.dVdc[(static_cast<long>(zj2) * nrad + mu) * nq + be];
              row[md.c_index(zi, zj2, mu, be)] = w == 0 ? g.v : g.d;
            }
      }
    }
  }
  return 0;
}

// Extrapolation grade (Section II.D): for every row b_k, c = b_k A^{-1} by LU with partial
// pivoting of A^T (textbook Doolittle) and two triangular solves; gamma_k = max_p |c_p|,
// argmax_k = the lowest p attaining it.  Ainv (m x m, row-major) is written if non-NULL.
// Returns -1 if a pivot is exactly zero.
int oracle_grade(int64_t m, const double* A, int64_t n, const double* brows, double* gamma,
                 int32_t* argmax, double* Ainv) {
  std::vector<double> LU(m * m);
  for (int64_t r = 0; r < m; ++r)
    for (int64_t c = 0; c < m; ++c) LU[r * m + c] = A[c * m + r];   // A^T
  std::vector<int64_t> piv(m);
  for (int64_t k = 0; k < m; ++k) {
    int64_t p = k;
    double best = std::fabs(LU[k * m + k]);
    for (int64_t r = k + 1; r < m; ++r)
      if (std::fabs(LU[r * m + k]) > best) { best = std::fabs(LU[r * m + k]); p = r; }
    if (best == 0.0) return -1;
    piv[k] = p;
    if (p != k)
      for (int64_t c = 0; c < m; ++c) std::swap(LU[k * m + c], LU[p * m + c]);
    for (int64_t r = k + 1; r < m; ++r) {
      LU[r * m + k] /= LU[k * m + k];
      double l = LU[r * m + k];
      for (int64_t c = k + 1; c < m; ++c) LU[r * m + c] -= l * LU[k * m + c];
    }
  }
  auto solve = [&](const double* rhs, double* y) {
    for (int64_t r = 0; r < m; ++r) y[r] = rhs[r];
    for (int64_t k = 0; k < m; ++k) std::swap(y[k], y[piv[k]]);
    for (int64_t r = 0; r < m; ++r)
      for (int64_t c = 0; c < r; ++c) y[r] -= LU[r * m + c] * y[c];
    for (int64_t r = m - 1; r >= 0; --r) {
      for (int64_t c = r + 1; c < m; ++c) y[r] -= LU[r * m + c] * y[c];
      y[r] /= LU[r * m + r];
    }
  };
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < n; ++k) {
    std::vector<double> y(m);
    solve(brows + k * m, y.data());
    double g = -1.0;
    int32_t a = 0;
    for (int64_t p = 0; p < m; ++p)
      if (std::fabs(y[p]) > g) { g = std::fabs(y[p]); a = static_cast<int32_t>(p); }
    gamma[k] = g;
    if (argmax) argmax[k] = a;
  }
  if (Ainv) {
    // row p of A^{-1} = e_p A^{-1}, i.e. the solution for b = e_p.
    std::vector<double> e(m, 0.0), y(m);
    for (int64_t p = 0; p < m; ++p) {
      e[p] = 1.0;
      solve(e.data(), y.data());
      for (int64_t c = 0; c < m; ++c) Ainv[p * m + c] = y[c];
      e[p] = 0.0;
    }
  }
  return 0;
}

}  // extern "C"

// Host-side basis enumeration and contraction schedule (see schedule.cpp).
#pragma once

#include <array>
#include <cstdint>
#include <functional>
#include <vector>

namespace mtp {

struct Schedule {
  int n_types = 0, lev_max = 0, n_q = 0;
  int n_lin = 0, n_rad = 0, n_moments = 0, nu_max = 0;
  int64_t n_params = 0;
  // basis (canonical order)
  std::vector<int> basis_P;
  std::vector<std::array<int, 4>> basis_mu, basis_nu;
  std::vector<std::array<int, 6>> basis_edges;
  // moment components in value order
  int n_mom_comps = 0;
  std::vector<int> comp_mu;
  std::vector<std::array<int, 3>> comp_exp;
  // v[n_mom_comps + d] = sum_{t in [dst_ptr[d], dst_ptr[d+1])} tri_c[t] v[tri_a[t]] v[tri_b[t]]
  int n_values = 0;
  std::vector<int> dst_ptr, tri_a, tri_b;
  std::vector<double> tri_c;
  std::vector<int> basis_idx;  // value index of each basis function
};

// Throws std::invalid_argument on a descriptor outside the supported range.
Schedule build_schedule(int n_types, int lev_max, int n_q);

// n_rad (n_rad + 1) / 2 null directions of the parameter rows for parameters theta (rows of D).
void gauge_directions(const Schedule& S, const double* theta, double* D);

}  // namespace mtp

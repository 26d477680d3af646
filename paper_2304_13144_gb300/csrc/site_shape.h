// Compile-time shape of the moment set of the specialised mixed-path kernels (site_fast.cu,
// site_split.cu): at every level the moments of radial index mu are M_{mu,nu} for all
// nu <= nu_max(mu) = max(nu_0 - 2 mu, 0) (eq. 3 with the level rule of eqs. 5-6), so the
// components of mu are exactly the monomials x^a y^b z^c of degree <= nu_max(mu).  The value
// index of component (mu, monomial k) is comp_base(mu) + k; monomials are numbered by degree,
// then by descending a, then descending b.
#pragma once

#include <cuda_runtime.h>

#include <type_traits>
#include <utility>

namespace mtp {
namespace shape {

constexpr int nmono_upto(int d) { return d < 0 ? 0 : (d + 1) * (d + 2) * (d + 3) / 6; }
constexpr int mono_index(int a, int b, int c) {
  return nmono_upto(a + b + c - 1) + (b + c) * (b + c + 1) / 2 + c;
}

template <int NR, int NU0>
struct Shape {
  static constexpr int numax(int mu) { return NU0 - 2 * mu > 0 ? NU0 - 2 * mu : 0; }
  static constexpr int NMONO = nmono_upto(NU0);
  static constexpr int comp_base(int mu) {
    int s = 0;
    for (int m = 0; m < mu; ++m) s += nmono_upto(numax(m));
    return s;
  }
  static constexpr int NCOMP = comp_base(NR);
  static constexpr int NCHUNK = (NCOMP + 31) / 32;
};

template <int N>
struct MonoTab {
  int a[N], b[N], c[N], deg[N], parent[N], axis[N], lx[N], ly[N], lz[N];
};

template <int NU0>
constexpr MonoTab<nmono_upto(NU0)> make_mono() {
  MonoTab<nmono_upto(NU0)> t{};
  int k = 0;
  for (int d = 0; d <= NU0; ++d)
    for (int a = d; a >= 0; --a)
      for (int b = d - a; b >= 0; --b) {
        const int c = d - a - b;
        t.a[k] = a; t.b[k] = b; t.c[k] = c; t.deg[k] = d;
        t.lx[k] = a > 0 ? mono_index(a - 1, b, c) : -1;
        t.ly[k] = b > 0 ? mono_index(a, b - 1, c) : -1;
        t.lz[k] = c > 0 ? mono_index(a, b, c - 1) : -1;
        if (a > 0) { t.parent[k] = t.lx[k]; t.axis[k] = 0; }
        else if (b > 0) { t.parent[k] = t.ly[k]; t.axis[k] = 1; }
        else if (c > 0) { t.parent[k] = t.lz[k]; t.axis[k] = 2; } else { t.parent[k] = -1; t.axis[k] = -1; }
        ++k;
      }
  return t;
}

// slots of the moment pass: (monomial k, mu) in monomial-major order; first = first slot of k
template <int N>
struct SlotTab {
  int k[N], mu[N], comp[N], first[N];
};

template <int NR, int NU0>
constexpr SlotTab<Shape<NR, NU0>::NCOMP> make_slots() {
  using Sh = Shape<NR, NU0>;
  SlotTab<Sh::NCOMP> t{};
  constexpr auto M = make_mono<NU0>();
  int s = 0;
  for (int k = 0; k < Sh::NMONO; ++k) {
    bool first = true;
    for (int mu = 0; mu < NR; ++mu)
      if (M.deg[k] <= Sh::numax(mu)) {
        t.k[s] = k; t.mu[s] = mu; t.comp[s] = Sh::comp_base(mu) + k; t.first[s] = first ? 1 : 0;
        first = false;
        ++s;
      }
  }
  return t;
}

template <int NR, int NU0>
struct Tab {
  static constexpr MonoTab<nmono_upto(NU0)> mono = make_mono<NU0>();
  static constexpr SlotTab<Shape<NR, NU0>::NCOMP> slots = make_slots<NR, NU0>();
};

// f(integral_constant<I>), f(integral_constant<I + 1>), ..., f(integral_constant<N - 1>) in order
// (a fold over an index sequence: no recursion depth, for the 286 monomials of degree <= 10)
template <int I, class F, int... K>
__device__ __forceinline__ void static_for_seq(F& f, std::integer_sequence<int, K...>) {
  (f(std::integral_constant<int, I + K>{}), ...);
}
template <int I, int N, class F>
__device__ __forceinline__ void static_for(F&& f) {
  if constexpr (I < N) static_for_seq<I>(f, std::make_integer_sequence<int, N - I>{});
}

__device__ __forceinline__ float axis_val(int ax, float x, float y, float z) { return ax == 0 ? x : (ax == 1 ? y : z); }

// v[0..31] on every lane -> on lane l, v[0] = sum over lanes of the original v[l].
__device__ __forceinline__ void transpose_reduce(float (&v)[32], int lane) {
  static_for<0, 5>([&](auto S) {
    constexpr int s = 16 >> decltype(S)::value;
    const bool up = (lane & s) != 0;
    static_for<0, s>([&](auto I) {
      constexpr int i = decltype(I)::value;
      const float send = up ? v[i] : v[i + s];
      const float keep = up ? v[i + s] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, s);
    });
  });
}


// radial functions f_mu, f'_mu (eq. 4) for one pair; Q_b written to Qrow if given
template <int NR, int NQ>
__device__ __forceinline__ void radial(float rr, const float* cz, float rmin, float rcut, float (&f)[NR],
                                       float (&df)[NR], float* Qrow) {
  const float x = (2.f * rr - (rmin + rcut)) * (1.f / (rcut - rmin));
  const float w = rcut - rr;
  const float w2 = w * w;
  const float dxdr = 2.f / (rcut - rmin);
  float t0 = 1.f, t1 = x, d0 = 0.f, d1 = 1.f;
#pragma unroll
  for (int mu = 0; mu < NR; ++mu) { f[mu] = 0.f; df[mu] = 0.f; }
#pragma unroll
  for (int b = 0; b < NQ; ++b) {
    float tb, db;
    if (b == 0) { tb = t0; db = d0; }
    else if (b == 1) { tb = t1; db = d1; } else {
      const float t2 = 2.f * x * t1 - t0;
      const float d2 = 2.f * t1 + 2.f * x * d1 - d0;
      t0 = t1; t1 = t2; d0 = d1; d1 = d2;
      tb = t2; db = d2;
    }
    const float q = tb * w2;
    const float dq = db * dxdr * w2 - 2.f * tb * w;
    if (Qrow) Qrow[b] = q;
#pragma unroll
    for (int mu = 0; mu < NR; ++mu) {
      const float c = cz[mu * NQ + b];
      f[mu] = fmaf(c, q, f[mu]);
      df[mu] = fmaf(c, dq, df[mu]);
    }
  }
}

template <int NR, int NU0>
__device__ __forceinline__ void adjoint_pass(float rx, float ry, float rz, const float (&f)[NR], const float* grads,
                                             float (&g)[NR], float& gx, float& gy, float& gz) {
  using Sh = Shape<NR, NU0>;
  using Tb = Tab<NR, NU0>;
  float mono[Sh::NMONO];
  static_for<0, Sh::NMONO>([&](auto K) {
    constexpr int k = decltype(K)::value;
    if constexpr (k == 0) {
      mono[0] = 1.f;
    } else {
      constexpr int par = Tb::mono.parent[k];
      constexpr int ax = Tb::mono.axis[k];
      mono[k] = mono[par] * axis_val(ax, rx, ry, rz);
    }
    float h = 0.f;
    static_for<0, NR>([&](auto MU) {
      constexpr int mu = decltype(MU)::value;
      constexpr int dk = Tb::mono.deg[k];
      if constexpr (dk <= Sh::numax(mu)) {
        const float G = grads[Sh::comp_base(mu) + k];
        g[mu] = fmaf(G, mono[k], g[mu]);
        h = fmaf(G, f[mu], h);
      }
    });
    constexpr int ea = Tb::mono.a[k], eb = Tb::mono.b[k], ec = Tb::mono.c[k];
    constexpr int lx = Tb::mono.lx[k], ly = Tb::mono.ly[k], lz = Tb::mono.lz[k];
    if constexpr (ea > 0) gx = fmaf(h * static_cast<float>(ea), mono[lx], gx);
    if constexpr (eb > 0) gy = fmaf(h * static_cast<float>(eb), mono[ly], gy);
    if constexpr (ec > 0) gz = fmaf(h * static_cast<float>(ec), mono[lz], gz);
    // fence per degree: keeps the broadcast loads of dV/dM from being hoisted wholesale
    if constexpr (k + 1 == nmono_upto(Tb::mono.deg[k])) __syncwarp();
  });
}

}  // namespace shape
}  // namespace mtp

// Per-neighborhood kernel of the MTP hot path (one warp per atomic neighborhood).
//
// For atom i with neighbors j (Section II.A):
//   radial basis   Q_b(r) = T_b(x) (R_cut - r)^2, x = (2r - R_min - R_cut)/(R_cut - R_min)   (eq. 4)
//   radial funcs   f_mu = sum_b c[z_i][z_j][mu][b] Q_b                                          (eq. 4)
//   moments        M_{mu,(a,b,c)} = sum_j f_mu(r_ij) x^a y^b z^c   (symmetric storage)          (eq. 3)
//   basis          flattened contraction triples v[d] = sum c v[a] v[b]                        (eqs. 5-6)
//   site energy    V_i = s_{z_i} + sum_a xi_a B_a                                               (eq. 2)
// and the hand-written adjoint: dV/dv by the transposed triple list (gather form, no atomics),
// then per pair dV_i/dr_ij = sum_{mu,k} dV/dM_{mu,k} [f'_mu r^/|r| x^k + f_mu grad(x^k)].
// The same code, instantiated on dual numbers, gives the tangent of the parameter row
// b_i = dV_i/dtheta (eq. 9) used by the force and stress terms of the loss gradient (eq. 7).
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>

#include "mtp_internal.h"
#include "profiler.h"

namespace mtp {
namespace {

template <class R>
struct Dual {
  R v, d;
};
template <class R> __device__ __forceinline__ Dual<R> operator+(Dual<R> a, Dual<R> b) { return {a.v + b.v, a.d + b.d}; }
template <class R> __device__ __forceinline__ Dual<R> operator-(Dual<R> a, Dual<R> b) { return {a.v - b.v, a.d - b.d}; }
template <class R> __device__ __forceinline__ Dual<R> operator*(Dual<R> a, Dual<R> b) {
  return {a.v * b.v, a.d * b.v + a.v * b.d};
}
template <class R> __device__ __forceinline__ Dual<R> operator*(R s, Dual<R> b) { return {s * b.v, s * b.d}; }
template <class R> __device__ __forceinline__ Dual<R> operator*(Dual<R> b, R s) { return {s * b.v, s * b.d}; }
template <class R> __device__ __forceinline__ Dual<R> operator+(Dual<R> a, R s) { return {a.v + s, a.d}; }
template <class R> __device__ __forceinline__ Dual<R> operator-(R s, Dual<R> a) { return {s - a.v, -a.d}; }
template <class R> __device__ __forceinline__ Dual<R> operator-(Dual<R> a, R s) { return {a.v - s, a.d}; }
template <class R> __device__ __forceinline__ Dual<R> operator/(Dual<R> a, Dual<R> b) {
  R inv = R(1) / b.v;
  return {a.v * inv, (a.d - a.v * inv * b.d) * inv};
}
template <class R> __device__ __forceinline__ Dual<R>& operator+=(Dual<R>& a, Dual<R> b) { a.v += b.v; a.d += b.d; return a; }

template <class S> struct Traits;
template <> struct Traits<float> { using R = float; };
template <> struct Traits<double> { using R = double; };
template <> struct Traits<Dual<float>> { using R = float; };
template <> struct Traits<Dual<double>> { using R = double; };

template <class S> __device__ __forceinline__ S mk(typename Traits<S>::R v) {
  if constexpr (std::is_same<S, typename Traits<S>::R>::value) return v;
  else return S{v, typename Traits<S>::R(0)};
}
template <class S> __device__ __forceinline__ S mk2(typename Traits<S>::R v, typename Traits<S>::R d) {
  if constexpr (std::is_same<S, typename Traits<S>::R>::value) return v;
  else return S{v, d};
}
template <class S> __device__ __forceinline__ typename Traits<S>::R vpart(S x) {
  if constexpr (std::is_same<S, typename Traits<S>::R>::value) return x;
  else return x.v;
}
template <class S> __device__ __forceinline__ typename Traits<S>::R dpart(S x) {
  if constexpr (std::is_same<S, typename Traits<S>::R>::value) return typename Traits<S>::R(0);
  else return x.d;
}
__device__ __forceinline__ float ssqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double ssqrt(double x) { return sqrt(x); }
template <class R> __device__ __forceinline__ Dual<R> ssqrt(Dual<R> x) {
  R s = ssqrt(x.v);
  return {s, x.d / (R(2) * s)};
}
template <class S> __device__ __forceinline__ S shfl_xor(S x, int m) {
  if constexpr (std::is_same<S, typename Traits<S>::R>::value) return __shfl_xor_sync(0xffffffffu, x, m);
  else return S{__shfl_xor_sync(0xffffffffu, x.v, m), __shfl_xor_sync(0xffffffffu, x.d, m)};
}
template <class S> __device__ __forceinline__ S warp_sum(S x) {
  for (int m = 16; m; m >>= 1) x = x + shfl_xor(x, m);
  return x;
}

constexpr int kWarps = 4;

struct Layout {
  int NR, NQ, PWS, NV, CBN, NC;
  size_t c_bytes, warp_bytes, total;
};

template <class S, class R>
Layout make_layout(const DevSchedule& d, int warps) {
  Layout L;
  L.NR = d.n_rad;
  L.NQ = d.n_q;
  L.PWS = 6 * (d.nu_max + 1) + 1;
  L.NV = d.n_vals;
  L.CBN = d.n_types * d.n_rad * d.n_q;
  L.NC = d.n_types * L.CBN;
  L.c_bytes = (static_cast<size_t>(L.NC) * sizeof(R) + 15) & ~size_t(15);
  size_t nS = 2 * static_cast<size_t>(L.NV) + 32 * (3 * L.NR + L.NQ + L.PWS) + L.CBN;
  L.warp_bytes = (nS * sizeof(S) + 32 * sizeof(int) + 15) & ~size_t(15);
  L.total = L.c_bytes + warps * L.warp_bytes;
  return L;
}

struct SiteParams {
  DevSchedule d;
  DevNbr nb;
  const double* pos;
  const int* type;
  const double* cell;   // n_cfg x 9
  int64_t n_work;
  SiteOutputs o;
  Layout L;
  int warps_hint;   // warps per block requested (0: the largest that fits)
};

// Load r_ij (and its tangent) for pair p of center i.
template <class S, class R>
__device__ __forceinline__ void load_pair(const SiteParams& P, int64_t i, int64_t p, bool tangent, S& rx, S& ry,
                                          S& rz, int& zj) {
  int j = P.nb.pj[p];
  zj = P.type[j];
  R x, y, z;
  if constexpr (std::is_same<R, float>::value) {
    float4 v = P.nb.pr32[p];
    x = v.x; y = v.y; z = v.z;
  } else {
    int img = P.nb.pimg[p];
    int n0 = unpack_img(img, 0), n1 = unpack_img(img, 1), n2 = unpack_img(img, 2);
    const double* H = P.cell + 9 * P.nb.atom_cfg[i];
    double sh0 = n0 * H[0] + n1 * H[3] + n2 * H[6];
    double sh1 = n0 * H[1] + n1 * H[4] + n2 * H[7];
    double sh2 = n0 * H[2] + n1 * H[5] + n2 * H[8];
    x = (P.pos[3 * j + 0] + sh0) - P.pos[3 * i + 0];
    y = (P.pos[3 * j + 1] + sh1) - P.pos[3 * i + 1];
    z = (P.pos[3 * j + 2] + sh2) - P.pos[3 * i + 2];
  }
  if (tangent) {
    const double* U = P.o.U;
    const double* Sm = P.o.Scfg + 9 * P.nb.atom_cfg[i];
    R dx = R(U[3 * j + 0] - U[3 * i + 0]) + R(Sm[0]) * x + R(Sm[1]) * y + R(Sm[2]) * z;
    R dy = R(U[3 * j + 1] - U[3 * i + 1]) + R(Sm[3]) * x + R(Sm[4]) * y + R(Sm[5]) * z;
    R dz = R(U[3 * j + 2] - U[3 * i + 2]) + R(Sm[6]) * x + R(Sm[7]) * y + R(Sm[8]) * z;
    rx = mk2<S>(x, dx); ry = mk2<S>(y, dy); rz = mk2<S>(z, dz);
  } else {
    rx = mk<S>(x); ry = mk<S>(y); rz = mk<S>(z);
  }
}

// Radial basis, radial functions and power tables of one pair into the lane's smem rows.
template <class S, class R>
__device__ __forceinline__ void pair_setup(const SiteParams& P, const R* ctab, int zi, int zj, S rx, S ry, S rz,
                                           bool act, S& rr, S* PF, S* PDF, S* PQ, S* PW, int nu_max) {
  const Layout& L = P.L;
  const R rmin = R(P.d.r_min), rcut = R(P.d.r_cut);
  rr = ssqrt(rx * rx + ry * ry + rz * rz);
  S x = (R(2) * rr - (rmin + rcut)) * (R(1) / (rcut - rmin));
  S w = rcut - rr;
  S w2 = w * w;
  R dxdr = R(2) / (rcut - rmin);
  // Chebyshev T_b and dT_b/dx by the three-term recurrence
  S t0 = mk<S>(R(1)), t1 = x, d0 = mk<S>(R(0)), d1 = mk<S>(R(1));
  const R* cz = ctab + (static_cast<size_t>(zi) * P.d.n_types + zj) * L.NR * L.NQ;
  for (int mu = 0; mu < L.NR; ++mu) { PF[mu] = mk<S>(R(0)); PDF[mu] = mk<S>(R(0)); }
  for (int b = 0; b < L.NQ; ++b) {
    S tb, db;
    if (b == 0) { tb = t0; db = d0; }
    else if (b == 1) { tb = t1; db = d1; } else {
      S t2 = R(2) * x * t1 - t0;
      S d2 = R(2) * t1 + R(2) * x * d1 - d0;
      t0 = t1; t1 = t2; d0 = d1; d1 = d2;
      tb = t2; db = d2;
    }
    S q = tb * w2;
    S dq = db * dxdr * w2 - R(2) * tb * w;
    PQ[b] = q;
    if (act) {
      for (int mu = 0; mu < L.NR; ++mu) {
        R c = cz[mu * L.NQ + b];
        PF[mu] = PF[mu] + c * q;
        PDF[mu] = PDF[mu] + c * dq;
      }
    }
  }
  // powers x^k, y^k, z^k (k = 0..nu_max) and k x^(k-1) etc.
  const int np1 = nu_max + 1;
  S* px = PW;
  S* py = PW + np1;
  S* pz = PW + 2 * np1;
  S* dx = PW + 3 * np1;
  S* dy = PW + 4 * np1;
  S* dz = PW + 5 * np1;
  px[0] = py[0] = pz[0] = mk<S>(R(1));
  dx[0] = dy[0] = dz[0] = mk<S>(R(0));
  for (int k = 1; k <= nu_max; ++k) {
    px[k] = px[k - 1] * rx; py[k] = py[k - 1] * ry; pz[k] = pz[k - 1] * rz;
    dx[k] = R(k) * px[k - 1]; dy[k] = R(k) * py[k - 1]; dz[k] = R(k) * pz[k - 1];
  }
}

enum : int { M_EFS = 1, M_ROWS = 2, M_TAN = 4 };

template <class S, class R, int MODE>
__global__ void __launch_bounds__(kWarps * 32) site_kernel(SiteParams P) {
  extern __shared__ __align__(16) unsigned char smem[];
  const Layout& L = P.L;
  const DevSchedule& d = P.d;
  R* ctab = reinterpret_cast<R*>(smem);
  const R* theta = nullptr;
  const R* tri_c = nullptr;
  const R* use_c = nullptr;
  const R* seed = nullptr;
  if constexpr (std::is_same<R, float>::value) { theta = d.theta_f; tri_c = d.tri_cf; use_c = d.use_cf; seed = d.seed_f; } else { theta = d.theta_d; tri_c = d.tri_cd; use_c = d.use_cd; seed = d.seed_d; }
  const int T = d.n_types;
  const int64_t off_c = T + d.n_lin;
  for (int k = threadIdx.x; k < L.NC; k += blockDim.x) ctab[k] = theta[off_c + k];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nw = blockDim.x >> 5;   // at most kWarps (fewer for large models)
  unsigned char* wbase = smem + L.c_bytes + warp * L.warp_bytes;
  S* vals = reinterpret_cast<S*>(wbase);
  S* grads = vals + L.NV;
  S* PFb = grads + L.NV;               // 32 x NR
  S* PDFb = PFb + 32 * L.NR;           // 32 x NR
  S* GMb = PDFb + 32 * L.NR;           // 32 x NR
  S* PQb = GMb + 32 * L.NR;            // 32 x NQ
  S* PWb = PQb + 32 * L.NQ;            // 32 x PWS
  S* CB = PWb + 32 * L.PWS;            // CBN
  int* ZJ = reinterpret_cast<int*>(CB + L.CBN);
  // per-warp gradient accumulator for the tangent mode lives in the rows buffer region
  __syncthreads();
  const int nu_max = d.nu_max;
  const int np1 = nu_max + 1;

  double Wacc[9];
  for (int64_t wk = static_cast<int64_t>(blockIdx.x) * nw + warp; wk < P.n_work;
       wk += static_cast<int64_t>(gridDim.x) * nw) {
    const int64_t i = P.o.atom_list ? P.o.atom_list[wk] : wk;
    const int zi = P.type[i];
    const int64_t p0 = P.nb.off[i];
    const int np = static_cast<int>(P.nb.off[i + 1] - p0);
    for (int c = lane; c < d.n_mom; c += 32) vals[c] = mk<S>(R(0));
    if (MODE & (M_ROWS | M_TAN))
      for (int e = lane; e < L.CBN; e += 32) CB[e] = mk<S>(R(0));
    __syncwarp();
    // ---------------- moments (eq. 3) ----------------
    for (int base = 0; base < np; base += 32) {
      const int q = lane;
      const bool act = base + q < np;
      S rx = mk<S>(R(1)), ry = mk<S>(R(0)), rz = mk<S>(R(0));
      int zj = 0;
      if (act) load_pair<S, R>(P, i, p0 + base + q, (MODE & M_TAN) != 0, rx, ry, rz, zj);
      S rr;
      pair_setup<S, R>(P, ctab, zi, zj, rx, ry, rz, act, rr, PFb + L.NR * q, PDFb + L.NR * q, PQb + L.NQ * q,
                       PWb + L.PWS * q, nu_max);
      ZJ[q] = zj;
      __syncwarp();
      const int nq = min(32, np - base);
      for (int c = lane; c < d.n_mom; c += 32) {
        const int info = d.comp_info[c];
        const int mu = info & 255, a = (info >> 8) & 255, b = (info >> 16) & 255, cc = (info >> 24) & 255;
        S acc = mk<S>(R(0));
        for (int qq = 0; qq < nq; ++qq) {
          const S* W = PWb + L.PWS * qq;
          acc += PFb[L.NR * qq + mu] * W[a] * W[np1 + b] * W[2 * np1 + cc];
        }
        vals[c] += acc;
      }
      __syncwarp();
    }
    // ---------------- forward contraction (eqs. 5-6) ----------------
    for (int wv = 0; wv < d.n_fwaves; ++wv) {
      const int e1 = d.fwave_ptr[wv + 1];
      for (int e = d.fwave_ptr[wv] + lane; e < e1; e += 32) {
        const int dst = d.fdst[e];
        const int t0 = d.tri_ptr[dst - d.first_dst], t1 = d.tri_ptr[dst - d.first_dst + 1];
        S acc = mk<S>(R(0));
        for (int t = t0; t < t1; ++t) {
          const uint32_t ab = d.tri_ab[t];
          acc += tri_c[t] * (vals[ab & 0xffffu] * vals[ab >> 16]);
        }
        vals[dst] = acc;
      }
      __syncwarp();
    }
    // ---------------- site energy (eq. 2) ----------------
    if (MODE & M_EFS) {
      S acc = mk<S>(R(0));
      for (int a = lane; a < d.n_lin; a += 32) acc += theta[T + a] * vals[d.basis_idx[a]];
      acc = warp_sum(acc);
      if (lane == 0) P.o.V[i] = static_cast<double>(vpart(acc)) + d.theta_d[zi];
    }
    // ---------------- adjoint of the contraction (gather form) ----------------
    for (int wv = 0; wv < d.n_rwaves; ++wv) {
      const int e1 = d.rwave_ptr[wv + 1];
      for (int e = d.rwave_ptr[wv] + lane; e < e1; e += 32) {
        const int x = d.rval[e];
        S g = mk<S>(seed[x]);
        const int u1 = d.use_ptr[x + 1];
        for (int u = d.use_ptr[x]; u < u1; ++u) {
          const uint32_t od = d.use_od[u];
          g += use_c[u] * (vals[od & 0xffffu] * grads[od >> 16]);
        }
        grads[x] = g;
      }
      __syncwarp();
    }
    // ---------------- per-pair adjoint: dV/dr_ij, virial, radial block of b_i ----------------
    for (int k = 0; k < 9; ++k) Wacc[k] = 0.0;
    for (int base = 0; base < np; base += 32) {
      const int q = lane;
      const bool act = base + q < np;
      S rx = mk<S>(R(1)), ry = mk<S>(R(0)), rz = mk<S>(R(0));
      int zj = 0;
      if (act) load_pair<S, R>(P, i, p0 + base + q, (MODE & M_TAN) != 0, rx, ry, rz, zj);
      S* PF = PFb + L.NR * q;
      S* PDF = PDFb + L.NR * q;
      S* GM = GMb + L.NR * q;
      S* PQ = PQb + L.NQ * q;
      S* PW = PWb + L.PWS * q;
      S rr;
      pair_setup<S, R>(P, ctab, zi, zj, rx, ry, rz, act, rr, PF, PDF, PQ, PW, nu_max);
      ZJ[q] = zj;
      for (int mu = 0; mu < L.NR; ++mu) GM[mu] = mk<S>(R(0));
      if (act) {
        S gx = mk<S>(R(0)), gy = mk<S>(R(0)), gz = mk<S>(R(0));
        S gm = mk<S>(R(0));
        int cur_mu = d.comp_info[0] & 255;
        const S* px = PW;
        const S* py = PW + np1;
        const S* pz = PW + 2 * np1;
        const S* dxp = PW + 3 * np1;
        const S* dyp = PW + 4 * np1;
        const S* dzp = PW + 5 * np1;
        S fmu = PF[cur_mu];
        for (int c = 0; c < d.n_mom; ++c) {
          const int info = d.comp_info[c];
          const int mu = info & 255, a = (info >> 8) & 255, b = (info >> 16) & 255, cc = (info >> 24) & 255;
          if (mu != cur_mu) {
            GM[cur_mu] += gm;
            gm = mk<S>(R(0));
            cur_mu = mu;
            fmu = PF[mu];
          }
          const S G = grads[c];
          const S yz = py[b] * pz[cc];
          const S xa = px[a];
          gm += G * (xa * yz);
          if (MODE & M_EFS) {
            const S h = G * fmu;
            gx += h * (dxp[a] * yz);
            gy += h * (xa * (dyp[b] * pz[cc]));
            gz += h * (xa * (py[b] * dzp[cc]));
          }
        }
        GM[cur_mu] += gm;
        if (MODE & M_EFS) {
          S rad = mk<S>(R(0));
          for (int mu = 0; mu < L.NR; ++mu) rad += GM[mu] * PDF[mu];
          const S s = rad / rr;
          gx += s * rx; gy += s * ry; gz += s * rz;
          const int64_t p = p0 + base + q;
          R* Gout = static_cast<R*>(P.o.G);
          Gout[3 * p + 0] = vpart(gx);
          Gout[3 * p + 1] = vpart(gy);
          Gout[3 * p + 2] = vpart(gz);
          const double g3[3] = {static_cast<double>(vpart(gx)), static_cast<double>(vpart(gy)),
                                static_cast<double>(vpart(gz))};
          const double r3[3] = {static_cast<double>(vpart(rx)), static_cast<double>(vpart(ry)),
                                static_cast<double>(vpart(rz))};
          for (int a2 = 0; a2 < 3; ++a2)
            for (int b2 = 0; b2 < 3; ++b2) Wacc[3 * a2 + b2] -= g3[a2] * r3[b2];
        }
      }
      __syncwarp();
      if (MODE & (M_ROWS | M_TAN)) {
        const int nq = min(32, np - base);
        for (int e = lane; e < L.CBN; e += 32) {
          const int zj2 = e / (L.NR * L.NQ);
          const int mu = (e / L.NQ) % L.NR;
          const int b = e % L.NQ;
          S acc = mk<S>(R(0));
          for (int qq = 0; qq < nq; ++qq)
            if (ZJ[qq] == zj2) acc += GMb[L.NR * qq + mu] * PQb[L.NQ * qq + b];
          CB[e] += acc;
        }
      }
      __syncwarp();
    }
    if (MODE & M_EFS) {
      for (int k = 0; k < 9; ++k) {
        double v = Wacc[k];
        for (int m = 16; m; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
        Wacc[k] = v;
      }
      if (lane == 0)
        for (int k = 0; k < 9; ++k) P.o.Wat[9 * i + k] = Wacc[k];
    }
    if (MODE & M_ROWS) {
      const int64_t row = P.o.row_pos ? P.o.row_pos[i] : wk;
      const int64_t ld = P.o.rows_ld;
      const int cb_total = T * L.CBN;
      if (P.o.rows) {
        double* out = P.o.rows + row * ld;
        for (int k = lane; k < T; k += 32) out[k] = (k == zi) ? 1.0 : 0.0;
        for (int a = lane; a < d.n_lin; a += 32) out[T + a] = static_cast<double>(vpart(vals[d.basis_idx[a]]));
        for (int e = lane; e < cb_total; e += 32) {
          const int zblk = e / L.CBN;
          out[off_c + e] = (zblk == zi) ? static_cast<double>(vpart(CB[e - zblk * L.CBN])) : 0.0;
        }
        for (int k = static_cast<int>(d.n_params) + lane; k < ld; k += 32) out[k] = 0.0;
      }
      if (P.o.rows_hi) {
        float* hi = P.o.rows_hi + row * ld;
        float* lo = P.o.rows_lo ? P.o.rows_lo + row * ld : nullptr;
        auto put = [&](int64_t k, double v) {
          float h = static_cast<float>(v);
          if (lo) {
            h = tf32_rn(h);
            lo[k] = tf32_rn(static_cast<float>(v - static_cast<double>(h)));
          }
          hi[k] = h;
        };
        for (int k = lane; k < T; k += 32) put(k, (k == zi) ? 1.0 : 0.0);
        for (int a = lane; a < d.n_lin; a += 32) put(T + a, static_cast<double>(vpart(vals[d.basis_idx[a]])));
        for (int e = lane; e < cb_total; e += 32) {
          const int zblk = e / L.CBN;
          put(off_c + e, (zblk == zi) ? static_cast<double>(vpart(CB[e - zblk * L.CBN])) : 0.0);
        }
        for (int64_t k = d.n_params + lane; k < ld; k += 32) put(k, 0.0);
      }
    }
    if (MODE & M_TAN) {
      // accumulate coef * b_i - d/dt b_i into this warp's row of the partial-gradient buffer
      double* acc = P.o.grad_part + (static_cast<int64_t>(blockIdx.x) * nw + warp) * d.n_params;
      const double coef = P.o.coef[P.nb.atom_cfg[i]];
      if (lane == 0) acc[zi] += coef;
      for (int a = lane; a < d.n_lin; a += 32) {
        const S B = vals[d.basis_idx[a]];
        acc[T + a] += coef * static_cast<double>(vpart(B)) - static_cast<double>(dpart(B));
      }
      for (int e = lane; e < L.CBN; e += 32)
        acc[off_c + static_cast<int64_t>(zi) * L.CBN + e] +=
            coef * static_cast<double>(vpart(CB[e])) - static_cast<double>(dpart(CB[e]));
    }
    __syncwarp();
  }
}

// Launches the kernel; returns the warps per block used.
template <class S, class R, int MODE>
int launch_sites(const SiteParams& P0, int* grid_used, cudaStream_t s) {
  SiteParams P = P0;
  // as many warps per block (up to kWarps) as the per-warp value arrays leave room for
  int warps = (P.warps_hint > 0) ? std::min(P.warps_hint, kWarps) : kWarps;
  P.L = make_layout<S, R>(P.d, warps);
  while (warps > 1 && P.L.total > 227 * 1024) {
    warps >>= 1;
    P.L = make_layout<S, R>(P.d, warps);
  }
  if (P.L.total > 227 * 1024)
    throw Fail{MTP_ERR_UNSUPPORTED, "model too large for the per-neighborhood kernel's shared memory"};
  auto kern = site_kernel<S, R, MODE>;
  MTP_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(P.L.total)));
  int dev = 0, nsm = 0, per_sm = 0;
  MTP_CUDA(cudaGetDevice(&dev));
  MTP_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  MTP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, warps * 32, P.L.total));
  per_sm = std::max(per_sm, 1);
  int64_t need = (P.n_work + warps - 1) / warps;
  int grid = static_cast<int>(std::min<int64_t>(need, static_cast<int64_t>(nsm) * per_sm));
  grid = std::max(grid, 1);
  if (grid_used) {
    if (*grid_used > 0) grid = std::min(grid, *grid_used);
    *grid_used = grid;
  }
  if (P.n_work == 0) return warps;
  const char* name = (MODE & M_TAN) ? "site_tangent" : (MODE & M_EFS) ? ((MODE & M_ROWS) ? "site_efs_rows" : "site_efs") : "site_rows";
  ProfRegion pr(name, s);
  kern<<<grid, warps * 32, P.L.total, s>>>(P);
  ProfRegion::launched();
  MTP_CUDA(cudaGetLastError());
  return warps;
}

}  // namespace

int site_max_grid(mtp_model* m, bool fp64, bool tangent) {
  int dev = 0, nsm = 0;
  MTP_CUDA(cudaGetDevice(&dev));
  MTP_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  (void)m; (void)fp64; (void)tangent;
  return nsm * 8;
}

bool run_sites_fast(mtp_model* m, const mtp_batch* b, const mtp_nbr* nb, const SiteOutputs& o, cudaStream_t s);
bool run_sites_split(mtp_model* m, const mtp_batch* b, const mtp_nbr* nb, const SiteOutputs& o, cudaStream_t s);

void run_sites(mtp_model* m, const mtp_batch* b, const mtp_nbr* nb, bool fp64, const SiteOutputs& o,
               bool tangent, int* grid_used, cudaStream_t s) {
  m->last_split = false;
  if (!fp64 && !tangent && !m->force_generic && run_sites_split(m, b, nb, o, s)) return;
  if (!fp64 && !tangent && !m->force_generic && run_sites_fast(m, b, nb, o, s)) return;
  SiteParams P{};
  P.warps_hint = m->tune_warps_generic;
  m->last_fast = false;
  P.d = m->ds;
  P.nb = nb->dn;
  P.pos = b->pos;
  P.type = b->type;
  P.cell = b->cell;
  P.o = o;
  P.n_work = o.atom_list ? o.n_list : nb->n_atoms;
  const bool efs = o.V != nullptr;
  const bool rows = o.rows != nullptr || o.rows_hi != nullptr;
  if (tangent) {
    if (fp64) m->last_warps = launch_sites<Dual<double>, double, M_TAN>(P, grid_used, s);
    else m->last_warps = launch_sites<Dual<float>, float, M_TAN>(P, grid_used, s);
    return;
  }
  if (efs && rows) {
    if (fp64) m->last_warps = launch_sites<double, double, M_EFS | M_ROWS>(P, grid_used, s);
    else m->last_warps = launch_sites<float, float, M_EFS | M_ROWS>(P, grid_used, s);
  } else if (efs) {
    if (fp64) m->last_warps = launch_sites<double, double, M_EFS>(P, grid_used, s);
    else m->last_warps = launch_sites<float, float, M_EFS>(P, grid_used, s);
  } else if (rows) {
    if (fp64) m->last_warps = launch_sites<double, double, M_ROWS>(P, grid_used, s);
    else m->last_warps = launch_sites<float, float, M_ROWS>(P, grid_used, s);
  } else {
    throw Fail{MTP_ERR_ARG, "no output requested"};
  }
}

}  // namespace mtp

// Register-resident per-neighborhood kernel for the mixed path (FP32 arithmetic, FP64 sums).
//
// Same method as site.cu (eqs. 2-4, 5-6, 9 and the hand-written adjoint) specialised on the
// shape of the moment set: at every level the moments of radial index mu are M_{mu,nu} for
// all nu <= nu_max(mu) = max(nu_0 - 2 mu, 0), so the components of mu are exactly the
// monomials x^a y^b z^c of degree <= nu_max(mu).  With N_rad and nu_0 as template parameters
// every monomial index is a compile-time constant and a pair's monomials live in registers:
//   * moments (lane = pair): per 32-component chunk each lane forms f_mu(r) x^a y^b z^c for its
//     pair; a warp transpose-reduction leaves lane l with the sum over the 32 pairs of
//     component l, accumulated into the neighborhood's value array in shared memory;
//   * contraction and its adjoint: the flattened triple list, packed to one 32-bit word per
//     term (12-bit operands, 8-bit index into a coefficient table in shared memory);
//   * pair adjoint (lane = pair): dV/dr_ij from the broadcast dV/dM, monomials regenerated in
//     registers, gradient of every monomial from its lower-degree neighbours.
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>
#include <utility>

#include "mtp_internal.h"
#include "profiler.h"
#include "site_shape.h"

namespace mtp {
namespace {
using namespace shape;

struct FastParams {
  DevSchedule d;
  DevNbr nb;
  const int* type;
  int64_t n_work;
  SiteOutputs o;
  int NQ, CBN, NC, NV;  // NV: per-neighborhood value slots, padded to a multiple of 4
  bool row_stage;       // rows are assembled in the adjoint buffer and written as float4
  // aux_off > 0: the pair-adjoint scratch (dV/df per pair, Q per pair, species per pair, the
  // radial block of b_i) lives in the adjoint array of the neighborhood being finished, from slot
  // aux_off on: after the contraction only the adjoints of the moments (slots below the moment
  // count) are read again, so the rest of the array is free
  int aux_off;
  size_t c_bytes, tab_bytes, sched_bytes, warp_bytes, total;
  // word offsets of the schedule arrays inside the shared-memory copy
  int o_fslab, o_fround, o_frdst, o_rslab, o_rround, o_rrval, o_seed;
};

__device__ __forceinline__ void copy_words(uint32_t* dst, const uint32_t* src, int n) {
  for (int k = threadIdx.x; k < n; k += blockDim.x) dst[k] = src[k];
}

template <int NR, int NU0>
__device__ __forceinline__ void moments_pass(float rx, float ry, float rz, const float (&f)[NR], float* vals,
                                             const int* slot_comp, int lane) {
  using Sh = Shape<NR, NU0>;
  using Tb = Tab<NR, NU0>;
  float mono[Sh::NMONO];
  static_for<0, Sh::NCHUNK>([&](auto C) {
    constexpr int c = decltype(C)::value;
    float v[32];
    static_for<0, 32>([&](auto Tt) {
      constexpr int t = decltype(Tt)::value;
      constexpr int s = 32 * c + t;
      if constexpr (s < Sh::NCOMP) {
        constexpr int k = Tb::slots.k[s];
        constexpr int mu = Tb::slots.mu[s];
        constexpr int first = Tb::slots.first[s];
        if constexpr (first != 0) {
          if constexpr (k == 0) {
            mono[0] = 1.f;
          } else {
            constexpr int par = Tb::mono.parent[k];
            constexpr int ax = Tb::mono.axis[k];
            mono[k] = mono[par] * axis_val(ax, rx, ry, rz);
          }
        }
        v[t] = f[mu] * mono[k];
      } else {
        v[t] = 0.f;
      }
    });
    transpose_reduce(v, lane);
    const int s = 32 * c + lane;
    if (s < Sh::NCOMP) vals[slot_comp[s]] += v[0];
  });
}

constexpr int kMaxWarpsF = 8;
constexpr int kNQ = 8;   // radial polynomials of the specialised kernel (other N_Q: generic kernel)
enum : int { F_EFS = 1, F_ROWS = 2 };

// FG: the forward slab stays in global memory (read through L1) instead of shared memory, which
// leaves room for one more warp per SM on the level-20 shape.
template <int NR, int NU0, int MODE, bool FG>
__global__ void __launch_bounds__(kMaxWarpsF * 32, 1) site_fast_kernel(FastParams P) {
  using Sh = Shape<NR, NU0>;
  extern __shared__ __align__(16) unsigned char smem[];
  const DevSchedule& d = P.d;
  constexpr int NQ = kNQ;
  const int CBN = P.CBN, NV = P.NV;
  float* ctab = reinterpret_cast<float*>(smem);
  float* coef = reinterpret_cast<float*>(smem + P.c_bytes);
  int* slot_comp = reinterpret_cast<int*>(coef + 256);
  const int T = d.n_types;
  const int64_t off_c = T + d.n_lin;
  for (int k = threadIdx.x; k < P.NC; k += blockDim.x) ctab[k] = d.theta_f[off_c + k];
  for (int k = threadIdx.x; k < d.n_coef; k += blockDim.x) coef[k] = d.coef_f[k];
  // slot -> value index of the moment component (monomial-major order of the moment pass)
  for (int s = threadIdx.x; s < Sh::NCOMP; s += blockDim.x) {
    // recompute slot s -> comp on the device (same order as make_slots)
    int ss = 0, comp = 0;
    for (int k = 0; k < Sh::NMONO && ss <= s; ++k) {
      int dk = 0;
      while (nmono_upto(dk) <= k) ++dk;
      for (int mu = 0; mu < NR; ++mu)
        if (dk <= Sh::numax(mu)) {
          if (ss == s) comp = Sh::comp_base(mu) + k;
          ++ss;
        }
    }
    slot_comp[s] = comp;
  }
  // the contraction schedule, staged once per (persistent) block: every warp reads it per atom
  uint32_t* sched = reinterpret_cast<uint32_t*>(smem + P.c_bytes + P.tab_bytes);
  if (!FG) copy_words(sched + P.o_fslab, d.fslab, d.fslab_words);
  copy_words(sched + P.o_fround, reinterpret_cast<const uint32_t*>(d.fround), 4 * d.n_fround);
  copy_words(sched + P.o_frdst, reinterpret_cast<const uint32_t*>(d.fr_dst), 32 * d.n_fround);
  copy_words(sched + P.o_rslab, d.rslab, d.rslab_words);
  copy_words(sched + P.o_rround, reinterpret_cast<const uint32_t*>(d.rround), 4 * d.n_rround);
  copy_words(sched + P.o_rrval, reinterpret_cast<const uint32_t*>(d.rr_val), 32 * d.n_rround);
  copy_words(sched + P.o_seed, reinterpret_cast<const uint32_t*>(d.seed_f), d.n_vals);
  const uint32_t* s_fslab = FG ? d.fslab : sched + P.o_fslab;
  const int4* s_fround = reinterpret_cast<const int4*>(sched + P.o_fround);
  const int* s_frdst = reinterpret_cast<const int*>(sched + P.o_frdst);
  const uint32_t* s_rslab = sched + P.o_rslab;
  const int4* s_rround = reinterpret_cast<const int4*>(sched + P.o_rround);
  const int* s_rrval = reinterpret_cast<const int*>(sched + P.o_rrval);
  const float* s_seed = reinterpret_cast<const float*>(sched + P.o_seed);
  const int nwarps = blockDim.x >> 5;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // per warp: two neighborhoods carried through the contraction together
  unsigned char* wbase = smem + P.c_bytes + P.tab_bytes + P.sched_bytes + warp * P.warp_bytes;
  float* valsA[2];
  float* gradsA[2];
  valsA[0] = reinterpret_cast<float*>(wbase);
  gradsA[0] = valsA[0] + NV;
  valsA[1] = gradsA[0] + NV;
  gradsA[1] = valsA[1] + NV;
  // padding terms read vals[0] and grads[0]: keep every entry finite from the start
  for (int k = lane; k < 4 * NV; k += 32) valsA[0][k] = 0.f;
  // pair-adjoint scratch: [GM 32 x NR | PQ 32 x NQ | ZJ 32 | CB], per warp or per adjoint array
  float* const aux_warp = gradsA[1] + NV;
  __syncthreads();
  const float rmin = static_cast<float>(d.r_min), rcut = static_cast<float>(d.r_cut);

  // ---------------- moments of one neighborhood (eq. 3) ----------------
  auto moments = [&](int64_t i, float* vals) {
    const int zi = P.type[i];
    const int64_t p0 = P.nb.off[i];
    const int np = static_cast<int>(P.nb.off[i + 1] - p0);
    const float* czi = ctab + static_cast<size_t>(zi) * T * NR * NQ;
    for (int c = lane; c < Sh::NCOMP; c += 32) vals[c] = 0.f;
    __syncwarp();
    for (int base = 0; base < np; base += 32) {
      const bool act = base + lane < np;
      float rx = 1.f, ry = 0.f, rz = 0.f, rr = 1.f;
      int zj = 0;
      if (act) {
        const int64_t p = p0 + base + lane;
        const float4 v = P.nb.pr32[p];
        rx = v.x; ry = v.y; rz = v.z; rr = v.w;
        zj = P.type[P.nb.pj[p]];
      }
      float f[NR], df[NR];
      radial<NR, NQ>(rr, czi + zj * NR * NQ, rmin, rcut, f, df, nullptr);
      if (!act)
#pragma unroll
        for (int mu = 0; mu < NR; ++mu) f[mu] = 0.f;
      moments_pass<NR, NU0>(rx, ry, rz, f, vals, slot_comp, lane);
    }
    __syncwarp();
  };

  // ---------------- pair adjoint and outputs of one neighborhood ----------------
  auto finish = [&](int64_t wk, int64_t i, const float* vals, const float* grads) {
    float* const aux = P.aux_off > 0 ? const_cast<float*>(grads) + P.aux_off : aux_warp;
    float* const GMb = aux;                 // 32 x NR
    constexpr int PQS = NQ + 1;             // odd row stride: the lanes' Q_b stores hit distinct banks
    float* const PQb = GMb + 32 * NR;       // 32 x PQS
    int* const ZJ = reinterpret_cast<int*>(PQb + 32 * PQS);
    float* const CB = PQb + 32 * PQS + 32;  // CBN
    if (MODE & F_ROWS) {
      for (int e = lane; e < CBN; e += 32) CB[e] = 0.f;
      __syncwarp();
    }
    const int zi = P.type[i];
    const int64_t p0 = P.nb.off[i];
    const int np = static_cast<int>(P.nb.off[i + 1] - p0);
    const float* czi = ctab + static_cast<size_t>(zi) * T * NR * NQ;
    if (MODE & F_EFS) {
      float acc = 0.f;
      for (int a = lane; a < d.n_lin; a += 32) acc = fmaf(d.theta_f[T + a], vals[d.basis_idx[a]], acc);
      for (int m = 16; m; m >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, m);
      if (lane == 0) P.o.V[i] = static_cast<double>(acc) + d.theta_d[zi];
    }
    float Wl[9];   // this lane's pairs (at most a few terms)
#pragma unroll
    for (int k = 0; k < 9; ++k) Wl[k] = 0.f;
    for (int base = 0; base < np; base += 32) {
      const bool act = base + lane < np;
      float rx = 1.f, ry = 0.f, rz = 0.f, rr = 1.f;
      int zj = 0;
      const int64_t p = p0 + base + lane;
      if (act) {
        const float4 v = P.nb.pr32[p];
        rx = v.x; ry = v.y; rz = v.z; rr = v.w;
        zj = P.type[P.nb.pj[p]];
      }
      float f[NR], df[NR], g[NR];
      radial<NR, NQ>(rr, czi + zj * NR * NQ, rmin, rcut, f, df, (MODE & F_ROWS) ? PQb + PQS * lane : nullptr);
#pragma unroll
      for (int mu = 0; mu < NR; ++mu) g[mu] = 0.f;
      float gx = 0.f, gy = 0.f, gz = 0.f;
      adjoint_pass<NR, NU0>(rx, ry, rz, f, grads, g, gx, gy, gz);
      if (!act)
#pragma unroll
        for (int mu = 0; mu < NR; ++mu) g[mu] = 0.f;
      if (MODE & F_ROWS) {
#pragma unroll
        for (int mu = 0; mu < NR; ++mu) GMb[NR * lane + mu] = g[mu];
        ZJ[lane] = zj;
      }
      if ((MODE & F_EFS) && act) {
        float rad = 0.f;
#pragma unroll
        for (int mu = 0; mu < NR; ++mu) rad = fmaf(g[mu], df[mu], rad);
        const float s = rad / rr;
        gx = fmaf(s, rx, gx); gy = fmaf(s, ry, gy); gz = fmaf(s, rz, gz);
        float* Gout = static_cast<float*>(P.o.G);
        __stcs(Gout + 3 * p + 0, gx);
        __stcs(Gout + 3 * p + 1, gy);
        __stcs(Gout + 3 * p + 2, gz);
        const float g3[3] = {gx, gy, gz}, r3[3] = {rx, ry, rz};
#pragma unroll
        for (int a2 = 0; a2 < 3; ++a2)
#pragma unroll
          for (int b2 = 0; b2 < 3; ++b2) Wl[3 * a2 + b2] = fmaf(-g3[a2], r3[b2], Wl[3 * a2 + b2]);
      }
      __syncwarp();
      if (MODE & F_ROWS) {
        const int nq = min(32, np - base);
        for (int e = lane; e < CBN; e += 32) {
          const int zj2 = e / (NR * NQ);
          const int mu = (e / NQ) % NR;
          const int b = e % NQ;
          float acc = 0.f;
          for (int qq = 0; qq < nq; ++qq)
            if (ZJ[qq] == zj2) acc = fmaf(GMb[NR * qq + mu], PQb[PQS * qq + b], acc);
          CB[e] += acc;
        }
      }
      __syncwarp();
    }
    if (MODE & F_EFS) {
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        // the neighborhood's virial in FP32 like its forces (FP64 instructions are scarce on this
        // GPU); the sums over atoms are FP64
        float v = Wl[k];
        for (int m = 16; m; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
        if (lane == 0) P.o.Wat[9 * i + k] = static_cast<double>(v);
      }
    }
    const int64_t rw = P.o.row_pos ? P.o.row_pos[i] : wk;   // this neighborhood's row of b
    if ((MODE & F_ROWS) && !P.row_stage) {
      const int64_t ld = P.o.rows_ld;
      float* hi = P.o.rows_hi ? P.o.rows_hi + rw * ld : nullptr;
      float* lo = P.o.rows_lo ? P.o.rows_lo + rw * ld : nullptr;
      double* out64 = P.o.rows ? P.o.rows + rw * ld : nullptr;
      auto put = [&](int64_t k, float v) {
        if (out64) out64[k] = v;
        if (hi) {
          float h = v;
          if (lo) {
            h = tf32_rn(v);
            lo[k] = tf32_rn(v - h);
          }
          hi[k] = h;
        }
      };
      for (int k = lane; k < T; k += 32) put(k, (k == zi) ? 1.f : 0.f);
      for (int a = lane; a < d.n_lin; a += 32) put(T + a, vals[d.basis_idx[a]]);
      for (int zblk = 0; zblk < T; ++zblk)
        for (int e = lane; e < CBN; e += 32) put(off_c + zblk * CBN + e, (zblk == zi) ? CB[e] : 0.f);
      for (int64_t k = d.n_params + lane; k < ld; k += 32) put(k, 0.f);
    }
    if ((MODE & F_ROWS) && P.row_stage) {
      // assemble b_i (eq. 9) in the adjoint buffer -- its values are no longer needed -- and
      // write it with 16-byte stores
      const int64_t ld = P.o.rows_ld;
      float* row = const_cast<float*>(grads);
      __syncwarp();
      for (int k = lane; k < ld; k += 32) row[k] = 0.f;
      __syncwarp();
      if (lane == 0) row[zi] = 1.f;
      for (int a = lane; a < d.n_lin; a += 32) row[T + a] = vals[d.basis_idx[a]];
      for (int e = lane; e < CBN; e += 32) row[off_c + zi * CBN + e] = CB[e];
      __syncwarp();
      if (P.o.rows) {
        double* out64 = P.o.rows + rw * ld;
        for (int k = lane; k < d.n_params; k += 32) out64[k] = row[k];
      }
      if (P.o.rows_hi) {
        float4* hi = reinterpret_cast<float4*>(P.o.rows_hi + rw * ld);
        float4* lo = P.o.rows_lo ? reinterpret_cast<float4*>(P.o.rows_lo + rw * ld) : nullptr;
        const float4* src = reinterpret_cast<const float4*>(row);
        for (int k = lane; k < ld / 4; k += 32) {
          const float4 v = src[k];
          if (lo) {
            const float4 h = make_float4(tf32_rn(v.x), tf32_rn(v.y), tf32_rn(v.z), tf32_rn(v.w));
            __stcs(hi + k, h);
            __stcs(lo + k, make_float4(tf32_rn(v.x - h.x), tf32_rn(v.y - h.y), tf32_rn(v.z - h.z), tf32_rn(v.w - h.w)));
          } else {
            hi[k] = v;
          }
        }
      }
    }
    __syncwarp();
  };

  for (int64_t wp = static_cast<int64_t>(blockIdx.x) * nwarps + warp; 2 * wp < P.n_work;
       wp += static_cast<int64_t>(gridDim.x) * nwarps) {
    const int64_t wk0 = 2 * wp, wk1 = 2 * wp + 1;
    const bool two = wk1 < P.n_work;
    const int64_t i0 = P.o.atom_list ? P.o.atom_list[wk0] : wk0;
    const int64_t i1 = two ? (P.o.atom_list ? P.o.atom_list[wk1] : wk1) : i0;
    moments(i0, valsA[0]);
    if (two) moments(i1, valsA[1]);
    float* v0 = valsA[0];
    float* v1 = valsA[1];
    float* g0 = gradsA[0];
    float* g1 = gradsA[1];
    // the contraction for one slab-word format (inline coefficient or coefficient table)
    auto contract = [&](auto inl) {
      constexpr bool INL = decltype(inl)::value;
      auto decode = [&](uint32_t w, float& c, uint32_t& x, uint32_t& y) {
        if constexpr (INL) {
          c = __uint_as_float(((w >> 22) << 17) + 0x3F800000u);
          x = w & 2047u;
          y = (w >> 11) & 2047u;
        } else {
          c = coef[w >> 24];
          x = w & 4095u;
          y = (w >> 12) & 4095u;
        }
      };
      // ---------------- forward contraction (eqs. 5-6): both neighborhoods per term ----------------
      // round headers are read one round ahead (the schedule copy is never written)
      int4 rd_n = d.n_fround > 0 ? s_fround[0] : make_int4(0, 0, 0, 0);
      int dst_n = d.n_fround > 0 ? s_frdst[lane] : -1;
      for (int r = 0; r < d.n_fround; ++r) {
        const int4 rd = rd_n;
        const int dst = dst_n;
        if (r + 1 < d.n_fround) {
          rd_n = s_fround[r + 1];
          dst_n = s_frdst[32 * (r + 1) + lane];
        }
        const uint32_t* slab = s_fslab + rd.y + lane;
        float a0 = 0.f, a1 = 0.f, b0 = 0.f, b1 = 0.f;
        int it = 0;
        for (; it + 2 <= rd.x; it += 2) {
          const uint32_t w0 = FG ? __ldg(slab + 32 * it) : slab[32 * it];
          const uint32_t w1 = FG ? __ldg(slab + 32 * it + 32) : slab[32 * it + 32];
          float c0, c1;
          uint32_t x0, y0, x1, y1;
          decode(w0, c0, x0, y0);
          decode(w1, c1, x1, y1);
          a0 = fmaf(c0, v0[x0] * v0[y0], a0);
          b0 = fmaf(c0, v1[x0] * v1[y0], b0);
          a1 = fmaf(c1, v0[x1] * v0[y1], a1);
          b1 = fmaf(c1, v1[x1] * v1[y1], b1);
        }
        if (it < rd.x) {
          const uint32_t w0 = FG ? __ldg(slab + 32 * it) : slab[32 * it];
          float c0;
          uint32_t x0, y0;
          decode(w0, c0, x0, y0);
          a0 = fmaf(c0, v0[x0] * v0[y0], a0);
          b0 = fmaf(c0, v1[x0] * v1[y0], b0);
        }
        if (dst >= 0) {
          v0[dst] = a0 + a1;
          v1[dst] = b0 + b1;
        }
        if (rd.z) __syncwarp();
      }
      // ---------------- adjoint of the contraction (gather form): both neighborhoods ----------------
      rd_n = d.n_rround > 0 ? s_rround[0] : make_int4(0, 0, 0, 0);   // the adjoint's headers likewise
      int x_n = d.n_rround > 0 ? s_rrval[lane] : -1;
      float sd_n = x_n >= 0 ? s_seed[x_n] : 0.f;
      int x_nn = d.n_rround > 1 ? s_rrval[32 + lane] : -1;
      for (int r = 0; r < d.n_rround; ++r) {
        const int4 rd = rd_n;
        const int x = x_n;
        const float sd = sd_n;
        if (r + 1 < d.n_rround) {
          rd_n = s_rround[r + 1];
          x_n = x_nn;
          sd_n = x_n >= 0 ? s_seed[x_n] : 0.f;
        }
        if (r + 2 < d.n_rround) x_nn = s_rrval[32 * (r + 2) + lane];
        const uint32_t* slab = s_rslab + rd.y + lane;
        float a0 = sd, a1 = 0.f, b0 = sd, b1 = 0.f;
        int it = 0;
        for (; it + 2 <= rd.x; it += 2) {
          const uint32_t w0 = slab[32 * it], w1 = slab[32 * it + 32];
          float c0, c1;
          uint32_t x0, y0, x1, y1;
          decode(w0, c0, x0, y0);
          decode(w1, c1, x1, y1);
          a0 = fmaf(c0, v0[x0] * g0[y0], a0);
          b0 = fmaf(c0, v1[x0] * g1[y0], b0);
          a1 = fmaf(c1, v0[x1] * g0[y1], a1);
          b1 = fmaf(c1, v1[x1] * g1[y1], b1);
        }
        if (it < rd.x) {
          const uint32_t w0 = slab[32 * it];
          float c0;
          uint32_t x0, y0;
          decode(w0, c0, x0, y0);
          a0 = fmaf(c0, v0[x0] * g0[y0], a0);
          b0 = fmaf(c0, v1[x0] * g1[y0], b0);
        }
        if (x >= 0) {
          g0[x] = a0 + a1;
          g1[x] = b0 + b1;
        }
        if (rd.z) __syncwarp();
      }
    };
    if (d.coef_inline) contract(std::true_type{});
    else contract(std::false_type{});
    finish(wk0, i0, v0, g0);
    if (two) finish(wk1, i1, v1, g1);
  }
}

template <int NR, int NU0, int MODE, bool FG>
void launch_fast(FastParams P, int nwarps, cudaStream_t s) {
  auto kern = site_fast_kernel<NR, NU0, MODE, FG>;
  MTP_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(P.total)));
  int dev = 0, nsm = 0, per_sm = 0;
  MTP_CUDA(cudaGetDevice(&dev));
  MTP_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  MTP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, nwarps * 32, P.total));
  per_sm = std::max(per_sm, 1);
  const int64_t need = ((P.n_work + 1) / 2 + nwarps - 1) / nwarps;
  const int grid = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(need, static_cast<int64_t>(nsm) * per_sm)));
  if (P.n_work == 0) return;
  ProfRegion pr((MODE & F_EFS) ? ((MODE & F_ROWS) ? "site_efs_rows" : "site_efs") : "site_rows", s);
  kern<<<grid, nwarps * 32, P.total, s>>>(P);
  ProfRegion::launched();
  MTP_CUDA(cudaGetLastError());
}

template <int NR, int NU0, bool FG>
void dispatch_mode(FastParams P, int nwarps, bool efs, bool rows, cudaStream_t s) {
  if (efs && rows) launch_fast<NR, NU0, F_EFS | F_ROWS, FG>(P, nwarps, s);
  else if (efs) launch_fast<NR, NU0, F_EFS, FG>(P, nwarps, s);
  else launch_fast<NR, NU0, F_ROWS, FG>(P, nwarps, s);
}

}  // namespace

// Returns false when the model's shape has no specialised instantiation (the caller then uses
// the generic kernel).
bool run_sites_fast(mtp_model* m, const mtp_batch* b, const mtp_nbr* nb, const SiteOutputs& o, cudaStream_t s) {
  const DevSchedule& d = m->ds;
  if (!d.tri_pk || d.n_q != kNQ) return false;
  const bool efs = o.V != nullptr;
  const bool rows = o.rows != nullptr || o.rows_hi != nullptr;
  if (!efs && !rows) return false;
  FastParams P{};
  P.d = d;
  P.nb = nb->dn;
  P.type = b->type;
  P.n_work = o.atom_list ? o.n_list : nb->n_atoms;
  P.o = o;
  P.NQ = d.n_q;
  P.CBN = d.n_types * d.n_rad * d.n_q;
  P.NC = d.n_types * P.CBN;
  P.NV = padded_nv(d.n_vals);
  // the staged row overwrites adjoint slots [0, ld): it must spare the zero slot n_vals
  P.row_stage = o.rows_ld > 0 && o.rows_ld <= d.n_vals && (o.rows_ld & 3) == 0;
  P.c_bytes = (static_cast<size_t>(P.NC) * sizeof(float) + 15) & ~size_t(15);
  P.tab_bytes = ((256 + d.n_mom) * sizeof(float) + 15) & ~size_t(15);
  // pair-adjoint scratch inside the finished neighborhood's adjoint array when it fits above the
  // moment adjoints, with its radial block at or above the staged row (which rewrites [0, ld))
  // and below the zero slot n_vals; otherwise one scratch block per warp
  const int aux_head = 32 * (d.n_rad + d.n_q + 1) + 32;   // GM, PQ (odd stride), ZJ before the radial block
  const int aux_need = aux_head + P.CBN;
  int aux_off = std::max((d.n_mom + 3) & ~3, (P.row_stage ? static_cast<int>(o.rows_ld) : 0) - aux_head);
  aux_off = (aux_off + 3) & ~3;
  P.aux_off = (rows && aux_off + aux_need <= d.n_vals) ? aux_off : 0;
  P.warp_bytes = ((4 * static_cast<size_t>(P.NV) + (P.aux_off > 0 ? 0 : aux_need)) * sizeof(float) + 15) & ~size_t(15);
  // shared-memory copy of the schedule (32-bit words); fwd_global: without the forward slab
  const int nu0 = d.nu_max, nr = d.n_rad;
  const bool fg_shape = nr == 5 && nu0 == 8;   // the shape with a global-forward instantiation
  const size_t limit = 227 * 1024;
  auto layout = [&](bool fg, FastParams& Q) {
    int w = 0;
    auto take = [&](int n) { const int o = w; w += (n + 3) & ~3; return o; };
    Q.o_fslab = fg ? 0 : take(d.fslab_words);
    Q.o_fround = take(4 * d.n_fround);
    Q.o_frdst = take(32 * d.n_fround);
    Q.o_rslab = take(d.rslab_words);
    Q.o_rround = take(4 * d.n_rround);
    Q.o_rrval = take(32 * d.n_rround);
    Q.o_seed = take(d.n_vals);
    Q.sched_bytes = static_cast<size_t>(w) * 4;
    const size_t fixed = Q.c_bytes + Q.tab_bytes + Q.sched_bytes;
    if (fixed + 2 * Q.warp_bytes > limit) return 0;
    return static_cast<int>(std::min<size_t>(kMaxWarpsF, (limit - fixed) / Q.warp_bytes));
  };
  FastParams Ps = P, Pg = P;
  const int ws = layout(false, Ps);
  const int wg = fg_shape ? layout(true, Pg) : 0;
  // placement: the tuned one, else the one with more warps per SM once the global-forward
  // placement's default cap of 7 is applied (shared memory on ties: measured faster, the forward
  // slab then does not compete for L1)
  bool fg = m->tune_fwd_global >= 0 ? (m->tune_fwd_global == 1 && wg > 0) : (std::min(wg, 7) > ws);
  if (!fg && ws == 0) fg = wg > 0;
  if (!fg && ws == 0) return false;
  P = fg ? Pg : Ps;
  int nwarps = fg ? wg : ws;
  // untuned default: at most 7 warps with the forward schedule in global memory (8 fit at level
  // 20 but ran 5 % slower there); mtp_autotune times every shape
  if (m->tune_warps_fast > 0) nwarps = std::min(nwarps, m->tune_warps_fast);
  else if (fg) nwarps = std::min(nwarps, 7);
  m->last_warps = nwarps;
  m->last_fast = true;
  m->last_fwd_global = fg;
  P.total = P.c_bytes + P.tab_bytes + P.sched_bytes + nwarps * P.warp_bytes;
  if (fg) { dispatch_mode<5, 8, true>(P, nwarps, efs, rows, s); return true; }
  if (nr == 2 && nu0 == 2) { dispatch_mode<2, 2, false>(P, nwarps, efs, rows, s); return true; }
  if (nr == 3 && nu0 == 4) { dispatch_mode<3, 4, false>(P, nwarps, efs, rows, s); return true; }
  if (nr == 4 && nu0 == 6) { dispatch_mode<4, 6, false>(P, nwarps, efs, rows, s); return true; }
  if (nr == 5 && nu0 == 8) { dispatch_mode<5, 8, false>(P, nwarps, efs, rows, s); return true; }
  return false;
}

}  // namespace mtp

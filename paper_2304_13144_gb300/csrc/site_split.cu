// Mixed-path (FP32 arithmetic, FP64 sums) per-neighborhood pass as three kernels, each laid
// out for its own phase of the method:
//
//   k_moments   (eqs. 3-4)  8 lanes per neighborhood, 4 neighborhoods per warp.  The lanes
//               stage their pairs' r_ij and f_mu(r_ij) in shared memory, then for every
//               32-component chunk of the moment set each lane sums f_mu x^a y^b z^c over its
//               own pairs in registers and one 3-stage butterfly over the 8 lanes leaves each
//               lane with 4 component sums.  Output: the moments, FP32, [work x ldm].
//   k_contract  (eqs. 2, 5-6 and their adjoint)  one or two neighborhoods per warp carried
//               through the contraction schedule (32-lane slabs of packed triples in shared
//               memory, as in site_fast.cu), V_i = s_z + sum_a xi_a B_a, the reverse pass seeded
//               with xi, and the adjoints dV/dM written over the moments.  The basis part of
//               the parameter row b_i (eq. 9) is written here.
//   k_adjoint   (forces and virial; the radial block of eq. 9)  8 lanes per neighborhood: per
//               pair dV_i/dr_ij from dV/dM (monomials regenerated in registers), the per-pair
//               gradients for the force gather, the neighborhood's virial, and
//               sum_j g_mu(j) Q_b(r_ij) per neighbor species for b_i.
//
// Splitting frees each phase from the others' resources: the contraction runs without the
// per-pair phases' 255 registers (more warps per SM, deeper unrolling), and the per-pair phases
// fill their lanes (about 44 pairs over 8 lanes use 92 % of the lane slots; 32 lanes per
// neighborhood used 69 %).  The moments and their adjoints cross HBM once each way
// (4 ldm bytes per atom, each way).
#include <cuda_runtime.h>

#include <algorithm>
#include <string>
#include <vector>

#include "mtp_internal.h"
#include "profiler.h"
#include "site_shape.h"

namespace mtp {
namespace {
using namespace shape;

constexpr int kNQs = 8;      // radial polynomials of the specialised kernels
constexpr int LPN = 8;       // lanes per neighborhood in the per-pair kernels
constexpr int GPW = 32 / LPN;
constexpr int BATCH = 64;    // pairs staged per neighborhood at a time (moments)
constexpr int BATCH_A = 32;  // pairs staged per neighborhood at a time (pair adjoint)
constexpr int GS = 17;       // floats staged per pair for the radial block: g_mu, Q_b, species (odd)

// float4 arrays staged per pair by the moment kernel: (x, y, z, f_0), then f_1.. four at a time
__host__ __device__ constexpr int stage_f4(int nr) { return 1 + (nr - 1 + 3) / 4; }
// moment components held per lane by the contraction kernel (n_mom <= 32 PRE) and the species
// of the radial-block accumulators of the pair-adjoint kernel, per shape
__host__ __device__ constexpr int pre_of(int nr) { return nr <= 5 ? 10 : 19; }
__host__ __device__ constexpr int tmax_of(int nr) { return nr <= 5 ? 3 : 4; }

// shared-memory floats per neighborhood group of the pair-adjoint kernel: dV/dM (ldm rounded up
// to 32, plus 8) then the radial-block staging; the stride is 8 mod 32 banks, so the four groups'
// broadcast reads of one component hit four different banks, and with the odd per-pair stride
// the 32 lanes' staging stores hit 32 different banks
__host__ __device__ inline int adj_region(int ldm, bool rows) {
  return ((ldm + 31) & ~31) + 8 + (rows ? BATCH_A * GS : 0);
}

struct SplitArgs {
  DevSchedule d;
  DevNbr nb;
  const int* type;
  int64_t n_work;
  SiteOutputs o;
  float* mom;   // [n_work x ldm]: moments (k_moments), overwritten by dV/dM (k_contract), both in
                // slot order (monomial-major, the order of the moment pass's chunks)
  int ldm;
  const int* slot_comp;   // slot -> value index of the moment component
  int T, CBN, NC, NV;
  // contraction kernel: shared-memory layout (word offsets of the schedule arrays)
  size_t c_bytes, sched_bytes, warp_bytes, total;
  size_t ovf_bytes;   // schedule in tensor memory: the stream rows past its 512 columns
  int o_fslab, o_fround, o_frdst, o_rslab, o_rround, o_rrval, o_seed;
};

__device__ __forceinline__ int64_t atom_of(const SplitArgs& P, int64_t wk) {
  return P.o.atom_list ? P.o.atom_list[wk] : wk;
}

// Range-checked element access (compiled in with MTP_SPLIT_CHECK): an index outside [0, n) is
// recorded (the first one: check code and index) and the access goes to a scratch slot instead.
#ifdef MTP_SPLIT_CHECK
__device__ unsigned long long g_split_fault;
__device__ __align__(16) unsigned char g_split_dummy[64];
template <class T>
__device__ __forceinline__ T& AT(T* p, long long i, long long n, int code) {
  if (i < 0 || i >= n) {
    atomicCAS(&g_split_fault, 0ull,
              (static_cast<unsigned long long>(code) << 48) | (static_cast<unsigned long long>(i) & 0xFFFFFFFFFFFFull));
    return *reinterpret_cast<T*>(g_split_dummy);
  }
  return p[i];
}
__device__ __forceinline__ bool OK(long long i, long long n, int code) {
  if (i >= 0 && i < n) return true;
  atomicCAS(&g_split_fault, 0ull,
            (static_cast<unsigned long long>(code) << 48) | (static_cast<unsigned long long>(i) & 0xFFFFFFFFFFFFull));
  return false;
}
#else
template <class T>
__device__ __forceinline__ T& AT(T* p, long long i, long long, int) { return p[i]; }
__device__ __forceinline__ constexpr bool OK(long long, long long, int) { return true; }
#endif

// v[0..31] on each of the LPN lanes of a group -> lane q of the group holds, in v[0..3], the sums
// over the group of components 4q .. 4q+3 (recursive halving: the lane with bit s of q set keeps
// the upper half and receives its partner's upper half)
__device__ __forceinline__ void group_reduce32(float (&v)[32], int q) {
  static_assert(LPN == 8, "the butterfly is written for 8 lanes");
  static_for<0, 3>([&](auto S) {
    constexpr int st = decltype(S)::value;
    constexpr int s = 4 >> st;        // partner distance 4, 2, 1
    constexpr int h = 16 >> st;       // values exchanged: 16, 8, 4
    const bool up = (q & s) != 0;
    static_for<0, h>([&](auto I) {
      constexpr int i = decltype(I)::value;
      const float send = up ? v[i] : v[i + h];
      const float keep = up ? v[i + h] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, s);
    });
  });
}

__device__ __forceinline__ float group_sum(float v) {
  v += __shfl_xor_sync(0xffffffffu, v, 4);
  v += __shfl_xor_sync(0xffffffffu, v, 2);
  v += __shfl_xor_sync(0xffffffffu, v, 1);
  return v;
}

// x^A y^B z^C from the power tables (compile-time exponents, no multiply by 1)
template <int A, int B, int C, int D>
__device__ __forceinline__ float mono_of(const float (&px)[D], const float (&py)[D], const float (&pz)[D]) {
  if constexpr (A + B + C == 0) {
    return 1.f;
  } else if constexpr (A > 0 && B > 0 && C > 0) {
    return px[A] * py[B] * pz[C];
  } else if constexpr (A > 0 && B > 0) {
    return px[A] * py[B];
  } else if constexpr (A > 0 && C > 0) {
    return px[A] * pz[C];
  } else if constexpr (B > 0 && C > 0) {
    return py[B] * pz[C];
  } else if constexpr (A > 0) {
    return px[A];
  } else if constexpr (B > 0) {
    return py[B];
  } else {
    return pz[C];
  }
}

template <int NR, int NU0>
struct ChunkInfo {
  using Sh = Shape<NR, NU0>;
  using Tb = Tab<NR, NU0>;
  static constexpr int deg_hi(int c) {
    int d = 0;
    for (int s = 32 * c; s < 32 * c + 32 && s < Sh::NCOMP; ++s) d = Tb::mono.deg[Tb::slots.k[s]] > d ? Tb::mono.deg[Tb::slots.k[s]] : d;
    return d;
  }
};

// ------------------------------------------------------------------------------------
// moments (eqs. 3-4)
// ------------------------------------------------------------------------------------
template <int NR, int NU0>
__global__ void __launch_bounds__(256) k_moments(SplitArgs P) {
  using Sh = Shape<NR, NU0>;
  using Tb = Tab<NR, NU0>;
  using CI = ChunkInfo<NR, NU0>;
  constexpr int NQ = kNQs;
  constexpr int NF4 = stage_f4(NR);
  extern __shared__ __align__(16) unsigned char smem[];
  const DevSchedule& d = P.d;
  float* ctab = reinterpret_cast<float*>(smem);
  const int T = P.T;
  for (int k = threadIdx.x; k < P.NC; k += blockDim.x)
    if (OK(T + d.n_lin + k, d.n_params, 1)) ctab[k] = d.theta_f[T + d.n_lin + k];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, grp = lane / LPN, q = lane % LPN;
  const int nwarps = blockDim.x >> 5;
  // per group: (x, y, z, f_0), (f_1 .. f_4), (f_5, 0, 0, 0) of each staged pair as NF4 float4
  // arrays; the 8 lanes of a group read 8 consecutive float4 (one conflict-free phase of a
  // 128-bit load)
  float4* stg = reinterpret_cast<float4*>(smem + P.c_bytes) + (static_cast<size_t>(warp) * GPW + grp) * NF4 * BATCH;
  __syncthreads();
  const float rmin = static_cast<float>(d.r_min), rcut = static_cast<float>(d.r_cut);
  for (int64_t w0 = (static_cast<int64_t>(blockIdx.x) * nwarps + warp) * GPW; w0 < P.n_work;
       w0 += static_cast<int64_t>(gridDim.x) * nwarps * GPW) {
    const int64_t wk = w0 + grp;
    const bool live = wk < P.n_work;
    int np = 0, zi = 0;
    int64_t p0 = 0;
    if (live && OK(wk, P.nb.n_atoms, 3)) {
      const int64_t i = atom_of(P, wk);
      zi = P.type[i];
      p0 = P.nb.off[i];
      np = static_cast<int>(P.nb.off[i + 1] - p0);
      if (!OK(zi, T, 4) || !OK(p0 + np - 1 + (np == 0), P.nb.n_pairs + 1, 5)) { zi = 0; np = 0; }
    }
    // the warp walks the batches of its largest neighborhood (all lanes take part in the butterflies)
    int np_max = np;
    for (int m = 16; m; m >>= 1) np_max = max(np_max, __shfl_xor_sync(0xffffffffu, np_max, m));
    const float* czi = ctab + static_cast<size_t>(zi) * T * NR * NQ;
    float* out = live ? P.mom + wk * P.ldm : nullptr;
    // at least one pass, so that a neighborhood without pairs gets zero moments
    for (int base = 0; base < max(np_max, 1); base += BATCH) {
      const int nbt = min(BATCH, np - base);   // <= 0 for a group that is done
      __syncwarp();
      for (int t = q; t < nbt; t += LPN) {
        const int64_t p = p0 + base + t;
        if (!OK(p, P.nb.n_pairs, 6) || !OK(t, BATCH, 7)) continue;
        const float4 r = P.nb.pr32[p];
        const int jj = P.nb.pj[p];
        if (!OK(jj, P.nb.n_atoms, 8)) continue;
        const int zj = P.type[jj];
        if (!OK(zj, T, 9)) continue;
        float f[NR], df[NR];
        radial<NR, NQ>(r.w, czi + zj * NR * NQ, rmin, rcut, f, df, nullptr);
        float fe[4 * NF4 - 3];
#pragma unroll
        for (int k = 0; k < 4 * NF4 - 3; ++k) fe[k] = k < NR ? f[k < NR ? k : 0] : 0.f;
        stg[t] = make_float4(r.x, r.y, r.z, fe[0]);
#pragma unroll
        for (int k = 1; k < NF4; ++k) stg[k * BATCH + t] = make_float4(fe[4 * k - 3], fe[4 * k - 2], fe[4 * k - 1], fe[4 * k]);
      }
      __syncwarp();
      static_for<0, Sh::NCHUNK>([&](auto Cc) {
        constexpr int c = decltype(Cc)::value;
        constexpr int DH = CI::deg_hi(c);
        float acc[32];
#pragma unroll
        for (int t = 0; t < 32; ++t) acc[t] = 0.f;
        for (int t = q; t < nbt; t += LPN) {
          if (!OK(t, BATCH, 10)) continue;
          const float4 ea = stg[t];
          const float x = ea.x, y = ea.y, z = ea.z;
          float f[NR];
          f[0] = ea.w;
#pragma unroll
          for (int k = 1; k < NF4; ++k) {
            const float4 eb = stg[k * BATCH + t];
            const float e4[4] = {eb.x, eb.y, eb.z, eb.w};
#pragma unroll
            for (int u = 0; u < 4; ++u)
              if (4 * k - 3 + u < NR) f[4 * k - 3 + u < NR ? 4 * k - 3 + u : 0] = e4[u];
          }
          float px[DH + 1], py[DH + 1], pz[DH + 1];
          px[0] = py[0] = pz[0] = 1.f;
#pragma unroll
          for (int k = 1; k <= DH; ++k) {
            px[k] = k == 1 ? x : px[k - 1] * x;
            py[k] = k == 1 ? y : py[k - 1] * y;
            pz[k] = k == 1 ? z : pz[k - 1] * z;
          }
          float mk = 0.f;
          static_for<0, 32>([&](auto Tt) {
            constexpr int t2 = decltype(Tt)::value;
            constexpr int s = 32 * c + t2;
            if constexpr (s < Sh::NCOMP) {
              constexpr int k = Tb::slots.k[s];
              constexpr int mu = Tb::slots.mu[s];
              constexpr bool fresh = (t2 == 0) ? true : (Tb::slots.k[s > 0 ? s - 1 : 0] != k);
              if constexpr (fresh) mk = mono_of<Tb::mono.a[k], Tb::mono.b[k], Tb::mono.c[k]>(px, py, pz);
              acc[t2] = fmaf(f[mu], mk, acc[t2]);
            }
          });
        }
        group_reduce32(acc, q);
        // lane q holds slots 32c + 4q .. +3 (zeros past the last slot; ldm covers them)
        if (live && 32 * c + 4 * q < Sh::NCOMP && OK(wk * P.ldm + 32 * c + 4 * q + 3, P.n_work * P.ldm, 11)) {
          float4* o4 = reinterpret_cast<float4*>(out + 32 * c + 4 * q);
          float4 val = make_float4(acc[0], acc[1], acc[2], acc[3]);
          if (base > 0) {
            const float4 prev = *o4;
            val.x += prev.x; val.y += prev.y; val.z += prev.z; val.w += prev.w;
          }
          *o4 = val;
        }
      });
    }
  }
}

// ------------------------------------------------------------------------------------
// contraction and its adjoint (eqs. 2, 5-6); NB neighborhoods per warp
// ------------------------------------------------------------------------------------
__device__ __forceinline__ void copy_words_s(uint32_t* dst, const uint32_t* src, int n) {
  for (int k = threadIdx.x; k < n; k += blockDim.x) dst[k] = src[k];
}

// one slab word: a += c v[x] v[y] (forward) or a += c v[x] g[y] (reverse, w = the adjoint array)
template <int NB, bool INL>
__device__ __forceinline__ void slab_term(uint32_t wd, const float* coef, float* const (&v)[NB], float* const (&w)[NB],
                                          float (&a)[NB]) {
  float c;
  uint32_t x, y;
  if constexpr (INL) {
    c = __uint_as_float(((wd >> 22) << 17) + 0x3F800000u);
    x = wd & 2047u;
    y = (wd >> 11) & 2047u;
  } else {
    c = coef[wd >> 24];
    x = wd & 4095u;
    y = (wd >> 12) & 4095u;
  }
#pragma unroll
  for (int j = 0; j < NB; ++j) a[j] = fmaf(c, v[j][x] * w[j][y], a[j]);
}

// one round of 32 destination lists (L words per lane, lane stride 32) from a schedule in shared
// memory, UNR words per step, the next step's words loaded while the current ones are used;
// word it always goes to chain it % 2 (the sum is the same for every UNR, and for the streamed
// variant below, bit for bit)
template <int NB, bool INL, int UNR>
__device__ __forceinline__ void slab_round(const uint32_t* slab, int L, const float* coef, float* const (&v)[NB],
                                           float* const (&w)[NB], float (&acc)[NB]) {
  static_assert(UNR % 2 == 0, "whole pairs of words per iteration");
  float a[2][NB];
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int j = 0; j < NB; ++j) a[u][j] = 0.f;
  const int LU = L - L % UNR;   // rows of the whole steps
  uint32_t nxt[UNR];
  if (LU > 0) {
#pragma unroll
    for (int u = 0; u < UNR; ++u) nxt[u] = slab[32 * u];
  }
  for (int it = 0; it < LU; it += UNR) {
    uint32_t wd[UNR];
#pragma unroll
    for (int u = 0; u < UNR; ++u) wd[u] = nxt[u];
    if (it + UNR < LU) {
#pragma unroll
      for (int u = 0; u < UNR; ++u) nxt[u] = slab[32 * (it + UNR + u)];
    }
#pragma unroll
    for (int u = 0; u < UNR; ++u) slab_term<NB, INL>(wd[u], coef, v, w, a[u & 1]);
  }
  for (int it = LU; it < L; ++it) slab_term<NB, INL>(slab[32 * it], coef, v, w, a[it & 1]);
#pragma unroll
  for (int j = 0; j < NB; ++j) acc[j] += a[0][j] + a[1][j];
}

// Streamed schedule (a level whose schedule does not fit shared memory beside the value
// arrays): the forward and reverse slabs, one after the other, form a stream of rows (32 words,
// 128 B each) that repeats for every neighborhood iteration, padded to whole chunks of kCR rows.
// The block's threads copy chunk c into ring slot c % kRing with cp.async while chunk c - 1 is
// in use; every warp walks the same rows, so at the first row of chunk k all of them meet,
// wait for its copies, and start the copy of chunk k + kRing - 1 into the slot just freed.
constexpr int kCR = 32;     // rows per chunk (4 KB)
constexpr int kRing = 2;    // chunks in the ring
__host__ __device__ constexpr size_t ring_bytes() { return static_cast<size_t>(kRing) * kCR * 32 * 4; }

struct Stream {
  uint32_t* ring;
  const uint32_t* fsl;   // forward slab rows [0, FR), then reverse slab rows [FR, TR)
  const uint32_t* rsl;
  int FR, TR, TRp;       // TRp: TR rounded up to whole chunks
};

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// copy chunk c of the stream into its ring slot (all threads of the block; one commit group)
__device__ __forceinline__ void issue_chunk(const Stream& S, long long c) {
  const int local = static_cast<int>((c * kCR) % S.TRp);
  uint32_t* dst = S.ring + static_cast<int>(c % kRing) * kCR * 32;
  for (int u = threadIdx.x; u < kCR * 8; u += blockDim.x) {
    const int row = local + (u >> 3), l4 = (u & 7) * 4;
    const uint32_t* src = row < S.FR ? S.fsl + 32 * row + l4 : (row < S.TR ? S.rsl + 32 * (row - S.FR) + l4 : nullptr);
    if (src) cp_async16(dst + (u >> 3) * 32 + l4, src);
  }
  cp_async_commit();
}

// the round starting at stream row R0 (of this iteration's rows), L rows
template <int NB, bool INL, int UNR>
__device__ __forceinline__ void slab_round_stream(const Stream& S, long long R0, int L, int lane, const float* coef,
                                                  float* const (&v)[NB], float* const (&w)[NB], float (&acc)[NB]) {
  static_assert(UNR % 2 == 0, "whole pairs of words per iteration");
  float a[2][NB];
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int j = 0; j < NB; ++j) a[u][j] = 0.f;
  int it = 0;
  while (it < L) {
    const long long R = R0 + it;
    const int off = static_cast<int>(R % kCR);
    if (off == 0) {   // the first row of chunk k = R / kCR: the same point for every warp
      cp_async_wait<kRing - 2>();
      __syncthreads();
      issue_chunk(S, R / kCR + kRing - 1);
    }
    const int end = it + min(L - it, kCR - off);
    // rows it .. end - 1 of the round are rows off .. of the chunk's slot
    const uint32_t* slab = S.ring + static_cast<int>((R / kCR) % kRing) * kCR * 32 + (off - it) * 32 + lane;
    if ((it & 1) && it < end) {   // an odd first row: chains stay those of the round's row index
      slab_term<NB, INL>(slab[32 * it], coef, v, w, a[1]);
      ++it;
    }
    for (; it + UNR <= end; it += UNR) {
      uint32_t wd[UNR];
#pragma unroll
      for (int u = 0; u < UNR; ++u) wd[u] = slab[32 * (it + u)];
#pragma unroll
      for (int u = 0; u < UNR; ++u) slab_term<NB, INL>(wd[u], coef, v, w, a[u & 1]);
    }
    // fewer than UNR rows left, from an even row: chains 0, 1, 0, ...
#pragma unroll
    for (int u = 0; u < UNR - 1; ++u)
      if (it < end) {
        slab_term<NB, INL>(slab[32 * it], coef, v, w, a[u & 1]);
        ++it;
      }
  }
#pragma unroll
  for (int j = 0; j < NB; ++j) acc[j] += a[0][j] + a[1][j];
}

// Schedule in tensor memory (a level whose slab stream has few rows beyond 512): the first
// kTmemRows rows of the stream (forward slab rows, then reverse slab rows) sit in the block's
// 512 TMEM columns, row r in column r, lane l of the row in TMEM lane 32 q + l of every lane
// quarter q (a warp reads the quarter of its warp index mod 4); rows past them, the round
// headers, lane entries and seeds in shared memory.  This leaves shared memory to the value
// arrays (two neighborhoods per warp, 11 warps at level 20).  Words are read with tcgen05.ld (32 lanes x 32 bit, one column), the next step's in
// flight while the current step's are used; tcgen05.wait::ld names the loaded registers, so no
// use of them is scheduled before it.
constexpr int kTmemRows = 512;

template <int N>
__device__ __forceinline__ void tmem_ld_rows(uint32_t taddr, uint32_t (&w)[N]) {
#pragma unroll
  for (int u = 0; u < N; ++u)
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(w[u]) : "r"(taddr + u) : "memory");
}
template <int N>
__device__ __forceinline__ void tmem_wait_rows(uint32_t (&w)[N]) {
  if constexpr (N == 1) asm volatile("tcgen05.wait::ld.sync.aligned;" : "+r"(w[0])::"memory");
  else if constexpr (N == 2) asm volatile("tcgen05.wait::ld.sync.aligned;" : "+r"(w[0]), "+r"(w[1])::"memory");
  else if constexpr (N == 4)
    asm volatile("tcgen05.wait::ld.sync.aligned;" : "+r"(w[0]), "+r"(w[1]), "+r"(w[2]), "+r"(w[3])::"memory");
  else if constexpr (N == 8)
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(w[0]), "+r"(w[1]), "+r"(w[2]), "+r"(w[3]), "+r"(w[4]), "+r"(w[5]), "+r"(w[6]), "+r"(w[7])::"memory");
  else static_assert(N == 1 || N == 2 || N == 4 || N == 8, "steps of 1, 2, 4 or 8 words");
}

// the round starting at stream row R0, L rows: rows below kTmemRows from TMEM (tq = the TMEM
// address of column 0 in this warp's lane quarter), the others from `ovf` (shared memory, row
// kTmemRows first, this lane's word at ovf[32 (row - kTmemRows)])
template <int NB, bool INL, int UNR>
__device__ __forceinline__ void slab_round_tmem(uint32_t tq, const uint32_t* ovf, int R0, int L, const float* coef,
                                                float* const (&v)[NB], float* const (&w)[NB], float (&acc)[NB]) {
  static_assert(UNR % 2 == 0, "whole pairs of words per iteration");
  float a[2][NB];
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int j = 0; j < NB; ++j) a[u][j] = 0.f;
  const int Lt = max(0, min(L, kTmemRows - R0));   // rows in tensor memory
  const int LU = Lt - Lt % UNR;
  if (LU > 0) {
    uint32_t nxt[UNR];
    tmem_ld_rows<UNR>(tq + R0, nxt);
    tmem_wait_rows<UNR>(nxt);
    for (int it = 0; it < LU; it += UNR) {
      uint32_t wd[UNR];
#pragma unroll
      for (int u = 0; u < UNR; ++u) wd[u] = nxt[u];
      const bool more = it + UNR < LU;
      if (more) tmem_ld_rows<UNR>(tq + R0 + it + UNR, nxt);
#pragma unroll
      for (int u = 0; u < UNR; ++u) slab_term<NB, INL>(wd[u], coef, v, w, a[u & 1]);
      if (more) tmem_wait_rows<UNR>(nxt);
    }
  }
  int it = LU;
#pragma unroll
  for (int u = 0; u < UNR - 1; ++u)   // fewer than UNR rows left, from an even row: chains 0, 1, 0
    if (it < Lt) {
      uint32_t t1[1];
      tmem_ld_rows<1>(tq + R0 + it, t1);
      tmem_wait_rows<1>(t1);
      slab_term<NB, INL>(t1[0], coef, v, w, a[u & 1]);
      ++it;
    }
  if (it < L) {   // rows past tensor memory
    const uint32_t* slab = ovf + 32 * (R0 - kTmemRows);
    if ((it & 1) && it < L) {
      slab_term<NB, INL>(slab[32 * it], coef, v, w, a[1]);
      ++it;
    }
    for (; it + 2 <= L; it += 2) {
      const uint32_t w0 = slab[32 * it], w1 = slab[32 * (it + 1)];
      slab_term<NB, INL>(w0, coef, v, w, a[0]);
      slab_term<NB, INL>(w1, coef, v, w, a[1]);
    }
    if (it < L) slab_term<NB, INL>(slab[32 * it], coef, v, w, a[0]);
  }
#pragma unroll
  for (int j = 0; j < NB; ++j) acc[j] += a[0][j] + a[1][j];
}

// partial sums of a list split over an aligned group of 2^lg lanes (lane entry bits 16..19):
// after the butterfly every lane of the group holds the group's total (idle lanes: garbage)
template <int NB>
__device__ __forceinline__ void group_combine(float (&acc)[NB], int ent) {
  const int g = 1 << ((ent >> 16) & 15);
#pragma unroll
  for (int s = 1; s < 32; s <<= 1) {
#pragma unroll
    for (int j = 0; j < NB; ++j) {
      const float t = __shfl_xor_sync(0xffffffffu, acc[j], s);
      if (g > s) acc[j] += t;
    }
  }
}

// PRE: moment components per lane prefetched in registers (n_mom <= 32 PRE).  GSCH: the schedule
// stays in global memory (a level whose schedule does not fit shared memory next to the value
// arrays): the slab words are streamed through a two-chunk ring in shared memory (Stream above),
// the round headers and lane entries read from global memory (L1) a round ahead; every warp of
// a block runs the same number of neighborhood iterations (a warp past the end computes on zeros
// and writes nothing), so that all of them reach every chunk boundary.
template <int NB, bool INL, int UNR, int PRE, int SCH>
__global__ void __launch_bounds__(SCH == 1 ? 256 : (SCH == 2 ? 384 : 512), 1) k_contract(SplitArgs P) {
  constexpr bool GSCH = SCH == 1;   // streamed through the shared ring
  constexpr bool TMS = SCH == 2;    // in tensor memory
  extern __shared__ __align__(16) unsigned char smem[];
  const DevSchedule& d = P.d;
  const int NV = P.NV;
  float* coef = reinterpret_cast<float*>(smem);
  for (int k = threadIdx.x; k < d.n_coef; k += blockDim.x)
    if (OK(k * 4 + 3, static_cast<long long>(P.c_bytes), 20)) coef[k] = d.coef_f[k];
  const uint32_t* s_fslab;
  const int4* s_fround;
  const int* s_frdst;
  const uint32_t* s_rslab;
  const int4* s_rround;
  const int* s_rrval;
  const float* s_seed;
  Stream S{};
  __shared__ uint32_t tmem_slot;
  uint32_t tq = 0;              // TMS: TMEM address of column 0 in this warp's lane quarter
  const uint32_t* ovf = nullptr;   // TMS: stream rows past tensor memory (this lane's word)
  if constexpr (TMS) {
    const int nw = blockDim.x >> 5, wp = threadIdx.x >> 5, ln = threadIdx.x & 31;
    if (wp == 0) {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                       static_cast<unsigned>(__cvta_generic_to_shared(&tmem_slot))),
                   "r"(512));
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int FR = d.pfslab_words / 32, TR = FR + d.prslab_words / 32, TT = min(TR, kTmemRows);
    const int q = wp & 3;
    tq = tmem_slot + (static_cast<uint32_t>(32 * q) << 16);
    // the warps of lane quarter q write its copy of rows [0, TT), one column per store
    const int nq = (nw - q + 3) / 4, kq = wp >> 2;
    for (int r = kq; r < TT; r += nq) {
      const uint32_t word = r < FR ? d.pfslab[32 * r + ln] : d.prslab[32 * (r - FR) + ln];
      asm volatile("tcgen05.st.sync.aligned.32x32b.x1.b32 [%0], {%1};" ::"r"(tq + r), "r"(word) : "memory");
    }
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    uint32_t* o = reinterpret_cast<uint32_t*>(smem + P.c_bytes);
    for (int k = threadIdx.x; k < 32 * (TR - TT); k += blockDim.x) {
      const int r = TT + k / 32;
      o[k] = r < FR ? d.pfslab[32 * r + (k & 31)] : d.prslab[32 * (r - FR) + (k & 31)];
    }
    ovf = o + ln;
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    S.FR = FR;
  }
  if constexpr (GSCH || TMS) {
    if constexpr (GSCH) {
      S.ring = reinterpret_cast<uint32_t*>(smem + P.c_bytes);
      S.fsl = d.pfslab;
      S.rsl = d.prslab;
      S.FR = d.pfslab_words / 32;
      S.TR = S.FR + d.prslab_words / 32;
      S.TRp = (S.TR + kCR - 1) / kCR * kCR;
    }
    s_fslab = d.pfslab;
    s_fround = reinterpret_cast<const int4*>(d.pfround);
    s_frdst = d.pfr_dst;
    s_rslab = d.prslab;
    s_rround = reinterpret_cast<const int4*>(d.prround);
    s_rrval = d.prr_val;
    s_seed = d.seed_f;
    if constexpr (TMS) {
      // round headers, lane entries and seeds in shared memory after the overflow rows (one warp
      // fewer than with them read through L1, 13.10 against 13.51 ms at level 20)
      const int TR = (d.pfslab_words + d.prslab_words) / 32, TT = min(TR, kTmemRows);
      uint32_t* h = reinterpret_cast<uint32_t*>(smem + P.c_bytes) + 32 * (TR - TT);
      int o = 0;
      auto put = [&](const uint32_t* src, int n) {
        copy_words_s(h + o, src, n);
        const int at = o;
        o += (n + 3) & ~3;
        return h + at;
      };
      s_fround = reinterpret_cast<const int4*>(put(reinterpret_cast<const uint32_t*>(d.pfround), 4 * d.n_pfround));
      s_frdst = reinterpret_cast<const int*>(put(reinterpret_cast<const uint32_t*>(d.pfr_dst), 32 * d.n_pfround));
      s_rround = reinterpret_cast<const int4*>(put(reinterpret_cast<const uint32_t*>(d.prround), 4 * d.n_prround));
      s_rrval = reinterpret_cast<const int*>(put(reinterpret_cast<const uint32_t*>(d.prr_val), 32 * d.n_prround));
      s_seed = reinterpret_cast<const float*>(put(reinterpret_cast<const uint32_t*>(d.seed_f), d.n_vals));
      __syncthreads();
    }
  } else {
    uint32_t* sched = reinterpret_cast<uint32_t*>(smem + P.c_bytes);
    copy_words_s(sched + P.o_fslab, d.pfslab, d.pfslab_words);
    copy_words_s(sched + P.o_fround, reinterpret_cast<const uint32_t*>(d.pfround), 4 * d.n_pfround);
    copy_words_s(sched + P.o_frdst, reinterpret_cast<const uint32_t*>(d.pfr_dst), 32 * d.n_pfround);
    copy_words_s(sched + P.o_rslab, d.prslab, d.prslab_words);
    copy_words_s(sched + P.o_rround, reinterpret_cast<const uint32_t*>(d.prround), 4 * d.n_prround);
    copy_words_s(sched + P.o_rrval, reinterpret_cast<const uint32_t*>(d.prr_val), 32 * d.n_prround);
    copy_words_s(sched + P.o_seed, reinterpret_cast<const uint32_t*>(d.seed_f), d.n_vals);
    s_fslab = sched + P.o_fslab;
    s_fround = reinterpret_cast<const int4*>(sched + P.o_fround);
    s_frdst = reinterpret_cast<const int*>(sched + P.o_frdst);
    s_rslab = sched + P.o_rslab;
    s_rround = reinterpret_cast<const int4*>(sched + P.o_rround);
    s_rrval = reinterpret_cast<const int*>(sched + P.o_rrval);
    s_seed = reinterpret_cast<const float*>(sched + P.o_seed);
  }
  const int nwarps = blockDim.x >> 5;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // per warp: NB (values, adjoints) array pairs, each adjoint array NV after its values
  float* const wbase =
      reinterpret_cast<float*>(smem + P.c_bytes + (GSCH ? ring_bytes() : (TMS ? P.ovf_bytes : P.sched_bytes)) +
                               warp * P.warp_bytes);
  for (int k = lane; k < 2 * NB * NV; k += 32) wbase[k] = 0.f;   // the zero slot n_vals stays 0
  float* v[NB];
  float* g[NB];
#pragma unroll
  for (int j = 0; j < NB; ++j) {
    v[j] = wbase + 2 * j * NV;
    g[j] = v[j] + NV;
  }
  const int T = P.T;
  const int n_mom = d.n_mom;
  // this lane's moment slots (the same for every neighborhood) and their value indices
  int sc[PRE];
#pragma unroll
  for (int r = 0; r < PRE; ++r) {
    const int k = lane + 32 * r;
    sc[r] = k < n_mom ? P.slot_comp[k] : -1;
    if (sc[r] >= 0 && !OK(sc[r], NV, 21)) sc[r] = -1;
  }
  const int64_t stride = static_cast<int64_t>(gridDim.x) * nwarps * NB;
  // moments of the next neighborhoods, loaded one iteration ahead (their global latency overlaps
  // the contraction of the current ones)
  float pre[NB][PRE];
  auto fetch = [&](int64_t w0) {
#pragma unroll
    for (int j = 0; j < NB; ++j) {
      const bool live = w0 + j < P.n_work;
      const float* src = P.mom + (w0 + j) * P.ldm;
#pragma unroll
      for (int r = 0; r < PRE; ++r) {
        const int k = lane + 32 * r;
        pre[j][r] = (live && sc[r] >= 0 && OK((w0 + j) * P.ldm + k, P.n_work * P.ldm, 22)) ? __ldcs(src + k) : 0.f;
      }
    }
  };
  // the block's first neighborhood: with GSCH the loop runs while the block has any work left
  const int64_t bfirst = static_cast<int64_t>(blockIdx.x) * nwarps * NB;
  int64_t w0 = bfirst + static_cast<int64_t>(warp) * NB;
  if (w0 < P.n_work) fetch(w0);
  __syncthreads();
  long long vbase = 0;   // GSCH: the stream row of this iteration's first row
  if constexpr (GSCH) {
#pragma unroll
    for (int c = 0; c < kRing - 1; ++c) issue_chunk(S, c);
  }
  for (int64_t b0 = bfirst; GSCH ? b0 < P.n_work : w0 < P.n_work; b0 += stride, w0 += stride, vbase += S.TRp) {
    int64_t wk[NB];
    bool live[NB];
#pragma unroll
    for (int j = 0; j < NB; ++j) {
      wk[j] = w0 + j;
      live[j] = wk[j] < P.n_work;
#pragma unroll
      for (int r = 0; r < PRE; ++r)
        if (sc[r] >= 0) v[j][sc[r]] = live[j] ? pre[j][r] : 0.f;
    }
    if (w0 + stride < P.n_work) fetch(w0 + stride);
    __syncwarp();
    // ---------------- forward contraction (eqs. 5-6) ----------------
    int4 rd_n = d.n_pfround > 0 ? s_fround[0] : make_int4(0, 0, 0, 0);
    int dst_n = d.n_pfround > 0 ? s_frdst[lane] : -1;
    for (int r = 0; r < d.n_pfround; ++r) {
      int4 rd = rd_n;
      const int ent = dst_n;
      if (r + 1 < d.n_pfround) {
        rd_n = s_fround[r + 1];
        dst_n = s_frdst[32 * (r + 1) + lane];
      }
      if (!OK(rd.y + 32 * (rd.x > 0 ? rd.x - 1 : 0) + 31, d.pfslab_words, 23)) rd.x = 0;
      float acc[NB];
#pragma unroll
      for (int j = 0; j < NB; ++j) acc[j] = 0.f;
      if constexpr (GSCH) slab_round_stream<NB, INL, UNR>(S, vbase + (rd.y >> 5), rd.x, lane, coef, v, v, acc);
      else if constexpr (TMS) slab_round_tmem<NB, INL, UNR>(tq, ovf, rd.y >> 5, rd.x, coef, v, v, acc);
      else slab_round<NB, INL, UNR>(s_fslab + rd.y + lane, rd.x, coef, v, v, acc);
      if (rd.w) group_combine<NB>(acc, ent);
      const int dst = ent & 0xffff;
      if (ent >= 0 && ((ent >> 20) & 1) && OK(dst, NV, 26)) {
#pragma unroll
        for (int j = 0; j < NB; ++j) v[j][dst] = acc[j];
      }
      if (rd.z) __syncwarp();
    }
    // ---------------- site energy (eq. 2) ----------------
#pragma unroll
    for (int j = 0; j < NB; ++j) {
      if (!live[j]) continue;
      const int64_t i = atom_of(P, wk[j]);
      if (P.o.V) {
        float acc = 0.f;
        for (int a = lane; a < d.n_lin; a += 32)
          if (OK(d.basis_idx[a], NV, 27)) acc = fmaf(d.theta_f[T + a], v[j][d.basis_idx[a]], acc);
        for (int m = 16; m; m >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, m);
        if (lane == 0) P.o.V[i] = static_cast<double>(acc) + d.theta_d[P.type[i]];
      }
    }
    // ---------------- adjoint of the contraction (gather form), seeded with xi ----------------
    rd_n = d.n_prround > 0 ? s_rround[0] : make_int4(0, 0, 0, 0);
    int x_n = d.n_prround > 0 ? s_rrval[lane] : -1;
    int x_nn = d.n_prround > 1 ? s_rrval[32 + lane] : -1;
    for (int r = 0; r < d.n_prround; ++r) {
      int4 rd = rd_n;
      const int ent = x_n;
      if (r + 1 < d.n_prround) {
        rd_n = s_rround[r + 1];
        x_n = x_nn;
      }
      if (r + 2 < d.n_prround) x_nn = s_rrval[32 * (r + 2) + lane];
      const int x = ent & 0xffff;
      const bool lead = ent >= 0 && ((ent >> 20) & 1);
      const float sd = (lead && OK(x, d.n_vals, 28)) ? s_seed[x] : 0.f;
      if (!OK(rd.y + 32 * (rd.x > 0 ? rd.x - 1 : 0) + 31, d.prslab_words, 29)) rd.x = 0;
      float acc[NB];
#pragma unroll
      for (int j = 0; j < NB; ++j) acc[j] = sd;
      if constexpr (GSCH) slab_round_stream<NB, INL, UNR>(S, vbase + S.FR + (rd.y >> 5), rd.x, lane, coef, v, g, acc);
      else if constexpr (TMS) slab_round_tmem<NB, INL, UNR>(tq, ovf, S.FR + (rd.y >> 5), rd.x, coef, v, g, acc);
      else slab_round<NB, INL, UNR>(s_rslab + rd.y + lane, rd.x, coef, v, g, acc);
      if (rd.w) group_combine<NB>(acc, ent);
      if (lead && OK(x, NV, 32)) {
#pragma unroll
        for (int j = 0; j < NB; ++j) g[j][x] = acc[j];
      }
      if (rd.z) __syncwarp();
    }
    __syncwarp();
    // ---------------- outputs: dV/dM over the moments, the basis part of b_i ----------------
#pragma unroll
    for (int j = 0; j < NB; ++j) {
      if (!live[j]) continue;
      float* dst = P.mom + wk[j] * P.ldm;
#pragma unroll
      for (int r = 0; r < PRE; ++r)
        if (sc[r] >= 0 && OK(wk[j] * P.ldm + lane + 32 * r, P.n_work * P.ldm, 34)) __stcs(dst + lane + 32 * r, g[j][sc[r]]);
      const int64_t i = atom_of(P, wk[j]);
      const int64_t rw = P.o.row_pos ? P.o.row_pos[i] : wk[j];
      if (P.o.rows_hi) {
        const int zi = P.type[i];
        float* hi = P.o.rows_hi + rw * P.o.rows_ld;
        float* lo = P.o.rows_lo ? P.o.rows_lo + rw * P.o.rows_ld : nullptr;
        for (int k = lane; k < T + d.n_lin; k += 32) {
          if (!OK(rw * P.o.rows_ld + k, P.nb.n_atoms * P.o.rows_ld, 35)) continue;
          if (k >= T && !OK(d.basis_idx[k - T], NV, 36)) continue;
          const float val = k < T ? (k == zi ? 1.f : 0.f) : v[j][d.basis_idx[k - T]];
          if (lo) {
            const float h = tf32_rn(val);
            __stcs(hi + k, h);
            __stcs(lo + k, tf32_rn(val - h));
          } else {
            __stcs(hi + k, val);
          }
        }
      }
    }
    __syncwarp();
  }
  if constexpr (GSCH) cp_async_wait<0>();   // the chunks copied ahead of the last rows
  if constexpr (TMS) {   // every warp is past its last tensor-memory read
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_slot), "r"(512));
    }
  }
}

// ------------------------------------------------------------------------------------
// pair adjoint: per-pair gradients, the neighborhood's virial, the radial block of b_i
// ------------------------------------------------------------------------------------
template <int NR, int NU0, bool ROWS>
__global__ void __launch_bounds__(256) k_adjoint(SplitArgs P) {
  using Sh = Shape<NR, NU0>;
  constexpr int NQ = kNQs;
  static_assert(NR + NQ + 1 <= GS, "radial-block staging");
  extern __shared__ __align__(16) unsigned char smem[];
  const DevSchedule& d = P.d;
  const int T = P.T;
  float* ctab = reinterpret_cast<float*>(smem);
  for (int k = threadIdx.x; k < P.NC; k += blockDim.x) ctab[k] = d.theta_f[T + d.n_lin + k];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, grp = lane / LPN, q = lane % LPN;
  const int nwarps = blockDim.x >> 5;
  const int gstride = adj_region(P.ldm, ROWS);
  float* gM = reinterpret_cast<float*>(smem + P.c_bytes) + (static_cast<size_t>(warp) * GPW + grp) * gstride;
  float* rstg = gM + ((P.ldm + 31) & ~31) + 8;
  __syncthreads();
  const float rmin = static_cast<float>(d.r_min), rcut = static_cast<float>(d.r_cut);
  for (int64_t w0 = (static_cast<int64_t>(blockIdx.x) * nwarps + warp) * GPW; w0 < P.n_work;
       w0 += static_cast<int64_t>(gridDim.x) * nwarps * GPW) {
    const int64_t wk = w0 + grp;
    const bool live = wk < P.n_work;
    int np = 0, zi = 0;
    int64_t p0 = 0, i = 0;
    if (live && OK(wk, P.nb.n_atoms, 40)) {
      i = atom_of(P, wk);
      zi = P.type[i];
      p0 = P.nb.off[i];
      np = static_cast<int>(P.nb.off[i + 1] - p0);
      if (!OK(zi, T, 41) || !OK(p0 + np - 1 + (np == 0), P.nb.n_pairs + 1, 42)) { zi = 0; np = 0; }
    }
    int np_max = np;
    for (int m = 16; m; m >>= 1) np_max = max(np_max, __shfl_xor_sync(0xffffffffu, np_max, m));
    __syncwarp();
    if (live) {
      const float* src = P.mom + wk * P.ldm;
      for (int k = q; k < Sh::NCOMP; k += LPN)
        if (OK(P.slot_comp[k], P.ldm, 43) && OK(wk * P.ldm + k, P.n_work * P.ldm, 44)) gM[P.slot_comp[k]] = __ldcs(src + k);
    }
    __syncwarp();
    const float* czi = ctab + static_cast<size_t>(zi) * T * NR * NQ;
    float Wl[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) Wl[k] = 0.f;
    // radial block accumulators: lane q owns beta = q for every (species, mu)
    constexpr int TM = tmax_of(NR);
    float cb[TM][NR];
#pragma unroll
    for (int z = 0; z < TM; ++z)
#pragma unroll
      for (int mu = 0; mu < NR; ++mu) cb[z][mu] = 0.f;
    float* Gout = static_cast<float*>(P.o.G);
    for (int base = 0; base < np_max; base += BATCH_A) {
      const int nbt = min(BATCH_A, np - base);
      // every lane of the warp runs the same number of iterations (adjoint_pass has warp-wide
      // __syncwarp fences); lanes without a pair of their own work on a dummy one
      const int nbt_w = min(BATCH_A, np_max - base);
      for (int t0 = 0; t0 < nbt_w; t0 += LPN) {
        const int t = t0 + q;
        const int64_t p = p0 + base + t;
        bool act = t < nbt;
        if (act && (!OK(p, P.nb.n_pairs, 45) || (ROWS && !OK(t * GS + GS - 1, BATCH_A * GS, 46)))) act = false;
        float4 r = make_float4(1.f, 0.f, 0.f, 1.f);
        int zj = 0;
        if (act) {
          r = P.nb.pr32[p];
          const int jj = P.nb.pj[p];
          if (OK(jj, P.nb.n_atoms, 47)) zj = P.type[jj];
          if (!OK(zj, T, 48)) zj = 0;
        }
        float f[NR], df[NR], g[NR];
        radial<NR, NQ>(r.w, czi + zj * NR * NQ, rmin, rcut, f, df, (ROWS && act) ? rstg + t * GS + NR : nullptr);
#pragma unroll
        for (int mu = 0; mu < NR; ++mu) g[mu] = 0.f;
        float gx = 0.f, gy = 0.f, gz = 0.f;
        adjoint_pass<NR, NU0>(r.x, r.y, r.z, f, gM, g, gx, gy, gz);
        if (!act) continue;
        float rad = 0.f;
#pragma unroll
        for (int mu = 0; mu < NR; ++mu) rad = fmaf(g[mu], df[mu], rad);
        const float sc = rad / r.w;
        gx = fmaf(sc, r.x, gx);
        gy = fmaf(sc, r.y, gy);
        gz = fmaf(sc, r.z, gz);
        if (Gout && OK(3 * p + 2, 3 * P.nb.n_pairs, 53)) {
          __stcs(Gout + 3 * p + 0, gx);
          __stcs(Gout + 3 * p + 1, gy);
          __stcs(Gout + 3 * p + 2, gz);
        }
        const float g3[3] = {gx, gy, gz}, r3[3] = {r.x, r.y, r.z};
#pragma unroll
        for (int a2 = 0; a2 < 3; ++a2)
#pragma unroll
          for (int b2 = 0; b2 < 3; ++b2) Wl[3 * a2 + b2] = fmaf(-g3[a2], r3[b2], Wl[3 * a2 + b2]);
        if (ROWS) {
          float* e = rstg + t * GS;
#pragma unroll
          for (int mu = 0; mu < NR; ++mu) e[mu] = g[mu];
          e[NR + NQ] = __int_as_float(zj);
        }
      }
      if (ROWS) {
        __syncwarp();
        // sum_j g_mu(j) Q_b(r_ij) per neighbor species: lane q takes b = q over the staged pairs
        for (int t = 0; t < nbt; ++t) {
          if (!OK(t * GS + GS - 1, BATCH_A * GS, 49)) continue;
          const float* e = rstg + t * GS;
          const float qb = e[NR + q];
          const int zj = __float_as_int(e[NR + NQ]);
#pragma unroll
          for (int mu = 0; mu < NR; ++mu) {
            const float pr = e[mu] * qb;
#pragma unroll
            for (int z = 0; z < TM; ++z) cb[z][mu] += (zj == z) ? pr : 0.f;
          }
        }
        __syncwarp();
      }
    }
    // the neighborhood's virial (FP32 over its pairs, like its forces; sums over atoms are FP64)
#pragma unroll
    for (int k = 0; k < 9; ++k) Wl[k] = group_sum(Wl[k]);
    if (live && P.o.Wat && q == 0 && OK(9 * i + 8, 9 * P.nb.n_atoms, 50)) {
#pragma unroll
      for (int k = 0; k < 9; ++k) P.o.Wat[9 * i + k] = static_cast<double>(Wl[k]);
    }
    if (ROWS && live && P.o.rows_hi) {
      const int64_t rw = P.o.row_pos ? P.o.row_pos[i] : wk;
      const int64_t ld = P.o.rows_ld;
      const int off_c = T + d.n_lin;
      float* hi = P.o.rows_hi + rw * ld;
      float* lo = P.o.rows_lo ? P.o.rows_lo + rw * ld : nullptr;
      auto put = [&](int64_t k, float val) {
        if (!OK(rw * ld + k, P.nb.n_atoms * ld, 51) || !OK(k, ld, 52)) return;
        if (lo) {
          const float h = tf32_rn(val);
          __stcs(hi + k, h);
          __stcs(lo + k, tf32_rn(val - h));
        } else {
          __stcs(hi + k, val);
        }
      };
      // block zi holds the sums; the other species' blocks and the padding past m are zero
      for (int k = off_c + q; k < ld; k += LPN) {
        const int e = k - off_c;
        if (e / P.CBN != zi || k >= d.n_params) put(k, 0.f);
      }
#pragma unroll
      for (int z = 0; z < TM; ++z) {
        if (z < T) {
#pragma unroll
          for (int mu = 0; mu < NR; ++mu) put(off_c + static_cast<int64_t>(zi) * P.CBN + (z * NR + mu) * NQ + q, cb[z][mu]);
        }
      }
    }
    __syncwarp();
  }
}

template <class K>
int blocks_per_sm(K kern, int threads, size_t smem) {
  int per = 0;
  MTP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, threads, smem));
  return std::max(per, 1);
}

int num_sms() {
  int dev = 0, nsm = 0;
  MTP_CUDA(cudaGetDevice(&dev));
  MTP_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  return nsm;
}

template <int NR, int NU0>
void launch_split(SplitArgs P, int warps_pair, int nb_contract, int unroll, int sch, bool efs, bool rows,
                  cudaStream_t s) {
  const int nsm = num_sms();
  const int64_t groups = (P.n_work + GPW - 1) / GPW;
  // ---- moments ----
  {
    const size_t smem = P.c_bytes + static_cast<size_t>(warps_pair) * GPW * stage_f4(NR) * BATCH * sizeof(float4);
    auto kern = k_moments<NR, NU0>;
    MTP_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)));
    const int per = blocks_per_sm(kern, warps_pair * 32, smem);
    const int grid = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>((groups + warps_pair - 1) / warps_pair,
                                                                              static_cast<int64_t>(nsm) * per)));
    ProfRegion pr("site_moments", s);
    kern<<<grid, warps_pair * 32, smem, s>>>(P);
    ProfRegion::launched();
    MTP_CUDA(cudaGetLastError());
  }
  // ---- contraction ----
  {
    const size_t sched = sch == 2 ? ring_bytes() : (sch == 3 ? P.ovf_bytes : P.sched_bytes);
    const int wpb = std::max(1, static_cast<int>((227 * 1024 - P.c_bytes - sched) / P.warp_bytes));
    // the streamed variant is built for <= 256 threads, the tensor-memory one for <= 384
    const int warps = std::min(wpb, sch == 2 ? 8 : (sch == 3 ? 12 : 16));
    const bool inl = P.d.coef_inline;
    auto launch = [&](auto kern) {
      size_t sm = P.c_bytes + sched + static_cast<size_t>(warps) * P.warp_bytes;
      // a block that holds all 512 tensor-memory columns: more than half the shared memory, so
      // that no second block shares its SM (it would wait for the columns)
      if (sch == 3) sm = std::max<size_t>(sm, 120 * 1024);
      MTP_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sm)));
      const int per = blocks_per_sm(kern, warps * 32, sm);
      const int64_t need = (P.n_work + nb_contract - 1) / nb_contract;
      const int grid = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>((need + warps - 1) / warps,
                                                                                static_cast<int64_t>(nsm) * per)));
      ProfRegion pr("site_contract", s);
      kern<<<grid, warps * 32, sm, s>>>(P);
      ProfRegion::launched();
      MTP_CUDA(cudaGetLastError());
    };
    constexpr int PRE = pre_of(NR);
    // the level-24 shape (6, 10) only has the streamed, 12-bit-index variant (its 3,853 values
    // need 12-bit indices, its schedule fits neither shared nor tensor memory; the caller checks)
    auto pick = [&](auto nbc, auto unr) {
      constexpr int NBc = decltype(nbc)::value, U = decltype(unr)::value;
      if constexpr (NR >= 6) {
        launch(k_contract<NBc, false, U, PRE, 1>);
      } else if (sch == 2) {
        if (inl) launch(k_contract<NBc, true, U, PRE, 1>);
        else launch(k_contract<NBc, false, U, PRE, 1>);
      } else if (sch == 3) {
        if (inl) launch(k_contract<NBc, true, U, PRE, 2>);
        else launch(k_contract<NBc, false, U, PRE, 2>);
      } else {
        if (inl) launch(k_contract<NBc, true, U, PRE, 0>);
        else launch(k_contract<NBc, false, U, PRE, 0>);
      }
    };
    if (nb_contract == 2) {
      if (unroll == 8 && NR < 6) pick(std::integral_constant<int, 2>{}, std::integral_constant<int, 8>{});
      else if (unroll == 4) pick(std::integral_constant<int, 2>{}, std::integral_constant<int, 4>{});
      else pick(std::integral_constant<int, 2>{}, std::integral_constant<int, 2>{});
    } else {
      if (unroll == 4) pick(std::integral_constant<int, 1>{}, std::integral_constant<int, 4>{});
      else pick(std::integral_constant<int, 1>{}, std::integral_constant<int, 2>{});
    }
  }
  // ---- pair adjoint ----
  if (efs || rows) {
    const size_t gstride = static_cast<size_t>(adj_region(P.ldm, rows));
    const size_t smem = P.c_bytes + static_cast<size_t>(warps_pair) * GPW * gstride * sizeof(float);
    auto go = [&](auto kern) {
      MTP_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)));
      const int per = blocks_per_sm(kern, warps_pair * 32, smem);
      const int grid = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>((groups + warps_pair - 1) / warps_pair,
                                                                                static_cast<int64_t>(nsm) * per)));
      ProfRegion pr("site_adjoint", s);
      kern<<<grid, warps_pair * 32, smem, s>>>(P);
      ProfRegion::launched();
      MTP_CUDA(cudaGetLastError());
    };
    if (rows) go(k_adjoint<NR, NU0, true>);
    else go(k_adjoint<NR, NU0, false>);
  }
}

template <int NR, int NU0>
std::vector<int> slot_table() {
  using Sh = Shape<NR, NU0>;
  constexpr auto S = make_slots<NR, NU0>();
  return std::vector<int>(S.comp, S.comp + Sh::NCOMP);
}

}  // namespace

// Uploads the slot -> component table of the model's shape (at load time, so that the split
// pass allocates nothing when it runs); leaves it empty for shapes without a split kernel.
void split_prepare(mtp_model* m) {
  const DevSchedule& d = m->ds;
  std::vector<int> t;
  if (d.n_q == kNQs) {
    if (d.n_rad == 2 && d.nu_max == 2) t = slot_table<2, 2>();
    else if (d.n_rad == 3 && d.nu_max == 4) t = slot_table<3, 4>();
    else if (d.n_rad == 4 && d.nu_max == 6) t = slot_table<4, 6>();
    else if (d.n_rad == 5 && d.nu_max == 8) t = slot_table<5, 8>();
    else if (d.n_rad == 6 && d.nu_max == 10) t = slot_table<6, 10>();
  }
  if (t.empty() || static_cast<int>(t.size()) != d.n_mom) return;
  m->split_tab.ensure(t.size() * sizeof(int), 0);
  MTP_CUDA(cudaMemcpy(m->split_tab.p, t.data(), t.size() * sizeof(int), cudaMemcpyHostToDevice));
}

// The three-kernel mixed pass.  Returns false (nothing launched) when the model's shape has no
// specialised instantiation, when the outputs are not the step's (FP64 rows, an explicit atom
// list), or when no moment workspace was given; the caller then uses another kernel.
bool run_sites_split(mtp_model* m, const mtp_batch* b, const mtp_nbr* nb, const SiteOutputs& o, cudaStream_t s) {
  const DevSchedule& d = m->ds;
  float* mom_ws = o.mom;
  if (!mom_ws || !split_wanted(m) || !d.tri_pk || d.n_q != kNQs || d.n_types > tmax_of(d.n_rad)) return false;
  if (o.rows || o.atom_list) return false;
  const bool efs = o.V != nullptr;
  const bool rows = o.rows_hi != nullptr;
  if (!efs && !rows) return false;
  if (efs && (!o.G || !o.Wat)) return false;
  const int nr = d.n_rad, nu0 = d.nu_max;
  const bool shape_ok = (nr == 2 && nu0 == 2) || (nr == 3 && nu0 == 4) || (nr == 4 && nu0 == 6) ||
                        (nr == 5 && nu0 == 8) || (nr == 6 && nu0 == 10);
  if (!shape_ok || d.n_mom > 32 * pre_of(nr)) return false;
  SplitArgs P{};
  P.d = d;
  P.nb = nb->dn;
  P.type = b->type;
  P.n_work = nb->n_atoms;
  P.o = o;
  P.mom = mom_ws;
  P.ldm = split_ldm(d.n_mom);
  P.slot_comp = m->split_tab.as<int>();
  P.T = d.n_types;
  P.CBN = d.n_types * d.n_rad * d.n_q;
  P.NC = d.n_types * P.CBN;
  P.NV = padded_nv(d.n_vals);
  P.c_bytes = (static_cast<size_t>(std::max(P.NC, d.n_coef)) * sizeof(float) + 15) & ~size_t(15);
  int w = 0;
  auto take = [&](int n) { const int o2 = w; w += (n + 3) & ~3; return o2; };
  P.o_fslab = take(d.pfslab_words);
  P.o_fround = take(4 * d.n_pfround);
  P.o_frdst = take(32 * d.n_pfround);
  P.o_rslab = take(d.prslab_words);
  P.o_rround = take(4 * d.n_prround);
  P.o_rrval = take(32 * d.n_prround);
  P.o_seed = take(d.n_vals);
  P.sched_bytes = static_cast<size_t>(w) * 4;
  const int nbc = m->tune_split_nb > 0 ? m->tune_split_nb : 1;
  P.warp_bytes = static_cast<size_t>(2 * nbc * P.NV) * sizeof(float);
  // the schedule in shared memory when it fits beside at least four warps' value arrays (unless
  // global memory is asked for), else read from global memory (level 24: 0.4 MB of slab words)
  // where the contraction reads its schedule: 1 shared memory (when it fits beside at least four
  // warps' value arrays), 2 streamed through a shared ring (level 24: 0.35 MB of slab words),
  // 3 tensor memory (the first 512 rows; the rest in shared memory), as asked or automatic
  const int rows_total = (d.pfslab_words + d.prslab_words) / 32;
  P.ovf_bytes = static_cast<size_t>(std::max(0, rows_total - kTmemRows)) * 128;
  P.ovf_bytes += static_cast<size_t>(((4 * d.n_pfround + 3) & ~3) + 32 * d.n_pfround + ((4 * d.n_prround + 3) & ~3) +
                                     32 * d.n_prround + ((d.n_vals + 3) & ~3)) * 4;   // headers, lane entries, seeds
  const bool fits = P.c_bytes + P.sched_bytes + 4 * P.warp_bytes <= 227 * 1024;
  const int ask = m->tune_split_sched;
  int sch = fits ? 1 : 2;
  if (ask == 2) sch = 2;
  if (ask == 3 && nr < 6 && P.c_bytes + P.ovf_bytes + 4 * P.warp_bytes <= 227 * 1024) sch = 3;
  if ((nr >= 6 && sch != 2) || (nr >= 6 && d.coef_inline)) return false;
  if (sch != 1 && (d.pfslab_words % 32 != 0 || d.prslab_words % 32 != 0)) return false;   // whole rows
  const size_t sbytes = sch == 2 ? ring_bytes() : (sch == 3 ? P.ovf_bytes : P.sched_bytes);
  if (P.c_bytes + sbytes + P.warp_bytes > 227 * 1024) return false;
  P.total = P.c_bytes + sbytes + P.warp_bytes;
  const int wp = m->tune_split_warps > 0 ? m->tune_split_warps : 8;
  m->last_fast = true;
  m->last_split = true;
  m->last_split_sched = sch;
  m->last_warps = wp;
  if (P.n_work == 0) return true;
  const int unr = m->tune_split_unroll == 4 ? 4 : (m->tune_split_unroll == 8 && nbc == 2 ? 8 : 2);
  if (nr == 2) launch_split<2, 2>(P, wp, nbc, unr, sch, efs, rows, s);
  else if (nr == 3) launch_split<3, 4>(P, wp, nbc, unr, sch, efs, rows, s);
  else if (nr == 4) launch_split<4, 6>(P, wp, nbc, unr, sch, efs, rows, s);
  else if (nr == 5) launch_split<5, 8>(P, wp, nbc, unr, sch, efs, rows, s);
  else launch_split<6, 10>(P, wp, nbc, unr, sch, efs, rows, s);
#ifdef MTP_SPLIT_CHECK
  unsigned long long fault = 0;
  MTP_CUDA(cudaStreamSynchronize(s));
  MTP_CUDA(cudaMemcpyFromSymbol(&fault, g_split_fault, sizeof(fault)));
  if (fault) {
    const unsigned long long zero = 0;
    MTP_CUDA(cudaMemcpyToSymbol(g_split_fault, &zero, sizeof(zero)));
    throw Fail{MTP_ERR_NUMERIC, "split pass: index out of range, check " + std::to_string(fault >> 48) + " index " +
                                    std::to_string(static_cast<long long>(fault & 0xFFFFFFFFFFFFull))};
  }
#endif
  return true;
}

}  // namespace mtp

// Neighbor build (Section II.A: the neighborhood n_i of atom i is every (j, image) with
// 0 < |r_ij| < R_cut).  Cell list over fractional coordinates of every configuration:
//   1. wrap periodic fractional coordinates into [0,1), bin atoms (bins of height >= R_cut),
//      count / scan / scatter, then sort each bin by atom index (deterministic order);
//   2. per atom, visit the bins within +-ceil(R_cut nb / h) along each axis (periodic axes
//      wrap and carry an image shift); count accepted pairs, scan to CSR, fill;
//   3. reverse-pair index: pair (i -> j, n) is matched with (j -> i, -n).  The decision is
//      symmetric (below) and the bin scan order point-symmetric, so when the count pass records,
//      per atom and scanned bin, the accepted slots and the pairs before that bin, the fill pass
//      computes each pair's reverse index directly; a search of j's list is the fallback (atoms
//      past slot 31 of their bin, or cells that scan more than 32 bins).
// Pair vectors are formed in double-single arithmetic (error-free TwoSum of the FP32 halves of
// the wrapped positions and of the image shift), so the FP32 copy is the correctly rounded
// r_ij without any FP64 arithmetic on the hot path; the rare pairs within a relative 4e-6 of
// the cut-off are decided by an FP64 recomputation of r_ij = (x_j + n.H) - x_i, always formed
// from the same end of the pair (the lower atom index, or the image with a positive leading
// component), so (i -> j, n) and (j -> i, -n) get bitwise the same |r|^2 and the same decision.
#include <cub/cub.cuh>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "mtp_internal.h"
#include "profiler.h"

namespace mtp {
namespace {

struct DevCfg {
  double H[9];
  double Hinv[9];
  int nb[3], kb[3], pbc[3];
  int K;
  long long bin_base, shift_base;
  float rc2f, rcm2f;
  double rc2;
  int qd[32];   // scanned bin q -> packed offsets (d0 + 64) | (d1 + 64) << 8 | (d2 + 64) << 16
};

struct NbrArgs {
  int64_t n_atoms;
  int n_cfg;
  const int64_t* atom_offset;
  const double* pos;
  const int* type;
  int n_types;
  const DevCfg* cfg;
  const float4* sh_hi;   // shift table (double-single halves)
  const float4* sh_lo;
  int* atom_cfg;
  int* wrap;             // packed integer wrap of each atom
  long long* atom_bin;   // global bin of each atom
  int* bcoord;           // the atom's bin coordinates within its configuration, 10 bits each
  float4* ph;            // wrapped position hi (.w = atom index bits)
  float4* pl;            // wrapped position lo (.w = packed wrap of the atom)
  int* bin_count;
  int* bin_fill;
  long long* bin_start;  // [n_bins + 1]
  int* bin_atoms;
  float4* bph;           // binned copies
  float4* bpl;
  long long* cnt;        // per atom neighbor count [n_atoms + 1]
  const long long* off;
  int* pj;
  int* pimg;
  float4* pr32;
  int* prev;
  uint2* rv;             // [scanned bin q x n_atoms], by bin-order position t: .x = accepted bits of
                         // the bin's first 32 slots, .y = the atom's pairs before bin q (count
                         // pass writes, fill reads); null when a configuration scans > 32 bins
  uint32_t* mask;        // [kMaskWords x n_atoms] accepted bits of the first kMaskBits candidates
                         // in scan order, by bin-order position (count pass writes, fill reads)
  unsigned* err;
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__global__ void k_prep(NbrArgs A) {
  int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i >= A.n_atoms) return;
  // configuration of atom i (binary search over atom_offset)
  int lo = 0, hi = A.n_cfg - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (A.atom_offset[mid] <= i) lo = mid; else hi = mid - 1;
  }
  const int k = lo;
  A.atom_cfg[i] = k;
  const DevCfg& C = A.cfg[k];
  const int t = A.type[i];
  if (t < 0 || t >= A.n_types) atomicOr(A.err, ERRF_SPECIES);
  double x[3] = {A.pos[3 * i], A.pos[3 * i + 1], A.pos[3 * i + 2]};
  if (!isfinite(x[0]) || !isfinite(x[1]) || !isfinite(x[2])) {
    atomicOr(A.err, ERRF_NONFINITE);
    x[0] = x[1] = x[2] = 0.0;
  }
  int w[3];
  int b[3];
  for (int a = 0; a < 3; ++a) {
    double s = x[0] * C.Hinv[0 * 3 + a] + x[1] * C.Hinv[1 * 3 + a] + x[2] * C.Hinv[2 * 3 + a];
    w[a] = 0;
    if (C.pbc[a]) {
      double f = floor(s);
      s -= f;
      w[a] = static_cast<int>(f);
      if (s >= 1.0) { s -= 1.0; w[a] += 1; }
    }
    int bi = static_cast<int>(floor(s * C.nb[a]));
    b[a] = min(max(bi, 0), C.nb[a] - 1);
  }
  const int wpk = pack_img(w[0], w[1], w[2]);
  A.wrap[i] = wpk;
  double xw[3];
  for (int c = 0; c < 3; ++c) xw[c] = x[c] - (w[0] * C.H[0 * 3 + c] + w[1] * C.H[1 * 3 + c] + w[2] * C.H[2 * 3 + c]);
  float h[3], l[3];
  for (int c = 0; c < 3; ++c) { h[c] = __double2float_rn(xw[c]); l[c] = __double2float_rn(xw[c] - static_cast<double>(h[c])); }
  A.ph[i] = make_float4(h[0], h[1], h[2], __int_as_float(static_cast<int>(i)));

  A.pl[i] = make_float4(l[0], l[1], l[2], __int_as_float(wpk));   // .w: the packed wrap
  long long bin = C.bin_base + (static_cast<long long>(b[0]) * C.nb[1] + b[1]) * C.nb[2] + b[2];
  A.atom_bin[i] = bin;
  A.bcoord[i] = b[0] | (b[1] << 10) | (b[2] << 20);
  atomicAdd(&A.bin_count[bin], 1);
}

__global__ void k_scatter(NbrArgs A) {
  int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i >= A.n_atoms) return;
  long long bin = A.atom_bin[i];
  int slot = atomicAdd(&A.bin_fill[bin], 1);
  A.bin_atoms[A.bin_start[bin] + slot] = static_cast<int>(i);
}

__global__ void k_sort_bins(NbrArgs A, long long n_bins) {
  long long bn = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
  if (bn >= n_bins) return;
  long long s0 = A.bin_start[bn], s1 = A.bin_start[bn + 1];
  for (long long a = s0 + 1; a < s1; ++a) {
    int v = A.bin_atoms[a];
    long long b = a - 1;
    while (b >= s0 && A.bin_atoms[b] > v) { A.bin_atoms[b + 1] = A.bin_atoms[b]; --b; }
    A.bin_atoms[b + 1] = v;
  }
  for (long long a = s0; a < s1; ++a) {
    int v = A.bin_atoms[a];
    A.bph[a] = A.ph[v];
    A.bpl[a] = A.pl[v];
  }
}

// Decide pair (i -> j, nrel) and form r_ij; returns 1 if accepted.
__device__ __forceinline__ int decide(const NbrArgs& A, const DevCfg& C, int64_t i, int j, const float4& xi_h,
                                      const float4& xi_l, const float4& xj_h, const float4& xj_l, int n0, int n1,
                                      int n2, float4& r_out, int& img_out) {
  const int K = C.K;
  const long long sidx = C.shift_base + ((static_cast<long long>(n0 + K) * (2 * K + 1) + (n1 + K)) * (2 * K + 1) + (n2 + K));
  const float4 sh = A.sh_hi[sidx];
  const float ax = (xj_h.x - xi_h.x) + sh.x, ay = (xj_h.y - xi_h.y) + sh.y, az = (xj_h.z - xi_h.z) + sh.z;
  if (ax * ax + ay * ay + az * az > C.rcm2f) return 0;
  const float4 sl = A.sh_lo[sidx];
  float r[3];
  const float xh[3] = {xj_h.x, xj_h.y, xj_h.z}, xih[3] = {xi_h.x, xi_h.y, xi_h.z};
  const float xl[3] = {xj_l.x, xj_l.y, xj_l.z}, xil[3] = {xi_l.x, xi_l.y, xi_l.z};
  const float shh[3] = {sh.x, sh.y, sh.z}, shl[3] = {sl.x, sl.y, sl.z};
  for (int c = 0; c < 3; ++c) {
    float s1, e1, s2, e2;
    two_sum(xh[c], -xih[c], s1, e1);
    two_sum(s1, shh[c], s2, e2);
    const float low = __fadd_rn(__fadd_rn(e1, e2), __fadd_rn(__fsub_rn(xl[c], xil[c]), shl[c]));
    r[c] = __fadd_rn(s2, low);
  }
  const float d2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
  const int wi = __float_as_int(xi_l.w), wj = __float_as_int(xj_l.w);   // packed wraps
  const int m0 = n0 - unpack_img(wj, 0) + unpack_img(wi, 0);
  const int m1 = n1 - unpack_img(wj, 1) + unpack_img(wi, 1);
  const int m2 = n2 - unpack_img(wj, 2) + unpack_img(wi, 2);
  bool accept;
  if (fabsf(d2 - C.rc2f) <= 4e-6f * C.rc2f || d2 < 1e-10f) {
    // formed from the canonical end: (x_b + s m.H) - x_a with (a, b, s) = (i, j, +1) or (j, i, -1);
    // (-m).H is the exact negation of m.H, so both ends give the same rounded |r|^2
    const bool flip = j < i || (j == i && (m0 < 0 || (m0 == 0 && (m1 < 0 || (m1 == 0 && m2 < 0)))));
    const long long ia = flip ? j : i, ib = flip ? i : j;
    const double sg = flip ? -1.0 : 1.0;
    double rr[3];
    for (int c = 0; c < 3; ++c) {
      const double sh64 = __dadd_rn(__dadd_rn(__dmul_rn(sg * m0, C.H[0 * 3 + c]), __dmul_rn(sg * m1, C.H[1 * 3 + c])),
                                    __dmul_rn(sg * m2, C.H[2 * 3 + c]));
      rr[c] = __dsub_rn(__dadd_rn(A.pos[3 * ib + c], sh64), A.pos[3 * ia + c]);
    }
    const double d64 = __dadd_rn(__dadd_rn(__dmul_rn(rr[0], rr[0]), __dmul_rn(rr[1], rr[1])), __dmul_rn(rr[2], rr[2]));
    if (d64 < 1e-16) { atomicOr(A.err, ERRF_GEOMETRY); return 0; }
    accept = d64 < C.rc2;
  } else {
    accept = d2 < C.rc2f;
  }
  if (!accept) return 0;
  r_out = make_float4(r[0], r[1], r[2], sqrtf(d2));
  img_out = pack_img(m0, m1, m2);
  return 1;
}

constexpr int kWarpScan = 32;    // the warp fill and the reverse record: at most 32 scanned bins
constexpr int kMaskWords = 16;   // accepted-candidate bits per atom recorded by the count pass
constexpr int kMaskBits = 32 * kMaskWords;

// (at most 64 registers, 8 CTAs of 128 threads per SM: with the per-bin reverse record the
// count pass measured 1.77 ms at 1M atoms against 1.91 ms at 48 registers / 10 CTAs and at
// 80 registers / 6 CTAs; a warp-per-atom count pass with ballots measured 2.86 ms)
#ifndef MTP_NB_MINB
#define MTP_NB_MINB 8
#endif
template <bool FILL>
__global__ void __launch_bounds__(128, MTP_NB_MINB) k_pairs(NbrArgs A) {
  // threads take the atoms in bin order, so that a warp's atoms scan the same or adjacent bins
  const int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (t >= A.n_atoms) return;
  const int64_t i = A.bin_atoms[t];
  const int k = A.atom_cfg[i];
  const DevCfg& C = A.cfg[k];
  const int bc = A.bcoord[i];
  const int b0 = bc & 1023, b1 = (bc >> 10) & 1023, b2 = (bc >> 20) & 1023;
  const float4 xi_h = A.ph[i], xi_l = A.pl[i];
  long long out = FILL ? A.off[i] : 0;
  const long long out_end = FILL ? A.off[i + 1] : 0;
  long long count = 0;
  int cand = 0;          // candidate index in scan order (the self candidate included)
  uint32_t mword = 0;    // count pass: accepted bits of the current mask word
  // bins are scanned in increasing q = ((d0 + kb0) w1 + (d1 + kb1)) w2 + (d2 + kb2)
  const int w1 = 2 * C.kb[1] + 1, w2 = 2 * C.kb[2] + 1;
  for (int d0 = -C.kb[0]; d0 <= C.kb[0]; ++d0) {
    int t0 = b0 + d0, n0 = 0;
    if (C.pbc[0]) {
      if (t0 < 0 || t0 >= C.nb[0]) { n0 = (t0 >= 0) ? t0 / C.nb[0] : -((-t0 + C.nb[0] - 1) / C.nb[0]); t0 -= n0 * C.nb[0]; }
    } else if (t0 < 0 || t0 >= C.nb[0]) {
      continue;
    }
    for (int d1 = -C.kb[1]; d1 <= C.kb[1]; ++d1) {
      int t1 = b1 + d1, n1 = 0;
      if (C.pbc[1]) {
        if (t1 < 0 || t1 >= C.nb[1]) { n1 = (t1 >= 0) ? t1 / C.nb[1] : -((-t1 + C.nb[1] - 1) / C.nb[1]); t1 -= n1 * C.nb[1]; }
      } else if (t1 < 0 || t1 >= C.nb[1]) {
        continue;
      }
      for (int d2 = -C.kb[2]; d2 <= C.kb[2]; ++d2) {
        int t2 = b2 + d2, n2 = 0;
        if (C.pbc[2]) {
          if (t2 < 0 || t2 >= C.nb[2]) { n2 = (t2 >= 0) ? t2 / C.nb[2] : -((-t2 + C.nb[2] - 1) / C.nb[2]); t2 -= n2 * C.nb[2]; }
        } else if (t2 < 0 || t2 >= C.nb[2]) {
          continue;
        }
        const int q = ((d0 + C.kb[0]) * w1 + (d1 + C.kb[1])) * w2 + (d2 + C.kb[2]);
        const long long tb = C.bin_base + (static_cast<long long>(t0) * C.nb[1] + t1) * C.nb[2] + t2;
        const long long s0 = A.bin_start[tb], s1 = A.bin_start[tb + 1];
        // candidate s of this bin: 1 if (i -> j, n) is a pair (written out in the fill pass)
        auto test = [&](long long s) -> int {
          const float4 xj_h = A.bph[s];
          const int j = __float_as_int(xj_h.w);
          if (j == static_cast<int>(i) && n0 == 0 && n1 == 0 && n2 == 0) return 0;
          float4 r;
          int img;
          if (!decide(A, C, i, j, xi_h, xi_l, xj_h, A.bpl[s], n0, n1, n2, r, img)) return 0;
          if (FILL && out < out_end) {
            A.pj[out] = j;
            A.pimg[out] = img;
            A.pr32[out] = r;
            ++out;
          }
          ++count;
          return 1;
        };
        long long s = s0;
        if (FILL && A.mask) {
          // replay the count pass's decisions: only its accepted candidates are formed again
          while (s < s1 && cand < kMaskBits) {
            const int wb = cand & 31;
            const int span = static_cast<int>(min(static_cast<long long>(32 - wb), s1 - s));
            uint32_t word = A.mask[static_cast<long long>(cand >> 5) * A.n_atoms + t] >> wb;
            if (span < 32) word &= (1u << span) - 1u;
            while (word) {
              const int b = __ffs(word) - 1;
              word &= word - 1u;
              test(s + b);
            }
            s += span;
            cand += span;
          }
        }
        const unsigned before = static_cast<unsigned>(count);
        uint32_t slots = 0;   // count pass: accepted bits of this bin's first 32 slots
        for (; s < s1; ++s, ++cand) {
          const int acc = test(s);
          if (!FILL && A.mask && cand < kMaskBits) {
            mword |= static_cast<uint32_t>(acc) << (cand & 31);
            if ((cand & 31) == 31) {
              A.mask[static_cast<long long>(cand >> 5) * A.n_atoms + t] = mword;
              mword = 0;
            }
          }
          if (!FILL && s - s0 < 32) slots |= static_cast<uint32_t>(acc) << (s - s0);
        }
        if (!FILL && A.rv) A.rv[static_cast<long long>(q) * A.n_atoms + t] = make_uint2(slots, before);
      }
    }
  }
  if (!FILL && A.mask && cand < kMaskBits && (cand & 31) != 0)
    A.mask[static_cast<long long>(cand >> 5) * A.n_atoms + t] = mword;
  if (!FILL) A.cnt[i] = count;
  else if (count != out_end - A.off[i]) atomicOr(A.err, ERRF_CAPACITY);
}

// Fill pass with one warp per atom (bin order), for configurations that scan at most 32 bins:
// lane q owns scanned bin q (its first binned atom, size, image and first candidate index), the
// count pass's accepted bits are located by prefix popcounts, and lane k forms the atom's k-th
// pair, so consecutive lanes write consecutive slots.  Candidates past the recorded bits are
// decided again, 32 at a time, and compacted by ballot.
// Reverse index: pair (i -> j) found in i's scanned bin q at j's binned position t_j is found
// from j in j's mirror bin n_scan - 1 - q (the scan order is point-symmetric) at i's slot in
// its own bin, so its place in j's list is off[j] + (j's pairs before that bin) + (j's accepted
// slots of that bin below i's slot), all recorded by the count pass.  Atoms past slot 31 of
// their bin leave -1 and ERRF_REVPEND for the search pass.
__device__ __forceinline__ int nth_set_bit(uint32_t m, int rem) {   // position of set bit #rem (0-based)
  int pos = 0;
#pragma unroll
  for (int width = 16; width; width >>= 1) {
    const int low = __popc(m & ((1u << width) - 1u));
    if (rem >= low) { rem -= low; m >>= width; pos += width; }
  }
  return pos;
}

__global__ void __launch_bounds__(256, 4) k_fill_warp(NbrArgs A) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int64_t t = (blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x) >> 5;
  if (t >= A.n_atoms) return;   // whole warps leave together
  const int64_t i = A.bin_atoms[t];
  const DevCfg& C = A.cfg[A.atom_cfg[i]];
  const int bc = A.bcoord[i];
  const int b[3] = {bc & 1023, (bc >> 10) & 1023, (bc >> 20) & 1023};
  const float4 xi_h = A.ph[i], xi_l = A.pl[i];
  const long long out0 = A.off[i], out1 = A.off[i + 1];
  const int w1 = 2 * C.kb[1] + 1, w2 = 2 * C.kb[2] + 1;
  const int n_scan = (2 * C.kb[0] + 1) * w1 * w2;
  const int slot_i = static_cast<int>(t - A.bin_start[A.atom_bin[i]]);   // i's slot in its bin
  // scanned bin of this lane (same order as k_pairs): first binned atom, size, image
  int n[3] = {0, 0, 0};
  long long s0 = 0;
  int sz = 0;
  if (lane < n_scan) {
    const int qd = C.qd[lane];
    const int d[3] = {(qd & 255) - 64, ((qd >> 8) & 255) - 64, ((qd >> 16) & 255) - 64};
    int tt[3];
    bool ok = true;
    for (int a = 0; a < 3; ++a) {
      tt[a] = b[a] + d[a];
      if (C.pbc[a]) {
        if (tt[a] < 0 || tt[a] >= C.nb[a]) {
          n[a] = (tt[a] >= 0) ? tt[a] / C.nb[a] : -((-tt[a] + C.nb[a] - 1) / C.nb[a]);
          tt[a] -= n[a] * C.nb[a];
        }
      } else if (tt[a] < 0 || tt[a] >= C.nb[a]) {
        ok = false;
      }
    }
    if (ok) {
      const long long tb = C.bin_base + (static_cast<long long>(tt[0]) * C.nb[1] + tt[1]) * C.nb[2] + tt[2];
      s0 = A.bin_start[tb];
      sz = static_cast<int>(A.bin_start[tb + 1] - s0);
    }
  }
  // first candidate index of each scanned bin (exclusive prefix of the sizes)
  int cst0 = sz;
  for (int m = 1; m < 32; m <<= 1) {
    const int v = __shfl_up_sync(full, cst0, m);
    if (lane >= m) cst0 += v;
  }
  const int ctot = __shfl_sync(full, cst0, 31);
  cst0 -= sz;
  const int cst = lane < n_scan ? cst0 : 0x7fffffff;   // lanes past the scan never match
  auto bin_of = [&](int c) {   // the scanned bin holding candidate c: the last lane with cst <= c
    int lo = 0, hi = 31;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (__shfl_sync(full, cst, mid) <= c) lo = mid; else hi = mid - 1;
    }
    return lo;
  };
  // the count pass's bits of the first min(ctot, kMaskBits) candidates, one word per lane
  const int nbits = min(ctot, kMaskBits);
  uint32_t word = 0;
  if (lane < kMaskWords && 32 * lane < nbits) {
    word = A.mask[static_cast<long long>(lane) * A.n_atoms + t];
    const int valid = nbits - 32 * lane;
    if (valid < 32) word &= (1u << valid) - 1u;
  }
  int wpre = __popc(word);
  for (int m = 1; m < 32; m <<= 1) {
    const int v = __shfl_up_sync(full, wpre, m);
    if (lane >= m) wpre += v;
  }
  const int nmask = __shfl_sync(full, wpre, 31);
  wpre -= __popc(word);
  // decide candidate c of scanned bin q again (every lane takes part in the shuffles)
  auto form = [&](int c, int q, bool act, int& j, int& img, float4& r, long long& sidx) -> int {
    const long long sb = __shfl_sync(full, s0, q);
    const int cq = __shfl_sync(full, cst0, q);
    const int n0 = __shfl_sync(full, n[0], q), n1 = __shfl_sync(full, n[1], q), n2 = __shfl_sync(full, n[2], q);
    if (!act) return 0;
    sidx = sb + (c - cq);
    const float4 xj_h = A.bph[sidx];
    j = __float_as_int(xj_h.w);
    if (j == static_cast<int>(i) && n0 == 0 && n1 == 0 && n2 == 0) return 0;
    return decide(A, C, i, j, xi_h, xi_l, xj_h, A.bpl[sidx], n0, n1, n2, r, img);
  };
  auto put = [&](long long o, int j, int img, const float4& r, int q, long long tj) {
    if (o >= out1) return;
    A.pj[o] = j;
    A.pimg[o] = img;
    A.pr32[o] = r;
    int rev = -1;
    if (slot_i < 32) {
      const uint2 e = A.rv[static_cast<long long>(n_scan - 1 - q) * A.n_atoms + tj];
      const long long oj = A.off[j], oj1 = A.off[j + 1];
      const long long pr = oj + e.y + __popc(e.x & ((1u << slot_i) - 1u));
      if (pr < oj1) rev = static_cast<int>(pr);
      else atomicOr(A.err, ERRF_REVERSE);   // j's record disagrees with its list
    } else {
      atomicOr(A.err, ERRF_REVPEND);
    }
    A.prev[o] = rev;
  };
  // accepted candidates among the recorded bits: lane k forms the atom's k-th pair
  for (int kb = 0; kb < nmask; kb += 32) {
    const int k = kb + lane;
    const bool act = k < nmask;
    int lo = 0, hi = kMaskWords - 1;   // the last word whose prefix count is <= k
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (__shfl_sync(full, wpre, mid) <= k) lo = mid; else hi = mid - 1;
    }
    const uint32_t ww = __shfl_sync(full, word, lo);
    const int wp = __shfl_sync(full, wpre, lo);
    const int c = act ? 32 * lo + nth_set_bit(ww, k - wp) : 0;
    const int q = bin_of(c);
    int j = 0, img = 0;
    float4 r;
    long long tj = 0;
    if (form(c, q, act, j, img, r, tj)) put(out0 + k, j, img, r, q, tj);
    else if (act) atomicOr(A.err, ERRF_CAPACITY);   // the replay disagrees with the count
  }
  long long written = nmask;
  // candidates past the recorded bits, decided again and compacted in scan order
  for (int cb = kMaskBits; cb < ctot; cb += 32) {
    const int c = cb + lane;
    const bool act = c < ctot;
    const int q = bin_of(act ? c : cb);
    int j = 0, img = 0;
    float4 r;
    long long tj = 0;
    const int acc = form(c, q, act, j, img, r, tj);
    const unsigned bal = __ballot_sync(full, acc != 0);
    if (acc) put(out0 + written + __popc(bal & ((1u << lane) - 1u)), j, img, r, q, tj);
    written += __popc(bal);
  }
  if (lane == 0 && written != out1 - out0) atomicOr(A.err, ERRF_CAPACITY);
}

// prev[p] = index of the reverse pair (j -> i, -image) of pair p = (i -> j, image), by a search
// of j's list: one warp per atom i (its pairs over the lanes).  MISSING: only the pairs the fill
// pass left at -1.
template <bool MISSING>
__global__ void k_reverse(NbrArgs A) {
  const int lane = threadIdx.x & 31;
  const long long wpb = blockDim.x >> 5;
  const long long nw = static_cast<long long>(gridDim.x) * wpb;
  for (long long i = blockIdx.x * wpb + (threadIdx.x >> 5); i < A.n_atoms; i += nw) {
    const long long p1 = A.off[i + 1];
    for (long long p = A.off[i] + lane; p < p1; p += 32) {
      if (MISSING && A.prev[p] >= 0) continue;
      const int j = A.pj[p];
      if (j < 0 || j >= A.n_atoms) {   // a list that disagrees with its count
        atomicOr(A.err, ERRF_REVERSE);
        A.prev[p] = static_cast<int>(p);
        continue;
      }
      const int img = A.pimg[p];
      const int want = pack_img(-unpack_img(img, 0), -unpack_img(img, 1), -unpack_img(img, 2));
      int found = -1;
      const long long q1 = A.off[j + 1];
      for (long long q = A.off[j]; q < q1; ++q)
        if (A.pj[q] == static_cast<int>(i) && A.pimg[q] == want) { found = static_cast<int>(q); break; }
      if (found < 0) atomicOr(A.err, ERRF_REVERSE);
      A.prev[p] = found < 0 ? static_cast<int>(p) : found;
    }
  }
}

template <class T>
void scan_exclusive(const T* in, T* out, int64_t n, DevBuf& tmp, cudaStream_t s) {
  size_t bytes = 0;
  MTP_CUDA(cub::DeviceScan::ExclusiveSum(nullptr, bytes, in, out, n, s));
  tmp.ensure(bytes, s);
  MTP_CUDA(cub::DeviceScan::ExclusiveSum(tmp.p, bytes, in, out, n, s));
}

int blocks_for(int64_t n, int t) { return static_cast<int>(std::max<int64_t>(1, (n + t - 1) / t)); }

}  // namespace

void build_neighbors(mtp_model* m, const mtp_batch* b, mtp_nbr* nb, cudaStream_t s) {
  const int n_cfg = b->n_cfg;
  if (n_cfg <= 0 || !b->atom_offset || !b->pos || !b->type || !b->cell || !b->pbc)
    throw Fail{MTP_ERR_ARG, "batch: null array or n_cfg <= 0"};
  std::vector<int64_t> ao(n_cfg + 1);
  std::vector<double> cell(9 * static_cast<size_t>(n_cfg));
  std::vector<uint8_t> pbc(3 * static_cast<size_t>(n_cfg));
  MTP_CUDA(cudaMemcpyAsync(ao.data(), b->atom_offset, ao.size() * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  MTP_CUDA(cudaMemcpyAsync(cell.data(), b->cell, cell.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
  MTP_CUDA(cudaMemcpyAsync(pbc.data(), b->pbc, pbc.size(), cudaMemcpyDeviceToHost, s));
  MTP_CUDA(cudaStreamSynchronize(s));
  if (ao[0] != 0) throw Fail{MTP_ERR_ARG, "atom_offset[0] must be 0"};
  for (int k = 0; k < n_cfg; ++k)
    if (ao[k + 1] < ao[k]) throw Fail{MTP_ERR_ARG, "atom_offset must be non-decreasing"};
  const int64_t N = ao[n_cfg];
  if (N <= 0) throw Fail{MTP_ERR_ARG, "empty batch"};
  if (N >= (int64_t(1) << 31)) throw Fail{MTP_ERR_UNSUPPORTED, "more than 2^31 atoms"};
  const double rc = m->desc.r_cut;
  std::vector<DevCfg> cfgs(n_cfg);
  std::vector<float4> shi, slo;
  long long bins = 0;
  nb->seg_host.clear();
  for (int k = 0; k < n_cfg; ++k) {
    DevCfg& C = cfgs[k];
    const double* H = &cell[9 * k];
    for (int q = 0; q < 9; ++q) C.H[q] = H[q];
    double c0[3] = {H[4] * H[8] - H[5] * H[7], H[5] * H[6] - H[3] * H[8], H[3] * H[7] - H[4] * H[6]};
    double c1[3] = {H[7] * H[2] - H[8] * H[1], H[8] * H[0] - H[6] * H[2], H[6] * H[1] - H[7] * H[0]};
    double c2[3] = {H[1] * H[5] - H[2] * H[4], H[2] * H[3] - H[0] * H[5], H[0] * H[4] - H[1] * H[3]};
    const double vol = H[0] * c0[0] + H[1] * c0[1] + H[2] * c0[2];
    if (!(std::fabs(vol) > 1e-9) || !std::isfinite(vol)) throw Fail{MTP_ERR_GEOMETRY, "degenerate cell"};
    for (int c = 0; c < 3; ++c) { C.Hinv[c * 3 + 0] = c0[c] / vol; C.Hinv[c * 3 + 1] = c1[c] / vol; C.Hinv[c * 3 + 2] = c2[c] / vol; }
    const double* cc[3] = {c0, c1, c2};
    int Kmax = 0;
    for (int a = 0; a < 3; ++a) {
      const double h = std::fabs(vol) / std::sqrt(cc[a][0] * cc[a][0] + cc[a][1] * cc[a][1] + cc[a][2] * cc[a][2]);
      C.pbc[a] = pbc[3 * k + a] ? 1 : 0;
      int n = static_cast<int>(std::floor(h / rc));
      n = std::max(1, std::min(n, 1024));
      C.nb[a] = n;
      C.kb[a] = static_cast<int>(std::ceil(rc * n / h - 1e-12));
      if (!C.pbc[a]) C.kb[a] = std::min(C.kb[a], n);
      if (C.pbc[a]) Kmax = std::max(Kmax, (C.kb[a] + n - 1) / n + 1);
      if (C.kb[a] > 64) throw Fail{MTP_ERR_GEOMETRY, "cell too thin for the cut-off (more than 64 images)"};
    }
    C.K = Kmax;
    {
      const int v1 = 2 * C.kb[1] + 1, v2 = 2 * C.kb[2] + 1, ns = (2 * C.kb[0] + 1) * v1 * v2;
      for (int q = 0; q < 32; ++q)
        C.qd[q] = q < ns ? ((q / (v1 * v2) - C.kb[0] + 64) | (((q / v2) % v1 - C.kb[1] + 64) << 8) |
                            ((q % v2 - C.kb[2] + 64) << 16))
                         : 0;
    }
    C.bin_base = bins;
    bins += static_cast<long long>(C.nb[0]) * C.nb[1] * C.nb[2];
    C.shift_base = static_cast<long long>(shi.size());
    for (int n0 = -Kmax; n0 <= Kmax; ++n0)
      for (int n1 = -Kmax; n1 <= Kmax; ++n1)
        for (int n2 = -Kmax; n2 <= Kmax; ++n2) {
          float hh[3], ll[3];
          for (int c = 0; c < 3; ++c) {
            const double v = n0 * H[0 * 3 + c] + n1 * H[1 * 3 + c] + n2 * H[2 * 3 + c];
            hh[c] = static_cast<float>(v);
            ll[c] = static_cast<float>(v - static_cast<double>(hh[c]));
          }
          shi.push_back(make_float4(hh[0], hh[1], hh[2], 0.f));
          slo.push_back(make_float4(ll[0], ll[1], ll[2], 0.f));
        }
    C.rc2 = rc * rc;
    C.rc2f = static_cast<float>(rc * rc);
    C.rcm2f = static_cast<float>((rc + 1e-3) * (rc + 1e-3));
    for (int64_t a0 = ao[k]; a0 < ao[k + 1]; a0 += 4096) {
      nb->seg_host.push_back(k);
      nb->seg_host.push_back(a0);
      nb->seg_host.push_back(std::min<int64_t>(a0 + 4096, ao[k + 1]));
    }
  }
  nb->n_atoms = N;
  nb->n_cfg = n_cfg;
  nb->atom_offset = ao;
  nb->n_bins_total = bins;
  nb->n_seg = static_cast<int64_t>(nb->seg_host.size() / 3);
  // device buffers
  nb->plan.ensure(cfgs.size() * sizeof(DevCfg) + 2 * shi.size() * sizeof(float4) + 64, s);
  DevCfg* d_cfg = nb->plan.as<DevCfg>();
  float4* d_shi = reinterpret_cast<float4*>(reinterpret_cast<char*>(d_cfg) + ((cfgs.size() * sizeof(DevCfg) + 15) & ~size_t(15)));
  float4* d_slo = d_shi + shi.size();
  MTP_CUDA(cudaMemcpyAsync(d_cfg, cfgs.data(), cfgs.size() * sizeof(DevCfg), cudaMemcpyHostToDevice, s));
  MTP_CUDA(cudaMemcpyAsync(d_shi, shi.data(), shi.size() * sizeof(float4), cudaMemcpyHostToDevice, s));
  MTP_CUDA(cudaMemcpyAsync(d_slo, slo.data(), slo.size() * sizeof(float4), cudaMemcpyHostToDevice, s));
  nb->seg.ensure(nb->seg_host.size() * sizeof(int64_t), s);
  MTP_CUDA(cudaMemcpyAsync(nb->seg.p, nb->seg_host.data(), nb->seg_host.size() * sizeof(int64_t),
                           cudaMemcpyHostToDevice, s));
  nb->atom_cfg.ensure(N * sizeof(int), s);
  nb->wrap.ensure(N * sizeof(int) + N * sizeof(long long) + 2 * N * sizeof(float4) + N * sizeof(int) + 64, s);
  int* d_wrap = nb->wrap.as<int>();
  long long* d_abin = reinterpret_cast<long long*>(reinterpret_cast<char*>(d_wrap) + ((N * sizeof(int) + 15) & ~size_t(15)));
  float4* d_ph = reinterpret_cast<float4*>(reinterpret_cast<char*>(d_abin) + ((N * sizeof(long long) + 15) & ~size_t(15)));
  float4* d_pl = d_ph + N;
  int* d_bcoord = reinterpret_cast<int*>(d_pl + N);
  const size_t bin_bytes = (bins + 1) * (2 * sizeof(int) + sizeof(long long)) + N * sizeof(int) + 2 * N * sizeof(float4) + 256;
  nb->bins.ensure(bin_bytes, s);
  char* bp = nb->bins.as<char>();
  long long* d_bstart = reinterpret_cast<long long*>(bp);
  int* d_bcount = reinterpret_cast<int*>(d_bstart + (bins + 1));
  int* d_bfill = d_bcount + (bins + 1);
  int* d_batoms = d_bfill + (bins + 1);
  float4* d_bph = reinterpret_cast<float4*>((reinterpret_cast<uintptr_t>(d_batoms + N) + 15) & ~uintptr_t(15));
  float4* d_bpl = d_bph + N;
  nb->counts.ensure((N + 1) * sizeof(long long), s);
  nb->off.ensure((N + 1) * sizeof(long long), s);
  m->err_flag.ensure(sizeof(unsigned), s);
  MTP_CUDA(cudaMemsetAsync(m->err_flag.p, 0, sizeof(unsigned), s));
  MTP_CUDA(cudaMemsetAsync(d_bcount, 0, 2 * (bins + 1) * sizeof(int), s));
  MTP_CUDA(cudaMemsetAsync(nb->counts.p, 0, (N + 1) * sizeof(long long), s));

  NbrArgs A{};
  A.n_atoms = N;
  A.n_cfg = n_cfg;
  A.atom_offset = b->atom_offset;
  A.pos = b->pos;
  A.type = b->type;
  A.n_types = m->desc.n_types;
  A.cfg = d_cfg;
  A.sh_hi = d_shi;
  A.sh_lo = d_slo;
  A.atom_cfg = nb->atom_cfg.as<int>();
  A.wrap = d_wrap;
  A.atom_bin = d_abin;
  A.bcoord = d_bcoord;
  A.ph = d_ph;
  A.pl = d_pl;
  A.bin_count = d_bcount;
  A.bin_fill = d_bfill;
  A.bin_start = d_bstart;
  A.bin_atoms = d_batoms;
  A.bph = d_bph;
  A.bpl = d_bpl;
  A.cnt = nb->counts.as<long long>();
  A.off = nb->off.as<long long>();
  A.err = m->err_flag.as<unsigned>();
  nb->masks.ensure(static_cast<size_t>(N) * kMaskWords * sizeof(uint32_t), s);
  A.mask = nb->masks.as<uint32_t>();
  // the warp fill and the reverse record, when every configuration scans at most 32 bins
  int max_scan = 0;
  for (const DevCfg& C : cfgs) max_scan = std::max(max_scan, (2 * C.kb[0] + 1) * (2 * C.kb[1] + 1) * (2 * C.kb[2] + 1));
  const bool warp_fill = max_scan <= kWarpScan;
  A.rv = nullptr;
  if (warp_fill) {
    nb->segs.ensure(static_cast<size_t>(max_scan) * N * sizeof(uint2), s);
    A.rv = nb->segs.as<uint2>();
  }
  const int TB = 256;
  {
    ProfRegion pr1("neighbors_bin_count", s);
    k_prep<<<blocks_for(N, TB), TB, 0, s>>>(A);
    ProfRegion::launched();
    MTP_CUDA(cudaGetLastError());
    // bin_count has bins+1 entries (last = 0) -> bin_start[bins] = N
    {
      // scan int counts into long long starts
      size_t bytes = 0;
      MTP_CUDA(cub::DeviceScan::ExclusiveSum(nullptr, bytes, d_bcount, d_bstart, bins + 1, s));
      nb->scratch.ensure(bytes, s);
      MTP_CUDA(cub::DeviceScan::ExclusiveSum(nb->scratch.p, bytes, d_bcount, d_bstart, bins + 1, s));
    }
    k_scatter<<<blocks_for(N, TB), TB, 0, s>>>(A);
    ProfRegion::launched();
    MTP_CUDA(cudaGetLastError());
    k_sort_bins<<<blocks_for(bins, TB), TB, 0, s>>>(A, bins);
    ProfRegion::launched();
    MTP_CUDA(cudaGetLastError());
    k_pairs<false><<<blocks_for(N, 128), 128, 0, s>>>(A);
    ProfRegion::launched();
    MTP_CUDA(cudaGetLastError());
    scan_exclusive<long long>(nb->counts.as<long long>(), nb->off.as<long long>(), N + 1, nb->scratch, s);
  }
  long long total = 0;
  unsigned flag = 0;
  MTP_CUDA(cudaMemcpyAsync(&total, nb->off.as<long long>() + N, sizeof(long long), cudaMemcpyDeviceToHost, s));
  MTP_CUDA(cudaMemcpyAsync(&flag, m->err_flag.p, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  MTP_CUDA(cudaStreamSynchronize(s));
  if (flag & ERRF_SPECIES) throw Fail{MTP_ERR_ARG, "species outside [0, n_types)"};
  if (flag & ERRF_NONFINITE) throw Fail{MTP_ERR_NUMERIC, "non-finite position"};
  if (flag & ERRF_GEOMETRY) throw Fail{MTP_ERR_GEOMETRY, "coincident atoms (|r_ij| < 1e-8 A)"};
  if (total >= (1LL << 31)) throw Fail{MTP_ERR_UNSUPPORTED, "more than 2^31 pairs"};
  nb->n_pairs = total;
  const int64_t P = std::max<long long>(total, 1);
  nb->pj.ensure(P * sizeof(int), s);
  nb->pimg.ensure(P * sizeof(int), s);
  nb->prev.ensure(P * sizeof(int), s);
  nb->pr32.ensure(P * sizeof(float4), s);
  A.pj = nb->pj.as<int>();
  A.pimg = nb->pimg.as<int>();
  A.pr32 = nb->pr32.as<float4>();
  A.prev = nb->prev.as<int>();
  // fill (at the counted offsets) with the reverse pairs; a fill that disagrees with its count
  // sets ERRF_CAPACITY: the pass is repeated once, then the build fails with MTP_ERR_CAPACITY
  for (int attempt = 0;; ++attempt) {
    {
      ProfRegion pr2("neighbors_fill", s);
      if (warp_fill) {
        k_fill_warp<<<blocks_for(N * 32, 256), 256, 0, s>>>(A);
        ProfRegion::launched();
      } else {
        k_pairs<true><<<blocks_for(N, 128), 128, 0, s>>>(A);
        ProfRegion::launched();
      }
      MTP_CUDA(cudaGetLastError());
    }
    if (!warp_fill && total > 0) {
      ProfRegion pr3("neighbors_reverse", s);
      k_reverse<false><<<blocks_for(N * 32, 256), 256, 0, s>>>(A);
      ProfRegion::launched();
      MTP_CUDA(cudaGetLastError());
    }
    MTP_CUDA(cudaMemcpyAsync(&flag, m->err_flag.p, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    MTP_CUDA(cudaStreamSynchronize(s));
    if (take_injected(g_inject_overflow)) flag |= ERRF_CAPACITY;
    if (flag & ERRF_GEOMETRY) throw Fail{MTP_ERR_GEOMETRY, "coincident atoms (|r_ij| < 1e-8 A)"};
    if (!(flag & ERRF_CAPACITY)) break;
    if (attempt == 1) throw Fail{MTP_ERR_CAPACITY, "neighbor fill overflowed its counted capacity twice"};
    MTP_CUDA(cudaMemsetAsync(m->err_flag.p, 0, sizeof(unsigned), s));
  }
  if ((flag & ERRF_REVPEND) && !(flag & ERRF_REVERSE)) {
    // atoms past slot 31 of their bin: their pairs' reverses by search
    {
      ProfRegion pr3("neighbors_reverse", s);
      k_reverse<true><<<blocks_for(N * 32, 256), 256, 0, s>>>(A);
      ProfRegion::launched();
      MTP_CUDA(cudaGetLastError());
    }
    MTP_CUDA(cudaMemcpyAsync(&flag, m->err_flag.p, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    MTP_CUDA(cudaStreamSynchronize(s));
  }
  if (flag & ERRF_REVERSE) throw Fail{MTP_ERR_NUMERIC, "inconsistent neighbor list (reverse-pair mismatch)"};
  DevNbr& D = nb->dn;
  D.n_atoms = N;
  D.n_pairs = total;
  D.off = reinterpret_cast<const int64_t*>(nb->off.p);
  D.pj = nb->pj.as<int>();
  D.pimg = nb->pimg.as<int>();
  D.prev = nb->prev.as<int>();
  D.pr32 = nb->pr32.as<float4>();
  D.atom_cfg = nb->atom_cfg.as<int>();
}

}  // namespace mtp

// Spherical cut of neighborhoods into non-periodic clusters (Section II.E, option (ii)).
//
// For a center atom c of configuration k: every atom j of k and periodic image n (periodic
// axes only) with |x_j + n H - x_c| < radius, the center itself first at the origin, then in
// ascending (j, n0, n1, n2).  One warp per center: the lanes take 32 consecutive atoms j, each
// lane walks its images in order, and a warp prefix sum places the lanes' hits in j order, so
// the output order is fixed.  Two passes (count, then fill at the scanned offsets).
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include <cub/cub.cuh>

#include "mtp_internal.h"
#include "profiler.h"

namespace mtp {
namespace {

constexpr unsigned ERR_CENTER = 1u;
constexpr unsigned ERR_FILL = 2u;
constexpr int kMaxImages = 64;   // per axis and direction

struct CutArgs {
  const int64_t* atom_offset;
  int n_cfg;
  const double* pos;
  const int32_t* type;
  const double* cell;     // n_cfg x 9, rows = lattice vectors
  const uint8_t* pbc;     // n_cfg x 3
  const int64_t* centers;
  int64_t n;
  double radius;
  long long* count;       // [n + 1]
  const long long* off;   // [n + 1] (fill pass)
  double* out_pos;
  int32_t* out_type;
  int64_t* out_src;
  unsigned* err;
};

__device__ int config_of(const CutArgs& A, int64_t atom) {
  int lo = 0, hi = A.n_cfg - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (A.atom_offset[mid] <= atom) lo = mid; else hi = mid - 1;
  }
  return lo;
}

template <bool FILL>
__global__ void k_cut(CutArgs A) {
  const int lane = threadIdx.x & 31;
  const int64_t q = blockIdx.x * static_cast<int64_t>(blockDim.x >> 5) + (threadIdx.x >> 5);
  if (q >= A.n) return;
  const int64_t c = A.centers[q];
  const int64_t n_atoms = A.atom_offset[A.n_cfg];
  if (c < 0 || c >= n_atoms) {
    if (lane == 0) { atomicOr(A.err, ERR_CENTER); if (!FILL) A.count[q] = 0; }
    return;
  }
  const int k = config_of(A, c);
  const int64_t a0 = A.atom_offset[k], a1 = A.atom_offset[k + 1];
  const double* H = A.cell + 9 * static_cast<int64_t>(k);
  // reciprocal rows (fractional coordinates) and face distances
  double G[9];
  const double c0[3] = {H[4] * H[8] - H[5] * H[7], H[5] * H[6] - H[3] * H[8], H[3] * H[7] - H[4] * H[6]};
  const double c1[3] = {H[7] * H[2] - H[8] * H[1], H[8] * H[0] - H[6] * H[2], H[6] * H[1] - H[7] * H[0]};
  const double c2[3] = {H[1] * H[5] - H[2] * H[4], H[2] * H[3] - H[0] * H[5], H[0] * H[4] - H[1] * H[3]};
  const double vol = H[0] * c0[0] + H[1] * c0[1] + H[2] * c0[2];
  for (int d = 0; d < 3; ++d) { G[0 * 3 + d] = c0[d] / vol; G[1 * 3 + d] = c1[d] / vol; G[2 * 3 + d] = c2[d] / vol; }
  int K[3];
  const double* cc[3] = {c0, c1, c2};
  for (int a = 0; a < 3; ++a) {
    const double h = fabs(vol) / sqrt(cc[a][0] * cc[a][0] + cc[a][1] * cc[a][1] + cc[a][2] * cc[a][2]);
    K[a] = A.pbc[3 * k + a] ? min(kMaxImages, static_cast<int>(ceil(A.radius / h)) + 1) : 0;
  }
  const double xc[3] = {A.pos[3 * c], A.pos[3 * c + 1], A.pos[3 * c + 2]};
  const double rad = A.radius;
  long long base = FILL ? A.off[q] : 0;
  if (FILL && lane == 0) {
    // the center first
    A.out_pos[3 * base] = 0.0; A.out_pos[3 * base + 1] = 0.0; A.out_pos[3 * base + 2] = 0.0;
    A.out_type[base] = A.type[c];
    A.out_src[base] = c;
  }
  base += 1;
  long long total = 1;
  for (int64_t j0 = a0; j0 < a1; j0 += 32) {
    const int64_t j = j0 + lane;
    const bool act = j < a1;
    // image of j nearest to c along each periodic axis: n = m - round(f)
    int s[3] = {0, 0, 0};
    double xj[3] = {0.0, 0.0, 0.0};
    if (act) {
      for (int d = 0; d < 3; ++d) xj[d] = A.pos[3 * j + d];
      for (int a = 0; a < 3; ++a) {
        const double f = (xj[0] - xc[0]) * G[a] + (xj[1] - xc[1]) * G[3 + a] + (xj[2] - xc[2]) * G[6 + a];
        s[a] = A.pbc[3 * k + a] ? static_cast<int>(rint(f)) : 0;
      }
    }
    // pass over this lane's images in ascending (n0, n1, n2): count, or count and write
    auto visit = [&](auto emit) {
      int hits = 0;
      if (!act) return hits;
      for (int m0 = -K[0]; m0 <= K[0]; ++m0)
        for (int m1 = -K[1]; m1 <= K[1]; ++m1)
          for (int m2 = -K[2]; m2 <= K[2]; ++m2) {
            const int n0 = m0 - s[0], n1 = m1 - s[1], n2 = m2 - s[2];
            if (j == c && n0 == 0 && n1 == 0 && n2 == 0) continue;
            double r[3];
            for (int d = 0; d < 3; ++d) {
              const double sh = __dadd_rn(__dadd_rn(__dmul_rn(static_cast<double>(n0), H[d]),
                                                    __dmul_rn(static_cast<double>(n1), H[3 + d])),
                                          __dmul_rn(static_cast<double>(n2), H[6 + d]));
              r[d] = __dsub_rn(__dadd_rn(xj[d], sh), xc[d]);
            }
            const double rr = __dadd_rn(__dadd_rn(__dmul_rn(r[0], r[0]), __dmul_rn(r[1], r[1])), __dmul_rn(r[2], r[2]));
            if (__dsqrt_rn(rr) < rad) { emit(hits, r); ++hits; }
          }
      return hits;
    };
    const int mine = visit([](int, const double*) {});
    // warp exclusive prefix of the lanes' hits (lanes hold ascending j)
    int incl = mine;
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    const int excl = incl - mine;
    const int round_total = __shfl_sync(0xffffffffu, incl, 31);
    if (FILL) {
      const long long at = base + excl;
      const long long end = A.off[q + 1];
      visit([&](int h, const double* r) {
        const long long o = at + h;
        if (o < end) {
          A.out_pos[3 * o] = r[0]; A.out_pos[3 * o + 1] = r[1]; A.out_pos[3 * o + 2] = r[2];
          A.out_type[o] = A.type[j];
          A.out_src[o] = j;
        } else {
          atomicOr(A.err, ERR_FILL);
        }
      });
    }
    base += round_total;
    total += round_total;
  }
  if (!FILL && lane == 0) A.count[q] = total;
  if (FILL && lane == 0 && base != A.off[q + 1]) atomicOr(A.err, ERR_FILL);
}

}  // namespace

int64_t run_cut_clusters(const mtp_batch* b, const int64_t* centers, int64_t n, double radius, int64_t* off,
                         double* pos, int32_t* type, int64_t* src, int64_t capacity, cudaStream_t s) {
  DevBuf work;
  work.ensure((n + 1) * sizeof(long long) + 64, s);
  long long* cnt = work.as<long long>();
  unsigned* err = reinterpret_cast<unsigned*>(cnt + n + 1);
  MTP_CUDA(cudaMemsetAsync(err, 0, sizeof(unsigned), s));
  MTP_CUDA(cudaMemsetAsync(cnt + n, 0, sizeof(long long), s));
  CutArgs A{};
  A.atom_offset = b->atom_offset;
  A.n_cfg = b->n_cfg;
  A.pos = b->pos;
  A.type = b->type;
  A.cell = b->cell;
  A.pbc = b->pbc;
  A.centers = centers;
  A.n = n;
  A.radius = radius;
  A.count = cnt;
  A.err = err;
  const unsigned g = static_cast<unsigned>(std::max<int64_t>(1, (n + 7) / 8));
  ProfRegion pr("cut_clusters", s);
  k_cut<false><<<g, 256, 0, s>>>(A);
  ProfRegion::launched();
  MTP_CUDA(cudaGetLastError());
  // offsets: exclusive scan of the counts into off[0..n]
  DevBuf scan_tmp;
  size_t bytes = 0;
  long long* offl = reinterpret_cast<long long*>(off);
  MTP_CUDA(cub::DeviceScan::ExclusiveSum(nullptr, bytes, cnt, offl, static_cast<int>(n + 1), s));
  scan_tmp.ensure(bytes, s);
  MTP_CUDA(cub::DeviceScan::ExclusiveSum(scan_tmp.p, bytes, cnt, offl, static_cast<int>(n + 1), s));
  long long total = 0;
  unsigned flag = 0;
  MTP_CUDA(cudaMemcpyAsync(&total, offl + n, sizeof(long long), cudaMemcpyDeviceToHost, s));
  MTP_CUDA(cudaMemcpyAsync(&flag, err, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  MTP_CUDA(cudaStreamSynchronize(s));
  if (flag & ERR_CENTER) throw Fail{MTP_ERR_ARG, "center atom index out of range"};
  if (!pos || !type || !src || total > capacity) return total;
  A.off = offl;
  A.out_pos = pos;
  A.out_type = type;
  A.out_src = src;
  k_cut<true><<<g, 256, 0, s>>>(A);
  ProfRegion::launched();
  MTP_CUDA(cudaGetLastError());
  MTP_CUDA(cudaMemcpyAsync(&flag, err, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  MTP_CUDA(cudaStreamSynchronize(s));
  if (flag) throw Fail{MTP_ERR_NUMERIC, "cluster cut: count and fill passes disagree"};
  return total;
}

}  // namespace mtp

// Forces, per-configuration sums, flag compaction, neighborhood extraction and the loss
// reductions of the training step.
//
// Forces (F = -dE/dx, used by eq. 7): with G_p = dV_i/dr_ij for pair p = (i -> j, n) and
// rev(p) = (j -> i, -n),  F_i = sum_{p in nbh(i)} (G_p - G_rev(p)); a deterministic gather in
// FP64 (no atomics).  Energies (eq. 1) and virials are summed per configuration over fixed
// atom segments, then per configuration over its segments, in a fixed order.
#include <cub/cub.cuh>
#include <thrust/iterator/counting_iterator.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "mtp_internal.h"
#include "profiler.h"

namespace mtp {
namespace {

int nblk(int64_t n, int t) { return static_cast<int>(std::max<int64_t>(1, (n + t - 1) / t)); }

// FP64 gradients: one thread per atom, pairs in list order
__global__ void k_forces(DevNbr nb, const double* G, double* F) {
  int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i >= nb.n_atoms) return;
  double f0 = 0, f1 = 0, f2 = 0;
  for (int64_t p = nb.off[i]; p < nb.off[i + 1]; ++p) {
    const int64_t q = nb.prev[p];
    f0 += G[3 * p + 0] - G[3 * q + 0];
    f1 += G[3 * p + 1] - G[3 * q + 1];
    f2 += G[3 * p + 2] - G[3 * q + 2];
  }
  F[3 * i + 0] = f0;
  F[3 * i + 1] = f1;
  F[3 * i + 2] = f2;
}

// FP32 gradients, LPA lanes per atom: each component summed as an unevaluated pair hi + lo of
// floats with error-free additions (TwoSum), as accurate as an FP64 accumulation on the FP32
// pipes (FP64 throughput is a small fraction of FP32 on this GPU); lane k of an atom's group
// takes pairs k, k + LPA, ..., and the group combines its partial pairs in a fixed tree
template <int LPA>
__global__ void k_forces_grp(DevNbr nb, const float* G, double* F) {
  const int64_t gid = (blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x) / LPA;
  const int k = threadIdx.x & (LPA - 1);
  const bool act = gid < nb.n_atoms;
  const int64_t i = act ? gid : 0;
  float h[3] = {0.f, 0.f, 0.f}, l[3] = {0.f, 0.f, 0.f};
  auto two = [](float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  };
  if (act) {
    const int64_t p1 = nb.off[i + 1];
    for (int64_t p = nb.off[i] + k; p < p1; p += LPA) {
      const int64_t q = nb.prev[p];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        float s, e;
        two(h[c], G[3 * p + c], s, e);
        h[c] = s; l[c] = __fadd_rn(l[c], e);
        two(h[c], -G[3 * q + c], s, e);
        h[c] = s; l[c] = __fadd_rn(l[c], e);
      }
    }
  }
#pragma unroll
  for (int m = LPA / 2; m; m >>= 1)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float oh = __shfl_xor_sync(0xffffffffu, h[c], m), ol = __shfl_xor_sync(0xffffffffu, l[c], m);
      // the lower lane of each pair adds the upper one's, so both get the same sum
      float s, e;
      if (k & m) two(oh, h[c], s, e); else two(h[c], oh, s, e);
      h[c] = s;
      l[c] = __fadd_rn(__fadd_rn((k & m) ? ol : l[c], (k & m) ? l[c] : ol), e);
    }
  if (act && k < 3) {
    const float hv = k == 0 ? h[0] : (k == 1 ? h[1] : h[2]);
    const float lv = k == 0 ? l[0] : (k == 1 ? l[1] : l[2]);
    F[3 * i + k] = static_cast<double>(hv) + static_cast<double>(lv);
  }
}

// one block per segment (cfg, a0, a1): partial[seg][0] = sum V, [1..9] = sum W
__global__ void k_seg_sums(const int64_t* seg, const double* V, const double* Wat, double* part) {
  const int64_t s = blockIdx.x;
  const int64_t a0 = seg[3 * s + 1], a1 = seg[3 * s + 2];
  __shared__ double red[10][256];
  double acc[10];
  for (int k = 0; k < 10; ++k) acc[k] = 0.0;
  for (int64_t a = a0 + threadIdx.x; a < a1; a += blockDim.x) {
    if (V) acc[0] += V[a];
    if (Wat)
      for (int k = 0; k < 9; ++k) acc[1 + k] += Wat[9 * a + k];
  }
  for (int k = 0; k < 10; ++k) red[k][threadIdx.x] = acc[k];
  __syncthreads();
  for (int w = blockDim.x / 2; w; w >>= 1) {
    if (threadIdx.x < w)
      for (int k = 0; k < 10; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < 10) part[10 * s + threadIdx.x] = red[threadIdx.x][0];
}

__global__ void k_cfg_sums(const int64_t* seg, int64_t n_seg, const double* part, int n_cfg, double* E, double* W) {
  // warp per config; the config's segments (contiguous in seg) are taken by lane s mod 32 in
  // order, then summed over the lanes in a fixed shuffle tree
  const int lane = threadIdx.x & 31;
  const int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (k >= n_cfg) return;   // whole warps
  int64_t lo = 0, hi = n_seg;   // first segment of config k
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (seg[3 * mid] < k) lo = mid + 1; else hi = mid;
  }
  double acc[10];
  for (int q = 0; q < 10; ++q) acc[q] = 0.0;
  for (int64_t s = lo + lane; s < n_seg && seg[3 * s] == k; s += 32)
    for (int q = 0; q < 10; ++q) acc[q] += part[10 * s + q];
  for (int m = 16; m; m >>= 1)
    for (int q = 0; q < 10; ++q) {
      const double o = __shfl_xor_sync(0xffffffffu, acc[q], m);
      acc[q] = (lane & m) ? o + acc[q] : acc[q] + o;   // both lanes of a pair form the same sum
    }
  if (lane == 0) {
    if (E) E[k] = acc[0];
    if (W)
      for (int q = 0; q < 9; ++q) W[9 * k + q] = acc[1 + q];
  }
}

struct AboveThreshold {
  const double* gamma;
  double thr;
  __device__ bool operator()(int i) const { return gamma[i] > thr; }
};

__global__ void k_extract_counts(DevNbr nb, const int32_t* idx, int64_t n, long long* cnt, unsigned* bad) {
  int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (k > n) return;
  if (k == n) { cnt[k] = 0; return; }
  const int i = idx[k];
  if (i < 0 || i >= nb.n_atoms) { atomicOr(bad, 1u); cnt[k] = 0; return; }
  cnt[k] = nb.off[i + 1] - nb.off[i];
}

__global__ void k_extract_fill(DevNbr nb, const double* pos, const int* type, const double* cell,
                               const int32_t* idx, int64_t n, const long long* off, double* r, int32_t* ty,
                               int32_t* jout) {
  int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (k >= n) return;
  const int i = idx[k];
  if (i < 0 || i >= nb.n_atoms) return;
  const double* H = cell + 9 * nb.atom_cfg[i];
  int64_t o = off[k];
  for (int64_t p = nb.off[i]; p < nb.off[i + 1]; ++p, ++o) {
    const int j = nb.pj[p];
    const int img = nb.pimg[p];
    const int n0 = unpack_img(img, 0), n1 = unpack_img(img, 1), n2 = unpack_img(img, 2);
    if (r)
      for (int c = 0; c < 3; ++c) {
        const double sh = n0 * H[c] + n1 * H[3 + c] + n2 * H[6 + c];
        r[3 * o + c] = (pos[3 * j + c] + sh) - pos[3 * i + c];
      }
    if (ty) ty[o] = type[j];
    if (jout) jout[o] = j;
  }
}

// U_i = 2 w_f (F_i - F*_i); per-block partial of sum |F - F*|^2
__global__ void k_train_forces(int64_t n, const double* F, const double* Fref, double w_f, double* U, double* part) {
  __shared__ double red[256];
  double acc = 0.0;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    for (int c = 0; c < 3; ++c) {
      const double d = F[3 * i + c] - Fref[3 * i + c];
      U[3 * i + c] = 2.0 * w_f * d;
      acc += d * d;
    }
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = blockDim.x / 2; w; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void k_train_cfg(int n_cfg, const double* E, const double* Eref, const double* W, const double* Wref,
                            double w_e, double w_f, double w_s, const double* fpart, int n_fpart, double* coef,
                            double* S, double* loss) {
  __shared__ double red[256];
  double acc = 0.0;
  for (int k = threadIdx.x; k < n_cfg; k += blockDim.x) {
    const double dE = E[k] - Eref[k];
    coef[k] = 2.0 * w_e * dE;
    acc += w_e * dE * dE;
    for (int q = 0; q < 9; ++q) {
      const double dW = (w_s != 0.0 && Wref) ? W[9 * k + q] - Wref[9 * k + q] : 0.0;
      S[9 * k + q] = 2.0 * w_s * dW;
      acc += w_s * dW * dW;
    }
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = blockDim.x / 2; w; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double f = 0.0;
    for (int b = 0; b < n_fpart; ++b) f += fpart[b];
    loss[0] = red[0] + w_f * f;
  }
}

__global__ void k_sum_rows(const double* part, int nrows, int64_t m, double* out) {
  int64_t c = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (c >= m) return;
  double acc = 0.0;
  for (int r = 0; r < nrows; ++r) acc += part[static_cast<int64_t>(r) * m + c];
  out[c] = acc;
}

}  // namespace

void run_forces(const mtp_nbr* nb, bool fp64, const void* G, double* F, cudaStream_t s) {
  ProfRegion pr("force_gather", s);
  if (fp64) {
    k_forces<<<nblk(nb->n_atoms, 256), 256, 0, s>>>(nb->dn, static_cast<const double*>(G), F);
    ProfRegion::launched();
  } else {
    k_forces_grp<8><<<nblk(nb->n_atoms * 8, 256), 256, 0, s>>>(nb->dn, static_cast<const float*>(G), F);
    ProfRegion::launched();
  }
  MTP_CUDA(cudaGetLastError());
}

void run_config_sums(const mtp_nbr* nb, const double* V, const double* Wat, double* E, double* W, DevBuf& tmp,
                     cudaStream_t s) {
  tmp.ensure(nb->n_seg * 10 * sizeof(double), s);
  ProfRegion pr("config_sums", s);
  k_seg_sums<<<static_cast<unsigned>(nb->n_seg), 256, 0, s>>>(nb->seg.as<int64_t>(), V, Wat, tmp.as<double>());
  ProfRegion::launched();
  MTP_CUDA(cudaGetLastError());
  k_cfg_sums<<<nblk(nb->n_cfg * 32, 128), 128, 0, s>>>(nb->seg.as<int64_t>(), nb->n_seg, tmp.as<double>(),
                                                 static_cast<int>(nb->n_cfg), E, W);
  ProfRegion::launched();
  MTP_CUDA(cudaGetLastError());
}

void run_config_sums_into(const mtp_nbr* nb, const double* V, const double* Wat, double* E, double* W, double* part,
                          cudaStream_t s) {
  ProfRegion pr("config_sums", s);
  k_seg_sums<<<static_cast<unsigned>(nb->n_seg), 256, 0, s>>>(nb->seg.as<int64_t>(), V, Wat, part);
  ProfRegion::launched();
  MTP_CUDA(cudaGetLastError());
  k_cfg_sums<<<nblk(nb->n_cfg * 32, 128), 128, 0, s>>>(nb->seg.as<int64_t>(), nb->n_seg, part, static_cast<int>(nb->n_cfg),
                                                 E, W);
  ProfRegion::launched();
  MTP_CUDA(cudaGetLastError());
}

namespace {
__global__ void k_iota64(int64_t n, int64_t* out) {
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i < n) out[i] = i;
}
__global__ void k_rank64(int64_t n, const int64_t* order, int64_t* rank) {
  const int64_t r = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (r < n) rank[order[r]] = r;
}
}  // namespace

void run_species_order(const int32_t* type, int64_t N, int n_types, int32_t* zrow, int64_t* order, DevBuf& tmp,
                       cudaStream_t s) {
  // a stable radix sort of the atom indices by species (ties keep index order)
  ProfRegion pr("grade_row_order", s);
  int bits = 1;
  while ((1 << bits) < n_types) ++bits;
  int64_t* iota = order + N;   // the caller provides 2N entries
  k_iota64<<<nblk(N, 256), 256, 0, s>>>(N, iota);
  ProfRegion::launched();
  MTP_CUDA(cudaGetLastError());
  size_t bytes = 0;
  MTP_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, bytes, type, zrow, iota, order, static_cast<int>(N), 0, bits, s));
  tmp.ensure(bytes, s);
  MTP_CUDA(cub::DeviceRadixSort::SortPairs(tmp.p, bytes, type, zrow, iota, order, static_cast<int>(N), 0, bits, s));
  k_rank64<<<nblk(N, 256), 256, 0, s>>>(N, order, order + N);   // the sort's input is no longer needed
  ProfRegion::launched();
  MTP_CUDA(cudaGetLastError());
}

void run_flag(int64_t N, const double* gamma, double threshold, int32_t* flagged, int64_t* n_flagged, DevBuf& tmp,
              cudaStream_t s) {
  AboveThreshold pred{gamma, threshold};
  ProfRegion pr("flag_compact", s);
  thrust::counting_iterator<int> it(0);
  size_t bytes = 0;
  MTP_CUDA(cub::DeviceSelect::If(nullptr, bytes, it, flagged, n_flagged, static_cast<int>(N), pred, s));
  tmp.ensure(bytes, s);
  MTP_CUDA(cub::DeviceSelect::If(tmp.p, bytes, it, flagged, n_flagged, static_cast<int>(N), pred, s));
}

int64_t run_extract(const mtp_nbr* nb, const mtp_batch* b, const int32_t* idx, int64_t n, int64_t* off, double* r,
                    int32_t* type, int32_t* j, int64_t capacity, DevBuf& tmp, cudaStream_t s) {
  tmp.ensure((n + 1) * sizeof(long long) + 64, s);
  long long* cnt = tmp.as<long long>();
  unsigned* bad = reinterpret_cast<unsigned*>(cnt + n + 1);
  MTP_CUDA(cudaMemsetAsync(bad, 0, sizeof(unsigned), s));
  k_extract_counts<<<nblk(n + 1, 256), 256, 0, s>>>(nb->dn, idx, n, cnt, bad);
  ProfRegion::launched();
  MTP_CUDA(cudaGetLastError());
  DevBuf scan_tmp;
  size_t bytes = 0;
  long long* offl = reinterpret_cast<long long*>(off);
  MTP_CUDA(cub::DeviceScan::ExclusiveSum(nullptr, bytes, cnt, offl, n + 1, s));
  scan_tmp.ensure(bytes, s);
  MTP_CUDA(cub::DeviceScan::ExclusiveSum(scan_tmp.p, bytes, cnt, offl, n + 1, s));
  long long total = 0;
  unsigned badh = 0;
  MTP_CUDA(cudaMemcpyAsync(&total, offl + n, sizeof(long long), cudaMemcpyDeviceToHost, s));
  MTP_CUDA(cudaMemcpyAsync(&badh, bad, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  MTP_CUDA(cudaStreamSynchronize(s));
  scan_tmp.release();
  if (badh) throw Fail{MTP_ERR_ARG, "atom index out of range"};
  if (total > capacity) return total;
  if (n > 0) {
    k_extract_fill<<<nblk(n, 128), 128, 0, s>>>(nb->dn, b->pos, b->type, b->cell, idx, n, offl, r, type, j);
    ProfRegion::launched();
    MTP_CUDA(cudaGetLastError());
  }
  return total;
}

void run_train_prep(const mtp_nbr* nb, int n_cfg, const double* E, const double* F, const double* W,
                    const double* E_ref, const double* F_ref, const double* W_ref, double w_e, double w_f,
                    double w_s, double* coef, double* U, double* Scfg, double* loss, DevBuf& tmp, cudaStream_t s) {
  const int nb_f = 256;
  tmp.ensure(nb_f * sizeof(double), s);
  ProfRegion pr("train_residuals", s);
  k_train_forces<<<nb_f, 256, 0, s>>>(nb->n_atoms, F, F_ref, w_f, U, tmp.as<double>());
  ProfRegion::launched();
  MTP_CUDA(cudaGetLastError());
  k_train_cfg<<<1, 256, 0, s>>>(n_cfg, E, E_ref, W, W_ref, w_e, w_f, w_s, tmp.as<double>(), nb_f, coef, Scfg, loss);
  ProfRegion::launched();
  MTP_CUDA(cudaGetLastError());
}

void run_sum_rows(const double* part, int nrows, int64_t m, double* out, cudaStream_t s) {
  ProfRegion pr("train_grad_sum", s);
  k_sum_rows<<<nblk(m, 128), 128, 0, s>>>(part, nrows, m, out);
  ProfRegion::launched();
  MTP_CUDA(cudaGetLastError());
}

}  // namespace mtp

// Configuration-level grades (Sections II.D-II.E).
//
//   b(cfg_k) = dE_k/dtheta = sum_{i in k} b_i        configuration rows (eq. 1 with eq. 9)
//   gamma(cfg_k) = max_j |(b(cfg_k) A^-1)_j|          configuration mode (A from configuration rows)
//   gamma(cfg_k) = max_{i in k} gamma_i               neighborhood mode
//   class_k = [gamma > gamma_save] + [gamma > gamma_break]   (0 continue, 1 save, 2 stop)
//
// Sums over a configuration's atoms go through the fixed segments of the neighbor list
// (at most 4096 atoms each, in order) and then over the segments in order: deterministic.
#include <cuda_runtime.h>

#include <algorithm>

#include "mtp_internal.h"
#include "profiler.h"

namespace mtp {
namespace {

unsigned blocks(int64_t n, int t) { return static_cast<unsigned>(std::max<int64_t>(1, (n + t - 1) / t)); }

// part[s][p] = sum over the atoms of segment s of rows[a][p]
__global__ void k_seg_row_sums(const int64_t* seg, const double* __restrict__ rows, int64_t m, double* part) {
  const int64_t s = blockIdx.x;
  const int64_t p = blockIdx.y * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (p >= m) return;
  const int64_t a0 = seg[3 * s + 1], a1 = seg[3 * s + 2];
  double acc = 0.0;
  for (int64_t a = a0; a < a1; ++a) acc += rows[a * m + p];
  part[s * m + p] = acc;
}

// first segment of configuration k (segments are sorted by configuration)
__device__ int64_t first_segment(const int64_t* seg, int64_t n_seg, int64_t k) {
  int64_t lo = 0, hi = n_seg;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (seg[3 * mid] < k) lo = mid + 1; else hi = mid;
  }
  return lo;
}

__global__ void k_cfg_row_sums(const int64_t* seg, int64_t n_seg, const double* __restrict__ part, int64_t m,
                               int64_t n_cfg, double* out) {
  const int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (t >= n_cfg * m) return;
  const int64_t k = t / m, p = t - k * m;
  double acc = 0.0;
  for (int64_t s = first_segment(seg, n_seg, k); s < n_seg && seg[3 * s] == k; ++s) acc += part[s * m + p];
  out[t] = acc;
}

// per segment: the largest gamma_i and the lowest atom attaining it
__global__ void k_seg_gamma_max(const int64_t* seg, const double* __restrict__ gamma, double* gmax, int64_t* amax) {
  const int64_t s = blockIdx.x;
  const int64_t a0 = seg[3 * s + 1], a1 = seg[3 * s + 2];
  double best = -1.0;
  int64_t arg = -1;
  for (int64_t a = a0 + threadIdx.x; a < a1; a += blockDim.x)
    if (gamma[a] > best) { best = gamma[a]; arg = a; }
  __shared__ double sb[256];
  __shared__ int64_t sa[256];
  sb[threadIdx.x] = best;
  sa[threadIdx.x] = arg;
  __syncthreads();
  for (int w = blockDim.x / 2; w; w >>= 1) {
    if (threadIdx.x < w) {
      const double ob = sb[threadIdx.x + w];
      const int64_t oa = sa[threadIdx.x + w];
      if (oa >= 0 && (ob > sb[threadIdx.x] || (ob == sb[threadIdx.x] && (sa[threadIdx.x] < 0 || oa < sa[threadIdx.x])))) {
        sb[threadIdx.x] = ob;
        sa[threadIdx.x] = oa;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) { gmax[s] = sb[0]; amax[s] = sa[0]; }
}

__global__ void k_cfg_gamma_max(const int64_t* seg, int64_t n_seg, const double* gmax, const int64_t* amax,
                                int64_t n_cfg, double* gamma_cfg, int64_t* worst) {
  const int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (k >= n_cfg) return;
  double best = 0.0;
  int64_t arg = -1;
  for (int64_t s = first_segment(seg, n_seg, k); s < n_seg && seg[3 * s] == k; ++s)
    if (amax[s] >= 0 && (arg < 0 || gmax[s] > best)) { best = gmax[s]; arg = amax[s]; }
  gamma_cfg[k] = best;
  if (worst) worst[k] = arg;
}

__global__ void k_classify(const double* gamma, int64_t n, double g_save, double g_break, int32_t* cls) {
  const int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (k >= n) return;
  const double g = gamma[k];
  cls[k] = (g > g_save ? 1 : 0) + (g > g_break ? 1 : 0);
}

// vector-Jacobian product of the configuration energies (eq. 1): dtheta[p] = sum_k gE[k] R[k][p]
// with R the configuration rows, summed over k in order (deterministic)
__global__ void k_vjp_theta(const double* R, const double* gE, int n_cfg, int64_t m, double* g) {
  const int64_t p = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (p >= m) return;
  double acc = 0.0;
  for (int k = 0; k < n_cfg; ++k) acc = fma(gE[k], R[k * m + p], acc);
  g[p] = acc;
}

// dE_k/dx_i = -F_i for the atoms i of configuration k, scaled by gE[k]
__global__ void k_vjp_pos(const double* F, const double* gE, const int* atom_cfg, int64_t N, double* g) {
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i >= N) return;
  const double w = gE[atom_cfg[i]];
  for (int c = 0; c < 3; ++c) g[3 * i + c] = -w * F[3 * i + c];
}

__global__ void k_widen_argmax(const int32_t* in, int64_t n, int64_t* out) {
  const int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (k < n) out[k] = in[k];
}

}  // namespace

void run_config_row_sums(const mtp_nbr* nb, const double* rows, int64_t m, double* out, DevBuf& tmp, cudaStream_t s) {
  tmp.ensure(static_cast<size_t>(nb->n_seg) * m * sizeof(double), s);
  ProfRegion pr("config_rows_sum", s);
  const dim3 g(static_cast<unsigned>(nb->n_seg), blocks(m, 128));
  if (nb->n_seg > 0) {
    k_seg_row_sums<<<g, 128, 0, s>>>(nb->seg.as<int64_t>(), rows, m, tmp.as<double>());
    ProfRegion::launched();
  }
  k_cfg_row_sums<<<blocks(nb->n_cfg * m, 256), 256, 0, s>>>(nb->seg.as<int64_t>(), nb->n_seg, tmp.as<double>(), m,
                                                           nb->n_cfg, out);
  ProfRegion::launched();
  MTP_CUDA(cudaGetLastError());
}

void run_config_gamma_max(const mtp_nbr* nb, const double* gamma, double* gamma_cfg, int64_t* worst, DevBuf& tmp,
                          cudaStream_t s) {
  tmp.ensure(static_cast<size_t>(std::max<int64_t>(nb->n_seg, 1)) * (sizeof(double) + sizeof(int64_t)), s);
  double* gmax = tmp.as<double>();
  int64_t* amax = reinterpret_cast<int64_t*>(gmax + std::max<int64_t>(nb->n_seg, 1));
  ProfRegion pr("config_gamma_max", s);
  if (nb->n_seg > 0) {
    k_seg_gamma_max<<<static_cast<unsigned>(nb->n_seg), 256, 0, s>>>(nb->seg.as<int64_t>(), gamma, gmax, amax);
    ProfRegion::launched();
  }
  k_cfg_gamma_max<<<blocks(nb->n_cfg, 128), 128, 0, s>>>(nb->seg.as<int64_t>(), nb->n_seg, gmax, amax, nb->n_cfg,
                                                        gamma_cfg, worst);
  ProfRegion::launched();
  MTP_CUDA(cudaGetLastError());
}

void run_classify(const double* gamma, int64_t n, double g_save, double g_break, int32_t* cls, cudaStream_t s) {
  if (n == 0) return;
  k_classify<<<blocks(n, 256), 256, 0, s>>>(gamma, n, g_save, g_break, cls);
  ProfRegion::launched();
  MTP_CUDA(cudaGetLastError());
}

void run_energy_vjp(const mtp_nbr* nb, const double* R, const double* gE, int64_t m, const double* F, double* g_pos,
                    double* g_theta, cudaStream_t s) {
  ProfRegion pr("energy_vjp", s);
  if (g_theta && m > 0) {
    k_vjp_theta<<<blocks(m, 128), 128, 0, s>>>(R, gE, static_cast<int>(nb->n_cfg), m, g_theta);
    ProfRegion::launched();
  }
  if (g_pos && nb->n_atoms > 0) {
    k_vjp_pos<<<blocks(nb->n_atoms, 256), 256, 0, s>>>(F, gE, nb->dn.atom_cfg, nb->n_atoms, g_pos);
    ProfRegion::launched();
  }
  MTP_CUDA(cudaGetLastError());
}

void run_widen_argmax(const int32_t* in, int64_t n, int64_t* out, cudaStream_t s) {
  if (n == 0) return;
  k_widen_argmax<<<blocks(n, 256), 256, 0, s>>>(in, n, out);
  ProfRegion::launched();
  MTP_CUDA(cudaGetLastError());
}

}  // namespace mtp

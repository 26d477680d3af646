// Active-set inverse (FP64 LU with partial pivoting) and the SIMT grade product.
//
// Sections II.C-D: the grade of neighborhood i is gamma_i = max_p |(b_i A^-1)_p| for the
// active-set matrix A (rows = parameter rows of the active neighborhoods).  A^-1 is formed
// once per active set: right-looking LU with partial pivoting, P A = L U, then the columns of
// A^-1 by forward and back substitution, one column per thread (coalesced row-major writes).
// The grade product C = B A^-1 is fused with its row epilogue (max |C_ip| and the lowest p
// attaining it), so C is never written.  This SIMT kernel serves the FP64 path; the mixed
// path uses the tensor-core kernel in grade_tc.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "mtp_internal.h"
#include "profiler.h"

namespace mtp {
namespace {

__global__ void k_maxabs(const double* A, int64_t n, double* out) {
  __shared__ double red[1024];
  double v = 0.0;
  for (int64_t k = threadIdx.x; k < n; k += blockDim.x) v = fmax(v, fabs(A[k]));
  red[threadIdx.x] = v;
  __syncthreads();
  for (int w = blockDim.x / 2; w; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = red[0];
}

// pivot search in column k, row swap, singularity flag
__global__ void k_pivot(double* LU, int64_t m, int64_t k, int* piv, const double* maxabs, unsigned* flag) {
  __shared__ double bv[1024];
  __shared__ int64_t bi[1024];
  double best = -1.0;
  int64_t bidx = k;
  for (int64_t r = k + threadIdx.x; r < m; r += blockDim.x) {
    const double v = fabs(LU[r * m + k]);
    if (v > best) { best = v; bidx = r; }
  }
  bv[threadIdx.x] = best;
  bi[threadIdx.x] = bidx;
  __syncthreads();
  for (int w = blockDim.x / 2; w; w >>= 1) {
    if (threadIdx.x < w) {
      const double o = bv[threadIdx.x + w];
      const int64_t oi = bi[threadIdx.x + w];
      if (o > bv[threadIdx.x] || (o == bv[threadIdx.x] && oi < bi[threadIdx.x])) { bv[threadIdx.x] = o; bi[threadIdx.x] = oi; }
    }
    __syncthreads();
  }
  const int64_t p = bi[0];
  if (threadIdx.x == 0) {
    piv[k] = static_cast<int>(p);
    if (!(bv[0] > 1e-13 * maxabs[0])) atomicOr(flag, 1u);
  }
  if (p != k)
    for (int64_t c = threadIdx.x; c < m; c += blockDim.x) {
      const double t = LU[k * m + c];
      LU[k * m + c] = LU[p * m + c];
      LU[p * m + c] = t;
    }
}

__global__ void k_lcol(double* LU, int64_t m, int64_t k) {
  const int64_t r = k + 1 + blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (r >= m) return;
  const double d = LU[k * m + k];
  LU[r * m + k] = d != 0.0 ? LU[r * m + k] / d : 0.0;
}

__global__ void k_trail(double* LU, int64_t m, int64_t k) {
  const int64_t c = k + 1 + blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  const int64_t r = k + 1 + blockIdx.y;
  if (c >= m || r >= m) return;
  LU[r * m + c] -= LU[r * m + k] * LU[k * m + c];
}

// column c of A^-1: solve L U x = P e_c
__global__ void k_inverse_cols(const double* LU, const int* piv, int64_t m, double* X) {
  const int64_t c = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (c >= m) return;
  // y = P e_c : apply the row swaps in order to the unit vector
  int64_t pos = c;  // position of the 1 after the swaps
  for (int64_t k = 0; k < m; ++k) {
    const int64_t p = piv[k];
    if (pos == k) pos = p;
    else if (pos == p) pos = k;
  }
  for (int64_t r = 0; r < m; ++r) {
    double v = (r == pos) ? 1.0 : 0.0;
    for (int64_t k = 0; k < r; ++k) v -= LU[r * m + k] * X[k * m + c];
    X[r * m + c] = v;
  }
  for (int64_t r = m - 1; r >= 0; --r) {
    double v = X[r * m + c];
    for (int64_t k = r + 1; k < m; ++k) v -= LU[r * m + k] * X[k * m + c];
    X[r * m + c] = v / LU[r * m + r];
  }
}

// Split A^-1 into TF32 pieces hi + lo (each rounded to nearest TF32), transposed to K-major
// [n][k] and zero-padded to ld x ld: the B operand of the tensor-core grade.
__global__ void k_split_ainv(const double* X, int64_t m, int64_t ld, float* hi, float* lo) {
  const int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (idx >= ld * ld) return;
  const int64_t n = idx / ld, k = idx % ld;   // output row n (= column of A^-1), col k
  const double v = (n < m && k < m) ? X[k * m + n] : 0.0;
  const float h = tf32_rn(static_cast<float>(v));
  hi[idx] = h;
  lo[idx] = tf32_rn(static_cast<float>(v - static_cast<double>(h)));
}

// Grade product with fused row epilogue.  Block: 256 threads, 64 rows; column tiles of 64;
// K steps of 16; each thread owns a 4 x 4 micro-tile.
template <class T>
__global__ void __launch_bounds__(256) k_grade_simt(const T* B, int64_t ldb, const T* X, int64_t m, int64_t N,
                                                     double* gamma, int32_t* argmax) {
  __shared__ T sB[16][64 + 1];
  __shared__ T sX[16][64 + 1];
  __shared__ double rowmax[64];
  __shared__ int rowarg[64];
  __shared__ double tmax[16][64];
  __shared__ int targ[16][64];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int64_t row0 = static_cast<int64_t>(blockIdx.x) * 64;
  if (threadIdx.x < 64) { rowmax[threadIdx.x] = -1.0; rowarg[threadIdx.x] = 0; }
  for (int64_t col0 = 0; col0 < m; col0 += 64) {
    T acc[4][4];
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
    for (int64_t k0 = 0; k0 < m; k0 += 16) {
      for (int e = threadIdx.x; e < 16 * 64; e += 256) {
        const int kk = e / 64, rr = e % 64;
        const int64_t gr = row0 + rr, gk = k0 + kk;
        sB[kk][rr] = (gr < N && gk < m) ? B[gr * ldb + gk] : T(0);
        const int64_t gc = col0 + rr;
        sX[kk][rr] = (gk < m && gc < m) ? X[gk * m + gc] : T(0);
      }
      __syncthreads();
      for (int kk = 0; kk < 16; ++kk) {
        T bv[4], xv[4];
        for (int a = 0; a < 4; ++a) bv[a] = sB[kk][ty * 4 + a];
        for (int b = 0; b < 4; ++b) xv[b] = sX[kk][tx * 4 + b];
        for (int a = 0; a < 4; ++a)
          for (int b = 0; b < 4; ++b) acc[a][b] += bv[a] * xv[b];
      }
      __syncthreads();
    }
    for (int a = 0; a < 4; ++a) {
      double best = -1.0;
      int barg = 0;
      for (int b = 0; b < 4; ++b) {
        const int64_t gc = col0 + tx * 4 + b;
        const double v = fabs(static_cast<double>(acc[a][b]));
        if (gc < m && v > best) { best = v; barg = static_cast<int>(gc); }
      }
      tmax[tx][ty * 4 + a] = best;
      targ[tx][ty * 4 + a] = barg;
    }
    __syncthreads();
    if (threadIdx.x < 64) {
      double best = rowmax[threadIdx.x];
      int barg = rowarg[threadIdx.x];
      for (int t = 0; t < 16; ++t) {
        const double v = tmax[t][threadIdx.x];
        const int g = targ[t][threadIdx.x];
        if (v > best || (v == best && g < barg)) { best = v; barg = g; }
      }
      rowmax[threadIdx.x] = best;
      rowarg[threadIdx.x] = barg;
    }
    __syncthreads();
  }
  if (threadIdx.x < 64) {
    const int64_t gr = row0 + threadIdx.x;
    if (gr < N) {
      gamma[gr] = rowmax[threadIdx.x];
      if (argmax) argmax[gr] = rowarg[threadIdx.x];
    }
  }
}

__global__ void k_to_float(const double* X, int64_t n, float* Y) {
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i < n) Y[i] = static_cast<float>(X[i]);
}

}  // namespace

void run_lu_inverse(mtp_model* md, const double* A, int64_t m, cudaStream_t s) {
  DevBuf work;
  work.ensure(m * m * sizeof(double) + m * sizeof(int) + 64, s);
  double* LU = work.as<double>();
  int* piv = reinterpret_cast<int*>(LU + m * m);
  md->err_flag.ensure(sizeof(unsigned), s);
  md->ws_misc.ensure(sizeof(double), s);
  MTP_CUDA(cudaMemsetAsync(md->err_flag.p, 0, sizeof(unsigned), s));
  MTP_CUDA(cudaMemcpyAsync(LU, A, m * m * sizeof(double), cudaMemcpyDeviceToDevice, s));
  ProfRegion pr("active_set_lu_inverse", s);
  k_maxabs<<<1, 1024, 0, s>>>(A, m * m, md->ws_misc.as<double>());
  ProfRegion::launched();
  for (int64_t k = 0; k < m; ++k) {
    k_pivot<<<1, 1024, 0, s>>>(LU, m, k, piv, md->ws_misc.as<double>(), md->err_flag.as<unsigned>());
    ProfRegion::launched();
    const int64_t rem = m - k - 1;
    if (rem > 0) {
      k_lcol<<<static_cast<unsigned>((rem + 255) / 256), 256, 0, s>>>(LU, m, k);
      ProfRegion::launched();
      dim3 g(static_cast<unsigned>((rem + 127) / 128), static_cast<unsigned>(rem));
      k_trail<<<g, 128, 0, s>>>(LU, m, k);
      ProfRegion::launched();
    }
  }
  MTP_CUDA(cudaGetLastError());
  md->ainv_d.ensure(m * m * sizeof(double), s);
  k_inverse_cols<<<static_cast<unsigned>((m + 63) / 64), 64, 0, s>>>(LU, piv, m, md->ainv_d.as<double>());
  ProfRegion::launched();
  MTP_CUDA(cudaGetLastError());
  // mixed-path copies: K-major padded split (tensor cores) and plain FP32 (SIMT)
  const int64_t ld = grade_tc_ld(m);
  md->ainv_ld = ld;
  md->ainv_f.ensure((2 * ld * ld + m * m) * sizeof(float), s);
  float* hi = md->ainv_f.as<float>();
  k_split_ainv<<<static_cast<unsigned>((ld * ld + 255) / 256), 256, 0, s>>>(md->ainv_d.as<double>(), m, ld, hi, hi + ld * ld);
  ProfRegion::launched();
  k_to_float<<<static_cast<unsigned>((m * m + 255) / 256), 256, 0, s>>>(md->ainv_d.as<double>(), m * m, hi + 2 * ld * ld);
  ProfRegion::launched();
  MTP_CUDA(cudaGetLastError());
  unsigned flag = 0;
  MTP_CUDA(cudaMemcpyAsync(&flag, md->err_flag.p, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  MTP_CUDA(cudaStreamSynchronize(s));
  work.release();
  if (flag) throw Fail{MTP_ERR_SINGULAR, "active-set matrix is singular (LU pivot below 1e-13 max|A|)"};
  md->m_active = m;
  md->have_ainv = true;
}

void run_grade_simt(mtp_model* md, int64_t N, bool fp64, const double* rows, const float* rows_f, int64_t ld,
                    double* gamma, int32_t* argmax, cudaStream_t s) {
  const int64_t m = md->m_active;
  const unsigned g = static_cast<unsigned>((N + 63) / 64);
  if (N == 0) return;
  ProfRegion pr(fp64 ? "grade_simt_fp64" : "grade_simt_fp32", s);
  if (fp64) {
    k_grade_simt<double><<<g, 256, 0, s>>>(rows, ld, md->ainv_d.as<double>(), m, N, gamma, argmax);
    ProfRegion::launched();
  } else {
    k_grade_simt<float><<<g, 256, 0, s>>>(rows_f, ld, md->ainv_f.as<float>() + 2 * md->ainv_ld * md->ainv_ld, m, N,
                                               gamma, argmax);
    ProfRegion::launched();
  }
  MTP_CUDA(cudaGetLastError());
}

}  // namespace mtp

// MaxVol update of the active set (Section II.D, D-optimality), FP64 on the GPU.
//
// The active set is the m x m matrix A of maximal |det A|.  For candidate rows B (n x m),
// C = B A^-1; replacing active row j by candidate row i multiplies |det A| by |C_ij|.  While the
// largest |C_ij| exceeds 1 + eps the swap is made and C and A^-1 follow by rank-one corrections
// (Sherman-Morrison):
//   u = (C_i. - e_j) / C_ij,   C <- C - C_.j u,   A^-1 <- A^-1 - (A^-1)_.j u,   A_j. <- B_i.
// (row i of C becomes e_j, so a candidate enters at most once; the row swapped out is dropped).
// At the end A^-1 is formed afresh from the final A by LU, which also refreshes the split copies
// used by the mixed-precision grade.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "mtp_internal.h"
#include "profiler.h"

namespace mtp {

void run_lu_inverse(mtp_model* md, const double* A, int64_t m, cudaStream_t s);

namespace {

constexpr int GT = 32;   // GEMM tile (rows, columns and k)
constexpr int GR = 8;    // thread rows per tile (each thread computes GT / GR outputs)

// C[n x m] = B[n x m] X[m x m] (row-major, FP64)
__global__ void __launch_bounds__(GT * GR) k_gemm(const double* __restrict__ B, const double* __restrict__ X,
                                                  double* __restrict__ C, int64_t n, int m) {
  __shared__ double sB[GT][GT + 1];
  __shared__ double sX[GT][GT + 1];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int col = blockIdx.x * GT + tx;
  const int64_t row_tiles = (n + GT - 1) / GT;
  for (int64_t rt = blockIdx.y; rt < row_tiles; rt += gridDim.y) {
    const int64_t row0 = rt * GT;
    double acc[GT / GR];
#pragma unroll
    for (int q = 0; q < GT / GR; ++q) acc[q] = 0.0;
    for (int k0 = 0; k0 < m; k0 += GT) {
      for (int r = ty; r < GT; r += GR) {
        const int64_t gr = row0 + r;
        const int gk = k0 + tx;
        sB[r][tx] = (gr < n && gk < m) ? B[gr * m + gk] : 0.0;
        const int xr = k0 + r;
        sX[r][tx] = (xr < m && col < m) ? X[static_cast<int64_t>(xr) * m + col] : 0.0;
      }
      __syncthreads();
#pragma unroll 8
      for (int k = 0; k < GT; ++k) {
        const double x = sX[k][tx];
#pragma unroll
        for (int q = 0; q < GT / GR; ++q) acc[q] = fma(sB[ty + GR * q][k], x, acc[q]);
      }
      __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < GT / GR; ++q) {
      const int64_t gr = row0 + ty + GR * q;
      if (gr < n && col < m) C[gr * m + col] = acc[q];
    }
  }
}

struct Best {
  double v;
  long long idx;
};

__device__ __forceinline__ Best better(Best a, Best b) {
  return (b.v > a.v || (b.v == a.v && b.idx < a.idx)) ? b : a;
}

__device__ Best block_best(Best b) {
  __shared__ Best sh[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int o = 16; o; o >>= 1) {
    Best t;
    t.v = __shfl_xor_sync(0xffffffffu, b.v, o);
    t.idx = __shfl_xor_sync(0xffffffffu, b.idx, o);
    b = better(b, t);
  }
  if (lane == 0) sh[w] = b;
  __syncthreads();
  if (w == 0) {
    b = lane < static_cast<int>(blockDim.x >> 5) ? sh[lane] : Best{-1.0, 0x7fffffffffffffffLL};
    for (int o = 16; o; o >>= 1) {
      Best t;
      t.v = __shfl_xor_sync(0xffffffffu, b.v, o);
      t.idx = __shfl_xor_sync(0xffffffffu, b.idx, o);
      b = better(b, t);
    }
  }
  return b;
}

// largest |C| and its lowest flat (row-major) index: per-block partials, then one block
__global__ void k_argmax_part(const double* __restrict__ C, long long total, Best* part) {
  Best b{-1.0, 0x7fffffffffffffffLL};
  for (long long t = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; t < total;
       t += static_cast<long long>(gridDim.x) * blockDim.x) {
    const double v = fabs(C[t]);
    if (v > b.v) b = Best{v, t};   // grid-stride order is ascending per thread: keeps the lowest index
  }
  b = block_best(b);
  if (threadIdx.x == 0) part[blockIdx.x] = b;
}

__global__ void k_argmax_final(const Best* part, int n_part, Best* out) {
  Best b{-1.0, 0x7fffffffffffffffLL};
  for (int t = threadIdx.x; t < n_part; t += blockDim.x) b = better(b, part[t]);
  b = block_best(b);
  if (threadIdx.x == 0) *out = b;
}

// u = (C_i. - e_j) / C_ij, v = C_.j, w = (A^-1)_.j, then A_j. = B_i.
__global__ void k_swap_vectors(const double* __restrict__ C, const double* __restrict__ Ainv,
                               const double* __restrict__ B, double* __restrict__ A, int64_t n, int m, int64_t i,
                               int j, double* u, double* v, double* w) {
  const double cij = C[i * m + j];
  for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < std::max<int64_t>(n, m);
       t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    if (t < m) {
      u[t] = (C[i * m + t] - (t == j ? 1.0 : 0.0)) / cij;
      w[t] = Ainv[t * m + j];
      A[static_cast<int64_t>(j) * m + t] = B[i * m + t];
    }
    if (t < n) v[t] = C[t * m + j];
  }
}

// M[r][c] -= left[r] * right[c]
__global__ void k_rank1(double* __restrict__ M, int64_t rows, int m, const double* __restrict__ left,
                        const double* __restrict__ right) {
  const long long total = rows * static_cast<long long>(m);
  for (long long t = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; t < total;
       t += static_cast<long long>(gridDim.x) * blockDim.x) {
    const long long r = t / m;
    const int c = static_cast<int>(t - r * m);
    M[t] = fma(-left[r], right[c], M[t]);
  }
}

}  // namespace

int64_t run_maxvol(mtp_model* md, const double* B, int64_t n, double eps, int64_t max_swaps, int64_t* source,
                   cudaStream_t s) {
  const int64_t m = md->m_active;
  std::vector<int64_t> src(static_cast<size_t>(m), -1);
  int64_t swaps = 0;
  if (n > 0) {
    int dev = 0, nsm = 0;
    MTP_CUDA(cudaGetDevice(&dev));
    MTP_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const int n_part = nsm * 4;
    DevBuf work;
    const size_t cbytes = static_cast<size_t>(n) * m * sizeof(double);
    work.ensure(cbytes + (n + 2 * m) * sizeof(double) + (n_part + 1) * sizeof(Best) + 256, s);
    double* C = work.as<double>();
    double* v = C + n * m;
    double* u = v + n;
    double* w = u + m;
    Best* part = reinterpret_cast<Best*>(w + m);
    Best* best_d = part + n_part;
    ProfRegion pr("active_set_maxvol", s);
    {
      const dim3 blk(GT, GR);
      const dim3 grd(static_cast<unsigned>((m + GT - 1) / GT),
                     static_cast<unsigned>(std::min<int64_t>((n + GT - 1) / GT, 65535)));
      k_gemm<<<grd, blk, 0, s>>>(B, md->ainv_d.as<double>(), C, n, static_cast<int>(m));
      ProfRegion::launched();
      MTP_CUDA(cudaGetLastError());
    }
    const long long total = static_cast<long long>(n) * m;
    const unsigned g_nm = static_cast<unsigned>(std::min<long long>((total + 255) / 256, nsm * 16LL));
    const unsigned g_mm = static_cast<unsigned>(std::min<long long>((m * m + 255) / 256, nsm * 16LL));
    const unsigned g_v = static_cast<unsigned>(std::min<long long>((std::max(n, m) + 255) / 256, nsm * 4LL));
    Best best{};
    while (swaps < max_swaps) {
      k_argmax_part<<<n_part, 256, 0, s>>>(C, total, part);
      ProfRegion::launched();
      k_argmax_final<<<1, 1024, 0, s>>>(part, n_part, best_d);
      ProfRegion::launched();
      MTP_CUDA(cudaGetLastError());
      MTP_CUDA(cudaMemcpyAsync(&best, best_d, sizeof(Best), cudaMemcpyDeviceToHost, s));
      MTP_CUDA(cudaStreamSynchronize(s));
      if (!(best.v > 1.0 + eps)) break;
      const int64_t i = best.idx / m;
      const int j = static_cast<int>(best.idx - i * m);
      k_swap_vectors<<<g_v, 256, 0, s>>>(C, md->ainv_d.as<double>(), B, md->a_d.as<double>(), n, static_cast<int>(m),
                                         i, j, u, v, w);
      ProfRegion::launched();
      k_rank1<<<g_nm, 256, 0, s>>>(C, n, static_cast<int>(m), v, u);
      ProfRegion::launched();
      k_rank1<<<g_mm, 256, 0, s>>>(md->ainv_d.as<double>(), m, static_cast<int>(m), w, u);
      ProfRegion::launched();
      MTP_CUDA(cudaGetLastError());
      src[static_cast<size_t>(j)] = i;
      ++swaps;
    }
    MTP_CUDA(cudaStreamSynchronize(s));
    work.release();
  }
  if (source) {
    MTP_CUDA(cudaMemcpyAsync(source, src.data(), m * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    MTP_CUDA(cudaStreamSynchronize(s));
  }
  if (swaps > 0) run_lu_inverse(md, md->a_d.as<double>(), m, s);
  return swaps;
}

}  // namespace mtp

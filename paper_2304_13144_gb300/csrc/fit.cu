// BFGS fit of the parameters (Section II.B, eq. 7) and the fitting-error report.
//
// The loss and its gradient come from mtp_train_step (GPU); the driver is host code: the
// parameters are scaled, u = theta / D with D_p = max(|theta0_p|, 1e-12 max|theta0|) (they span
// many orders of magnitude); textbook BFGS on u with the inverse-Hessian update
//   H <- (I - r s y^T) H (I - r y s^T) + r s s^T,  r = 1 / s.y   (skipped when s.y <= 0),
// H = I rescaled to (s.y / y.y) I just before the first update; a backtracking Armijo line
// search (step 1, halved up to 40 times, L(u + t d) <= L(u) + 1e-4 t g.d); stop when
// max|g_u| <= gtol max(1, |L|), after max_iter accepted steps, or when no step is accepted.
//
// Errors: energy per atom |E_k - E*_k| / N_k (max, mean, RMS over configurations), force
// |F_i - F*_i| (max, mean, RMS over atoms; per-block partials on the GPU summed in order on
// the host), virial |W_ab - W*_ab| (max, mean, RMS over configurations and components).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "mtp_internal.h"
#include "profiler.h"

extern "C" mtp_status mtp_set_params(mtp_model* model, const double* theta, int64_t m);
extern "C" mtp_status mtp_train_step(mtp_model* model, const mtp_batch* batch, const mtp_nbr* nbr, mtp_precision prec,
                                     const double* E_ref, const double* F_ref, const double* W_ref, double w_e,
                                     double w_f, double w_s, double* loss, double* grad, void* stream);
extern "C" mtp_status mtp_energy_forces_stress(mtp_model* model, const mtp_batch* batch, const mtp_nbr* nbr,
                                               mtp_precision prec, double* energy, double* site_energy,
                                               double* forces, double* virial, void* stream);

namespace mtp {
namespace {

constexpr int kErrBlocks = 256;

// per block: max |dF_i|, sum |dF_i|, sum |dF_i|^2 over a contiguous range of atoms
__global__ void k_force_err(const double* __restrict__ F, const double* __restrict__ Fr, int64_t n, double* part) {
  const int64_t per = (n + gridDim.x - 1) / gridDim.x;
  const int64_t a0 = blockIdx.x * per, a1 = std::min<int64_t>(n, a0 + per);
  double mx = 0.0, s1 = 0.0, s2 = 0.0;
  for (int64_t a = a0 + threadIdx.x; a < a1; a += blockDim.x) {
    const double dx = F[3 * a] - Fr[3 * a], dy = F[3 * a + 1] - Fr[3 * a + 1], dz = F[3 * a + 2] - Fr[3 * a + 2];
    const double q = dx * dx + dy * dy + dz * dz;
    const double d = sqrt(q);
    mx = fmax(mx, d);
    s1 += d;
    s2 += q;
  }
  __shared__ double r[3][256];
  r[0][threadIdx.x] = mx;
  r[1][threadIdx.x] = s1;
  r[2][threadIdx.x] = s2;
  __syncthreads();
  for (int w = blockDim.x / 2; w; w >>= 1) {
    if (threadIdx.x < w) {
      r[0][threadIdx.x] = fmax(r[0][threadIdx.x], r[0][threadIdx.x + w]);
      r[1][threadIdx.x] += r[1][threadIdx.x + w];
      r[2][threadIdx.x] += r[2][threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[3 * blockIdx.x] = r[0][0];
    part[3 * blockIdx.x + 1] = r[1][0];
    part[3 * blockIdx.x + 2] = r[2][0];
  }
}

void check(mtp_status st) {
  if (st != MTP_OK) throw Fail{st, mtp_last_error()};
}

}  // namespace
}  // namespace mtp

using namespace mtp;

extern "C" mtp_status mtp_fit_bfgs(mtp_model* md, const mtp_batch* b, const mtp_nbr* nb, mtp_precision prec,
                                   const double* E_ref, const double* F_ref, const double* W_ref, double w_e,
                                   double w_f, double w_s, int64_t max_iter, double gtol, double* loss_out,
                                   int64_t* iters_out, void* stream) {
  try {
    if (!md || !b || !nb || !E_ref || !F_ref) throw Fail{MTP_ERR_ARG, "null argument"};
    if (max_iter < 0 || !(gtol >= 0.0)) throw Fail{MTP_ERR_ARG, "max_iter and gtol must be non-negative"};
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t m = md->sched.n_params;
    const std::vector<double> theta0 = md->theta;
    std::vector<double> D(m, 1.0);
    double top = 0.0;
    for (double v : theta0) top = std::max(top, std::fabs(v));
    if (top > 0.0)
      for (int64_t p = 0; p < m; ++p) D[p] = std::max(std::fabs(theta0[p]), 1e-12 * top);
    DevBuf dev;
    dev.ensure((m + 1) * sizeof(double), s);
    double* grad_d = dev.as<double>();
    double* loss_d = grad_d + m;
    std::vector<double> th(m), gh(m);
    // L(u) and dL/du at u
    auto eval = [&](const std::vector<double>& u, double& L, std::vector<double>& g) {
      for (int64_t p = 0; p < m; ++p) th[p] = D[p] * u[p];
      check(mtp_set_params(md, th.data(), m));
      check(mtp_train_step(md, b, nb, prec, E_ref, F_ref, W_ref, w_e, w_f, w_s, loss_d, grad_d, stream));
      MTP_CUDA(cudaMemcpyAsync(&L, loss_d, sizeof(double), cudaMemcpyDeviceToHost, s));
      MTP_CUDA(cudaMemcpyAsync(gh.data(), grad_d, m * sizeof(double), cudaMemcpyDeviceToHost, s));
      MTP_CUDA(cudaStreamSynchronize(s));
      g.resize(m);
      for (int64_t p = 0; p < m; ++p) g[p] = D[p] * gh[p];
    };
    std::vector<double> u(m), g, un(m), gn, d(m), sv(m), yv(m), Hy(m), H;
    for (int64_t p = 0; p < m; ++p) u[p] = theta0[p] / D[p];
    double L = 0.0, Ln = 0.0;
    eval(u, L, g);
    int64_t it = 0;
    bool have_h = false;
    while (it < max_iter) {
      double gmax = 0.0;
      for (double v : g) gmax = std::max(gmax, std::fabs(v));
      if (gmax <= gtol * std::max(1.0, std::fabs(L))) break;
      // d = -H g
      if (have_h) {
        for (int64_t p = 0; p < m; ++p) {
          double acc = 0.0;
          for (int64_t q = 0; q < m; ++q) acc += H[p * m + q] * g[q];
          d[p] = -acc;
        }
      } else {
        for (int64_t p = 0; p < m; ++p) d[p] = -g[p];
      }
      double gd = 0.0;
      for (int64_t p = 0; p < m; ++p) gd += g[p] * d[p];
      double t = 1.0;
      bool ok = false;
      for (int k = 0; k < 41; ++k) {
        for (int64_t p = 0; p < m; ++p) un[p] = u[p] + t * d[p];
        eval(un, Ln, gn);
        if (Ln <= L + 1e-4 * t * gd) { ok = true; break; }
        t *= 0.5;
      }
      if (!ok) break;
      double sy = 0.0, yy = 0.0;
      for (int64_t p = 0; p < m; ++p) {
        sv[p] = un[p] - u[p];
        yv[p] = gn[p] - g[p];
        sy += sv[p] * yv[p];
        yy += yv[p] * yv[p];
      }
      if (!have_h) {
        H.assign(static_cast<size_t>(m * m), 0.0);
        const double sc = sy > 0.0 ? sy / yy : 1.0;
        for (int64_t p = 0; p < m; ++p) H[p * m + p] = sc;
        have_h = true;
      }
      if (sy > 0.0) {
        // H <- (I - r s y^T) H (I - r y s^T) + r s s^T
        //    = H - r (s (H y)^T + (H y) s^T) + (r^2 y.Hy + r) s s^T   (H symmetric)
        const double r = 1.0 / sy;
        double yHy = 0.0;
        for (int64_t p = 0; p < m; ++p) {
          double acc = 0.0;
          for (int64_t q = 0; q < m; ++q) acc += H[p * m + q] * yv[q];
          Hy[p] = acc;
          yHy += yv[p] * acc;
        }
        const double c = r * r * yHy + r;
        for (int64_t p = 0; p < m; ++p)
          for (int64_t q = 0; q < m; ++q)
            H[p * m + q] += -r * (sv[p] * Hy[q] + Hy[p] * sv[q]) + c * sv[p] * sv[q];
      }
      u.swap(un);
      g.swap(gn);
      L = Ln;
      ++it;
    }
    // leave the model at the accepted parameters
    for (int64_t p = 0; p < m; ++p) th[p] = D[p] * u[p];
    check(mtp_set_params(md, th.data(), m));
    MTP_CUDA(cudaStreamSynchronize(s));
    if (loss_out) *loss_out = L;
    if (iters_out) *iters_out = it;
    return MTP_OK;
  } catch (const Fail& e) {
    set_error(e.msg);
    return e.st;
  } catch (const std::exception& e) {
    set_error(e.what());
    return MTP_ERR_CUDA;
  }
}

extern "C" mtp_status mtp_fit_errors(mtp_model* md, const mtp_batch* b, const mtp_nbr* nb, mtp_precision prec,
                                     const double* E_ref, const double* F_ref, const double* W_ref, double* report,
                                     void* stream) {
  try {
    if (!md || !b || !nb || !E_ref || !F_ref || !report) throw Fail{MTP_ERR_ARG, "null argument"};
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t N = nb->n_atoms, K = nb->n_cfg;
    DevBuf dev;
    dev.ensure((std::max<int64_t>(N, 1) * 3 + K * 10 + 2 * K * 9 + K + 3 * kErrBlocks) * sizeof(double), s);
    double* F = dev.as<double>();
    double* E = F + std::max<int64_t>(N, 1) * 3;
    double* W = E + K;
    double* part = W + 9 * K;
    double* Er = part + 3 * kErrBlocks;
    double* Wr = Er + K;
    check(mtp_energy_forces_stress(md, b, nb, prec, E, nullptr, F, W, stream));
    if (N > 0) {
      k_force_err<<<kErrBlocks, 256, 0, s>>>(F, F_ref, N, part);
      ProfRegion::launched();
      MTP_CUDA(cudaGetLastError());
    }
    MTP_CUDA(cudaMemcpyAsync(Er, E_ref, K * sizeof(double), cudaMemcpyDeviceToDevice, s));
    if (W_ref) MTP_CUDA(cudaMemcpyAsync(Wr, W_ref, 9 * K * sizeof(double), cudaMemcpyDeviceToDevice, s));
    std::vector<double> hE(K), hEr(K), hW(9 * K), hWr(9 * K), hp(3 * kErrBlocks, 0.0);
    MTP_CUDA(cudaMemcpyAsync(hE.data(), E, K * sizeof(double), cudaMemcpyDeviceToHost, s));
    MTP_CUDA(cudaMemcpyAsync(hEr.data(), Er, K * sizeof(double), cudaMemcpyDeviceToHost, s));
    MTP_CUDA(cudaMemcpyAsync(hW.data(), W, 9 * K * sizeof(double), cudaMemcpyDeviceToHost, s));
    if (W_ref) MTP_CUDA(cudaMemcpyAsync(hWr.data(), Wr, 9 * K * sizeof(double), cudaMemcpyDeviceToHost, s));
    if (N > 0) MTP_CUDA(cudaMemcpyAsync(hp.data(), part, 3 * kErrBlocks * sizeof(double), cudaMemcpyDeviceToHost, s));
    MTP_CUDA(cudaStreamSynchronize(s));
    double emx = 0, es1 = 0, es2 = 0;
    for (int64_t k = 0; k < K; ++k) {
      const double n = static_cast<double>(std::max<int64_t>(nb->atom_offset[k + 1] - nb->atom_offset[k], 1));
      const double e = std::fabs(hE[k] - hEr[k]) / n;
      emx = std::max(emx, e);
      es1 += e;
      es2 += e * e;
    }
    double fmx = 0, fs1 = 0, fs2 = 0;
    for (int q = 0; q < kErrBlocks; ++q) {
      fmx = std::max(fmx, hp[3 * q]);
      fs1 += hp[3 * q + 1];
      fs2 += hp[3 * q + 2];
    }
    double wmx = 0, ws1 = 0, ws2 = 0;
    if (W_ref)
      for (int64_t q = 0; q < 9 * K; ++q) {
        const double w = std::fabs(hW[q] - hWr[q]);
        wmx = std::max(wmx, w);
        ws1 += w;
        ws2 += w * w;
      }
    const double nk = K > 0 ? static_cast<double>(K) : 1.0, na = N > 0 ? static_cast<double>(N) : 1.0;
    const double out[9] = {emx, es1 / nk, std::sqrt(es2 / nk), fmx, fs1 / na, std::sqrt(fs2 / na),
                           wmx, ws1 / (9 * nk), std::sqrt(ws2 / (9 * nk))};
    std::copy(out, out + 9, report);
    return MTP_OK;
  } catch (const Fail& e) {
    set_error(e.msg);
    return e.st;
  } catch (const std::exception& e) {
    set_error(e.what());
    return MTP_ERR_CUDA;
  }
}

// Arithmetic peaks of the current GPU, measured by the library's own microbenchmarks: the
// denominators of the roofline fractions of the per-neighborhood kernel (FP32 FMA, FP64 FMA)
// and of the tensor-core grade (TF32 tcgen05.mma).  The paper has no counterpart.
//
//   FFMA / DFMA: every thread runs 8 independent multiply-add chains (enough independent work to
//     cover the pipeline latency at full occupancy); 2 flops per FMA.
//   TF32: one CTA per SM, one thread issues tcgen05.mma.kind::tf32 (M 128, N 256, K 8) on fixed
//     operand tiles in shared memory, accumulating into tensor memory; 2 M N K flops per MMA.
//     The operands never change, so this is the issue-rate ceiling of the tensor pipe for that
//     shape (no operand traffic).  Its one wait (all MMAs done) is bounded.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "mtp_internal.h"

namespace mtp {
namespace {

template <class T>
__global__ void __launch_bounds__(512) k_fma_peak(T* sink, int iters, T mul, T add) {
  T a[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) a[j] = static_cast<T>(threadIdx.x + j) * static_cast<T>(1e-3);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = a[j] * mul + add;   // contracted to one FMA
  }
  T s = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) s += a[j];
  if (s == static_cast<T>(-1.2345)) sink[0] = s;   // keeps the chains live; never true here
}

constexpr int TM = 128, TN = 256, TK = 32;   // operand tiles: 128 x 32 and 256 x 32 FP32, 128-byte swizzle
constexpr uint32_t kWaitLimit = 1u << 24;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t sw128_desc(const void* p) {
  const uint64_t addr = smem_u32(p);
  uint64_t d = 0;
  d |= (addr >> 4) & 0x3FFFull;
  d |= 1ull << 16;
  d |= (1024ull >> 4) << 32;
  d |= 1ull << 46;
  d |= 2ull << 61;
  return d;
}

__global__ void __launch_bounds__(128, 1) k_tf32_peak(int iters, unsigned* err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  float* A = reinterpret_cast<float*>(smem);
  float* B = A + TM * TK;
  uint64_t* bar = reinterpret_cast<uint64_t*>(B + TN * TK);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 1);
  for (int k = threadIdx.x; k < (TM + TN) * TK; k += blockDim.x)
    A[k] = __uint_as_float((0x3F800000u + (static_cast<uint32_t>(k) * 2654435761u >> 9)) & 0xffffe000u);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic-proxy stores -> MMA reads
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)), "r"(TN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  if (threadIdx.x == 0) {
    const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | (static_cast<uint32_t>(TN >> 3) << 17) |
                           (static_cast<uint32_t>(TM >> 4) << 24);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int ks = 0; ks < TK / 8; ++ks) {
        const uint64_t ad = sw128_desc(reinterpret_cast<unsigned char*>(A) + ks * 32);
        const uint64_t bd = sw128_desc(reinterpret_cast<unsigned char*>(B) + ks * 32);
        const uint32_t acc = (it > 0 || ks > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
            ::"r"(tmem), "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
      }
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
    bool done = false;
    for (uint32_t t = 0; t < kWaitLimit && !done; ++t) {
      uint32_t ok;
      asm volatile(
          "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
          : "=r"(ok)
          : "r"(smem_u32(bar)), "r"(0)
          : "memory");
      done = ok != 0;
      if (!done && t > 64) __nanosleep(256);
    }
    if (!done) atomicOr(err, 1u);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TN));
  }
}

}  // namespace
}  // namespace mtp

using namespace mtp;

extern "C" mtp_status mtp_measure_peak(int kind, double* tflops, double* ms, void* stream) {
  try {
    if (!tflops || kind < 0 || kind > 2) throw Fail{MTP_ERR_ARG, "kind must be 0 (FP32 FMA), 1 (FP64 FMA) or 2 (TF32 MMA)"};
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0, nsm = 0;
    MTP_CUDA(cudaGetDevice(&dev));
    MTP_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    DevBuf buf;
    buf.ensure(64, s);
    MTP_CUDA(cudaMemsetAsync(buf.p, 0, 64, s));
    cudaEvent_t e0, e1;
    MTP_CUDA(cudaEventCreate(&e0));
    MTP_CUDA(cudaEventCreate(&e1));
    double flops = 0.0;
    float best = 0.f;
    // operand tiles + barrier + alignment slack, padded so that one CTA fills an SM's shared memory
    const size_t tc_smem = std::max<size_t>((TM + TN) * TK * sizeof(float) + 64 + 1024, 160 * 1024);
    if (kind == 2) {
      MTP_CUDA(cudaFuncSetAttribute(k_tf32_peak, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(tc_smem)));
    }
    for (int rep = 0; rep < 4; ++rep) {   // the first run warms up; the best of the others is kept
      MTP_CUDA(cudaEventRecord(e0, s));
      if (kind == 0) {
        const int iters = 1 << 16, threads = 512, grid = nsm * 4;
        k_fma_peak<float><<<grid, threads, 0, s>>>(buf.as<float>(), iters, 0.999999f, 1e-6f);
        flops = 2.0 * 8 * iters * static_cast<double>(threads) * grid;
      } else if (kind == 1) {
        const int iters = 1 << 12, threads = 512, grid = nsm * 4;
        k_fma_peak<double><<<grid, threads, 0, s>>>(buf.as<double>(), iters, 0.999999, 1e-6);
        flops = 2.0 * 8 * iters * static_cast<double>(threads) * grid;
      } else {
        const int iters = 8192;
        k_tf32_peak<<<nsm, 128, tc_smem, s>>>(iters, buf.as<unsigned>());
        flops = 2.0 * TM * TN * TK * static_cast<double>(iters) * nsm;
      }
      MTP_CUDA(cudaGetLastError());
      MTP_CUDA(cudaEventRecord(e1, s));
      MTP_CUDA(cudaEventSynchronize(e1));
      float t = 0.f;
      MTP_CUDA(cudaEventElapsedTime(&t, e0, e1));
      if (rep == 1 || (rep > 1 && t < best)) best = t;
    }
    unsigned err = 0;
    if (kind == 2) MTP_CUDA(cudaMemcpy(&err, buf.p, sizeof(unsigned), cudaMemcpyDeviceToHost));
    MTP_CUDA(cudaEventDestroy(e0));
    MTP_CUDA(cudaEventDestroy(e1));
    MTP_CUDA(cudaStreamSynchronize(s));
    buf.release();
    if (err) throw Fail{MTP_ERR_TIMEOUT, "tensor-core peak: the completion wait expired"};
    *tflops = flops / (best * 1e-3) / 1e12;
    if (ms) *ms = best;
    return MTP_OK;
  } catch (const Fail& e) {
    set_error(e.msg);
    return e.st;
  } catch (...) {
    set_error("unknown error");
    return MTP_ERR_CUDA;
  }
}

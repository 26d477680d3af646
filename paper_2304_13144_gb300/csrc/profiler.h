// Kernel-level tracing regions (see profiler.cu).
#pragma once
#include <cuda_runtime.h>

namespace mtp {
// Records a CUDA event pair around the launches made during its lifetime, on stream s,
// when tracing is enabled (mtp_profiler_enable), and opens an NVTX range of the same name.
// launched() after each of the library's own kernel launches counts it in the innermost open
// region of the calling thread.
class ProfRegion {
 public:
  ProfRegion(const char* name, cudaStream_t s);
  ~ProfRegion();
  ProfRegion(const ProfRegion&) = delete;
  ProfRegion& operator=(const ProfRegion&) = delete;
  static void launched();

 private:
  const char* name_;
  cudaStream_t s_;
  cudaEvent_t a_ = nullptr, b_ = nullptr;
  int kernels_ = 0;
  ProfRegion* outer_ = nullptr;
};
}  // namespace mtp

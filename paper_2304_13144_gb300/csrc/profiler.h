// Kernel-level tracing regions (see profiler.cu).
#pragma once
#include <cuda_runtime.h>

namespace mtp {
// Records a CUDA event pair around the launches made during its lifetime, on stream s,
// when tracing is enabled (mtp_profiler_enable), and opens an NVTX range of the same name.
class ProfRegion {
 public:
  ProfRegion(const char* name, cudaStream_t s);
  ~ProfRegion();
  ProfRegion(const ProfRegion&) = delete;
  ProfRegion& operator=(const ProfRegion&) = delete;

 private:
  const char* name_;
  cudaStream_t s_;
  cudaEvent_t a_ = nullptr, b_ = nullptr;
};
}  // namespace mtp

// Energies, forces and virial without any device allocation.
//
// Some callers cannot allocate device memory when they call in: an MD engine or an inference
// server that owns the whole device-memory budget through its own pool allocator and does not
// allow foreign allocations, or a time-step loop where an allocation's implicit device
// synchronisation and its possible failure are not acceptable.  This entry point runs the same
// kernels as mtp_energy_forces_stress but keeps its scratch (per-pair gradients, per-atom
// energies and virials, per-segment partial sums) in one file-scope device array of fixed size
// instead of the model's workspace.  The array belongs to this file's device module: the CUDA
// runtime commits it on a device when the module is loaded there, which mtp_load forces (it
// looks up the array's device address with the model's device current), so the memory is taken
// when a model is created, not at the first call, and stays until the process exits.  A call on
// a device where no model was loaded since the last device reset looks the address up itself,
// so that first call should come before any stream capture.  All calls share the one array:
// calls whose work overlaps on the GPU (other streams, other threads) race on it and must be
// serialised by the caller.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <string>

#include "mtp_internal.h"
#include "profiler.h"

namespace mtp {

void run_config_sums_into(const mtp_nbr* nb, const double* V, const double* Wat, double* E, double* W, double* part,
                          cudaStream_t s);

namespace {

constexpr int64_t kMaxAtoms = 32768;
constexpr int64_t kMaxPairs = 524288;
constexpr int64_t kMaxSegments = 1024;
constexpr size_t kAlign = 256;
constexpr size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }
// gradients (FP64 at most) + site energies + per-atom virials + segment partials
constexpr size_t kScratchBytes = align_up(kMaxPairs * 3 * sizeof(double)) + align_up(kMaxAtoms * sizeof(double)) +
                                 align_up(kMaxAtoms * 9 * sizeof(double)) + align_up(kMaxSegments * 10 * sizeof(double));

static __device__ __align__(256) unsigned char g_efs_scratch[kScratchBytes];

std::mutex g_mu;
void* g_addr[256] = {nullptr};

// Device address of the scratch array on `device` (the current device); refresh = look it up
// again even if known (mtp_load does, so a model created after a device reset sees the array
// of the new context; models themselves do not survive a reset).
void* scratch_address(int device, bool refresh) {
  if (device < 0 || device >= 256) throw Fail{MTP_ERR_ARG, "device index out of range"};
  std::lock_guard<std::mutex> lk(g_mu);
  if (refresh || !g_addr[device]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_efs_scratch);
    if (e != cudaSuccess || !p)
      throw Fail{MTP_ERR_CUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e)};
    g_addr[device] = p;
  }
  return g_addr[device];
}

}  // namespace

// Called by mtp_load with the model's device current: loads this file's module on the device
// (committing the scratch array there) and records the array's address.
void noalloc_prepare(int device) { scratch_address(device, true); }

}  // namespace mtp

using namespace mtp;

extern "C" mtp_status mtp_energy_forces_stress_noalloc(mtp_model* md, const mtp_batch* b, const mtp_nbr* nb,
                                                       mtp_precision prec, double* energy, double* site_energy,
                                                       double* forces, double* virial, void* stream) {
  try {
    check_run(md, b, nb);
    if (prec != MTP_FP64 && prec != MTP_MIXED) throw Fail{MTP_ERR_ARG, "unknown precision"};
    if (!energy && !site_energy && !forces && !virial) throw Fail{MTP_ERR_ARG, "no output requested"};
    if (nb->n_atoms > kMaxAtoms || nb->n_pairs > kMaxPairs || nb->n_seg > kMaxSegments)
      throw Fail{MTP_ERR_CAPACITY, "the allocation-free path holds at most " + std::to_string(kMaxAtoms) + " atoms, " +
                                       std::to_string(kMaxPairs) + " pairs and " + std::to_string(kMaxSegments) +
                                       " configuration segments; this call has " + std::to_string(nb->n_atoms) +
                                       " atoms, " + std::to_string(nb->n_pairs) + " pairs and " +
                                       std::to_string(nb->n_seg) + " segments"};
    const bool fp64 = prec == MTP_FP64;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = -1;
    MTP_CUDA(cudaGetDevice(&dev));
    unsigned char* base = static_cast<unsigned char*>(scratch_address(dev, false));
    unsigned char* pG = base;
    double* pV = reinterpret_cast<double*>(base + align_up(kMaxPairs * 3 * sizeof(double)));
    double* pW = pV + align_up(kMaxAtoms * sizeof(double)) / sizeof(double);
    double* pPart = pW + align_up(kMaxAtoms * 9 * sizeof(double)) / sizeof(double);
    SiteOutputs o;
    o.V = site_energy ? site_energy : pV;
    o.Wat = pW;
    o.G = pG;
    // every entry of G, V and W is written by the kernels: nothing needs clearing
    run_sites(md, b, nb, fp64, o, false, nullptr, s);
    if (forces) run_forces(nb, fp64, o.G, forces, s);
    if (energy || virial) run_config_sums_into(nb, o.V, o.Wat, energy, virial, pPart, s);
    return MTP_OK;
  } catch (const Fail& e) {
    set_error(e.msg);
    return e.st;
  } catch (const std::exception& e) {
    set_error(e.what());
    return MTP_ERR_CUDA;
  } catch (...) {
    set_error("unknown error");
    return MTP_ERR_CUDA;
  }
}

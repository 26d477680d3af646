// Internal declarations shared by the CUDA translation units of the MTP library.
#pragma once

#include <cuda_runtime.h>

#include <atomic>

#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/mtp.h"
#include "schedule.h"

namespace mtp {

// ------------------------------------------------------------------------------------
// error reporting
// ------------------------------------------------------------------------------------
void set_error(const std::string& msg);
struct Fail {
  mtp_status st;
  std::string msg;
};
#define MTP_CUDA(call)                                                                    \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      throw ::mtp::Fail{MTP_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)}; \
  } while (0)

// device error flag bits
enum : unsigned { ERRF_GEOMETRY = 1u, ERRF_SPECIES = 2u, ERRF_CAPACITY = 4u, ERRF_NONFINITE = 8u,
                  ERRF_REVERSE = 16u, ERRF_REVPEND = 32u };

// ------------------------------------------------------------------------------------
// device buffer owned by a handle (stream-ordered allocation, grows only)
// ------------------------------------------------------------------------------------
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  void ensure(size_t need, cudaStream_t s);
  void release();
  template <class T> T* as() const { return static_cast<T*>(p); }
};

// ------------------------------------------------------------------------------------
// schedule and parameters on the device (one copy per model)
// ------------------------------------------------------------------------------------
struct DevSchedule {
  int n_types, n_q, n_rad, n_lin;
  int64_t n_params;
  int n_mom, n_vals, first_dst, nu_max;
  int n_fwaves, n_rwaves;
  double r_min, r_cut;
  const int* comp_info;     // per moment component: mu | a<<8 | b<<16 | c<<24
  const int* fwave_ptr;     // [n_fwaves+1] into fdst
  const int* fdst;          // destination value index, grouped by depth
  const int* tri_ptr;       // [n_vals - n_mom + 1]
  const uint32_t* tri_ab;   // a | b << 16
  const float* tri_cf;
  const double* tri_cd;
  const int* rwave_ptr;     // [n_rwaves+1] into rval
  const int* rval;          // value index, grouped by height (sinks first)
  const int* use_ptr;       // [n_vals+1]
  const uint32_t* use_od;   // other operand | dst << 16
  const float* use_cf;
  const double* use_cd;
  const int* basis_idx;     // [n_lin]
  // packed copies for the specialised mixed-path kernel (nullptr when n_vals > 4096 or more
  // than 256 distinct coefficients): a | b << 12 | coef_index << 24, other | dst << 12 | ci << 24
  const uint32_t* tri_pk;
  const uint32_t* use_pk;
  const float* coef_f;
  int n_coef;
  // slab words carry their coefficient inline: a | b << 11 | code << 22, with the float
  // rebuilt as bits (code << 17) + 0x3F800000; padding terms read the always-zero value slot
  // n_vals.  Otherwise a | b << 12 | ci << 24 with ci into coef_f (padding: coefficient 0).
  bool coef_inline;
  int n_tri, n_use;         // lengths of the triple and use lists
  // "slab" form of the packed lists for warp-per-neighborhood execution: rounds of 32
  // destinations; word (round r, iteration it, lane l) at off_r + 32 it + l, lists padded to the
  // round's longest with zero-coefficient terms.  round = {L, off, end_of_wave, 0}
  const uint32_t* fslab;
  const int4* fround;
  const int* fr_dst;        // [n_fround * 32], -1 = idle lane
  int n_fround, fslab_words;
  const uint32_t* rslab;
  const int4* rround;
  const int* rr_val;        // [n_rround * 32], -1 = idle lane
  int n_rround, rslab_words;
  // packed rounds of the three-kernel pass's contraction: a long list takes an aligned group of
  // 2..32 lanes (equal shares, combined by a butterfly); lane entry -1 (idle) or
  // index | log2(group) << 16 | leader << 20; round = {L, off, end_of_wave, grouped}
  const uint32_t* pfslab;
  const int4* pfround;
  const int* pfr_dst;
  int n_pfround, pfslab_words;
  const uint32_t* prslab;
  const int4* prround;
  const int* prr_val;
  int n_prround, prslab_words;
  const double* theta_d;    // [n_params]
  const float* theta_f;
  const double* seed_d;     // [n_vals] sum of xi over basis functions stored at that value
  const float* seed_f;
};

// ------------------------------------------------------------------------------------
// neighbor list on the device
// ------------------------------------------------------------------------------------
struct CfgPlan {
  double H[9];        // rows = lattice vectors
  double Hinv[9];     // s = x Hinv
  int nb[3], kb[3], pbc[3];
  int K;              // image table half-width: nrel in [-K, K]^3
  int64_t bin_base;
  int64_t shift_base; // offset into the shift table ((2K+1)^3 entries)
  double rc2;
};

struct DevNbr {
  int64_t n_atoms, n_pairs;
  const int64_t* off;   // [n_atoms+1]
  const int* pj;        // neighbor atom
  const int* pimg;      // packed image (3 x 10-bit signed) relative to the given positions
  const int* prev;      // index of the reverse pair
  const float4* pr32;   // r_ij rounded from a double-single evaluation, .w = |r_ij|
  const int* atom_cfg;  // configuration of each atom
};

// Round an FP32 value to the nearest TF32 (10 explicit mantissa bits, ties away from zero);
// the result is exactly representable, so tensor cores consume it without further rounding.
inline __host__ __device__ float tf32_rn(float x) {
#ifdef __CUDA_ARCH__
  return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xffffe000u);
#else
  uint32_t u;
  std::memcpy(&u, &x, 4);
  u = (u + 0x1000u) & 0xffffe000u;
  float y;
  std::memcpy(&y, &u, 4);
  return y;
#endif
}

inline __host__ __device__ int pack_img(int a, int b, int c) {
  return (a & 1023) | ((b & 1023) << 10) | ((c & 1023) << 20);
}
inline __host__ __device__ int unpack_img(int v, int k) {
  int x = (v >> (10 * k)) & 1023;
  return x >= 512 ? x - 1024 : x;
}

// ------------------------------------------------------------------------------------
// handles
// ------------------------------------------------------------------------------------
struct ModelHost;
}  // namespace mtp

struct mtp_model {
  int device = 0;
  mtp_desc desc{};
  mtp::Schedule sched;
  mtp::DevSchedule ds{};
  mtp::DevBuf sched_buf;       // all schedule arrays
  mtp::DevBuf theta_buf;       // theta_d, theta_f, seed_d, seed_f
  std::vector<double> theta;   // host copy
  // active set
  bool have_ainv = false;
  int64_t m_active = 0;
  mtp::DevBuf a_d;             // m x m FP64 active-set matrix (rows = active neighborhoods)
  mtp::DevBuf ainv_d;          // m x m FP64
  mtp::DevBuf ainv_f;          // padded FP32 (hi) and (lo) for the mixed grade
  int64_t ainv_ld = 0;
  // workspaces
  mtp::DevBuf ws_pair;         // per-pair gradients
  mtp::DevBuf ws_atom;         // per-atom V, W
  mtp::DevBuf ws_rows;         // parameter rows for the grade
  mtp::DevBuf ws_grade;        // per-pass partial row maxima of the tensor-core grade
  mtp::DevBuf ws_sort;         // species order of the rows for the tensor-core grade
  mtp::DevBuf ws_misc;
  mtp::DevBuf ws_red;          // reductions
  mtp::DevBuf err_flag;        // unsigned
  // errors of asynchronous kernels (bit 1: a bounded wait of the tensor-core grade expired),
  // allocated and zeroed by mtp_load, OR-ed by the kernels, read and cleared by mtp_sync
  mtp::DevBuf async_err;
  bool force_generic = false;  // route the mixed path through the generic kernel (cross-checks)
  // launch shape of the per-neighborhood kernels: warps per block (0 = largest that fits),
  // chosen by mtp_autotune; last_warps records the shape of the latest launch
  int tune_warps_fast = 0;
  int tune_fwd_global = -1;    // forward schedule in global memory: -1 automatic, 0 no, 1 yes
  bool last_fwd_global = false;
  int tune_warps_generic = 0;
  int last_warps = 0;
  bool last_fast = false;
  // mixed pass: caller's choice (0 automatic, 1 single kernel, 2 three kernels), the
  // autotuner's choice for "automatic" (-1 untuned, 0 single, 1 three kernels), and the
  // three-kernel pass's warps per block of its per-pair kernels and neighborhoods per warp of its
  // contraction (0: defaults)
  int mixed_pass = 0;
  int tune_split = -1;
  int tune_split_warps = 0;
  int tune_split_nb = 0;
  int tune_split_unroll = 0;   // words in flight per lane in the contraction (2 or 4; 0 = 2)
  int tune_split_sched = 0;    // contraction schedule: 0 = shared memory where it fits, 1 = shared
                               // memory, 2 = streamed through a shared ring, 3 = tensor memory
  bool last_split = false;
  int last_split_sched = 0;   // where the last three-kernel pass read its schedule (1, 2 or 3 as above)
  mtp::DevBuf split_tab;       // slot -> component table of the split pass (uploaded by mtp_load)
  mtp::DevBuf ws_mom;          // moments / their adjoints of the split pass
};

struct mtp_nbr {
  int device = 0;
  int64_t n_atoms = 0, n_pairs = 0, n_cfg = 0;
  mtp::DevNbr dn{};
  mtp::DevBuf off, pj, pimg, prev, pr32, atom_cfg;
  mtp::DevBuf segs;   // per scanned bin and atom: accepted slots and pairs before the bin (neighbors.cu)
  mtp::DevBuf masks;  // per-atom accepted-candidate bits of the count pass (neighbors.cu)
  mtp::DevBuf bins, plan, shifts, wrap, scratch, counts;
  std::vector<mtp::CfgPlan> plans;
  std::vector<int64_t> atom_offset;   // host copy
  int64_t n_bins_total = 0;
  // segments for deterministic per-config reductions: [cfg, atom_begin, atom_end]
  std::vector<int64_t> seg_host;
  mtp::DevBuf seg;
  int64_t n_seg = 0;
};

namespace mtp {

// kernels / launchers implemented in the .cu files
void upload_schedule(mtp_model* m);
void upload_theta(mtp_model* m);
void build_neighbors(mtp_model* m, const mtp_batch* b, mtp_nbr* nb, cudaStream_t s);
unsigned read_and_clear_flag(mtp_model* m, cudaStream_t s);

struct SiteOutputs {
  double* V = nullptr;          // per atom
  void* G = nullptr;            // per pair gradient (R x 3)
  double* Wat = nullptr;        // per atom virial (9)
  double* rows = nullptr;       // parameter rows (FP64), ld = n_params
  float* rows_hi = nullptr;     // parameter rows split for the tensor-core grade
  float* rows_lo = nullptr;
  int64_t rows_ld = 0;
  const int64_t* atom_list = nullptr;  // optional explicit atoms (rows follow list order)
  const int64_t* row_pos = nullptr;    // optional row of each atom's b_i (rows in another order)
  int64_t n_list = 0;
  // workspace of the three-kernel mixed pass (moments, then their adjoints; split_ldm(n_mom)
  // floats per atom); null: the single-kernel pass
  float* mom = nullptr;
  // tangent mode (training)
  const double* U = nullptr;    // per atom 3
  const double* Scfg = nullptr; // per config 9
  const double* coef = nullptr; // per config energy coefficient
  double* grad_part = nullptr;  // [gridDim x n_params]
};

void run_sites(mtp_model* m, const mtp_batch* b, const mtp_nbr* nb, bool fp64, const SiteOutputs& o,
               bool tangent, int* grid_used, cudaStream_t s);
void run_forces(const mtp_nbr* nb, bool fp64, const void* G, double* F, cudaStream_t s);
// atom indices sorted (stably) by species into order[0, N), their species into zrow, and each
// atom's position in that order into order[N, 2N)
void run_species_order(const int32_t* type, int64_t N, int n_types, int32_t* zrow, int64_t* order, DevBuf& tmp,
                       cudaStream_t s);
void run_config_sums(const mtp_nbr* nb, const double* V, const double* Wat, double* E, double* W,
                     DevBuf& tmp, cudaStream_t s);
void run_lu_inverse(mtp_model* m, const double* A, int64_t n, cudaStream_t s);
void run_config_row_sums(const mtp_nbr* nb, const double* rows, int64_t m, double* out, DevBuf& tmp, cudaStream_t s);
void run_config_gamma_max(const mtp_nbr* nb, const double* gamma, double* gamma_cfg, int64_t* worst, DevBuf& tmp,
                          cudaStream_t s);
void run_classify(const double* gamma, int64_t n, double g_save, double g_break, int32_t* cls, cudaStream_t s);
void run_widen_argmax(const int32_t* in, int64_t n, int64_t* out, cudaStream_t s);
// g_theta = sum_k gE[k] R[k] (R: n_cfg x m configuration rows), g_pos[i] = -gE[cfg(i)] F[i]
void run_energy_vjp(const mtp_nbr* nb, const double* R, const double* gE, int64_t m, const double* F, double* g_pos,
                    double* g_theta, cudaStream_t s);
int64_t run_cut_clusters(const mtp_batch* b, const int64_t* centers, int64_t n, double radius, int64_t* off,
                         double* pos, int32_t* type, int64_t* src, int64_t capacity, cudaStream_t s);
// host-side fault injection (mtp_debug_inject): armed counts, each consumed by one event
extern std::atomic<int> g_inject_alloc;
extern std::atomic<int> g_inject_overflow;
extern std::atomic<int> g_inject_grade_wait;
bool take_injected(std::atomic<int>& c);
// per-neighborhood value slots of the specialised kernel's shared-memory arrays: the values,
// one always-zero slot (index n_values), padded to a multiple of 4
inline int padded_nv(int n_values) { return (n_values + 1 + 3) & ~3; }
// per-atom stride (floats) of the split pass's moment workspace
inline int split_ldm(int n_mom) { return (n_mom + 3) & ~3; }
void split_prepare(mtp_model* m);
// whether the mixed path takes the three-kernel pass (caller's setting, else the autotuner's)
inline bool split_wanted(const mtp_model* m) {
  return m->split_tab.p && (m->mixed_pass == 2 || (m->mixed_pass == 0 && m->tune_split != 0));
}
int64_t run_maxvol(mtp_model* md, const double* B, int64_t n, double eps, int64_t max_swaps, int64_t* source,
                   cudaStream_t s);
void run_grade(mtp_model* m, int64_t N, bool fp64, const double* rows, const float* rows_hi,
               const float* rows_lo, int64_t ld, double* gamma, int32_t* argmax, cudaStream_t s);
void run_flag(int64_t N, const double* gamma, double threshold, int32_t* flagged, int64_t* n_flagged,
              DevBuf& tmp, cudaStream_t s);
int64_t run_extract(const mtp_nbr* nb, const mtp_batch* b, const int32_t* idx, int64_t n, int64_t* off,
                    double* r, int32_t* type, int32_t* j, int64_t capacity, DevBuf& tmp, cudaStream_t s);
void run_train_prep(const mtp_nbr* nb, int n_cfg, const double* E, const double* F, const double* W,
                    const double* E_ref, const double* F_ref, const double* W_ref, double w_e,
                    double w_f, double w_s, double* coef, double* U, double* Scfg, double* loss,
                    DevBuf& tmp, cudaStream_t s);
void run_sum_rows(const double* part, int nrows, int64_t m, double* out, cudaStream_t s);
// argument checks shared by the entry points that run the per-neighborhood pass
void check_run(const mtp_model* m, const mtp_batch* b, const mtp_nbr* nb);
// loads the allocation-free path's module on `device` (current) and records its scratch address
void noalloc_prepare(int device);
int64_t grade_tc_ld(int64_t m);   // row stride of the split parameter rows and of A^-1

}  // namespace mtp

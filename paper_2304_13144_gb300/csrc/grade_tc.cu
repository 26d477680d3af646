// Tensor-core grade product for the mixed path (sm_103a: TMA + tcgen05 + TMEM).
//
// Section II.D: gamma_i = max_p |(b_i A^-1)_p|.  C = B X with B the parameter rows (N x K) and
// X = A^-1 (K x K), both split into TF32 pieces v = hi + lo (hi, lo rounded to nearest TF32), and
// C ~ B_hi X_hi + B_hi X_lo + B_lo X_hi accumulated in FP32 in tensor memory (each product then
// has a relative error of about 2^-22, the size of the FP32 rows' own rounding).  The
// row epilogue (max |C_ip| and the lowest p attaining it) is fused: C never leaves the SM.
//
// One persistent CTA per SM, 6 warps:
//   warp 0: TMA producer (128B-swizzled fp32 tiles of B and X into a 2-stage ring),
//   warp 1: allocates TMEM and issues tcgen05.mma (M = 128, N = 224, K = 8 per instruction),
//   warps 2-5: epilogue, one row per thread (tcgen05.ld 32x32b), two TMEM accumulators so the
//              epilogue of one 224-column pass overlaps the MMAs of the next.
// Every mbarrier wait is bounded (a.wait_limit tries): on expiry the kernel records an error in
// the model's latch, stops issuing, waits for its own copies and MMAs in flight (bounded by the
// default limit, whatever a.wait_limit is), frees TMEM and returns.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "mtp_internal.h"
#include "profiler.h"

namespace mtp {
namespace {

constexpr int BM = 128;            // rows per tile (TMEM lanes)
constexpr int BN = 224;            // columns per pass (MMA N)
constexpr int BK = 32;             // fp32 elements per 128-byte swizzle row
constexpr int KSTEP = 8;           // K per tcgen05.mma kind::tf32
constexpr int STAGES = 2;
constexpr int A_BYTES = BM * BK * 4;   // 16 KB
constexpr int B_BYTES = BN * BK * 4;   // 28 KB
constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;
constexpr int TMEM_COLS = 512;
constexpr int THREADS = 192;
constexpr uint32_t WAIT_LIMIT = 1u << 24;   // default tries per wait (>= 1 s with the back-off)
constexpr size_t SMEM_BYTES = STAGES * STAGE_BYTES + 256 + 1024;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait of at most `limit` tries; false = gave up (abort flag set by the caller)
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                          uint32_t limit = WAIT_LIMIT) {
  for (uint32_t it = 0; it < limit; ++it) {
    if (mbar_try(bar, parity)) return true;
    if (*abort_flag) return false;
    if (it > 64) __nanosleep(64);
  }
  return false;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// K-major, 128-byte swizzle, 8-row groups 1024 bytes apart
__device__ __forceinline__ uint64_t smem_desc(const void* p) {
  const uint64_t addr = smem_u32(p);
  uint64_t d = 0;
  d |= (addr >> 4) & 0x3FFFull;           // start address
  d |= 1ull << 16;                        // leading byte offset (unused for swizzled K-major)
  d |= (1024ull >> 4) << 32;              // stride byte offset
  d |= 1ull << 46;                        // descriptor version
  d |= 2ull << 61;                        // SWIZZLE_128B
  return d;
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
      ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

struct TcArgs {
  int64_t N;           // rows
  int m;               // valid columns
  int n_pass;          // ld / BN
  int k_chunks;        // ld / BK
  int64_t n_tiles;     // ceil(N / BM)
  int64_t n_work;      // n_tiles * n_pass work items (tile, pass)
  float* pbest;        // [n_pass x N] per-pass row maxima
  int32_t* parg;       // [n_pass x N] and their columns
  unsigned* err;       // the model's asynchronous error latch (bit 1: a wait expired)
  uint32_t wait_limit; // tries per wait in normal operation (the drain waits use WAIT_LIMIT)
  // rows grouped by the center's species (zrow[r], ascending) or zrow == null: the radial block
  // of b_i is zero outside the center's species, so a K chunk that lies in the blocks of species
  // absent from a tile (or in the padding past n_params) is skipped for that tile
  const int32_t* zrow;
  int off_c, cbn, n_params;
};

// true when every row of a tile whose species lie in [zlo, zhi] is zero in K chunk kc
__device__ __forceinline__ bool chunk_zero(const TcArgs& a, int kc, int zlo, int zhi) {
  if (!a.zrow) return false;
  const int lo = kc * BK;
  if (lo < a.off_c) return false;
  const int hi = min(lo + BK, a.n_params) - 1;   // the chunk's last real column
  if (hi < lo) return true;                       // padding only
  const int z0 = (lo - a.off_c) / a.cbn, z1 = (hi - a.off_c) / a.cbn;
  return z1 < zlo || z0 > zhi;
}

__device__ __forceinline__ void tile_species(const TcArgs& a, int64_t tile, int& zlo, int& zhi) {
  zlo = 0;
  zhi = 0;
  if (!a.zrow) return;
  zlo = a.zrow[tile * BM];
  zhi = a.zrow[min(a.N, (tile + 1) * BM) - 1];
}

// gamma_i and argmax_i from the per-pass partials: passes in column order, strict '>' keeps the
// lowest column on ties; a NaN partial (a pass that did not run) makes gamma_i NaN; row r is atom
// row_atom[r] when rows were grouped by species
__global__ void k_grade_combine(int64_t N, int n_pass, const float* pbest, const int32_t* parg, const int64_t* row_atom,
                                double* gamma, int32_t* argmax) {
  const int64_t r = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (r >= N) return;
  float best = -1.f;
  int arg = 0;
  bool nan = false;
  for (int p = 0; p < n_pass; ++p) {
    const float v = pbest[p * N + r];
    nan = nan || (v != v);
    if (v > best) { best = v; arg = parg[p * N + r]; }
  }
  const int64_t o = row_atom ? row_atom[r] : r;
  gamma[o] = nan ? __longlong_as_double(0x7ff8000000000000LL) : static_cast<double>(best);
  if (argmax) argmax[o] = arg;
}

__global__ void __launch_bounds__(THREADS, 1) k_grade_tc(const __grid_constant__ CUtensorMap mAh,
                                                          const __grid_constant__ CUtensorMap mAl,
                                                          const __grid_constant__ CUtensorMap mBh,
                                                          const __grid_constant__ CUtensorMap mBl, TcArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* ring = smem;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
  uint64_t* full = bars;              // [STAGES]
  uint64_t* empty = bars + 2;         // [STAGES]
  uint64_t* accf = bars + 4;          // [2]
  uint64_t* acce = bars + 6;          // [2]
  uint64_t* drain = bars + 8;         // [1]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 9);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(bars + 10);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
    for (int b = 0; b < 2; ++b) { mbar_init(&accf[b], 1); mbar_init(&acce[b], 4); }
    mbar_init(drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      uint32_t it = 0;
      // work item w = (tile w / n_pass, pass w % n_pass); the grid is a multiple of n_pass, so the
      // CTAs of one tile run its passes side by side (the row tile is read from DRAM once) and
      // each CTA keeps one column slab of A^-1
      for (int64_t w = blockIdx.x; w < a.n_work && !*abort_flag; w += gridDim.x) {
        const int64_t tile = w / a.n_pass;
        const int pass = static_cast<int>(w - tile * a.n_pass);
        int zlo, zhi;
        tile_species(a, tile, zlo, zhi);
          for (int kc = 0; kc < a.k_chunks; ++kc) {
            if (chunk_zero(a, kc, zlo, zhi)) continue;
            const uint32_t s = it % STAGES, n = it / STAGES;
            if (n > 0 && !mbar_wait(&empty[s], (n - 1) & 1, abort_flag, a.wait_limit)) { *abort_flag = 1; break; }
            unsigned char* st = ring + s * STAGE_BYTES;
            mbar_expect_tx(&full[s], STAGE_BYTES);
            const int x = kc * BK, yr = static_cast<int>(tile * BM), yc = pass * BN;
            tma_load_2d(st, &mAh, x, yr, &full[s]);
            tma_load_2d(st + A_BYTES, &mAl, x, yr, &full[s]);
            tma_load_2d(st + 2 * A_BYTES, &mBh, x, yc, &full[s]);
            tma_load_2d(st + 2 * A_BYTES + B_BYTES, &mBl, x, yc, &full[s]);
            ++it;
          }
      }
      if (*abort_flag) {
        // let the copies already issued land before the CTA's shared memory goes away
        for (uint32_t j = (it > STAGES ? it - STAGES : 0); j < it; ++j) {
          volatile int no_abort = 0;
          mbar_wait(&full[j % STAGES], (j / STAGES) & 1, &no_abort);
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | (static_cast<uint32_t>(BN >> 3) << 17) |
                             (static_cast<uint32_t>(BM >> 4) << 24);
      uint32_t it = 0, acc_it = 0;
      bool issued = false;
      for (int64_t w = blockIdx.x; w < a.n_work && !*abort_flag; w += gridDim.x, ++acc_it) {
        {
          const uint32_t b = acc_it & 1, na = acc_it >> 1;
          if (na > 0 && !mbar_wait(&acce[b], (na - 1) & 1, abort_flag, a.wait_limit)) { *abort_flag = 1; break; }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t dtm = tmem + b * BN;
          int zlo, zhi;
          tile_species(a, w / a.n_pass, zlo, zhi);
          for (int kc = 0; kc < a.k_chunks; ++kc) {
            if (chunk_zero(a, kc, zlo, zhi)) continue;   // chunk 0 never is: the first MMA sets D
            const uint32_t s = it % STAGES, n = it / STAGES;
            if (!mbar_wait(&full[s], n & 1, abort_flag, a.wait_limit)) { *abort_flag = 1; break; }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            unsigned char* st = ring + s * STAGE_BYTES;
#pragma unroll
            for (int ks = 0; ks < BK / KSTEP; ++ks) {
              const uint32_t off = ks * KSTEP * 4;
              const uint64_t ah = smem_desc(st + off), al = smem_desc(st + A_BYTES + off);
              const uint64_t bh = smem_desc(st + 2 * A_BYTES + off), bl = smem_desc(st + 2 * A_BYTES + B_BYTES + off);
              mma_tf32(dtm, ah, bh, idesc, (kc > 0 || ks > 0) ? 1u : 0u);
              mma_tf32(dtm, ah, bl, idesc, 1u);
              mma_tf32(dtm, al, bh, idesc, 1u);
            }
            mma_commit(&empty[s]);
            issued = true;
            ++it;
          }
          if (*abort_flag) break;
          mma_commit(&accf[b]);
        }
      }
      if (issued) {
        // all MMAs of this thread complete before TMEM is released
        mma_commit(drain);
        volatile int no_abort = 0;
        mbar_wait(drain, 0, &no_abort);
      }
    }
    __syncwarp();
  } else {
    const int q = warp & 3;   // TMEM lane quarter accessible to this warp
    uint32_t acc_it = 0;
    for (int64_t w = blockIdx.x; w < a.n_work && !*abort_flag; w += gridDim.x) {
      const int64_t tile = w / a.n_pass;
      const int pass = static_cast<int>(w - tile * a.n_pass);
      float best = -1.f;
      int barg = 0;
      {
        const uint32_t b = acc_it & 1, na = acc_it >> 1;
        ++acc_it;
        bool ok = true;
        if (lane == 0) ok = mbar_wait(&accf[b], na & 1, abort_flag, a.wait_limit);
        ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
        if (!ok) { if (lane == 0) *abort_flag = 1; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t tbase = tmem + (static_cast<uint32_t>(q * 32) << 16) + b * BN;
#pragma unroll 1
        for (int c0 = 0; c0 < BN; c0 += 32) {
          float v[32];
          tmem_ld32(tbase + c0, v);
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const int col = pass * BN + c0 + j;
            const float av = fabsf(v[j]);
            if (col < a.m && av > best) { best = av; barg = col; }
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(&acce[b]);
      }
      if (*abort_flag) break;
      const int64_t row = tile * BM + q * 32 + lane;
      if (row < a.N) {
        a.pbest[pass * a.N + row] = best;
        a.parg[pass * a.N + row] = barg;
      }
    }
  }
  if (threadIdx.x == 0 && *abort_flag) atomicOr(a.err, 1u);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
  }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    MTP_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q));
    if (q != cudaDriverEntryPointSuccess || !p) throw Fail{MTP_ERR_CUDA, "cuTensorMapEncodeTiled unavailable"};
    fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

CUtensorMap make_map(const float* base, int64_t rows, int64_t ld, int box_rows) {
  CUtensorMap m;
  const cuuint64_t dims[2] = {static_cast<cuuint64_t>(ld), static_cast<cuuint64_t>(rows)};
  const cuuint64_t strides[1] = {static_cast<cuuint64_t>(ld) * 4};
  const cuuint32_t box[2] = {BK, static_cast<cuuint32_t>(box_rows)};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = encode_fn()(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box,
                                 estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                 CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) throw Fail{MTP_ERR_CUDA, "cuTensorMapEncodeTiled failed"};
  return m;
}

}  // namespace

int64_t grade_tc_ld(int64_t m) { return ((m + BN - 1) / BN) * BN; }

bool grade_tc_available(const mtp_model* md) {
  static int cached = -1;
  if (cached < 0) {
    cudaDeviceProp prop;
    cached = (cudaGetDeviceProperties(&prop, md->device) == cudaSuccess && prop.major == 10 && prop.minor == 3) ? 1 : 0;
  }
  return cached == 1 && md->ainv_ld % BN == 0 && md->ainv_ld % BK == 0;
}

void run_grade_tc(mtp_model* md, int64_t N, const float* hi, const float* lo, int64_t ld, double* gamma,
                  int32_t* argmax, const int32_t* zrow, const int64_t* row_atom, cudaStream_t s) {
  if (N == 0) return;
  if (ld != md->ainv_ld || ld % BN != 0) throw Fail{MTP_ERR_ARG, "grade: row stride mismatch"};
  const float* xh = md->ainv_f.as<float>();
  const float* xl = xh + ld * ld;
  const CUtensorMap mAh = make_map(hi, N, ld, BM), mAl = make_map(lo, N, ld, BM);
  const CUtensorMap mBh = make_map(xh, ld, ld, BN), mBl = make_map(xl, ld, ld, BN);
  TcArgs a;
  a.N = N;
  a.m = static_cast<int>(md->m_active);
  a.n_pass = static_cast<int>(ld / BN);
  a.k_chunks = static_cast<int>(ld / BK);
  a.n_tiles = (N + BM - 1) / BM;
  a.n_work = a.n_tiles * a.n_pass;
  md->ws_grade.ensure(static_cast<size_t>(a.n_pass) * N * (sizeof(float) + sizeof(int32_t)), s);
  a.pbest = md->ws_grade.as<float>();
  a.parg = reinterpret_cast<int32_t*>(a.pbest + static_cast<size_t>(a.n_pass) * N);
  // partials start as NaN: a pass that does not run (a bounded wait expired) leaves gamma NaN
  MTP_CUDA(cudaMemsetAsync(a.pbest, 0xFF, static_cast<size_t>(a.n_pass) * N * sizeof(float), s));
  a.err = md->async_err.as<unsigned>();
  // host-side fault injection: a single try per wait makes the first unsatisfied wait expire
  a.wait_limit = take_injected(g_inject_grade_wait) ? 1u : WAIT_LIMIT;
  a.zrow = zrow;
  a.off_c = md->sched.n_types + md->sched.n_lin;
  a.cbn = md->sched.n_types * md->sched.n_rad * md->sched.n_q;
  a.n_params = md->sched.n_params;
  MTP_CUDA(cudaFuncSetAttribute(k_grade_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(SMEM_BYTES)));
  int nsm = 0;
  MTP_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, md->device));
  const int per = nsm >= a.n_pass ? (nsm / a.n_pass) * a.n_pass : nsm;   // a multiple of n_pass
  const int grid = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(a.n_work, per)));
  ProfRegion pr("grade_tc_tf32x3", s);
  k_grade_tc<<<grid, THREADS, SMEM_BYTES, s>>>(mAh, mAl, mBh, mBl, a);
  ProfRegion::launched();
  MTP_CUDA(cudaGetLastError());
  k_grade_combine<<<static_cast<unsigned>((N + 255) / 256), 256, 0, s>>>(N, a.n_pass, a.pbest, a.parg, row_atom,
                                                                         gamma, argmax);
  ProfRegion::launched();
  MTP_CUDA(cudaGetLastError());
}

}  // namespace mtp

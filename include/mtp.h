/*
 * mtp.h - C ABI of the GB300-native Moment Tensor Potential hot path
 * (the neighborhood-level method of MLIP-3, arXiv 2304.13144).
 *
 * Conventions (all entry points):
 *  - Every array argument is caller-owned.  "device" arrays live in CUDA device memory of
 *    the current device; "host" arrays in host memory.  The library never frees them.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).  Work is
 *    enqueued on it; calls that must read a size back from the GPU (neighbor build,
 *    extraction) synchronise that stream.
 *  - Handles (mtp_model, mtp_nbr) and their scratch are owned by the library and released
 *    by mtp_free_model / mtp_free_nbr.
 *  - No C++ exception crosses the ABI.  A failing call returns a non-zero mtp_status,
 *    leaves its outputs unspecified and its handles valid; mtp_last_error() gives a
 *    thread-local message for the last failure on this thread.
 *  - Parameter layout (the paper fixes none; see the design notes):
 *      theta = [ s_z (n_types) | xi_a (n_lin, canonical basis order) |
 *                c[z_i][z_j][mu][beta] (n_types^2 * n_rad * n_q, row-major) ],
 *    m = n_types + n_lin + n_types^2 n_rad n_q.
 *  - Units: positions and cells in Angstrom, energies in eV, forces in eV/A,
 *    virial W_ab = -dE/d(eps_ab) in eV (not divided by the volume).
 */
#ifndef MTP_H
#define MTP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mtp_model mtp_model; /* opaque: descriptor, schedule, parameters, A^-1 */
typedef struct mtp_nbr mtp_nbr;     /* opaque: neighbor list in device memory */

typedef enum {
  MTP_OK = 0,
  MTP_ERR_ARG = 1,         /* invalid argument (null pointer, size, species out of range) */
  MTP_ERR_CUDA = 2,        /* a CUDA runtime call failed */
  MTP_ERR_CAPACITY = 3,    /* a caller-provided output buffer is too small */
  MTP_ERR_SINGULAR = 4,    /* active-set matrix singular (LU pivot below tolerance) */
  MTP_ERR_GEOMETRY = 5,    /* coincident atoms (|r_ij| < 1e-8 A) or a degenerate cell */
  MTP_ERR_NUMERIC = 6,     /* non-finite input */
  MTP_ERR_UNSUPPORTED = 7, /* request outside what this build supports */
  MTP_ERR_TIMEOUT = 8      /* a bounded wait inside a kernel expired (reported by mtp_sync) */
} mtp_status;

typedef enum { MTP_FP64 = 0, MTP_MIXED = 1 } mtp_precision;

/* Model descriptor.  Section II.A: n_types species, MTP level lev_max (eqs. 5-6), n_q
 * radial polynomials (Chebyshev T_0..T_{n_q-1} on [r_min, r_cut], eq. 4), cut-off r_cut. */
typedef struct {
  int32_t n_types;
  int32_t lev_max;
  int32_t n_q;
  int32_t reserved;
  double r_min;
  double r_cut;
} mtp_desc;

/* Sizes derived from a descriptor (mtp_describe / mtp_model_sizes). */
typedef struct {
  int64_t n_params;     /* m */
  int32_t n_lin;        /* number of basis functions B_a (eq. 2) */
  int32_t n_rad;        /* number of radial functions f_mu (eq. 4) */
  int32_t n_moments;    /* distinct moments M_{mu,nu} used by the basis (eq. 3) */
  int32_t n_mom_comps;  /* symmetric-storage components of those moments */
  int32_t n_values;     /* per-atom value array: components + intermediates */
  int32_t n_triples;    /* flattened contraction triples (dst += c * a * b) */
  int32_t nu_max;       /* largest tensor rank used */
  int32_t n_gauge;      /* n_rad (n_rad + 1) / 2 null directions of the parameter rows */
} mtp_sizes;

/* A batch of configurations (Section III.A: size, types, positions, supercell).
 * All pointers are caller-owned DEVICE memory. */
typedef struct {
  int32_t n_cfg;
  int32_t reserved;
  const int64_t* atom_offset; /* n_cfg + 1, atoms of config k are [atom_offset[k], atom_offset[k+1]) */
  const double* pos;          /* N x 3, A */
  const int32_t* type;        /* N, 0 .. n_types - 1 */
  const double* cell;         /* n_cfg x 3 x 3, row a = lattice vector a, A */
  const uint8_t* pbc;         /* n_cfg x 3, non-zero = periodic along that lattice vector */
} mtp_batch;

/* ---------------------------------------------------------------------------------- */
/* Library and model                                                                  */
/* ---------------------------------------------------------------------------------- */

const char* mtp_version(void);
const char* mtp_last_error(void); /* thread-local; never NULL */

/* Host-only: sizes of the basis of `desc` (Section II.A, eqs. 5-6).  Calls no CUDA API. */
mtp_status mtp_describe(const mtp_desc* desc, mtp_sizes* out);

/* Host-only: the canonical basis (Section II.A).  Function a is a multigraph on P[a] <= 4
 * moment factors with labels (mu[4a+p], nu[4a+p]) and edge multiplicities
 * edges[6a+e] over node pairs (0,1),(0,2),(0,3),(1,2),(1,3),(2,3).  Arrays are host
 * memory of capacity n_lin (mu, nu: 4 n_lin; edges: 6 n_lin).  Calls no CUDA API. */
mtp_status mtp_describe_basis(const mtp_desc* desc, int32_t* P, int32_t* mu, int32_t* nu,
                              int32_t* edges);

/* Host-only: the flattened contraction schedule (host arrays sized from mtp_sizes):
 * comp_mu[n_mom_comps], comp_exp[3 n_mom_comps] (exponents a,b,c of x^a y^b z^c),
 * dst_ptr[n_values - n_mom_comps + 1], tri_a/tri_b[n_triples], tri_c[n_triples],
 * basis_idx[n_lin].  Value d >= n_mom_comps equals
 * sum_{t in [dst_ptr[d-n_mom_comps], dst_ptr[d-n_mom_comps+1])} tri_c[t] v[tri_a[t]] v[tri_b[t]].
 * Calls no CUDA API. */
mtp_status mtp_describe_schedule(const mtp_desc* desc, int32_t* comp_mu, int32_t* comp_exp,
                                 int32_t* dst_ptr, int32_t* tri_a, int32_t* tri_b,
                                 double* tri_c, int32_t* basis_idx);

/* Host-only: the n_gauge = n_rad (n_rad + 1) / 2 null directions of the parameter rows
 * (rows of D, host, n_gauge x m).  V is unchanged when the radial functions are mixed
 * lower-triangularly, f_mu -> f_mu + eps f_mu' (mu' <= mu, eq. 4), with xi compensating
 * (eqs. 2, 5-6), so b_i . d = 0 for every neighborhood and direction d: an active set of m
 * raw rows is always singular, and a full-rank one takes m - n_gauge rows plus these
 * directions.  The paper does not discuss this.  Calls no CUDA API. */
mtp_status mtp_gauge_directions(const mtp_desc* desc, const double* theta, int64_t m, double* D);

/* Create a model on the current device.  theta: host, m doubles (layout above).
 * Enumerates the basis (Section II.A), compiles the contraction schedule and uploads it. */
mtp_status mtp_load(const mtp_desc* desc, const double* theta, int64_t m, mtp_model** out);
void mtp_free_model(mtp_model* model);
int64_t mtp_num_params(const mtp_model* model);
mtp_status mtp_model_sizes(const mtp_model* model, mtp_sizes* out);

/* Replace theta (host, m doubles); used by training loops (eq. 7). */
mtp_status mtp_set_params(mtp_model* model, const double* theta, int64_t m);

/* Active set (Sections II.C-D): A is DEVICE memory, m x m row-major FP64, row k = the
 * parameter row of active-set entry k.  A^-1 is formed on the GPU by FP64 LU with partial
 * pivoting and kept in the model.  MTP_ERR_SINGULAR if a pivot is below 1e-13 max|A|.
 * Synchronises `stream`. */
mtp_status mtp_set_active_set(mtp_model* model, const double* A, int64_t m, void* stream);

/* Copy A^-1 (m x m, row-major FP64) to DEVICE memory `Ainv`. */
mtp_status mtp_get_active_inverse(const mtp_model* model, double* Ainv, void* stream);

/* ---------------------------------------------------------------------------------- */
/* Neighborhoods                                                                      */
/* ---------------------------------------------------------------------------------- */

/* Build or rebuild the neighbor list (Section II.A): for every atom i all (j, image n)
 * with 0 < |r_ij| < r_cut, r_ij = x_j + n.H - x_i, n = 0 along non-periodic axes, by a
 * cell list over every configuration of the batch.  The full list is kept (both i->j and
 * j->i), with the index of each pair's reverse.  *inout may be NULL (allocated) or a
 * previous list (reused, grown if needed).  Synchronises `stream` (sizes are read back).
 * MTP_ERR_GEOMETRY on coincident atoms or a degenerate cell, MTP_ERR_ARG on a species
 * outside [0, n_types). */
mtp_status mtp_build_neighbors(mtp_model* model, const mtp_batch* batch, mtp_nbr** inout,
                               void* stream);
void mtp_free_nbr(mtp_nbr* nbr);
mtp_status mtp_nbr_size(const mtp_nbr* nbr, int64_t* n_atoms, int64_t* n_pairs);

/* Copy the list to DEVICE arrays: off[n_atoms+1], j[n_pairs], image[3 n_pairs] (integer
 * image n of each pair), r[3 n_pairs] (r_ij, FP64).  Any pointer may be NULL. */
mtp_status mtp_nbr_export(const mtp_nbr* nbr, const mtp_batch* batch, int64_t* off, int32_t* j,
                          int32_t* image, double* r, void* stream);

/* Copy the reverse-pair index to DEVICE rev[n_pairs]: rev[p] is the position of (j -> i, -n) for
 * pair p = (i -> j, n), so rev[rev[p]] = p (the force gather F_i = sum_p (G_p - G_rev(p)) reads
 * it).  MTP_ERR_ARG on a null list or a null rev with pairs present. */
mtp_status mtp_nbr_reverse(const mtp_nbr* nbr, int32_t* rev, void* stream);

/* ---------------------------------------------------------------------------------- */
/* Hot path                                                                           */
/* ---------------------------------------------------------------------------------- */

/* Energies, forces and virial (eqs. 1-4; forces and stresses as used by eq. 7).
 * Outputs are DEVICE memory, any may be NULL except that at least one is given:
 *   energy[n_cfg] = sum_i V_i per configuration (FP64 accumulation),
 *   site_energy[N] = V_i, forces[N x 3] = -dE/dx, virial[n_cfg x 9] = -dE/deps (eV).
 * MTP_MIXED: radial basis, moments, contractions and adjoint in FP32, energy/virial sums
 * in FP64.  MTP_FP64: everything in FP64.  The neighbor list must have been built for
 * this batch (same positions for FP64 parity). */
mtp_status mtp_energy_forces_stress(mtp_model* model, const mtp_batch* batch, const mtp_nbr* nbr,
                                    mtp_precision prec, double* energy, double* site_energy,
                                    double* forces, double* virial, void* stream);

/* mtp_energy_forces_stress plus the per-atom virials (DEVICE site_virial[N x 9], or NULL):
 * W_i[a][b] = -sum_j (dV_i/dr_ij)_a (r_ij)_b, the site-based split of the virial (per-atom
 * stress times volume); sum_{i in k} W_i = virial[k].  The split is a convention (not unique); this one
 * charges each neighborhood's derivative to its center. */
mtp_status mtp_energy_forces_stress_atoms(mtp_model* model, const mtp_batch* batch, const mtp_nbr* nbr,
                                          mtp_precision prec, double* energy, double* site_energy,
                                          double* forces, double* virial, double* site_virial, void* stream);

/* Allocation-free variant of mtp_energy_forces_stress (the paper has no counterpart).
 * For callers that may not allocate device memory at call time (an engine that owns the whole
 * device-memory budget through its own allocator, or a time-step loop that cannot afford an
 * allocation's synchronisation or failure).  Same arguments, outputs and precision as
 * mtp_energy_forces_stress (NULL outputs allowed likewise); the scratch lives in a fixed 16 MiB
 * device array inside the library.  That array is committed on a device when the library's
 * module is loaded there, which mtp_load does (so it is taken when a model is created, before
 * a caller's pool grabs the rest of the memory), and it is held until the process exits.
 * Limits: at most 32768 atoms, 524288 pairs and 1024 configuration segments (4096-atom pieces
 * of the configurations), else MTP_ERR_CAPACITY.  Calls no cudaMalloc/cudaFree.  The CUDA
 * runtime still loads each kernel's code on its first launch (lazy loading) unless
 * CUDA_MODULE_LOADING=EAGER; one call of mtp_energy_forces_stress at start-up loads the same
 * kernels.  A device reset invalidates every model (their device memory is gone); a model
 * loaded afterwards looks the array up again.  Calls share the array: calls that overlap on the
 * GPU race and must be serialised by the caller. */
mtp_status mtp_energy_forces_stress_noalloc(mtp_model* model, const mtp_batch* batch, const mtp_nbr* nbr,
                                            mtp_precision prec, double* energy, double* site_energy,
                                            double* forces, double* virial, void* stream);

/* Per-atom parameter rows b_i = dV_i/dtheta (eq. 9), DEVICE rows[n x m] FP64 for the atoms
 * listed in DEVICE atoms[n] (atoms == NULL: all atoms, n = N). */
mtp_status mtp_param_rows(mtp_model* model, const mtp_batch* batch, const mtp_nbr* nbr,
                          mtp_precision prec, const int64_t* atoms, int64_t n, double* rows,
                          void* stream);

/* Per-atom extrapolation grade (Section II.D): gamma_i = max_p |(b_i A^-1)_p|,
 * argmax_i = the lowest p attaining it, and the compacted list of atoms with
 * gamma_i > threshold (Section II.E, flag iff strictly greater), ascending.
 * DEVICE outputs: gamma[N] (FP64), argmax[N] or NULL, flagged[N] or NULL,
 * n_flagged[1] (int64) or NULL.  Requires mtp_set_active_set.  MTP_MIXED forms the
 * product with split-precision tensor-core arithmetic (FP32-level accuracy); MTP_FP64
 * in FP64.  Every wait inside the tensor-core kernel is bounded: if one expires, the kernel
 * stops, and the gamma_i it did not finish are NaN (never flagged). */
mtp_status mtp_grade(mtp_model* model, const mtp_batch* batch, const mtp_nbr* nbr,
                     mtp_precision prec, double threshold, double* gamma, int32_t* argmax,
                     int32_t* flagged, int64_t* n_flagged, void* stream);

/* Copy of the current active-set matrix A (DEVICE out, m x m FP64, row-major; row j is the
 * parameter row of the j-th active neighborhood).  Requires mtp_set_active_set. */
mtp_status mtp_get_active_set(const mtp_model* model, double* A, void* stream);

/* MaxVol update of the active set (Section II.D, D-optimality: the active set is the m x m
 * matrix of maximal |det A|).  With C = B A^-1 for the candidate rows B, replacing active row
 * j by candidate row i multiplies |det A| by |C_ij|; the update repeatedly makes the swap at
 * the largest |C_ij| (ties: lowest i, then lowest j) while it exceeds 1 + eps, following C and
 * A^-1 by rank-one corrections in FP64, then forms A^-1 afresh from the final A by LU.  A row
 * swapped out is dropped (it is not a candidate); a candidate enters at most once.
 *   B        DEVICE [n x m] FP64 candidate rows (e.g. mtp_param_rows of flagged atoms)
 *   eps      >= 0; max_swaps >= 0 bounds the number of swaps
 *   source   DEVICE [m] int64 out, or NULL: -1 for a kept active row, else the index in B of
 *            the candidate now in its place
 *   n_swaps  HOST out, or NULL: swaps made
 * Requires mtp_set_active_set; MTP_ERR_SINGULAR if the final A cannot be factorised. */
mtp_status mtp_maxvol(mtp_model* model, const double* B, int64_t n, double eps, int64_t max_swaps,
                      int64_t* source, int64_t* n_swaps, void* stream);

/* Configuration rows b(cfg_k) = dE_k/dtheta = sum_{i in k} b_i (eq. 1 with eq. 9): DEVICE
 * rows[n_cfg x m] FP64 out (sums over a configuration's atoms in a fixed order). */
mtp_status mtp_config_rows(mtp_model* model, const mtp_batch* batch, const mtp_nbr* nbr,
                           mtp_precision prec, double* rows, void* stream);

/* Vector-Jacobian product of the configuration energies E_k (eq. 1) for reverse-mode
 * differentiation: given DEVICE gE[n_cfg] (dL/dE_k),
 *   g_theta[m] = sum_k gE_k dE_k/dtheta = sum_k gE_k sum_{i in k} b_i   (b_i of eq. 9; DEVICE, or NULL)
 *   g_pos[N x 3] = dL/dx_i = -gE_{k(i)} F_i                               (DEVICE, or NULL)
 * with F the forces of the forward pass (DEVICE forces[N x 3], required when g_pos is given).
 * Sums run in a fixed order (deterministic).  Synchronises `stream`. */
mtp_status mtp_energy_vjp(mtp_model* model, const mtp_batch* batch, const mtp_nbr* nbr, mtp_precision prec,
                          const double* gE, const double* forces, double* g_pos, double* g_theta, void* stream);

typedef enum {
  MTP_GRADE_NEIGHBORHOOD = 0,   /* gamma(cfg) = max over the configuration's atoms of gamma_i */
  MTP_GRADE_CONFIGURATION = 1   /* gamma(cfg) = max_j |(b(cfg) A^-1)_j|, A from configuration rows */
} mtp_grade_mode;

/* Configuration grades and the learning-on-the-fly classes (Sections II.D-II.E).
 *   gamma_cfg  DEVICE [n_cfg] FP64 out
 *   worst      DEVICE [n_cfg] int64 out, or NULL: neighborhood mode -> the atom with the
 *              largest gamma_i (lowest index on ties, -1 for an empty configuration);
 *              configuration mode -> the active row j attaining the maximum
 *   cls        DEVICE [n_cfg] int32 out, or NULL: 0 if gamma <= gamma_save (continue),
 *              1 if gamma_save < gamma <= gamma_break (save), 2 if gamma > gamma_break (stop)
 * The active set must match the mode (rows of neighborhoods or of configurations).  The
 * configuration-mode product is formed in FP64; prec sets the arithmetic of the rows (and of
 * the per-atom grade in neighborhood mode). */
mtp_status mtp_config_grade(mtp_model* model, const mtp_batch* batch, const mtp_nbr* nbr,
                            mtp_precision prec, mtp_grade_mode mode, double gamma_save,
                            double gamma_break, double* gamma_cfg, int64_t* worst, int32_t* cls,
                            void* stream);

/* One step of MD with extrapolation control (Section III.B): energies, forces, virial and
 * the grade from a single pass over the neighborhoods.  Arguments as in
 * mtp_energy_forces_stress and mtp_grade; gamma may be NULL to skip the grade. */
mtp_status mtp_step(mtp_model* model, const mtp_batch* batch, const mtp_nbr* nbr,
                    mtp_precision prec, double* energy, double* site_energy, double* forces,
                    double* virial, double threshold, double* gamma, int32_t* argmax,
                    int32_t* flagged, int64_t* n_flagged, void* stream);

/* Neighborhoods of selected atoms (Section II.E step 3(ii), Section III.A
 * cut_extrapolative_neighborhood): for the n DEVICE atom indices idx[], write the
 * R_cut neighborhood of each as CSR: off[n+1] (int64), then per neighbor its relative
 * vector r[3] (FP64, A), species type[] and atom index j[] (any of r/type/j may be NULL).
 * `capacity` is the room in r/type/j (neighbors); *total (host) receives the number of
 * neighbors.  MTP_ERR_CAPACITY if capacity < total.  Synchronises `stream`. */
mtp_status mtp_extract_neighborhoods(const mtp_nbr* nbr, const mtp_batch* batch,
                                     const int32_t* idx, int64_t n, int64_t* off, double* r,
                                     int32_t* type, int32_t* j, int64_t capacity,
                                     int64_t* total, void* stream);

/* BFGS fit of theta (Section II.B: minimise the loss of eq. 7 with BFGS), starting from the
 * model's parameters; loss and gradient from mtp_train_step (arguments as there).  Variables
 * u = theta / D, D_p = max(|theta0_p|, 1e-12 max|theta0|); textbook BFGS inverse-Hessian update
 * (skipped when s.y <= 0; H = (s.y / y.y) I before the first update); backtracking Armijo line
 * search (step 1, halved up to 40 times, c1 = 1e-4).  Stops when max|dL/du| <= gtol max(1,|L|),
 * after max_iter accepted steps, or when no step is accepted.  The model is left at the
 * accepted parameters (read them with mtp_get_params).  HOST outputs (or NULL): the final
 * loss and the number of accepted steps.  Host driver; each evaluation runs on `stream` and
 * synchronises it. */
mtp_status mtp_fit_bfgs(mtp_model* model, const mtp_batch* batch, const mtp_nbr* nbr,
                        mtp_precision prec, const double* E_ref, const double* F_ref,
                        const double* W_ref, double w_e, double w_f, double w_s, int64_t max_iter,
                        double gtol, double* loss, int64_t* iters, void* stream);

/* Autotuner for the per-neighborhood kernel's launch shape (the paper has no counterpart):
 * times the pass that mtp_step makes (energies, forces, virial, and the grade when an active
 * set is loaded) on this batch at every feasible number of warps per block (1..8 for the
 * specialised single-kernel mixed pass, 1, 2, 4 for the generic kernel; blocks per SM then
 * follow from the occupancy) and, for the level-20 shape of the single kernel, with the
 * forward part of the contraction schedule in shared or in global memory; for the mixed path
 * also the three-kernel pass (4 or 8 warps per block, 1 or 2 neighborhoods per contraction
 * warp) unless mtp_set_mixed_pass fixed the single kernel.  Keeps the fastest in the model for
 * later calls of this precision (with mixed pass 0, also which pass), and returns the single
 * kernel's warps (HOST warps) and the best time of three of the chosen shape (HOST ms) --
 * either may be NULL.  Synchronises `stream`. */
mtp_status mtp_autotune(mtp_model* model, const mtp_batch* batch, const mtp_nbr* nbr,
                        mtp_precision prec, int32_t* warps, double* ms, void* stream);

/* The launch shapes the autotuner left in the model (HOST outputs, any may be NULL):
 * warps_fast = warps per block of the specialised mixed kernel (0: untuned, the default shape),
 * fwd_global = forward contraction schedule in global (1) or shared (0) memory (-1: untuned),
 * warps_generic = warps per block of the generic kernel (0: untuned).  No GPU work. */
mtp_status mtp_get_launch_shape(const mtp_model* model, int32_t* warps_fast, int32_t* fwd_global,
                                int32_t* warps_generic);

/* Which pass the mixed path runs (no counterpart in the paper; both compute the same method):
 * 1 = one kernel per neighborhood (moments, contraction, adjoint and rows in one pass, the
 * allocation-free entry point's kernel), 2 = three kernels (moments; contraction and its
 * adjoint; pair adjoint), with the moments and their adjoints in a library workspace of
 * 4 ceil4(n_moment_components) bytes per atom; 0 = automatic: the three kernels where the
 * model's shape has them, unless mtp_autotune found the single kernel faster.  Results of the
 * two passes agree to FP32 rounding; each pass is bitwise reproducible under every launch shape.
 * MTP_ERR_UNSUPPORTED for 2 when the shape has no three-kernel pass.  No GPU work. */
mtp_status mtp_set_mixed_pass(mtp_model* model, int pass);

/* Launch shape of the three-kernel pass (what mtp_autotune sets): warps per block of its
 * per-pair kernels (4 or 8; 0 = default 8), neighborhoods per warp of its contraction (1 or 2;
 * 0 = default 1), schedule words per step per lane there (2 or 4, or 8 with two neighborhoods per
 * warp; 0 = default 2) and where the
 * contraction reads its schedule (1 = shared memory; 2 = streamed from global memory through a
 * shared-memory ring, the block's warps in step; 3 = tensor memory, the first 512 rows of 128 B,
 * the rest in shared memory; 0 = shared memory where it fits beside four warps' value arrays).
 * A schedule that fits neither shared nor tensor memory is always streamed; a placement that
 * does not apply falls back to the automatic one.  Results do not depend on it.  MTP_ERR_ARG
 * outside these values.  No GPU work. */
mtp_status mtp_set_split_shape(mtp_model* model, int warps_pair, int nb_contract, int unroll, int schedule);

/* The shape set above (or by mtp_autotune), HOST outputs, any may be NULL; *schedule_used is
 * where the last three-kernel pass read its schedule (1, 2 or 3 as above; 0 before any). */
mtp_status mtp_get_split_shape(const mtp_model* model, int32_t* warps_pair, int32_t* nb_contract, int32_t* unroll,
                               int32_t* schedule, int32_t* schedule_used);

/* The setting above, the pass the next mixed call will run (1 or 2), and the three-kernel
 * pass's tuned shape (warps per block of its per-pair kernels, neighborhoods per warp of its
 * contraction; 0 = default).  HOST outputs, any may be NULL. */
mtp_status mtp_get_mixed_pass(const mtp_model* model, int32_t* setting, int32_t* in_use, int32_t* split_warps,
                              int32_t* split_nb);

/* Checkpoint (the paper keeps theta, the active set and its mode in its .almtp file): the
 * model's descriptor, theta and, if loaded, the active-set matrix A, in a HOST byte buffer
 * (magic "MTP1", version 1, then mtp_desc, m, theta[m] FP64, a flag and A[m x m] FP64, native
 * byte order).  buffer == NULL queries the size (*size, HOST); MTP_ERR_CAPACITY if capacity <
 * size.  mtp_restore makes a new model from such a buffer (A re-factorised on the GPU); the
 * caller frees it with mtp_free_model. */
mtp_status mtp_save(const mtp_model* model, void* buffer, int64_t capacity, int64_t* size, void* stream);
mtp_status mtp_restore(const void* buffer, int64_t size, mtp_model** model, void* stream);

/* Host-side fault injection for tests of the failure paths (no GPU fault is made):
 * MTP_FAULT_DEVICE_ALLOC makes the next `count` growths of a library workspace fail as a device
 * allocation failure (MTP_ERR_CUDA); MTP_FAULT_NEIGHBOR_OVERFLOW flags the next `count`
 * neighbor fills as overflowing their counted capacity (the build repeats a failed fill once,
 * then returns MTP_ERR_CAPACITY); MTP_FAULT_GRADE_WAIT gives every wait of the next `count`
 * tensor-core grade launches a single try, so the first wait not already satisfied expires and
 * the kernel takes its abort path (stops, drains its own copies and MMAs with the default
 * bound, frees tensor memory, leaves the unfinished gamma NaN; mtp_sync then returns
 * MTP_ERR_TIMEOUT).  count = 0 disarms.  Process-wide. */
enum { MTP_FAULT_DEVICE_ALLOC = 1, MTP_FAULT_NEIGHBOR_OVERFLOW = 2, MTP_FAULT_GRADE_WAIT = 3 };
mtp_status mtp_debug_inject(int fault, int count);

/* Synchronise `stream` and report errors that asynchronous kernels of this model latched on
 * the device since the last mtp_sync (mtp_grade and mtp_step return before their kernels run):
 * MTP_ERR_TIMEOUT if a bounded wait of the tensor-core grade expired (the gamma_i it did not
 * finish are NaN).  Clears the latch. */
mtp_status mtp_sync(mtp_model* model, void* stream);

/* Current parameter vector theta (HOST out, m FP64). */
mtp_status mtp_get_params(const mtp_model* model, double* theta, int64_t m);

/* Fitting errors of the current parameters (the check_errors report), HOST report[9]:
 * energy per atom |E_k - E*_k| / N_k: max, mean, RMS over configurations; force |F_i - F*_i|:
 * max, mean, RMS over atoms; virial |W_ab - W*_ab| (eV): max, mean, RMS over configurations
 * and components (zeros if W_ref is NULL).  DEVICE references as in mtp_train_step. */
mtp_status mtp_fit_errors(mtp_model* model, const mtp_batch* batch, const mtp_nbr* nbr,
                          mtp_precision prec, const double* E_ref, const double* F_ref,
                          const double* W_ref, double* report, void* stream);

/* Spherical cut (Section II.E step 3, option (ii): an extrapolative neighborhood is cut out
 * and treated as a non-periodic cluster; the paper's cut radius is 8 A).  For each of the n
 * DEVICE center atoms, every atom j of its configuration and periodic image n (periodic axes
 * only) with |x_j + n H - x_c| < radius: CSR off[n+1] (int64, DEVICE), then per cluster atom
 * its position relative to the center pos[3] (FP64, A; the center itself first, at the
 * origin, then ascending (j, n0, n1, n2)), species type[] and source atom src[] (int64).
 * pos/type/src may all be NULL to query the size; *total (HOST) receives the number of
 * cluster atoms; MTP_ERR_CAPACITY if an output is given and capacity < total.  Needs no
 * model or neighbor list.  Synchronises `stream`. */
mtp_status mtp_cut_clusters(const mtp_batch* batch, const int64_t* centers, int64_t n, double radius,
                            int64_t* off, double* pos, int32_t* type, int64_t* src,
                            int64_t capacity, int64_t* total, void* stream);

/* Loss of eq. 7 and its gradient with respect to theta:
 *   L = sum_k [ w_e (E_k - E*_k)^2 + w_f sum_i |F_ik - F*_ik|^2 + w_s sum_ab (W_k,ab - W*_k,ab)^2 ].
 * DEVICE inputs E_ref[n_cfg], F_ref[N x 3], W_ref[n_cfg x 9] (NULL allowed if w_s == 0);
 * DEVICE outputs loss[1] and grad[m] (FP64).  The force and stress terms use a
 * forward-over-reverse tangent pass through the hand-written adjoint. */
mtp_status mtp_train_step(mtp_model* model, const mtp_batch* batch, const mtp_nbr* nbr,
                          mtp_precision prec, const double* E_ref, const double* F_ref,
                          const double* W_ref, double w_e, double w_f, double w_s, double* loss,
                          double* grad, void* stream);

/* Arithmetic peak of the current GPU by the library's own microbenchmark (no counterpart in
 * the paper; the denominators of the kernels' roofline fractions): kind 0 = FP32 FMA, 1 = FP64
 * FMA (8 independent FMA chains per thread, full occupancy), 2 = TF32 tensor-core MMA
 * (tcgen05.mma.kind::tf32, M 128, N 256, K 8, one issuing thread per SM, operands fixed in
 * shared memory).  HOST out tflops (2 flops per multiply-add) and ms (best of three timed runs
 * after one warm-up, CUDA events on `stream`).  Synchronises `stream`. */
mtp_status mtp_measure_peak(int kind, double* tflops, double* ms, void* stream);

/* ---------------------------------------------------------------------------------- */
/* Tracing (no counterpart in the paper)                                              */
/* ---------------------------------------------------------------------------------- */

/* Enable (on != 0) or disable kernel-level tracing: while enabled, every kernel region
 * the library launches records a CUDA event pair on the stream it runs on. */
mtp_status mtp_profiler_enable(int on);

/* Synchronise the recorded events, then report per region name (in order of first
 * appearance, at most `capacity` regions): names[48*k] (NUL-terminated), total device
 * time ms[k] and launches[k] = launches of the library's own kernels inside the region (the
 * CUB scan, sort and select kernels it also runs are not counted); *count = regions written.
 * Clears the record.  Host arrays; any of names/ms/launches may be NULL. */
mtp_status mtp_profiler_read(int32_t capacity, char* names, double* ms, int64_t* launches, int32_t* count);

#ifdef __cplusplus
}
#endif

#endif /* MTP_H */

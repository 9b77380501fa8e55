/*
 * soapgap.h -- C ABI of the GB300 library for the separable-density SOAP descriptor
 * and the GAP energy / forces / virial built on it (Caro, arXiv:1905.02142).
 *
 * Problem statement (Sec. I-IV of the paper): given periodic structures (Cartesian
 * positions, lattice vectors, species), a cutoff r_cut, basis sizes n_max, l_max and the
 * atom widths, compute for every atom i
 *   c_nlm(i)  the expansion coefficients of its smoothed neighbour density (Eqs. 01, 05,
 *             08, 15; the density smoothing of Sec. III.B; the radial recursion Eq. 04),
 *   p_nn'l(i) = sum_m c_nlm c_n'lm   (Eq. 09),   q(i) = p(i) / |p(i)|   (Sec. I),
 *   eps_i     = sum_s alpha_s (q_i . q_s)^zeta  over a sparse set (Sec. IV.A),
 * the energy of each structure, the forces -dE/dx and the virial -dE/dstrain; and, for
 * fitting the alpha_s (Sec. IV.A), the kernel rows k(i, s) = (q_i . q_s)^zeta, their sums
 * over each structure and their derivatives with respect to every position
 * (soapgap_design, soapgap_kernel_rows).
 *
 * Conventions
 *   - Lengths in Angstrom.  cell rows are the lattice vectors.  Positions may lie anywhere:
 *     the neighbour search maps an atom whose fractional coordinates are outside
 *     [-1e-9, 1 + 1e-9) into its cell (x - n h) first, and atoms already inside are used
 *     exactly as given.  A non-finite position gives SOAPGAP_E_INVALID_ARG.
 *   - Neighbours: every atom j in every periodic image S with |x_j + S.h - x_i| < r_cut
 *     (strict), except (i, i, S = 0); atom i itself enters once as the central term.
 *   - Species map to separate density channels: channel = species(j) * n_max + n.
 *   - Angular functions are real spherical harmonics; p is identical to Eq. 09's.
 *   - Packed descriptor layout (length D = n_ch (n_ch+1)/2 * (l_max+1), n_ch = n_species
 *     * n_max): for each channel pair c1 <= c2 (row-major upper triangle) and each
 *     l = 0..l_max, p[c1][c2][l] times sqrt(2) when c1 != c2, so that dot products of
 *     packed vectors equal the full sums over (n, n', l).  q uses this layout.
 *   - Virial: W_ab = -sum over pairs (dE/dr_ij)_a (r_ij)_b  (= -dE/dstrain_ab).
 *
 * Precision (soapgap_params.precision)
 *   SOAPGAP_FP64  every step in FP64: the radial recursion per pair in the primitive basis,
 *                 the orthonormalisation W = S^-1/2 per atom, FP64 GEMM for the GAP kernel.
 *   SOAPGAP_MIXED pair and power-spectrum kernels in FP32 with radial functions taken from
 *                 FP64-built tables of the orthonormal-basis coefficients (the adjoint's
 *                 with coarser nodes: it only feeds forces and virial); GAP products on the
 *                 tensor cores with FP32 accumulation; FP64 per-structure sums.
 *   Float outputs typed "real" below are float for MIXED and double for FP64.
 *
 * Errors: every call returns 0 (SOAPGAP_OK) or a negative code; soapgap_last_error()
 * returns a message for the last failure on that handle.  No call throws.
 * Memory: the caller owns every input and output buffer.  The handle owns a device
 * workspace that grows on demand and lives until soapgap_destroy.
 * Streams: device work is enqueued on the caller's stream.  soapgap_compute and
 * soapgap_backward synchronise that stream once (to size the pair list) and again at
 * the end to report device-side errors.
 */
#ifndef SOAPGAP_H
#define SOAPGAP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* return codes */
#define SOAPGAP_OK 0
#define SOAPGAP_E_INVALID_ARG (-1) /* bad pointer, size, parameter, non-finite position */
#define SOAPGAP_E_UNSUPPORTED (-2) /* n_max or l_max outside the supported range, a
                                      batch of 2^28 atoms or more (n_atoms n_species < 2^30),
                                      or one whose pair list may reach 2^31 pairs (atoms x
                                      per-atom neighbour slots, about 1.3 x the densest
                                      structure's neighbours + 32) */
#define SOAPGAP_E_CAPACITY (-3)    /* a fixed-size buffer is too small (see message)    */
#define SOAPGAP_E_CUDA (-4)        /* a CUDA runtime call or kernel failed              */
#define SOAPGAP_E_STATE (-5)       /* call order violated (no model / no forward pass)  */

/* precision */
#define SOAPGAP_FP64 0
#define SOAPGAP_MIXED 1

/* soapgap_compute flags */
#define SOAPGAP_DESC 1u   /* write q and |p|                            */
#define SOAPGAP_ENERGY 2u /* write e_atom and e_struct (needs a model)  */
#define SOAPGAP_FORCES 4u /* write forces (needs a model)               */
#define SOAPGAP_VIRIAL 8u /* write virial (needs a model)               */
#define SOAPGAP_TIMING 16u /* record per-stage device times (soapgap_stage_times) */
#define SOAPGAP_ASYNC 32u  /* no allocation and no host synchronisation: capturable in a
                              CUDA graph (see soapgap_compute)                         */

/* soapgap_design flags (rows of the sparse-GAP fitting matrices) */
#define SOAPGAP_DESIGN_K 64u       /* kernel rows k_atom                        */
#define SOAPGAP_DESIGN_KSTRUCT 128u /* per-structure energy rows k_struct       */
#define SOAPGAP_DESIGN_DK 256u     /* force rows dk                             */

/* Stages reported by soapgap_design_times, in this order. */
#define SOAPGAP_N_DESIGN_STAGES 4  /* descriptors (neighbours to q), kernel_rows (with the
                                      per-structure sums), jacobian, force_rows */

/* Stages reported by soapgap_stage_times, in this order. */
#define SOAPGAP_N_STAGES 7 /* neighbours, pair_forward, power_spectrum, gap_forward,
                              gap_backward, pair_adjoint, finish */

/* Limits: 2 <= n_max <= 12 (the basis degenerates beyond 12, Sec. III.A),
 * 0 <= l_max <= 12, 1 <= n_species <= 8. */
#define SOAPGAP_MAX_NMAX 12
#define SOAPGAP_MAX_LMAX 12
#define SOAPGAP_MAX_SPECIES 8

/* Hyperparameters (Eq. 15 and Sec. III.A-B).
 *   r_cut          hard cutoff r_hard (> 0)
 *   r_soft         start of the buffer zone, 0 < r_soft <= r_cut (== r_cut: no buffer)
 *   sigma_r0       sigma_{0,r} (> 0), also the width of the Gaussian basis function
 *   sigma_p0       sigma_{0,perp} (> 0)
 *   alpha_r        d sigma_r / d r_j  (>= 0)
 *   alpha_p        d sigma_perp / d r_j (>= 0)
 *   amp_a          exponent a of the amplitude polynomial (>= 0)
 *   n_f            filter parameter of the buffer zone (> 0; the paper uses 4)
 *   central_weight weight of the central atom's own Gaussian (1 = counted once)
 *   eq08_weight    0: angular weight 4 pi e^{-z} i_l(z) (projection of the Kaufmann
 *                  expansion); 1: Eq. 08 as printed, with an extra (2l+1).            */
typedef struct soapgap_params {
    double r_cut, r_soft;
    double sigma_r0, sigma_p0, alpha_r, alpha_p, amp_a, n_f, central_weight;
    int32_t n_max, l_max, n_species;
    int32_t precision;   /* SOAPGAP_FP64 or SOAPGAP_MIXED */
    int32_t eq08_weight; /* 0 or 1 */
} soapgap_params;

/* A batch of periodic structures stored back to back.
 *   atom_offs_host [n_struct+1] host int64, atom_offs_host[0] = 0, nondecreasing,
 *                  atom_offs_host[n_struct] = n_atoms; atoms of structure s are
 *                  atom_offs_host[s] .. atom_offs_host[s+1]-1
 *   cell_host      [n_struct][3][3] host double, rows = lattice vectors, det != 0
 *   pos            [n_atoms][3] DEVICE double, Cartesian (see the conventions above)
 *   species        [n_atoms] DEVICE int32 in [0, n_species)                          */
typedef struct soapgap_batch {
    int32_t n_struct;
    int32_t n_atoms;
    const int64_t* atom_offs_host;
    const double* cell_host;
    const double* pos;
    const int32_t* species;
} soapgap_batch;

typedef struct soapgap_handle soapgap_handle;

/* Create a handle: validates the parameters, builds W = S^-1/2 in FP64 on the host
 * (Sec. III.A) and, for MIXED, the radial table on the device.  *out is NULL on error. */
int soapgap_create(const soapgap_params* params, soapgap_handle** out);

/* The radial orthonormaliser W = S^-1/2 of Sec. III.A for (n_max, r_cut, sigma_r0), as the
 * handle uses it: W [n_max][n_max] HOST double, row-major (g_n = sum_a W[n][a] phi_a).
 * S is built and diagonalised in binary128 on the host and W rounded to FP64; no device
 * work.  SOAPGAP_E_UNSUPPORTED if n_max is outside [2, 12] or S is not positive definite. */
int soapgap_orthonormaliser(int32_t n_max, double r_cut, double sigma_r0, double* W);

/* Packed descriptor length D. */
int soapgap_descriptor_dim(const soapgap_handle* h, int32_t* dim);

/* Set the GAP model (Sec. IV.A): q_sparse [M][D] host double, packed layout, each row a
 * normalised descriptor; alpha [M] host double; zeta > 0.  Copies to the device and
 * synchronises.  M >= 1.  SOAPGAP_E_INVALID_ARG for a NULL pointer, M < 1, zeta <= 0 or a
 * non-finite entry; the handle keeps its previous model then.  Past those checks the
 * previous model is dropped first, so after any later failure (SOAPGAP_E_CUDA) the handle
 * has none and calls that need one return SOAPGAP_E_STATE.  A new model requires a new
 * ENERGY evaluation before soapgap_backward. */
int soapgap_set_model(soapgap_handle* h, const double* q_sparse, const double* alpha,
                      int32_t m, double zeta);

/* Forward evaluation on `stream` (a cudaStream_t, NULL = default stream).
 * flags: any of SOAPGAP_DESC | ENERGY | FORCES | VIRIAL.  Outputs are DEVICE pointers;
 * a NULL output is skipped, but every output selected by `flags` must be non-NULL:
 *   q        [n_atoms][D] real      pnorm   [n_atoms] real   (|p| per atom)
 *   e_atom   [n_atoms] real         e_struct [n_struct] double
 *   forces   [n_atoms][3] double    virial  [n_struct][3][3] double
 * With ENERGY the handle keeps what soapgap_backward needs. */
int soapgap_compute(soapgap_handle* h, const soapgap_batch* batch, uint32_t flags,
                    void* q, void* pnorm, void* e_atom, double* e_struct, double* forces,
                    double* virial, void* stream);

/* Asynchronous evaluation (flags | SOAPGAP_ASYNC, not with SOAPGAP_TIMING).  The call enqueues
 * its work on `stream` and returns without waiting: it allocates nothing and never
 * synchronises, so it may be captured in a CUDA graph (stream capture) and replayed.
 * Requirements and behaviour:
 *   - an earlier synchronous call on this handle with the same batch shape (n_atoms,
 *     n_struct) and flags must have sized the workspace; otherwise SOAPGAP_E_STATE;
 *   - the neighbour-pair count is not read back.  The pair buffers of the earlier calls
 *     (their size plus 25 %) bound it; if a configuration needs more pairs, every output of
 *     the call is invalid and soapgap_sync_status reports SOAPGAP_E_CAPACITY;
 *   - pos and species are read from their device pointers when the work runs (at every
 *     replay); the cell and atom_offs are taken at call (capture) time through the
 *     handle's pinned staging, so the handle must not be used for another batch shape
 *     between replays of a captured graph;
 *   - a captured graph holds the device buffers of the model it was captured with:
 *     capture again after soapgap_set_model (a larger sparse set reallocates them);
 *   - device-detected errors (non-finite position, coincident atoms, pair capacity) are
 *     reported by soapgap_sync_status, not by the return value. */

/* Wait for `stream` and report the device error word of the last asynchronous call:
 * SOAPGAP_OK, SOAPGAP_E_CAPACITY (pair buffers too small), SOAPGAP_E_INVALID_ARG (atom
 * non-finite position, coincident atoms) or SOAPGAP_E_CUDA; soapgap_last_error has the text. */
int soapgap_sync_status(soapgap_handle* h, void* stream);

/* Autotuner (the paper has no counterpart: it picks launch shapes of this library's kernels).
 * Runs one synchronous ENERGY|FORCES|VIRIAL evaluation of `batch` (device pos/species, as
 * for soapgap_compute; it also sizes the workspace for asynchronous calls), then times on
 * it, stage by stage, the candidates of a tile plan of SOAPGAP_PLAN_LEN entries:
 *   plan[0]  the tensor-core adjoint: 2, 3 or 4 = mma.sync with that many warps (32-pair
 *            batches) per block; 5 = tcgen05 with the per-atom contraction accumulated in
 *            tensor memory (exact class sizes n_max = l_max = 6, 8, 10, 12 only; other sizes
 *            run the mma.sync kernel with 4 warps)
 *   plan[1]  tile configuration of the GAP forward product (columns per tile, pipeline
 *            stages, epilogue warps): 0 = (256, 4, 8), 1 = (128, 6, 4), 2 = (128, 6, 8)
 *   plan[2]  the same for the GAP backward product: 0 = (224, 5, 4), 1 = (128, 6, 4),
 *            2 = (192, 5, 4), 3 = (256, 4, 4), 4 = (160, 6, 4)
 *   plan[3]  the neighbour sweep: 1 = one block per bin, the bin's candidates staged once in
 *            shared memory; 2 = one warp per atom; 0 = per bin for a single structure with at
 *            least 8 bins per SM, else per atom (timed only without a Verlet skin)
 *   plan[4]  the forward pair kernel's neighbour contraction c[n][lm] += b_n a_lm: 1 = FP32
 *            FMA on the lanes; 2 = tensor cores (mma.sync m16n8k16, FP16 hi/lo operands,
 *            three products, FP32 accumulation); 0 = FP32 FMA
 * and keeps the fastest of each for the batch's problem class (basis class, species count,
 * 32-pair batches per atom, power of two of the atom count).  Later calls on the handle
 * in that class use the plan; classes without one use {0 (by pairs per atom), 0, 0, 0, 0}.  The
 * results do not depend on the plan beyond the order of floating-point sums.  `plan` (may
 * be NULL) receives the choice (on the FP64 path only the neighbour sweep is tuned).
 * Synchronises; afterwards soapgap_backward needs a new evaluation. */
#define SOAPGAP_PLAN_LEN 5
int soapgap_autotune(soapgap_handle* h, const soapgap_batch* batch, int32_t* plan, void* stream);

/* Tile plan of the batch's problem class: soapgap_get_plan writes it to plan[SOAPGAP_PLAN_LEN]
 * (the defaults {0, 0, 0, 0, 0} if none was tuned or set); soapgap_set_plan installs one (e.g. read
 * back from a cache of earlier tuning runs).  Both need a synchronous evaluation of this
 * batch on the handle first (its pair count fixes the class): SOAPGAP_E_STATE otherwise;
 * SOAPGAP_E_INVALID_ARG for an entry out of range (plan[0] may also be 0: chosen by the
 * pairs per atom). */
int soapgap_get_plan(soapgap_handle* h, const soapgap_batch* batch, int32_t* plan);
int soapgap_set_plan(soapgap_handle* h, const soapgap_batch* batch, const int32_t* plan);

/* Verlet skin (neighbour-list reuse).  skin >= 0 (A); 0 (the default) builds the list at
 * every call.  With skin > 0 the list holds all pairs within r_cut + skin and is rebuilt only
 * when an atom has moved by skin/2 or more since the positions of the last build (checked on
 * the device at every call), or when the batch shape or a cell changed.  Between rebuilds
 * every pair's separation is recomputed from its (j, S) and the current positions, and pairs
 * beyond r_cut contribute exactly nothing, so results equal those of a fresh list up to the
 * order of floating-point sums.  Asynchronous calls take the decision on the device (and
 * are therefore capturable); the cell and the species must not change between them.
 * soapgap_export_pairs returns the list (pairs within r_cut + skin).  Setting the skin
 * forces a rebuild at the next call. */
int soapgap_set_skin(soapgap_handle* h, double skin);

/* Whether the last soapgap_compute rebuilt the neighbour list: 1 yes, 0 reused (skin),
 * -1 decided on the device (asynchronous call with a skin). */
int soapgap_last_rebuild(const soapgap_handle* h, int32_t* rebuilt);

/* Velocity-Verlet half step for molecular dynamics around the evaluation (units: A, fs,
 * amu, eV; 1 eV/(A amu) = 0.009648533212 A/fs^2), enqueued on `stream` (capturable):
 *   v += (dt/2) F / m                  (drift = 0: the closing kick)
 *   v += (dt/2) F / m;  x += dt v      (drift != 0: kick and drift)
 * Positions are not wrapped (the neighbour search maps them into their cells itself, and
 * unwrapped positions keep a Verlet-skin list valid when atoms cross a cell face).
 * pos [n_atoms][3], vel [n_atoms][3] DEVICE double, updated in place; forces [n_atoms][3]
 * DEVICE double (F = -dE/dx, as written by soapgap_compute); inv_mass [n_atoms] DEVICE
 * double (1/amu).  One step: verlet(drift=1), compute(FORCES), verlet(drift=0). */
int soapgap_verlet(soapgap_handle* h, const soapgap_batch* batch, double* pos, double* vel,
                   const double* forces, const double* inv_mass, double dt, int32_t drift,
                   void* stream);

/* Adjoint of the last ENERGY evaluation on this handle, for the same batch:
 * dE_dEstruct [n_struct] DEVICE double (weights of each structure's energy);
 * grad_pos [n_atoms][3] DEVICE double receives d(sum_s w_s E_s)/dx (i.e. minus the
 * force when w = 1); virial [n_struct][3][3] DEVICE double or NULL.
 * Returns SOAPGAP_E_STATE without a model, or without a preceding ENERGY evaluation
 * under the current model. */
int soapgap_backward(soapgap_handle* h, const soapgap_batch* batch, const double* dE_dEstruct,
                     double* grad_pos, double* virial, void* stream);

/* Rows of the sparse-GAP fitting matrices for a batch of training structures (Sec. IV.A:
 * the weights alpha_s are fitted to the energies and forces of N_t training environments,
 * with the sparse set as basis; kernel of Sec. I), against the sparse set of the last
 * soapgap_set_model (its alpha and the model's energies are not used):
 *   k_atom[i][s]    = k(i, s) = (q_i . q_s)^zeta                      (SOAPGAP_DESIGN_K)
 *   k_struct[t][s]  = sum over the atoms i of structure t of k(i, s) (SOAPGAP_DESIGN_KSTRUCT)
 *   dk[k][a][s]     = d/dx_{k,a} of sum over i in the structure of atom k of k(i, s)
 *                                                                     (SOAPGAP_DESIGN_DK)
 * so that a model with weights alpha has E_t = k_struct[t] . alpha and the force
 * F_{k,a} = -dk[k][a] . alpha.  Layouts: k_atom [n_atoms][M], dk [n_atoms][3][M] DEVICE,
 * float for MIXED, double for FP64; k_struct [n_struct][M] DEVICE double.  Outputs not
 * requested may be NULL.  flags may add SOAPGAP_TIMING (soapgap_design_times).
 * Precision (MIXED): kernel rows from the same split tensor-core products as the energy
 * (relative error ~1e-7, on top of the descriptors' own error); force rows from single FP16
 * products of the centred sparse rows with power-of-two scaled FP16 descriptor Jacobians
 * projected orthogonally to the owner's descriptor (RMS relative error ~1e-4).
 * Workspace: the Jacobian columns, 3 (P + n_atoms) of them for P neighbour pairs, each of
 * D + 2 padded to 64 halves (MIXED) or D doubles (FP64), plus 24 (MIXED) or 40 (FP64)
 * bytes each, and n_atoms x M weights.  Synchronises `stream`; SOAPGAP_E_STATE without a model,
 * SOAPGAP_E_UNSUPPORTED if the descriptor is too large for the Jacobian kernel's shared
 * memory or the column count exceeds 2^31. */
int soapgap_design(soapgap_handle* h, const soapgap_batch* batch, uint32_t flags, void* k_atom,
                   double* k_struct, void* dk, void* stream);

/* Device time in milliseconds of each stage of the last soapgap_design call made with
 * SOAPGAP_TIMING: ms[SOAPGAP_N_DESIGN_STAGES] host double (0 for stages that did not run). */
int soapgap_design_times(const soapgap_handle* h, double* ms);

/* Kernel rows of any descriptors against the sparse set of the last soapgap_set_model:
 * k[i][s] = (q_i . q_s)^zeta.  q [n][D] DEVICE (float for MIXED, double for FP64; rows as
 * written by soapgap_compute with SOAPGAP_DESC), k [n][M] DEVICE of the same type.  With
 * the sparse rows themselves this is the K_MM block of the fit.  Synchronises `stream`. */
int soapgap_kernel_rows(soapgap_handle* h, const void* q, int32_t n, void* k, void* stream);

/* Same as soapgap_compute, but pos/species and every output are HOST pointers; the
 * library copies inputs to its workspace and results back on `stream` and returns
 * after the stream has finished. */
int soapgap_compute_host(soapgap_handle* h, const soapgap_batch* batch, uint32_t flags,
                         void* q, void* pnorm, void* e_atom, double* e_struct, double* forces,
                         double* virial, void* stream);

/* Device time in milliseconds of each stage of the last soapgap_compute call made with
 * SOAPGAP_TIMING (CUDA events recorded on the caller's stream): ms[SOAPGAP_N_STAGES] host
 * double; stages that did not run report 0.  SOAPGAP_E_STATE if timing was not on. */
int soapgap_stage_times(const soapgap_handle* h, double* ms);

/* Diagnostic: C = A B^T on the tensor cores with the library's tcgen05 GEMM (the kernel
 * behind the mixed-precision GAP products).  A [m][k], B [n][k] DEVICE FP16 row-major
 * (k a multiple of 64; rows 16-byte aligned), C [m][n] DEVICE float.  Uses the handle's
 * error word; synchronises `stream`. */
int soapgap_tc_gemm_f16(soapgap_handle* h, const void* a, int32_t m, const void* b, int32_t n,
                        int32_t k, float* c, void* stream);

/* Number of kernels the last soapgap_compute / soapgap_backward call launched. */
int soapgap_last_launch_count(const soapgap_handle* h, int64_t* n);

/* Number of neighbour pairs found by the last compute call (diagnostics). */
int soapgap_last_pair_count(const soapgap_handle* h, int64_t* n_pairs);

/* Copy the pair list of the last synchronous list build to HOST arrays, in canonical order
 * (centre, neighbour species, neighbour, then shift S lexicographically):
 *   centre[P], neighbour[P] int32 atom indices; shift[P][3] int32 image S (x_j + S.h).
 * With a Verlet skin the list holds the pairs within r_cut + skin of its build.
 * `capacity` is the length of the arrays; SOAPGAP_E_CAPACITY if it is below P.
 * SOAPGAP_E_STATE if no synchronous call has completed a list since the last failed or
 * asynchronous rebuild. */
int soapgap_export_pairs(soapgap_handle* h, int64_t capacity, int32_t* centre,
                         int32_t* neighbour, int32_t* shift);

/* GAP local energies eps_i = sum_s alpha_s (q_i . q_s)^zeta for callers that cannot
 * allocate device memory.  The paper has no counterpart: this is a service of the library.
 * Who needs it: applications that own all device memory through their own pool and forbid
 * other allocations, and loops that cannot accept the device-wide synchronisation that
 * cudaMalloc/cudaFree may cause.  The call allocates nothing (no cudaMalloc, cudaFree or
 * allocating library routine): its scratch, n * ceil(m/64) floats of per-tile partial
 * sums, lives in a fixed 16 MiB array in the library's device memory, which every GPU
 * that loads the library keeps until the process exits.
 *   q [n][d], q_sparse [m][d], alpha [m], e_atom [n]: DEVICE float (MIXED layout of q);
 *   zeta > 0; work is enqueued on `stream` (a cudaStream_t, NULL = default stream).
 * Returns SOAPGAP_E_CAPACITY, before any device work, when n * ceil(m/64) > 4194304 or
 * n > 4194240 (65535 rows of 64 atoms, the launch grid's limit).
 * The first call on each device looks up the array's device address (cudaGetSymbolAddress)
 * with that device current; make that first call before any stream capture.  A device
 * reset destroys the array with its context: the next call on that device, in the new
 * context, looks the address up again (it must then also come before any capture).
 * All calls share the one array and it keeps the last call's contents (each call writes
 * every entry it reads, so nothing needs clearing); calls that overlap on the GPU, on
 * different streams of the same device, race on it. */
int soapgap_gap_energy_noalloc(const float* q, const float* q_sparse, const float* alpha,
                               int32_t n, int32_t m, int32_t d, double zeta, float* e_atom,
                               void* stream);

/* Number of FP16 products of the mixed path's GAP energy (Sec. IV.A, eps_i = sum_s alpha_s
 * (q_i . q_s)^zeta on the tensor cores; the paper has no GPU design to follow here).  The
 * products are taken about the sparse-set mean, q = qbar + n u, as u_i . u_s on FP16
 * operands: one product hi.hi, or three, hi.hi + hi.lo + lo.hi, with u = hi + lo.  At
 * soapgap_set_model the library evaluates the local energies of the sparse rows themselves
 * with one product and with three, and uses one product when their relative difference
 * (|d eps|_2 / |eps|_2) is at most 1e-5, ten times below the 1e-4 energy bar; otherwise three.
 * soapgap_set_gap_terms(h, terms): 0 = that automatic choice (default), 1 or 3 = forced; it
 * applies to the current model and to later ones; SOAPGAP_E_INVALID_ARG for other values.
 * soapgap_gap_terms(h, &terms, &probe_err): the number in use (0 without a mixed-precision
 * model) and the measured one-product error (-1 without one; probe_err may be NULL).
 * The kernel rows of the fitting matrices always take three products; the FP64 path has none. */
int soapgap_set_gap_terms(soapgap_handle* h, int32_t terms);
int soapgap_gap_terms(const soapgap_handle* h, int32_t* terms, double* probe_err);

/* Arithmetic peak of the current device, measured (the paper has no counterpart: this is
 * the denominator of the roofline reported for the pair kernels and the FP64 path).
 * kind SOAPGAP_PEAK_FP32_FMA or SOAPGAP_PEAK_FP64_FMA: a kernel of independent fused
 * multiply-add chains on every SM (8 blocks of 256 threads per SM), timed with CUDA events
 * on `stream` (a cudaStream_t, NULL = default stream), best of three launches after one
 * warm-up.  Writes *tflops (TFLOP/s, one FMA = 2 flop) and, if sm_count is not NULL, the
 * device's SM count.  Synchronises `stream`; runs for a few tens of milliseconds.
 * SOAPGAP_E_INVALID_ARG for an unknown kind or a NULL tflops. */
#define SOAPGAP_PEAK_FP32_FMA 0
#define SOAPGAP_PEAK_FP64_FMA 1
int soapgap_measure_alu_peak(int32_t kind, double* tflops, int32_t* sm_count, void* stream);

/* Message describing the last error on h ("" if none); valid until the next call. */
const char* soapgap_last_error(const soapgap_handle* h);

/* Release the handle and its workspace (NULL is ignored). */
void soapgap_destroy(soapgap_handle* h);

#ifdef __cplusplus
}
#endif
#endif /* SOAPGAP_H */

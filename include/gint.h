/*
 * gint.h -- C ABI of the GB300 real-space grid integration library (libgint.so).
 *
 * The library evaluates the three-centre grid integrals of numerical-atomic-
 * orbital DFT that the paper (arXiv 2409.09399, Section 2.2) identifies as the
 * grid-integration hot path, on one NVIDIA GB300 (sm_103a):
 *
 *   H^V_IJ(T)[mu,nu] = sum_g sum_T1 phi_Imu(r_g - R_I - T1) V_g
 *                                    phi_Jnu(r_g - R_J - T1 - T) dV      (Eq. 2)
 *   rho_g            = sum over neighbour pairs ((I,T1),(J,T2)) of
 *                      phi_Imu(r_g-R_I-T1) D_IJ(T2-T1)[mu,nu] phi_Jnu(r_g-R_J-T2)  (Eq. 3)
 *   F_I              = -dE/dR_I at fixed V, E = sum_g V_g rho_g dV        (Eq. 4)
 *   sigma            = -(1/Omega) dE/d(strain) at fixed V_g and dV        (Eq. 5)
 *
 * Conventions (all calls):
 *   - Units: bohr and hartree.  Cell rows are the lattice vectors a1, a2, a3.
 *   - Grid: r_g = sum_i (g_i/n_i) a_i, g_i in [0, n_i); dV = Omega/(n1 n2 n3).
 *     Grid arrays (V, rho) are float64, C order [n1][n2][n3] (g3 fastest).
 *   - Basis: phi = R_l(|d|) Y_lm(d/|d|) for |d| < rc of the atom's species,
 *     R the cubic Hermite interpolant of the tabulated (y_k, y'_k) on knots
 *     r_k = k*dr; Y_lm real, normalised, no Condon-Shortley phase, l <= 3.
 *     Orbitals of an atom are ordered: l ascending, then radial functions in
 *     the order given, then m = -l..l.
 *   - Sparse matrices (H, D) live on the pair pattern: every block (I, J, T)
 *     with |R_J + T - R_I| < rc_I + rc_J (Section 2.2: the pairs with
 *     overlapping cutoff radii), sorted by (I, J, t1, t2, t3), T = sum t_i a_i.
 *     Block b is row-major nw_I x nw_J float64 at offsets[b] (in elements).
 *   - Device pointers are CUDA device (or managed) memory of the device the
 *     handle was created on; the caller owns them.  The handle owns its
 *     pattern, bricks, tables and scratch.
 *   - Every compute call is asynchronous on the given stream (0 = legacy
 *     default stream).  Arguments are validated on the host before anything is
 *     enqueued; a failed call enqueues nothing and returns a status.  No call
 *     traps or aborts.  Device-side anomalies raise a flag that gint_sync()
 *     reports.
 *   - A handle is not thread safe: calls on one handle must not overlap in
 *     time on the host, and kernels from two calls on one handle must not run
 *     concurrently on the device (they share the handle's scratch).
 */
#ifndef GINT_H
#define GINT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gint_handle gint_handle;
/* Same type as cudaStream_t; 0 is the legacy default stream. */
typedef struct CUstream_st* gint_stream;

typedef enum {
    GINT_OK = 0,
    GINT_ERR_INVALID_ARG = 1,      /* a null pointer, a size out of range, bad tables */
    GINT_ERR_CUDA = 2,             /* a CUDA runtime call failed; see gint_last_error() */
    GINT_ERR_OOM = 3,              /* device memory allocation failed */
    GINT_ERR_PATTERN_MISMATCH = 4, /* a pair met on the grid is missing from the pattern */
    GINT_ERR_TIMEOUT = 5,          /* a bounded device wait gave up */
    GINT_ERR_UNSUPPORTED = 6,      /* a precision or basis this build does not implement */
    GINT_ERR_DEVICE = 7            /* a device-side check failed; see gint_last_error() */
} gint_status;

/* Arithmetic of the per-batch work.  In every form the atom-to-brick offsets,
 * the accumulation of batch results into H, rho, F and sigma, and the final
 * reductions are FP64; the forms differ in the orbital values and the batch
 * contractions.  GINT_FP64 is the plain FP64 form. */
typedef enum {
    GINT_FP64 = 0,
    GINT_FP32 = 1,     /* FP32 orbital values and FP32 SIMT contractions */
    GINT_TF32 = 2,     /* not implemented (GINT_ERR_UNSUPPORTED): TF32 keeps 10 mantissa bits per
                          operand and accumulates in FP32 like the 16-bit splits, so it has their
                          accumulation bias without their 22-bit operands */
    GINT_BF16X3 = 3,   /* H^V, rho and force on the tensor cores: operands split
                          x = hi + lo in bf16, products hi*hi + hi*lo + lo*hi, FP32
                          accumulation per brick (H^V) or per 128-point tile (rho, force) */
    GINT_BF16X6 = 4,   /* not implemented (GINT_ERR_UNSUPPORTED): a three-piece split with six
                          products; GINT_FP16X4 below is the ~FP32-accurate split this library
                          provides (its leading term accumulates exactly, which a six-product
                          bf16 split would not) */
    GINT_FP16X3 = 5,   /* as GINT_BF16X3 with fp16 pieces (22-bit products) */
    GINT_FP16X4 = 6    /* tensor cores, exact leading term: each operand value x is written
                          x / q = n + l1 + l2 with q a power of two (per orbital for the
                          orbital values, per (atom, orbital row) for D), n an integer of
                          <= 8 bits (exact in fp16) and l1, l2 fp16 pieces of the rest;
                          the products n*n accumulate exactly in FP32, the cross terms
                          n*l1 + l1*n + l1*l1 + n*l2 + l2*n in a second FP32 accumulator */
} gint_precision;

/* One tabulated radial function R(r): y[k] = R(k*dr), dy[k] = R'(k*dr),
 * k = 0..n_knots-1.  Host pointers, read during gint_setup only. */
typedef struct {
    int l;              /* angular momentum, 0..3 */
    int n_knots;        /* >= 2 */
    double dr;          /* knot spacing (bohr), > 0; the same for all radials of a species */
    const double* y;    /* n_knots values */
    const double* dy;   /* n_knots derivatives (required) */
} gint_radial;

typedef struct {
    double rc;                 /* cutoff radius (bohr); the table must cover [0, rc] */
    int n_radial;              /* 1..16 */
    const gint_radial* radial; /* n_radial entries; all with the same dr and n_knots */
} gint_species;

typedef struct {
    int precision;   /* gint_precision */
    int brick[3];    /* grid points per batch along a1, a2, a3; 0 = default (8, 8, 8).
                        The product must be <= 2048. */
    int device;      /* CUDA device ordinal; -1 = current device */
    int reserved[5]; /* must be zero */
} gint_options;

/* Create a handle: uploads geometry and tables, builds the pair pattern
 * (Section 2.2) and the batch/atom neighbour lists (Section 2.3.2) on the
 * device.  Synchronous.
 *   n_atoms  >= 1; pos[n_atoms][3] (host, bohr); species[n_atoms] (host) in [0, n_species);
 *   cell[9] (host) rows a1, a2, a3 (bohr), right- or left-handed, non-singular;
 *   sp[n_species] (host); grid[3] (host) each >= 1;
 *   opt may be NULL for defaults; out receives the handle (NULL on failure). */
gint_status gint_setup(int n_atoms, const double* pos, const int* species, const double* cell,
                       int n_species, const gint_species* sp, const int* grid,
                       const gint_options* opt, gint_handle** out);

/* Release a handle and all device memory it owns.  NULL is a no-op. */
void gint_destroy(gint_handle* h);

/* The pair pattern.  *blocks points to device memory holding n_blocks rows of
 * (I, J, t1, t2, t3) int32; *offsets to device memory holding n_blocks+1 int64
 * element offsets (offsets[n_blocks] = n_values).  Both stay owned by the
 * handle and valid until gint_destroy or gint_update_positions.  Any output
 * pointer may be NULL. */
gint_status gint_pattern(const gint_handle* h, int64_t* n_blocks, int64_t* n_values,
                         const int32_t** blocks, const int64_t** offsets);

/* Select the arithmetic of later calls (gint_precision).  Host only: it sets
 * a field of the handle and touches no device memory, so a caller may give
 * each call its own form (every per-form table, such as the tensor-core copy
 * of D, is made inside the call that uses it).  Calls already enqueued keep
 * the form they were enqueued with.  GINT_ERR_INVALID_ARG for an unknown
 * value; whether the handle's bricks suit a tensor-core form is reported by
 * gint_check and by the compute calls. */
gint_status gint_set_precision(gint_handle* h, int precision);

/* H^V (Eq. 2).  V: device [n1][n2][n3] float64.  H: device, n_values float64
 * on the pattern.  accumulate = 0 overwrites H; accumulate = 1 adds into the
 * canonical blocks (I < J, or I == J and T >= 0 lexicographically) and then
 * rewrites every other block as the transpose of its mirror, so H must be
 * symmetric (H_JI(-T) = H_IJ(T)^T) on entry. */
gint_status gint_vlocal(gint_handle* h, const double* V, double* H, int accumulate, gint_stream stream);

/* rho (Eq. 3).  D: device, n_values float64 on the pattern; it must be
 * symmetric (D_JI(-T) = D_IJ(T)^T): only the canonical blocks are read.
 * rho: device [n1][n2][n3] float64, every element written. */
gint_status gint_rho(gint_handle* h, const double* D, double* rho, gint_stream stream);

/* Pulay force and stress (Eq. 4, 5) of E = sum_g V_g rho_g[D] dV at fixed V.
 * V, D as above (D symmetric, canonical blocks read).  Outputs (device, float64,
 * every non-NULL one overwritten):
 *   F[n_atoms][3]            F_I = -dE/dR_I
 *   sigma[3][3]              -(1/Omega) dE/d(eps_ab), eps a homogeneous strain
 *                            applied to atoms, images and grid points alike
 *   virial_atom[n_atoms][3][3]  per-atom parts Pi_I with sigma = -sum_I Pi_I / Omega
 *   E[1]                     sum_g V_g rho_g dV
 * At least one output must be non-NULL. */
gint_status gint_force_stress(gint_handle* h, const double* V, const double* D, double* F,
                              double* sigma, double* virial_atom, double* E, gint_stream stream);

/* Gradients of the grid energy E = sum_g V_g rho_g[D] dV = sum_blocks D . H^V (Eq. 2-5), the
 * adjoint of the three calls above, each output re-evaluating the orbital values (nothing is
 * kept from an earlier call):
 *   dE_dR[n_atoms][3]   dE/dR_I = -F_I                        (Eq. 4, at fixed V and D)
 *   dE_deps[3][3]       dE/d(eps_ab) = sum_I Pi_I = -Omega sigma  (Eq. 5, homogeneous strain of
 *                       atoms, images and grid points at fixed V_g and dV)
 *   dE_dV[n1][n2][n3]   dE/dV_g = rho_g dV                    (Eq. 3)
 *   dE_dD (n_values)    dE/dD = H^V on every block of the pattern (Eq. 2)
 *   E[1]                E itself (not scaled)
 * Every gradient is multiplied by *grad_E (a device scalar, the upstream gradient of a
 * reverse-mode chain; NULL means 1).  All pointers are device memory of the handle's device;
 * NULL outputs are skipped, at least one must be non-NULL.  V and D as for gint_force_stress
 * (D symmetric, canonical blocks read).  With a brick selection (gint_select_bricks) E and its
 * gradients are those of the selected bricks' grid points (dE_dV is zero elsewhere).  Errors
 * as for gint_force_stress. */
gint_status gint_energy_grads(gint_handle* h, const double* V, const double* D, const double* grad_E, double* dE_dR,
                              double* dE_deps, double* dE_dV, double* dE_dD, double* E, gint_stream stream);

/* New atom positions (and optionally a new cell) for an existing handle: the pair pattern,
 * the atom images, the brick lists, pair tables and tile masks are rebuilt for the new
 * geometry in place (the handle pointer stays valid); the grid dimensions, species tables,
 * precision, brick shape, brick selection and wait limit are kept.  This is the step of the
 * ionic loop of the paper's Fig. 1 between two force evaluations.
 *   pos[n_atoms][3] (host, bohr); cell[9] (host) or NULL to keep the cell.
 *   keep_pattern = 1: the new geometry must have exactly the same pattern (so D and H laid
 *     out on it stay valid, e.g. for small displacements); if it does not, nothing changes and
 *     GINT_ERR_PATTERN_MISMATCH is returned.
 *   keep_pattern = 0: the pattern may change; *pattern_changed (may be NULL) is set to 1 if it
 *     did (then gint_pattern gives the new block list and offsets).
 * Synchronous (waits for the device).  On any error the handle is unchanged.  Batches made
 * from the handle before the call are stale: gint_batch_run rejects them. */
gint_status gint_update_positions(gint_handle* h, const double* pos, const double* cell, int keep_pattern,
                                  int* pattern_changed);

/* Restrict later calls to a subset of the bricks (the batches of grid points of Section 2.3.2),
 * the unit of work that the paper's task decomposition deals to processes (Section 2.3.1,
 * Fig. 5).  Brick b covers grid points [b0 B0, (b0+1) B0) x [b1 B1, ...) x [b2 B2, ...) with
 * b = (b0 nb1 + b1) nb2 + b2, nb_i = ceil(n_i / B_i), B the brick shape (gint_get_info).
 *   bricks: host array of n brick ids in [0, nb0 nb1 nb2) (duplicates allowed), or NULL for every
 *   brick (the default).
 * With a selection, gint_vlocal and gint_force_stress return the contributions of the selected
 * bricks' grid points only (the results of disjoint selections covering the grid add up to the
 * full results), and gint_rho writes rho on the selected bricks' points only (other elements are
 * left untouched).  Synchronous; GINT_ERR_INVALID_ARG for an id out of range. */
gint_status gint_select_bricks(gint_handle* h, int64_t n, const int64_t* bricks);

/* Work of every brick, for partitioning the bricks by cost: n_images[b] (host, one entry per
 * brick, n_bricks of gint_get_info) = number of atom images whose cutoff sphere meets brick b. */
gint_status gint_brick_loads(const gint_handle* h, int64_t* n_images);

/* Number of polls after which a wait of the tensor-core pipelines (producers, copies and MMA
 * issue handing buffers to one another) gives up: the kernel then stops its work, raises a
 * flag that gint_sync reports as GINT_ERR_TIMEOUT, and returns.  0 = the default (2^26 polls,
 * far above any normal wait).  The waits that drain the tensor pipe before tensor memory is
 * released always use the default.  Host only. */
gint_status gint_set_wait_limit(gint_handle* h, int64_t polls);

/* Test hook: the n-th device allocation the library makes from now on (n >= 1) fails the way
 * cudaMalloc fails on a full device, so that out-of-memory paths can be exercised without
 * filling a GPU; 0 disables.  Process-wide.  gint_setup then returns GINT_ERR_OOM having
 * released everything it allocated. */
gint_status gint_debug_fail_alloc(int n);

/* The local potential from rho, the step of Fig. 1 that precedes the grid integrals (Section
 * 2.2, the text after Eq. 2: V is the sum of the local pseudopotentials, the Hartree and the
 * exchange-correlation potentials):
 *   V_out = V_ext + V_H + v_xc,
 *   V_H:  periodic solution of lap V_H = -4 pi (rho - mean rho) on the handle's grid and cell,
 *         V_H(G) = 4 pi rho(G) / |G|^2 with V_H(G = 0) = 0 (on the Nyquist index of an even axis
 *         the kernel is the mean over G and -G, which keeps V_H real);
 *   v_xc: LDA, Slater exchange + Perdew-Zunger (1981) correlation, spin unpolarised, in hartree;
 *         0 where rho <= 0;
 *   energies[0] = E_H = 1/2 sum_g rho_g V_H,g dV, energies[1] = E_xc = sum_g rho_g eps_xc,g dV.
 * rho, V_ext, V_out, V_H: device grid arrays [n1][n2][n3] float64; V_ext may be NULL (zero);
 * V_H may be NULL (not returned) and otherwise must not alias rho; V_out must not alias rho;
 * energies: device double[2] or NULL.  rho is read only.  The two 3-D FFTs are cuFFT's,
 * loaded at run time (GINT_ERR_UNSUPPORTED if libcufft cannot be loaded); the first call on a
 * handle makes the FFT plans and a half-spectrum buffer (16 (n1 n2 (n3/2 + 1)) bytes), so make
 * it before any stream capture.  Asynchronous on `stream`; grids above 2^31 points are
 * GINT_ERR_UNSUPPORTED.  The brick selection does not apply (the whole grid is used). */
gint_status gint_local_potential(gint_handle* h, const double* rho, const double* V_ext, double* V_out, double* V_H,
                                 double* energies, gint_stream stream);

/* H^V in the FP64 form, like gint_vlocal(h, V, H, 0, stream), without any
 * device allocation.  For callers that cannot let a library call cudaMalloc
 * (it synchronises the device and fails once a framework's caching allocator
 * has reserved the free memory): the kernel's orbital-value scratch is a fixed
 * 64 MiB array inside libgint.  The paper has no counterpart of this call.
 *   - Always FP64, whatever gint_set_precision selected; H is overwritten.
 *   - gint_setup maps the array on the handle's device (cudaGetSymbolAddress,
 *     with that device current), which reserves its 64 MiB there until the
 *     process exits; the call itself only reads the address kept in the handle.
 *     If the mapping failed at set-up, the call returns GINT_ERR_CUDA.
 *   - A brick whose scratch slice exceeds 64 MiB is rejected with
 *     GINT_ERR_UNSUPPORTED (use smaller bricks); with fewer slices than the
 *     handle's CTA count the kernel runs on fewer CTAs.
 *   - Every call, on every handle, shares the one array: calls whose kernels
 *     overlap on the GPU race and give wrong results.  Nothing in the array
 *     needs to start at zero (each brick's slice is written before it is read).
 *   - Calls no cudaMalloc, cudaFree or other allocating routine. */
gint_status gint_vlocal_static(gint_handle* h, const double* V, double* H, gint_stream stream);

/* Bloch sum of H^V (the step after the grid integrals, Section 2.4 setting):
 *   H(k)_{I mu, J nu} = sum over pattern blocks (I, J, t) of exp(2 pi i k . t) H_IJ(t)[mu, nu],
 * k given in fractions of the reciprocal lattice vectors (k . T = 2 pi kfrac . t).
 * H: device, the full block list (as gint_vlocal writes it).  Hk: device, dense
 * n_orbitals x n_orbitals complex matrix, row-major with leading dimension ld (complex
 * elements, ld >= n_orbitals), real and imaginary parts interleaved (complex128); rows
 * and columns in atom order, each atom's orbitals in the pattern's order.  Hk is
 * overwritten.  Asynchronous on `stream`; host validation only. */
gint_status gint_fold_k(const gint_handle* h, const double* H, const double kfrac[3], double* Hk, int64_t ld,
                        gint_stream stream);

/* Whether the kernels of the handle's current precision accept its bricks
 * (the tensor-core forms bound the orbitals, atom images and points of one
 * brick).  GINT_OK, or GINT_ERR_UNSUPPORTED with the limits in
 * gint_last_error(); host only, launches nothing. */
gint_status gint_check(const gint_handle* h);

/* Many cells in one launch (the uneven multi-cell workload: many small
 * periodic cells, each with its own handle).  gint_batch_create takes n
 * handles of one device (the handles must outlive the batch).  gint_batch_run
 * runs, for every cell i, gint_vlocal (if H[i]), gint_rho (if rho[i]) and
 * gint_force_stress (if F[i], sigma[i] or E[i]); the pointer arrays are host
 * arrays of n device pointers (H, rho, F, sigma, E may be NULL as a whole).
 * The first call captures all these calls into one CUDA graph on an internal
 * stream; later calls with the same buffers launch that graph as one unit,
 * ordered after the work already queued on `stream` and before later work on
 * it.  Changing a buffer re-captures.  Errors of the individual calls are
 * reported as they would be by those calls. */
typedef struct gint_batch gint_batch;
gint_status gint_batch_create(int n, gint_handle* const* handles, gint_batch** out);
gint_status gint_batch_run(gint_batch* b, const double* const* V, const double* const* D, double* const* H,
                           double* const* rho, double* const* F, double* const* sigma, double* const* E,
                           gint_stream stream);
void gint_batch_destroy(gint_batch* b);

/* Wait for the handle's work on `stream` and report (then clear) any flag a
 * device-side check raised since the last call. */
gint_status gint_sync(gint_handle* h, gint_stream stream);

/* Statistics of the handle's batches (for tests and benchmarks). */
typedef struct {
    int64_t n_blocks, n_values;   /* pattern size */
    int64_t n_ext_atoms;          /* atom images whose cutoff sphere meets the grid */
    int64_t n_bricks;             /* batches of grid points */
    int64_t n_bricks_nonempty;    /* batches with at least one atom in range */
    int64_t n_brick_atoms;        /* sum over batches of atoms in range */
    int64_t n_brick_pairs;        /* sum over batches of atom pairs in the pattern */
    int max_brick_atoms;          /* largest atom list of one batch */
    int max_brick_orbitals;       /* largest orbital count of one batch */
    int brick[3];
    int precision;
    int64_t scratch_bytes;        /* device scratch owned by the handle */
    int64_t n_orbitals;           /* sum over atoms of their orbitals: the dimension of H(k) */
} gint_info;

gint_status gint_get_info(const gint_handle* h, gint_info* info);

/* Exact work of the grid integrals (for roofline accounting): over every grid
 * point r, n_o(r) = number of orbitals phi_Imu(r - R_I - T) with |r - R_I - T| < rc.
 * Writes sum_r n_o(r) and sum_r n_o(r)^2.  Runs a counting kernel and
 * synchronises the device.  Outputs are host pointers. */
gint_status gint_work_stats(gint_handle* h, int64_t* sum_orbitals, int64_t* sum_orbitals_sq);

/* Message of the last failed call on this host thread.  gint_setup, the
 * compute calls (gint_vlocal, gint_rho, gint_force_stress, gint_vlocal_static,
 * gint_fold_k), gint_check and gint_batch_create/run clear it when they start,
 * so after one of them succeeds it is "". */
const char* gint_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* GINT_H */

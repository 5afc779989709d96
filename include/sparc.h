/*
 * sparc.h — C ABI of the GB300 CheFSI library (libsparc.so).
 *
 * One Chebyshev-filtered subspace iteration (CheFSI) step of real-space
 * Kohn-Sham DFT, as in Algorithm 1 of "GPU acceleration of local and semilocal
 * density functional calculations in the SPARC electronic structure code"
 * (arXiv 2302.09708): Chebyshev filtering, projection, subspace
 * diagonalisation and rotation, with the matrix-free Hamiltonian of Sec. II A
 *
 *   H X = -1/2 Lap X + Veff o X + sum_J chi_J Gamma_J h^3 chi_J^T X ,
 *
 * Lap the 12th-order (radius 6) central finite-difference Laplacian on a
 * uniform grid (periodic or Dirichlet per axis), Veff a diagonal potential and
 * chi_J the Kleinman-Bylander projectors of atom J on its support points.
 *
 * Conventions shared by every call
 *  - Every function returns an int status (sparc_status below); no C++
 *    exception crosses the ABI.  sparc_last_error() gives a message.
 *  - Grid point (i, j, k) has linear index i + nx (j + ny k) (x fastest).
 *  - An orbital block X is an Nd x Ns column-major matrix (one orbital per
 *    column) with leading dimension ld >= Nd elements, of element type dtype
 *    (SPARC_F64 or SPARC_F32); rows Nd..ld-1 are ignored and never written.
 *    Blocks passed to the calls are owned by the caller.  Device pointers
 *    (cudaMalloc, torch.empty(..., device="cuda")) run without staging; where a
 *    call says "device or host", a host pointer is copied through a library
 *    buffer inside the call.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Work is
 *    enqueued on it; calls return without waiting unless stated.  The calls
 *    that wait for the stream before returning are sparc_spectrum_bounds,
 *    sparc_chefsi_step, sparc_subspace_eig, sparc_batch_chefsi_step, the
 *    calls given a host block, and sparc_project / sparc_rotate whenever they
 *    run the tensor-core form (every mixed handle, and FP64 handles without
 *    options flag bit 1).  Kernels that wait on barriers bound every wait; if
 *    one runs out the kernel stops and records SPARC_ERR_TIMEOUT, which the
 *    next of those waiting calls on the handle returns.
 *  - All inputs given at create time are copied; the caller may free them.
 *  - The library owns its workspace (two Nd x ns_max blocks of the working
 *    precision plus the Ns x Ns subspace buffers), sized at create time.
 */
#ifndef SPARC_H
#define SPARC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SPARC_OK = 0,
  SPARC_ERR_INVALID_ARG = 1, /* bad shape, pointer, bound or option           */
  SPARC_ERR_CUDA = 2,        /* a CUDA runtime call failed                     */
  SPARC_ERR_OOM = 3,         /* device allocation failed                       */
  SPARC_ERR_NOT_SPD = 4,     /* the overlap Ms is not positive definite        */
  SPARC_ERR_NUMERIC = 5,     /* NaN/Inf or a non-converging iteration          */
  SPARC_ERR_TIMEOUT = 6      /* a bounded device wait ran out                  */
} sparc_status;

enum { SPARC_PERIODIC = 0, SPARC_DIRICHLET = 1 };
enum { SPARC_F64 = 0, SPARC_F32 = 1, SPARC_C128 = 2 /* complex FP64, (re, im) pairs */ };
enum { SPARC_PREC_FP64 = 0, SPARC_PREC_MIXED = 1 };

typedef struct sparc_context* sparc_handle;

/* Uniform grid: nx, ny, nz >= 1 points, spacing h > 0 (bohr), bc[d] per axis. */
typedef struct {
  int nx, ny, nz;
  double h;
  int bc[3];
} sparc_grid;

/*
 * Nonlocal projectors, per atom J = 0..natoms-1 (Sec. II A: "stored as a dense
 * matrix" per atom and applied to the components of X on its support):
 *  supp_ptr[J]..supp_ptr[J+1]-1  range of atom J's support points in supp_idx
 *  supp_idx[]                    linear grid indices (0 <= idx < Nd)
 *  nproj[J]                      number of projectors of atom J (>= 0)
 *  chi_ptr[J]                    offset of atom J's column-major
 *                                n_supp x nproj[J] block in chi[]
 *  proj_ptr[J]                   offset of atom J's nproj[J] energies in gamma[]
 *  gamma[]                       projector energies Gamma (Ha)
 * natoms = 0 (all pointers may be NULL) gives a purely local Hamiltonian.
 */
typedef struct {
  int natoms;
  const int64_t* supp_ptr;
  const int32_t* supp_idx;
  const int32_t* nproj;
  const int64_t* chi_ptr;
  const double* chi;
  const int64_t* proj_ptr;
  const double* gamma;
} sparc_nonlocal;

typedef struct {
  int precision; /* SPARC_PREC_FP64: FP64 everywhere.  SPARC_PREC_MIXED: FP32
                    orbital storage and filtering, split-precision tensor-core
                    projection/rotation, FP64 bounds/Cholesky/eigensolve.      */
  int ns_max;    /* largest Ns passed to any call on this handle (>= 1)        */
  int device;    /* CUDA device ordinal                                        */
  int flags;     /* bit 0: use the generic stencil kernel instead of the TMA
                    plane-ring form (for cross-checking).
                    bit 1 (FP64 handles): projection and rotation on the FP64
                    SIMT pipe instead of the FP64-accurate six-digit
                    tensor-core split (about 2^-45 relative to sum |x_k y_k|).
                    bit 2 (FP64 handles): H x of FP64 blocks in double-FP32
                    arithmetic (48-bit pairs on the FP32 pipe, ~5x faster,
                    ~1e-13 relative; Ritz values stay within 1e-8 Ha, the
                    subspace of nearly degenerate top states may move by
                    ~1e-7).  Mixed handles always evaluate their FP64 Yt this
                    way.
                    bit 3 (test hook for the timeout path): every launch of the
                    ring stencil first waits on a barrier that nothing
                    completes, so that wait runs out after timeout_cycles, the
                    kernel stops (its loads in flight land first) and the next
                    waiting call returns SPARC_ERR_TIMEOUT.  Other bits 0.     */
  int stencil_shape; /* thread shape of the ring stencil: 0 = chosen by timing
                    the shapes that fit the grid on the first filter or H x call
                    with a given ns (that call waits for its stream); k >= 1 =
                    shape k - 1 always (see sparc_get_tuning).  The shapes give
                    bit-identical results.  Shapes (planes per step, threads):
                    FP64 blocks 0 (2, 384), 1 (1, 576); FP32 blocks 0 (4, 384),
                    1 (1, 576), 2 (2, 512).                                    */
  int reserved;  /* must be 0                                                  */
  int64_t timeout_cycles; /* bound of every device-side wait, in SM clock cycles
                    (0 = 4e9, about two seconds); a wait that runs out stops its
                    kernel and the next waiting call returns SPARC_ERR_TIMEOUT */
} sparc_options;

/* Thread shape of the ring stencil in use on a handle and the timings that
 * chose it (sparc_get_tuning).  shape = -1: no ring-form stencil has run. */
typedef struct {
  int shape;            /* index of the shape in use                          */
  int rows_per_thread;  /* grid rows a thread computes per plane              */
  int planes_per_step;  /* planes per move of the thread's z register queue   */
  int slab_rows;        /* y rows of the slab one CTA owns                    */
  int threads;          /* threads per CTA                                    */
  int ns;               /* orbital count of the timed launches                */
  int candidates;       /* number of shapes                                   */
  float candidate_ms[8];/* one stencil launch per shape (0: did not fit)      */
} sparc_tuning;

/* Stage times (ms) of the last sparc_chefsi_step on the handle (CUDA events)
 * and the number of library kernels it launched.  bounds_ms includes the
 * host-to-device staging of a host block; total_ms runs from the call's first
 * event to the end of the rotation.  stage_in_ms / stage_out_ms: the event-
 * timed host-to-device and device-to-host copies of a host block (0 for
 * device blocks).  host_ms: wall time of the whole call on the host clock,
 * from entry to return (for host blocks this includes the final copy and
 * synchronisation; for device blocks the step's own synchronisation on its
 * status word). */
typedef struct {
  float bounds_ms, filter_ms, hx_ms, project_ms, eig_ms, rotate_ms, total_ms;
  int64_t launches;
  float stage_in_ms, stage_out_ms, host_ms;
  /* inside filter_ms, on grids that run the ring stencil: the summed durations
     of the local stencil launches and of the nonlocal passes that follow them
     (0 on the generic path), and the number of filter degrees they cover */
  float stencil_ms, nonlocal_ms;
  int32_t stencil_launches;
} sparc_timings;

/*
 * sparc_create — build a handle for one Hamiltonian (Sec. II A).
 * veff: Nd host doubles.  nl may be NULL (no projectors).  opt may be NULL
 * (FP64, ns_max = 1, device 0).  Validates: n >= 1 per axis, h > 0, bc in
 * {PERIODIC, DIRICHLET}, support indices in range, nonnegative counts.
 * Errors: INVALID_ARG, OOM, CUDA.  On error *out is NULL.
 */
int sparc_create(const sparc_grid* g, const double* veff, const sparc_nonlocal* nl,
                 const sparc_options* opt, sparc_handle* out);

/*
 * sparc_create_kpoint — a handle for H(k) at the Bloch wavevector k (kvec, three
 * components in 1/bohr; components on Dirichlet axes are unused).  The paper
 * computes in real arithmetic at Gamma; at any other wavevector of a
 * Brillouin-zone sampling every operation of Algorithm 1 is complex (Sec. III
 * and the k-point slabs of Sec. IV):
 *   - Bloch condition psi(r + L_d e_d) = exp(i k_d L_d) psi(r) on periodic axes
 *     (L_d = N_d h): a stencil neighbour index j is read at j mod N_d and
 *     multiplied by exp(i k_d L_d floor(j / N_d));
 *   - projectors are Bloch sums: chi^k(r_i) = chi(r_i - R_J - T_i) exp(i k.T_i)
 *     with T_i the periodic image nearest r_i (the cut-off must be below half of
 *     every periodic cell length); positions: natoms x 3 host doubles (bohr), R_J;
 *   - Hs = Xt^H Yt, Ms = Xt^H Xt, Hs Z = Ms Z D with Z^H Ms Z = I.
 * g, veff, nl and opt as in sparc_create; opt->precision must be SPARC_PREC_FP64
 * and ns_max <= 1022.  Orbital blocks of the handle are SPARC_C128 device blocks
 * (column-major, interleaved (re, im) doubles, ld counted in complex entries).
 * Calls accepted: sparc_hpsi, sparc_spectrum_bounds, sparc_cheb_filter,
 * sparc_project, sparc_subspace_eig, sparc_rotate (their ns x ns matrices are
 * complex, column-major, interleaved: 2 ns^2 doubles each; lam stays real;
 * sparc_project makes Hs and Ms Hermitian from their upper triangles, so their
 * diagonals are real),
 * sparc_chefsi_step, sparc_occupations, sparc_get_timings; the others return
 * INVALID_ARG.  The subspace eigensolve uses cyclic Jacobi rotations (returns
 * NUMERIC if 40 sweeps do not converge).  Errors: as sparc_create.
 */
int sparc_create_kpoint(const sparc_grid* g, const double* veff, const sparc_nonlocal* nl,
                        const double* positions, const sparc_options* opt, const double* kvec,
                        sparc_handle* out);

/* sparc_destroy — free the handle and all its device memory; NULL is a no-op. */
int sparc_destroy(sparc_handle h);

/* Last error message of the handle (or of the last failed create if h is NULL). */
const char* sparc_last_error(sparc_handle h);

/*
 * sparc_hpsi — Y = H X for ns columns (Sec. II A, the filtering kernel HX).
 * X, Y: device blocks of type dtype with leading dimension ld (>= Nd); X and Y
 * must not overlap (INVALID_ARG if X == Y).  1 <= ns <= ns_max.  Asynchronous.
 */
int sparc_hpsi(sparc_handle h, const void* X, void* Y, int ns, int64_t ld, int dtype,
               void* stream);

/*
 * sparc_spectrum_bounds — Lanczos estimate of the spectrum ends (Algorithm 1
 * needs lambda_Nd, the largest eigenvalue of H).  `iters` Lanczos steps in FP64
 * from the start vector v_i = u(seed, i) - 1/2, u the counter-based splitmix64
 * uniform.  Writes *a0 = smallest Ritz value, *b = largest Ritz value + |beta_k|
 * (an upper bound of the spectrum).  Synchronous (waits for the stream).
 * 2 <= iters <= 512.
 */
int sparc_spectrum_bounds(sparc_handle h, int iters, uint64_t seed, double* a0, double* b,
                          void* stream);

/*
 * sparc_cheb_filter — X <- p_m((H - c)/e) X / p_m((a0 - c)/e) (Algorithm 1,
 * filtering) with c = (b + a)/2, e = (b - a)/2, m = degree, by the scaled
 * three-term Chebyshev recurrence.  a is the filter cut-off lambda_c, b an upper
 * bound of the spectrum, a0 an estimate of its lower end; requires
 * a0 < a < b and degree >= 1 (INVALID_ARG otherwise).  X: device or host block
 * of type dtype (SPARC_F64 on FP64 handles, SPARC_F32 on mixed handles),
 * overwritten with the result.  Asynchronous for device X.
 */
int sparc_cheb_filter(sparc_handle h, void* X, int ns, int64_t ld, int dtype, int degree,
                      double a, double b, double a0, void* stream);

/*
 * sparc_project — Hs = Xt^T Yt and Ms = Xt^T Xt (Algorithm 1, projection).
 * Xt, Yt: device blocks (dtype, ld).  Hs, Ms: device ns x ns FP64 column-major
 * outputs.  Both are symmetrised from their upper triangles.  Asynchronous on
 * the FP64 SIMT form; the tensor-core form waits for the stream and returns
 * TIMEOUT if one of its bounded waits ran out.
 */
int sparc_project(sparc_handle h, const void* Xt, const void* Yt, int ns, int64_t ld,
                  int dtype, double* Hs, double* Ms, void* stream);

/*
 * sparc_subspace_eig — solve Hs Z = Ms Z D (Algorithm 1, diagonalisation) in
 * FP64: Cholesky Ms = L L^T, A = L^-1 Hs L^-T, A = V D V^T, Z = L^-T V.
 * Hs, Ms: device ns x ns column-major (symmetric; read only).  lam: device ns
 * doubles, ascending.  Z: device ns x ns column-major, Z^T Ms Z = I, each
 * column's largest-magnitude entry positive.  Returns NOT_SPD if the Cholesky
 * meets a non-positive pivot and NUMERIC on NaN/Inf; synchronous (reads the
 * status word back).
 */
int sparc_subspace_eig(sparc_handle h, const double* Hs, const double* Ms, int ns, double* lam,
                       double* Z, void* stream);

/*
 * sparc_rotate — Xout = Xt Z (Algorithm 1, rotation).  Xt, Xout: device
 * blocks (dtype, ld), not overlapping.  Z: device ns x ns FP64 column-major.
 * Asynchronous on the FP64 SIMT form; the tensor-core form waits for the
 * stream, as sparc_project does.
 */
int sparc_rotate(sparc_handle h, const void* Xt, void* Xout, const double* Z, int ns, int64_t ld,
                 int dtype, void* stream);

/*
 * sparc_chefsi_step — one full CheFSI step (Algorithm 1): filter X, Yt = H Xt,
 * project, diagonalise, rotate; X is replaced by Xt Z.
 * bounds: {a, b, a0} host doubles, or NULL: then b and a0 come from a cached
 * 32-step Lanczos run (seed 0) made on the first such call, and a is the
 * largest Ritz value of the previous step on this handle (first step:
 * a0 + 0.1 (b - a0)).  eig: ns Ritz values, ascending, written to host memory
 * if eig_on_host is nonzero, else to device memory (may be NULL).  X: device
 * or host block.  Synchronous: the call waits for the stream at its end, to
 * read the status word of the step's kernels and the largest Ritz value (the
 * next step's cut-off).  Errors: INVALID_ARG, NOT_SPD, NUMERIC, TIMEOUT, CUDA,
 * OOM.
 */
int sparc_chefsi_step(sparc_handle h, void* X, int ns, int64_t ld, int dtype, int degree,
                      const double* bounds, double* eig, int eig_on_host, void* stream);

/*
 * sparc_get_timings — the stage times and launch count of the last
 * sparc_chefsi_step on the handle, into *t (see sparc_timings).  Waits for
 * that step's last stage event.  Errors: INVALID_ARG (null arguments, or no
 * step has run on the handle), CUDA.
 */
int sparc_get_timings(sparc_handle h, sparc_timings* t);

/*
 * sparc_get_tuning — the thread shape the handle's ring stencil uses for the
 * most recent ns it tuned (or was given), with the per-shape times measured on
 * the handle's workspace blocks (stencil_shape 0), into *t.  Errors:
 * INVALID_ARG (null arguments).
 */
int sparc_get_tuning(sparc_handle h, sparc_tuning* t);

/*
 * sparc_occupations — Fermi-Dirac occupations of the Ritz values (the smeared
 * occupation a self-consistent cycle applies after each CheFSI step, Sec. 2.1):
 * f_n = 1 / (1 + exp((lam_n - mu) / kT)), with the Fermi level mu found by
 * bisection on [min lam - 1, max lam + 1] until |2 sum_n f_n - ne| < 1e-12
 * (at most 400 halvings).  lam: ns device doubles (any order).  occ: ns device
 * doubles (output).  mu: one device double (output).  Requires 1 <= ns,
 * kT > 0 and 0 < ne < 2 ns (else INVALID_ARG).  Asynchronous.
 */
int sparc_occupations(sparc_handle h, const double* lam, int ns, double ne, double kT,
                      double* occ, double* mu, void* stream);

/*
 * sparc_density — electron density of the occupied orbitals,
 * rho_i = (2 / h^3) sum_n occ_n X_{i n}^2 for i < Nd (spin-degenerate, with
 * X^T X = I so that h^3 sum_i rho_i = 2 sum_n occ_n).  X: device block (dtype,
 * ld >= Nd, 0 <= ns <= ns_max; ns = 0 gives rho = 0).  occ: ns device doubles.
 * rho: Nd device doubles (output).  FP64 blocks sum in FP64; FP32 blocks sum
 * groups of 16 orbitals in FP32 and the groups in FP64.  Uses the handle's
 * filter workspace as scratch.  Errors: INVALID_ARG, CUDA.  Asynchronous.
 */
int sparc_density(sparc_handle h, const void* X, int ns, int64_t ld, int dtype, const double* occ,
                  double* rho, void* stream);

/*
 * sparc_nonlocal_forces — nonlocal Hellmann-Feynman forces on the atoms (the
 * force kernels the paper runs on the GPU beside the filter, Sec. III: the
 * gradient of the orbitals, then the nonlocal projectors applied to it):
 *   F_Jd = -4 sum_n occ_n sum_p gamma_Jp (h^3 <chi_Jp|X_n>) (h^3 <chi_Jp|D_d X_n>),
 * for real orbitals with spin degeneracy 2, with D_d the radius-6 central first
 * derivative along axis d (x, y, z) under the grid's boundary conditions.
 * - X: device block (dtype of the handle, ld >= Nd, 0 <= ns <= ns_max).
 * - occ: ns device doubles.
 * - F: 3 * natoms device doubles (output), atom-major (F[3 J + d]) in Ha/bohr.
 *   ns = 0 gives F = 0; a handle without atoms returns at once and F may be
 *   NULL.
 * Arithmetic is FP64 for both dtypes (FP32 blocks are widened on load), with a
 * fixed summation order: results are deterministic. The handle's filter
 * workspace is scratch and must hold natoms * ns * 3 doubles (else
 * INVALID_ARG). Errors: INVALID_ARG, CUDA.  Asynchronous.
 */
int sparc_nonlocal_forces(sparc_handle h, const void* X, int ns, int64_t ld, int dtype,
                          const double* occ, double* F, void* stream);

/*
 * Batched form — many independent systems (the paper treats the eigenproblems
 * of different k-points / spins / configurations as independent, Sec. II).
 * A batch is built from existing handles (same precision and device; each keeps
 * its own workspace).  One batched step runs Algorithm 1 on every member, the
 * whole step one CUDA graph: each member's filter, Yt = H Xt and projection
 * (the kernels of sparc_chefsi_step) run as one chain on one of the library's
 * streams, the members concurrently; then one batched eigensolve for all
 * members (see sparc_batch_subspace_eig); then the rotations.  The graph is
 * captured on the first call and replayed while the X pointers, ld, ns,
 * degrees and bounds stay the same; otherwise it is captured again and the
 * executable graph updated.
 */
typedef struct sparc_batch_context* sparc_batch;

/* sparc_batch_create — hs: n >= 1 handles (borrowed: they must outlive the
 * batch).  Errors: INVALID_ARG, OOM, CUDA (message via sparc_last_error(NULL)). */
int sparc_batch_create(const sparc_handle* hs, int n, sparc_batch* out);

/* sparc_batch_destroy — frees the batch (not the handles); NULL is a no-op. */
int sparc_batch_destroy(sparc_batch b);

/* Last error message of a batch call. */
const char* sparc_batch_last_error(sparc_batch b);

/*
 * sparc_batch_chefsi_step — one CheFSI step of every member i = 0..n-1.
 * X[i]: device block of member i (dtype, ld[i] >= Nd_i), replaced by Xt Z.
 * ns[i] must equal member i's ns_max.  degree[i] >= 1.  bounds: 3n host
 * doubles {a, b, a0} per member, or NULL (library bounds per member as in
 * sparc_chefsi_step).  eig: n host pointers to ns[i] doubles (ascending Ritz
 * values), or NULL.  Synchronous.  Errors as sparc_chefsi_step; the failing
 * member is named in the message.
 */
int sparc_batch_chefsi_step(sparc_batch b, void* const* X, const int* ns, const int64_t* ld,
                            int dtype, const int* degree, const double* bounds,
                            double* const* eig, void* stream);

/* Kernel launches per batched step (nodes of the captured graph). */
int sparc_batch_get_info(sparc_batch b, int64_t* launches_per_step);

/*
 * sparc_batch_subspace_eig — the generalised eigensolve of sparc_subspace_eig
 * (Algorithm 1, diagonalisation) for every member i = 0..n-1 at once.
 * Hs[i], Ms[i]: device ns[i] x ns[i] FP64 column-major, symmetric, read only;
 * lam[i]: device ns[i] doubles (ascending); Z[i]: device ns[i] x ns[i]
 * column-major with Z^T Ms Z = I and each column's largest-magnitude entry
 * positive.  1 <= ns[i] <= member i's ns_max.  Members with ns[i] <= 512 are
 * solved together, one launch per cluster size: one thread-block cluster per
 * member runs the steps of sparc_subspace_eig (Cholesky, reduction to
 * standard form, Householder tridiagonalisation, bisection, inverse
 * iteration with Cholesky-QR, back-transformation) with cluster barriers
 * between them; larger members use sparc_subspace_eig's solver one after
 * another.  Uses each member's eigensolver workspace.  Synchronous.  Errors:
 * INVALID_ARG, NOT_SPD, NUMERIC, TIMEOUT, CUDA; the message names the first
 * failing member.  sparc_batch_chefsi_step runs the same solver.
 */
int sparc_batch_subspace_eig(sparc_batch b, const double* const* Hs, const double* const* Ms,
                             const int* ns, double* const* lam, double* const* Z, void* stream);

/*
 * sparc_project_noalloc — the FP64 projection of sparc_project (Hs = Xt^T Yt,
 * Ms = Xt^T Xt) on the FP64 SIMT pipe (the form FP64 handles use when created
 * with sparc_options.flags bit 1), without a handle and without
 * allocating any device memory.
 * The paper has no counterpart; this entry point exists for callers that may
 * not call cudaMalloc: code whose device memory is owned by another allocator
 * (a framework's caching pool or a pre-partitioned budget) that a raw
 * cudaMalloc would bypass, and latency-critical loops that cannot afford the
 * device-wide synchronisation cudaMalloc/cudaFree may cause.
 *
 * Xt, Yt: device FP64 blocks, Nd x ns column-major with leading dimension
 * ld >= nd.  Hs, Ms: device ns x ns FP64 column-major outputs, symmetrised from
 * their upper triangles, as in sparc_project.  The caller passes (and owns) all
 * inputs and outputs.
 *
 * Scratch: the split-K partial sums live in one library-owned, file-scope
 * device array of 4,194,304 doubles (32 MiB) that every GPU which loads the
 * library holds until the process exits.  ns may be at most 1448 (two ns x ns
 * partials must fit); larger ns returns INVALID_ARG without launching work.
 * The first call on a device looks up that array's device address (once per
 * device, with that device current) and keeps it for the life of the process;
 * make that first call before any CUDA stream capture.  A cudaDeviceReset
 * invalidates the kept address: do not call this entry point on a device
 * after resetting it.  Xt, Yt, Hs and Ms must be memory of the current
 * device (or managed memory); a pointer to another GPU's memory returns
 * INVALID_ARG.  All calls share the array and it keeps the last call's
 * contents; every value a call reads from it is written earlier by the same
 * call, so nothing needs clearing, but calls that overlap on the GPU (for
 * example on two streams at once) race on it and must be serialised by the
 * caller.  Errors: INVALID_ARG (null or host pointers, bad sizes), CUDA; the
 * message is available from sparc_last_error(NULL).  Asynchronous.
 */
int sparc_project_noalloc(const double* Xt, const double* Yt, int ns, int64_t nd, int64_t ld,
                          double* Hs, double* Ms, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SPARC_H */

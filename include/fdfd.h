/*
 * fdfd.h -- C ABI of libfdfd: cached direct solves of the 2D TM (Ez)
 * finite-difference frequency-domain system for adjoint inverse design, on
 * one NVIDIA GB300 (sm_103a).
 *
 * Paper: "Computational Scaling in Inverse Photonic Design Through
 * Factorization Caching" (arXiv 2307.05388).  Section numbers and equation
 * numbers below refer to it.
 *
 * Operator (Eq. 1-2).  The paper's
 *     (-omega^2 eps0 eps_r + mu0^-1 curl curl) E = -i omega J
 * is discretised on a Yee grid of nx x ny cells of size dx with a
 * stretched-coordinate PML of npml cells on every side (counted inside the
 * grid) and a zero field one cell beyond the grid (PEC).  The library works
 * with the dimensionless operator obtained by multiplying by mu0 dx^2:
 *     A = -dx^2 Lap_s - (k0 dx)^2 diag(eps_r),   k0 = omega / c,
 *     A[(i,j),(i+-1,j)] = -1 / (sx(i+1/2) sx(i+1/2 +- 1/2)),  same in y,
 *     A[(i,j),(i,j)]    = -(sum of the four neighbour coefficients) - (k0 dx)^2 eps[i,j],
 *     s(u) = 1 - i [-(order+1) ln R / (2 k0 dx npml)] d(u)^order,  d = depth / npml,
 * with cell (i, j) centred at ((i + 1/2) dx, (j + 1/2) dx) and the time
 * convention e^{+i omega t} implied by the -i omega J right-hand side.  The
 * unknown of cell (i, j) has flat index n = i*ny + j.  A right-hand side b is
 * the caller's (for Eq. 2 it is -i omega mu0 dx^2 J).
 *
 * Method (Sec. II).  Symbolic factorisation once per grid (nested-dissection
 * ordering aligned to the design box, elimination tree, fronts), reused for
 * every wavelength and iteration; numeric factorisation per wavelength
 * (batched dense complex LU of same-level fronts with extend-add); the
 * adjoint solve A^T x = b reuses the same factors (Eq. 6); a design update
 * refactors only the fronts whose subtree holds a design pixel; many
 * right-hand sides share one factorisation.  In the default mixed mode the
 * factors are complex FP32 and every solve is refined by flexible GMRES with
 * FP64 residuals and updates, so that results match a complex128 direct solve.
 *
 * Conventions for every call:
 *  - Pointers named *_dev are device memory owned by the caller, read or
 *    written on the context's CUDA stream (asynchronously: synchronise the
 *    stream before reading results on the host).  Pointers named *_host are
 *    host memory, read before the call returns.
 *  - Complex numbers are interleaved (re, im) doubles, i.e. CUDA double2.
 *  - Field arrays have layout [n_omega][nrhs][nx*ny] (system s = w*nrhs + r).
 *  - Design arrays have layout [w][h]: pixel (i, j) of the box, at grid cell
 *    (x0 + i, y0 + j), has index i*h + j.
 *  - Every call returns a status; fdfd_last_error() gives a one-line reason.
 *    No call aborts the process.  A failed call leaves the context usable
 *    unless the status is FDFD_ERR_CUDA.
 */
#ifndef FDFD_H_
#define FDFD_H_

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fdfd_ctx fdfd_ctx;

typedef enum {
  FDFD_OK = 0,
  FDFD_ERR_ARG = 1,            /* invalid argument (sizes, null pointers, box outside grid) */
  FDFD_ERR_STATE = 2,          /* call out of order (e.g. solve before factor) */
  FDFD_ERR_OOM = 3,            /* device memory allocation failed */
  FDFD_ERR_CUDA = 4,           /* a CUDA runtime error; text in fdfd_last_error */
  FDFD_ERR_PIVOT = 5,          /* pivot growth above the bound even in FP64 */
  FDFD_ERR_NOT_CONVERGED = 6,  /* refinement stopped above the tolerance; best x returned */
  FDFD_ERR_TIMEOUT = 7         /* a bounded device wait of a dataflow sweep gave up (a front it
                                  depends on never completed); reported by the call that
                                  synchronises next, the context stays usable */
} fdfd_status;

typedef struct { int nx, ny; } fdfd_grid;

/* PML thickness in cells (npml_x, npml_y; 0 disables that axis), ln of the
 * target normal-incidence reflection (default ln 1e-8) and grading order
 * (default 3). */
typedef struct { int npml_x, npml_y; double ln_R; double order; } fdfd_pml;

/* design region in cells: [x0, x0+w) x [y0, y0+h); w = h = 0 for none */
typedef struct { int x0, y0, w, h; } fdfd_box;

typedef enum {
  FDFD_MODE_MIXED = 0,         /* cached complex FP32 factors + FP64 FGMRES refinement */
  FDFD_MODE_F64 = 1,           /* cached complex FP64 factors, no refinement */
  FDFD_MODE_PLAIN = 2          /* no caching (paper's reference arm, Sec. III): every solve
                                  re-runs the symbolic phase and a full FP64 factorisation */
} fdfd_mode;

typedef struct {
  int mode;                    /* fdfd_mode */
  double ir_tol;               /* FGMRES stop: ||b - A x|| <= ir_tol ||b|| per system (default 1e-9) */
  int ir_max_iter;             /* FGMRES iterations per solve across restarts (default 40);
                                  0 returns the raw FP32-factor solution */
  int gmres_restart;           /* Krylov vectors per cycle, 1..16 (default 8) */
  double growth_bound;         /* largest |L| entry expected of an FP32 front (default 1e7, where
                                  the FP32 unit roundoff times the growth reaches about 0.6); above
                                  it a factorisation with block-local pivoting (or the symmetric
                                  form) is redone in FP32 with partial pivoting over all pivot
                                  rows.  FP32 factors whose growth stays finite are then kept for
                                  refined solves: one that does not converge on them sends the
                                  factorisation to FP64, as does an infinite or NaN growth (a zero
                                  or non-finite pivot), or a raw solve (ir_max_iter = 0). */
  int leaf_area;               /* nested-dissection leaf size in cells (default 32) */
  int pivoting;                /* row pivoting in large fronts: 0 = partial pivoting over all the
                                  front's pivot rows, 1 = partial pivoting within each 32 x 32
                                  diagonal block of the panel (default; faster, rows below are
                                  eliminated against it).  Small fronts and the FP64 fallback
                                  always use full partial pivoting. */
  int tensor_form;             /* update matrices S = F22 - L21 U12 of complex FP32 fronts with
                                  m >= tensor_min_m on the tensor cores (tcgen05, FP32 accumulation):
                                  0 = off (SIMT FP32), 1 = TF32 operands, 2 = TF32 hi + lo (three
                                  products), 3 = BF16 three-way split, six products (default) */
  int tensor_min_m;            /* smallest boundary size m sent to the tensor cores (default 128) */
  int tensor_min_tiles;        /* CTAs a level's tensor-core update matrices should fill: 0 = the
                                  device's SM count, one wave (default).  A level whose eligible
                                  fronts make fewer 128 x 128 output tiles (over all wavelengths)
                                  splits each tile's contraction over up to 16 CTAs (4 k-tiles of
                                  8 pivots at least each); if even then it fills less than half
                                  of them, its update matrices run SIMT.  1 = never split. */
  int factor_form;             /* complex FP32 factors: 0 = LU of A with the pivoting above (default);
                                  1 = symmetric form: D A, with D = diag(s_x s_y) at the cell centres,
                                  is complex symmetric (reciprocity) and is factored as L diag(d) L^T
                                  in the elimination order with no pivoting, lower triangles only
                                  (half the update flops; the solves run the L and L^T sweeps with
                                  D and 1 / d applied between them).  If its pivot growth exceeds
                                  growth_bound it falls back to LU with partial pivoting over all
                                  pivot rows, then to FP64, as above; the next design refactor then
                                  refactors the whole symmetric form again.  FP64 factors are
                                  always LU. */
  int sweep_rhs_pairs;         /* 1: the sweeps of complex FP32 factors take the right-hand sides of a
                                  wavelength two at a time when their count is even (each factor entry
                                  loaded once for both; twice the shared memory per CTA); 0: one at a
                                  time (default: the second system's reads mostly hit the caches, and
                                  the pairs' shared memory lowers residency; measured C3 +1%, C5 -7%). */
  int tensor_offdiag;          /* 1: complex FP32 LU fronts whose update matrices go to the tensor cores
                                  (tensor_form > 0, block-local pivoting) also form L21 = F21 U11^-1 and
                                  U12 = L11^-1 P F12 there, as products with the triangular inverses, and
                                  their panel steps factor only the pivot block; 0 (default): the panel
                                  steps form L21 and U12 by substitution.  The products are faster but
                                  carry the conditioning of U11 and L11 into the factors (more FGMRES
                                  iterations on ill-conditioned fronts). */
} fdfd_options;
/* fdfd_create rejects a mode outside fdfd_mode with FDFD_ERR_ARG and clamps the
 * other fields: gmres_restart to 1..16, ir_max_iter and tensor_min_tiles to >= 0,
 * tensor_min_m to >= 1; leaf_area < 1, tensor_form outside 0..3, and ir_tol or
 * growth_bound that are not positive numbers take their defaults; any nonzero
 * pivoting means 1; factor_form outside 0..1 takes 0; any nonzero sweep_rhs_pairs or tensor_offdiag means 1. */

typedef struct {
  long long sf;                /* symbolic factorisations performed */
  long long nf;                /* numeric factorisations (one per wavelength, full or design refactor) */
  long long bs;                /* back substitutions (one per system solved: wavelength x rhs) */
  long long sweeps;            /* triangular sweep pairs executed (including refinement) */
  long long ir_iters;          /* FGMRES iterations in the last solve (max over systems) */
  double ir_resid;             /* largest relative residual at the end of the last solve */
  long long fallbacks;         /* factorisations redone in FP64 (pivot growth or no convergence) */
  double growth;               /* largest |L| entry in the last factorisation */
  int n_fronts, n_levels, max_front;
  long long factor_entries;    /* stored L and U entries per wavelength */
  long long store_bytes;       /* device bytes of front storage (all wavelengths) */
  double flops_factor;         /* full factorisation flops per wavelength (8 per complex FMA) */
  double flops_design;         /* flops of a design refactor per wavelength */
  long long repivots;          /* complex FP32 factorisations redone with partial pivoting over all
                                  pivot rows after block-local pivoting (or the symmetric form)
                                  exceeded growth_bound */
  int factor_form;             /* form of the current complex FP32 factors (0 LU, 1 symmetric) */
} fdfd_stats;

/* Fills *opt with the defaults listed above. */
void fdfd_default_options(fdfd_options* opt);

/* Creates a context (host only, no device work yet).
 * k0_host: [n_omega] free-space wavenumbers k0 = omega / c, in inverse units of
 * dx (e.g. 2 pi / lambda with lambda and dx in micrometres).  cuda_stream: the
 * cudaStream_t all work is issued on (NULL = legacy default stream).  The
 * context owns every device buffer it allocates; the caller owns *out and
 * frees it with fdfd_destroy.  opt may be NULL (defaults). */
fdfd_status fdfd_create(fdfd_ctx** out, fdfd_grid grid, double dx, const double* k0_host, int n_omega,
                        fdfd_pml pml, fdfd_box design, const fdfd_options* opt, void* cuda_stream);

/* Symbolic phase (Sec. II, Fig. 1): nested-dissection ordering aligned to the
 * design box, elimination tree, fronts and index maps, computed on the host and
 * uploaded once.  Idempotent: a second call does nothing (in plain mode it is
 * repeated inside every solve instead). */
fdfd_status fdfd_analyze(fdfd_ctx* ctx);

/* Numeric factorisation of A(eps) for every wavelength (Sec. II).
 * eps_dev: [nx*ny] relative permittivity (device, read once; the context keeps
 * a copy).  Runs the symbolic phase first if it has not run. */
fdfd_status fdfd_factor(fdfd_ctx* ctx, const double* eps_dev);

/* Design update: replaces the permittivity of the design box by eps_design_dev
 * ([w*h], device) and refactors only the fronts whose subtree holds a design
 * pixel, reusing the cached factors and update matrices of every other front.
 * The result is bit-identical to fdfd_factor on the full updated eps.
 * Requires an earlier fdfd_factor. */
fdfd_status fdfd_refactor_design(fdfd_ctx* ctx, const double* eps_design_dev);

/* Solves A x = b (transpose = 0, Eq. 5) or A^T x = b (transpose = 1, Eq. 4/6)
 * for all wavelengths and nrhs right-hand sides on the cached factors.
 * b_dev, x_dev: [n_omega][nrhs][nx*ny] complex128 (device); x may not alias b.
 * In mixed mode, refinement that stops above ir_tol on the complex FP32 factors
 * sends the factorisation to FP64 (counted in fdfd_stats.fallbacks) and the solve
 * is repeated; FDFD_ERR_NOT_CONVERGED (x holds the last iterate) is returned only
 * when it stops above ir_tol on FP64 factors as well. */
fdfd_status fdfd_solve(fdfd_ctx* ctx, const double* b_dev, double* x_dev, int nrhs, int transpose);

/* Mode-overlap objective and its adjoint source (Eq. 4):
 *   o_s = sum_j g_s[j] x_s[col_s*ny + j],   F = sum_s weight_s |o_s|^2,
 *   b_adj_s = weight_s conj(o_s) g_s on column col_s, zero elsewhere
 * (the Wirtinger derivative dF/dE with E* held fixed, transposed).
 * x_dev: [n_omega][nrhs][nx*ny]; cols_dev: [n_omega*nrhs] int; g_dev:
 * [n_omega*nrhs][ny] complex128; weight_dev: [n_omega*nrhs] or NULL (all 1);
 * o_dev: [n_omega*nrhs] complex128 out; F_dev: one double out; b_adj_dev:
 * [n_omega][nrhs][nx*ny] out or NULL. */
fdfd_status fdfd_objective(fdfd_ctx* ctx, const double* x_dev, int nrhs, const int* cols_dev,
                           const double* g_dev, const double* weight_dev, double* o_dev, double* F_dev,
                           double* b_adj_dev);

/* The same with transmission targets (Sec. III-IV: the duplexer's and the mode
 * multiplexer's objectives are the differences between calculated and target
 * transmissions, minimised):
 *   o_s = sum_j g_s[j] x_s[col_s*ny + j],   F = sum_s weight_s (|o_s|^2 - target_s)^2,
 *   b_adj_s = 2 weight_s (|o_s|^2 - target_s) conj(o_s) g_s on column col_s, zero elsewhere.
 * target_dev: [n_omega*nrhs] double (device); NULL gives fdfd_objective's F = sum weight |o|^2.
 * Other arguments as for fdfd_objective. */
fdfd_status fdfd_objective_target(fdfd_ctx* ctx, const double* x_dev, int nrhs, const int* cols_dev,
                                  const double* g_dev, const double* weight_dev, const double* target_dev,
                                  double* o_dev, double* F_dev, double* b_adj_dev);

/* Pixel gradient (Eq. 3) over the design box:
 *   grad[p] (+)= sum_s weight_s * 2 (k0 dx)^2 Re(x_adj_s[p] x_fwd_s[p]),
 * i.e. dF/deps_p = -2 Re{x_adj^T (dA/deps_p) x_fwd} with dA/deps_p = -(k0 dx)^2 e_p e_p^T,
 * given x_adj = A^-T (dF/dx)^T.  x_fwd_dev, x_adj_dev: [n_omega][nrhs][nx*ny];
 * weight_dev: [n_omega*nrhs] or NULL; grad_dev: [w*h]; accumulate = 1 adds. */
fdfd_status fdfd_grad(fdfd_ctx* ctx, const double* x_fwd_dev, const double* x_adj_dev, int nrhs,
                      const double* weight_dev, double* grad_dev, int accumulate);

/* One whole forward + adjoint design iteration in one call (Sec. II; Eq. 3-6):
 * design refactor with eps_design ([w*h], the box's permittivity), forward solves
 * of b_dev for every wavelength and source, the objective of fdfd_objective_target
 * (target_dev NULL: F = sum weight |o|^2) and its adjoint source, transpose solves
 * on the same factors, and the pixel gradient dF/deps of fdfd_grad.
 * flags: FDFD_HOST_EPS = eps_design is host memory (copied to the device inside
 * the call; pinned memory keeps the copy asynchronous); FDFD_HOST_OUT = F_out
 * (one double) and grad_out ([w*h]) are host memory, and the call returns after
 * the stream has written them.  Without the flags those pointers are device
 * memory written on the context's stream.  x_dev, xadj_dev: [n_omega][nrhs][nx*ny]
 * complex128 device buffers that receive the forward and adjoint fields, or NULL
 * (context-owned buffers, kept until the next call).  b_dev, cols_dev, g_dev,
 * weight_dev, target_dev: as for fdfd_solve and fdfd_objective_target.
 * Requires an earlier fdfd_factor (the full permittivity) and a design box
 * (FDFD_ERR_STATE); statuses of the steps pass through. */
#define FDFD_HOST_EPS 1
#define FDFD_HOST_OUT 2
fdfd_status fdfd_design_iteration(fdfd_ctx* ctx, const double* eps_design, const double* b_dev, int nrhs,
                                  const int* cols_dev, const double* g_dev, const double* weight_dev,
                                  const double* target_dev, double* F_out, double* grad_out, double* x_dev,
                                  double* xadj_dev, int flags);

/* Applies the FP64 operator: y = A x (transpose 0) or A^T x, all systems. */
fdfd_status fdfd_apply(fdfd_ctx* ctx, const double* x_dev, double* y_dev, int nrhs, int transpose);

/* Guided modes of an x-invariant cross-section, for eigenmode sources and mode
 * monitors (the multi-mode devices of Sec. III).  Host-only: needs no context and
 * no GPU, and touches no device memory.
 *
 * A guide eps[i][j] = eps_line[j] carries source-free fields
 * E[i][j] = phi[j] exp(-i theta i) of the operator of Eq. 1-2 when
 * (k0dx^2 diag(eps_line) + tridiag(1, -2, 1)) phi = mu phi with
 * mu = 4 sin^2(theta / 2): the y-part of the stencil with PEC one cell beyond
 * both ends and no PML on the cross-section (a bound mode has decayed before it).
 *
 *   ny        cells of the cross-section (>= 1)
 *   k0dx      free-space wavenumber times the cell size
 *   eps_line  [ny] relative permittivity along y (host)
 *   n_modes   1..ny: the n_modes largest mu are returned
 *   mu        [n_modes] out (host), descending; a mode is bound when
 *             mu > k0dx^2 max(eps_line[0], eps_line[ny-1])
 *   theta     [n_modes] out (host) or NULL: propagation constant times dx,
 *             NaN where mu is outside (0, 4) (no propagation along x on the grid)
 *   phi       [n_modes][ny] out (host), unit 2-norm, sign fixed so that the
 *             first entry whose magnitude reaches half the largest is positive
 *
 * Method: bisection on Sturm counts for mu (full double precision), inverse
 * iteration with partial pivoting for phi.  Errors: FDFD_ERR_ARG for sizes out
 * of range, NULL eps_line/mu/phi or non-finite inputs; FDFD_ERR_PIVOT if an
 * inverse iteration breaks down. */
fdfd_status fdfd_slab_modes(int ny, double k0dx, const double* eps_line, int n_modes, double* mu,
                            double* theta, double* phi);

/* Replaces the solve options (ir_tol, ir_max_iter, gmres_restart) at run time.
 * mode, growth_bound, leaf_area, pivoting and the tensor_* fields are fixed at
 * creation and ignored here. */
fdfd_status fdfd_set_options(fdfd_ctx* ctx, const fdfd_options* opt);

/* Counters and sizes (synchronises the context's stream). */
fdfd_status fdfd_stats_get(fdfd_ctx* ctx, fdfd_stats* out);

/* Symbolic plan introspection for host-side tests (valid after fdfd_analyze):
 * per front its pivot count k, boundary count m, parent (-1 root), level and
 * design flag; idx receives the grid cells of every front ([k pivots | m
 * boundary] concatenated in front order, sum of (k+m) entries).  Any output
 * pointer may be NULL.  Host memory. */
fdfd_status fdfd_plan_fronts(fdfd_ctx* ctx, int* k_host, int* m_host, int* parent_host, int* level_host,
                             int* design_host, int* idx_host);

/* More plan introspection: per front its size n = k + m, the row stride ld of its
 * storage and the row stride ldk of its inverse block (host memory; NULL skips). */
fdfd_status fdfd_plan_sizes(fdfd_ctx* ctx, int* n_host, int* ld_host, int* ldk_host);

/* Factor introspection for tests: copies front f of wavelength w of the current
 * factorisation to host memory (synchronises the stream): front_host receives
 * n x ld entries (row-major; complex64, or complex128 if the factorisation is in
 * FP64: L21 below the pivot rows, U12 right of them (LU form only) and the update
 * matrix S in the trailing block, lower triangle only in the symmetric form), inv_host
 * k x ldk entries of the inverse block (L11^-1 strictly below the diagonal; U11^-1 on
 * and above it in the LU form, 1 / d on the diagonal in the symmetric form).  Either
 * pointer may be NULL.  FDFD_ERR_STATE before a factorisation. */
fdfd_status fdfd_front_copy(fdfd_ctx* ctx, int w, int f, void* front_host, void* inv_host);

/* Per-kernel profile: while enabled, every kernel launch of the solver is
 * bracketed by CUDA events on the context's stream and its algorithmic work
 * (flops at 8 per complex multiply-add, and the bytes the method must move) is
 * recorded.  Enabling (or disabling) clears the records.  Profiling adds event
 * records between launches, so time the unprofiled path separately. */
typedef struct {
  char name[32];               /* kernel class, e.g. "lu_gemm", "sweep_L" */
  long long launches;
  double ms;                   /* summed event time of its launches */
  double flops;                /* summed algorithmic flops */
  double bytes;                /* summed algorithmic bytes */
} fdfd_kernel_profile;
fdfd_status fdfd_profile_enable(fdfd_ctx* ctx, int on);
/* Writes up to max_out kernel classes to out and their count to *n_out
 * (synchronises the context's stream).  out is host memory. */
fdfd_status fdfd_profile_get(fdfd_ctx* ctx, fdfd_kernel_profile* out, int max_out, int* n_out);

/* Resets the SF/NF/BS counters. */
void fdfd_reset_counters(fdfd_ctx* ctx);

/* Self-test of the failure path of the dataflow sweeps (the paper has no
 * counterpart).  Every wait of a sweep task on the fronts it depends on polls
 * a completion counter a bounded number of times (about a second) and then
 * gives up: it sets the context's device error word and its CTA stops, so a
 * front that never completes ends the launch with FDFD_ERR_TIMEOUT instead of
 * hanging the GPU.  This call runs one such wait on a counter that nothing
 * increments (one small kernel on the context's stream, synchronised) and
 * returns FDFD_ERR_TIMEOUT when the wait gave up as designed; the error word
 * is cleared and the context stays usable.  Any other status is a failure. */
fdfd_status fdfd_selftest_wait(fdfd_ctx* ctx);

/* Self-test of the failure path of the tensor-core update-matrix pipeline (the paper
 * has no counterpart).  The copy, MMA and accumulation roles of that kernel wait on
 * shared-memory mbarriers with a bounded wait (by global time); a wait that gives up
 * sets the context's error word to 2 and the CTA frees its tensor memory and returns.
 * This call runs that same bounded wait, with a 1 ms limit, on an mbarrier that
 * nothing arrives at (one small kernel on the context's stream, synchronised), and
 * returns FDFD_ERR_TIMEOUT when it gave up as designed; the error word is cleared and
 * the context stays usable.  Any other status is a failure. */
fdfd_status fdfd_selftest_mbar_wait(fdfd_ctx* ctx);

/* The same bounded wait as fdfd_selftest_wait, left for the caller to find: the
 * probe kernel and the copy of the error word back to the host are queued on the
 * context's stream and the call returns FDFD_OK without synchronising.  Once the
 * stream has run them, the next call that checks the error word (fdfd_solve,
 * fdfd_solve_raw_noalloc, fdfd_selftest_*) returns FDFD_ERR_TIMEOUT and clears
 * it, exactly as after a sweep whose wait gave up; the context stays usable. */
fdfd_status fdfd_selftest_wait_async(fdfd_ctx* ctx);

/* Self-test of the tensor-core update-matrix product (Sec. II: S = F22 - L21 U12 of
 * a front), on one caller-supplied front: front_dev is a (k + m) x ld row-major
 * complex64 matrix in device memory (8-byte aligned, ld >= k + m, interleaved
 * re/im) whose block [k:, k:] is overwritten with F22 - L21 U12, L21 = rows k..
 * columns ..k, U12 = rows ..k columns k..; nothing else is written.  planes is
 * the operand form of tensor_form (1 TF32, 2 TF32 hi + lo, 3 BF16 three-way split).  Runs the same pack and product kernels as the factorisation on
 * the context's stream and synchronises; FDFD_ERR_ARG on bad arguments,
 * FDFD_ERR_TIMEOUT if a pipeline wait gave up. */
fdfd_status fdfd_selftest_schur_tc(fdfd_ctx* ctx, void* front_dev, int k, int m, int ld, int planes);

/* Text of the last error on this context ("" if none); valid until the next call. */
const char* fdfd_last_error(const fdfd_ctx* ctx);

/* Frees every device and host buffer of the context (synchronises its stream). */
void fdfd_destroy(fdfd_ctx* ctx);

/* Solve on the cached factors without allocating any device memory.
 * (The paper has no counterpart: this is a library convenience.)
 *
 * For callers that cannot call cudaMalloc at solve time: code that must not
 * let the allocator synchronise the device inside a latency-critical loop,
 * processes whose device memory is budgeted or owned by another allocator
 * pool, and embedding applications that forbid allocation after set-up.
 *
 * Computes x = (P^T L U)^-1 b (transpose = 0) or x = (P^T L U)^-T b
 * (transpose = 1) with the cached factorisation: the raw forward and backward
 * sweeps only, without refinement (the same result as fdfd_solve with
 * ir_max_iter = 0).  b_dev, x_dev: [n_omega][nrhs][nx*ny] complex128 (device,
 * caller-owned); x may not alias b.  All temporary storage lives in one fixed
 * device array of fdfd_noalloc_scratch_bytes() bytes (32 MiB) that every GPU
 * loading this library holds until the process exits; a solve whose front
 * vectors and sweep counters (4 bytes per front and wavelength, twice) do not
 * fit is rejected with FDFD_ERR_ARG before any device work.  The first call on a device looks up
 * the array's device address (with that device current); make that first call
 * before any stream capture.  Every call shares the array and leaves its last
 * contents there (nothing in it needs to start at zero); calls that overlap on
 * the GPU race on it and must be serialised by the caller.  Requires an earlier
 * fdfd_factor (FDFD_ERR_STATE otherwise) and the context's device to be the
 * current device (FDFD_ERR_STATE otherwise); if that FP32 factorisation exceeded
 * the growth bound, returns FDFD_ERR_PIVOT (fdfd_solve redoes it in FP64, which
 * allocates).  The first call after each factorisation synchronises the stream
 * once to read the factorisation's growth figure; other calls do not synchronise.
 * A bounded device wait that gave up earlier (in a factorisation or a sweep)
 * is reported at entry as FDFD_ERR_TIMEOUT; one that gives up in this call's own
 * sweeps is reported by the next call on the context that checks it (this call
 * only queues the copy of the error word back to the host). */
fdfd_status fdfd_solve_raw_noalloc(fdfd_ctx* ctx, const double* b_dev, double* x_dev, int nrhs, int transpose);
/* Size in bytes of the fixed scratch array used by fdfd_solve_raw_noalloc. */
size_t fdfd_noalloc_scratch_bytes(void);

/* Smoothing filter and projection of the design density (Sec. III: a smoothing
 * filter of 200 nm radius and a sigmoid-like projection binarise the geometry;
 * the forms used are a conic filter and a tanh projection):
 *   rho~_i = sum_j w_ij rho_j / N_i,  w_ij = max(0, radius - |p_i - p_j|),  N_i = sum_j w_ij,
 *   rho^_i = (tanh(beta eta) + tanh(beta (rho~_i - eta))) / (tanh(beta eta) + tanh(beta (1 - eta))),
 *   eps_i  = eps_lo + rho^_i (eps_hi - eps_lo),
 * with pixel distances |p_i - p_j| in cells and the sums over the context's
 * design box (w x h pixels, x-major: pixel (i, j) at i*h + j, the layout of
 * fdfd_refactor_design).  rho_dev, eps_dev: [w*h] double (device); work_dev:
 * [2*w*h] double (device, caller-owned), filled with what the adjoint needs
 * (the slope d eps_i / d rho~_i, then N_i).  FDFD_ERR_ARG unless 0 < radius
 * <= 25, beta > 0, 0 < eta < 1 and the context has a design box.  Runs on the
 * context's stream. */
fdfd_status fdfd_filter_project(fdfd_ctx* ctx, const double* rho_dev, double radius, double beta, double eta,
                                double eps_lo, double eps_hi, double* eps_dev, double* work_dev);

/* Permittivity of the design box from an unfiltered density (Sec. III's design
 * pixels between eps_SiO2 and eps_Si): eps_i = eps_lo + rho_i (eps_hi - eps_lo)
 * for the w*h pixels of the context's design box.  rho_dev, eps_dev: [w*h] double
 * (device; may alias).  Runs on the context's stream.  The chain rule is a scale:
 * dF/drho = (eps_hi - eps_lo) dF/deps.  FDFD_ERR_ARG without a design box. */
fdfd_status fdfd_density_eps(fdfd_ctx* ctx, const double* rho_dev, double eps_lo, double eps_hi, double* eps_dev);

/* Chain rule of fdfd_filter_project back to the density:
 *   g_rho_j = sum_i w_ij g_eps_i s_i / N_i
 * with s_i and N_i from the work_dev of the forward call (same radius).
 * g_eps_dev, g_rho_dev: [w*h] double (device); g_rho may not alias g_eps. */
fdfd_status fdfd_filter_project_adjoint(fdfd_ctx* ctx, const double* g_eps_dev, const double* work_dev,
                                        double radius, double* g_rho_dev);

#ifdef __cplusplus
}
#endif

#endif /* FDFD_H_ */

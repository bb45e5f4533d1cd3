/*
 * sg.h -- C ABI of the GB300 stochastic Galerkin Helmholtz solver.
 *
 * The library solves the linear system A V = b that a finite-difference
 * (FD) discretisation in space and a stochastic Galerkin (SG) projection in
 * the random variables produce for
 *
 *     -Laplace(u) - k(x, xi)^2 u = f,    k(x, xi) = k_0(x) + sum_l xi_l k_l(x),
 *
 * with homogeneous Dirichlet or absorbing (d_n u - i k u = 0) boundary
 * conditions and independent xi_l ~ U[-1, 1] (Pulch & Sete, "The Helmholtz
 * equation with uncertainties in the wavenumber", Sec. 2 and Sec. 3).
 *
 * Conventions shared by every entry point:
 *   - All pointers named X, Y, R, Z, b, x, x0 are caller-owned buffers of
 *     N = n * P complex numbers stored as interleaved (re, im) pairs,
 *     complex128 for SG_FP64 and complex64 for SG_FP32.  They live in device
 *     memory unless an entry point says otherwise.  Ordering is the paper's:
 *     V = [V_0; V_1; ...; V_{P-1}] (mode-major, Sec. 3.1), each V_i over the
 *     n grid unknowns with x fastest (Theorems A.5/A.6).
 *   - n = number of grid unknowns (Dirichlet nodes are eliminated, absorbing
 *     boundary nodes are kept), P = (s+r)!/(s! r!) chaos modes (Sec. 2.3).
 *   - Chaos modes are ordered by total degree; inside one degree by
 *     descending lexicographic order of the multi-index (alpha_1..alpha_s).
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls are asynchronous on that stream unless stated.
 *   - Every call returns an sg_status.  On failure sg_last_error() returns
 *     a thread-local message; outputs are left unspecified.  No entry point
 *     falls back to the CPU.
 *   - The library owns the handle, its device fields, factors and
 *     workspace (allocated by sg_assemble / the first sg_gmres call, freed by
 *     sg_destroy).  Handles are not thread-safe; use one per host thread.
 *   - One CUDA device per process: kernel attributes and SM counts are set
 *     up on the device of the first sg_assemble, and sg_assemble on another
 *     device returns SG_EUNSUPPORTED (run one process per GPU).
 */
#ifndef SG_GB300_H
#define SG_GB300_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sg_handle sg_handle;

typedef enum {
  SG_OK = 0,
  SG_EINVAL = 1,        /* bad argument (size, NULL pointer, NaN, k <= 0 ...) */
  SG_ENOMEM = 2,        /* device or host allocation failed */
  SG_ECUDA = 3,         /* a CUDA runtime call failed */
  SG_ENOTCONV = 4,      /* GMRES stopped at maxit above tol (x = best iterate) */
  SG_EBREAKDOWN = 5,    /* Arnoldi breakdown or non-finite value in the solve */
  SG_ESINGULAR = 6,     /* zero pivot in a preconditioner factorisation */
  SG_ETIMEOUT = 7,      /* a bounded device-side wait gave up (kernel returned, context usable) */
  SG_EUNSUPPORTED = 8   /* valid input the library does not implement */
} sg_status;

typedef enum { SG_BC_DIRICHLET = 0, SG_BC_ABSORBING = 1 } sg_bc;

/* Preconditioners (Sec. 4, Sec. 5, Sec. 6.3):
 *   SG_PREC_MEAN      mean-value A_0 = I_P (x) S(xi_bar), xi_bar = 0 for
 *                     uniform variables, so S(xi_bar) is the FD matrix of the
 *                     wavenumber k_0 (Sec. 5, Remark 6.1);
 *   SG_PREC_CSL_MEAN  mean-value complex shifted Laplace
 *                     M_0 = I_P (x) (S(xi_bar) - i beta D_2(k_0^2)) (Sec. 6.3);
 *   SG_PREC_CSL       the coupled complex shifted Laplace matrix
 *                     M(beta) = A - i beta K, K = [C_ij] the k^2 part of A
 *                     (Sec. 4; the paper uses it in 1D), factored as a band
 *                     with the unknowns numbered point by point (kl = ku = P in
 *                     1D, mx P in 2D) on first use; SG_EUNSUPPORTED when that
 *                     band is too wide (most 2D problems). */
typedef enum { SG_PREC_NONE = 0, SG_PREC_MEAN = 1, SG_PREC_CSL_MEAN = 2, SG_PREC_CSL = 3 } sg_prec;

/* SG_FP64: complex128 operands and arithmetic.
 * SG_FP32: complex64 operands and arithmetic (reductions accumulate in FP64
 *          across thread blocks).
 * SG_MIXED (sg_gmres only): complex64 inner GMRES inside an FP64 iterative
 *          refinement loop; b, x, x0 are complex128.
 * SG_TF32 (sg_precond only): complex64 operands, the 2D fast-diagonalisation
 *          transforms in plain TF32 on the tensor cores (relative error of
 *          the apply ~2e-3).  Not in the paper.
 * SG_FP16 (sg_precond only): complex64 operands, transforms 2-4 of the same
 *          apply on binary16 operands (tensor-core kind::f16, FP32
 *          accumulation) with binary16 intermediates, scaled to stay near 1
 *          (the input by 1 / ||R||); the same 11-bit significands as TF32.
 *          Where it exists (sg_info.fp16_route) the complex64 inner cycles
 *          of sg_gmres use it (see there), else SG_TF32.  Not in the paper. */
typedef enum { SG_FP64 = 0, SG_FP32 = 1, SG_MIXED = 2, SG_TF32 = 3, SG_FP16 = 4 } sg_precision;

/* Problem description (Sec. 2.2 wavenumber model; Appendix A grids).
 *   dim    1 or 2 (unit interval / unit square).
 *   nx,ny  grid nodes per direction INCLUDING boundary nodes (q+2 in the
 *          paper's notation); ny = 1 when dim = 1.  h = mesh width.
 *   bc     {left x=0, right x=1, bottom y=0, top y=1}; dim = 1 reads bc[0],
 *          bc[1] (they may differ); dim = 2 requires all four equal
 *          (Theorem A.5 all Dirichlet or Theorem A.6 all absorbing).
 *   s, r   number of random variables and total chaos degree.
 *   k0     host, nx*ny doubles: k_0 at every node, x fastest.
 *   kl     host, s*nx*ny doubles, layout [l][node]: k_1..k_s (may be NULL
 *          when s = 0).  k_0 - sum_l |k_l| must be > 0 at every node, the
 *          positivity the paper assumes in Sec. 3.2.
 *   f      host, nx*ny doubles: source values at the nodes (before FD
 *          weights).  May be NULL (zero source).
 *   beta   CSL shift for SG_PREC_CSL_MEAN (Sec. 4; the paper uses 1/2).
 *   point_source, point_x, point_y
 *          if point_source != 0, a unit point source delta(x - a) at
 *          a = point_x (1D) or (point_x, point_y) (2D) is added to f, with
 *          the discretisation of App. A.3: 1/h^dim at the grid node closest
 *          to a (of two equally close nodes, the one with the smaller index;
 *          for a = 1/2 the node t = ceil(q/2)), zero elsewhere.  a must lie
 *          in [0, 1] per coordinate (else SG_EINVAL); a source on an
 *          eliminated Dirichlet node contributes nothing.
 * The host arrays are read during sg_assemble only. */
typedef struct {
  int dim;
  int nx, ny;
  double h;
  int bc[4];
  int s, r;
  const double* k0;
  const double* kl;
  const double* f;
  double beta;
  int point_source;
  double point_x, point_y;
} sg_desc;

typedef struct {
  int dim;
  int mx, my;          /* unknown grid (x, y); n = mx * my */
  int n;               /* grid unknowns */
  int P;               /* chaos modes */
  long long N;         /* n * P */
  int s, r;
  int terms;           /* distinct coefficient fields of the coupling (2s + s(s-1)/2) */
  int coupling_nnz;    /* nonzeros of the union P x P coupling pattern (incl. diagonal) */
  int separable;       /* 1 if k_0 is constant: 2D preconditioners available */
  int specialised;     /* 1 if a register-resident matvec kernel serves (s, r) */
  int fast_diag;       /* 1 if FP32 2D preconditioner applies use the fast diagonalisation
                          (both directions transformed, tensor-core GEMMs; lines <= 320) */
  double eig_orth_err; /* separable 2D: max |Q^T Q - I| of the 1D pencils' eigenvector
                          factors (set-up rejects > 1e-10); 0 otherwise */
  double eig_kappa;    /* separable 2D: cond(Q) of those factors (set-up rejects > 100) */
  int tf32_route;      /* 1 if SG_TF32 applies are available (separable 2D, any line length);
                          the complex64 GMRES cycles then run flexible GMRES with them */
  int fp16_route;      /* 1 if SG_FP16 applies are available (and the complex64 GMRES
                          cycles use them unless sg_tune.tf32_transforms is set) */
} sg_info;

/* Builds the SG operator of Theorem 3.4 / Theorems A.1, A.2, A.5, A.6:
 * chaos tables, node fields on the device, and the factorisations of the
 * mean-value and CSL blocks (1D: tridiagonal LU with partial pivoting;
 * 2D with constant k_0: eigenvectors of the 1D pencil in x plus tridiagonal
 * LU with partial pivoting along y, all pivots in FP64).
 * Returns SG_EINVAL on inconsistent sizes (or more than 2^30 nodes), NaN/Inf fields or k <= 0,
 * SG_ESINGULAR if a factorisation meets a zero pivot.  *out is set only on
 * success. */
sg_status sg_assemble(const sg_desc* desc, void* stream, sg_handle** out);

/* Frees everything the handle owns (synchronises the device first).  NULL
 * is ignored. */
void sg_destroy(sg_handle* h);

sg_status sg_get_info(const sg_handle* h, sg_info* info);

/* Writes the SG right-hand side b = e_0 (x) b_0 of Sec. 3.1, b_0 = D_2
 * weights times f on the unknowns (F_0 of Theorem A.2, b_0 of Theorem A.6),
 * into the device buffer b (N complex, precision prec: FP64 or FP32). */
sg_status sg_rhs(sg_handle* h, sg_precision prec, void* b, void* stream);

/* Y = A X, the SG matrix A = I_P (x) L - i[B_ij] - [C_ij] of Theorem 3.4,
 * applied matrix-free: per grid point, the FD stencil of L on every mode
 * plus the P x P coupling sum_t c_t(x) G_t (Sec. 3.2, c_ij and b_ij of the
 * SG-then-FD route).  X and Y: device, N complex each, precision FP64 or
 * FP32, must not overlap. */
sg_status sg_matvec(sg_handle* h, sg_precision prec, const void* X, void* Y, void* stream);

/* Z = (I_P (x) S_blk)^-1 R for the chosen block (see sg_prec), one
 * factorisation applied to all P modes at once (the reshape of Sec. 6.3).
 * SG_PREC_NONE copies R to Z.  R and Z: device, N complex; Z may equal R
 * (in place).  prec SG_FP64, SG_FP32, SG_TF32 or SG_FP16 (complex64 data;
 * separable 2D problems only, SG_EUNSUPPORTED otherwise; SG_FP16 where
 * sg_info.fp16_route).
 * Returns SG_EUNSUPPORTED for 2D problems whose k_0 varies in space (no
 * separable factorisation).  Asynchronous: a bounded wait that gives up
 * inside a tensor-core transform sets the handle's device flag, which the
 * next sg_gmres call on the handle reports as SG_ETIMEOUT. */
sg_status sg_precond(sg_handle* h, sg_prec kind, sg_precision prec, const void* R, void* Z,
                     void* stream);

/* Largest N (= n * P complex values) sg_precond_noalloc accepts. */
#define SG_NOALLOC_MAX_N 524288

/* Allocation-free form of sg_precond (the paper has no counterpart: this is
 * an interface for callers, not part of the method).  Same result as
 * sg_precond for SG_PREC_MEAN and SG_PREC_CSL_MEAN, but the intermediate
 * vectors live in a fixed array inside the library image instead of the
 * handle's scratch, and the call allocates no device or host memory.  It is
 * meant for callers that cannot call cudaMalloc while they run (allocation
 * forbidden or too slow in their context, or device memory owned by another
 * allocator's pool); the handle itself must still come from sg_assemble.
 *   - N must be <= SG_NOALLOC_MAX_N, else SG_EINVAL with a message.
 *   - The array holds 2 * SG_NOALLOC_MAX_N complex128 values (16 MiB) on the
 *     device, until the process exits.  sg_assemble looks up its device
 *     address (cudaGetSymbolAddress), which is also what loads it under lazy
 *     module loading, so no call of this entry point loads code or commits
 *     memory.
 *   - All calls share the array: calls that overlap on the GPU (several
 *     streams or host threads) race.  Each call overwrites what it reads, so
 *     no clearing is needed between calls.
 *   - SG_FP32 on a 2D handle with the tensor-core transforms shares the
 *     handle's device timeout flag with sg_precond: a bounded wait that gives
 *     up there is reported by the next sg_gmres on the handle (SG_ETIMEOUT).
 * R, Z: device, N complex of precision prec (FP64 or FP32); Z may equal R. */
sg_status sg_precond_noalloc(sg_handle* h, sg_prec kind, sg_precision prec, const void* R, void* Z,
                             void* stream);

/* Use of a supplied initial guess (not in the paper, which starts from zero).
 *   SG_X0_AS_GIVEN:  start from x0.
 *   SG_X0_FALLBACK:  start from x0 unless ||b - A x0|| > ||b|| (or is not
 *                    finite); then start from zero.
 *   SG_X0_SCALED:    start from zeta x0 with zeta = (A x0)^H b / ||A x0||^2,
 *                    the multiple of x0 with the smallest residual (the
 *                    initial-guess scaling of Hegedus), so the starting
 *                    residual never exceeds ||b|| up to rounding; falls back
 *                    to zero like SG_X0_FALLBACK if it does.  Costs one extra
 *                    operator application and one reduction. */
typedef enum { SG_X0_AS_GIVEN = 0, SG_X0_FALLBACK = 1, SG_X0_SCALED = 2 } sg_x0_policy;

typedef struct {
  int restart;          /* Krylov basis length per cycle; <= 0 means full GMRES (no restart) */
  int maxit;            /* cap on total Arnoldi steps; <= 0 means N (FP64/FP32) */
  int max_outer;        /* SG_MIXED: cap on refinement steps; <= 0 means 20 */
  double tol;           /* stop when ||b - A x||_2 / ||b||_2 <= tol (Sec. 6.3) */
  double inner_tol;     /* SG_MIXED: inner relative reduction per refinement step (a step that can
                           reach tol within 20x of it aims at tol directly); <= 0 means 1e-5
                           (1e-3 with the binary16 basis, see basis16) */
  sg_prec prec;         /* right preconditioner M: A M^-1 y = b, x = M^-1 y (Sec. 6.3) */
  sg_precision mode;    /* SG_FP64, SG_FP32 or SG_MIXED */
  const void* x0;       /* initial guess (same memory space and precision as x); NULL = zero */
  int host_io;          /* 1: b, x0, x are HOST buffers (copied in and out inside the call) */
  int check_every;      /* steps between host reads of the convergence flag; <= 0 means 8 */
  int x0_policy;        /* sg_x0_policy: how a supplied x0 is used (0 = as given) */
  int side;             /* 0: right preconditioning A M^-1 y = b, x = M^-1 y, stopping on
                           ||b - A x|| / ||b||; 1: left, M^-1 A x = M^-1 b, stopping on
                           ||M^-1 (b - A x)|| / ||M^-1 b|| (Sec. 6.3 compares both; SG_FP64 and
                           SG_FP32 only) */
  int basis16;          /* SG_MIXED with right preconditioning on a problem whose binary16 route
                           runs (sg_info.fp16_route, transforms not tuned to TF32): 0 (default)
                           stores the cycles' Krylov basis as binary16 pairs (half the
                           orthogonalisation traffic; each cycle then reduces the residual by
                           about 1e-3, so inner_tol <= 0 means 1e-3 there, and the FP64
                           refinement takes one more step); -1 keeps it in complex64 */
} sg_gmres_opts;

typedef struct {
  int iters;            /* Arnoldi steps over all cycles (and refinement steps) */
  int outer;            /* SG_MIXED refinement steps (0 otherwise) */
  int cycles;           /* restart cycles */
  double relres;        /* final ||b - A x|| / ||b|| computed in FP64 (FP32 for SG_FP32) */
  sg_status status;
  double relres_prec;   /* the stopping quantity: ||M^-1 (b - A x)|| / ||M^-1 b|| for side = 1,
                           relres otherwise */
  int graph_outer;      /* sg_gmres_batched: refinement steps run inside the one-graph launch
                           (0 on the per-system route and for sg_gmres) */
} sg_gmres_info;

/* Solves A x = b with restarted, right-preconditioned GMRES: Arnoldi by
 * classical Gram-Schmidt applied twice, complex Givens rotations in FP64 on
 * the device, lazy normalisation of the basis (Sec. 6.3 names GMRES, this
 * library fixes the variant).  Complex64 cycles (SG_FP32, and the inner
 * cycles of SG_MIXED) on 2D problems whose preconditioner has the SG_TF32
 * route run flexible GMRES with that preconditioner (its SG_FP16 form where
 * it exists): z_j = M^-1 v_j is kept
 * for every step and the correction is sum_j y_j z_j, so the inexact
 * preconditioner changes the iteration count, not the attainable residual
 * (the workspace then holds restart more complex64 vectors).  b and x: N complex (complex128 for FP64 and
 * MIXED, complex64 for FP32), device memory unless opts->host_io.  Blocks
 * the calling host thread until the solve ends.  Returns SG_OK when relres
 * <= tol, SG_ENOTCONV with the last iterate in x otherwise, SG_EBREAKDOWN on
 * non-finite values, SG_ETIMEOUT if a bounded device-side wait gave up
 * during the solve (or in an earlier sg_precond on the handle; the flag is
 * cleared).  info may be NULL. */
sg_status sg_gmres(sg_handle* h, const sg_gmres_opts* opts, const void* b, void* x,
                   sg_gmres_info* info, void* stream);

/* Solves `count` independent SG systems (different grids, chaos sizes and
 * wavenumbers allowed) with the same options.
 *   - One-graph route (SG_MIXED, device buffers, right or no
 *     preconditioning, zero initial guesses or per-system guesses x0[k]
 *     under any x0_policy, opts->x0 NULL; taken unless concurrency < 0):
 *     the whole batch
 *     is ONE CUDA graph launch.  Each system is a chain of conditional nodes
 *     (refinement steps, chunks of 8 Arnoldi steps) whose conditions its own
 *     kernels set on the device, so restarts, refinements and convergence
 *     are decided without the host; per-system records are read back once.
 *     The graph is built and instantiated on the first call with a given
 *     set of handles, vectors and options and reused afterwards.  It unrolls
 *     4 refinement steps; a system still above tol after them continues on
 *     the per-system route from its current iterate (its info sums both);
 *     a system whose guess is worse than zero, or whose b is zero while a
 *     guess is given, is solved again on that route from the start (as
 *     sg_gmres restarts it).  Arithmetic per system is sg_gmres's, so the
 *     result equals a solve of that system alone.
 *   - Per-system route (otherwise): each system runs sg_gmres on its own
 *     internal CUDA stream, and up to `concurrency` systems (<= 0 means
 *     min(count, 16)) are in flight at once, driven by a pool of host
 *     threads.
 * Workspaces are allocated for all handles before any solve starts.  The solves wait for work already queued on
 * `stream` and are complete when the call returns.  h[k], b[k], x[k] as in
 * sg_gmres (opts->host_io is honoured per system); x0 (may be NULL): per
 * system initial guesses overriding opts->x0 (entries may be NULL = zero).
 * infos (may be NULL) gets one record per system.  Returns SG_OK if every
 * system converged, SG_ENOTCONV if some did not, otherwise the first error
 * met.  The handles must be distinct.  (The paper solves one system at a
 * time; batching is this library's throughput mode.) */
sg_status sg_gmres_batched(sg_handle* const* h, int count, const sg_gmres_opts* opts, const void* const* b,
                           void* const* x, const void* const* x0, sg_gmres_info* infos, int concurrency,
                           void* stream);

/* Stationary iteration with the mean-value splitting (Sec. 5; Sec. 7 runs it
 * with A_0): B x^(i+1) = b - (A - B) x^(i), i.e.
 * x^(i+1) = x^(i) + B^-1 (b - A x^(i)), with B = I_P (x) S_blk the block of
 * opts->prec (SG_PREC_MEAN: A_0; SG_PREC_CSL_MEAN: M_0).  It converges when
 * the spectral radius of I - B^-1 A is below one (small theta) and diverges
 * otherwise (the paper's wedge: theta = 0.1 converges, theta = 0.2 does not).
 *   x0_given  1: x holds the initial iterate on entry; 0: x^(0) = 0 (then
 *             x^(1) = B^-1 b, the paper's starting vector).
 *   maxit     steps at most; tol: stop when ||b - A x|| / ||b|| <= tol.
 *   mode      SG_FP64 (complex128 b, x) or SG_FP32 (complex64).
 * history (host, may be NULL): maxit + 1 doubles, relres of x^(0), x^(1), ...
 * up to the last iterate.  info (may be NULL): steps taken, final relres,
 * status, and diverged = 1 if the residual ended above 1e6 times the first
 * one (or became non-finite).  Returns SG_OK at tol, SG_ENOTCONV at maxit,
 * SG_EBREAKDOWN on a non-finite residual.  Device buffers; blocks the host
 * thread until done. */
typedef struct {
  sg_prec prec;
  sg_precision mode;
  int maxit;
  double tol;
  int x0_given;
} sg_stationary_opts;

typedef struct {
  int iters;
  double relres;
  int diverged;
  sg_status status;
} sg_stationary_info;

sg_status sg_stationary(sg_handle* h, const sg_stationary_opts* opts, const void* b, void* x,
                        sg_stationary_info* info, double* history, void* stream);

/* Post-processing of an SG solution V (N complex of precision prec, device;
 * Sec. 7): with the orthonormal chaos basis the expected value of
 * u~(x, xi) = sum_i V_i(x) phi_i(xi) is V_0(x), and the variances of its real
 * and imaginary parts are sum_{i>=1} (Re V_i(x))^2 and sum_{i>=1} (Im V_i(x))^2.
 *   mean     device, n complex (prec) or NULL
 *   var_re, var_im  device, n reals (prec) or NULL
 *   gamma    host, r + 1 doubles or NULL: gamma_j = max { ||V_i||_inf :
 *            total degree of phi_i = j }, j = 0..r (the magnitudes the paper
 *            plots against the degree); the call then synchronises `stream`.
 * The first call with gamma allocates a P-entry device buffer in the handle. */
sg_status sg_statistics(sg_handle* h, sg_precision prec, const void* V, void* mean, void* var_re, void* var_im,
                        double* gamma, void* stream);

/* ---------------------------------------------------------------------------
 * Learned initial guess (not in the paper: a throughput aid whose result is
 * always finished by sg_gmres to the same tolerance; the zero guess remains
 * the fallback).  A multilayer perceptron maps workload parameters to the
 * coefficients c of a rank-R basis U (rows U_i of N complex64 values, from a
 * POD of training solutions), and the guess is x0 = sum_i c_i U_i.
 * ------------------------------------------------------------------------- */
typedef struct sg_mlp sg_mlp;

/* in_dim -> width (tanh) x hidden -> out_dim (linear).  Parameters start at
 * zero; set them with sg_mlp_set_params.  Flat FP32 parameter layout:
 * for each layer l: W_l (d_{l+1} x d_l, row-major) then b_l (d_{l+1}). */
sg_status sg_mlp_create(int in_dim, int width, int hidden, int out_dim, sg_mlp** out);
void sg_mlp_destroy(sg_mlp* m);
long long sg_mlp_num_params(const sg_mlp* m);
/* src/dst: device, num_params FP32 values.  set also resets the Adam state. */
sg_status sg_mlp_set_params(sg_mlp* m, const float* src, void* stream);
sg_status sg_mlp_get_params(const sg_mlp* m, float* dst, void* stream);
/* Y = net(X); X: device batch x in_dim FP32, Y: device batch x out_dim FP32.
 * Products read bf16 copies of the weights and accumulate in FP32. */
sg_status sg_mlp_forward(sg_mlp* m, const float* X, int batch, float* Y, void* stream);
/* Mean squared error against T (batch x out_dim) and its gradient with
 * respect to every parameter (grad: device, num_params FP32; may be NULL).
 * *loss (host, may be NULL) is written after the call synchronises. */
sg_status sg_mlp_loss_grad(sg_mlp* m, const float* X, const float* T, int batch, double* loss, float* grad,
                           void* stream);
/* `epochs` passes over the nsamples rows of X, T (device) in mini-batches of
 * `batch` rows taken in order, one Adam step (lr; beta 0.9 / 0.999; eps
 * 1e-8) per mini-batch.  loss_history (host, epochs entries, may be NULL):
 * mean loss per epoch. */
sg_status sg_mlp_train(sg_mlp* m, const float* X, const float* T, int nsamples, int batch, int epochs, float lr,
                       double* loss_history, void* stream);

/* C[i][j] = sum_t conj(A[i][t]) B[j][t] for complex64 rows A_i (m rows,
 * stride lda) and B_j (n rows, stride ldb) of length k; C: m x n complex64
 * row-major.  workspace: device, m * n complex128 (FP64 accumulation of the
 * split long dimension).  Gram matrices and projections onto a basis. */
sg_status sg_cgemm_hn(const void* A, long long lda, const void* B, long long ldb, int m, int n, long long k, void* C,
                      void* workspace, void* stream);
/* C = A B for row-major complex64 A (m x k), B (k x n); C row-major m x n,
 * complex128 if out_c128 else complex64.  Expansion x = c U of a basis. */
sg_status sg_cgemm_nn(const void* A, const void* B, int m, int n, int k, void* C, int out_c128, void* stream);

/* A trained warm-start model: the network (not owned: it must outlive the
 * model), a copy of the decoder D = scale * U (rank rows of N complex64
 * values, device, row-major: the scaled rank-R basis of training
 * solutions) and the box [lo, hi] (host, in_dim doubles each, lo < hi) that
 * the network's inputs are normalised from.  The network's output width must
 * be 2 * rank (rank complex coefficients as interleaved pairs). */
typedef struct sg_warmstart sg_warmstart;
sg_status sg_warmstart_create(sg_mlp* net, const void* D, int rank, long long N, const double* lo, const double* hi,
                              sg_warmstart** out);
void sg_warmstart_destroy(sg_warmstart* w);
/* Initial guesses x0 for `count` parameter rows (params: host, count x
 * in_dim doubles, e.g. (kbar, sigma, correlation length, x_s, y_s)):
 * x0 (device, count x N complex128, row k for row k of params) =
 * net(2 (p - lo) / (hi - lo) - 1) viewed as rank complex values, times D.
 * Every step runs on the device in the library's kernels; the first call
 * with a larger count allocates the model's small input/output buffers.
 * Pass a row of x0 to sg_gmres as opts.x0 (with SG_X0_SCALED or
 * SG_X0_FALLBACK, so that a poor guess never starts above the zero guess). */
sg_status sg_warmstart_predict(sg_warmstart* w, const double* params, int count, void* x0, void* stream);

/* Message of the last failing call on this host thread ("" if none). */
const char* sg_last_error(void);

/* One of the four plain-TF32 transforms of the 2D fast-diagonalisation
 * preconditioner (the SG_TF32 apply of sg_precond is t = 0, 1, 2, 3 in turn;
 * the block solve for all P modes at once of Sec. 6.3, with S_blk^-1 =
 * (Qhat_y (x) Qhat_x) diag(1 / (lambda_y,j + lambda_x,i + shift))
 * (Qhat_y (x) Qhat_x)^T).  complex64, device buffers, per mode p (mxp, myp =
 * mx, my rounded up to even; pad entries of Y are written as zero):
 *   t = 0: Y_p = (X_p Qhat_x)^T        X [P][my][mx],  Y [P][mx][myp]
 *   t = 1: Y_p = L^-1 o (X_p Qhat_y)   X, Y [P][mx][myp]  (L^-1 of `kind`)
 *   t = 2: Y_p = (X_p Qhat_y^T)^T      X [P][mx][myp], Y [P][my][mxp]
 *   t = 3: Y_p = X_p Qhat_x^T          X [P][my][mxp], Y [P][my][mx]
 * kind: SG_PREC_MEAN or SG_PREC_CSL_MEAN.  X and Y must not overlap.  The
 * same kernels as the apply (a primitive for timing one transform and for
 * callers that fuse their own steps between them); SG_EUNSUPPORTED without the
 * fast-diagonalisation route.  Asynchronous on `stream`.
 * prec SG_TF32: the layouts above in complex64.  prec SG_FP16 (where
 * sg_info.fp16_route): the binary16 route of the solver's cycles: X of t = 0
 * and Y of t = 3 complex64, the others binary16 pairs with rows padded to a
 * multiple of 4 pairs (mx4, my4 in place of mxp, myp); t = 0 scales by
 * sqrt(N) (the input taken as unit norm), t = 1 by 1 / max |L^-1|, t = 3
 * divides both out. */
sg_status sg_fd_transform(sg_handle* h, sg_prec kind, sg_precision prec, int t, const void* X, void* Y,
                          void* stream);

/* One pass of the CGS2 orthogonalisation of Arnoldi step j in the complex64
 * flexible cycles that SG_MIXED runs with the mean-value preconditioner on 2D
 * separable problems (the step's largest kernels), in the form sg_gmres runs
 * by default (on the binary16 route: the binary16 basis), launched on
 * `stream` over the handle's GMRES workspace so that a caller can time it
 * with events on that stream:
 *   pass 0  prepares: sizes the workspace for GMRES(restart) (restart <= 0:
 *           30) as sg_gmres would and zeroes basis slots 0..j+1 and the
 *           device scalars;
 *   pass 1  the dots of w (the operator's output) with slots 0..j and, on
 *           the binary16 basis, of slot j with slots 0..j-1 (its delayed
 *           second projection), and the scale of the new slot;
 *   pass 2  the projection update of w, the new slot j+1 (binary16 on the
 *           binary16 basis), its norm and the Givens column of step j.
 * Values are meaningless (zeros); the work and the memory traffic are a
 * step's.  Each pass first clears the workspace's done flag (a 64-byte
 * memset on the stream).  SG_EINVAL for j out of the workspace or a pass out
 * of range, SG_EUNSUPPORTED where the two-pass form does not run.
 * Overwrites the workspace; must not run concurrently with another call on
 * the handle. */
sg_status sg_cgs2_pass(sg_handle* h, int restart, int j, int pass, void* stream);

/* ---------------------------------------------------------------- launch-shape tuning
 * Three launch shapes of the hot path depend on the problem (grid, P) and
 * are not fixed by the method (the paper times whole solves only):
 *   cgs_blocks_per_sm  grid of the CGS2 passes of every Arnoldi step, in
 *                      blocks per SM (1 .. 8); 0: the built-in rule (4);
 *   op_ctas_per_sm     CTAs per SM of the persistent complex64 SG operator
 *                      (1 .. 16, clamped to what fits); 0: as many as fit;
 *                      ignored by problems without that kernel;
 *   tc_tile_n          output tile width of the tensor-core transforms of 2D
 *                      separable preconditioners (64 or 128 real columns);
 *                      256: the binary16 transforms (SG_FP16) in the paired
 *                      form, two CTAs of a cluster on adjacent row tiles
 *                      sharing each B stage by multicast copies, the TF32
 *                      ones at 128 (SG_EUNSUPPORTED without the binary16
 *                      route or on a GPU that cannot hold such clusters);
 *                      0: the built-in rule per transform;
 *   tf32_transforms    1: the complex64 GMRES cycles apply the SG_TF32 form
 *                      of the preconditioner even where the SG_FP16 form
 *                      exists; 0: SG_FP16 where it exists.
 * None changes the operator, the preconditioner or the method: the operator
 * and the transforms give the same bits for every choice; the CGS2 grid
 * changes the order of the block sums of the inner products (rounding only,
 * still reproducible for a fixed choice); the transform precision changes the
 * preconditioner within its ~2e-3 accuracy (the flexible cycles absorb it).
 * The *_us fields are filled by sg_autotune: measured times of one step's
 * CGS2 passes at step restart / 2, one complex64 operator application and
 * one preconditioner apply of the cycles' form, as an Arnoldi step after
 * the first runs it (binary16 from the workspace's binary16 copy of the
 * basis vector where there is one; 0 where not timed). */
typedef struct {
  int cgs_blocks_per_sm;
  int op_ctas_per_sm;
  int tc_tile_n;
  int tf32_transforms;
  double cgs_us;
  double op_us;
  double apply_us;
} sg_tune;

/* Times the candidate shapes on this handle's problem (CUDA events on
 * `stream`, after warm-up; CGS2 with the complex64 basis of GMRES(restart),
 * restart <= 0 meaning 30, allocated like sg_gmres would) and applies the
 * fastest of each; *out (may be NULL) receives the choices and their times.
 * Overwrites the handle's GMRES workspace; must not run concurrently with
 * another call on the same handle.  Blocks until done. */
sg_status sg_autotune(sg_handle* h, int restart, sg_tune* out, void* stream);

/* The shapes in effect for this handle (0 = built-in rule), with the times
 * of the last sg_autotune (zeros if it never ran). */
sg_status sg_tune_get(const sg_handle* h, sg_tune* out);

/* Applies stored shapes (e.g. a table of sg_autotune results for this
 * problem size); the *_us fields are ignored.  SG_EINVAL for values out of
 * range.  Releases the GMRES workspace if the CGS2 grid changes (the next
 * solve allocates it again).  Must not run concurrently with another call
 * on the same handle. */
sg_status sg_tune_set(sg_handle* h, const sg_tune* t);

/* Number of CUDA kernels this library has launched in this process so far
 * (all handles, all threads; a diagnostic for benchmarks). */
long long sg_kernel_launches(void);

/* ABI version: 100 * major + minor. */
int sg_version(void);

/* Measured arithmetic peak of the GPU's CUDA cores (not in the paper: a
 * diagnostic for roofline figures).  Runs a kernel of independent fused
 * multiply-add chains (FP64 if fp64 != 0, else FP32) over the whole GPU,
 * timed with CUDA events, and writes the rate in TFLOP/s (2 flop per FMA) to
 * *tflops.  Synchronises `stream`; allocates and frees a small buffer. */
sg_status sg_alu_peak(int fp64, double* tflops, void* stream);

/* Check of the device-side failure detection (not in the paper).  Launches
 * one warp that waits, through the bounded mbarrier wait of the
 * preconditioner's tensor-core transform kernel, for a barrier phase that
 * nothing completes (count 1, no arrival, no copy in flight).  The wait gives
 * up after its limit (0.5 s of %globaltimer), the kernel records that in a
 * device flag, as the transform kernel does, and returns; the CUDA context
 * stays usable.
 *   stream     CUDA stream (NULL: legacy default stream); the call synchronises it.
 *   timed_out  host int, out: 1 if the wait gave up, 0 if it completed.
 *   seconds    host double, out (may be NULL): kernel time by CUDA events.
 * Returns SG_ETIMEOUT when the wait gave up (the designed outcome), SG_OK if
 * the barrier completed (a defect of the wait), SG_EINVAL for NULL timed_out,
 * SG_ECUDA on a CUDA error or if the kernel did not reach its end.  Allocates
 * and frees 8 bytes of device memory. */
sg_status sg_selftest_wait_timeout(void* stream, int* timed_out, double* seconds);

#ifdef __cplusplus
}
#endif
#endif

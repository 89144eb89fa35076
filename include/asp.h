/*
 * asp.h -- C ABI of the GB300 additive sweeping preconditioner library (libasp.so).
 *
 * The library solves the PML-truncated Helmholtz equation
 *     Delta u + omega^2 / c(x)^2 u = f   on (0,1)^d,  u = 0 on the boundary,
 * (Liu & Ying, "Additive Sweeping Preconditioner for the Helmholtz Equation",
 * 2016, Section 1, Eq. (1)) discretized by the central-difference scheme with a
 * perfectly matched layer on every side (Section 2, Eq. (2); Section 3.1, Eq. (4);
 * Section 3.2 puts the PML on all sides), preconditioned by the additive sweeping
 * preconditioner (Section 3.1, Algorithms 1 and 2) inside flexible GMRES
 * (Section 3.2).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Grid.  n interior nodes per axis, h = 1/(n+1), node i at x = i*h (Section 2).
 *        dim = 2 or 3 (Section 4 for 3D).
 * Vectors.  A batch of nrhs grid functions is stored point-major with the
 *        right-hand side fastest ("RHS-interleaved"):
 *            2D: element (i1, i2, r)     at ((i2-1)*n + (i1-1))*nrhs + r,
 *            3D: element (i1, i2, i3, r) at (((i3-1)*n + (i2-1))*n + (i1-1))*nrhs + r,
 *        i.e. for nrhs = 1 exactly the paper's column-major ordering (x1 fastest,
 *        Section 3.1).  The sweep axis is the slowest one: x2 in 2D, x3 in 3D
 *        (layers are columns in 2D and slabs of planes in 3D).  Complex numbers are interleaved
 *        (re, im) pairs: complex128 = two doubles.  All vector arguments are
 *        DEVICE pointers unless the name says _host.
 * Streams.  `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *        stream).  Work is enqueued on it; calls return once it is enqueued, except
 *        where a call says it synchronizes.
 * Ownership.  The caller owns every pointer it passes; the library copies what it
 *        keeps (the velocity field).  The library owns the device memory it
 *        allocates for a handle (factors, transfer maps, Krylov workspace) and
 *        frees it in asp_destroy.
 * Threads.  One handle is used by one thread at a time (calls on the same
 *        handle are not synchronized against each other); different handles may
 *        be used concurrently from different threads, each on its own stream
 *        (the serving loop does so).  Library-wide state (job-list caches, kernel
 *        attributes, the test hook) is synchronized internally.
 * Errors.  Every int-returning call returns ASP_OK (0) or a negative ASP_ERR_*
 *        code; asp_error_string() names it and asp_last_error_detail() gives a
 *        one-line description of the most recent failure on the calling thread.
 *        No call traps, asserts or spins without a bound on the device: device
 *        waits have iteration limits and report ASP_ERR_TIMEOUT.
 */
#ifndef ASP_H
#define ASP_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ------------------------------------------------------- */
#define ASP_OK 0
#define ASP_ERR_INVALID -1        /* argument out of range / inconsistent sizes   */
#define ASP_ERR_OOM -2            /* device allocation failed                     */
#define ASP_ERR_CUDA -3           /* a CUDA runtime call failed                   */
#define ASP_ERR_SMALL_PIVOT -4    /* zero or non-finite pivot in a layer factor   */
#define ASP_ERR_NOT_CONVERGED -5  /* FGMRES hit maxit before the tolerance        */
#define ASP_ERR_TIMEOUT -6        /* a bounded device-side wait gave up           */
#define ASP_ERR_STATE -7          /* call made in the wrong order (e.g. no factor) */
#define ASP_ERR_UNSUPPORTED -8    /* valid request this build does not implement  */

/* ---- precision of the layer factors and preconditioner applies ---------- */
#define ASP_PREC_C128 0 /* complex128 factors and applies (plain FP64 path)      */
#define ASP_PREC_C64 1  /* complex64 factors and applies inside FP64 FGMRES      */
/* complex64 as ASP_PREC_C64, with every 2D layer factor block stored as the
 * packed upper triangle of the complex-symmetric W_k Delta (Section 3.1,
 * practical remark 4: the symmetric version saves memory): half the factor
 * bytes, at the cost of expanding each block in shared memory during the
 * layer solves (slower applies).  Not available in 3D (ASP_ERR_UNSUPPORTED). */
#define ASP_PREC_C64_SYM 2

/* ---- solver of the 3D slab subproblems ---------------------------------- */
/* block elimination over the x2 planes: n dense blocks of n*w unknowns per
 * slab, each inverted (Gauss-Jordan, tensor-core updates for complex64)      */
#define ASP_SLAB_BLOCK 0
/* nested dissection (Section 4, Algorithms 3 and 4): the unknowns of a slab
 * grouped along x3 into columns, the n x n grid of columns ordered by nested
 * dissection, a multifrontal factorization with dense fronts (partial
 * Gauss-Jordan with pivoting inside the fully summed rows); fewer flops and
 * factor bytes than ASP_SLAB_BLOCK.  3D only.                                  */
#define ASP_SLAB_ND 1

/* Problem parameters (Section 2 and Section 3.1 notation).
 *   dim        spatial dimension (2 or 3)
 *   n          interior nodes per axis; h = 1/(n+1)
 *   omega      angular frequency (> 0)
 *   pml        gamma: boundary PML width eta = gamma*h (>= 2)
 *   pml_aux    gamma_a: width of the auxiliary PMLs of the padded layer grids
 *              (Section 3.1, practical remark 2); 0 means gamma_a = gamma
 *   b          interior layer width in grid columns (planes in 3D) along the
 *              sweep axis (>= 1); with P = n + 2 - 2*gamma physical columns there
 *              are m = floor(P/b) layers and the last one absorbs the remainder
 *              P - m*b
 *   C          PML strength: sigma = (C/eta) (d/eta)^2 at distance d past the
 *              physical edge (Section 2); > 0
 *   factor_prec ASP_PREC_C128, ASP_PREC_C64 or ASP_PREC_C64_SYM
 *   max_rhs    largest nrhs that later calls will pass (1..256); sizes the
 *              apply and Krylov workspaces
 *   restart    FGMRES restart length the workspace is sized for (1..64)
 *   slab_solver ASP_SLAB_BLOCK (0, the default) or ASP_SLAB_ND; 3D only       */
typedef struct asp_params {
  int dim;
  int n;
  double omega;
  int pml;
  int pml_aux;
  int b;
  double C;
  int factor_prec;
  int max_rhs;
  int restart;
  int slab_solver;
} asp_params;

typedef struct asp_handle asp_handle;

/* Per-right-hand-side result of asp_gmres_solve (host memory, caller-owned). */
typedef struct asp_solve_info {
  int iterations;       /* preconditioner applications until the estimate met tol */
  int converged;        /* 1 if the true relative residual is <= tol               */
  double rel_res_est;   /* FGMRES residual estimate / ||f|| at exit                */
  double rel_res_true;  /* ||f - A u|| / ||f|| recomputed in FP64 at exit          */
} asp_solve_info;

/* asp_setup: validate `p`, build the layer partition (Section 3.1: X_p, X_q^M,
 * X_p^R, X_p^L), compute the PML profiles, copy the velocity c (n^dim doubles,
 * natural ordering, HOST memory if c_is_device == 0, else DEVICE) and allocate
 * the handle's device memory.  Returns ASP_ERR_INVALID for out-of-range
 * parameters or a non-positive / non-finite velocity, ASP_ERR_UNSUPPORTED for a
 * valid problem this build does not take (2D: a padded layer wider than 64
 * columns, or n above 16 * (SMs / 2) = 1216 on a 152-SM GPU with three or more
 * layers, since the sweep chain holds at most 16 map rows per CTA on half of
 * the SMs; 3D: a slab block n * (padded width) above 3072 unknowns),
 * ASP_ERR_OOM if the footprint does not fit.  Synchronizes the device before
 * returning. */
int asp_setup(const asp_params* p, const double* c, int c_is_device, asp_handle** out);

/* asp_setup_layers: asp_setup with layers of arbitrary physical widths
 * (Section 3.1, practical remark 3: the widths need not be equal and can be
 * chosen larger where the velocity varies heavily).  widths (HOST, nwidths
 * entries) are the numbers of physical columns (planes in 3D) of layers
 * 1..m along the sweep axis, each >= 1, summing to n + 2 - 2*gamma; X_1 also
 * holds the gamma - 1 boundary-PML columns before it and X_m those after it.
 * p->b is not used for the partition.  widths = NULL gives asp_setup's
 * partition.  Every other rule of asp_setup applies (2D padded widths
 * 2*gamma_a + b_p - 2 <= 64, the auxiliary padding of the second and the
 * second-to-last layer inside the grid: gamma_a <= gamma + min(b_1, b_m)). */
int asp_setup_layers(const asp_params* p, const int* widths, int nwidths, const double* c, int c_is_device,
                     asp_handle** out);

/* Layer widths chosen from the velocity (Section 3.1, practical remark 3):
 * layers of at least b_min physical columns, grown (up to b_max) while the
 * next column boundary falls where the velocity jumps heavily along the sweep
 * axis (relative jump above 4 times its median over the physical region, and
 * above 1e-3), so that auxiliary PMLs are placed where the medium is smooth;
 * the last layer takes the remainder.  c: HOST, n^dim doubles, natural
 * ordering.  Writes at most `capacity` widths and returns their number m, or
 * ASP_ERR_INVALID.  Host-only; no device work. */
int asp_layer_widths_from_velocity(const asp_params* p, const double* c, int b_min, int b_max, int* widths,
                                   int capacity);

/* Host-only check of the nested-dissection plan (ASP_SLAB_ND) of an n x n
 * grid of columns with w planes each (Section 4: unknowns grouped along x3,
 * nested dissection of the column grid).  Fills up to `nstats` (<= 9) of:
 * [0] tree nodes, [1] largest depth, [2] largest front (unknowns), [3] factor
 * entries ([X; L] and P of every front), [4] stencil entries the fronts
 * assemble, [5] nonzeros of the slab's 7-point operator, [6] couplings
 * assembled more than once, [7] couplings never assembled, [8] complex
 * multiply-adds of the fronts' Gauss-Jordan steps.  A valid plan has
 * [4] == [5] and [6] == [7] == 0.  Returns ASP_ERR_INVALID for n < 1 or w < 1.
 * No device work. */
int asp_nd_plan_check(int n, int w, long long* stats, int nstats);

/* Bytes of device memory asp_setup + asp_factor will hold for these
 * parameters (factors, transfer maps, apply and Krylov workspaces).  Pure
 * function of `p` and the device's SM count (152 without a device); 0 for
 * invalid or unsupported parameters. */
size_t asp_footprint_bytes(const asp_params* p);
/* The same for asp_setup_layers' partition (widths = NULL: uniform). */
size_t asp_footprint_bytes_layers(const asp_params* p, const int* widths, int nwidths);

/* Number of layers m, and the partition of layer p (1-based): X_p = [x_lo, x_hi]
 * along the sweep axis (global 1-based indices).  Returns ASP_ERR_INVALID for a
 * bad p. */
int asp_num_layers(const asp_handle* h);
int asp_layer_range(const asp_handle* h, int p, int* x_lo, int* x_hi);

/* asp_factor: Algorithm 1.  Factors H_q^M (q=1..m), H_p^R (p=2..m) and H_p^L
 * (p=1..m-1) in the precision chosen at setup, all in one batched launch, and
 * builds the dense trace-transfer maps of the R and L sweeps (the linear maps
 * from a layer's incoming boundary trace to the outgoing trace of G~_p^R /
 * G~_p^L, Section 3.1 "Putting together").  In 3D every slab subproblem is
 * factored by blocked Gauss-Jordan over its x2 planes (dense blocks of
 * n*w unknowns; complex64 factors do the rank-256 Schur updates on the tensor
 * cores) and no transfer maps are built.  Enqueued on `stream`; the pivot
 * check synchronizes `stream` and returns ASP_ERR_SMALL_PIVOT if any block
 * pivot was zero or non-finite. */
int asp_factor(asp_handle* h, void* stream);

/* z = M^-1 r: Algorithm 2 (M-solves of every layer, right-going and
 * left-going sweeps with accumulated boundary values, and the sum), for nrhs
 * right-hand sides.  r and z are complex128 DEVICE vectors in the
 * RHS-interleaved layout; they may not alias.  1 <= nrhs <= max_rhs.  Requires
 * asp_factor.  Enqueued on `stream`. */
int asp_apply_preconditioner(asp_handle* h, const void* r, void* z, int nrhs, void* stream);

/* y = A x: the 5-point operator of Eq. (4) with the PML on all four sides (3D:
 * the 7-point operator, PML on all six sides), for nrhs complex128 DEVICE
 * vectors (RHS-interleaved, no aliasing).  Needs only asp_setup.  Enqueued on
 * `stream`. */
int asp_matvec(asp_handle* h, const void* x, void* y, int nrhs, void* stream);

/* One layer subproblem on its own (for checking): v = H^-1 g for the
 * subproblem kind (0 = H_p^M, 1 = H_p^R, 2 = H_p^L) of layer p, with g and v
 * complex128 DEVICE arrays of shape [w][n][nrhs] (2D: padded x2 columns of the
 * subproblem outermost, x1, then the right-hand side) or [w][n][n][nrhs] (3D:
 * padded x3 planes, x2, x1, right-hand side), w = asp_subproblem_width.
 * Uses the stored factors.  Enqueued on `stream`. */
int asp_subproblem_width(const asp_handle* h, int kind, int p);
int asp_subproblem_solve(asp_handle* h, int kind, int p, const void* g, void* v, int nrhs,
                         void* stream);

/* asp_gmres_solve: right-preconditioned flexible GMRES (Section 3.2), zero
 * initial guess, restart `restart` (<= the setup value), FP64 Arnoldi
 * (classical Gram-Schmidt, with a second pass for a right-hand side whose new
 * vector lost more than a factor 1000 of its norm) and Givens rotations on the
 * device,
 * independent Krylov spaces per right-hand side.  Stops a right-hand side when
 * its residual estimate / ||f|| <= tol; stops when all have stopped or after
 * `maxit` iterations.  tol = 0 with maxit = k runs exactly k iterations.
 * f and u are complex128 DEVICE vectors (RHS-interleaved); u is written even
 * when ASP_ERR_NOT_CONVERGED is returned.  info_host (nrhs entries, HOST) may
 * be NULL.  Synchronizes `stream` once per iteration to read the convergence
 * flags, and before returning. */
int asp_gmres_solve(asp_handle* h, const void* f, void* u, int nrhs, double tol, int restart,
                    int maxit, asp_solve_info* info_host, void* stream);

/* asp_autotune: choose the launch shapes of the layer solves of an apply
 * with nrhs right-hand sides by timing them.  For the M-solves and for the
 * sweep fills it times, on this handle's own factors, each candidate shape --
 * right-hand sides per job (the tile's column capacity) and the compiled tile
 * variant: the default capacity for nrhs, its alternative tile where one
 * exists (complex64 at 32 and at 1 right-hand side), and the next smaller
 * capacity -- one untimed and three timed launches each, and keeps the
 * fastest for later applies with this nrhs.  The input contents are not used
 * for the choice (the apply workspace is timed as it is).  choice_host (HOST,
 * 4 ints, may be NULL): capacity and variant chosen for the M-solves, then for
 * the fills.  ms_host (HOST, 6 doubles, may be NULL): mean milliseconds of each
 * candidate (M-solves first, 0 where a candidate does not exist or does not
 * fit the widths).  Requires asp_factor; 3D handles have nothing to tune
 * (ASP_OK).  Synchronizes `stream`. */
int asp_autotune(asp_handle* h, int nrhs, int* choice_host, double* ms_host, void* stream);

/* asp_set_solve_shape: use the launch shape (cap, variant) -- one of the
 * candidates asp_autotune times, listed there -- for the layer solves of kind
 * 0 (M-solves) or 1 (sweep fills) in later applies with `nrhs` right-hand
 * sides, instead of the default or the autotuned choice (2D handles).  Every
 * shape computes the same result; this fixes the choice (reproducible runs,
 * tests of each compiled tile).  ASP_ERR_INVALID for a shape that is not a
 * candidate at this nrhs, ASP_ERR_UNSUPPORTED on 3D handles.  Host-only. */
int asp_set_solve_shape(asp_handle* h, int nrhs, int kind, int cap, int variant);

/* Number of kernel launches this handle has issued since the last call (the
 * counter is reset by the call).  Used to report how many of the library's
 * kernels ran in a timed region. */
long long asp_take_launch_count(asp_handle* h);

/* Phase timing (measurement).  When enabled, the library records a CUDA event
 * before and after each of its launches on the launching stream and attributes
 * the interval to a phase:
 *   0 factor (block inversions)      1 transfer maps     2 M-solves (EMBED)
 *   3 sweep chain                    4 sweep fills       5 sum
 *   6 matvec                         7 FGMRES vector kernels
 *   8 3D tensor-core Schur updates (the rank-256 updates of the slab factor;
 *     their time is also part of phase 0)
 *   9 diagonal blocks of the sweep subproblems' inverses (complex64 maps built
 *     on the tensor cores; phase 1 is then the tensor-core map kernel alone)
 * In 3D, phase 0 is the whole slab factor per stream, phase 2 the launch of
 * all M-slab solves and phase 4 the paired sweep launches.
 * asp_phase_times synchronizes the device, writes per-phase total milliseconds
 * and launch counts (HOST arrays of nphases <= ASP_NUM_PHASES entries) and
 * resets the records.  Timing adds two event records per launch; it is off by
 * default. */
#define ASP_NUM_PHASES 10
int asp_set_phase_timing(asp_handle* h, int enable);
int asp_phase_times(asp_handle* h, double* ms, long long* launches, int nphases);

/* ---- allocation-free residual check ------------------------------------
 * asp_residual_norms_noalloc: rel_res[r] = ||f_r - A u_r|| / ||f_r|| (0 when
 * f_r = 0) for r < nrhs, with A the operator of asp_matvec for the problem in
 * `p` (dim, n, omega, pml, C are read; the other fields are ignored).  The
 * paper has no counterpart of this call.  It is for callers that cannot
 * allocate device memory -- a process whose device memory belongs to another
 * allocator (a framework's caching pool, a fixed arena), or a serving loop
 * that must not allocate once it runs -- and therefore takes no handle.
 *   c        DEVICE, n*n doubles, the velocity in the natural ordering; every
 *            entry must be positive and finite, else every rel_res entry is NaN
 *   f, u     DEVICE complex128 vectors, RHS-interleaved as everywhere
 *   rel_res  DEVICE, nrhs doubles, written
 * It allocates nothing: its temporaries live in one fixed device array inside
 * the library (about 0.7 MB, held on every GPU that loads the library until the
 * process exits), sized for n <= ASP_NOALLOC_MAX_N and nrhs <=
 * ASP_NOALLOC_MAX_RHS; larger requests return ASP_ERR_INVALID.  The first call
 * on a device looks up that array's device address (cudaGetSymbolAddress), so
 * make the first call on each device before any stream capture.  All calls
 * share the array: calls that overlap on the GPU race and may return wrong
 * values, so order them (one stream, or events).  Enqueued on `stream`. */
#define ASP_NOALLOC_MAX_N 4096
#define ASP_NOALLOC_MAX_RHS 64
int asp_residual_norms_noalloc(const asp_params* p, const double* c, const void* f, const void* u, int nrhs,
                               double* rel_res, void* stream);

/* Self-test of failure detection on the device.  Launches one CTA that waits,
 * with the library's bounded mbarrier wait and a limit of `polls` polls, on a
 * barrier that nothing arrives on.  Every device-side wait of the library gives
 * up the same way (after 2^26 polls) and reports through the error word; this
 * call runs that path on purpose with a short limit.  Expected result:
 * ASP_ERR_TIMEOUT, with the context still usable for further calls.  ASP_OK would
 * mean the barrier completed (a library defect).  polls: 1 .. 2^26, else
 * ASP_ERR_INVALID.  Allocates and frees 8 bytes of device memory; synchronizes
 * `stream`. */
int asp_selftest_bounded_wait(int polls, void* stream);

/* Host-side fault injection for tests of the allocation-failure path: after
 * `after` more device allocations made by asp_setup / asp_setup_layers (0: the
 * next one), one allocation is reported as failed without calling the CUDA
 * allocator; the hook then disarms itself.  The setup must return ASP_ERR_OOM
 * and leave no device memory behind.  after < 0 disarms the hook.  Host-only
 * state, process-wide; returns ASP_OK. */
int asp_testhook_fail_device_alloc(int after);

/* Free everything the handle owns.  NULL is accepted; calling it twice on the
 * same pointer is undefined (the handle is gone after the first call). */
void asp_destroy(asp_handle* h);

/* Static name of an error code ("ASP_OK", "ASP_ERR_INVALID", ...). */
const char* asp_error_string(int code);

/* One-line description of the last failure on the calling thread (static
 * thread-local storage, overwritten by the next failure). */
const char* asp_last_error_detail(void);

#ifdef __cplusplus
}
#endif

#endif /* ASP_H */

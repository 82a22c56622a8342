/*
 * st.h -- C ABI of the GB300 space-time Petrov-Galerkin heat solver.
 *
 * The solver computes the discrete solution of the heat equation
 * u_t + A u = f, u(0) = 0, discretised in space and time together with the
 * Petrov-Galerkin pair "hat functions in time (x) X_h" (trial) and
 * "piecewise constants in time (x) X_h" (test) of Henning, Palitta, Simoncini
 * and Urban, "Matrix oriented reduction of space-time Petrov-Galerkin
 * variational problems" (arXiv:1912.10082), Section 3.  The linear system
 * B u = f with B = D_t (x) M + C_t (x) A (Section 3, eq. par1) is never
 * assembled; it is handled in its matrix form (Section 4)
 *
 *     M U D_t^T + A U C_t^T = F,   F = F1 F2^T                      (1)
 *
 * U is N_h x N_t, column k holding the coefficients of the trial function
 * sigma^k (nodal values at t^k = k dt).  D_t = bidiag(1 | -1) and
 * C_t = (dt/2) bidiag(1 | 1) are lower bidiagonal (rows: test functions).
 * M and A are the spatial mass and operator matrices on a shared CSR pattern.
 *
 * Conventions
 *  - Every call returns an int status: ST_OK (0) or a negative ST_E* code.
 *    No C++ exception crosses this boundary.
 *  - Dense matrices are column-major with an explicit leading dimension.
 *  - "device" pointers are CUDA global memory of the current device; a few
 *    inputs also accept host memory, as documented per argument (the library
 *    tells them apart with cudaPointerGetAttributes).
 *  - A problem handle is not thread-safe; distinct handles are independent.
 *    Work is issued on the handle's stream.  Calls that return results through
 *    host memory synchronise that stream before returning.
 *  - Spatial nodes are the interior nodes of a box, numbered lexicographically
 *    with x fastest (homogeneous Dirichlet data, Section 2).
 */
#ifndef ST_H_
#define ST_H_

#ifdef __cplusplus
extern "C" {
#endif

#define ST_ABI_VERSION 1

/* status codes */
#define ST_OK          0
#define ST_EINVAL     -1   /* invalid argument (sizes, pointers, descriptor) */
#define ST_ENOMEM     -2   /* a device or host allocation failed */
#define ST_ENOTCONV   -3   /* maxit or max_basis reached above tol; best iterate returned */
#define ST_EBREAKDOWN -4   /* the Krylov block lost rank and nothing was left to add */
#define ST_ECUDA      -5   /* a CUDA runtime call or kernel launch failed */
#define ST_ETIMEOUT   -6   /* a bounded device-side wait gave up */
#define ST_ENOTSUP    -7   /* the requested operation needs a feature this problem lacks */

/* precision modes of st_solve */
#define ST_FP64  0   /* every N_h-sized step in FP64 */
#define ST_MIXED 1   /* FP32 fast-diagonalisation solves refined to FP64 accuracy (Section 4 solve, see st_solve) */

/* element types of st_apply */
#define ST_F64 0
#define ST_F32 1

/* spatial operators (Section 2: A elliptic, a coercive) */
#define ST_HEAT     0   /* a(u,v) = kappa (grad u, grad v) */
#define ST_CONVDIFF 1   /* a(u,v) = eps (grad u, grad v) + (beta . grad u, v) */

typedef struct st_problem st_problem;

/* Problem description, read by st_setup only.  Zero-initialise, then set. */
typedef struct st_desc {
    int dim;            /* 1, 2 or 3: uniform box grid, P1 (dim 1) / Q1 (dim 2, 3) elements;
                           0: user-supplied CSR matrices (fields n_h ... a_vals) */
    int n[3];           /* interior nodes per direction (x, y, z); n[d] >= 1 */
    double length[3];   /* box edge lengths; <= 0 means 1.0 */
    int op;             /* ST_HEAT or ST_CONVDIFF */
    double kappa;       /* ST_HEAT diffusion coefficient (> 0; 0 means 1.0) */
    double eps;         /* ST_CONVDIFF diffusion (> 0) */
    double beta[3];     /* ST_CONVDIFF velocity */
    int n_t;            /* number of uniform time intervals N_t (>= 1) */
    double T;           /* final time (> 0); dt = T / N_t (Section 3) */
    /* dim == 0 only: host arrays copied by st_setup; shared sorted CSR pattern */
    int n_h;            /* number of spatial unknowns */
    int nnz;
    const int* row_ptr; /* n_h + 1 entries, row_ptr[0] == 0 */
    const int* col_idx; /* nnz entries, ascending within each row */
    const double* m_vals; /* mass matrix values M */
    const double* a_vals; /* operator matrix values A */
    /* solver controls */
    int precision;      /* ST_FP64 or ST_MIXED */
    double tol;         /* target relative residual ||F - op(U)||_F / ||F||_F; <= 0 means 1e-8 (Section 5) */
    int maxit;          /* maximum rational Krylov iterations; <= 0 means 400 */
    int max_basis;      /* maximum basis columns; <= 0 means 2048 */
    void* stream;       /* cudaStream_t to issue work on; NULL = default stream */
} st_desc;

/* Low-rank solution U ~= V Y returned by st_solve. */
typedef struct st_solution {
    int n_h, n_t, k;      /* V is n_h x k, Y is k x n_t */
    const double* V;      /* device, column-major, ld = n_h; owned by the handle,
                             valid until the next st_solve or st_destroy */
    const double* Y;      /* device, column-major, ld = k; owned by the handle */
    double* U_dense;      /* in: optional caller-owned device buffer for U = V Y (NULL: skip) */
    int ldu;              /* in: leading dimension of U_dense (>= n_h) */
} st_solution;

/* Statistics of one st_solve. */
typedef struct st_stats {
    int iterations;       /* rational Krylov iterations (shifted solves) */
    int basis_cols;       /* k = columns of V; memory is k * (N_h + N_t) numbers (Section 5, Table 1 mu_mem) */
    int rank;             /* numerical rank of U: #{singular values of Y > 1e-8 * largest} */
    int p;                /* rank of F after compression */
    int converged;        /* 1 if relres <= tol */
    int residual_checks;  /* how many times the projected equation was solved */
    int mu_mem;           /* basis columns allocated, including the block computed at the last
                             iteration (Section 5, Table 1: mu_mem = Its + 1 for a rank-1 load) */
    double relres;        /* final relative residual, FP64 */
    double ms_total;      /* wall time of the call (host clock) */
    double ms_phase[8];   /* host clock between synchronisation points: 0 compress, 1 shifted solves and
                             block Gram-Schmidt, 2 block QR, 3 products of the new block,
                             4 projected solve, 5 residual, 6 output, 7 other */
    double shift_min, shift_max;  /* extremes of the shifts s used, as (A + s M)^{-1} */
    int inner_iterations; /* convection-diffusion: preconditioned FGMRES steps of all shifted solves */
} st_stats;

/* st_setup -- build a problem handle (Section 3: spatial matrices M_h, A_h;
 * time grid t^k = k dt).  For dim 1..3 the library assembles the P1/Q1 mass
 * and operator matrices on the device (Kronecker products of 1D
 * M = h/6 tridiag(1,4,1), K = 1/h tridiag(-1,2,-1), G = 1/2 tridiag(-1,0,1))
 * and tables for the fast-diagonalisation shifted solve.  For dim == 0 the
 * CSR arrays are copied from host memory (st_solve, st_shift_solve and
 * st_solve_lrfgmres then use the algebraic inner solver for heat problems;
 * st_timestep_cn returns ST_ENOTSUP: it needs the tensor-grid solver).
 * Ownership: the handle owns every device buffer it allocates until
 * st_destroy.  Errors: ST_EINVAL (bad sizes or fields, nnz > INT_MAX),
 * ST_ENOMEM, ST_ECUDA.  *out is NULL on error. */
int st_setup(const st_desc* d, st_problem** out);

/* st_destroy -- free the handle and everything it owns.  NULL is accepted.
 * The handle's pinned host staging goes back to a library-wide pool for the
 * next handle or batch instead of being freed: freeing pinned memory (like a
 * synchronous device free) waits for the whole device, which would stall the
 * solves of other handles.  The pool keeps its buffers for the life of the
 * process (at most the largest staging in use at once, per size class). */
int st_destroy(st_problem* p);

/* st_problem_info -- sizes of a problem (host outputs, any may be NULL). */
int st_problem_info(const st_problem* p, int* n_h, int* n_t, int* nnz, double* dt);

/* st_p1_mesh_csr -- P1 mass matrix M and heat operator A = kappa (grad u, grad v) of a simplex mesh on its
 * interior nodes (paper Section 3: X_h the continuous piecewise linear functions vanishing on the boundary;
 * Example 1 uses such meshes), assembled on the host in CSR form with one shared, sorted pattern -- the input of
 * st_setup's dim == 0 path (st_desc.row_ptr, col_idx, m_vals, a_vals).
 *   dim            2 (triangles) or 3 (tetrahedra)
 *   n_nodes, xyz   node coordinates, n_nodes x dim, row-major (node i at xyz[i*dim .. i*dim+dim-1])
 *   n_elems, elems vertex indices, n_elems x (dim+1), row-major
 *   interior       n_nodes flags: nonzero for the nodes that carry unknowns (Dirichlet nodes are 0); the
 *                  unknowns are numbered in node order
 *   row_ptr (n_h+1), col_idx, m_vals, a_vals (nnz): caller-owned outputs; pass NULL for all four to get
 *                  the sizes only, then call again with arrays of those sizes
 *   n_h, nnz       outputs: interior node count and nonzeros of the shared pattern
 * Element T, vertices x_0..x_d, B = [x_1 - x_0, ..., x_d - x_0]: |T| = |det B| / d!, barycentric gradients the
 * rows of B^-1 and minus their sum; local stiffness kappa |T| grad l_i . grad l_j, local mass
 * |T| (1 + delta_ij) / ((d+1)(d+2)).  Host only (no GPU call).  ST_EINVAL on bad sizes, an index out of
 * range or a degenerate element. */
int st_p1_mesh_csr(int dim, int n_nodes, const double* xyz, int n_elems, const int* elems,
                   const unsigned char* interior, double kappa, int* row_ptr, int* col_idx, double* m_vals,
                   double* a_vals, int* n_h, int* nnz);

/* st_wave_matrices -- the one-dimensional matrices of the wave equation's space-time system (paper Section 3
 * "The Wave Equation", Section 4 eq. 3terms; Section 5 Example 2's cubic B-splines), assembled on the host:
 * test space R (x) Z with Z the cubic B-splines of an open uniform knot vector on n_x intervals of (0, 1) without
 * the two that are nonzero at an end point (N_h = n_x + 1, Dirichlet), R the cubic B-splines on n_t intervals of
 * (0, T) without the two that are nonzero in value or slope at T (N_t = n_t + 1).  Outputs (any may be NULL),
 * dense column-major: Mh = (psi_i, psi_j), Ah = (psi_i', psi_j'), Qh = (psi_i'', psi_j'') (N_h x N_h);
 * Mt = (rho^k, rho^l), Dt[k][l] = ((rho^k)'', rho^l), Qt = ((rho^k)'', (rho^l)'') (N_t x N_t).  4-point
 * Gauss-Legendre on every knot interval (exact).  Host only.  ST_EINVAL for n_x < 4, n_t < 4 or T <= 0. */
int st_wave_matrices(int n_x, int n_t, double T, double* Mh, double* Ah, double* Qh, double* Mt, double* Dt,
                     double* Qt);

/* st_wave_solve -- the wave equation's space-time system, M_h U Q_t^T + A_h U (D_t + D_t^T) + Q_h U M_t = F1 F2^T
 * (Section 4 eq. 3terms; matrices of st_wave_matrices, unknown U N_h x N_t, U[i][k] the coefficient of the trial
 * function (rho^k)'' psi_i + rho^k A psi_i), by GMRES on vec(U) (X_0 = 0, no restart, classical Gram-Schmidt
 * twice) right-preconditioned by M_h W Q_t^T + Q_h W M_t = V, solved by diagonalising the pencils (Q_h, M_h)
 * and (Q_t, M_t) on the host ("GMRES+LYAP").  Stops when the residual estimate |g_{j+1}| / ||F||_F <= tol, or
 * after maxit steps (ST_ENOTCONV, the last iterate returned).  F1 (N_h x p, ld ldf1), F2 (N_t x p, ld ldf2) host
 * or device; U (N_h x N_t, ld ldu) host or device, written.  stats (may be NULL): iterations, relres (the
 * estimate), converged, ms_total, ms_phase[0] = host set-up (matrices and eigendecompositions).  stream: the
 * caller's stream (NULL: the legacy stream); device memory (about (maxit + 8) N_h N_t doubles) is taken and
 * released on it.  Synchronises.  Errors: ST_EINVAL, ST_ENOMEM, ST_EBREAKDOWN, ST_ECUDA. */
int st_wave_solve(int n_x, int n_t, double T, const double* F1, int ldf1, const double* F2, int ldf2, int p,
                  double tol, int maxit, double* U, int ldu, st_stats* stats, void* stream);

/* st_get_csr -- copy the assembled matrices to host arrays (sizes from
 * st_problem_info): row_ptr (n_h+1), col_idx (nnz), m_vals, a_vals (nnz).
 * Any pointer may be NULL.  Synchronises the stream. */
int st_get_csr(st_problem* p, int* row_ptr, int* col_idx, double* m_vals, double* a_vals);

/* st_apply -- Y = M U D_t^T + A U C_t^T (Section 4, the vec identity
 * (D (x) A) vec(X) = vec(A X D^T) applied to B = D_t (x) M + C_t (x) A).
 * Column l of Y is P u_l - N u_{l-1} with P = M + dt/2 A, N = M - dt/2 A,
 * u_0 = 0.  U and Y: device, n_h x n_t, dtype ST_F64 (double) or ST_F32
 * (float), ldu, ldy >= n_h; U and Y must not overlap.  Asynchronous. */
int st_apply(st_problem* p, int dtype, const void* U, int ldu, void* Y, int ldy);

/* st_rhs_manufactured -- load factors of the manufactured solution
 * u = sin(pi t) prod_d sin(pi x_d / L_d) with exact integrals (Section 3,
 * eq. par2): F1 = [g, g] (n_h x 2), F2 = [h_a, h_b] (n_t x 2) with
 * g_j = (prod_d sin(pi x_d/L_d), phi_j), h_a[l] = (pi cos(pi t), tau^l),
 * h_b[l] = (kappa sum_d (pi/L_d)^2 sin(pi t), tau^l).  Heat problems on boxes
 * only (ST_ENOTSUP otherwise).  Outputs: device arrays.  Asynchronous. */
int st_rhs_manufactured(st_problem* p, double* F1, int ldf1, double* F2, int ldf2);

/* st_shift_solve -- W = (A + s M)^{-1} M X for p columns (Section 4: the
 * resolvent (A_h - sigma M_h)^{-1} M_h with sigma = -s < 0).  Heat: fast
 * diagonalisation on the tensor grid; precision ST_FP64 computes the
 * transforms in FP64, ST_MIXED computes them in FP32 and refines once with an
 * FP64 residual.  Asynchronous.  Convection-diffusion: flexible GMRES
 * right-preconditioned by the fast-diagonalisation solve of eps K + s M (its
 * transforms in FP64, or FP32 under ST_MIXED), all columns advanced together,
 * stopped at a relative residual of 1e-12 per column; synchronises with the
 * host every few steps.  X, W: device double, n_h x p, ld >= n_h; may alias.
 * s > -lambda_min (of eps K for convection-diffusion).  Heat problems given
 * as user CSR matrices (dim == 0; M and A symmetric positive definite):
 * Jacobi-preconditioned conjugate gradients, all columns advanced together,
 * to a relative residual of 1e-12 per column, FP64 whatever the precision;
 * synchronises every few iterations.  ST_ENOTSUP for convection-diffusion
 * given by user matrices. */
int st_shift_solve(st_problem* p, double s, const double* X, int ldx, int ncols,
                   double* W, int ldw, int precision);

/* st_shift_solve_noalloc -- the FP64 shifted solve of st_shift_solve,
 * W = (A + s M)^{-1} M X, for callers that cannot allocate device memory
 * while they run: code recording its own stream capture, or a real-time
 * loop whose memory is fixed after start-up, where a cudaMalloc (which can
 * synchronise the device or fail) is not allowed.  st_shift_solve may grow a
 * workspace owned by the handle; this call allocates nothing (no cudaMalloc,
 * cudaFree or allocating library routine).  The paper has no counterpart.
 * Scratch: a file-scope device array of 4,194,304 doubles (32 MiB); calls
 * with n_h * ncols above that return ST_EINVAL (text in st_last_error).  The
 * first call on a device loads the library's device code there, which
 * reserves the array on that device until the process exits, and looks up
 * its device address: make that first call before any stream capture.  Every
 * later call allocates nothing.  The problem's device (current at st_setup)
 * must be the current device (else ST_EINVAL).  The call never times launch
 * variants (st_autotune): it uses the tuned or built-in choices as they are.
 * Every call shares the array (each call overwrites it completely before
 * reading it), so calls that overlap on the GPU, on any stream, race.  X and
 * W: device double, n_h x ncols, ld >= n_h, may alias (also W == X).  Work is
 * issued on the handle's stream; asynchronous.  ST_ENOTSUP without the
 * tensor-grid heat solver. */
int st_shift_solve_noalloc(st_problem* p, double s, const double* X, int ldx, int ncols, double* W, int ldw);

/* st_shift_solve_noalloc_max -- capacity of that scratch array in doubles. */
unsigned long st_shift_solve_noalloc_max(void);

/* st_autotune -- pick, by timing on this GPU, the launch variants of the
 * kernels behind the shifted solves of Section 4 for this problem's shapes
 * (the paper has no counterpart: its solves ran on CPUs).  Tuned: the tile
 * edge (16, 32 or 64) of the fast-diagonalisation mode products, and the
 * x-line tridiagonal solve of the convection-diffusion preconditioner (a warp
 * per row for rows of at most 256 points, or a thread per row loading 64 or
 * 16 steps at a time).  Runs st_shift_solve once at shift s (same domain) on
 * ncols (1..16) internal seeded columns in the given precision; the first
 * launch of each shape missing from the table runs every valid variant on
 * its own operands, four interleaved rounds of three launches timed with
 * CUDA events on the handle's stream (the first round discarded), and keeps
 * the fastest, unless it beats the built-in choice by 3% or less.  The
 * choices are kept, process-wide, for every later launch of the same kernel
 * shape on any handle and thread (a shape: precision, grid direction and
 * length, columns per launch); RKSM solves with p columns after rank
 * compression use the shapes of ncols = p.  All variants compute the same
 * quantity; they may differ in rounding.  Allocates and frees 3 n_h ncols
 * doubles of device memory (besides the handle workspace st_shift_solve
 * may grow); synchronises; call it with the GPU otherwise
 * idle, outside stream capture (a captured stream is never tuned).  *tuned
 * (may be NULL): shapes added.  Errors: ST_EINVAL, ST_ENOTSUP (as
 * st_shift_solve), ST_ENOMEM, ST_ECUDA. */
int st_autotune(st_problem* p, double s, int ncols, int precision, int* tuned);

/* st_autotune_reset -- forget every tuned choice; later launches take the
 * built-in choices again.  Not to be called while solves run. */
int st_autotune_reset(void);

/* st_autotune_count -- number of kernel shapes with a tuned choice. */
int st_autotune_count(void);

/* st_autotune_save -- write every tuned choice to a text file at path
 * ("st-autotune 1", "device <device_tag>", then one sorted line per shape),
 * so that a later process on the same kind of GPU can skip the timing.
 * device_tag: caller-chosen identity of the GPU (name, SM count, compute
 * capability...), non-empty, at most 199 characters, no line breaks.  Host
 * only; no CUDA call.  Errors: ST_EINVAL (NULL or bad tag, file not writable;
 * text in st_last_error). */
int st_autotune_save(const char* path, const char* device_tag);

/* st_autotune_load -- add the choices of a file written by st_autotune_save
 * to the table (replacing those of the same shapes) when its device tag
 * equals device_tag; otherwise load nothing and return ST_OK with
 * *loaded = 0.  Entries of unknown kernel families, element sizes or variant
 * indices are skipped; every loaded choice is still checked against the
 * shape of each launch before use (a variant that cannot run the shape is
 * replaced by the built-in choice).  *loaded (may be NULL): entries added.
 * Host only; no CUDA call.  Errors: ST_EINVAL (NULL or bad tag, unreadable
 * file, bad header, a malformed line: then nothing is loaded). */
int st_autotune_load(const char* path, const char* device_tag, int* loaded);

/* st_solve -- rational Krylov Galerkin projection (RKSM) for (1) (Section 4):
 * compress F to a full-column-rank F1 (QR + SVD), grow an orthonormal basis
 * V of the rational Krylov space of the pencil (A, M) started from M^{-1} F1
 * with adaptive shifts, impose V^T R = 0, solve the projected equation
 * (V^T M V) Y D_t^T + (V^T A V) Y C_t^T = (V^T F1) F2^T by the time
 * recurrence of the triangular time pencil, and stop when the relative
 * residual (Frobenius, FP64, evaluated from low-rank factors) is <= tol.
 * F1: n_h x p (ld ldf1), F2: n_t x p (ld ldf2), double, host OR device.
 * 1 <= p <= 16.  Output in *sol (V, Y owned by the handle; U_dense filled if
 * given).  stats may be NULL.  Synchronises.  Returns ST_OK, ST_ENOTCONV
 * (best iterate returned), ST_EBREAKDOWN, ST_ENOTSUP (convection-diffusion
 * given as user matrices), ST_EINVAL
 * (also for a NaN or Inf in F1 or F2, or an F1 whose Gram matrix overflows).
 * Heat (ST_HEAT): the shifted solves are exact fast-diagonalisation
 * transforms.  Convection-diffusion (ST_CONVDIFF, A nonsymmetric): each
 * shifted solve is flexible GMRES (all columns advanced together)
 * right-preconditioned by the x-line solve of eps K + beta_x Gx (x) M_rest
 * + s M when |beta_x| is the largest component (else by the
 * fast-diagonalisation solve of eps K + s M), to 1e-3 tol relative (at least
 * 1e-13); the projected matrices are not symmetrised and the projected time
 * recurrence uses LU.  ST_MIXED: FP32 transforms (refined to FP64 accuracy,
 * or inside FGMRES as the preconditioner), basis products in double-float
 * arithmetic on the FP32 pipes (about 48 significant bits), and on
 * convection-diffusion grids of at least 2^15 points FGMRES cycles in FP32
 * refined on the FP64 residual.  Heat given as user CSR matrices (dim == 0,
 * e.g. P1 on a simplex mesh from st_p1_mesh_csr; M and A symmetric positive
 * definite): the shifted solves and the start block's M^{-1} F1 are
 * Jacobi-preconditioned conjugate gradients (to 1e-12 / 1e-13 relative per
 * column), the pencil interval of the adaptive shifts is estimated at the
 * first solve (power and inverse iteration), and the solve runs in FP64
 * whatever the requested precision. */
int st_solve(st_problem* p, const double* F1, int ldf1, const double* F2, int ldf2, int ncols,
             st_solution* sol, st_stats* stats);

/* st_solve_lrfgmres -- LR-FGMRES+RKSM, the comparison solver of Section 5,
 * Example 1 (Table 1): flexible GMRES (no restart, X_0 = 0) on (1) with every
 * Krylov vector held as a low-rank pair P Q^T (P on the device, Q on the host),
 * inner product trace(X^T Y), every sum and operator product truncated (thin
 * QRs of both factors and an SVD of the core; singular values at or below
 * trunc times the largest dropped), right-preconditioned by st_solve's RKSM
 * stopped after precond_iters shifted solves on the vector's factors (blocks
 * of at most 16 columns, their results summed).  Stops when the least-squares
 * residual estimate is <= the problem's tol, or after maxit steps.  Heat
 * problems, on box grids or as user CSR matrices (ST_ENOTSUP otherwise).  F1, F2 as st_solve (host or
 * device, 1 <= ncols).  Output in *sol: V = P (n_h x k), Y = Q^T (k x n_t),
 * owned by the handle (valid until its next solve or st_destroy), U_dense
 * filled if given.  stats (may be NULL): iterations = GMRES steps, basis_cols
 * = k, mu_mem = stored columns of every factor pair V_1..V_{m+1}, Z_1..Z_m
 * (Table 1's memory count), relres = the final least-squares estimate,
 * inner_iterations = RKSM iterations of all preconditioner calls.  Returns
 * ST_OK, ST_ENOTCONV (best iterate returned), ST_EINVAL, ST_ENOTSUP, ST_ENOMEM,
 * ST_ECUDA.  Synchronises. */
int st_solve_lrfgmres(st_problem* p, const double* F1, int ldf1, const double* F2, int ldf2, int ncols,
                      int maxit, int precond_iters, double trunc, st_solution* sol, st_stats* stats);

/* Statistics of one st_solve_batch call. */
typedef struct st_batch_stats {
    int instances;          /* problems in the call */
    int grouped;            /* problems solved on the grouped lock-step path */
    int rounds;             /* lock-step iterations (the most iterations of a grouped problem) */
    int grouped_launches;   /* grouped kernel launches issued */
    int groups;             /* lock-step groups run concurrently, each on its own stream */
    double ms_total;        /* wall time of the call (host clock) */
    double ms_phase[8];     /* wall time: 0 rank compression, 1 shifted solves and block Gram-Schmidt
                               (and the start blocks), 2 block QR decisions on the host (with the
                               per-problem fallbacks), 3 block QR on the device and products of the
                               new blocks, 4 projected solves, 5 residual checks, 6 output, 7 shifts */
} st_batch_stats;

/* st_solve_batch -- st_solve for `count` independent problems at once
 * (Section 4's method for each; the paper solves one problem at a time).
 * The problems advance in lock step, one rational Krylov iteration per
 * round: every device step of a round (the shifted solves, block
 * Gram-Schmidt, block QR and products of the new blocks, the residual
 * checks) is ONE launch of a grouped kernel over all problems still
 * iterating, and each round synchronises with the host once per phase for
 * the whole group; the small host problems of a round (rank decisions,
 * shifts, projected solves) run on a pool of host threads.  The problems
 * run as `groups` such lock-step groups (<= 0: about 8 problems a group, at
 * most 32 groups; problems dealt by decreasing size) on streams and host threads of their
 * own, so one group's host work overlaps the others' device work; `stream`
 * waits for all of them.  Each problem
 * takes exactly the steps and decisions st_solve takes on it, and the
 * grouped kernels run the per-problem kernels' tiles, so problems[i]'s
 * result does not depend on the other problems of the call.
 * problems: distinct handles of the current device.  The grouped path
 * covers box heat problems of dimension 2 or 3 with at least 3 points a
 * side; the others (dimension 1, user matrices, convection-diffusion) are
 * solved one after another by st_solve's driver on the same stream.
 * F1[i] (n_h x ncols[i], ld ldf1[i]) and F2[i] (n_t x ncols[i], ld ldf2[i]):
 * host or device, 1 <= ncols[i] <= 16.  Outputs per problem (arrays of
 * count entries): sols (may be NULL; as st_solve, V and Y owned by the
 * handle, U_dense filled if given), stats (may be NULL), status (required:
 * st_solve's return value for that problem).  Work runs on `stream` (NULL:
 * default stream); each handle's own stream is restored on return.  Returns
 * ST_OK when the call ran (see status[]), ST_EINVAL for bad arguments, or
 * ST_ENOMEM / ST_ECUDA when a failure stopped the whole call.  bstats may be
 * NULL.  Synchronises. */
int st_solve_batch(int count, st_problem* const* problems, const double* const* F1, const int* ldf1,
                   const double* const* F2, const int* ldf2, const int* ncols, st_solution* sols,
                   st_stats* stats, int* status, void* stream, int groups, st_batch_stats* bstats);

/* st_residual -- relres = ||F - M U D_t^T - A U C_t^T||_F / ||F1 F2^T||_F in
 * FP64 for a dense U (device double, ld >= n_h) (Section 5 stopping
 * quantity).  F1, F2 host or device.  relres: host.  Synchronises. */
int st_residual(st_problem* p, const double* U, int ldu, const double* F1, int ldf1,
                const double* F2, int ldf2, int ncols, double* relres);

/* st_residual_lowrank -- the same for U = V Y (V device n_h x k, Y device
 * k x n_t), from the factors [F1, M V, A V] and [F2, -D_t Y^T, -C_t Y^T]
 * without forming U or the Kronecker product (Section 4).  Synchronises. */
int st_residual_lowrank(st_problem* p, const double* V, int ldv, const double* Y, int ldy, int k,
                        const double* F1, int ldf1, const double* F2, int ldf2, int ncols,
                        double* relres);

/* st_timestep_cn -- Crank-Nicolson time stepping on the same load matrix
 * (Section 3: the scheme equals CN; Section 5 comparison):
 * (M + dt/2 A) u_l = F[:, l] + (M - dt/2 A) u_{l-1}, l = 1..N_t, one
 * fast-diagonalisation spatial solve per step, FP64.  U: device double,
 * n_h x n_t, ld >= n_h, caller-owned (the full N_h * N_t storage of
 * Section 5).  F1, F2 host or device.  Asynchronous after the inputs are
 * staged. */
int st_timestep_cn(st_problem* p, const double* F1, int ldf1, const double* F2, int ldf2, int ncols,
                   double* U, int ldu);

/* st_set_coefficients -- change the operator and its coefficients of a box
 * problem in place (same grid, time grid and controls): op ST_HEAT with
 * kappa (> 0; 0 means 1.0), or ST_CONVDIFF with eps > 0 and beta[3]
 * (beta may be NULL for zero velocity).  Re-runs the device assembly of
 * M, A, P = M + dt/2 A, N = M - dt/2 A (Section 3) on the handle's stream;
 * the grid-only fast-diagonalisation tables are kept.  Asynchronous.
 * ST_ENOTSUP for user CSR problems (dim == 0). */
int st_set_coefficients(st_problem* p, int op, double kappa, double eps, const double* beta);

/* st_error_string -- static text for a status code. */
const char* st_error_string(int status);

/* st_last_error -- text of the last failure recorded on the calling thread:
 * a CUDA error (call, file, line) or a message of a call that returned an
 * error status (sizes, files, solver state).  Per thread; never cleared. */
const char* st_last_error(void);

/* ---- many independent solves on one GPU: batched and served workloads ----
 * The paper solves one problem at a time; the executor runs many solves of
 * the Section 4 method at once.  `slots` worker threads each own a CUDA
 * stream; problem handles live in a pool shared by the slots and keyed by
 * geometry (operators and fast-diagonalisation tables stay on the device
 * between requests; a new coefficient re-runs the assembly only; at most
 * 4 x slots handles are kept, and none whose operators exceed 512 MB).
 * Device memory of handles comes from the stream-ordered allocator, so one
 * slot's allocations never synchronise the others.  Requests are admitted in arrival
 * order as long as their estimated device footprint (st_request_bytes) fits
 * the free part of the HBM budget; a request that does not fit is passed
 * over until memory frees up, and one larger than the whole budget runs when
 * nothing else does.  A slot takes the next admissible request as soon as its
 * previous one finishes (continuous batching): work of requests that arrived
 * at different times overlaps on the device.  A solve reads and writes only
 * its own handle, so its result is the same alone and in a mix. */
typedef struct st_executor st_executor;

typedef struct st_request {
    st_desc desc;            /* box problem (dim 1..3) and solver controls; desc.stream is ignored */
    const double* F1;        /* n_h x p load factor, host or device; valid until the result is returned */
    int ldf1;
    const double* F2;        /* n_t x p load factor, host or device */
    int ldf2;
    int p;                   /* 1 <= p <= 16 */
    double* U_out;           /* optional n_h x n_t buffer (host or device) receiving U; NULL: none */
    int ldu;                 /* leading dimension of U_out (>= n_h) */
    unsigned long long tag;  /* the caller's identifier, returned with the result */
    int method;              /* ST_METHOD_RKSM (st_solve) or ST_METHOD_CN (st_timestep_cn; U is
                                written to U_out, or to a buffer of the slot when U_out is NULL) */
} st_request;

#define ST_METHOD_RKSM 0
#define ST_METHOD_CN   1

typedef struct st_result {
    unsigned long long tag;  /* st_request.tag */
    int status;              /* status of the solve (ST_OK, ST_ENOTCONV, ...) or of its set-up */
    int slot;                /* worker slot that ran the request */
    int k;                   /* basis columns of the solution */
    double bytes_reserved;   /* admission estimate held while the request ran */
    double t_submit, t_start, t_end;   /* seconds on the executor clock (st_executor_now) */
    st_stats stats;          /* statistics of the solve */
    char message[160];       /* on failure, the worker's st_last_error text ("" on success) */
} st_result;

/* st_request_bytes -- admission estimate of a request's device footprint
 * in bytes: the CSR operators (P, N, M, A in FP64 and FP32), the
 * fast-diagonalisation tables, a basis of k = min(max_basis + 16,
 * p (min(maxit, m) + 1)) columns with m = 80 for heat and 200 for
 * convection-diffusion, stored as V and M V (plus the float-pair copy of V
 * under ST_MIXED), 12 p N_h-sized work columns and Y (k x N_t); for
 * convection-diffusion also the flexible GMRES blocks (84 N_h doubles per
 * column, at most 16 columns and 4 GB).  Host only.  0 for invalid
 * descriptors (NULL, dim outside 1..3, p < 1). */
double st_request_bytes(const st_desc* d, int p);

/* st_executor_create -- start `slots` (1..256) worker threads on the current
 * device with an HBM budget in bytes (<= 0: 80% of the free memory). */
int st_executor_create(int slots, double hbm_budget_bytes, st_executor** out);

/* A request that runs out of device memory (ST_ENOMEM) while other requests
 * run is queued again, at most twice, with an estimate of the whole budget,
 * so that it runs alone; its result is reported only then.
 *
 * st_executor_submit -- queue a request (copied; the F1, F2 and U_out
 * buffers it points to must stay valid until its result is returned).
 * ST_EINVAL for bad sizes or after st_executor_destroy began. */
int st_executor_submit(st_executor* ex, const st_request* req);

/* st_executor_wait -- move up to `max` finished results into out[] (out may be
 * NULL to discard them), waiting up to timeout_s seconds for the first one
 * (<= 0: do not wait).  *count receives the number moved. */
int st_executor_wait(st_executor* ex, st_result* out, int max, int* count, double timeout_s);

/* st_executor_set_policy -- order in which waiting requests are admitted.
 * ST_SCHED_FIFO (the default): arrival order, skipping requests that do not
 * fit the free HBM.  ST_SCHED_HRRN: the request with the highest response
 * ratio (wait + estimated service) / estimated service, admitted when it
 * fits the free HBM (until then nothing else is admitted), so short requests
 * overtake long ones while no request waits for ever (its ratio grows with
 * its wait).  The service estimate of a request
 * is 2 ms plus n_h * n_t times a rate per class (operator, method,
 * dimension), learned from the finished requests of that class (prior rate
 * 3e-9 s for heat RKSM, 2e-8 s for convection-diffusion RKSM, 1e-9 s for
 * CN).  Takes effect from the next admission; ST_EINVAL for an unknown
 * policy. */
#define ST_SCHED_FIFO 0
#define ST_SCHED_HRRN 1
int st_executor_set_policy(st_executor* ex, int policy);

/* st_executor_pending -- requests still queued and running (host outputs, may be NULL). */
int st_executor_pending(st_executor* ex, int* queued, int* running);

/* st_executor_now -- seconds since the executor was created (its clock). */
double st_executor_now(st_executor* ex);

/* st_executor_destroy -- drop queued requests, let running ones finish, join
 * the workers and free their handles.  NULL is accepted. */
int st_executor_destroy(st_executor* ex);

/* ---- launch accounting and kernel timing (tracing; no counterpart in the paper) ---- */

/* Per-kernel totals of a profiling region. */
typedef struct st_kernel_time {
    char name[24];        /* kernel tag, e.g. "apply", "fd_gemm", "ts_tn" */
    int launches;         /* launches recorded in the region */
    double ms;            /* summed durations between the event pair around each launch */
    double bytes;         /* summed algorithmic bytes (each input read once, each output written once) */
    double flops;         /* summed algorithmic floating-point operations */
} st_kernel_time;

/* st_launch_count -- number of kernels this library has launched in the
 * process (graph replays count every kernel node). */
unsigned long long st_launch_count(void);

/* st_profile_begin -- start recording an event pair on the launching stream
 * around every tagged kernel launch (not inside graph capture). */
int st_profile_begin(void);

/* st_profile_end -- stop recording, wait for the events and aggregate per tag
 * into out[0 .. min(*count, max)).  *count receives the number of tags. */
int st_profile_end(st_kernel_time* out, int max, int* count);

#ifdef __cplusplus
}
#endif

#endif /* ST_H_ */

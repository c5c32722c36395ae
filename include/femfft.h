/*
 * femfft -- fast direct solver for the tensor-product nth-order FEM
 * discretisation of a generalised Poisson equation on a rectangular
 * parallelepiped with homogeneous Dirichlet conditions, on one NVIDIA GB300
 * (sm_103a).
 *
 * Method: A. Zlotnik and I. Zlotnik, "On fast Fourier solvers for the tensor
 * product high-order FEM for a generalized Poisson equation" (arXiv:1701.03967).
 *   Problem (Section 4, the N-dimensional boundary value problem and its FEM
 *   operator form, with per-axis coefficients a_i and zeroth-order term c):
 *       -sum_i a_i d^2u/dx_i^2 + c u = f  on (0,X_1) x ... x (0,X_N),  u = 0 on the boundary,
 *       L = sum_i a_i (4/h_i^2) calA_i (x) prod_{j!=i} calC_j + c prod_j calC_j,   L u = b,
 *   where calA_i, calC_i are the h-free 1D stiffness and mass operators of
 *   Section 2 (K_i uniform elements of order n on [0, X_i], h_i = X_i / K_i)
 *   and b is the "FEM average" right-hand side f^h.
 *   Solve (Section 4, algorithm (a)): direct FC_n-transform along every axis
 *   (Section 3, Theorem 2, item 2), division by sum_i a_i 4 h_i^-2 lambda_i + c,
 *   inverse F_n-transform along every axis (Theorem 2, item 1).  Algorithm (b)
 *   of Section 4 (transforms along x_2..x_N, band solves along x_1) is
 *   selected per plan by fem_fft_set_algorithm.
 *
 * Data layout (all entry points): a field is a C-order array
 *   [nrhs][M_1][M_2]...[M_N] of float64, M_i = n K_i - 1, axis N contiguous.
 * Along an axis, index m (0-based) is the FEM node at x = (m+1) h / n: element e
 * (0-based) owns indices n e .. n e + n - 2 (its interior nodes, l = 1..n-1)
 * and n e + n - 1 (its right vertex); the two boundary vertices are not stored.
 * Spectral arrays (fem_fft_forward / fem_fft_inverse) have the same shape;
 * along an axis, coefficient sigma (0-based) is mode (k, l) with
 * sigma + 1 = n k + slot: the n-1 bubble modes k = 0 (slot l = 1..n-1) first,
 * then for k = 1..K-1 the n modes slot = l-1 = 0..n-1 in ascending eigenvalue
 * order, with the eigenvectors normalised as in Section 3, Theorem 1 (node
 * values sin(pi k j / K); bubble interiors (-P)^{j-1} e^(l), C~e.e = 1).
 *
 * Pointers: every array argument named d_* is a device pointer owned by the
 * caller (for example a contiguous torch tensor's data_ptr()); h_* arguments
 * are host pointers.  The library never frees caller memory.  A plan owns its
 * device tables and workspace.  Streams are passed as cudaStream_t cast to
 * void* (NULL = legacy default stream).  All calls are asynchronous on that
 * stream unless stated otherwise; a plan's workspace is shared by all calls
 * on it, so calls on one plan must be issued on one stream (or serialised).
 *
 * nrhs = 0 is a no-op (array pointers may then be NULL).
 *
 * Errors: every entry point returns 0 (FEM_FFT_OK) or a negative status.  No
 * exception crosses the ABI.  An asynchronous device error from an earlier
 * call surfaces as FEM_FFT_ERR_CUDA at a later synchronising call.
 */
#ifndef FEMFFT_H_
#define FEMFFT_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fem_fft_plan_s* fem_fft_plan;
typedef struct fem_fft_batch_s* fem_fft_batch;

enum fem_fft_status {
  FEM_FFT_OK = 0,
  FEM_FFT_ERR_ARG = -1,           /* invalid argument or unsupported size */
  FEM_FFT_ERR_ASSUMPTION_A = -2,  /* a 1D eigenproblem failed (Section 3, assumption (A)) */
  FEM_FFT_ERR_OOM = -3,           /* device allocation failed */
  FEM_FFT_ERR_CUDA = -4,          /* CUDA runtime error (message: fem_fft_last_error) */
  FEM_FFT_ERR_TIMEOUT = -5,       /* a bounded device wait expired */
  FEM_FFT_ERR_NOT_CONVERGED = -6, /* refinement stopped above the requested tolerance */
  FEM_FFT_ERR_NONFINITE = -7      /* NaN or Inf in a right-hand side or a residual */
};

enum fem_fft_precision {
  FEM_FFT_FP64 = 0,  /* transforms, divide and everything else in float64 */
  FEM_FFT_MIXED = 1  /* float32 transforms + float64 matrix-free residual refinement */
};

/*
 * fem_fft_plan_create -- Section 4 (problem statement) and Section 3
 * (1D eigenpairs, Theorem 1).  Precomputes, on the host in double-double
 * arithmetic, the reference matrices A, C (Section 2), the bubble eigenpairs
 * of A~ e = lambda C~ e, for every axis and k = 1..K_i-1 the n eigenpairs
 * lambda_k^(l), p_k^(l) and norms ||s_k^(l)||_C^2, and the transform tables;
 * uploads them and allocates the workspace for up to max_nrhs right-hand
 * sides per call (larger nrhs are processed in groups).  Synchronous.
 *   N         number of axes, 1..3
 *   n         element order, 1..9, on every axis (per-axis orders:
 *             fem_fft_plan_create_orders)
 *   h_K[N]    elements per axis; each K_i >= 2 of the form 2^p 3^q with p >= 1
 *   h_X[N]    axis lengths X_i > 0
 *   h_a[N]    coefficients a_i > 0
 *   c         zeroth-order coefficient, c > -pi^2 sum_i a_i / X_i^2 (so L is
 *             positive definite, Section 4)
 *   precision FEM_FFT_FP64 or FEM_FFT_MIXED
 *   max_nrhs  >= 1
 *   stream    stream for the table uploads
 * Returns FEM_FFT_ERR_ARG for out-of-range arguments, FEM_FFT_ERR_OOM,
 * FEM_FFT_ERR_CUDA, or FEM_FFT_ERR_ASSUMPTION_A.  *out is NULL on failure.
 */
int fem_fft_plan_create(fem_fft_plan* out, int N, int n, const int64_t* h_K, const double* h_X,
                        const double* h_a, double c, int precision, int64_t max_nrhs, void* stream);

/*
 * fem_fft_plan_create_orders -- as fem_fft_plan_create with an element order
 * per axis, h_n[N] (each 1..9): Section 4 states the N-D problem with the
 * 1D spaces S_{K_i}^{(n_i)} of their own orders.  Axis i then has
 * M_i = n_i K_i - 1 unknowns and its own eigenpairs, transforms and element
 * matrices; the spectral denominators sum the axes' eigenvalues as before.
 * A batch (fem_fft_batch_create) holding such a plan runs in stream mode only.
 */
int fem_fft_plan_create_orders(fem_fft_plan* out, int N, const int* h_n, const int64_t* h_K, const double* h_X,
                               const double* h_a, double c, int precision, int64_t max_nrhs, void* stream);

/*
 * fem_fft_plan_set_coefficients -- replace a_i and c of an existing plan
 * (Section 4 operator).  The 1D eigenpairs do not depend on them, so only the
 * denominator tables a_i 4 h_i^-2 lambda are recomputed and re-uploaded;
 * this is what differentiation with respect to a_i, c iterates on.
 * Same validity rules as fem_fft_plan_create.  Synchronous on stream.
 */
int fem_fft_plan_set_coefficients(fem_fft_plan plan, const double* h_a, double c, void* stream);

/* Frees the plan's device tables and workspace (synchronises its stream). */
int fem_fft_plan_destroy(fem_fft_plan plan);

/*
 * fem_fft_solve -- u = L^{-1} b, Section 4, algorithm (a).
 *   d_b, d_u  [nrhs][M_1..M_N] float64; d_b == d_u (in place) is allowed in
 *             FP64 precision, and in MIXED precision only with refinement
 *             disabled (max_iter = 0), else FEM_FFT_ERR_ARG.
 * FP64: 2N-1 pencil passes in float64.  MIXED: the passes in float32, then
 * max_iter (default 2) refinement steps r = b - L u (float64, matrix-free),
 * u += L^{-1} r (float32 passes), stopping early when the relative residual
 * ||r||_2 / ||b||_2 <= rtol (default 0: always take max_iter steps).  The
 * residual norms are read back at the end of each step only when rtol > 0;
 * then, when the steps run out, the final iterate's residual is evaluated as
 * well and a value above rtol returns FEM_FFT_ERR_NOT_CONVERGED (u holds the
 * last iterate).  Non-finite right-hand sides: the first pass flags any NaN
 * or Inf it reads in b, without synchronising; fem_fft_last_info reports it
 * (FEM_FFT_ERR_NONFINITE), and with rtol > 0 the solve itself returns it.
 */
int fem_fft_solve(fem_fft_plan plan, const double* d_b, double* d_u, int64_t nrhs, void* stream);

/* fem_fft_apply -- d_b = L d_u in float64, matrix-free (Section 4, operator
 * form; element blocks of Section 2).  d_u != d_b. */
int fem_fft_apply(fem_fft_plan plan, const double* d_u, double* d_b, int64_t nrhs, void* stream);

/*
 * fem_fft_apply_mass -- d_b = (calC_1 (x) ... (x) calC_N) d_u in float64,
 * matrix-free: the mass operator of the N-D space (the global mass matrices
 * of Section 2 in tensor products as in Section 4; the c-term of L with c = 1).
 * With it, one implicit Euler step of calC u' + L u = b,
 * (calC + tau L) u_new = calC u + tau b, is a solve with a plan whose
 * coefficients are (tau a_i, 1 + tau c): calC + tau L has the form of L.
 * Layout and errors as fem_fft_apply; d_u != d_b.  Asynchronous on stream.
 */
int fem_fft_apply_mass(fem_fft_plan plan, const double* d_u, double* d_b, int64_t nrhs, void* stream);

/*
 * fem_fft_dirichlet_rhs -- non-zero Dirichlet data (Section 4, u = g on the
 * boundary instead of 0): d_b -= L_full G on the interior nodes, where G is
 * the FEM function with g's values at the boundary nodes and 0 inside and
 * L_full the operator of Section 4 on the space that keeps the boundary
 * nodes.  Then fem_fft_solve of the corrected d_b gives the interior values
 * of the solution (u - G has zero boundary values).
 *   d_g  nrhs fields extended by the boundary node at each end of every axis:
 *        [nrhs][M_1 + 2]...[M_N + 2] float64, C order, fine index m of axis i
 *        (the node at x_i = m h_i / n, m = 0 .. n K_i) at position m; only the
 *        boundary entries are read (the interior is taken as 0)
 *   d_b  [nrhs][M_1]...[M_N] float64, corrected in place (typically f^h)
 * Float64 operator products on the extended fields; temporaries of 2, 4 or
 * 5 extended fields (N = 1, 2, 3) come from the stream-ordered allocator
 * (cudaMallocAsync) and are released on the stream.  FEM_FFT_ERR_OOM if they
 * cannot be had.  Asynchronous on stream.  A MIXED solve of the corrected
 * right-hand side (which carries the boundary layer of the data) can need a
 * third refinement step (fem_fft_set_refinement): on the 2D n = 9 K = 1024
 * problem two steps left 1.7e-10, three 3.1e-13.
 */
int fem_fft_dirichlet_rhs(fem_fft_plan plan, const double* d_g, double* d_b, int64_t nrhs, void* stream);

/*
 * fem_fft_set_algorithm -- the solver of fem_fft_solve (N >= 2):
 * FEM_FFT_ALGO_A (default) is algorithm (a) of Section 4 (FC_n / F_n
 * transforms along every axis and the spectral division); FEM_FFT_ALGO_B is
 * algorithm (b): the transforms along x_2..x_N only and, for every position
 * of those axes, the 1D problem [a_1 4 h_1^-2 calA_1 + (sum_{i>=2} a_i
 * 4 h_i^-2 lambda_i + c) calC_1] v = f~ along x_1, a symmetric positive
 * definite band system solved by static condensation of the element
 * interiors and a tridiagonal vertex solve.  Both give the solution of
 * L u = b.  Setting B computes its tables (one row of n + 2 values per
 * position of x_2..x_N) and a scratch of max_nrhs * (K_1 - 1) * M_2..M_N
 * values; synchronises stream.  FEM_FFT_ERR_ARG for N = 1.  A batch
 * (fem_fft_batch_create) runs each plan's algorithm as set when the batch is
 * created.
 */
enum { FEM_FFT_ALGO_A = 0, FEM_FFT_ALGO_B = 1 };
int fem_fft_set_algorithm(fem_fft_plan plan, int algo, void* stream);

/*
 * fem_fft_plan_tune -- time the plan's pencil passes (the launches of
 * fem_fft_solve, on the plan's own zeroed workspace) for every admissible
 * tile shape (pencils per CTA, powers of two) and FFT values per thread
 * (4, 8 or 6, 12), and keep the fastest per pass for later solves.  No paper
 * counterpart (a launch-configuration tuner).  Synchronises stream; about a
 * second for large plans.  Results are exact-arithmetic neutral: every
 * shape computes the same transforms.
 */
int fem_fft_plan_tune(fem_fft_plan plan, void* stream);

/*
 * fem_fft_solve_host -- u = L^{-1} b for right-hand sides in HOST memory
 * (the solve of fem_fft_solve, Section 4), with the copies pipelined inside
 * the library: two device slots of max_nrhs fields (allocated at the first
 * call, owned by the plan) alternate between successive calls (and groups of
 * max_nrhs right-hand sides), and the upload of one and the download of the
 * one before run on the plan's own copy streams under the solve of the
 * current one.  No paper counterpart (a serving path).
 *   h_b  [nrhs][M..] float64 host memory, read by the upload; it must hold
 *        the data when the call is made and stay unchanged until the upload
 *        has run (use pinned memory for asynchronous, overlapped copies)
 *   h_u  [nrhs][M..] float64 host memory, written by the download
 *   stream  work on it before the call precedes the uploads; h_u is complete
 *        once the stream has passed fem_fft_host_wait(plan, stream)
 * Asynchronous.  Other calls on the plan must not run between a host solve
 * and the wait that completes it (they share the plan's workspace).
 * fem_fft_host_wait -- make `stream` wait for every download issued so far.
 */
int fem_fft_solve_host(fem_fft_plan plan, const double* h_b, double* h_u, int64_t nrhs, void* stream);
int fem_fft_host_wait(fem_fft_plan plan, void* stream);

/* Refinement controls of the MIXED precision (ignored in FP64). */
int fem_fft_set_refinement(fem_fft_plan plan, double rtol, int max_iter);

/*
 * fem_fft_set_residual_precision -- arithmetic of the refinement residual
 * r = b - L u of a MIXED plan: FEM_FFT_RESIDUAL_DF64 (default) evaluates it in
 * double-float arithmetic (pairs of floats, about 48 significant bits, on the
 * float pipes: no float64 instruction), FEM_FFT_RESIDUAL_F64 in float64.  The
 * refined solution's accuracy floor is ~1e-12 relative with DF64 and ~1e-13
 * with F64 (2D, n = 9, K = 1024), both far below the 1e-10 target.
 * fem_fft_apply is always float64.  Returns FEM_FFT_ERR_ARG for another mode.
 */
enum { FEM_FFT_RESIDUAL_F64 = 0, FEM_FFT_RESIDUAL_DF64 = 1 };
int fem_fft_set_residual_precision(fem_fft_plan plan, int mode);

/* Iterations and relative residual ||b - L u|| / ||b|| of the last MIXED
 * solve whose residual was evaluated (-1 if unknown).  Waits for the last
 * solve on its stream and returns its status: FEM_FFT_ERR_NONFINITE if its
 * right-hand side held NaN or Inf, FEM_FFT_ERR_NOT_CONVERGED if rtol > 0 was
 * missed, else FEM_FFT_OK (any precision). */
int fem_fft_last_info(fem_fft_plan plan, int* iters, double* rel_residual);

/*
 * fem_fft_forward -- direct FC_n-transform along every axis (Section 3,
 * Theorem 2, item 2; Section 4, the multiple expansion of f^h):
 * d_y (field) -> d_c (spectral coefficients, layout above), float64 path.
 * fem_fft_inverse -- inverse F_n-transform along every axis (Theorem 2,
 * item 1): d_c (spectral) -> d_w (field).  d_in may equal d_out.
 */
int fem_fft_forward(fem_fft_plan plan, const double* d_y, double* d_c, int64_t nrhs, void* stream);
int fem_fft_inverse(fem_fft_plan plan, const double* d_c, double* d_w, int64_t nrhs, void* stream);

/*
 * fem_fft_forward_fn -- direct F_n-transform along every axis (Section 3,
 * Theorem 2, item 3): d_w (field) -> d_c, the coefficients w_kl of the
 * expansion of w in the eigenvectors s_k^(l), w_kl = (calC w, s_k^(l)) /
 * ||s_k^(l)||_C^2 (calC the N-D mass operator), in the spectral layout above;
 * the inverse is fem_fft_inverse.  The mass product is folded into the
 * forward maps as in the theorem's second formula (node sums weighted by
 * 2 [c_0 + c.p + theta_k (c_n + c.p^)], interior sums by q = C~ p + c; bubble
 * maps by C~ e), so the transform takes the passes of fem_fft_forward and no
 * separate mass product.  Float64 path; d_w may equal d_c.
 */
int fem_fft_forward_fn(fem_fft_plan plan, const double* d_w, double* d_c, int64_t nrhs, void* stream);

/*
 * fem_fft_heat_step -- one implicit Euler step of calC u' + L u = b
 * (Section 4 operator; the heat-equation use of the solver):
 * (calC + tau L) u_new = calC u + tau b.  The plan must represent
 * calC + tau L, i.e. be created (or set with fem_fft_plan_set_coefficients)
 * with coefficients (tau a_i, 1 + tau c); its solve then divides by
 * 1 + tau (sum_i a_i 4 h_i^-2 lambda_i + c).  The library forms the
 * right-hand side calC u + tau b (float64 mass product and axpy) and solves.
 *   tau            > 0, finite
 *   d_u, d_b       [nrhs][M..] float64 (read)
 *   d_u_new        [nrhs][M..] float64 (written); distinct from d_u and d_b
 * FP64 plans and MIXED plans without refinement form the right-hand side in
 * d_u_new; other MIXED plans in a stream-ordered temporary (cudaMallocAsync,
 * released on the stream; FEM_FFT_ERR_OOM if it cannot be had).  Asynchronous.
 */
int fem_fft_heat_step(fem_fft_plan plan, double tau, const double* d_u, const double* d_b, double* d_u_new,
                      int64_t nrhs, void* stream);

/*
 * fem_fft_grad_coeffs -- derivatives of a scalar loss through u = L^{-1} f
 * with respect to the coefficients (derived from Section 4: dL/da_i =
 * 4 h_i^-2 calA_i (x) prod_{j!=i} calC_j, dL/dc = prod_j calC_j, so
 * dloss/da_i = -lam^T (dL/da_i) u and dloss/dc = -lam^T (dL/dc) u with
 * lam = L^{-1} dloss/du).  Inputs: d_u = L^{-1} f and d_lam = L^{-1} g
 * (both [nrhs][M..]).  Outputs h_grad_a[N] and *h_grad_c on the host (sums
 * over all right-hand sides), evaluated matrix-free in float64.  Synchronises.
 */
int fem_fft_grad_coeffs(fem_fft_plan plan, const double* d_u, const double* d_lam, int64_t nrhs,
                        double* h_grad_a, double* h_grad_c, void* stream);

/*
 * Plan queries (host, synchronous): sizes and the 1D tables of axis i, for
 * tests.  h_lam/h_cnorm receive M_i values (h-free eigenvalues and C-norms in
 * the spectral order above); h_p receives K_i * n * (n-1) values: p_k^(l)
 * for k >= 1 at [k][l-1][:], e^(l) at [0][l-1][:].  Any pointer may be NULL.
 */
int fem_fft_plan_dims(fem_fft_plan plan, int* N, int* n, int64_t* h_M, int* precision);
/* the element order of every axis (h_n[N]); fem_fft_plan_dims reports n = 0
 * when they differ */
int fem_fft_plan_orders(fem_fft_plan plan, int* h_n);
int fem_fft_axis_tables(fem_fft_plan plan, int axis, double* h_lam, double* h_cnorm, double* h_p);

/*
 * fem_fft_axis_precompute -- host only (no device call): the 1D tables of
 * one axis exactly as fem_fft_plan_create computes them (Section 3,
 * Theorem 1; double-double precompute).  h_lam, h_cnorm: M = nK-1 values in
 * the spectral order above; h_p: K*n*(n-1) values as in fem_fft_axis_tables.
 * Any output pointer may be NULL.  Returns FEM_FFT_ERR_ARG for n outside
 * 1..9 or K outside the supported set, FEM_FFT_ERR_ASSUMPTION_A if an
 * eigenproblem fails.
 */
int fem_fft_axis_precompute(int n, int64_t K, double X, double* h_lam, double* h_cnorm, double* h_p);

/*
 * Kernel timing (tracing; no paper counterpart).  fem_fft_profile(plan, 1)
 * starts recording a CUDA event pair around every kernel the plan launches
 * (on the launch stream), with the algorithmic HBM bytes and arithmetic of
 * that launch; fem_fft_profile(plan, 0) stops and clears.  Kinds: 0 forward
 * pencil pass, 1 fused forward/divide/inverse pass, 2 inverse pass,
 * 3 matrix-free operator apply in float64 (arithmetic: float64 flops, FMA = 2),
 * 4 operator apply in double-float (arithmetic: float32 operations of the
 * double-float algorithm).  fem_fft_profile_read synchronises and returns,
 * for one kind, the launch count, summed device milliseconds, summed
 * algorithmic bytes and arithmetic (any pointer may be NULL).
 */
int fem_fft_profile(fem_fft_plan plan, int enable);
int fem_fft_profile_read(fem_fft_plan plan, int kind, int64_t* launches, double* ms, double* bytes,
                         double* flops64);

/*
 * fem_fft_apply_noalloc -- d_b = L d_u (float64, matrix-free, the same
 * operator as fem_fft_apply) for callers that cannot allocate device memory at
 * the point of the call: it needs no plan and calls no cudaMalloc/cudaFree or
 * allocating library routine (for example a host callback or allocator hook
 * that must not re-enter the allocator, or a framework that forbids device
 * allocation after its warm-up).  The paper has no counterpart; this is a
 * service entry point of the library.
 *   N, n, h_K, h_X, h_a, c  as for fem_fft_plan_create, with the same
 *             validity rules (FEM_FFT_ERR_ARG otherwise)
 *   d_u, d_b  caller-owned device arrays [nrhs][M_1..M_N]; the two ranges
 *             must not overlap (FEM_FFT_ERR_ARG)
 * The float64 temporaries live in one static device array of 64 MiB that
 * every GPU loading this library holds until the process exits; a problem
 * needing more than 8 * DOF * T bytes (T = 3, 4 temporaries for N = 2, 3;
 * N = 1 needs none and is limited to 9 * 2^20 unknowns) returns
 * FEM_FFT_ERR_ARG before any launch.  All calls share that array and it keeps
 * the last call's contents (every temporary is written before it is read):
 * calls whose kernels overlap on the GPU race and must be serialised.  The
 * first call on a device looks up the array's address (cudaGetSymbolAddress,
 * with that device current) and caches it; make that first call before any
 * stream capture.  Asynchronous on stream.
 */
int fem_fft_apply_noalloc(int N, int n, const int64_t* h_K, const double* h_X, const double* h_a, double c,
                          const double* d_u, double* d_b, int64_t nrhs, void* stream);

/*
 * Batched solves (many problems of uneven N, n, K and right-hand-side counts
 * replayed from one CUDA graph: per element order present, one
 * dependency-driven kernel launch that runs every step of every problem of
 * that order from a ticket-ordered work list).  Each problem
 * is solved as fem_fft_solve would solve it with a mixed-precision plan:
 * the plan's algorithm of Section 4 ((a), or (b) with its band solve as three
 * batch steps) in float32, then `steps` float64 residual refinement steps.  The batch is an execution schedule over existing plans;
 * it owns no copy of their tables or workspaces.
 *
 * fem_fft_batch_create -- record the solve chains of nprob plans and build
 * the work list.
 *   plans    nprob distinct plans, each created with FEM_FFT_MIXED; they
 *            must outlive the batch, and their own solves must not run
 *            concurrently with the batch's (the workspaces are shared)
 *   h_nrhs   right-hand sides per problem, 1 <= h_nrhs[p] <= the plan's max_nrhs
 *   steps    refinement steps (0..16; 2 reaches float64 accuracy)
 *   tune_cache  path of a JSON autotune cache (NULL: none).  Entries for this
 *            GPU are read; new ones are written back.
 *   tune     1: time candidate tile shapes (pencils per tile) and radix
 *            schedules for every (n, K, contiguous/strided, pass) the batch
 *            uses and is missing from the cache (a few seconds); 0: use the
 *            cache, else the stand-alone passes' choices
 *   stream   used for the tuning launches; the call synchronises it
 * Returns FEM_FFT_ERR_ARG for a non-mixed or repeated plan or a pencil too
 * large for the persistent kernel's shared memory.  When some plan has
 * different element orders on its axes (fem_fft_plan_create_orders) nothing
 * is recorded: the batch starts in FEM_FFT_BATCH_STREAMS mode (four streams)
 * and FEM_FFT_BATCH_GRAPH is refused (the batched kernel runs one element
 * order per launch).
 */
int fem_fft_batch_create(fem_fft_batch* out, const fem_fft_plan* plans, int nprob, const int64_t* h_nrhs,
                         int steps, const char* tune_cache, int tune, void* stream);
int fem_fft_batch_destroy(fem_fft_batch batch);

/*
 * fem_fft_batch_layout -- the packed layout of the batch's fields: problem p
 * occupies float64 elements [h_offsets[p], h_offsets[p] + nrhs_p * DOF_p) of
 * one buffer of *total_len elements, in the layout of fem_fft_solve
 * ([nrhs][M_1..M_N], C order).  Also the number of steps (pencil passes and
 * operator applies of all chains) and work items.  Any pointer may be NULL.
 */
int fem_fft_batch_layout(fem_fft_batch batch, int64_t* h_offsets, int64_t* total_len, int64_t* n_steps,
                         int64_t* n_items);

/*
 * fem_fft_batch_solve -- d_u = L_p^-1 d_b for every problem p, both packed
 * device buffers of total_len float64 (distinct; d_b is not modified).
 * Asynchronous on stream: one graph launch (per element order, a counter
 * reset and one kernel).  When d_b or d_u differ from the previous call the step table is
 * rewritten first (this synchronises stream).  Device-side waits are bounded:
 * check fem_fft_batch_status after the solve.
 */
int fem_fft_batch_solve(fem_fft_batch batch, const double* d_b, double* d_u, void* stream);

/*
 * fem_fft_batch_set_mode -- how fem_fft_batch_solve executes (no paper
 * counterpart; the arithmetic is the same Section 4 solve either way, the
 * results agree to rounding).
 *   FEM_FFT_BATCH_GRAPH    the recorded work list in one graph launch (above;
 *                          the default)
 *   FEM_FFT_BATCH_STREAMS  every problem solved by its own plan
 *                          (fem_fft_solve with the batch's refinement steps,
 *                          the plan's own tuned kernels) on one of nstreams
 *                          (1..64) streams owned by the batch, forked from and
 *                          joined back into the solve's stream; problems are
 *                          assigned largest first to the least loaded stream.
 *                          fem_fft_batch_status reports no device wait in this
 *                          mode; each plan's fem_fft_last_info holds its status.
 * Synchronises the device.  FEM_FFT_ERR_ARG for an unknown mode or nstreams
 * out of range.
 */
enum { FEM_FFT_BATCH_GRAPH = 0, FEM_FFT_BATCH_STREAMS = 1 };
int fem_fft_batch_set_mode(fem_fft_batch batch, int mode, int nstreams);

/*
 * fem_fft_batch_status -- synchronise stream and return the status of the
 * last solve: FEM_FFT_OK, or FEM_FFT_ERR_TIMEOUT when a dependency wait gave
 * up (the results are then incomplete; *h_step names the waiting step).
 */
int fem_fft_batch_status(fem_fft_batch batch, void* stream, int* h_status, int64_t* h_step);

/*
 * fem_fft_batch_tuning -- the tuned (n, K, strided, mode, W, V, split)
 * entries of the passes the batch uses, 7 ints each in h_entries (mode: 0
 * forward, 1 inverse, 2 fused pass; W pencils per tile; V FFT values per
 * thread; split: the fused pass runs as forward-with-division + inverse), and
 * microseconds per pencil in h_us.  Returns the entry count (at most
 * max_entries are written).
 */
int fem_fft_batch_tuning(fem_fft_batch batch, int max_entries, int* h_entries, double* h_us);

/* Time limit of one device-side dependency wait (default 2 s). */
int fem_fft_batch_set_wait_limit(fem_fft_batch batch, double seconds);

/*
 * fem_fft_batch_hold_step -- test hook of the bounded waits: step `step`
 * (which must have a predecessor) waits for one item more than its
 * predecessor has, so that its waits run out; -1 restores the schedule.
 * Takes effect at the next solve.
 */
int fem_fft_batch_hold_step(fem_fft_batch batch, int64_t step);

/*
 * fem_fft_batch_order -- the level order of the work list (host only): the
 * steps of nprob chains of nsteps[p] steps, step 0 of every problem first
 * (problems by decreasing `work`, which may be NULL), then step 1, and so on.
 * Writes (problem, step) pairs to h_prob/h_step (sum of nsteps entries) and
 * returns their count.
 */
int fem_fft_batch_order(int nprob, const int* nsteps, const double* work, int* h_prob, int* h_step);

/*
 * fem_fft_apply_tiling -- the block tiling of the operator apply launches
 * (host only; no paper counterpart): for an axis of K elements with `outer`
 * positions before it and `inner` after it (inner == 1: the contiguous axis),
 * *h_tw positions per block (lines of the contiguous axis when inner == 1
 * and *h_tw > 1, each with 256 / *h_tw element slots) and *h_blocks blocks.
 * Either pointer may be NULL.  FEM_FFT_ERR_ARG for a non-positive size.
 */
int fem_fft_apply_tiling(int64_t inner, int64_t outer, int64_t K, int* h_tw, int64_t* h_blocks);

/*
 * fem_fft_apply_block_map -- the thread map of one block of that tiling
 * (host only; no paper counterpart), computed by the same decode the apply
 * kernels run: for each of the block's 256 threads t, the outer index
 * h_o[t], the position h_w[t] (the line in lines mode) and the element h_e[t]
 * it applies, or -1 in all three when the thread has no element.  Host
 * arrays of 256 entries.  FEM_FFT_ERR_ARG for a non-positive size, a NULL
 * array or a block outside [0, blocks).
 */
int fem_fft_apply_block_map(int64_t inner, int64_t outer, int64_t K, int64_t block, int64_t* h_o, int64_t* h_w,
                            int64_t* h_e);

/*
 * fem_fft_divide_check -- the float64 division of the spectral divide
 * (Section 4, algorithm (a): coefficient / (sum_i a_i s_i lambda_i + c)) as
 * the float64 passes compute it -- a float reciprocal seed refined by two
 * Newton steps, then one product -- next to CUDA's float64 division, for n
 * pairs (no paper counterpart; a diagnostic for tests).  d_q[i] = the passes'
 * x[i] / d[i], d_ref[i] = CUDA's.  Device arrays of n float64; d[i] must lie
 * in the float range (|d| between 2^-126 and 2^127), as every divisor of a
 * plan does.  Asynchronous on stream.  FEM_FFT_ERR_ARG for n < 0 or a NULL
 * pointer with n > 0.
 */
int fem_fft_divide_check(const double* d_x, const double* d_d, double* d_q, double* d_ref, int64_t n, void* stream);

/* Static text for a status code; fem_fft_last_error: the last CUDA error
 * text recorded by this thread (empty if none). */
const char* fem_fft_strerror(int code);
const char* fem_fft_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* FEMFFT_H_ */

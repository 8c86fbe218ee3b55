/*
 * ddeig.h -- C ABI of the GB300 two-level domain-decomposition eigensolver.
 *
 * Computes the ground state (lambda_1, phi) of the Schroedinger eigenproblem
 *     -Laplace(phi) + V phi = lambda phi  on  (0,L)^p x (0,ell),  phi = 0 on the boundary
 * (Theisen & Stamm, arXiv 2311.08757: the Schroedinger equation and box geometry of Sec. 1)
 * discretised by Q1 finite elements on the uniform grid h = 1/n (Sec. 2, discrete weak
 * form): A x = lambda B x with A = K + M_V, B = M.  The method is the shifted inverse
 * iteration x_{k+1} = A_sigma^{-1} B x_k of Sec. 2, sigma the lowest eigenvalue of the
 * x-periodic unit-cell problem (cell problem of Sec. 1, weak cell problem of Sec. 2).  Each
 * shifted system A_sigma w = b (A_sigma = A - sigma M) is solved by conjugate gradients
 * preconditioned with the two-level additive Schwarz operator M_AS2^{-1} (Sec. 2.2, Sec. 3.1)
 * (one overlapping subdomain per unit cell, PerFact coarse space of Definition 2.1).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Supported geometry: p in {1, 2} expanding directions, q = 1 fixed direction.
 *  - Vectors over the box are FP64 arrays of length
 *        ndof = (L n - 1)^p (ell n - 1)
 *    holding the values at the interior nodes, y fastest, then x_p, ..., x_1 slowest:
 *    node (a, j) (1 <= a <= Ln-1, 1 <= j <= ell n - 1) is entry (a-1)(ell n-1) + (j-1);
 *    for p = 2, node (a1, a2, j) is ((a1-1)(Ln-1) + (a2-1))(ell n-1) + (j-1).
 *  - Cell vectors (psi) have length n^p (ell n - 1): node (a, j), 0 <= a < n, is entry
 *    a(ell n - 1) + (j-1) (p = 2: ((a1 n + a2)(ell n - 1) + j - 1)).
 *  - V_cell_qp: the potential sampled on the unit cell at tensor Gauss-Legendre points,
 *    quad_pts per direction.  Element-major: elements (ex, ey) (p = 2: (ex1, ex2, ey)),
 *    ey fastest, element (ex, ey) = [ex h, (ex+1) h] x [ey h, (ey+1) h]; inside an element
 *    the quad_pts^(p+1) points are ordered (qx, qy) (p = 2: (qx1, qx2, qy)), qy fastest.
 *    Length n^p (ell n) quad_pts^(p+1).  V must be 1-periodic in x (assumption A1).
 *  - Pointer arguments marked "host or device" may point to device memory or to host
 *    memory (pageable or pinned); host buffers are staged through the context's device
 *    buffers inside the call.  The caller owns every buffer it passes; the context owns
 *    everything it allocates.
 *  - Calls run on the CUDA stream given to dd_setup and return after the work has
 *    completed (each call synchronises that stream before returning its scalars).
 *  - Every call returns DD_OK (0) or a negative status; no exception crosses the ABI and
 *    nothing aborts the process.  dd_status_string() names a status; dd_last_error()
 *    gives a message for the last failure in the context.
 */
#ifndef DDEIG_H
#define DDEIG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DD_OK           0
#define DD_EINVAL      -1   /* bad argument or grid (L < 1, n < 3, delta < 1, 2 delta >= n, nV mismatch ...) */
#define DD_ESTATE      -2   /* call out of order (e.g. pcg_solve before coarse_build) */
#define DD_ENOMEM      -3   /* device allocation failed */
#define DD_ECUDA       -4   /* CUDA runtime error */
#define DD_ENAN        -5   /* non-finite input or iterate */
#define DD_ENOTSPD     -6   /* non-positive pivot or p^T A p <= 0 (operator or shift not SPD) */
#define DD_EMAXIT      -7   /* iteration limit reached; outputs hold the last iterate */
#define DD_ETIMEOUT    -8   /* a bounded device-side wait gave up; the context must be destroyed */
#define DD_EUNSUPPORTED -9  /* option combination not built (e.g. a precision for this size) */

/* Local-inverse precision (the only place below FP64). */
#define DD_PREC_FP64 0      /* local solves by FP64 banded Cholesky (plain method) */
#define DD_PREC_TF32 1      /* dense local inverses, TF32 tensor-core GEMM, FP32 accumulate */
#define DD_PREC_BF16 2      /* dense local inverses, BF16 tensor-core GEMM, FP32 accumulate */
#define DD_PREC_FP8  3      /* dense local inverses, FP8 (E4M3) tensor-core GEMM, FP32 accumulate;
                               A_T^{-1} scaled per type and R_i r per subdomain to the E4M3 range
                               before rounding, the product scaled back in the GEMM's epilogue.
                               The preconditioner is within a few percent of M_AS2^{-1}, but for
                               the shifted local problems of this method that is not close
                               enough: the flexible CG stagnates or diverges (the eigen-solves
                               then end with DD_EMAXIT).  Use BF16 or TF32 for solves. */

/* Partition of unity D_i (Sec. 2.2 equal weights; Sec. 4.1.2 distance based). */
#define DD_PU_EQUAL    0
#define DD_PU_DISTANCE 1

typedef struct {
    int    p;          /* expanding directions: 1 or 2                                     */
    int    q;          /* fixed directions: must be 1                                      */
    int    L;          /* domain length in unit cells, >= 1 (Sec. 1 box geometry, L in N)  */
    double ell;        /* fixed-direction length; ell * n must be an integer >= 2         */
    int    n;          /* elements per unit length, h = 1/n, n >= 3                        */
    int    overlap;    /* delta >= 1 element layers added on each x side (Sec. 3.1), 2 delta < n */
    int    quad_pts;   /* Gauss points per direction for int V phi v: 1..4 (default 2)   */
    int    pu_kind;    /* DD_PU_EQUAL or DD_PU_DISTANCE                                   */
    int    precision;  /* DD_PREC_*                                                        */
    int    coarse;     /* 1: two-level M_AS2 (Sec. 2.2); 0: one-level M_AS1 ablation       */
} dd_grid;

typedef struct dd_ctx dd_ctx;    /* opaque; owns every device buffer it allocates */

/* Sizes and state of a context (filled by dd_query). */
typedef struct {
    long long ndof;          /* interior unknowns of the box                               */
    long long ncell;         /* unknowns of the periodic cell problem                       */
    int       nsub;          /* subdomains N = L^p                                          */
    int       ntypes;        /* distinct local matrices (left/interior/right per axis)      */
    int       nloc_max;      /* largest local problem |N_i|                                 */
    int       kpad;          /* local size padded for the tensor-core GEMM                  */
    int       band_local;    /* half bandwidth of the local matrices                        */
    double    sigma;         /* cell shift (valid after dd_cell_eigenpair)                  */
    int       cell_iters;    /* inverse iterations used by the cell solve                   */
    int       stage;         /* 1 set up, 2 cell eigenpair done, 3 coarse built             */
    long long device_bytes;  /* device memory held by the context                           */
    int       gemm_tile_n;   /* N tile of the mixed local-solve contraction chosen at
                                dd_coarse_build (128, 160 or 256; 0 before it and in FP64)   */
    int       reserved_;     /* zero                                                         */
} dd_info;

/*
 * dd_setup -- validate the grid, allocate the context, upload V and build the periodic
 * stencil tables of A = K + M_V and M (Sec. 2: translated cell meshes make every box row
 * a translated cell row, and V is periodic by assumption A1).
 *   g          grid and options (copied)
 *   V_cell_qp  host or device, nV doubles, layout above; non-finite values -> DD_ENAN
 *   stream     cudaStream_t to run on (NULL = the legacy default stream)
 *   out        receives the context; *out = NULL on failure
 */
int dd_setup(const dd_grid* g, const double* V_cell_qp, size_t nV, void* stream, dd_ctx** out);

/*
 * dd_set_potential -- replace V on an existing context (same grid): uploads V_cell_qp (host or
 * device, nV doubles, layout above), rebuilds the stencil tables of A = K + M_V and M and
 * returns the context to the state after dd_setup (dd_cell_eigenpair and dd_coarse_build
 * must follow).  Lets one context serve many potentials without re-allocating.
 * DD_EINVAL on a size mismatch, DD_ENAN on non-finite values.
 */
int dd_set_potential(dd_ctx* ctx, const double* V_cell_qp, size_t nV);

/*
 * dd_cell_eigenpair -- lowest eigenpair (sigma, psi) of the x-periodic, y-Dirichlet cell
 * problem (cell problem of Sec. 1, weak cell problem of Sec. 2), psi > 0, psi^T M_# psi = 1;
 * then forms A_sigma = A - sigma M (Sec. 1.1) and the coarse weights D_i R_i E^# psi (Def. 2.1).
 *   sigma_out     host, receives sigma (may be NULL)
 *   psi_cell_out  host or device, n^p (ell n - 1) doubles, or NULL
 */
int dd_cell_eigenpair(dd_ctx* ctx, double* sigma_out, double* psi_cell_out);

/*
 * dd_coarse_build -- local matrices A_{sigma,i} = R_i A_sigma R_i^T per distinct subdomain
 * type, factorised (FP64 banded Cholesky) and, for TF32/BF16, inverted and rounded; the
 * coarse matrix A_{sigma,0} = R_0 A_sigma R_0^T (Sec. 3.1) assembled and factorised.
 * DD_ENOTSPD if a local or coarse matrix is not positive definite.
 */
int dd_coarse_build(dd_ctx* ctx);

/*
 * dd_pcg_solve -- solve A_sigma x = b by CG preconditioned with M_AS2^{-1} (Sec. 3.1; the
 * one-level M_AS1^{-1} when grid.coarse = 0); flexible CG (Polak-Ribiere beta) when the
 * local inverses are rounded (TF32/BF16).  Stops when ||r_k||_2 <= rtol ||r_0||_2 (Sec. 4.1).
 *   b          host or device, ndof doubles
 *   x          host or device, ndof doubles; in: initial guess, out: solution
 *   iters_out  host, iterations used (may be NULL);  relres_out host, ||r_k||/||r_0|| (may be NULL)
 * DD_EMAXIT when maxit is reached (x holds the last iterate).
 */
int dd_pcg_solve(dd_ctx* ctx, const double* b, double* x, double rtol, int maxit,
                 int* iters_out, double* relres_out);

/*
 * dd_gmres_solve -- A_sigma x = b by right-preconditioned restarted GMRES (flexible form, so
 * a rounded preconditioner is allowed) with the context's two-level Schwarz preconditioner,
 * M_RAS2^{-1} or M_AS2^{-1} (DD_OPT_PRECOND; Sec. 2.2 pairs the restricted one with GMRES),
 * restart length DD_OPT_RESTART.  Arnoldi by classical Gram-Schmidt applied twice.
 *   b        host or device, ndof doubles
 *   x        host or device, ndof doubles; in: initial guess, out: solution
 *   stops when the method's own residual (the least-squares residual of the Arnoldi relation,
 *   as PCG stops on its recursive residual) is <= rtol ||b - A_sigma x_0||_2; each restart
 *   begins from the true residual.  relres_out is that residual over ||b - A_sigma x_0||_2.
 * DD_EMAXIT after maxit iterations (x holds the last iterate).  dd_pcg_solve returns
 * DD_EINVAL while the restricted preconditioner is selected.
 */
int dd_gmres_solve(dd_ctx* ctx, const double* b, double* x, double rtol, int maxit, int* iters_out,
                   double* relres_out);

/*
 * dd_inverse_iterate -- shifted inverse iteration (Sec. 2): b = M x_k, solve A_sigma w = b
 * by dd_pcg_solve with zero initial guess and relative tolerance rtol_inner, x_{k+1} =
 * w / ||w||_M (sign: sum x > 0); rho = x^T A x, eta = ||A x - rho M x||_2 / (|rho| ||M x||_2).
 * Stops when eta <= tol_res and |rho_k - rho_{k-1}| <= tol_lam |rho_k|.
 *   x                host or device, ndof doubles; in: x_0 (any nonzero vector; its M-norm is
 *                    normalised), out: phi (M-normalised)
 *   lambda_out       host, the Rayleigh quotient rho of the returned x (may be NULL)
 *   outer_out, inner_total_out, inner_max_out  host iteration counts (may be NULL)
 */
int dd_inverse_iterate(dd_ctx* ctx, double* x, double tol_res, double tol_lam, int maxit_outer,
                       double rtol_inner, double* lambda_out, int* outer_out,
                       int* inner_total_out, int* inner_max_out);

/*
 * dd_lopcg -- inexact shift-and-invert preconditioned LOPCG (Algorithm 1, Sec. 2.1; inner
 * strategies of Sec. 4.3).  Outer residual r_o = A x_k - rho_k M x_k (x_k M-normalised,
 * rho_k its Rayleigh quotient); inner step w_k:
 *   DD_INNER_FIXED     PCG on A_sigma w = r_o from zero to relative residual rtol_inner
 *   DD_INNER_ADAPTIVE  the same to relative residual min(0.1, ||r_o||_2)
 *   DD_INNER_FUSED     w = M_AS2^{-1} r_o: one application of the two-level Schwarz
 *                      preconditioner, no inner Krylov loop
 * then x_{k+1} = the lowest Ritz vector of span{x_k, w_k, x_{k-1}} (M-orthonormalised basis
 * in the order x_k, w_k, x_{k-1}; a direction whose M-norm drops below 1e-10 of its norm
 * before orthogonalisation is dropped), M-normalised with sum x > 0.  x_0 = e_1 (the first
 * interior node), x_1 = the caller's x.  Stops like dd_inverse_iterate: eta <= tol_res and
 * |rho_k - rho_{k-1}| <= tol_lam |rho_k|.
 *   x                 host or device, ndof doubles; in: x_1 (nonzero), out: phi
 *   inner_total_out   inner PCG iterations summed (preconditioner applications when fused)
 * DD_EINVAL for a bad mode or tolerance, DD_EMAXIT after maxit_outer steps (x holds the
 * last iterate), DD_ENOTSPD / DD_ENAN if the Rayleigh-Ritz basis degenerates.
 */
#define DD_INNER_FIXED    0
#define DD_INNER_ADAPTIVE 1
#define DD_INNER_FUSED    2
int dd_lopcg(dd_ctx* ctx, double* x, int inner, double tol_res, double tol_lam, int maxit_outer,
             double rtol_inner, double* lambda_out, int* outer_out, int* inner_total_out,
             int* inner_max_out);

/*
 * dd_potential_gradient -- gradient of a function of the ground state with respect to the
 * potential values V_cell_qp (the layout of dd_setup's V).  The potential enters only through
 * M_V (Sec. 1: (V phi, v) by tensor Gauss quadrature), so for the M-normalised ground state
 * (lambda, phi):
 *   d lambda / dV_cell_qp[e, q] = sum over the copies of cell element e of h^d W_q phi_h(z_q)^2
 *     (Hellmann-Feynman: d lambda = phi^T dA phi),
 * and for a loss l(phi) with g = dl/dphi, with w the solution of the projected singular
 * system (A - lambda M) w = g - M phi (phi^T g), phi^T M w = 0, solved by projected PCG with
 * the two-level Schwarz preconditioner of the context (preconditioned residuals projected
 * M-orthogonally to phi, so A - lambda M is positive definite on every search direction even
 * with lambda, phi only as accurate as the eigen-solve):
 *   dl / dV_cell_qp[e, q] = - sum over the copies of h^d W_q w_h(z_q) phi_h(z_q).
 * Writes dV = g_lambda * d lambda/dV + dl/dV (the second term only when g_phi != NULL).
 *   phi        host or device, ndof doubles: the M-normalised ground state (dd_inverse_iterate
 *              or dd_lopcg output) of the context's potential; lambda its eigenvalue
 *   g_phi      host or device, ndof doubles, or NULL
 *   rtol       relative residual of the adjoint PCG (e.g. 1e-10)
 *   dV         host or device, nV = n^p ny Q^(p+1) doubles (output)
 *   iters_out  adjoint PCG iterations (0 without g_phi; may be NULL)
 * Needs dd_coarse_build.  DD_EINVAL on a size mismatch, DD_EMAXIT if the adjoint PCG does not
 * converge in 10000 iterations.
 */
int dd_potential_gradient(dd_ctx* ctx, const double* phi, double lambda, double g_lambda,
                          const double* g_phi, double rtol, double* dV, size_t nV, int* iters_out);

/*
 * dd_eigenpair -- convenience: dd_setup, dd_cell_eigenpair, dd_coarse_build and
 * dd_inverse_iterate from x_0 = 1 with tol_res = 1e-8, tol_lam = 1e-10, rtol_inner = 1e-8,
 * maxit_outer = 100, then dd_destroy.
 *   phi_out     host or device, ndof doubles (may be NULL)
 *   lambda_out, sigma_out   host (may be NULL)
 */
int dd_eigenpair(const dd_grid* g, const double* V_cell_qp, size_t nV, void* stream,
                 double* lambda_out, double* phi_out, double* sigma_out);

/*
 * Batched ground states (many independent instances: uneven L, own potential and shift).
 * dd_batch_create sets up one context per instance (grids[i], V[i] of nV[i] doubles, host or
 * device, as for dd_setup; all on the caller's stream).  dd_batch_ground_states runs every
 * instance's whole pipeline -- dd_cell_eigenpair and dd_coarse_build on a pool of `threads`
 * host threads (<= 0: min(count, 16)), largest instance first, each on its own context
 * stream, then from x_0 = 1:
 *   DD_BATCH_IPM             the shifted inverse iteration (tol_res 1e-8, tol_lam 1e-10,
 *                            rtol_inner 1e-8, as dd_inverse_iterate)
 *   DD_BATCH_LOPCG_FUSED     SI-LOPCG with the fused inner step (dd_lopcg, DD_INNER_FUSED)
 *   DD_BATCH_LOPCG_ADAPTIVE  dd_lopcg with DD_INNER_ADAPTIVE, per instance, concurrently
 *   DD_BATCH_IPM_CONCURRENT  dd_inverse_iterate per instance on the thread pool (the instances'
 *                            own launches overlap on the GPU)
 * DD_BATCH_IPM and DD_BATCH_LOPCG_FUSED run BATCHED when the instances share p = 1, the
 * precision (BF16 or TF32), h, delta, ell, quadrature and partition of unity: the instances
 * are split into G groups of about equal total size, each driven by one host thread on its own
 * streams; within a group every kernel of an iteration is one launch over all the group's
 * instances (the blocks of each instance's own launch side by side; the local solves one
 * grouped tensor-core contraction over the instances' tiles), a block of PCG iterations is one
 * CUDA graph, each instance keeps its own device scalars, kernels of an instance whose solve is
 * done return at once, an instance joins its group's iteration as soon as its own set-up is
 * done and drops out when its eigen-iteration stops.  G (1, 2, 4 or 8) is set by
 * dd_batch_set_groups, or, with 0 (the default), chosen by timing: each count is tried on
 * successive calls (its first use builds it) and the fastest is kept; -1 runs every method per
 * instance.  Otherwise these two methods run per instance, concurrently.
 * Outputs per instance (arrays of count entries, each may be NULL): lambda, outer and inner
 * iteration counts, wall seconds from the start of the call to the instance's eigenpair;
 * phi_out[i] (host or device, ndof_i doubles; phi_out or an entry may be NULL).
 * Returns the first failing instance's status (the others still run).  Results equal those
 * of the single-instance calls bit for bit (same arithmetic per instance, deterministic
 * reductions), batched or not, for every G.
 * dd_batch_context gives instance i's context (owned by the batch) for options and queries;
 * a context with timing, GMRES, the restricted preconditioner, the dense coarse solve or the
 * two-kernel p update selected makes these methods run per instance.  dd_batch_info reports
 * whether the batch qualifies for the batched kernels, whether the last call ran them, the N
 * tile of the grouped contraction of its first group (timed on the group's operands when the
 * group was built), the number of groups, and the wall seconds of the last call's set-up phase
 * (until every instance's coarse build is done) and of the whole last call (each may be NULL).
 */
typedef struct dd_batch dd_batch;
#define DD_BATCH_IPM            0
#define DD_BATCH_LOPCG_FUSED    1
#define DD_BATCH_LOPCG_ADAPTIVE 2
#define DD_BATCH_IPM_CONCURRENT 3
int dd_batch_create(const dd_grid* grids, const double* const* V, const size_t* nV, int count, void* stream,
                    dd_batch** out);
int dd_batch_ground_states(dd_batch* b, int method, int threads, double* lambda_out, double* const* phi_out,
                           int* outer_out, int* inner_out, double* seconds_out);
int dd_batch_size(const dd_batch* b);
int dd_batch_set_groups(dd_batch* b, int groups);
int dd_batch_info(const dd_batch* b, int* batchable_out, int* last_batched_out, int* gemm_tile_n_out,
                  int* groups_out, double* setup_seconds_out, double* total_seconds_out);
dd_ctx* dd_batch_context(dd_batch* b, int i);
void dd_batch_destroy(dd_batch* b);

/* dd_destroy -- free the context and everything it owns (NULL is ignored). */
void dd_destroy(dd_ctx* ctx);

/* dd_status_string -- static name of a status code. */
const char* dd_status_string(int status);

/* dd_last_error -- message of the last failure recorded in ctx ("" if none; ctx may be NULL
 * for failures of dd_setup itself, which are kept per thread). */
const char* dd_last_error(const dd_ctx* ctx);

/* dd_query -- sizes and state of a context. */
int dd_query(const dd_ctx* ctx, dd_info* info);

/* ---------------------------------------------------------------------------------------
 * Operator-level entry points (same layouts as above).  They expose the individual steps
 * of the iteration so that each can be checked against an independent implementation.
 * ------------------------------------------------------------------------------------- */

#define DD_OP_ASIGMA 0   /* y = A_sigma x  (needs dd_cell_eigenpair)        */
#define DD_OP_MASS   1   /* y = M x                                          */
#define DD_OP_A      2   /* y = (K + M_V) x                                  */

/* y = op x over the box (x, y host or device, ndof doubles). */
int dd_apply_operator(dd_ctx* ctx, int op, const double* x, double* y);

/* y = A_sigma x evaluated by the float-pair pass of the PCG iteration (DD_OPT_PAIRS: each
 * coefficient and x value split into two floats, error-free products and sums on the FP32
 * pipe, y = hi + lo in FP64), whatever DD_OPT_PAIRS is set to: p = 1 the fused p-update pass
 * with beta = 0, p = 2 the split p update and the (tiled, where DD_OPT_TILED3 and the box
 * allow) pair matvec.  It exposes that arithmetic for checking against dd_apply_operator
 * (DD_OP_ASIGMA).  Per node, |y_pairs - y| relative to the sum of |a_ij x_j| over the row: the
 * splits and the dropped lo * lo product leave 2.5 * 2^-47 of each term; the FP32 roundings of
 * the low-order accumulator add an amount that grows with the number of taps.  Largest ratios
 * measured: 8.5 * 2^-47 with the 9 taps of p = 1, 13.4 * 2^-47 with the 27 of p = 2 (tested
 * against 2^-42).  x, y host or device, ndof doubles; needs dd_cell_eigenpair; DD_EINVAL for
 * null pointers or a p = 1 box with more than 256 padded rows (Ypad). */
int dd_apply_asigma_pairs(dd_ctx* ctx, const double* x, double* y);

/* z = M_AS2^{-1} r (or M_AS1^{-1} r), Sec. 3.1 (r, z host or device, ndof doubles);
 * needs dd_coarse_build. */
int dd_apply_preconditioner(dd_ctx* ctx, const double* r, double* z);

/* Coarse matrix A_{sigma,0} = R_0 A_sigma R_0^T copied to host as a dense nsub x nsub
 * row-major array (needs dd_coarse_build; grid.coarse = 1). */
int dd_coarse_matrix(dd_ctx* ctx, double* A0_host);

/* Options of the iteration engine (defaults in brackets):
 *   DD_OPT_CHECK_EVERY  iterations between host convergence checks (iterations after the stop
 *                       return at once) [16]
 *   DD_OPT_USE_GRAPH    replay the PCG iteration as a CUDA graph [1]
 *   DD_OPT_FLEXIBLE     -1 automatic (flexible iff rounded local inverses) / 0 / 1 [-1]
 *   DD_OPT_TIMING       1: time every kernel class with CUDA events (eager launches) [0]
 *   DD_OPT_KRYLOV       inner solver of dd_inverse_iterate / dd_lopcg: 0 PCG, 1 GMRES [0]
 *   DD_OPT_PRECOND      0 M_AS2^{-1} (symmetric, for CG), 1 M_RAS2^{-1} (restricted: local
 *                       solutions weighted by the partition of unity D_i; GMRES only) [0]
 *   DD_OPT_RESTART      GMRES restart length, 1..200, fixed by the first GMRES solve [30]
 *   DD_OPT_COARSE_SOLVE coarse solve u_0 = A_0^{-1} c: 1 cyclic reduction of the tridiagonal A_0
 *                       (p = 1 only), 2 dense A_0^{-1} from its banded Cholesky factor applied
 *                       as a GEMV, 0 = automatic (cyclic reduction for p = 1: measured faster
 *                       beside the local GEMM at 2048 subdomains, and no N^2 set-up; dense for
 *                       p = 2); read by dd_coarse_build [0]
 *   DD_OPT_GEMM_TILE_N  N tile of the mixed local-solve contraction: 128, 160 or 256, 0 = chosen
 *                       by timing each on the context's operands at dd_coarse_build (cached per
 *                       problem shape); the result does not depend on it [0]
 *   DD_OPT_LOCAL_RHS    FP64 local solves: subdomains of one type solved together by one warp,
 *                       1, 2 or 4 (capped by shared memory), 0 = default (2 where allowed) [0]; the result
 *                       does not depend on it (same operations per vector)
 *   DD_OPT_FUSED_PQ     p = 1: -1 automatic / 1 one kernel stages p = z + beta p in shared memory
 *                       and applies the stencil from there (one node per thread and pass), 2 the
 *                       same with two nodes per thread and pass (their tap chains interleaved),
 *                       0 a vector update then the stencil from global memory (the p = 2 form);
 *                       the result is the same bits for 1 and 2; automatic = 2 [-1]
 *   DD_OPT_PROLONG_TABLES p = 1: 1 reads the owners of every node and their packed rows from
 *                       index tables in the prolong-sum; 0 computes them in closed form where
 *                       set-up found the formula equal to the tables (same values, two dependent
 *                       loads fewer per node, but more integer work: 28.1 against 24.5 us per
 *                       launch on the L = 2048, h = 1/32 box) [1]
 *   DD_OPT_PAIRS        the matvec q = A_sigma p of the PCG iteration in float pairs on the FP32
 *                       pipe: each coefficient and p value split into hi + lo (48 significand
 *                       bits), error-free products and sums, q = hi + lo in FP64; q agrees with
 *                       the FP64 stencil to within 2^-42 times the sum of the taps' magnitudes
 *                       (measured up to 13.4 * 2^-47; the FP64 one: about 2^-53; see
 *                       dd_apply_asigma_pairs).  p = 1: inside the fused p update pass; p = 2: the p
 *                       update also stores p split.  p, q, x, r, z and their updates, every dot
 *                       product, the coarse solve, the outer iteration's residuals and Rayleigh
 *                       quotients, the stop rules and dd_apply_operator stay FP64.  0: the FP64
 *                       matvec.  p = 1 needs at most 256 padded rows (Ypad).  -1: 1 when the
 *                       local inverses are rounded (precision other than FP64), else 0 [-1]
 *   DD_OPT_PDL          1: the kernels of the PCG iteration's chain (fused p update, x/r update,
 *                       restriction packing, local contraction, prolong-sum) are launched with
 *                       programmatic dependent launch, so that each one's blocks are scheduled
 *                       while its predecessor drains (each waits for the predecessor's results
 *                       before reading anything); 0: plain launches.  The same results; on the
 *                       L = 2048, h = 1/32 box the ground state took 24.0 ms with it against
 *                       23.3 ms without, hence off by default [0]
 *   DD_OPT_FUSE_XR      p = 1, BF16/TF32 local inverses, fused p update, at most 4096
 *                       subdomains: 1 runs the iteration's x, r update inside the restriction
 *                       packing (each subdomain's block forms r - alpha q for its packed row and,
 *                       on the node columns it owns, updates x (unless DD_OPT_X_LAG) and sums
 *                       (r, r) and takes the stop test), and the prolong-sum stores r - alpha q;
 *                       one kernel fewer per iteration.  x and r take the same values as with
 *                       0; (r, r) is summed in another order.  On the L = 2048, h = 1/32 box a
 *                       PCG iteration took 104.5 us against 99.3 us with 0 (106.0 us without
 *                       DD_OPT_X_LAG): the packing blocks, one per overlapping subdomain, form
 *                       r - alpha q and (r, r) slower than the separate update does, so off by
 *                       default; -1: off [0]
 *   DD_OPT_TILED3       p = 2 with float pairs: 1 evaluates q = A_sigma p tile by tile from
 *                       shared memory (each block takes the planes of one residue a1 mod n, so
 *                       it stages the n Ypad classes of the split table once, and for every tile
 *                       the split p of three planes), where n Ypad <= 448; 0 reads the table and
 *                       p through the caches.  The same q; (p, q) summed in another order [1]
 *   DD_OPT_X_LAG        1: the PCG update x_{k+1} = x_k + alpha_k p_k is made by iteration k + 1's
 *                       p update (which reads p_k anyway), and once more after the last
 *                       iteration, so the x/r update streams only r and q; the same FMA on the
 *                       same operands, so x is bit-identical to 0 (x updated with r); with
 *                       DD_OPT_FUSE_XR the fused packing then leaves x alone too [1] */
#define DD_OPT_CHECK_EVERY 0
#define DD_OPT_USE_GRAPH   1
#define DD_OPT_FLEXIBLE    2
#define DD_OPT_TIMING      3
#define DD_OPT_LOCAL_RHS   4
#define DD_OPT_KRYLOV      5
#define DD_OPT_PRECOND     6
#define DD_OPT_RESTART     7
#define DD_OPT_GEMM_TILE_N 8
#define DD_OPT_COARSE_SOLVE 9
#define DD_OPT_FUSED_PQ    10
#define DD_OPT_PROLONG_TABLES 11
#define DD_OPT_PAIRS       12
#define DD_OPT_PDL         13
#define DD_OPT_FUSE_XR     14
#define DD_OPT_TILED3      15
#define DD_OPT_X_LAG       16
int dd_set_option(dd_ctx* ctx, int option, int value);

/* Per-kernel-class timing collected while DD_OPT_TIMING = 1: for class k (0 <= k < count),
 * names[k] (static string), launches[k] and total device milliseconds ms[k].  Pass NULL
 * arrays to get only *count.  dd_reset_timings zeroes the counters. */
int dd_kernel_timings(dd_ctx* ctx, int* count, const char** names, long long* launches, double* ms);
int dd_reset_timings(dd_ctx* ctx);

/* Number of kernel launches this library has issued in the process so far (a replayed CUDA
 * graph counts each of its kernel nodes); differences bracket a region of interest. */
long long dd_kernel_launch_count(void);

/* Self-test of the tensor-core contraction used for the local solves (no paper counterpart;
 * it checks the kernel in isolation): D[n][m] = sum_k A[m][k] B[n][k] for host row-major
 * A (M x K) and B (N x K), rounded to BF16 (precision = DD_PREC_BF16, nearest even), to
 * E4M3 (DD_PREC_FP8, nearest even, saturating; unscaled) or read as TF32 (DD_PREC_TF32),
 * FP32 accumulation; D is host N x M row-major.  Allocates and
 * frees its own device buffers.  DD_ETIMEOUT if a bounded device wait expired. */
int dd_tc_gemm_test(int precision, int M, int N, int K, const float* A_host, const float* B_host, float* D_host);

/* Self-test of the device precision conversions of the mixed form (no paper counterpart;
 * they round the restrictions R_i r to the GEMM's operand type and widen its FP32 results
 * with integer operations, off GB300's narrow FP64 pipe).  n host values in, n host values out:
 *   kind 0: double -> BF16 bits (uint16), IEEE round to nearest even;
 *   kind 1: double -> TF32 (float whose low 13 mantissa bits are zero), nearest, ties away;
 *   kind 2: float -> double (exact).
 * Allocates and frees its own device buffers.  DD_EINVAL for a bad kind, n < 1 or a null
 * pointer. */
int dd_convert_test(int kind, long long n, const void* in_host, void* out_host);

/* Self-test of the arithmetic pipes that bound the FP64 vector kernels (no paper counterpart;
 * it measures their roofline denominators on the GPU at hand): kind 0 the FP64 fused
 * multiply-add (DFMA) pipe, kind 1 the FP32 one (FFMA).  Every thread of 8 blocks of 256 per
 * SM runs 8 independent FMA chains; *tflops_out receives 2 flops per FMA over the CUDA-event
 * time of the fastest of `reps` launches (1..100, after one untimed launch), in TFLOP/s.
 * Allocates and frees its own device buffers.  DD_EINVAL for a bad kind or reps or a null
 * pointer. */
int dd_alu_peak_test(int kind, int reps, double* tflops_out);

/* Allocation-free form of the same tensor-core contraction (the paper has no counterpart: it
 * exists for callers that cannot allocate device memory where they need the product, such as
 * a server whose device memory is reserved up front by its own arena, or a latency-critical
 * path where cudaMalloc/cudaFree would synchronise the device).
 *   D[n][m] = sum_k A[m][k] B[n][k], FP32 accumulation.
 *   A_dev  device, M x K row-major: BF16 (precision = DD_PREC_BF16) or FP32 read as TF32
 *   B_dev  device, N x K row-major, same type;  D_dev device, N x M row-major FP32
 *   K must be a multiple of 64; ceil(M/128) * ceil(N/256) <= 4096, otherwise DD_EINVAL.
 *   stream cudaStream_t (NULL = legacy default); the call returns after the product is done.
 * Allocates nothing: the kernel's scratch (tile list, error word of its bounded waits) is a
 * fixed 64 KB array in the library's static device memory, present on every GPU that loads
 * the library until the process exits.  The first call on a device looks up that array's
 * device address (cudaGetSymbolAddress) and caches it.  No call may be made while its
 * stream is being captured into a CUDA graph: every call copies its tile list from host
 * memory and synchronises the stream before it returns.  All calls share the array and it
 * keeps the last call's contents, so calls that overlap on the GPU (concurrent streams or
 * threads) race and must be serialised by the caller.  DD_ETIMEOUT if a bounded device
 * wait expired. */
int dd_tc_gemm_noalloc(int precision, int M, int N, int K, const void* A_dev, const void* B_dev, float* D_dev,
                       void* stream);

#ifdef __cplusplus
}
#endif

#endif /* DDEIG_H */

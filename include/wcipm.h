/*
 * wcipm.h -- C ABI of the GB300 library for the inner Newton solve of a
 * primal-dual interior-point method on low-rank SDPs, following
 * Chiu & Zhang, "Well-conditioned primal-dual interior-point method for
 * accurate low-rank semidefinite programming" (arXiv 2407.14013).
 *
 * Problem (Section 1, eq. sdp-pd):  min <C,X>  s.t.  A(X) = b,  X PSD,
 * with A(X) = [<A_i, X>]_{i=1..m}.  Given the eigen-decomposition of the
 * Nesterov-Todd scaling point W = V diag(lam) V^T and the residuals
 * (C~, b~), one call of sdp_newton_solve returns the Newton direction of
 * (Newt-eps) (Section 3):
 *
 *   [ -(W (x)s W)^{-1}  A^T ] [svec dX]   [svec C~]
 *   [        A           0  ] [  dy   ] = [   b~  ],   dS = C~ - A^T(dy),
 *
 * computed, as the paper proposes, through the well-conditioned augmented
 * system (eq. augsys) solved by PCG with the indefinite preconditioner of
 * Cor. pcg, then recovered with eq. recover.  Every step runs in the
 * library's own CUDA kernels (sm_103a) on the stream given at setup.
 *
 * Conventions shared by every entry point
 *   - Symmetric n x n matrices are full, column-major, FP64 (row- and
 *     column-major coincide; both triangles must be filled).
 *   - Unless a function says otherwise, array arguments are DEVICE pointers
 *     that the caller allocates and owns; they must stay valid until the
 *     call returns (all calls return after their work has completed on the
 *     handle's stream).
 *   - The handle owns all scratch memory.  The Newton solve's workspace is
 *     allocated once in sdp_setup (sized for the largest rank the options
 *     allow); sdp_newton_solve, sdp_newton_resolve, sdp_newton_solve_host and
 *     sdp_grad allocate nothing.  Three workspaces are allocated on first use
 *     and kept by the handle: the interior-point loop's (ipm_step, sdp_solve,
 *     sdp_scaling_point, sdp_center, sdp_solve_slack, sdp_solve_batch: about
 *     24 n^2 doubles), the linear block's (sdp_set_linear_diag, sdp_grad_slack:
 *     m + m d_max doubles) and the slack variables' (sdp_solve_slack: 14 m
 *     doubles); each reports SDP_ENOMEM if it cannot be allocated.
 *   - Status codes are returned; sdp_last_error() gives a message.  A CUDA
 *     error reported by the runtime is returned as SDP_ECUDA and leaves the
 *     handle unusable except for sdp_destroy.
 *   - A handle may be used by one host thread at a time.
 */
#ifndef WCIPM_H
#define WCIPM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sdp_handle sdp_handle;

typedef enum {
  SDP_OK = 0,
  SDP_EINVAL = 1,        /* bad argument: shape, NULL pointer, r out of range, unsorted COO ... */
  SDP_ENOMEM = 2,        /* workspace allocation failed in sdp_setup                            */
  SDP_ECUDA = 3,         /* a CUDA runtime error; see sdp_last_error                            */
  SDP_ENOTCONV = 4,      /* PCG reached max_pcg without the stopping test; outputs hold the last iterate */
  SDP_ENUMERIC = 5,      /* non-finite or non-positive PCG scalar, or a non-positive pivot     */
  SDP_ETIMEOUT = 6,      /* a bounded device-side wait gave up (sdp_set_tc_wait_limit_ns)          */
  SDP_EUNSUPPORTED = 7   /* option combination not built                                        */
} sdp_status;

/* Storage kinds of the constraint operator A (eq. sdp-pd; rows svec(A_i) of (Newt-eps)). */
typedef enum {
  SDP_A_DIAG = 0,        /* A_i = e_i e_i^T, m = n: A(X) = diag(X)                               */
  SDP_A_SPARSE_COO = 1,  /* entries (con, row, col, val), row >= col, sorted by con (ascending):
                            <A_i, X> = sum over entries of con i of val * X[row,col] * (row==col ? 1 : 2).
                            Repeated positions within a constraint add up.  sdp_setup copies the
                            entries to the host once, validates them (EINVAL: an unsorted or
                            out-of-range con, col > row, row >= n, a non-finite val, a constraint
                            with no entry, nnz < 1 or nnz > 2^31 - 1) and uploads two index tables
                            into the workspace (entries by constraint, entries by position); the
                            handle keeps reading the caller's four arrays.  The mixed forms are not
                            built for this kind (EUNSUPPORTED).                                    */
  SDP_A_DENSE_SVEC = 2   /* a_dense: m x n(n+1)/2 row-major, row i = svec(A_i): lower triangle
                            column by column, off-diagonal entries times sqrt(2) (Notations)     */
} sdp_a_kind;

typedef enum {
  SDP_FP64 = 0,          /* every product in FP64 (the plain form)                                */
  SDP_MIXED_FP32 = 1,    /* FP64 iterative refinement of the augmented-system solution from x = 0:
                            the FP64 residual rho = g - M x, then the same PCG on M~ delta = rho
                            from delta0 = P^{-1}[0; rho_v], x += delta, until the FP64 residual
                            passes the stop test.  M~ forms the block A E A^T from an FP32 copy
                            of A (DENSE) or of E o E (DIAG) with FP32 products; its rows with
                            B = A Q, the vectors, scalars and the preconditioner stay FP64.
                            If a correction solve breaks down, or max_refine corrections do not
                            reach the stop test, the FP64 PCG continues from the refined iterate
                            (its iterations count in pcg_iters).                              */
  SDP_MIXED_TF32 = 2,    /* as SDP_MIXED_FP32, with the n^3 products E Y E of the correction
                            operator (DENSE kind) run on the tensor cores (tcgen05 kind::tf32,
                            FP32 accumulation in TMEM), each FP32 operand split into TF32 parts
                            hi + lo and the product taken as hi hi + hi lo + lo hi (three MMAs
                            per step, about FP32 accuracy); the passes over A stream its FP32
                            copy.  DIAG kind: the same as SDP_MIXED_FP32 (its A E A^T block,
                            (E o E) p_u, has no matrix product)                              */
  SDP_MIXED_BF16 = 3     /* as SDP_MIXED_FP32 with a BF16 copy of A (DENSE kind, 2 bytes per
                            entry, rows zero-padded to a multiple of 8 entries) or of E o E
                            (DIAG kind), BF16 products summed in FP32 in the passes, and E Y E
                            as BF16 tensor-core products (tcgen05 kind::f16, FP32 accumulation);
                            the FP64 refinement recovers the accuracy of the direction        */
} sdp_precision;

typedef struct {
  int32_t n;             /* matrix order, >= 2                                                  */
  int32_t m;             /* number of constraints, >= 1                                          */
  int32_t kind;          /* sdp_a_kind                                                          */
  int32_t pad_;
  int64_t nnz;           /* SPARSE_COO: number of entries                                        */
  const int32_t* a_con;  /* SPARSE_COO: device int32[nnz], constraint index, nondecreasing        */
  const int32_t* a_row;  /* SPARSE_COO: device int32[nnz]                                        */
  const int32_t* a_col;  /* SPARSE_COO: device int32[nnz], a_col <= a_row                        */
  const double* a_val;   /* SPARSE_COO: device double[nnz]                                       */
  const double* a_dense; /* DENSE_SVEC: device double[m * n(n+1)/2]                              */
} sdp_problem;

typedef struct {
  int32_t r_fixed;       /* > 0: use this rank parameter r (1 <= r < n)                          */
  int32_t r_hat;         /* r_fixed == 0: r = argmax_{i <= r_hat} lam_i/lam_{i+1} (Section 7)     */
  int32_t precision;     /* sdp_precision                                                       */
  int32_t precond_space; /* 0 = auto (the smaller of m and d), 1 = d x d complement C (Section 6),
                            2 = m x m complement K = beta I + B D^{-1} B^T (same preconditioner),
                            3 = auto with a linear block (sdp_set_linear_diag): the m-space when
                            fewer than d rows have tau^-2 delta_i <= 1e8 beta (rows the other
                            slacks fix), else the d-space; without one, as 0.  3 reserves room
                            for both complements (not for the DIAG kind) */
  int32_t max_pcg;       /* iteration cap                                                       */
  int32_t check_every;   /* PCG iterations between host reads of the stop flag (>= 1)            */
  int32_t beta_rule;     /* 0: beta = median(eig E)^2 * ||A||_F^2/m;  1: median(eig E)^2 (Section 7 as printed) */
  int32_t use_graph;     /* 1: run the PCG iterations as replays of a captured CUDA graph of
                            check_every iterations (captured on a private stream, launched on
                            the handle's stream); 0: plain launches                            */
  double newton_rtol;    /* stop when ||r_k|| <= newton_rtol * ||[svec C~; b~]||; with the second
                            block of r_k at rounding level, ||r_k|| is the (Newt-eps) residual of
                            the recovered direction (Lemma smallres).  The mixed form applies the
                            same test to the FP64 residual g - M x                               */
  int32_t max_refine;    /* mixed form: refinement steps at most                                 */
  int32_t max_inner;     /* mixed form: PCG iterations per correction solve at most               */
  double inner_rtol;     /* mixed form: each correction solve stops at ||r|| <= inner_rtol ||r_0|| */
  int32_t pcg_start;     /* start of the FP64 PCG (both satisfy Cor. pcg: the second block of the
                            residual is zero):  0 = x0 = P^{-1}[0; g_v] (the preconditioner applied
                            to the second block of g), which keeps ||r_0|| of the size of ||g||;
                            1 = x0 = [0; -Sigma^{-1} Q^T c] as printed in Cor. pcg, whose first
                            block of r_0 grows like 1/mu^2 and sets a floor for the attainable
                            residual near the end of the interior-point path                     */
  int32_t tc_products;   /* 1 (default): the large dense FP64 products of a Newton solve (n >= 512:
                            E = Vs diag(e) Vs^T, E C~, the recovery, the complements B^T B and
                            B D^{-1} B^T) run on the BF16 tensor cores by exact slices (see
                            sdp_gemm_f64_tc; FP64 accuracy); 0: every product on the FP64 MMA
                            path.  The Cholesky and inverse of the complement stay FP64 MMA.     */
  int32_t krylov;        /* 0 (default): indefinite PCG with the Section 6 preconditioner
                            (Cor. pcg); 1: MINRES on eq. augsys with P = I from x0 = 0
                            (Cor. minres): no B = A Q and no Schur complement are formed, so the
                            workspace is O(n^2 + m + d) (the fallback when neither C nor K
                            fits), at the price of many more iterations (the condition number
                            of eq. augsys, not of the preconditioned operator); max_pcg bounds
                            its iterations and the stop test is the PCG one.  FP64 only
                            (a mixed form with krylov = 1: SDP_EUNSUPPORTED).               */
  int32_t int_passes;    /* DENSE_SVEC kind, FP64 operator (the FP64 form, and the FP64 residuals
                            of the mixed form): 1 (default) = the two passes over the svec rows,
                            A(Z) and A^T(y), stream an integer copy of A made at setup (two int32
                            digits per entry with a power-of-two scale per row, 8 bytes per
                            entry) and sum exact int64 digit products, whose error is within the
                            FP64 dot-product bound measured against the largest entry of the row
                            and of the vector; GB300's integer pipe keeps up with HBM where its
                            FP64 pipe does not.  The products E Y E of the operator (n < 512) are
                            summed the same way.  0 = FP64 FMAs over the caller's A (no copy)
                            and FP64 MMA products.                                              */
} sdp_options;

typedef struct {
  int32_t r;             /* rank parameter used                                                 */
  int32_t d;             /* n r - r(r-1)/2                                                      */
  int32_t pcg_iters;     /* PCG iterations performed (mixed form: of all correction solves)      */
  int32_t space;         /* 1 = d-space, 2 = m-space                                            */
  int32_t converged;     /* 1 if the stopping test held                                         */
  int32_t refine_steps;  /* mixed form: correction solves performed (0 in the plain form)        */
  double tau;            /* lambda_{r+1}(W)/2 (eq. EQSigdef)                                     */
  double beta;           /* preconditioner scale (Cor. pcg)                                      */
  double res_norm;       /* ||r_k|| at exit (plain: the PCG recurrence; mixed: the FP64 residual) */
  double rhs_norm;       /* ||[svec C~; b~]|| (right side of (Newt-eps))                          */
  double res0_norm;      /* ||r_0|| (mixed form: ||g||, the residual at x = 0)                   */
  double s_A;            /* ||A||_F^2 / m                                                       */
  double setup_ms;       /* device time of the split and the preconditioner setup (a1, a2)       */
  double pcg_ms;         /* device time from the right-hand side to the PCG stop (a3 - a6)       */
  double recover_ms;     /* device time of the recovery (a8)                                     */
  double prof_At_ms;     /* with profiling on: summed time of the A^T(y) passes over the dense A */
  double prof_A_ms;      /* with profiling on: summed time of the A(X) passes over the dense A   */
  int32_t prof_At_launches;  /* number of those A^T passes that did work                        */
  int32_t prof_A_launches;   /* number of those A passes that did work                          */
  double prof_At32_ms;   /* the same for the FP32 passes of the mixed form                       */
  double prof_A32_ms;
  int32_t prof_At32_launches;
  int32_t prof_A32_launches;
  double refine_rate;    /* mixed forms: (||rho_k|| / ||g||)^(1/k) after k corrections, the mean
                            contraction of the FP64 residual per correction solve -- the error of
                            the low-precision correction operator as the refinement sees it
                            (0 in the plain form)                                            */
} sdp_newton_info;

/* One outer interior-point iteration (ipm_step) or a whole solve (sdp_solve). */
typedef struct {
  int32_t iters;         /* outer iterations performed (sdp_solve) / 1 (ipm_step)                */
  int32_t converged;     /* 1 if rel_gap, pinf and dinf are all <= gap_tol at exit               */
  int32_t pcg_iters;     /* PCG iterations of all Newton solves                                  */
  int32_t eig_sweeps;    /* Jacobi sweeps of all eigen-decompositions                            */
  int32_t newton_inexact;/* Newton solves that stopped at max_pcg before the stopping test but whose
                            (Newt-eps) residual was below 0.1 gap_tol of the right side (their
                            directions are used as they are; a direction above that bound ends the
                            loop with SDP_ENOTCONV and the last iterate)                         */
  int32_t pad_;
  double pobj;           /* <C, X>                                                              */
  double dobj;           /* b^T y                                                               */
  double rel_gap;        /* |pobj - dobj| / (1 + |pobj| + |dobj|)                               */
  double pinf;           /* ||b - A(X)|| / (1 + ||b||)                                          */
  double dinf;           /* ||C - A^T(y) - S||_F / (1 + ||C||_F)                                */
  double mu;             /* <X, S> / n                                                          */
  double alpha_p;        /* last primal step length                                             */
  double alpha_d;        /* last dual step length                                               */
  double sigma;          /* last centring parameter                                             */
  double newton_ms;      /* device time in Newton solves                                        */
  double total_ms;       /* wall time of the call                                               */
} sdp_ipm_info;

/* Symmetric eigen-decomposition on the device by the parallel cyclic Jacobi method (FP64),
 * used by the outer loop: A = V diag(lam) V^T.  A (n x n, symmetric, column-major) is
 * destroyed; V (n x n), lam (n, in no particular order) are outputs.  Stops when the
 * off-diagonal Frobenius norm is <= tol times the Frobenius norm, or after max_sweeps sweeps
 * (then SDP_ENOTCONV).  work: device scratch of sdp_eigh_work_elems(n) doubles.  All on
 * `stream`, synchronous (one host read per sweep).  *sweeps (host, may be NULL) receives the
 * sweep count.  Not in the paper: its outer loop is an existing solver's (Section 7). */
int64_t sdp_eigh_work_elems(int32_t n);
sdp_status sdp_eigh(void* stream, int32_t n, double* A, double* V, double* lam, double tol, int32_t max_sweeps,
                    double* work, int64_t work_elems, int32_t* sweeps);

/* One iteration of the outer primal-dual interior-point method on the problem of the handle
 * with data (b, C): (X, y, S) -> (X + a_p dX, y + a_d dy, S + a_d dS) in place.  The method
 * (Section 7 keeps an existing solver's outer loop and does not describe it) is the textbook
 * infeasible NT path-following Mehrotra predictor-corrector also written in the oracle:
 *   W = L (L^T S L)^{-1/2} L^T with X = L L^T (eq. newt), G = L U Gamma^{-1/4} from
 *   L^T S L = U Gamma U^T (so W = G G^T and G^{-1} X G^{-T} = Gamma^{1/2} is diagonal);
 *   predictor: (Newt-eps) with b~ = b - A(X), C~ = R_d + S (R_c = -X), R_d = C - A^T(y) - S;
 *   sigma = (mu_aff / mu)^3; corrector: R_c = G R G^T with Lam R + R Lam =
 *   2 sigma mu I - 2 Lam^2 - (Dx Ds + Ds Dx), C~ = R_d - G^{-T} R G^{-1};
 *   steps: a = min(1, 0.98 * max{a : X + a dX PSD}) by the smallest eigenvalue of the scaled
 *   step, dS = R_d - A^T(dy).
 * Every Newton direction is one sdp_newton_solve on the reformulation (eig(W) by sdp_eigh).
 * b (m), C (n x n symmetric), X, S (n x n, positive definite), y (m): device pointers.
 * The first call allocates the loop's workspace (about 24 n^2 doubles). */
sdp_status ipm_step(sdp_handle* h, const double* b, const double* C, double* X, double* y, double* S,
                    sdp_ipm_info* info);

/* Whole solve from X = S = xi I, y = 0 (xi = max(10, sqrt n, max_i (1+|b_i|)/(1+||A_i||_F),
 * (1+||C||_F)/sqrt n)) until rel_gap, pinf and dinf are <= gap_tol (SDP_OK) or max_iter
 * iterations (SDP_ENOTCONV).  X, y, S: device outputs.  A Newton solve that reaches max_pcg
 * with a (Newt-eps) residual above 0.1 gap_tol times its right side also ends the loop with
 * SDP_ENOTCONV: no step is taken on that direction, X, y, S hold the last iterate and info the
 * measures of that iterate (ipm_step applies the same rule with gap_tol = 1e-8). */
sdp_status sdp_solve(sdp_handle* h, const double* b, const double* C, double* X, double* y, double* S,
                     double gap_tol, int32_t max_iter, sdp_ipm_info* info);

/* Linear block of the Newton system: nonnegative variables x >= 0 entering the constraints as
 * A(X) + G x = b, as in the robust problems of Section 7 (eq. rmc-sdp: x = [v; w], G = [I, -I]).
 * With D = diag(x / z) (NT scaling of the orthant), eliminating dx adds G D G^T to the Schur
 * matrix: the solve becomes (A (W (x)s W) A^T + diag(delta)) dy = b~ + A(W C~ W) with
 * delta = diag(G D G^T) (each variable in one constraint, so G D G^T is diagonal; for eq. rmc-sdp
 * delta = d_v + d_w).  In eq. augsys this is tau^-2 diag(delta) added to the (1,1) block, and the
 * Section 6 preconditioner takes Lam = beta I + tau^-2 diag(delta) in place of beta I (d-space:
 * C = tau^2 Sigma + B^T Lam^{-1} B; m-space: K = Lam + B (tau^2 Sigma)^{-1} B^T).  The caller
 * folds the linear block's right side into b~ (b~ + G D c~) and forms dx = D(G^T dy - c~).
 * delta: device pointer to m values >= 0, owned by the caller and read by every later Newton solve
 * of the handle, or NULL to remove the block.  DENSE_SVEC and SPARSE_COO kinds, FP64 form and
 * PCG only (otherwise SDP_EUNSUPPORTED); the setup of the next solve is redone (no resolve
 * before it).  While a block is set, sdp_solve, ipm_step, sdp_solve_batch and sdp_grad (which
 * have no nonnegative variables) return SDP_EUNSUPPORTED.
 * SDP_ENOMEM if the workspace of the block (m + m d_max doubles) cannot be allocated. */
sdp_status sdp_set_linear_diag(sdp_handle* h, const double* delta);

/* Whole solve of the robust form with slacks (Section 7, eq. rmc-sdp):
 *   min <C, X> + cv^T v + cw^T w   s.t.   A(X) + v - w = b,   X PSD,   v, w >= 0
 * (dual: max b^T y with C - A^T(y) = S PSD, zv = cv - y >= 0, zw = cw + y >= 0).  The method of
 * sdp_solve with the orthant added: mu = (<X, S> + v^T zv + w^T zw) / (n + 2 m), the Newton
 * directions with the linear block delta = v/zv + w/zw (sdp_set_linear_diag, set and removed by
 * this call), the ratio test for v, w (primal) and zv, zw (dual), and the stop test of sdp_solve
 * with the slack terms in the objective and in the dual residual.  Start X = S = xi I, y = 0,
 * v = w = zv = zw = xi.  cv, cw: device inputs (m, > 0); X, y, S, v, w, zv, zw: device outputs.
 * DENSE_SVEC and SPARSE_COO kinds, FP64 form, PCG (as sdp_set_linear_diag; otherwise
 * SDP_EUNSUPPORTED before any output is written).  SDP_EINVAL for a NULL handle or array, a
 * gap_tol <= 0 or max_iter < 0, SDP_EUNSUPPORTED while the caller has a linear block set,
 * SDP_ENOTCONV after max_iter iterations or on an unconverged Newton direction as in sdp_solve
 * (outputs hold the last iterate), SDP_ENOMEM if the 14 m
 * doubles of the slack workspace cannot be allocated. */
sdp_status sdp_solve_slack(sdp_handle* h, const double* b, const double* C, const double* cv, const double* cw,
                           double* X, double* y, double* S, double* v, double* w, double* zv, double* zw,
                           double gap_tol, int32_t max_iter, sdp_ipm_info* info);

/* Centring at a fixed mu: Newton steps towards the central-path point of parameter mu
 * (A(X) = b, A^T(y) + S = C, X S = mu I), each the NT direction (Section 3, (Newt-eps) through
 * the reformulated solve) of R_c = mu S^{-1} - X, i.e. Lam R + R Lam = 2 mu I - 2 Lam^2 in the
 * scaled frame of ipm_step, with one step length for X, y and S: min(1, 0.95 * 0.95 max step).
 * Stops (SDP_OK) when ||Lam^2 - mu I||_F / mu, pinf and dinf are all <= tol, or after max_iter
 * steps (SDP_ENOTCONV).  The paper has no counterpart: the derivative of the optimum (sdp_grad)
 * is that of the central-path point of its scaling point, which equals the derivative of the
 * optimum up to O(mu) only at a centred iterate, so a final iterate of sdp_solve is centred at
 * its own mu before it is differentiated.  X, y, S: device, in place (X, S positive definite);
 * b, C as for sdp_solve; info (may be NULL): iters, measures, and the final centrality in
 * info->sigma.  SDP_EINVAL for mu <= 0, tol <= 0 or max_iter < 0; the other codes as
 * ipm_step.  The interior-point workspace is allocated on first use. */
sdp_status sdp_center(sdp_handle* h, const double* b, const double* C, double* X, double* y, double* S, double mu,
                      double tol, int32_t max_iter, sdp_ipm_info* info);

/* The NT scaling point of an iterate (eq. newt), as the Newton solve and the adjoint take it:
 * W = L (L^T S L)^{-1/2} L^T with X = L L^T, computed as G G^T with G = L U Gamma^{-1/4}
 * (L^T S L = U Gamma U^T), and its eigen-decomposition W = V diag(lam) V^T (Jacobi, FP64; both
 * eigen-decompositions start from the handle's previous ones, e.g. those of the last
 * interior-point iteration, when there are any).  X, S: n x n positive definite (device);
 * V: out n x n, lam: out n (device, any order).  The interior-point workspace is allocated on
 * first use.  SDP_ENUMERIC when X is not positive definite or L^T S L is singular.  With
 * sdp_grad this gives the derivative of the optimum at the final iterate of sdp_solve. */
sdp_status sdp_scaling_point(sdp_handle* h, const double* X, const double* S, double* V, double* lam);

/* Many independent solves at once (batched SDPs of uneven size): sdp_solve of instance i on
 * hs[i] with (b[i], C[i]) into (X[i], y[i], S[i]), for i < count.  `workers` host threads
 * (<= 0: min(count, 16)) take the instances largest first; each solve runs on its own
 * handle's stream, so give every handle its own (non-blocking) stream for the solves to
 * overlap on the GPU: the small instances of a batch do not fill the GPU one at a time.
 * While batched, the eigensolver and the smallest-eigenvalue search take their
 * non-cooperative paths (no grid-wide barrier waits on blocks that share the GPU with other
 * solves); results agree with single solves to the solve tolerance, not bitwise.
 * Each workspace of the interior-point loop is allocated before the workers start.
 *   hs       count distinct handles (a handle must not appear twice: its workspace is shared)
 *   b, C, X, y, S   count device pointers each, as for sdp_solve
 *   infos    count host structs (may be NULL);  statuses  count host status codes (required)
 * Returns SDP_OK when every instance returned SDP_OK, else the status of the first failing
 * instance (by index); SDP_EINVAL for bad arguments (nothing is solved). */
sdp_status sdp_solve_batch(int32_t count, sdp_handle* const* hs, const double* const* b, const double* const* C,
                           double* const* X, double* const* y, double* const* S, double gap_tol, int32_t max_iter,
                           int32_t workers, sdp_ipm_info* infos, int32_t* statuses);

/* Fill *opt with the defaults: r_fixed 0, r_hat 10, FP64, auto space,
 * max_pcg 2000, check_every 8, beta_rule 0, use_graph 1, newton_rtol 1e-12, max_refine 10,
 * max_inner 500, inner_rtol 1e-6, pcg_start 0, tc_products 1, krylov 0, int_passes 1. */
void sdp_default_options(sdp_options* opt);

/* Validate the problem, record its (device) pointers -- the caller keeps
 * them alive for the handle's lifetime -- compute s_A = ||A||_F^2/m and
 * allocate all workspace for ranks up to r_fixed (or r_hat).
 * `stream` is a cudaStream_t (NULL = legacy default stream). */
sdp_status sdp_setup(const sdp_problem* prob, const sdp_options* opt, void* stream,
                     sdp_handle** out);

/* One Newton solve (Section 3 (Newt-eps) through eq. augsys + eq. recover).
 *   V    n x n column-major, orthonormal eigenvectors of W (any order)
 *   lam  n eigenvalues of W, all > 0, paired with the columns of V
 *   Ct   n x n symmetric residual C~;   bt  m residual b~
 *   dX   out n x n;  dy  out m;  dS  out n x n (= C~ - A^T(dy))
 *   info out (host pointer, may be NULL)
 * All array arguments are device pointers.  Returns SDP_ENOTCONV if the
 * stopping test did not hold within max_pcg iterations (outputs are still
 * written from the last iterate). */
sdp_status sdp_newton_solve(sdp_handle* h, const double* V, const double* lam,
                            const double* Ct, const double* bt,
                            double* dX, double* dy, double* dS, sdp_newton_info* info);

/* Another right side (C~, b~) at the scaling point of the most recent sdp_newton_solve on this
 * handle: the split and the preconditioner core (a1, a2: E, Sigma, B = A Q and the inverse of
 * the Schur complement) are reused, so only the right side, the PCG and the recovery run.
 * The interior-point corrector uses it (two right sides per scaling point).  SDP_EINVAL when
 * the handle has no usable previous solve (none yet, or its factorisation failed). */
sdp_status sdp_newton_resolve(sdp_handle* h, const double* Ct, const double* bt, double* dX, double* dy, double* dS,
                              sdp_newton_info* info);

/* One application of the augmented operator or of the preconditioner at the scaling point of the
 * most recent sdp_newton_solve on this handle (its split and preconditioner core): which = 0:
 * out = M pin with M = [[A E A^T, A Q], [Q^T A^T, -tau^2 Sigma]] (eq. augsys; the operator the
 * PCG applies, plus tau^-2 diag(delta) in its (1,1) block with a linear block set); which = 1:
 * out = P^{-1} pin, the block preconditioner of Section 6 in the handle's space (d- or m-space,
 * sdp_newton_info.space).  pin, out: device vectors of m + d doubles, [u; v] with v in the
 * h-coordinates [svec B; vec N] of range(Q) (d = sdp_newton_info.d of that solve); they may not
 * overlap.  FP64 in every precision form.  Asynchronous: the work is enqueued on the handle's
 * stream and the call returns without waiting (synchronize that stream, or order later work on
 * it, before reading out).  SDP_EINVAL for a NULL argument, a `which` other than 0 or 1, or a handle without a
 * usable previous solve; SDP_EUNSUPPORTED for which = 1 on a MINRES handle (no preconditioner).
 * This is the operator-only and preconditioner-only entry of the bench and of the parity tests
 * that compare each against the oracle's plain definition. */
sdp_status sdp_apply_augsys(sdp_handle* h, const double* pin, double* out, int32_t which);

/* Same as sdp_newton_solve with every array argument a HOST pointer
 * (pinned memory gives asynchronous copies); the copies to and from the
 * device are part of the call. */
sdp_status sdp_newton_solve_host(sdp_handle* h, const double* V, const double* lam,
                                 const double* Ct, const double* bt,
                                 double* dX, double* dy, double* dS, sdp_newton_info* info);

/* Vector-Jacobian product of the SDP optimum with respect to the data (C, b), by implicit
 * differentiation at the final iterate.  The linearised optimality conditions of Section 3,
 *   A(dX) = db,  A^T(dy) + dS = dC,  dX + W dS W = 0,
 * have the symmetric KKT matrix K of (Newt-eps), so the cotangents of the data are
 * [gC; gb] = K^{-1} [sym gX; gy]: one Newton solve on the reformulated operator and its
 * preconditioner with (C~, b~) = (sym gX, gy), gC = dX, gb = dy.  This is the derivative of
 * the central-path point at the scaling point W = V diag(lam) V^T; for W the NT scaling of a
 * well-centred iterate near the optimum it differs from the derivative of the optimum by
 * O(mu).  The paper states no such product; it reuses its Newton system.
 *   V, lam  eigen-decomposition of W (as for sdp_newton_solve)
 *   gX      n x n cotangent of X (its symmetric part is used);  gy  m cotangent of y
 *   gC      out n x n (symmetric);  gb  out m;  info as for sdp_newton_solve
 * All arrays are device pointers.  Same status codes as sdp_newton_solve. */
sdp_status sdp_grad(sdp_handle* h, const double* V, const double* lam, const double* gX, const double* gy,
                    double* gC, double* gb, sdp_newton_info* info);

/* Vector-Jacobian product of the optimum of the robust form with slacks (Section 7, eq. rmc-sdp:
 * min <C, X> + cv^T v + cw^T w  s.t.  A(X) + v - w = b, X PSD, v, w >= 0) with respect to its
 * data (C, b, cv, cw), at the scaling point of a final iterate: W = V diag(lam) V^T for (X, S) and
 * D = diag(d_v, d_w) with d_v = v / zv, d_w = w / zw for the orthant.  The linearised optimality
 * conditions have the symmetric KKT matrix of (Newt-eps) with the linear block, so the cotangents
 * of the data are one Newton solve with (C~, c~, b~) = (sym gX, (g_v, g_w), g_y): the linear
 * block delta = d_v + d_w is set for the solve, b~ = g_y + d_v g_v - d_w g_w, and then
 *   gC = dX,  gb = dy,  (gcv, gcw) = D (G^T dy - c~) = (d_v (dy - g_v), d_w (-dy - g_w)).
 * The paper has no such product; it reuses its Newton system.  V, lam as for sdp_newton_solve;
 * dv, dw, gy, gv, gw, gb, gcv, gcw: m (device); gX, gC: n x n (device).  DENSE_SVEC and SPARSE_COO
 * kinds, FP64 form, PCG (as sdp_set_linear_diag); SDP_EUNSUPPORTED while the caller has a linear
 * block set (it is set and removed by this call).  Same status codes as sdp_newton_solve. */
sdp_status sdp_grad_slack(sdp_handle* h, const double* V, const double* lam, const double* dv, const double* dw,
                          const double* gX, const double* gy, const double* gv, const double* gw, double* gC,
                          double* gb, double* gcv, double* gcw, sdp_newton_info* info);

/* Diagnostics: copy `count` doubles of an internal buffer of the most recent solve into the
 * device array `dst` (stream-ordered, synchronous).  which: 0 = E (n x n), 1 = D = tau^2 Sigma
 * (d), 2 = B = A Q (m x d, row-major), 3 = inverse of the preconditioner's Schur complement
 * (d x d or m x m), 4 = eigenvectors sorted by descending eigenvalue (n x n), 5 = the PCG
 * iterate [u; v] (m + d), 6 = the right side g of eq. augsys (m + d), 7 = the raw device
 * control block of the PCG loop (its size in doubles), 8..11 = the PCG vectors r, z, p and
 * A p (m + d each), 12 = the control block of the correction solve of the mixed form.  SDP_EINVAL if
 * `count` exceeds the buffer. */
sdp_status sdp_debug_copy(sdp_handle* h, int32_t which, double* dst, int64_t count);

/* Turn on (1) or off (0) CUDA-event timing of every pass over the dense constraint matrix
 * (reported in sdp_newton_info.prof_*).  Creates its events on first use. */
sdp_status sdp_set_profiling(sdp_handle* h, int32_t on);

/* Y = A^T(y) = sum_i y_i A_i (n x n, full, column-major) for the dense svec storage of A
 * (m x n(n+1)/2 row-major, as SDP_A_DENSE_SVEC), without allocating any device memory.
 * The paper has no counterpart: this entry point exists for callers that cannot call
 * cudaMalloc (code inside an allocator or memory-pool callback, a process whose device
 * memory another framework has reserved in full, a path that must not fail with an
 * out-of-memory error once started).  The caller passes the device arrays a_dense, y (m)
 * and Y (n x n); the only scratch, the row-group partial sums of A^T(y), lives in a fixed
 * 4 MiB array in the library's device data, held by every GPU that loads the library
 * until the process exits.  Limit: n(n+1)/2 <= 524288 (n <= 1023), else SDP_EINVAL.
 * Other errors: SDP_EINVAL for NULL arrays or n, m < 1; SDP_ECUDA if a CUDA call fails.
 * Every call looks up the array's device address (cudaGetSymbolAddress) for the device
 * current at the call, so it stays right after a context reset; the first call on a device
 * loads the library's device code there, so make that first call before any stream capture.  All calls
 * share the array, so calls that overlap on the GPU race; every value read is written
 * earlier in the same call, so nothing needs clearing between calls.  `stream` is a
 * cudaStream_t; the call returns after its work on that stream has completed. */
sdp_status sdp_adjoint_dense_noalloc(const double* a_dense, int32_t n, int32_t m, const double* y,
                                     double* Y, void* stream);

/* Double-precision matrix product on the BF16 tensor cores (tcgen05 with TMEM accumulators,
 * TMA-fed), C = alpha op(A) op(B) + beta C, column-major like BLAS dgemm (op = transpose when
 * tA / tB is nonzero; op(A) M x K, op(B) K x N).  The paper has no counterpart: its dense
 * products are FP64 (the n^3 products of Section 3 and the Schur complements of Section 6), and
 * the GPU's tensor cores have no FP64 kind.  The operands are split into eight exact BF16
 * integer slices per row of op(A) and column of op(B) (scaled by a power of two), the 36 slice
 * products that matter are accumulated exactly in FP32 over K-chunks of 4096 and summed in FP64:
 * the error is about K 2^-55 max_k|op(A)[i,k]| max_k|op(B)[k,j]| per entry, the FP64 bound when
 * rows and columns carry no large internal dynamic range.
 *   work   device scratch of sdp_gemm_f64_tc_work_bytes(M, N, K) bytes, 256-byte aligned
 *          (about 32 (M + N) K bytes: the slices)
 * All matrices are device pointers; `stream` is a cudaStream_t; the call returns after its work
 * on that stream has completed.  SDP_EINVAL for bad sizes, leading dimensions or work;
 * SDP_EUNSUPPORTED on a device that is not a Blackwell (sm_10x) GPU; SDP_ETIMEOUT if a bounded
 * wait inside the kernel gave up (about 2 s; the output is then not written). */
size_t sdp_gemm_f64_tc_work_bytes(int32_t M, int32_t N, int32_t K);
sdp_status sdp_gemm_f64_tc(void* stream, int32_t tA, int32_t tB, int32_t M, int32_t N, int32_t K, double alpha,
                           const double* A, int64_t lda, const double* B, int64_t ldb, double beta, double* C,
                           int64_t ldc, void* work, size_t work_bytes);

/* Inverse or Cholesky factor of a symmetric positive definite matrix, as the Newton solve forms
 * its preconditioner core (Section 6: C = tau^2 Sigma + beta^{-1} B^T B in the d-space, or the
 * m-space K, is inverted once per Newton solve so that every PCG application is one product).
 *   A      n x n, column-major, device; only the lower triangle is read.
 *          mode 0: overwritten with A^{-1} (both triangles);
 *          mode 1: overwritten with the Cholesky factor L (A = L L^T, lower, upper zeroed).
 *   Linv   mode 1 only, NULL or n x n device: L^{-1} (lower, upper zeroed).
 *   coop   1: for n <= 1024, one cooperative launch over the whole GPU (blocked right-looking
 *          Cholesky, L^{-1} by block forward substitution and L^{-T} L^{-1}, advanced together
 *          in 32-wide block steps); 0, larger n, or a device without cooperative launches: the
 *          chain of one-CTA diagonal-block factorisations and FP64 products.
 *   work   device scratch of sdp_spd_inverse_work_bytes(n) bytes, 256-byte aligned.
 * FP64 throughout.  Returns after the work on `stream` has completed; SDP_ENUMERIC when a pivot
 * is not positive and finite (A is not SPD to working precision; the output is then not
 * meaningful), SDP_EINVAL for bad arguments. */
size_t sdp_spd_inverse_work_bytes(int32_t n);
sdp_status sdp_spd_inverse(void* stream, int32_t n, double* A, double* Linv, int32_t mode, int32_t coop, void* work,
                           size_t work_bytes);

/* Limit in nanoseconds of every wait of the main loop of the tensor-core product (the TMA
 * copies, the products and the drain of an accumulator, each an mbarrier wait bounded by
 * %globaltimer), process-wide, for the products launched after the call; 0 restores the
 * default of 2 s.  When a wait runs out the kernel records an error word, stops issuing
 * copies and products, waits with the full 2 s bound for the ones already in flight, frees its
 * TMEM and returns; the call then returns SDP_ETIMEOUT with its output not written, and the
 * stream and the context stay usable.  The paper has no counterpart: this is the control that
 * lets a test make a bounded wait run out without faulting or hanging a GPU. */
void sdp_set_tc_wait_limit_ns(uint64_t ns);

/* Low-precision matrix product on the tensor cores, as the TF32 and BF16 forms run it (tcgen05 with
 * FP32 accumulators in TMEM, operands staged by TMA): C = alpha A_s^T B_s for A_s (K x M) and B_s
 * (K x N) column-major with leading dimensions lda, ldb, i.e. the rows of op(A) and the columns of
 * op(B) K-contiguous.  tf32 = 1: A_s, B_s are FP32 and read as TF32 (kind::tf32); tf32 = 0: they are
 * BF16 (kind::f16).  C: FP32, M x N column-major, ldc >= M.  Each product of two operands is exact
 * in the FP32 accumulator; the sums are FP32.  The paper has no counterpart (its products are
 * FP64); this entry point exposes the mixed forms' product for tests.  err_word: a device int32
 * (the bounded-wait error word, cleared by the call).  lda, ldb >= K with 16-byte rows, A and B
 * 16-byte aligned, M, N, K >= 1, else SDP_EINVAL; SDP_EUNSUPPORTED on a GPU that is not sm_10x;
 * SDP_ETIMEOUT as sdp_gemm_f64_tc.  Returns after the work on `stream` has completed. */
sdp_status sdp_gemm_tn_lp(void* stream, int32_t tf32, int32_t M, int32_t N, int32_t K, float alpha, const void* A,
                          int64_t lda, const void* B, int64_t ldb, float* C, int64_t ldc, int32_t* err_word);

/* Bounds report of the checked debug build (libwcipm_checked.so: the sparse-operator kernels of
 * section 4.2's A(.) and A^T(.) for SDP_A_SPARSE_COO compiled with -DSDP_CHECK_BOUNDS).  There,
 * every index that a gather or a scatter takes from an index table (the entries of a constraint,
 * the entries and row/column of a matrix position, the CSR pattern of A^T(y)) is compared with
 * the length of the array it addresses before it is used; an index out of range is skipped (the
 * access is not made) and recorded in device memory.  The call synchronizes the device, reads and
 * clears the records, and writes to *first the first violation kept (site << 48 | index mod 2^48,
 * site >= 1 naming the check; 0 when none) and to *count the number seen since the last call.
 * Returns SDP_OK when none was seen, SDP_EINVAL when one was (or first or count is NULL),
 * SDP_ECUDA when reading the records failed, and SDP_EUNSUPPORTED in the default build, which
 * has no checks (*first = *count = 0).  Not safe to call while another thread launches work. */
sdp_status sdp_bounds_report(uint64_t* first, uint64_t* count);

/* One bounds check of `index` against [0, bound) by the checked build's sparse translation unit,
 * with no access behind it: an index outside the range is recorded as a violation (reported by
 * the next sdp_bounds_report), one inside it is not.  The paper has no counterpart; this lets a
 * test see the record and the report work without an out-of-range index reaching an access.
 * Returns after the check on `stream` has completed; SDP_EUNSUPPORTED in the default build,
 * SDP_EINVAL for bound < 0. */
sdp_status sdp_bounds_selftest(void* stream, int64_t index, int64_t bound);

/* Bytes of device workspace owned by the handle. */
size_t sdp_workspace_bytes(const sdp_handle* h);

/* Number of kernel launches issued by the most recent solve call. */
int64_t sdp_last_launch_count(const sdp_handle* h);

/* Message for the most recent failure on this handle (or of sdp_setup when h is NULL). */
const char* sdp_last_error(const sdp_handle* h);

/* Release the handle: waits for the work on its stream, then frees its device workspace, its
 * pinned control block, the outer loop's buffers, its captured graphs, events and side streams
 * (the stream passed to sdp_setup stays the caller's).  NULL is ignored;
 * the handle must not be used afterwards.  Device pointers the caller passed in stay the
 * caller's. */
void sdp_destroy(sdp_handle* h);

#ifdef __cplusplus
}
#endif

#endif /* WCIPM_H */

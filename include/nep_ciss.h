/*
 * nep_ciss.h -- C ABI of the GB300 contour-integral (CISS) solver for nonlinear
 * eigenvalue problems in split form.
 *
 * Problem (Sec. 2, Eqs. (nep) and (split)): find (lambda, x), x != 0, with
 *     T(lambda) x = 0,    T(z) = sum_{i<l} A_i f_i(z),
 * A_i constant sparse n x n matrices, f_i scalar holomorphic functions (Sec. 3.2.2
 * function classes: rational, exp, principal sqrt, with argument/result scaling and
 * combinations). The solver returns every eigenpair inside an ellipse Gamma.
 *
 * Conventions
 *   - Complex numbers are interleaved doubles (re, im); a "complex array of length k"
 *     is 2k doubles. Dense blocks are column-major.
 *   - Every call returns int: NEP_OK (0) or a negative NEP_ERR_*; nep_last_error()
 *     gives a message (thread-local, valid until the next failing call on the thread).
 *   - Inputs are copied at the call; callers keep ownership of their buffers. Objects
 *     returned through an out-pointer are owned by the library until the matching
 *     *_free/*_destroy call.
 *   - Entry points that take device pointers ("_dev") expect memory of the current
 *     CUDA device; "stream" is a cudaStream_t passed as void* (NULL = legacy default stream).
 *   - All arithmetic is complex. Host callbacks are not supported: every f_i must be a
 *     closed-form kind below, because the Rayleigh-Ritz/Newton step evaluates f_i and
 *     f_i' on the device.
 */
#ifndef NEP_CISS_H
#define NEP_CISS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ status */
#define NEP_OK 0
#define NEP_ERR_ARG (-1)         /* invalid argument (sizes, CSR structure, options)    */
#define NEP_ERR_CUDA (-2)        /* a CUDA runtime call failed                           */
#define NEP_ERR_REGION (-3)      /* the closed region meets a pole or a branch cut       */
#define NEP_ERR_NOMEM (-4)       /* device or host allocation failed                      */
#define NEP_ERR_UNSUPPORTED (-5) /* valid request outside what the library implements    */
#define NEP_ERR_INTERNAL (-6)    /* device-side check failed (bounded wait, bad index)   */

/* warning flags of a result (bitwise or) */
#define NEP_WARN_SATURATED 1     /* Hankel rank m == L*M: the probe subspace may be too small */
#define NEP_WARN_REFINE 2        /* some quadrature solve missed the backward-error target */
#define NEP_WARN_SINGULAR_NODE 4 /* an exactly zero pivot at some quadrature node         */
#define NEP_WARN_NEWTON 8        /* a Newton iteration on the projected problem failed (singular */
                                 /* bordered system or a non-finite iterate); candidates whose   */
                                 /* iterates left the region are counted in nep_result_info_t's  */
                                 /* newton_left and raise no warning                              */
#define NEP_WARN_INTERP 16       /* NLEIGS: the interpolation degree test failed at max_degree */

/* arithmetic of the quadrature solves */
#define NEP_PREC_FP64 0  /* complex128 factors and solves ("plain FP64")                  */
#define NEP_PREC_MIXED 1 /* complex64 factors and solves, FP64 residuals and refinement  */

/* ------------------------------------------------------------------ problem objects */
typedef struct nep_split *nep_split_t;
typedef struct nep_result *nep_result_t;
typedef struct nep_plan *nep_plan_t;

/* CSR matrix (0-based). Column indices of each row must be strictly increasing and in
 * [0, n_cols). val_im may be NULL for a real matrix. */
typedef struct {
    int32_t n_rows, n_cols;
    const int64_t *rowptr; /* n_rows + 1 entries */
    const int32_t *col;    /* rowptr[n_rows] entries */
    const double *val_re;
    const double *val_im;
} nep_csr;

/* Scalar function g(z) = beta * h(alpha * z) (FNSetScale of Sec. 3.2.2), h by kind:
 *   NEP_FN_RATIONAL  h(x) = p(x) / q(x); num/den are complex arrays, highest degree
 *                    first (nnum, nden coefficients); nden == 0 means q = 1.
 *   NEP_FN_EXP       h(x) = exp(x).
 *   NEP_FN_SQRT      h(x) = sqrt(x - shift), principal branch (cut on x - shift <= 0).
 *   NEP_FN_COMBINE   h = a + b, a * b, a / b or a(b(.)) (op), a and b nested nep_fn.
 *   NEP_FN_CALLBACK  g is the user's host function eval (the callback form of Sec. 3.2.1): eval(z, count,
 *                    f, df, ctx) writes g(z_k) to f and g'(z_k) to df (complex arrays of count entries,
 *                    interleaved re, im; df may be NULL, then only f is wanted). alpha, beta are not
 *                    applied. The library copies eval and ctx and calls eval on the host only: at plan
 *                    creation for the quadrature nodes, and during the extraction step for the Newton
 *                    iterates and the returned eigenvalues (one call per term per Newton step, all
 *                    candidates at once); under the request server, from its worker threads (eval must
 *                    then be thread-safe). Device code never evaluates such a term: the projected
 *                    Newton steps run one per launch with the values passed in (slower than the
 *                    all-device path).
 *   NEP_FN_TABLE     g tabulated at the quadrature nodes of one solve: table holds table_count = N
 *                    complex values (interleaved), g(z_j) for the nodes z_j of nep_nodes(region, N)
 *                    in order; a solve with another N returns NEP_ERR_ARG. Values off the nodes (g and
 *                    g' at Newton iterates and eigenvalues) come from eval, which must then be given:
 *                    a table term without eval makes nep_plan_create / nep_ciss_solve return
 *                    NEP_ERR_UNSUPPORTED (the band assembly and solve entry points take coefficient
 *                    tables directly).
 * CALLBACK and TABLE terms appear only at the top level of a term (not inside COMBINE). Entry points
 * that evaluate the functions on the device elsewhere (nep_rii, nep_plan_polish, nep_left_eigvecs,
 * nep_plan_left, nep_nleigs_*) return NEP_ERR_UNSUPPORTED for a split with such terms. */
#define NEP_FN_RATIONAL 0
#define NEP_FN_EXP 1
#define NEP_FN_SQRT 2
#define NEP_FN_COMBINE 3
#define NEP_FN_CALLBACK 4
#define NEP_FN_TABLE 5
typedef void (*nep_fn_eval_t)(const double *z, int32_t count, double *f, double *df, void *ctx);
#define NEP_OP_ADD 0
#define NEP_OP_MUL 1
#define NEP_OP_DIV 2
#define NEP_OP_COMPOSE 3
typedef struct nep_fn {
    int32_t kind;
    double alpha_re, alpha_im, beta_re, beta_im;
    double shift_re, shift_im;
    int32_t nnum, nden;
    const double *num;
    const double *den;
    int32_t op;
    const struct nep_fn *a;
    const struct nep_fn *b;
    nep_fn_eval_t eval;      /* NEP_FN_CALLBACK, NEP_FN_TABLE (off the nodes); NULL otherwise */
    void *ctx;               /* passed to eval                                                */
    const double *table;     /* NEP_FN_TABLE: complex[table_count], copied at creation       */
    int32_t table_count;
} nep_fn;

/* Ellipse Gamma: z(t) = center + a cos t + i b sin t (a: real semi-axis, b: imaginary). */
typedef struct {
    double center_re, center_im, a, b;
} nep_region;

typedef struct {
    int32_t precision;   /* NEP_PREC_FP64 or NEP_PREC_MIXED                               */
    double rank_tol;     /* Hankel numerical rank: sigma_i > rank_tol * sigma_1 (1e-12)   */
    double basis_tol;    /* Rayleigh-Ritz basis rank, relative singular value (1e-6)     */
    double refine_tol;   /* per-solve normwise backward error target (1e-10)              */
    double step_tol;     /* relative refinement correction regarded as converged (1e-14) */
    int32_t refine_max;  /* maximum refinement sweeps (10)                                */
    double eig_tol;      /* scaled-residual acceptance of returned eigenpairs (1e-8)      */
    int32_t newton_max;  /* Newton steps on the projected problem (30)                    */
    double newton_tol;   /* |dlambda| <= newton_tol * max(1, |lambda|) (1e-14)            */
    uint64_t seed;       /* probe block V when none is passed                             */
    int32_t symmetric;   /* 1: solve only the nodes with Im z > 0 and take the others as   */
                         /* their complex conjugates (real-symmetric contour halving).    */
                         /* Needs a real operator (real A_i, f_i(conj z) = conj f_i(z) on */
                         /* the nodes), a region symmetric about the real axis (real      */
                         /* centre), an even N and a real V: plan creation returns        */
                         /* NEP_ERR_ARG otherwise (V is checked at execute). Then S_k =   */
                         /* 2 Re of the sum over those N/2 nodes. Default 0.              */
    int32_t newton_abandon;     /* shortcut: a Newton iterate still unconverged after this many  */
                                /* steps and outside Gamma by 10% (((Re(l-c))/a)^2 +             */
                                /* ((Im(l-c))/b)^2 > 1.21) is given up as having left the region */
                                /* (default 8; 0: never, iterate to newton_max)                   */
    int32_t refine_extrapolate; /* shortcut: a refinement sweep also stops when the contraction  */
                                /* seen so far puts the next correction below step_tol          */
                                /* (default 1; 0: stop only on step_tol or no halving)           */
    int32_t lu_kernel;  /* LU of complex64 bands with kl > 64: 0 the tuned or default choice, 1 tensor    */
                        /* core with TF32 hi/lo operands (3 products, ~FP32), 2 tensor core with TF32     */
                        /* operands (1 product), 3 FP32 SIMT kernel. Results of 1-3 differ by rounding.   */
                        /* For 32 <= kl <= 64, 1 and 2 select the tensor-core kernel in place of the      */
                        /* register-window one (the default, 0 or 3).                                      */
    int32_t solve_rh;   /* right-hand sides per warp of the narrow-band sweeps: 0 tuned or default, 1, 2, */
                        /* 4 (a launch shape only: results identical)                                     */
} nep_opts;

/* Defaults listed above. */
void nep_opts_default(nep_opts *o);

/* Builds the split operator T(z) = sum_i A_i f_i(z) (Sec. 3.2.2, NEPSetSplitOperator):
 * validates each CSR (square n x n, sorted in-range columns), forms the union sparsity
 * pattern with one value array per term, its bandwidths (kl, ku), ||A_i||_inf, and
 * copies everything to the current device. nterms >= 1; f has nterms entries.
 * Errors: NEP_ERR_ARG (bad sizes/CSR/function), NEP_ERR_CUDA, NEP_ERR_NOMEM. */
int nep_create_split(int32_t n, int32_t nterms, const nep_csr *A, const nep_fn *f, nep_split_t *out);
int nep_destroy(nep_split_t h);
/* Bandwidths and band leading dimension (ldab = 2 kl + ku + 1) of the union pattern. */
int nep_split_info(nep_split_t h, int32_t *n, int32_t *nterms, int32_t *kl, int32_t *ku, int32_t *ldab);

/* ------------------------------------------------------------------ whole solve */
/* Full contour-integral pass (all steps on the device): nodes and coefficients,
 * assembly, banded LU, solves refined to the backward-error target (residual in double-float
 * arithmetic with complex64 factors, in FP64 with complex128), moments, block-Hankel SVD and
 * reduced eigenproblem, Rayleigh-Ritz projection (Sec. 4.2 Eq. (narnoldi-split)) with
 * Newton steps (Sec. 4.1 Eq. (newton)), scaled residuals (Sec. 2 Eq. (sressplit)).
 * V_host: n x L complex probe block (column-major) or NULL (drawn from opts->seed).
 * N >= 2 quadrature points, 1 <= L <= n, M >= 1. Errors: NEP_ERR_ARG, NEP_ERR_REGION
 * (a rational pole or sqrt branch cut meets the closed region), NEP_ERR_CUDA,
 * NEP_ERR_NOMEM, NEP_ERR_INTERNAL. */
int nep_ciss_solve(nep_split_t h, const nep_region *r, int32_t N, int32_t L, int32_t M, const nep_opts *o,
                   const double *V_host, nep_result_t *out);

/* Results: nconv eigenpairs sorted by (Re, Im); lambda: complex[nconv]; X: n x nconv
 * complex, unit 2-norm columns, largest entry real positive; resid: eta per pair.
 * Pointers stay valid until nep_result_free. */
int nep_result_get(nep_result_t r, int32_t *nconv, const double **lambda, const double **X, const double **resid,
                   int32_t *hankel_rank, int32_t *flags);
/* Per quadrature point (the npts nodes solved: N, or N/2 under the conjugate-symmetric option, in
 * node order): refinement sweeps run, LU status (0, or 1 + the first column with an exactly zero
 * pivot: that node was dropped from the moments) and the last measured normwise backward error
 * (0 for a dropped node). Pointers (any may be NULL) stay valid until nep_result_free. Results of
 * NLEIGS carry no points (*npts = 0). */
int nep_result_points(nep_result_t r, int32_t *npts, const int32_t **sweeps, const int32_t **lu_info,
                      const double **backward);
typedef struct {
    int32_t n, N, L, M, precision;
    int32_t hankel_rank;    /* m */
    int32_t basis_rank;     /* Rayleigh-Ritz basis dimension */
    int32_t ncandidates;    /* Newton starts */
    int32_t max_sweeps;     /* refinement sweeps of the slowest point */
    int32_t svd_sweeps;     /* Jacobi sweeps of the Hankel SVD */
    int32_t flags;
    double max_backward;    /* max over points of the last measured backward error */
    double ms_assemble, ms_factor, ms_solve, ms_moments, ms_extract, ms_total;
    double ms_queued;       /* server requests: submit to start of execution (0 otherwise) */
    double ms_latency;      /* server requests: submit to result ready (0 otherwise) */
    int32_t newton_failed;  /* Newton runs that failed (these raise NEP_WARN_NEWTON)       */
    int32_t newton_left;    /* Newton runs whose iterate left the region (no warning)      */
    int32_t krylov_steps;   /* NLEIGS, Interpol: Arnoldi steps run, over all restart cycles */
    int32_t restarts;       /* NLEIGS, Interpol: Krylov-Schur restarts run                  */
} nep_result_info_t;
int nep_result_info(nep_result_t r, nep_result_info_t *info);
/* Singular values of the Hankel matrix (L*M of them, descending). */
int nep_result_hankel_sigma(nep_result_t r, const double **sigma, int32_t *count);
int nep_result_free(nep_result_t r);
const char *nep_last_error(void);
/* Number of CUDA kernels this library has launched in the process so far (diagnostics). */
uint64_t nep_kernel_launches(void);
/* Bound on every device-side wait of the library (the grid barriers of its cooperative kernels:
 * QR with column pivoting and the Jacobi SVD), in polls of the barrier word; process-wide, read
 * at each launch. Default 2^24 polls (seconds). A wait that reaches the bound records an error
 * and stops waiting, the kernel runs to its end without further waits (its loop bounds do not
 * depend on the data, so it stays in bounds) and the call returns NEP_ERR_INTERNAL with the
 * context usable. *previous (or NULL) receives the old bound. Errors: NEP_ERR_ARG (polls < 0). */
int nep_set_wait_limit(int64_t polls, int64_t *previous);

/* ------------------------------------------------------------------ device-resident plan */
/* A plan owns the device workspace of one (operator, region, N, L, M, opts) solve so
 * that repeated solves allocate nothing. nep_plan_execute reads V from device memory
 * (n x L complex128, column-major) and leaves all results on the device;
 * nep_plan_result copies them into a new result object. One plan serves one solve
 * at a time (calls on one plan must not overlap). */
int nep_plan_create(nep_split_t h, const nep_region *r, int32_t N, int32_t L, int32_t M, const nep_opts *o,
                    nep_plan_t *out);
int nep_plan_execute(nep_plan_t p, const void *V_dev, void *stream);
/* nep_plan_execute for several plans at once, with shared launches: the banded LU and the substitution
 * sweeps of all their quadrature points run in launches shared across the plans (one per kernel
 * instance: points of problems of uneven n, bandwidth, N and L share a launch when their band shapes
 * fall in the same class), the assembly, refinement residuals, moments and extraction per plan, in
 * plan order, all on one stream, with one host read of every plan's active count per refinement
 * sweep. Every point runs the kernel instance and arguments of its plan alone, so each plan's results
 * are bitwise those of nep_plan_execute. V_devs[i]: plan i's probe block (device memory). Plans of one
 * precision, each at most once, without callback or table terms.
 * Errors: NEP_ERR_ARG, NEP_ERR_UNSUPPORTED, and those of nep_plan_execute. */
int nep_plan_execute_batch(int32_t count, nep_plan_t *plans, const void *const *V_devs, void *stream);
int nep_plan_result(nep_plan_t p, nep_result_t *out);
int nep_plan_destroy(nep_plan_t p);
/* Device buffers of a plan (for inspection/tests): name in {"F","coef","ab","ut","ipiv","info",
 * "Y","S","mu","sigma","tnorm","beta","sweeps","H","newton_its","newton_ok","candidates",
 * "newton_lambda"}; returns the device pointer and its bytes ("ut" is empty for bands too wide
 * for the narrow-band sweeps). */
int nep_plan_buffer(nep_plan_t p, const char *name, void **dev_ptr, size_t *bytes);

/* ------------------------------------------------------------------ autotuning */
/* The implementation's own choices for a problem shape (the paper has no counterpart): nep_autotune
 * times full passes (nep_plan_execute; one warm-up, the mean of two, CUDA events on the stream) of
 * every candidate of opts->lu_kernel (complex64 bands with kl > 64: tensor core with TF32 hi/lo
 * operands, tensor core with TF32 operands, FP32 SIMT) times opts->solve_rh (1, 2, 4 for the narrow-band
 * sweeps), each on its own plan of this shape, and keeps the fastest candidate whose quadrature solves
 * all reach the backward-error target (no NEP_WARN_REFINE, max backward error <= refine_tol: accuracy
 * is part of the objective; a TF32-operand LU that refinement cannot repair is never chosen). The
 * choice goes into a process-wide table keyed by (n, kl, ku, L, precision), which later plans of that
 * shape use when their opts leave lu_kernel / solve_rh at 0, and, if cache_path is not NULL, is appended
 * to that text file (one line per tuned shape) for nep_tune_load. V_dev: the probe block (device).
 * Errors: NEP_ERR_ARG, NEP_ERR_UNSUPPORTED (callback or table terms), NEP_ERR_INTERNAL (no candidate
 * met the accuracy target), and those of nep_plan_create / nep_plan_execute. */
typedef struct {
    int32_t lu_kernel, solve_rh;  /* the choice (as nep_opts; 0: not applicable to this shape) */
    double ms;                    /* its device time per pass                              */
    int32_t candidates, accurate; /* candidates timed, and those meeting the accuracy target */
} nep_tune_result;
int nep_autotune(nep_split_t h, const nep_region *r, int32_t N, int32_t L, int32_t M, const nep_opts *o,
                 const void *V_dev, const char *cache_path, nep_tune_result *out, void *stream);
/* Loads a cache file written by nep_autotune into the process-wide table (later lines win);
 * *entries (or NULL) receives the number of lines read. Errors: NEP_ERR_ARG (no such file). */
int nep_tune_load(const char *path, int32_t *entries);

/* ------------------------------------------------------------------ residual inverse iteration */
/* Polish of eigenpair estimates by residual inverse iteration (Sec. 4.1, Algorithm (rii),
 * Neumaier's method), for P pairs at once. For pair p, sigma_p is its starting eigenvalue:
 * T(sigma_p) is assembled and factored once by the band LU (complex64 factors for
 * NEP_PREC_MIXED, complex128 for NEP_PREC_FP64). Each iteration solves T(sigma_p) with the FP64
 * residual T(lambda_k) x and the A_i x as right-hand sides, takes lambda from Newton's method on
 * x^* T(sigma_p)^{-1} T(z) x = 0 (written as x^* T(sigma_p)^{-1} (T(lambda_k) x + sum_i
 * (f_i(z) - f_i(lambda_k)) A_i x); stopped at |mu| < sqrt(eps) |lambda|), computes the FP64 scaled
 * residual eta (Sec. 2 Eq. (sressplit)) and stops the pair once eta < tol; otherwise
 * x <- x - T(sigma_p)^{-1} T(lambda) x, normalised.
 *   lam_dev: P complex128 (in: starting eigenvalues; out: results)
 *   X_dev:   n x P complex128, column-major (in: starting vectors; out: unit 2-norm, first entry
 *            of largest modulus real positive)
 *   eta_dev: P doubles (out); its_dev: P int32 vector updates per pair (out), or NULL
 * At most max_it + 1 iterations; *iterations (or NULL) receives the number run. All pointers are
 * the caller's device memory; the call allocates its work arrays (among them the factors of P
 * points) on the stream and returns when they are done.
 * Errors: NEP_ERR_ARG (P < 0, max_it < 0, NULL arrays with P > 0, unknown precision), CUDA errors. */
int nep_rii(nep_split_t h, int32_t precision, int32_t P, double *lam_dev, double *X_dev, double *eta_dev,
            int32_t *its_dev, double tol, int32_t max_it, int32_t *iterations, void *stream);
/* The same polish, in place, for the eigenpairs of the plan's last nep_plan_execute whose eta is
 * not below tol: nep_plan_result then returns the polished values (same pairs, same order).
 * *polished (or NULL) receives the number of pairs polished. Errors: NEP_ERR_ARG (NULL plan,
 * max_it < 0), CUDA errors. */
int nep_plan_polish(nep_plan_t p, double tol, int32_t max_it, int32_t *polished, int32_t *iterations, void *stream);

/* ------------------------------------------------------------------ left eigenvectors, resolvent */
/* Left eigenvectors y^* T(lambda) = 0 (Sec. 2 Eq. (nep-left): right eigenvectors of T(lambda)^*)
 * of P eigenpairs (lambda_p, x_p), requested through Sec. 3.2.5's interface. T(lambda_p)^* is
 * assembled (as a band with the bandwidths swapped) and factored once by the band LU (complex64
 * factors for NEP_PREC_MIXED, complex128 for NEP_PREC_FP64; an exactly zero pivot stands for a tiny
 * one; should a result not be finite, all pairs are recomputed with the factors of T(lambda_p) and
 * the conjugate-transpose solve); from y = x_p the first step is inverse iteration y <- T(lambda_p)^{-*} y,
 * later steps y <- y - T(lambda_p)^{-*} (T(lambda_p)^* y) with the residual in FP64, each
 * normalised to unit 2-norm. A pair stops when its left scaled residual
 *   eta_L = ||T(lambda)^* y||_2 / (sum_i |f_i(lambda)| ||A_i||_1 ||y||_2)
 * falls below tol, when a step gains less than a factor 2 (the floor set by the eigenvalue's own
 * error), or after max_it steps. Finally y is scaled to y^* T'(lambda) x = 1 (the normalisation of
 * Sec. 2 Eq. (resolvent)); a pair with y^* T'(lambda) x = 0 keeps its unit y and gets eta = +inf.
 *   lam_dev: P complex128 eigenvalues; X_dev: n x P complex128 right eigenvectors (read only)
 *   Y_dev:   n x P complex128, column-major (out)
 *   eta_dev: P doubles (out: eta_L of the unit vector before the scaling); its_dev: P int32 steps
 *            per pair (out), or NULL
 * *iterations (or NULL) receives the largest step count. The caller owns every array; work arrays
 * are allocated on the stream and the call returns when the stream is done.
 * Errors: NEP_ERR_ARG (P < 0, max_it < 1, NULL arrays with P > 0, unknown precision), CUDA errors. */
int nep_left_eigvecs(nep_split_t h, int32_t precision, int32_t P, const double *lam_dev, const double *X_dev,
                     double *Y_dev, double *eta_dev, int32_t *its_dev, double tol, int32_t max_it,
                     int32_t *iterations, void *stream);
/* nep_left_eigvecs for the eigenpairs that the plan's last nep_plan_execute returned (as after
 * nep_plan_polish, if called), in the order of nep_plan_result: Y_dev (n x capacity complex128)
 * and eta_dev (capacity doubles) receive the first *nconv columns / entries. *nconv (or NULL)
 * receives the number of returned pairs. Errors: NEP_ERR_ARG (NULL plan, max_it < 1, capacity < 0,
 * NULL arrays with capacity > 0, more returned pairs than capacity), CUDA errors. */
int nep_plan_left(nep_plan_t p, double tol, int32_t max_it, int32_t capacity, double *Y_dev, double *eta_dev,
                  int32_t *nconv, int32_t *iterations, void *stream);
/* Pole part of the resolvent, Keldysh's expansion (Sec. 2 Eq. (resolvent)) without its
 * holomorphic remainder R(z):  out_{j,k} = sum_i (z_j - lambda_i)^{-1} x_i (y_i^* v_k)
 * for nz points z_j and nv vectors v_k, with Keldysh-normalised left vectors y_i (as from
 * nep_left_eigvecs). Inside a region holding all P eigenvalues and away from them, this is
 * T(z)^{-1} v up to R(z) v. All arrays are the caller's device memory, complex128 column-major:
 * lam_dev[P], X_dev and Y_dev n x P, z_dev[nz], V_dev n x nv, out_dev n x (nz*nv) with column
 * j*nv + k for (z_j, v_k). Asynchronous on the stream (its work arrays are freed in stream order).
 * Errors: NEP_ERR_ARG (n < 1, negative counts, NULL arrays that the counts need), CUDA errors. */
int nep_apply_resolvent(int32_t n, int32_t P, const double *lam_dev, const double *X_dev, const double *Y_dev,
                        int32_t nz, const double *z_dev, int32_t nv, const double *V_dev, double *out_dev,
                        void *stream);

/* ------------------------------------------------------------------ NLEIGS (static variant) */
/* Options of the rational-interpolation solver (Sec. 4.5). Zero fields take the defaults. */
typedef struct {
    double tol;          /* degree test max_i |d_i^d| < tol max_i |d_i^0|; default 1e-13        */
    int32_t max_degree;  /* largest degree d; default 60, at most 63                             */
    int32_t nboundary;   /* points discretising the boundary of the region; default 1024         */
    int32_t krylov;      /* Arnoldi steps of a cycle (the basis size); default 100, at most 512  */
    int32_t has_shift;   /* nonzero: use shift_re/im as the shift sigma, else the region centre  */
    double shift_re, shift_im;
    uint64_t seed;       /* seeded start vector (SplitMix64 + Box-Muller)                         */
    double eig_tol;      /* acceptance: eta <= eig_tol and inside the region; default 1e-8        */
    int32_t exact_solves; /* nonzero: each Arnoldi solve gets two FP64-residual corrections; zero  */
                          /* (default): plain complex64 solves, then the Ritz pairs inside the     */
                          /* region with eta <= 1e-4 are polished by nep_rii's iteration (FP64     */
                          /* residuals, tol 1e-13, at most 10 iterations) before the acceptance    */
    int32_t full_basis;   /* nonzero: Arnoldi on full (d n)-vectors; zero (default): the compact TOAR   */
                          /* basis of Sec. 4.5.3, U (n x m, m <= d + krylov) and coefficient vectors    */
    int32_t max_restarts; /* Krylov-Schur restarts with locking after the first cycle of krylov steps;  */
                          /* 0 (default): one cycle, no restart                                          */
    int32_t keep;         /* vectors kept at a restart, < krylov; default krylov / 2                     */
    double restart_tol;   /* a Ritz pair has converged when |b^T s| <= restart_tol |theta|; default     */
                          /* 1e-10 with exact_solves, 1e-6 without                                       */
    int32_t nev;          /* restarts stop once nev wanted pairs have converged; 0 (default): once      */
                          /* every wanted Ritz pair of the cycle has converged (at least one)            */
} nep_nleigs_opts;
/* The rational interpolant R_d(z) = sum_j b_j(z) D_j, D_j = sum_i d_i^j A_i, of Sec. 4.5.1 on the
 * region (host computation):
 *   - boundary of the region at nboundary points z_k = c + a cos(2 pi k/nb) + i b sin(2 pi k/nb);
 *   - singularity set Xi: the roots of the denominators of rational nodes (and of the rational
 *     denominator of a quotient), each square-root branch cut sampled at distances 0 and
 *     10^(-4 + 8k/47), k < 48, from its branch point; exp contributes nothing; the outer function of
 *     a composition is not searched;
 *   - Leja-Bagby nodes sigma_j on the boundary and poles xi_j in Xi (Eq. (nleigsleja)), sigma_0 =
 *     z_0, each Xi point used at most once, infinity once none is left; scalings beta_j with
 *     max |b_j| = 1 on the boundary (Eq. (nleigsbj), beta_0 = 1);
 *   - divided differences d_i^j = e_j^T f_i(H K^{-1}) e_1 (Eq. (nleigsfdd)) through functions of
 *     the lower-triangular H K^{-1} (matrix polynomials and triangular solves, exp by scaling and
 *     squaring of its Taylor series, sqrt by the Bjorck-Hammarling recurrence); the degree d is
 *     the first d >= 1 whose last pole, taken as infinity (Eq. (nleigsmatlin)), gives
 *     max_i |d_i^d| < tol max_i |d_i^0|.
 * Host arrays with room for cap = d+1 entries (d <= max_degree): sigma, xi complex[cap] (xi[0] and
 * the last pole are infinity, written as (inf, 0)); beta double[cap]; dd complex[nterms*cap] with
 * dd[i + nterms*j] = d_i^j. *degree, *converged (1 if the test held), *nsing (points of Xi); any
 * output pointer may be NULL. Errors: NEP_ERR_ARG (bad region, cap < d+1, max_degree outside
 * 1..63). */
int nep_nleigs_interpolation(nep_split_t h, const nep_region *r, const nep_nleigs_opts *o, int32_t cap,
                             double *sigma, double *xi, double *beta, double *dd, int32_t *degree,
                             int32_t *converged, int32_t *nsing);
/* The same from the function descriptions alone (nterms of them, as for nep_create_split): a host
 * computation that touches no device, for callers without a split or without a GPU. */
int nep_nleigs_interpolation_fns(int32_t nterms, const nep_fn *f, const nep_region *r, const nep_nleigs_opts *o,
                                 int32_t cap, double *sigma, double *xi, double *beta, double *dd, int32_t *degree,
                                 int32_t *converged, int32_t *nsing);
/* NLEIGS, static variant (Sec. 4.5.2, 4.5.3): shift-and-invert Arnoldi with o->krylov steps on
 * S = (A - sigma B)^{-1} B for the linearisation (A, B) of Eq. (nleigsmatlin), applied through the
 * block recurrences of Eqs. (nleigstoarreca) and (nleigstoarrecb) with one band LU of R_d(sigma)
 * (complex64 factors) and per step one band solve (with two corrections against the FP64 residual of
 * R_d(sigma) when o->exact_solves is set). By default the basis is the compact one of Sec. 4.5.3
 * (Eqs. (nleigs-toar1)-(nleigs-toar4)): Krylov vectors (I_d (x) U) g with U orthonormal (n x m, one new
 * column per step, none when the new direction already lies in span U) and coefficient vectors g,
 * Gram-Schmidt on n-vectors for U and on d m coefficient vectors for the Arnoldi; o->full_basis
 * keeps full (d n)-vectors. Classical Gram-Schmidt twice in both. Ritz values theta (complex64 QR, then
 * FP64 inverse iteration on the projected matrix and a Rayleigh quotient) give lambda = sigma + 1/theta
 * and x the first block of the Ritz vector. With o->max_restarts > 0, Krylov-Schur restarts with
 * locking follow each cycle of krylov steps (Sec. 4.5.3): the Ritz pairs with lambda inside the region
 * are wanted, converged when |b^T s| <= restart_tol |theta| (b the last row of the (k+1) x k Arnoldi
 * matrix); the run stops once o->nev wanted pairs have converged (nev = 0: every wanted pair of the
 * cycle, at least one) or after max_restarts restarts; else
 * the basis is cut to the invariant subspace of p = max(keep, converged + 1) Ritz values (converged
 * first, then wanted, then the others, each nearest the shift first), Q = the leading p Schur vectors
 * of H after the FP64 Schur form is reordered to put those first, plus the last Arnoldi vector; H
 * becomes the leading p x p block of the reordered Schur factor with the coupling row b^T Q, whose
 * entries for the converged (locked) vectors are zeroed, and the compact basis is compressed to an
 * orthonormal basis W of the range of its coefficient blocks (U <- U W; QR with column pivoting
 * stopped at a relative Frobenius mass of 1e-13, at most d + kept vectors); the Arnoldi continues
 * from there. Pairs inside the region with FP64 eta (Sec. 2 Eq. (sressplit), of the full T) at most
 * eig_tol are returned, deduplicated and sorted as nep_ciss_solve does. *out receives a result
 * object (nep_result_get; hankel_rank there is 0; flags NEP_WARN_INTERP if the degree test failed
 * at max_degree, NEP_WARN_SINGULAR_NODE if R_d(sigma) had an exactly zero pivot); *degree (or NULL)
 * the interpolation degree; nep_result_info gives the Arnoldi steps run and the restarts. The call
 * allocates its work arrays on the stream ((d n) x (krylov+1) complex128 for the full basis, n x
 * (d + krylov + 1) for the compact one) and returns when they are done. Errors: NEP_ERR_ARG, NEP_ERR_REGION
 * (a singularity of some f_i inside or on the region), NEP_ERR_UNSUPPORTED (more than 8 terms),
 * CUDA errors. */
int nep_nleigs_solve(nep_split_t h, const nep_region *r, const nep_nleigs_opts *o, nep_result_t *out,
                     int32_t *degree, void *stream);

/* ------------------------------------------------------------------ Interpol (Chebyshev interpolation) */
/* Options of the polynomial interpolation solver (Sec. 4.4). Zero fields take the defaults. */
typedef struct {
    int32_t degree;       /* interpolation degree d, 2 .. 63 (the paper leaves it to the user); default 40 */
    int32_t krylov;       /* Arnoldi steps of a cycle (the basis size); default 60, at most 512            */
    int32_t has_shift;    /* nonzero: shift_re/im (a value of lambda) as the shift; else the interval's    */
    double shift_re, shift_im; /* centre                                                                */
    uint64_t seed;        /* seeded start vector (SplitMix64 + Box-Muller)                                 */
    double eig_tol;       /* acceptance: eta of T (Eq. (sressplit)) <= eig_tol inside the region; 1e-8     */
    int32_t fast_solves;  /* nonzero: plain complex64 solves, then residual inverse iteration on T for the  */
                          /* Ritz pairs inside the region with eta <= 1e-4 (their eigenvalues then are T's, */
                          /* not P_d's); zero (default): each solve gets two FP64-residual corrections      */
    int32_t max_restarts; /* Krylov-Schur restarts as for nep_nleigs_opts (0: none)                        */
    int32_t keep;         /* vectors kept at a restart, < krylov; default krylov / 2                        */
    double restart_tol;   /* convergence of a Ritz pair, as for nep_nleigs_opts (default 1e-10, fast 1e-6)  */
    int32_t nev;          /* wanted eigenvalues that end the restarts, as for nep_nleigs_opts              */
} nep_interpol_opts;
/* Chebyshev coefficients of the f_i on the interval I = [c - a, c + a], the real axis of the region's
 * ellipse (real centre c; a = real semi-axis), lambda = a theta + c (host computation, no device):
 * nodes nu_j = cos(omega_j), omega_j = (j + 1/2) pi / (d + 1), j = 0 .. d (Eq. (interpolnu)) and
 * c_ik = 2/(d+1) sum_j f_i(lambda(nu_j)) cos(k omega_j) (Eq. (polinterpcoef)), so that
 * P_d(theta) = sum_i (c_i0/2 + sum_{k>=1} c_ik tau_k(theta)) A_i. coef: complex[nterms * (d+1)] with
 * coef[i + nterms k] = c_ik. Errors: NEP_ERR_ARG (bad region, complex centre, degree outside 2 .. 63). */
int nep_interpol_coefficients(int32_t nterms, const nep_fn *f, const nep_region *r, int32_t degree, double *coef);
/* The polynomial interpolation solver (Sec. 4.4, "Interpol") for eigenvalues on or near a real interval:
 * the coefficients above, then the eigenproblem P_d(theta) x = 0 by shift-and-invert Arnoldi on its
 * Chebyshev-basis linearisation (block rows -theta u_0 + u_1 = 0, u_{k-1} - 2 theta u_k + u_{k+1} = 0 and
 * sum_{k<d} C'_k u_k + C_d (2 theta u_{d-1} - u_{d-2}) = 0 for u_k = tau_k(theta) x), applied through
 * the block recurrences with one band LU of P_d(sigma) (complex64 factors) and one band solve per step;
 * classical Gram-Schmidt twice, Ritz values and Krylov-Schur restarts (o->max_restarts) as
 * nep_nleigs_solve with its full basis. The region filter of Sec. 4.4: pairs
 * with lambda strictly inside the region's ellipse (its imaginary semi-axis sets the vicinity of the
 * interval) and the scaled residual of T itself <= eig_tol, sorted and deduplicated as nep_ciss_solve
 * does; x is the first block of the Ritz vector. *out receives a result object (hankel_rank 0, no
 * points; NEP_WARN_SINGULAR_NODE if P_d(sigma) had an exactly zero pivot). The call allocates its work
 * arrays on the stream ((d n) x (krylov+1) complex128) and returns when they are done.
 * Errors: NEP_ERR_ARG (bad region, complex centre, options out of range), NEP_ERR_REGION (a
 * singularity of some f_i inside or on the region), NEP_ERR_UNSUPPORTED (more than 8 terms, or
 * callback/table terms), CUDA errors. */
int nep_interpol_solve(nep_split_t h, const nep_region *r, const nep_interpol_opts *o, nep_result_t *out,
                       void *stream);

/* ------------------------------------------------------------------ serving */
/* Continuous-batching request server. Requests are admitted in arrival order as soon as a
 * worker is free and their device footprint (nep_plan_bytes) fits the remaining budget;
 * every worker drives its own CUDA stream, so the kernels of admitted requests overlap on
 * the device. Each request runs exactly the computation of nep_ciss_solve on its inputs
 * (same kernels, same launch shapes, no state shared between requests), so its result does
 * not depend on what else is in flight. The split handle passed to nep_submit must stay
 * alive until the request's result has been taken.
 * Hardware queues: CUDA gives a context 8 work queues unless the environment variable
 * CUDA_DEVICE_MAX_CONNECTIONS (read when the process creates its context) says otherwise.
 * With more busy streams than queues, streams share a queue and a request's short result copy
 * can wait behind another worker's whole pass. Set it to at least workers + 2 (32 at most)
 * before the first CUDA call; the Python binding sets 32 when it is imported, unless the
 * variable is already set. */
typedef struct nep_server *nep_server_t;
#define NEP_PENDING 1 /* nep_poll: the request has not finished yet */
/* workers >= 1 concurrent requests; hbm_budget_bytes == 0: 80% of the free device memory. */
int nep_server_create(int32_t workers, uint64_t hbm_budget_bytes, nep_server_t *out);
/* The same with shared launches: a free worker takes up to max_batch requests from the head of the
 * queue (in arrival order, while they fit the budget and share a precision; requests with callback or
 * table terms run alone) and runs them as one nep_plan_execute_batch, so the LU and the sweeps of all
 * their quadrature points share launches; each result stays bitwise the one it gets alone.
 * max_batch == 1 is nep_server_create. Errors: NEP_ERR_ARG (workers < 1, max_batch < 1), NEP_ERR_CUDA. */
int nep_server_create_batched(int32_t workers, int32_t max_batch, uint64_t hbm_budget_bytes, nep_server_t *out);
/* Copies the region, options and V (n x L complex, or NULL: drawn from opts->seed) and
 * enqueues the request; *ticket identifies it. NEP_ERR_NOMEM if it can never fit the budget. */
int nep_submit(nep_server_t s, nep_split_t h, const nep_region *r, int32_t N, int32_t L, int32_t M, const nep_opts *o,
               const double *V_host, uint64_t *ticket);
/* NEP_OK and *out (to be freed with nep_result_free) once done, NEP_PENDING before, or the
 * request's error code. A ticket's result can be taken once. */
int nep_poll(nep_server_t s, uint64_t ticket, nep_result_t *out);
/* Blocks until the request is done; same returns as nep_poll without NEP_PENDING. */
int nep_server_wait(nep_server_t s, uint64_t ticket, nep_result_t *out);
/* Waits for all admitted and queued requests, then stops the workers. */
int nep_server_destroy(nep_server_t s);
/* Device bytes one solve of this shape allocates with the full quadrature: an upper bound. Admission
 * charges each request its own footprint, which is smaller for a request with opts.symmetric set (only
 * the N/2 nodes above the real axis are held), so budgets sized with this figure are conservative. */
uint64_t nep_plan_bytes(nep_split_t h, int32_t N, int32_t L, int32_t M, int32_t precision);

/* ------------------------------------------------------------------ step entry points */
/* Trapezoid nodes on Gamma (host): theta_j = 2 pi (j + 1/2)/N, z_j, weights
 * w_j = (b cos theta_j + i a sin theta_j)/N, zeta_j = (z_j - c)/a; each complex[N]. */
int nep_nodes(const nep_region *r, int32_t N, double *z, double *w, double *zeta);
/* F[i + l*j] = f_i(z_j) (host, complex[l*N]); dF likewise with f_i'. dF may be NULL. */
int nep_coefficients(nep_split_t h, int32_t N, const double *z, double *F, double *dF);
/* Kernel (a): band storage of T(z_j) = sum_i F[i,j] A_i for npts points (F_dev complex[l*npts]
 * on the device). Row-oriented band: entry (r, k), r-kl <= k <= r+ku, of point j at
 * ab[j*n*ldab + r*ldab + (k - r + kl)], other entries of the row zero; complex64
 * (precision MIXED) or complex128 (FP64). tnorm_dev[j] = ||T(z_j)||_inf (may be NULL). */
int nep_assemble_band(nep_split_t h, int32_t npts, const double *F_dev, int32_t precision, void *ab_dev,
                      double *tnorm_dev, void *stream);
/* Kernel (b): in-place banded LU with partial pivoting of npts assembled bands
 * (pivot: max |Re|+|Im| within kl rows, first index on ties). Output layout per row c:
 * ab[c*ldab + t] = U(c, c+t) for t in [0, kl+ku]; ab[c*ldab + kl+ku+1 + i] = L(c+1+i, c)
 * for i in [0, kl). ipiv_dev[j*n + c] = pivot row (0-based). info_dev[j] = 0 or
 * 1 + first column with an exactly zero pivot. */
int nep_band_factor(nep_split_t h, int32_t npts, int32_t precision, void *ab_dev, int32_t *ipiv_dev,
                    int32_t *info_dev, void *stream);
/* Kernel (b): solve T(z_j) X_j = B_j with the factors, in place on B (npts x n x L,
 * column-major per point, element type of the precision). For narrow bands (kl+1 <= 288 and
 * kl+ku+1 <= 288) the call builds the column copy of U (nep_band_transpose_u) in a temporary
 * of its own; a caller solving repeatedly with the same factors builds it once and calls
 * nep_band_solve_cols instead. */
int nep_band_solve(nep_split_t h, int32_t npts, int32_t precision, const void *ab_dev, const int32_t *ipiv_dev,
                   int32_t L, void *B_dev, void *stream);
/* Conjugate-transpose solve T(z_j)^* X_j = B_j with the factors of nep_band_factor, in place on
 * B (npts x n x L, column-major per point, element type of the precision): U^* forward, then
 * the L factors' conjugate transposes and the interchanges in reverse order (the factorisation
 * reused, as Sec. 4.5.4 does for the conjugate-transpose operator). An exactly zero pivot
 * (info != 0) stands for a tiny one (1e-20 for complex64 factors, 1e-100 for complex128), which
 * inverse iteration on a singular matrix wants. Asynchronous on the stream. */
int nep_band_solve_adjoint(nep_split_t h, int32_t npts, int32_t precision, const void *ab_dev,
                           const int32_t *ipiv_dev, int32_t L, void *B_dev, void *stream);
/* U of the factored band by columns: ut[j][c*(kl+ku+1) + d] = U(c-d, c) for d in [0, kl+ku]
 * (zero where c-d < 0); ut_dev holds npts x n x (kl+ku+1) elements of the precision's type. */
int nep_band_transpose_u(nep_split_t h, int32_t npts, int32_t precision, const void *ab_dev, void *ut_dev,
                         void *stream);
/* nep_band_solve with the column copy of U made by nep_band_transpose_u from the same factors
 * (ut_dev may be NULL for bands too wide for the narrow-band sweeps). */
int nep_band_solve_cols(nep_split_t h, int32_t npts, int32_t precision, const void *ab_dev, const void *ut_dev,
                        const int32_t *ipiv_dev, int32_t L, void *B_dev, void *stream);
/* Kernel (c): FP64 split-form residual R_j = V - T(z_j) Y_j (npts x n x L complex128). */
int nep_split_residual(nep_split_t h, int32_t npts, const double *F_dev, int32_t L, const double *V_dev,
                       const double *Y_dev, double *R_dev, void *stream);
/* Kernel (d): S_k = sum_j coef[j + N*k] Y_j for k < K (Y: N x n x L, S: K x n x L complex128);
 * j summed in ascending order. */
int nep_moments(int32_t n, int32_t L, int32_t N, int32_t K, const double *coef_dev, const double *Y_dev, double *S_dev,
                void *stream);
/* One-sided Jacobi SVD (FP64, device): A (rows x cols complex, column-major, rows >= cols)
 * is overwritten by U Sigma; W_dev (cols x cols) receives W with A_in W = U Sigma; sigma
 * descending with the columns of A and W permuted to match. Runs on a cooperative grid whose
 * barriers wait a bounded time (nep_set_wait_limit; NEP_ERR_INTERNAL when one runs out), or, when
 * the environment variable NEP_JACOBI_CLUSTER is "1" at the call and rows, cols <= 256 fit, on one
 * thread-block cluster with the columns in distributed shared memory (more throughput beside
 * other work, more latency alone). The two differ in rounding only; the contour solver's
 * Hankel SVD takes the same choice. */
int nep_jacobi_svd(int32_t rows, int32_t cols, double *A_dev, double *W_dev, double *sigma_dev, void *stream);
/* The SVD of nep_jacobi_svd for callers that cannot allocate device memory (a host that
 * accounts for every device byte itself, or a loop that must not enter the CUDA allocator).
 * The paper has no counterpart: this is a deployment variant of the Jacobi SVD above.
 * Same arguments and results as nep_jacobi_svd; its work arrays live in one fixed block of
 * device memory compiled into the library (2 MiB + 256 bytes, held on every GPU that loads
 * the library until the process exits), so it accepts rows*cols + cols*cols <= 131072
 * (e.g. 256 x 256) and returns NEP_ERR_ARG beyond that. It calls no allocation routine.
 * The first call on a device looks the block's device address up on that device (make that
 * first call before any stream capture). All calls share the block and each call resets the
 * parts that must start at zero: calls that overlap on the GPU (other streams, other host
 * threads) race and must be serialised by the caller. Returns after the stream finished. */
int nep_jacobi_svd_noalloc(int32_t rows, int32_t cols, double *A_dev, double *W_dev, double *sigma_dev, void *stream);
/* Eigenvalues and eigenvectors of a small complex matrix (m x m, FP64, device):
 * Hessenberg reduction and shifted QR. evec_dev may be NULL. */
int nep_small_eig(int32_t m, const double *A_dev, double *eval_dev, double *evec_dev, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* NEP_CISS_H */

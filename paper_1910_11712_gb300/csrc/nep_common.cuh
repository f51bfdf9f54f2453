// Shared definitions of the CUDA library: complex arithmetic, the split operator on
// the device, scalar-function evaluation, error reporting and launch helpers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/nep_ciss.h"

namespace nep {

// ----------------------------------------------------------------- complex numbers
template <typename T>
struct alignas(2 * sizeof(T)) cx {
    T re, im;
};
typedef cx<double> zd;
typedef cx<float> zf;

template <typename T> __host__ __device__ __forceinline__ cx<T> mk(T r, T i) { cx<T> z; z.re = r; z.im = i; return z; }
template <typename T> __host__ __device__ __forceinline__ cx<T> operator+(cx<T> a, cx<T> b) { return mk(a.re + b.re, a.im + b.im); }
template <typename T> __host__ __device__ __forceinline__ cx<T> operator-(cx<T> a, cx<T> b) { return mk(a.re - b.re, a.im - b.im); }
template <typename T> __host__ __device__ __forceinline__ cx<T> operator-(cx<T> a) { return mk(-a.re, -a.im); }
template <typename T> __host__ __device__ __forceinline__ cx<T> operator*(cx<T> a, cx<T> b) {
    return mk(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <typename T> __host__ __device__ __forceinline__ cx<T> operator*(T s, cx<T> a) { return mk(s * a.re, s * a.im); }
template <typename T> __host__ __device__ __forceinline__ cx<T> conj(cx<T> a) { return mk(a.re, -a.im); }
template <typename T> __host__ __device__ __forceinline__ T abs1(cx<T> a) { return fabs(a.re) + fabs(a.im); }
template <typename T> __host__ __device__ __forceinline__ T norm2(cx<T> a) { return a.re * a.re + a.im * a.im; }
template <typename T> __host__ __device__ __forceinline__ T cabs_(cx<T> a) { return hypot(a.re, a.im); }
// acc - a*b with fused multiply-adds
template <typename T> __host__ __device__ __forceinline__ cx<T> fms(cx<T> acc, cx<T> a, cx<T> b) {
    acc.re = fma(-a.re, b.re, acc.re);
    acc.re = fma(a.im, b.im, acc.re);
    acc.im = fma(-a.re, b.im, acc.im);
    acc.im = fma(-a.im, b.re, acc.im);
    return acc;
}
// acc + a*b
template <typename T> __host__ __device__ __forceinline__ cx<T> fma_(cx<T> acc, cx<T> a, cx<T> b) {
    acc.re = fma(a.re, b.re, acc.re);
    acc.re = fma(-a.im, b.im, acc.re);
    acc.im = fma(a.re, b.im, acc.im);
    acc.im = fma(a.im, b.re, acc.im);
    return acc;
}
// acc + conj(a)*b
template <typename T> __host__ __device__ __forceinline__ cx<T> fmac(cx<T> acc, cx<T> a, cx<T> b) {
    acc.re = fma(a.re, b.re, acc.re);
    acc.re = fma(a.im, b.im, acc.re);
    acc.im = fma(a.re, b.im, acc.im);
    acc.im = fma(-a.im, b.re, acc.im);
    return acc;
}
// a / b with scaling against overflow (Smith's method)
template <typename T> __host__ __device__ __forceinline__ cx<T> cdiv(cx<T> a, cx<T> b) {
    if (fabs(b.re) >= fabs(b.im)) {
        T r = b.im / b.re, d = b.re + b.im * r;
        return mk((a.re + a.im * r) / d, (a.im - a.re * r) / d);
    } else {
        T r = b.re / b.im, d = b.im + b.re * r;
        return mk((a.re * r + a.im) / d, (a.im * r - a.re) / d);
    }
}
template <typename T> __host__ __device__ __forceinline__ cx<T> csqrt_(cx<T> z) {
    // principal square root; the cut lies on the negative real axis, the sign of a zero
    // imaginary part selects the side (as C99 csqrt)
    T x = z.re, y = z.im;
    if (x == 0 && y == 0) return mk<T>(0, y);
    T r = hypot(x, y);
    T s = sqrt((r + fabs(x)) * T(0.5));
    if (x >= 0) return mk(s, y / (T(2) * s));
    return mk(fabs(y) / (T(2) * s), copysign(s, y));
}
template <typename T> __host__ __device__ __forceinline__ cx<T> cexp_(cx<T> z) {
    T e = exp(z.re);
    return mk(e * cos(z.im), e * sin(z.im));
}
template <typename T, typename U> __host__ __device__ __forceinline__ cx<T> cvt(cx<U> a) {
    return mk<T>((T)a.re, (T)a.im);
}

// ----------------------------------------------------------------- scalar functions
// Flattened function tree: node k has kind/op, scaling alpha/beta, shift, coefficient
// ranges into a shared coefficient pool, and child node indices (combine).
// LU kernel choices for complex64 bands with kl > 64 (nep_opts.lu_kernel): the library's default
// (tensor core, 3 x TF32), the tensor core with TF32 operands, the FP32 SIMT kernel
enum { LU_AUTO = 0, LU_TC3 = 1, LU_TC1 = 2, LU_SIMT = 3 };

// One quadrature point of some problem in a launch shared by several problems: a kernel given an
// array of these takes block b's sizes and buffers from entry b instead of its uniform arguments
// (point index 0 within them), with the same arithmetic per point.
struct PointDesc {
    int n, kl, ku, ldab, L, RWp, CWp, pad;
    void* ab;           // this point's band (factors)
    const void* ut;     // its column copy of U (sweeps)
    int* ipiv;
    int* info;
    void* B;            // its right-hand sides, n x L column-major
    const int* active;  // its refinement flag, or nullptr
    void* win;          // its LU window (wide bands)
};

struct FnNode {
    int kind, op, a, b;
    int num_off, num_len, den_off, den_len;
    zd alpha, beta, shift;
};

struct FnEval {
    zd f, df;
};

// Evaluates node k at z: g(z) = beta h(alpha z), returns g and g'.
__host__ __device__ inline FnEval fn_eval(const FnNode* nodes, const zd* coef, int k, zd z, int depth = 0) {
    const FnNode nd = nodes[k];
    zd x = nd.alpha * z;
    zd h, dh;
    if (nd.kind == NEP_FN_RATIONAL) {
        zd p = mk(0.0, 0.0), dp = mk(0.0, 0.0);
        for (int t = 0; t < nd.num_len; ++t) {
            dp = dp * x + p;
            p = p * x + coef[nd.num_off + t];
        }
        if (nd.den_len > 0) {
            zd q = mk(0.0, 0.0), dq = mk(0.0, 0.0);
            for (int t = 0; t < nd.den_len; ++t) {
                dq = dq * x + q;
                q = q * x + coef[nd.den_off + t];
            }
            h = cdiv(p, q);
            dh = cdiv(dp * q - p * dq, q * q);
        } else {
            h = p;
            dh = dp;
        }
    } else if (nd.kind == NEP_FN_EXP) {
        h = cexp_(x);
        dh = h;
    } else if (nd.kind == NEP_FN_SQRT) {
        h = csqrt_(x - nd.shift);
        dh = cdiv(mk(0.5, 0.0), h);
    } else if (nd.kind == NEP_FN_CALLBACK || nd.kind == NEP_FN_TABLE) {
        // host-supplied functions have no device form; callers pass their values in instead
        h = mk((double)NAN, (double)NAN);
        dh = h;
    } else {  // combine
        if (depth > 16) return FnEval{mk(0.0, 0.0), mk(0.0, 0.0)};
        if (nd.op == NEP_OP_COMPOSE) {
            FnEval eb = fn_eval(nodes, coef, nd.b, x, depth + 1);
            FnEval ea = fn_eval(nodes, coef, nd.a, eb.f, depth + 1);
            h = ea.f;
            dh = ea.df * eb.df;
        } else {
            FnEval ea = fn_eval(nodes, coef, nd.a, x, depth + 1);
            FnEval eb = fn_eval(nodes, coef, nd.b, x, depth + 1);
            if (nd.op == NEP_OP_ADD) {
                h = ea.f + eb.f;
                dh = ea.df + eb.df;
            } else if (nd.op == NEP_OP_MUL) {
                h = ea.f * eb.f;
                dh = ea.df * eb.f + ea.f * eb.df;
            } else {
                h = cdiv(ea.f, eb.f);
                dh = cdiv(ea.df * eb.f - ea.f * eb.df, eb.f * eb.f);
            }
        }
    }
    return FnEval{nd.beta * h, nd.beta * nd.alpha * dh};
}

// ----------------------------------------------------------------- device split operator
// Union sparsity pattern of all terms in CSR, one FP64 value array per term (zero where a
// term has no entry), so a single pass over the pattern applies any combination of terms.
struct SplitDev {
    int n, nterms, kl, ku, ldab;
    int64_t nnz;
    const int64_t* rowptr;  // n+1
    const int32_t* col;     // nnz
    const double* val;      // nterms x nnz real parts
    const double* val_im;   // nterms x nnz imaginary parts, or nullptr if all terms are real
    const double* norms;    // nterms, ||A_i||_inf
    const double* norms1;   // nterms, ||A_i||_1
    const int64_t* colptr;  // n+1: the pattern by columns, rows ascending within a column
    const int64_t* cidx;    // nnz: union-pattern entry of each column-ordered entry
    const int32_t* crow;    // nnz: its row
    const FnNode* fn_nodes;
    const zd* fn_coef;
    const int* fn_root;     // nterms root node indices
};

// ----------------------------------------------------------------- errors
void set_error(const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what, const char* file, int line);

#define NEP_CUDA(call)                                                                  \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess) return ::nep::cuda_fail(e_, #call, __FILE__, __LINE__); \
    } while (0)
void count_launch();
// f_i (and f_i') of every term at count points on the host, F[i + nterms k]; host-supplied terms through
// the user's function (host_api.cu). NEP_ERR_UNSUPPORTED for a tabulated term without eval.
int host_terms(const ::nep_split* h, const zd* z, int count, zd* F, zd* dF);
// whether any term is host-supplied (callback or table): such splits have no device function tree
bool split_has_host_terms(const ::nep_split* h);
// polls a device-side wait makes before it gives up and records an error (nep_set_wait_limit)
long long wait_limit();
#define NEP_CHECK_LAUNCH()         \
    do {                           \
        ::nep::count_launch();     \
        NEP_CUDA(cudaGetLastError()); \
    } while (0)
#define NEP_TRY(call)            \
    do {                         \
        int rc_ = (call);        \
        if (rc_ != NEP_OK) return rc_; \
    } while (0)

static inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// The device's opt-in dynamic shared memory per block (queried once).
int smem_optin_bytes();
// Raises a kernel's dynamic shared-memory limit to that maximum (less its static shared memory).
// Every caller sets the same value,
// so calls from several host threads (the request server's workers, concurrent plans) cannot lower
// the limit between another thread's set and its launch; each launch still passes its own size.
// (done once per kernel and device; two threads racing to do it set the same value)
bool smem_limit_raised(const void* fn);
void smem_limit_mark(const void* fn);
template <typename K>
inline cudaError_t allow_max_dynamic_smem(K kernel) {
    if (smem_limit_raised((const void*)kernel)) return cudaSuccess;
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, kernel);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             smem_optin_bytes() - (int)a.sharedSizeBytes);
    if (e == cudaSuccess) smem_limit_mark((const void*)kernel);
    return e;
}

// ----------------------------------------------------------------- launchers (per file)
// assemble.cu
template <typename T>
int launch_assemble(const SplitDev& s, int npts, const zd* F, cx<T>* ab, double* tnorm, zd* tval, cudaStream_t st);
// band_lu.cu
// Register-window LU with one CTA barrier per column step (lu_col.cu): kl <= 64, kl + ku <= 128.
bool band_lu_col_fits(int kl, int ku);
template <typename T>
int launch_band_lu_col(const SplitDev& s, int npts, cx<T>* ab, int* ipiv, int* info, const int* active,
                       cudaStream_t st);
// Blocked LU for wide bands (lu_wide.cu): panel in shared memory, trailing window in global memory.
bool band_lu_wide_fits(int kl, int elem_bytes);
// Points of several problems in shared launches (PointDesc arrays on the device):
// the register-window LU's template instance of a band shape (points with equal instances share a launch)
int lu_col_instance(int kl, int ku);
template <typename T>
int launch_band_lu_col_batch(int instance, int count, const PointDesc* pd_dev, cudaStream_t st);
// the narrow-band sweeps' launch shape of a problem, and the sweeps over points of equal shape
template <typename T>
void sweep_key(int kl, int ku, int npts, int L, int* rplf, int* rplb, int* rh, int rh_force = 0);
template <typename T>
int band_sweeps_batch(int rplf, int rplb, int rh, int count, int maxL, const PointDesc* pd, cudaStream_t st);
// the tensor-core LU over points of several complex64 problems (each kl > 64)
int launch_band_lu_tc_batch(const std::vector<PointDesc>& items, cudaStream_t st, int passes = 3);

template <typename T>
int launch_band_lu_wide(const SplitDev& s, int npts, cx<T>* ab, int* ipiv, int* info, const int* active,
                        cudaStream_t st);
// The same blocked LU in complex64 with the trailing update on the tensor core (lu_tc.cu): TMA-staged
// operand tiles, tcgen05 MMA (TF32 hi/lo split, 4M complex form) into tensor memory. The default for
// kl > 64 (band_lu_tc_fits); it runs for kl >= 32 (band_lu_tc_can) when asked for explicitly.
bool band_lu_tc_fits(int kl);
bool band_lu_tc_can(int kl);
// passes: 3 (TF32 hi/lo split, ~FP32 products) or 1 (TF32 operands)
int launch_band_lu_tc(const SplitDev& s, int npts, zf* ab, int* ipiv, int* info, const int* active, cudaStream_t st,
                      int passes = 3);
// Whether complex64 wide-band LUs use the tensor-core kernel (default yes; NEP_LU_TC=0 selects the
// FP32 SIMT kernel, for comparisons).
bool lu_tc_enabled();
template <typename T>
int launch_band_lu(const SplitDev& s, int npts, cx<T>* ab, int* ipiv, int* info, const int* active, cudaStream_t st,
                   int lu_kernel = LU_AUTO);
// Narrow-band substitution sweeps (register windows of kl+1 and kl+ku+1 rows, up to 288).
inline bool band_sweeps_fit(int kl, int ku) { return kl >= 1 && kl + 1 <= 288 && kl + ku + 1 <= 288; }
// band_solve_blocked.cu: the blocked substitution for complex64 factors of wider bands (NB-step
// blocks, products for the rows beyond each block); NEP_ERR_UNSUPPORTED when its windows do not fit
int band_solve_blocked_rhs(int kl, int ku, int L);
int launch_band_solve_blocked(const SplitDev& s, int npts, const zf* ab, const int* ipiv, int L, zf* B,
                              const int* active, cudaStream_t st);
// ut (npts x n x (kl+ku+1)): the U factor by columns, written by band_transpose_u after the LU.
template <typename T>
int band_sweeps(const SplitDev& s, int npts, const cx<T>* ab, const cx<T>* ut, const int* ipiv, int L, cx<T>* B,
                const int* active, cudaStream_t st, int rh_force = 0);
template <typename T>
int band_transpose_u(const SplitDev& s, int npts, const cx<T>* ab, cx<T>* ut, cudaStream_t st);
// moments.cu: conjugate-symmetric quadrature helpers
int launch_double_real(int64_t count, zd* x, cudaStream_t st);
int launch_count_imag(int64_t count, const zd* x, int* out, cudaStream_t st);
// host_api.cu: seeded probe block (count complex entries; imaginary parts zero when real_only)
void draw_probe_block(uint64_t seed, size_t count, bool real_only, double* out);
template <typename T>
int launch_band_solve(const SplitDev& s, int npts, const cx<T>* ab, const cx<T>* ut, const int* ipiv, int L, cx<T>* B,
                      const int* active, cudaStream_t st, int rh_force = 0);
// spmv.cu
int launch_split_residual(const SplitDev& s, int npts, const zd* tval, int L, const zd* V, const zd* Y, zd* R,
                          double* nrm, const int* active, cudaStream_t st);
template <typename T>
int launch_convert_rhs(int npts, int n, int L, const zd* V, cx<T>* B, cudaStream_t st);
template <typename T>
int launch_widen(int npts, int n, int L, const cx<T>* B, zd* Y, cudaStream_t st);
template <typename T>
int launch_refine_prepare(int npts, int n, int L, const zd* R, cx<T>* D, const int* active, cudaStream_t st);
template <typename T>
int launch_refine_update(int npts, int n, int L, const cx<T>* D, zd* Y, double* dmax, double* ymax,
                         const int* active, cudaStream_t st);
int launch_refine_decide(int npts, int L, int sweep, int max_sweeps, double tol, double step_tol, int extrapolate,
                         const double* nrm,
                         const double* tnorm, const double* dmax, const double* ymax, double* prev, double* beta,
                         int* active, int* sweeps, int* nactive, cudaStream_t st);
// moments.cu
int launch_moments(int n, int L, int N, int K, const zd* coef, const zd* Y, zd* S, cudaStream_t st);
int launch_vh_times(int n, int L, int K, const zd* V, const zd* S, zd* mu, zd* part, cudaStream_t st);
int launch_hankel_build(int L, int M, const zd* mu, zd* H, zd* Hs, cudaStream_t st);
// extract.cu
int zgemm(int M, int N, int K, int opA, const zd* A, int lda, const zd* B, int ldb, zd* C, int ldc, zd* part,
          size_t part_elems, cudaStream_t st);
struct JacobiWork {
    zd* Vm;
    int* flags;
    int* sweeps;
    unsigned* bar;
    int* err;
};
int jacobi_svd(int rows, int cols, zd* A, zd* U, zd* W, double* sigma, JacobiWork w, cudaStream_t st);
int qrcp_jacobi_svd(int n, zd* A, zd* U, zd* W, double* sigma, zd* work1, zd* work2, zd* work3, zd* tau, int* perm,
                    double* nrm2, int* steps_dev, int* steps_host, double trunc, JacobiWork w, cudaStream_t st);
template <typename T>
int small_eig(int m, const zd* A, zd* eval, zd* evec, int* status, void* gbuf, cudaStream_t st);
template <typename T>
int small_eig_fast(int m, const zd* A, zd* eval, zd* evec, int* status, void* gbuf, cudaStream_t st);
// Krylov-Schur restart: the FP64 Schur form A = Z T Z^H (eval = diag T; gbuf 2 m (m+1) + m elements,
// needed when it does not fit in shared memory), and its reordering that brings the diagonal entries
// at positions sel[0 .. p) to the front in that order
int launch_ks_schur(int m, const zd* A, zd* eval, zd* T, zd* Z, int* status, zd* gbuf, cudaStream_t st);
int launch_ks_reorder(int m, int p, const int* sel, zd* T, zd* Z, cudaStream_t st);
// an orthonormal basis Q (rows x r) of the range of A (rows x cols, overwritten) by QR with column
// pivoting, stopped at a relative Frobenius mass trunc; r <= rmax
int qr_range_basis(int rows, int cols, zd* A, zd* Q, int rmax, double trunc, zd* tau, int* perm, double* nrm2,
                   int* steps_dev, unsigned* bar, int* err, int* r_out, cudaStream_t st);
// complex128-sized elements of one Newton candidate's work area (FP32 Jacobian + FP64 iterate)
size_t newton_scratch_bytes(int k, int nterms);
int launch_pchol(int m, const zd* G, double tol2, int* rank_out, zd* Z, zd* gwork, cudaStream_t st);
int launch_newton(const SplitDev& s, int k, int ncand, const zd* Bs, zf* Bs32, const zd* lam0, const zd* Y0, int ldy0,
                  zd c, double rad, double ea, double eb, int maxit, int abandon, double tol, zd* lam_out, zd* Yout, int* ok,
                  int* its, unsigned char* gscratch, cudaStream_t st, const zd* fv_ext = nullptr,
                  double* nstate = nullptr, int steps = 0);
int launch_scale_cols(int rows, int cols, zd* X, int ld, const double* s, int mode, cudaStream_t st);
int launch_scale_rows(int rows, int cols, zd* X, int ld, const double* s, cudaStream_t st);
int launch_candidates(int m, const zd* theta, zd c, double a, zd* lam, cudaStream_t st);
int launch_fill_int(int n, int* p, int v, cudaStream_t st);
int launch_drop_singular(int npts, int n, int L, const int* info, zd* Y, int* active, double* beta, cudaStream_t st);
// double-float refinement with complex64 factors (spmv.cu): a complex value as hi + lo FP32 pairs
struct zdf {
    float hr, hi, lr, li;  // (hr + lr) + i (hi + li)
};
int launch_split_df(int64_t count, const zd* x, zdf* out, cudaStream_t st);
int launch_widen_df(int npts, int n, int L, const zf* B, zdf* Y, cudaStream_t st);
int launch_split_residual_df(const SplitDev& s, int npts, const zdf* tval, int L, const zdf* V, const zdf* Y, zf* D,
                             double* nrm, const int* active, cudaStream_t st);
int launch_refine_update_df(int npts, int n, int L, const zf* D, zdf* Y, double* dmax, double* ymax, const int* active,
                            cudaStream_t st);
int launch_df_to_zd(int npts, int n, int L, void* Y, cudaStream_t st);
// moments.cu: the moments from double-float Y, which it returns to FP64 in place
int launch_moments_df(int n, int L, int N, int K, const zd* coef, void* Y, zd* S, cudaStream_t st);
int launch_rank(int n, const double* sigma, double tol, int* out, cudaStream_t st);
int launch_normalize_columns(int rows, int cols, zd* X, int fix_phase, double* nrm, cudaStream_t st);
int launch_term_spmm(const SplitDev& s, int k, const zd* Q, zd* out, cudaStream_t st);
int launch_eta(const SplitDev& s, int ncand, const zd* lam, const zd* X, double* eta, cudaStream_t st,
               const zd* fv_ext = nullptr);
int launch_select(int ncand, const zd* lam, const double* eta, const int* ok, const zd* G, zd c, double ea, double eb,
                  double eig_tol, int* order, cudaStream_t st);
// polish.cu: residual inverse iteration from P (lambda, x) estimates (x: n x P), T(sigma_p) factored at
// the starting eigenvalues in the precision T of the band LU; eta (P) and its (P) written;
// *max_its_host = outer iterations run.
template <typename T>
int rii_polish(const SplitDev& s, int P, zd* lam, zd* X, double* eta, int* its, double tol, int max_it,
               int* max_its_host, cudaStream_t st);
// dir 0: lam[q], X(:, q), eta[q] <- lam_c[idx[q]], X_c(:, idx[q]), eta_c[idx[q]]; dir 1: the reverse
int launch_rii_move(int n, int P, const int* idx, zd* lam_c, zd* X_c, double* eta_c, zd* lam, zd* X, double* eta,
                    int dir, cudaStream_t st);

// left.cu: conjugate-transpose solve T(z_j)^* W_j = B_j with the factors of T(z_j) (in place on B)
template <typename T>
int launch_band_solve_adjoint(const SplitDev& s, int npts, const cx<T>* ab, const int* ipiv, int L, cx<T>* B,
                              const int* active, cudaStream_t st);
// left eigenvectors Y (n x P) of P pairs (lam, X), Keldysh-normalised (y^* T'(lambda) x = 1); eta:
// left scaled residual before the normalisation, its: steps per pair, *steps_host: steps run
template <typename T>
int left_eigvecs(const SplitDev& s, int P, const zd* lam, const zd* X, zd* Y, double* eta, int* its, double tol,
                 int max_it, int* steps_host, cudaStream_t st);
// Stream-ordered work arrays of one call (cudaMallocAsync on st), freed in stream order on every
// return path.
// pinned host scalars (64 ints a slot) from a process-wide pool: no per-call pinning, and no
// device-wide synchronisation when a slot is given back (host_api.cu)
int* pinned_slot_get();
void pinned_slot_put(int* slot);

struct StreamScratch {
    std::vector<void*> bufs;
    cudaStream_t st;
    explicit StreamScratch(cudaStream_t s) : st(s) {}
    StreamScratch(const StreamScratch&) = delete;
    StreamScratch& operator=(const StreamScratch&) = delete;
    ~StreamScratch() {
        for (void* b : bufs) cudaFreeAsync(b, st);
    }
    template <typename U>
    int get(U** out, size_t count) {
        *out = nullptr;
        void* p = nullptr;
        const cudaError_t e = cudaMallocAsync(&p, sizeof(U) * (count ? count : 1), st);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync", __FILE__, __LINE__);
        bufs.push_back(p);
        *out = static_cast<U*>(p);
        return NEP_OK;
    }
};

// nleigs.cu: rational interpolation on the region (host) and shift-and-invert Arnoldi on its
// linearisation (device)
struct NleigsInterp {
    int d = 0, converged = 0, nsing = 0;
    std::vector<zd> sigma, xi;  // d+1 nodes; poles (xi[0] unused, infinity as (inf, 0))
    std::vector<double> beta;   // d+1 scalings
    std::vector<zd> dd;         // nterms x (d+1): dd[i + nterms j] = d_i^j
};
struct NleigsOut {
    std::vector<zd> lam, X, ritz;
    std::vector<double> eta;
    int steps = 0, restarts = 0, lu_info = 0, polished = 0, polish_its = 0;
};
// Krylov-Schur restarts of the shift-and-invert Arnoldi (NLEIGS, Interpol): none when max_restarts
// is 0 (one cycle); keep: vectors kept at a restart (at least one more than the converged ones);
// a Ritz pair has converged when its residual estimate |b^T s| <= tol |theta|; the restarts stop
// once nev wanted pairs have converged (nev = 0: all wanted pairs of the cycle, at least one)
struct KsOpts {
    int max_restarts = 0;
    int keep = 0;
    double tol = 1e-10;
    int nev = 0;
};
int nleigs_interpolation(const std::vector<FnNode>& nodes, const std::vector<zd>& pool, const std::vector<int>& roots,
                         zd c, double a, double b, double tol, int dmax, int nb, NleigsInterp* out);
// exact: complex64 solves with two FP64-residual corrections; otherwise plain complex64 solves and
// residual inverse iteration on the converged Ritz pairs inside the region
int nleigs_run(const SplitDev& s, const NleigsInterp& it, zd shift, int kmax, const double* start_host, zd c,
               double ea, double eb, double eig_tol, bool exact, NleigsOut* res, cudaStream_t st, bool toar = true,
               const KsOpts& ks = KsOpts());
// Interpol (Sec. 4.4): Krylov on the Chebyshev-basis linearisation of P_d; c: nt x (d+1) coefficients
// of Eq. (polinterpcoef), lambda = alpha theta + beta, sigma the shift in theta
int interpol_run(const SplitDev& s, const std::vector<zd>& c, int d, zd sigma, double alpha, double beta, int kmax,
                 const double* start_host, zd center, double ea, double eb, double eig_tol, bool exact, NleigsOut* res,
                 cudaStream_t st, const KsOpts& ks = KsOpts());
// out (n x nz*nv, column j*nv + k) = sum_i x_i (y_i^* v_k) / (z_j - lam_i)
int apply_resolvent(int n, int P, const zd* lam, const zd* X, const zd* Y, int nz, const zd* z, int nv, const zd* V,
                    zd* out, cudaStream_t st);

}  // namespace nep

// Residual inverse iteration (Sec. 4.1, Algorithm (rii); Neumaier's method) on the device, for
// P eigenpair estimates at once: the polish of contour-method eigenpairs whose scaled residual
// misses a tolerance.
//
// Per pair p, with sigma_p its starting eigenvalue (T(sigma_p) assembled and factored once, in
// the precision of the band LU: complex64 factors for mixed precision, complex128 for FP64), and
// M = T(sigma_p)^{-1} as the band solve applies it. Iteration k, from (lambda_k, x):
//   u_i = A_i x,  r0 = T(lambda_k) x = sum_i f_i(lambda_k) u_i           (FP64)
//   y_0 = M r0,  y_{1+i} = M u_i                        (one band solve with nterms+1 columns)
//   Newton on g(z) = x^* M T(z) x = x^* y_0 + sum_i (f_i(z) - f_i(lambda_k)) x^* y_{1+i},
//             g'(z) = sum_i f_i'(z) x^* y_{1+i}, from lambda_k until |mu| < sqrt(eps) |lambda|
//   eta = ||T(lambda_{k+1}) x|| / (sum_i |f_i| ||A_i||_inf ||x||)   (FP64, Sec. 2 Eq. (sressplit))
//   stop if eta < tol, else x <- (x - v) / ||x - v||,
//             v = M T(lambda_{k+1}) x = y_0 + sum_i (f_i(lambda_{k+1}) - f_i(lambda_k)) y_{1+i}
// The solve is linear, so these columns give both the scalar function of the inner Newton loop
// and the update of the algorithm, with no solve inside the inner loop. M is applied to the small
// residual r0 and to the u_i only with the small weights f_i(z) - f_i(lambda_k): applied to the
// u_i with the full f_i(z), the rounding of a complex64 solve would not cancel where the terms
// of T(z) x do, and would hold lambda at ~1e-7 relative. The iteration's fixed point
// (T(lambda) x = 0) does not depend on M, only its rate does, and the residual and eta are FP64.
#include <algorithm>
#include <vector>

#include "nep_common.cuh"

namespace nep {

// F[i + nterms p] = f_i(lam_p)
__global__ void rii_coeffs_kernel(SplitDev s, int P, const zd* __restrict__ lam, zd* __restrict__ F) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= P * s.nterms) return;
    const int i = t % s.nterms, p = t / s.nterms;
    F[t] = fn_eval(s.fn_nodes, s.fn_coef, s.fn_root[i], lam[p]).f;
}

// active[p] = the factorisation at sigma_p has no zero pivot; its[p] = 0
__global__ void rii_init_kernel(int P, const int* __restrict__ info, int* __restrict__ active, int* __restrict__ its) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    active[p] = info[p] == 0;
    its[p] = 0;
}

// Right-hand sides of pair p, in the solve precision (AX: nterms x P x n, Fk: f_i(lambda_k)):
// column 0 = r0 = sum_i Fk_i (A_i x_p) (formed in FP64), column 1+i = A_i x_p
template <typename T>
__global__ void rii_rhs_kernel(int n, int nt, int P, const zd* __restrict__ AX, const zd* __restrict__ Fk,
                               cx<T>* __restrict__ B) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)P * n) return;
    const int r = (int)(t % n), p = (int)(t / n);
    cx<T>* b = B + (int64_t)p * (nt + 1) * n + r;
    zd r0 = mk(0.0, 0.0);
    for (int i = 0; i < nt; ++i) {
        const zd u = AX[((int64_t)i * P + p) * n + r];
        r0 = fma_(r0, Fk[(int64_t)p * nt + i], u);
        b[(int64_t)(1 + i) * n] = cvt<T>(u);
    }
    b[0] = cvt<T>(r0);
}

// c[p nc + j] = x_p^H y_{p,j} (nc = nterms + 1 columns); one CTA per (j, p)
template <typename T>
__global__ void __launch_bounds__(256) rii_dots_kernel(int n, int nc, const zd* __restrict__ X,
                                                       const cx<T>* __restrict__ B, const int* __restrict__ active,
                                                       zd* __restrict__ c) {
    const int i = blockIdx.x, p = blockIdx.y;
    if (!active[p]) return;
    const zd* x = X + (int64_t)p * n;
    const cx<T>* y = B + ((int64_t)p * nc + i) * n;
    zd acc = mk(0.0, 0.0);
    for (int r = threadIdx.x; r < n; r += blockDim.x) acc = fmac(acc, x[r], cvt<double>(y[r]));
    __shared__ zd part[8];
    for (int o = 16; o > 0; o >>= 1) {
        acc.re += __shfl_xor_sync(0xffffffffu, acc.re, o);
        acc.im += __shfl_xor_sync(0xffffffffu, acc.im, o);
    }
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        zd sum = mk(0.0, 0.0);
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) sum = sum + part[w];
        c[(int64_t)p * nc + i] = sum;
    }
}

// Inner Newton loop of the algorithm on g(z) = c_0 + sum_i (f_i(z) - Fk_i) c_{1+i}, one thread
// per pair
__global__ void rii_scalar_kernel(SplitDev s, int P, const zd* __restrict__ c, const zd* __restrict__ Fk,
                                  const int* __restrict__ active, zd* __restrict__ lam, int inner_max,
                                  double inner_tol) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P || !active[p]) return;
    const int nt = s.nterms, nc = nt + 1;
    zd l = lam[p];
    for (int it = 0; it < inner_max; ++it) {
        zd g = c[(int64_t)p * nc], dg = mk(0.0, 0.0);
        for (int i = 0; i < nt; ++i) {
            const FnEval e = fn_eval(s.fn_nodes, s.fn_coef, s.fn_root[i], l);
            const zd ci = c[(int64_t)p * nc + 1 + i];
            g = g + (e.f - Fk[(int64_t)p * nt + i]) * ci;
            dg = dg + e.df * ci;
        }
        if (dg.re == 0.0 && dg.im == 0.0) break;
        const zd mu = cdiv(g, dg);
        l = l - mu;
        const double am = hypot(mu.re, mu.im), al = hypot(l.re, l.im);
        if ((al > 0.0 && am < inner_tol * al) || (al == 0.0 && am == 0.0) || !(am == am)) break;
    }
    lam[p] = l;
}

// eta_p < tol: the pair is done. Otherwise, unless this is the last iteration,
// x_p <- (x_p - v) / ||x_p - v||, v = y_0 + sum_i (f_i(lambda_p) - Fk_i) y_{1+i}. One CTA per pair.
template <typename T>
__global__ void __launch_bounds__(256) rii_update_kernel(SplitDev s, int n, const zd* __restrict__ lam,
                                                         const double* __restrict__ eta, double tol, int last,
                                                         const zd* __restrict__ Fk, const cx<T>* __restrict__ B,
                                                         zd* __restrict__ X,
                                                         int* __restrict__ active, int* __restrict__ its) {
    const int p = blockIdx.x;
    if (!active[p]) return;
    if (eta[p] < tol) {
        if (threadIdx.x == 0) active[p] = 0;
        return;
    }
    if (last) return;
    __shared__ zd fv[32];  // nterms <= 32
    __shared__ double part[8];
    __shared__ double scale;
    const int nt = s.nterms;
    if (threadIdx.x < nt)
        fv[threadIdx.x] = fn_eval(s.fn_nodes, s.fn_coef, s.fn_root[threadIdx.x], lam[p]).f - Fk[(int64_t)p * nt + threadIdx.x];
    __syncthreads();
    zd* x = X + (int64_t)p * n;
    const cx<T>* y = B + (int64_t)p * (nt + 1) * n;
    double ss = 0.0;
    for (int r = threadIdx.x; r < n; r += blockDim.x) {
        zd v = x[r] - cvt<double>(y[r]);
        for (int i = 0; i < nt; ++i) v = v - fv[i] * cvt<double>(y[(int64_t)(1 + i) * n + r]);
        x[r] = v;
        ss += norm2(v);
    }
    for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = ss;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
        scale = t > 0.0 ? 1.0 / sqrt(t) : 0.0;
        its[p] += 1;
    }
    __syncthreads();
    for (int r = threadIdx.x; r < n; r += blockDim.x) x[r] = scale * x[r];
}

__global__ void rii_count_kernel(int P, const int* __restrict__ active, int* __restrict__ out) {
    int cnt = 0;
    for (int p = threadIdx.x; p < P; p += blockDim.x) cnt += active[p];
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if (threadIdx.x == 0) *out = cnt;
}


template <typename T>
int rii_polish(const SplitDev& s, int P, zd* lam, zd* X, double* eta, int* its, double tol, int max_it,
               int* max_its_host, cudaStream_t st) {
    if (max_its_host) *max_its_host = 0;
    if (P <= 0) return NEP_OK;
    const int n = s.n, nt = s.nterms, kv = s.kl + s.ku;
    StreamScratch w(st);
    zd *F = nullptr, *Fk = nullptr, *AX = nullptr, *c = nullptr;
    const int nc = nt + 1;
    cx<T>*ab = nullptr, *ut = nullptr, *B = nullptr;
    int *ipiv = nullptr, *info = nullptr, *active = nullptr, *cnt = nullptr;
    NEP_TRY(w.get(&F, (size_t)nt * P));
    NEP_TRY(w.get(&Fk, (size_t)nt * P));
    NEP_TRY(w.get(&ab, (size_t)P * n * s.ldab));
    NEP_TRY(w.get(&ipiv, (size_t)P * n));
    NEP_TRY(w.get(&info, (size_t)P));
    NEP_TRY(w.get(&AX, (size_t)nt * n * P));
    NEP_TRY(w.get(&B, (size_t)P * nc * n));
    NEP_TRY(w.get(&c, (size_t)P * nc));
    NEP_TRY(w.get(&active, (size_t)P));
    NEP_TRY(w.get(&cnt, 1));
    if (band_sweeps_fit(s.kl, s.ku)) NEP_TRY(w.get(&ut, (size_t)P * n * (kv + 1)));
    // T(sigma_p) at the starting eigenvalues, factored once
    rii_coeffs_kernel<<<ceil_div(P * nt, 128), 128, 0, st>>>(s, P, lam, F);
    NEP_CHECK_LAUNCH();
    NEP_TRY(launch_assemble<T>(s, P, F, ab, nullptr, nullptr, st));
    NEP_TRY(launch_band_lu<T>(s, P, ab, ipiv, info, nullptr, st));
    if (ut) NEP_TRY(band_transpose_u<T>(s, P, ab, ut, st));
    rii_init_kernel<<<ceil_div(P, 128), 128, 0, st>>>(P, info, active, its);
    NEP_CHECK_LAUNCH();
    const double inner_tol = 1.4901161193847656e-08;  // sqrt(eps) of FP64
    int* host = nullptr;
    host = pinned_slot_get();
    if (!host) { set_error("no pinned host memory"); return NEP_ERR_NOMEM; }
    int rc = NEP_OK, k = 0;
    for (; k <= max_it; ++k) {
        rii_coeffs_kernel<<<ceil_div(P * nt, 128), 128, 0, st>>>(s, P, lam, Fk);
        count_launch();
        if ((rc = launch_term_spmm(s, P, X, AX, st))) break;
        rii_rhs_kernel<T><<<ceil_div((int64_t)P * n, 256), 256, 0, st>>>(n, nt, P, AX, Fk, B);
        count_launch();
        if ((rc = launch_band_solve<T>(s, P, ab, ut, ipiv, nc, B, active, st))) break;
        rii_dots_kernel<T><<<dim3(nc, P), 256, 0, st>>>(n, nc, X, B, active, c);
        count_launch();
        rii_scalar_kernel<<<ceil_div(P, 64), 64, 0, st>>>(s, P, c, Fk, active, lam, 30, inner_tol);
        count_launch();
        if ((rc = launch_eta(s, P, lam, X, eta, st))) break;
        rii_update_kernel<T><<<P, 256, 0, st>>>(s, n, lam, eta, tol, k == max_it, Fk, B, X, active, its);
        count_launch();
        rii_count_kernel<<<1, 32, 0, st>>>(P, active, cnt);
        count_launch();
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) { rc = cuda_fail(e, "rii kernels", __FILE__, __LINE__); break; }
        if (cudaMemcpyAsync(host, cnt, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            rc = NEP_ERR_CUDA;
            break;
        }
        if (*host == 0) break;
    }
    pinned_slot_put(host);
    if (rc) return rc;
    if (max_its_host) *max_its_host = std::min(k, max_it) + 1;  // outer iterations run
    // unit 2-norm, first entry of largest modulus real positive (the pipeline's convention)
    return launch_normalize_columns(n, P, X, 1, nullptr, st);
}

// Packed work block <-> candidate arrays: dir 0 gathers columns idx[q] into q, dir 1 scatters back.
__global__ void rii_move_kernel(int n, int P, const int* __restrict__ idx, zd* __restrict__ lam_c, zd* __restrict__ X_c,
                                double* __restrict__ eta_c, zd* __restrict__ lam, zd* __restrict__ X,
                                double* __restrict__ eta, int dir) {
    const int q = blockIdx.y, c = idx[q];
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
        if (dir == 0) X[(int64_t)q * n + r] = X_c[(int64_t)c * n + r];
        else X_c[(int64_t)c * n + r] = X[(int64_t)q * n + r];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (dir == 0) {
            lam[q] = lam_c[c];
            eta[q] = eta_c[c];
        } else {
            lam_c[c] = lam[q];
            eta_c[c] = eta[q];
        }
    }
}

int launch_rii_move(int n, int P, const int* idx, zd* lam_c, zd* X_c, double* eta_c, zd* lam, zd* X, double* eta,
                    int dir, cudaStream_t st) {
    if (P <= 0) return NEP_OK;
    rii_move_kernel<<<dim3(std::min(ceil_div(n, 256), 64), P), 256, 0, st>>>(n, P, idx, lam_c, X_c, eta_c, lam, X, eta,
                                                                           dir);
    NEP_CHECK_LAUNCH();
    return NEP_OK;
}

template int rii_polish<float>(const SplitDev&, int, zd*, zd*, double*, int*, double, int, int*, cudaStream_t);
template int rii_polish<double>(const SplitDev&, int, zd*, zd*, double*, int*, double, int, int*, cudaStream_t);

}  // namespace nep

// Kernel (c): FP64 split-form residual of the quadrature solves, R_j = V - T(z_j) Y_j, and
// the small kernels of FP64 iterative refinement around the banded solves.
//
// T(z_j) is applied on the union sparsity pattern with the FP64 values the assembly kernel
// produced (the split sum sum_i f_i(z_j) A_i of Sec. 2 Eq. (split), evaluated once per point);
// this is the residual r = sum_i f_i(lambda) A_i x of Sec. 5 (one SpMV per term in the
// paper's implementation, one fused pass here). One CTA handles 256 rows of one
// (point, right-hand side) pair so that the infinity norms of R, Y and V it produces reduce
// inside the CTA to one atomic maximum each.
//
// Refinement sweep per point (all points in one launch each, points that have converged
// are skipped through the `active` mask):
//   R = V - T Y (FP64);  beta = max_l ||R_l||_inf / (||T||_inf ||Y_l||_inf + ||V_l||_inf);
//   D = T^{-1} R with the stored factors (complex64 or complex128);  Y += D (FP64);
//   stop when beta <= tol and (||D||/||Y|| <= step_tol or ||D||/||Y|| stopped halving).
#include "df_arith.cuh"
#include "nep_common.cuh"

namespace nep {

__device__ __forceinline__ void atomic_max_nonneg_d(double* addr, double v) {
    atomicMax(reinterpret_cast<unsigned long long*>(addr), (unsigned long long)__double_as_longlong(v));
}

__device__ __forceinline__ double block_max(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    if (w == 0) {
        v = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    }
    return v;
}

// nrm[(j*L + l)*3 + {0,1,2}] = max |R|, max |Y|, max |V| of column l of point j.
__global__ void __launch_bounds__(256) split_residual_kernel(const int64_t* __restrict__ rowptr,
                                                             const int32_t* __restrict__ col, int64_t nnz, int n,
                                                             int L, const zd* __restrict__ tval,
                                                             const zd* __restrict__ V, const zd* __restrict__ Y,
                                                             zd* __restrict__ R, double* __restrict__ nrm,
                                                             const int* __restrict__ active) {
    __shared__ double red[32];
    const int jl = blockIdx.y;
    const int j = jl / L, l = jl % L;
    if (active && !active[j]) return;
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    const zd* y = Y + (int64_t)jl * n;
    const zd* tv = tval + (int64_t)j * nnz;
    double mr = 0.0, my = 0.0, mv = 0.0;
    if (r < n) {
        const zd v = V[(int64_t)l * n + r];
        zd acc = v;
        for (int64_t e = rowptr[r]; e < rowptr[r + 1]; ++e) acc = fms(acc, tv[e], y[col[e]]);
        R[(int64_t)jl * n + r] = acc;
        // squared moduli: the maxima are taken first and rooted once (FP64 issue is scarce)
        mr = norm2(acc);
        my = norm2(y[r]);
        mv = norm2(v);
    }
    if (!nrm) return;
    mr = block_max(mr, red);
    if (threadIdx.x == 0) atomic_max_nonneg_d(nrm + (int64_t)jl * 3 + 0, sqrt(mr));
    my = block_max(my, red);
    if (threadIdx.x == 0) atomic_max_nonneg_d(nrm + (int64_t)jl * 3 + 1, sqrt(my));
    mv = block_max(mv, red);
    if (threadIdx.x == 0) atomic_max_nonneg_d(nrm + (int64_t)jl * 3 + 2, sqrt(mv));
}

int launch_split_residual(const SplitDev& s, int npts, const zd* tval, int L, const zd* V, const zd* Y, zd* R,
                          double* nrm, const int* active, cudaStream_t st) {
    if (npts <= 0 || L <= 0) return NEP_OK;
    if (nrm) NEP_CUDA(cudaMemsetAsync(nrm, 0, sizeof(double) * 3 * npts * L, st));
    dim3 grid(ceil_div(s.n, 256), npts * L);
    split_residual_kernel<<<grid, 256, 0, st>>>(s.rowptr, s.col, s.nnz, s.n, L, tval, V, Y, R, nrm, active);
    NEP_CHECK_LAUNCH();
    return NEP_OK;
}

// B_j = V for every point (converted to the solve precision)
template <typename T>
__global__ void convert_rhs_kernel(int npts, int64_t nl, const zd* __restrict__ V, cx<T>* __restrict__ B) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nl * npts) return;
    B[i] = cvt<T>(V[i % nl]);
}

template <typename T>
__global__ void widen_kernel(int64_t total, const cx<T>* __restrict__ B, zd* __restrict__ Y) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    Y[i] = cvt<double>(B[i]);
}

template <typename T>
__global__ void prepare_kernel(int64_t per_point, int npts, const zd* __restrict__ R, cx<T>* __restrict__ D,
                               const int* __restrict__ active) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= per_point * npts) return;
    const int j = (int)(i / per_point);
    if (active && !active[j]) return;
    D[i] = cvt<T>(R[i]);
}

// Y += D; dmax[j] = max |D|, ymax[j] = max |Y| over the point's block.
template <typename T>
__global__ void __launch_bounds__(256) update_kernel(int64_t per_point, const cx<T>* __restrict__ D,
                                                     zd* __restrict__ Y, double* __restrict__ dmax,
                                                     double* __restrict__ ymax, const int* __restrict__ active) {
    __shared__ double red[32];
    const int j = blockIdx.y;
    if (active && !active[j]) return;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double md = 0.0, my = 0.0;
    if (i < per_point) {
        const int64_t g = (int64_t)j * per_point + i;
        const zd d = cvt<double>(D[g]);
        const zd y = Y[g] + d;
        Y[g] = y;
        md = norm2(d);
        my = norm2(y);
    }
    md = block_max(md, red);
    if (threadIdx.x == 0) atomic_max_nonneg_d(dmax + j, sqrt(md));
    my = block_max(my, red);
    if (threadIdx.x == 0) atomic_max_nonneg_d(ymax + j, sqrt(my));
}

// One thread per point: backward error of the residual just measured, stop rule, counters.
__global__ void decide_kernel(int npts, int L, int sweep, int max_sweeps, double tol, double step_tol, int extrapolate,
                              const double* __restrict__ nrm, const double* __restrict__ tnorm,
                              const double* __restrict__ dmax, const double* __restrict__ ymax,
                              double* __restrict__ prev, double* __restrict__ beta_out, int* __restrict__ active,
                              int* __restrict__ sweeps, int* __restrict__ nactive) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= npts || !active[j]) return;
    double beta = 0.0;
    for (int l = 0; l < L; ++l) {
        const double* q = nrm + ((int64_t)j * L + l) * 3;
        const double den = tnorm[j] * q[1] + q[2];
        const double b = den > 0 ? q[0] / den : 0.0;
        beta = fmax(beta, b);
    }
    const double d = ymax[j] > 0 ? dmax[j] / ymax[j] : 0.0;
    beta_out[j] = beta;
    sweeps[j] = sweep + 1;
    // prev starts at 0, read as "no previous correction". Converged: backward error at the target
    // and either the correction is at the FP64 level or it stopped halving. With extrapolate set,
    // a sweep is also saved when the contraction seen so far (d / prev) puts the next correction
    // at the FP64 level (the error left after this one): a shortcut, not a different target
    const double pv = prev[j];
    const bool small = d <= step_tol || (extrapolate && pv > 0 && d <= 0.5 * pv && d * (d / pv) <= step_tol);
    const bool conv = beta <= tol && (small || (pv > 0 && d > 0.5 * pv));
    prev[j] = d;
    if (conv || sweep + 1 >= max_sweeps) {
        active[j] = 0;
    } else {
        atomicAdd(nactive, 1);
    }
}

// A node whose factorisation met an exactly zero pivot (info != 0: T(z_j) singular, an eigenvalue
// on the contour at that node) has no resolvent to sample: its Y_j is set to zero, so it drops out
// of the moment sums, and it takes no refinement sweeps. One CTA per point.
__global__ void drop_singular_kernel(int npts, int64_t nl, const int* __restrict__ info, zd* __restrict__ Y,
                                     int* __restrict__ active, double* __restrict__ beta) {
    const int j = blockIdx.x;
    if (!info[j]) return;
    for (int64_t e = threadIdx.x; e < nl; e += blockDim.x) Y[(int64_t)j * nl + e] = mk(0.0, 0.0);
    if (threadIdx.x == 0) {
        active[j] = 0;
        beta[j] = 0.0;
    }
}
int launch_drop_singular(int npts, int n, int L, const int* info, zd* Y, int* active, double* beta, cudaStream_t st) {
    if (npts <= 0) return NEP_OK;
    drop_singular_kernel<<<npts, 256, 0, st>>>(npts, (int64_t)n * L, info, Y, active, beta);
    NEP_CHECK_LAUNCH();
    return NEP_OK;
}

template <typename T>
int launch_convert_rhs(int npts, int n, int L, const zd* V, cx<T>* B, cudaStream_t st) {
    const int64_t nl = (int64_t)n * L;
    convert_rhs_kernel<T><<<ceil_div(nl * npts, 256), 256, 0, st>>>(npts, nl, V, B);
    NEP_CHECK_LAUNCH();
    return NEP_OK;
}
template <typename T>
int launch_widen(int npts, int n, int L, const cx<T>* B, zd* Y, cudaStream_t st) {
    const int64_t total = (int64_t)npts * n * L;
    widen_kernel<T><<<ceil_div(total, 256), 256, 0, st>>>(total, B, Y);
    NEP_CHECK_LAUNCH();
    return NEP_OK;
}
template <typename T>
int launch_refine_prepare(int npts, int n, int L, const zd* R, cx<T>* D, const int* active, cudaStream_t st) {
    const int64_t pp = (int64_t)n * L;
    prepare_kernel<T><<<ceil_div(pp * npts, 256), 256, 0, st>>>(pp, npts, R, D, active);
    NEP_CHECK_LAUNCH();
    return NEP_OK;
}
template <typename T>
int launch_refine_update(int npts, int n, int L, const cx<T>* D, zd* Y, double* dmax, double* ymax,
                         const int* active, cudaStream_t st) {
    const int64_t pp = (int64_t)n * L;
    NEP_CUDA(cudaMemsetAsync(dmax, 0, sizeof(double) * npts, st));
    NEP_CUDA(cudaMemsetAsync(ymax, 0, sizeof(double) * npts, st));
    dim3 grid(ceil_div(pp, 256), npts);
    update_kernel<T><<<grid, 256, 0, st>>>(pp, D, Y, dmax, ymax, active);
    NEP_CHECK_LAUNCH();
    return NEP_OK;
}
int launch_refine_decide(int npts, int L, int sweep, int max_sweeps, double tol, double step_tol, int extrapolate,
                         const double* nrm,
                         const double* tnorm, const double* dmax, const double* ymax, double* prev, double* beta,
                         int* active, int* sweeps, int* nactive, cudaStream_t st) {
    NEP_CUDA(cudaMemsetAsync(nactive, 0, sizeof(int), st));
    decide_kernel<<<ceil_div(npts, 128), 128, 0, st>>>(npts, L, sweep, max_sweeps, tol, step_tol, extrapolate, nrm,
                                                      tnorm, dmax,
                                                      ymax, prev, beta, active, sweeps, nactive);
    NEP_CHECK_LAUNCH();
    return NEP_OK;
}

#define INST(T)                                                                                            \
    template int launch_convert_rhs<T>(int, int, int, const zd*, cx<T>*, cudaStream_t);                   \
    template int launch_widen<T>(int, int, int, const cx<T>*, zd*, cudaStream_t);                        \
    template int launch_refine_prepare<T>(int, int, int, const zd*, cx<T>*, const int*, cudaStream_t);   \
    template int launch_refine_update<T>(int, int, int, const cx<T>*, zd*, double*, double*, const int*, \
                                         cudaStream_t);
INST(float)
INST(double)
#undef INST


// ------------------------------------------------------------------ double-float refinement
// With complex64 factors the refinement keeps Y as an unevaluated sum hi + lo of two FP32 values per
// real component (about 48 significant bits) and forms the residual V - T(z_j) Y in that arithmetic:
// error-free products (p = a b, e = fma(a, b, -p)) and sums (Knuth's two-sum). The residual's
// rounding is then about 2^-48 sum |t| |y|, far below the backward-error target of the refinement,
// and the work runs on the FP32 pipe, about 68 times the FP64 rate of this part. The FP64 values of
// T(z_j) and V are split once per pass; Y returns to FP64 for the moments.

__device__ __forceinline__ float block_max_f(float v, float* red) {
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    if (w == 0) {
        v = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0f;
        for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    }
    return v;
}

// out[i] = x[i] as hi + lo FP32 pairs
__global__ void split_df_kernel(int64_t count, const zd* __restrict__ x, zdf* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const zd v = x[i];
    const float hr = (float)v.re, hi = (float)v.im;
    out[i] = zdf{hr, hi, (float)(v.re - (double)hr), (float)(v.im - (double)hi)};
}

// Y = B (the first solve), lo parts zero
__global__ void widen_df_kernel(int64_t total, const zf* __restrict__ B, zdf* __restrict__ Y) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    const zf b = B[i];
    Y[i] = zdf{b.re, b.im, 0.0f, 0.0f};
}

// D_j = V - T(z_j) Y_j rounded to complex64 (the next correction's right-hand side), and the maxima
// of |R|, |Y|, |V| per (point, column) as split_residual_kernel gives them
__global__ void __launch_bounds__(256) split_residual_df_kernel(const int64_t* __restrict__ rowptr,
                                                                const int32_t* __restrict__ col, int64_t nnz, int n,
                                                                int L, const zdf* __restrict__ tval,
                                                                const zdf* __restrict__ V, const zdf* __restrict__ Y,
                                                                zf* __restrict__ D, double* __restrict__ nrm,
                                                                const int* __restrict__ active) {
    __shared__ float red[32];
    const int jl = blockIdx.y;
    const int j = jl / L, l = jl % L;
    if (active && !active[j]) return;
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    const zdf* y = Y + (int64_t)jl * n;
    const zdf* tv = tval + (int64_t)j * nnz;
    float mr = 0.0f, my = 0.0f, mv = 0.0f;
    if (r < n) {
        const zdf v = V[(int64_t)l * n + r];
        float rh = v.hr, rl = v.lr, ih = v.hi, il = v.li;
        for (int64_t e = rowptr[r]; e < rowptr[r + 1]; ++e) {
            const zdf t = tv[e], x = y[col[e]];
            df_fms(rh, rl, t.hr, t.lr, x.hr, x.lr);    // re -= t.re x.re
            df_fms(rh, rl, -t.hi, -t.li, x.hi, x.li);  // re += t.im x.im
            df_fms(ih, il, t.hr, t.lr, x.hi, x.li);    // im -= t.re x.im
            df_fms(ih, il, t.hi, t.li, x.hr, x.lr);    // im -= t.im x.re
        }
        D[(int64_t)jl * n + r] = mk(rh + rl, ih + il);
        const zdf yr = y[r];
        mr = hypotf(rh, ih);
        my = hypotf(yr.hr, yr.hi);
        mv = hypotf(v.hr, v.hi);
    }
    if (!nrm) return;
    mr = block_max_f(mr, red);
    if (threadIdx.x == 0) atomic_max_nonneg_d(nrm + (int64_t)jl * 3 + 0, (double)mr);
    my = block_max_f(my, red);
    if (threadIdx.x == 0) atomic_max_nonneg_d(nrm + (int64_t)jl * 3 + 1, (double)my);
    mv = block_max_f(mv, red);
    if (threadIdx.x == 0) atomic_max_nonneg_d(nrm + (int64_t)jl * 3 + 2, (double)mv);
}

// Y += D in double-float; dmax[j] = max |D|, ymax[j] = max |Y| over the point's block
__global__ void __launch_bounds__(256) update_df_kernel(int64_t per_point, const zf* __restrict__ D,
                                                        zdf* __restrict__ Y, double* __restrict__ dmax,
                                                        double* __restrict__ ymax, const int* __restrict__ active) {
    __shared__ float red[32];
    const int j = blockIdx.y;
    if (active && !active[j]) return;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float md = 0.0f, my = 0.0f;
    if (i < per_point) {
        const int64_t g = (int64_t)j * per_point + i;
        const zf d = D[g];
        zdf y = Y[g];
        df_add1(y.hr, y.lr, d.re);
        df_add1(y.hi, y.li, d.im);
        Y[g] = y;
        md = hypotf(d.re, d.im);
        my = hypotf(y.hr, y.hi);
    }
    md = block_max_f(md, red);
    if (threadIdx.x == 0) atomic_max_nonneg_d(dmax + j, (double)md);
    my = block_max_f(my, red);
    if (threadIdx.x == 0) atomic_max_nonneg_d(ymax + j, (double)my);
}

// Y (double-float) -> FP64 in place
__global__ void df_to_zd_kernel(int64_t total, void* __restrict__ Y) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    const zdf y = reinterpret_cast<const zdf*>(Y)[i];
    reinterpret_cast<zd*>(Y)[i] = mk((double)y.hr + (double)y.lr, (double)y.hi + (double)y.li);
}

int launch_split_df(int64_t count, const zd* x, zdf* out, cudaStream_t st) {
    if (count <= 0) return NEP_OK;
    split_df_kernel<<<ceil_div(count, 256), 256, 0, st>>>(count, x, out);
    NEP_CHECK_LAUNCH();
    return NEP_OK;
}
int launch_widen_df(int npts, int n, int L, const zf* B, zdf* Y, cudaStream_t st) {
    const int64_t total = (int64_t)npts * n * L;
    widen_df_kernel<<<ceil_div(total, 256), 256, 0, st>>>(total, B, Y);
    NEP_CHECK_LAUNCH();
    return NEP_OK;
}
int launch_split_residual_df(const SplitDev& s, int npts, const zdf* tval, int L, const zdf* V, const zdf* Y, zf* D,
                             double* nrm, const int* active, cudaStream_t st) {
    if (npts <= 0 || L <= 0) return NEP_OK;
    if (nrm) NEP_CUDA(cudaMemsetAsync(nrm, 0, sizeof(double) * 3 * npts * L, st));
    dim3 grid(ceil_div(s.n, 256), npts * L);
    split_residual_df_kernel<<<grid, 256, 0, st>>>(s.rowptr, s.col, s.nnz, s.n, L, tval, V, Y, D, nrm, active);
    NEP_CHECK_LAUNCH();
    return NEP_OK;
}
int launch_refine_update_df(int npts, int n, int L, const zf* D, zdf* Y, double* dmax, double* ymax, const int* active,
                            cudaStream_t st) {
    if (npts <= 0) return NEP_OK;
    const int64_t per_point = (int64_t)n * L;
    NEP_CUDA(cudaMemsetAsync(dmax, 0, sizeof(double) * npts, st));
    NEP_CUDA(cudaMemsetAsync(ymax, 0, sizeof(double) * npts, st));
    dim3 grid(ceil_div(per_point, 256), npts);
    update_df_kernel<<<grid, 256, 0, st>>>(per_point, D, Y, dmax, ymax, active);
    NEP_CHECK_LAUNCH();
    return NEP_OK;
}
int launch_df_to_zd(int npts, int n, int L, void* Y, cudaStream_t st) {
    const int64_t total = (int64_t)npts * n * L;
    if (total <= 0) return NEP_OK;
    df_to_zd_kernel<<<ceil_div(total, 256), 256, 0, st>>>(total, Y);
    NEP_CHECK_LAUNCH();
    return NEP_OK;
}

}  // namespace nep

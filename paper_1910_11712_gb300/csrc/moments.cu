// Kernel (d): contour moments and the block Hankel matrices, FP64.
//
// By Keldysh's theorem (Sec. 2 Eq. (resolvent)) the quadrature of zeta^k T(z)^{-1} V over
// Gamma keeps only the eigenvalues inside Gamma. With the trapezoid nodes/weights:
//   S_k = sum_j w_j zeta_j^k Y_j  (Y_j = T(z_j)^{-1} V),    mu_k = V^H S_k,    k < 2M,
//   H = [mu_{a+b}],  H< = [mu_{a+b+1}]  (a, b < M; LM x LM, column-major).
// moments_kernel: one thread per entry (i, l) of the n x L block reads Y_j(i, l) once for
// every point j (ascending) and keeps the K = 2M complex accumulators in registers; the
// coefficients c_jk = w_j zeta_j^k sit in shared memory. Arithmetic is FP64 (1.75 FMA/clk/SM
// on this part), so with 2M*4 FMAs per 16 bytes read the kernel is bound by FP64 issue,
// not by HBM.
// vh_partial_kernel + vh_reduce_kernel: mu_k = V^H S_k over row chunks with a fixed-order
// reduction (no atomics), so results do not depend on scheduling.
#include <algorithm>

#include "df_arith.cuh"
#include "nep_common.cuh"

namespace nep {

template <int K>
__global__ void __launch_bounds__(256) moments_kernel(int64_t nl, int N, const zd* __restrict__ coef,
                                                      const zd* __restrict__ Y, zd* __restrict__ S) {
    extern __shared__ zd cs[];  // N x K
    for (int t = threadIdx.x; t < N * K; t += blockDim.x) cs[t] = coef[(t / K) + (int64_t)N * (t % K)];
    __syncthreads();
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nl) return;
    zd acc[K];
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] = mk(0.0, 0.0);
    for (int j = 0; j < N; ++j) {
        const zd y = Y[(int64_t)j * nl + e];
#pragma unroll
        for (int k = 0; k < K; ++k) acc[k] = fma_(acc[k], cs[j * K + k], y);
    }
#pragma unroll
    for (int k = 0; k < K; ++k) S[(int64_t)k * nl + e] = acc[k];
}

// generic K (loop over k in chunks of 8 accumulators)
__global__ void __launch_bounds__(256) moments_kernel_generic(int64_t nl, int N, int K, const zd* __restrict__ coef,
                                                              const zd* __restrict__ Y, zd* __restrict__ S) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nl) return;
    for (int k0 = 0; k0 < K; k0 += 8) {
        zd acc[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) acc[k] = mk(0.0, 0.0);
        for (int j = 0; j < N; ++j) {
            const zd y = Y[(int64_t)j * nl + e];
#pragma unroll
            for (int k = 0; k < 8; ++k)
                if (k0 + k < K) acc[k] = fma_(acc[k], coef[j + (int64_t)N * (k0 + k)], y);
        }
#pragma unroll
        for (int k = 0; k < 8; ++k)
            if (k0 + k < K) S[(int64_t)(k0 + k) * nl + e] = acc[k];
    }
}

int launch_moments(int n, int L, int N, int K, const zd* coef, const zd* Y, zd* S, cudaStream_t st) {
    const int64_t nl = (int64_t)n * L;
    const int blocks = ceil_div(nl, 256);
    const size_t sm = sizeof(zd) * (size_t)N * K;
    if (K == 16 && sm <= 96 * 1024) {
        NEP_CUDA(allow_max_dynamic_smem(moments_kernel<16>));
        moments_kernel<16><<<blocks, 256, sm, st>>>(nl, N, coef, Y, S);
    } else if (K == 8 && sm <= 96 * 1024) {
        NEP_CUDA(allow_max_dynamic_smem(moments_kernel<8>));
        moments_kernel<8><<<blocks, 256, sm, st>>>(nl, N, coef, Y, S);
    } else {
        moments_kernel_generic<<<blocks, 256, 0, st>>>(nl, N, K, coef, Y, S);
    }
    NEP_CHECK_LAUNCH();
    return NEP_OK;
}

// The moments from Y held as double-float pairs (complex64 factors, the refinement's form): the
// accumulation in double-float arithmetic (coefficients split once per CTA), S written in FP64,
// and each Y element returned to FP64 in place after it is read.
template <int K>
__global__ void __launch_bounds__(256) moments_df_kernel(int64_t nl, int N, const zd* __restrict__ coef,
                                                         void* __restrict__ Y, zd* __restrict__ S) {
    extern __shared__ zdf csf[];  // N x K
    for (int t = threadIdx.x; t < N * K; t += blockDim.x) {
        const zd c = coef[(t / K) + (int64_t)N * (t % K)];
        const float hr = (float)c.re, hi = (float)c.im;
        csf[t] = zdf{hr, hi, (float)(c.re - (double)hr), (float)(c.im - (double)hi)};
    }
    __syncthreads();
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nl) return;
    float rh[K], rl[K], ih[K], il[K];
#pragma unroll
    for (int k = 0; k < K; ++k) rh[k] = rl[k] = ih[k] = il[k] = 0.0f;
    zdf* Yd = reinterpret_cast<zdf*>(Y);
    zd* Yz = reinterpret_cast<zd*>(Y);
    for (int j = 0; j < N; ++j) {
        const zdf y = Yd[(int64_t)j * nl + e];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const zdf c = csf[j * K + k];
            df_fma(rh[k], rl[k], c.hr, c.lr, y.hr, y.lr);    // re += c.re y.re
            df_fms(rh[k], rl[k], c.hi, c.li, y.hi, y.li);    // re -= c.im y.im
            df_fma(ih[k], il[k], c.hr, c.lr, y.hi, y.li);    // im += c.re y.im
            df_fma(ih[k], il[k], c.hi, c.li, y.hr, y.lr);    // im += c.im y.re
        }
        Yz[(int64_t)j * nl + e] = mk((double)y.hr + (double)y.lr, (double)y.hi + (double)y.li);
    }
#pragma unroll
    for (int k = 0; k < K; ++k) S[(int64_t)k * nl + e] = mk((double)rh[k] + (double)rl[k], (double)ih[k] + (double)il[k]);
}

int launch_moments_df(int n, int L, int N, int K, const zd* coef, void* Y, zd* S, cudaStream_t st) {
    const int64_t nl = (int64_t)n * L;
    const int blocks = ceil_div(nl, 256);
    const size_t sm = sizeof(zdf) * (size_t)N * K;
    if (K == 16 && sm <= 96 * 1024) {
        NEP_CUDA(allow_max_dynamic_smem(moments_df_kernel<16>));
        moments_df_kernel<16><<<blocks, 256, sm, st>>>(nl, N, coef, Y, S);
    } else if (K == 8 && sm <= 96 * 1024) {
        NEP_CUDA(allow_max_dynamic_smem(moments_df_kernel<8>));
        moments_df_kernel<8><<<blocks, 256, sm, st>>>(nl, N, coef, Y, S);
    } else {  // other moment counts: Y to FP64, then the FP64 moments
        NEP_TRY(launch_df_to_zd(N, n, L, Y, st));
        return launch_moments(n, L, N, K, coef, reinterpret_cast<const zd*>(Y), S, st);
    }
    NEP_CHECK_LAUNCH();
    return NEP_OK;
}

// part[(chunk*K + k)*L*L + a + L*b] = sum_{i in chunk} conj(V(i,a)) S_k(i,b)
constexpr int VH_ROWS = 128;
__global__ void __launch_bounds__(256) vh_partial_kernel(int n, int L, int K, const zd* __restrict__ V,
                                                         const zd* __restrict__ S, zd* __restrict__ part) {
    extern __shared__ zd sh[];
    zd* vs = sh;                    // VH_ROWS x L
    zd* ss = sh + VH_ROWS * L;      // VH_ROWS x L
    const int chunk = blockIdx.x, k = blockIdx.y;
    const int i0 = chunk * VH_ROWS;
    const int rows = min(VH_ROWS, n - i0);
    const zd* Sk = S + (int64_t)k * n * L;
    for (int t = threadIdx.x; t < VH_ROWS * L; t += blockDim.x) {
        const int i = t % VH_ROWS, a = t / VH_ROWS;
        vs[t] = i < rows ? V[(int64_t)a * n + i0 + i] : mk(0.0, 0.0);
        ss[t] = i < rows ? Sk[(int64_t)a * n + i0 + i] : mk(0.0, 0.0);
    }
    __syncthreads();
    for (int ab = threadIdx.x; ab < L * L; ab += blockDim.x) {
        const int a = ab % L, b = ab / L;
        zd acc = mk(0.0, 0.0);
        for (int i = 0; i < rows; ++i) acc = fmac(acc, vs[a * VH_ROWS + i], ss[b * VH_ROWS + i]);
        part[((int64_t)chunk * K + k) * L * L + ab] = acc;
    }
}

__global__ void vh_reduce_kernel(int nchunks, int LL, int K, const zd* __restrict__ part, zd* __restrict__ mu) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= K * LL) return;
    const int k = t / LL, ab = t % LL;
    zd acc = mk(0.0, 0.0);
    for (int c = 0; c < nchunks; ++c) acc = acc + part[((int64_t)c * K + k) * LL + ab];
    mu[t] = acc;
}

int launch_vh_times(int n, int L, int K, const zd* V, const zd* S, zd* mu, zd* part, cudaStream_t st) {
    const int nch = ceil_div(n, VH_ROWS);
    const size_t sm = sizeof(zd) * 2 * VH_ROWS * L;
    if (sm > 200 * 1024) return NEP_ERR_UNSUPPORTED;
    NEP_CUDA(allow_max_dynamic_smem(vh_partial_kernel));
    vh_partial_kernel<<<dim3(nch, K), 256, sm, st>>>(n, L, K, V, S, part);
    NEP_CHECK_LAUNCH();
    vh_reduce_kernel<<<ceil_div(K * L * L, 256), 256, 0, st>>>(nch, L * L, K, part, mu);
    NEP_CHECK_LAUNCH();
    return NEP_OK;
}

// H(a*L + i, b*L + c) = mu_{a+b}(i, c), Hs likewise with mu_{a+b+1}; mu_k is L x L column-major.
__global__ void hankel_build_kernel(int L, int M, const zd* __restrict__ mu, zd* __restrict__ H, zd* __restrict__ Hs) {
    const int LM = L * M;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= LM * LM) return;
    const int row = t % LM, colm = t / LM;
    const int a = row / L, i = row % L, b = colm / L, c = colm % L;
    H[t] = mu[(int64_t)(a + b) * L * L + i + (int64_t)L * c];
    Hs[t] = mu[(int64_t)(a + b + 1) * L * L + i + (int64_t)L * c];
}

int launch_hankel_build(int L, int M, const zd* mu, zd* H, zd* Hs, cudaStream_t st) {
    const int LM = L * M;
    hankel_build_kernel<<<ceil_div(LM * LM, 256), 256, 0, st>>>(L, M, mu, H, Hs);
    NEP_CHECK_LAUNCH();
    return NEP_OK;
}


// ------------------------------------------------------------------ conjugate symmetry
// x <- 2 Re x (the sum of a term and its complex conjugate), count entries.
__global__ void double_real_kernel(int64_t count, zd* __restrict__ x) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < count) x[t] = mk(2.0 * x[t].re, 0.0);
}
int launch_double_real(int64_t count, zd* x, cudaStream_t st) {
    if (count <= 0) return NEP_OK;
    double_real_kernel<<<(int)((count + 255) / 256), 256, 0, st>>>(count, x);
    NEP_CHECK_LAUNCH();
    return NEP_OK;
}

// *out = number of entries of x with a nonzero imaginary part.
__global__ void count_imag_kernel(int64_t count, const zd* __restrict__ x, int* __restrict__ out) {
    int c = 0;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < count; t += (int64_t)gridDim.x * blockDim.x)
        c += x[t].im != 0.0;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}
int launch_count_imag(int64_t count, const zd* x, int* out, cudaStream_t st) {
    NEP_CUDA(cudaMemsetAsync(out, 0, sizeof(int), st));
    if (count <= 0) return NEP_OK;
    const int blocks = (int)std::min<int64_t>((count + 255) / 256, 1024);
    count_imag_kernel<<<blocks, 256, 0, st>>>(count, x, out);
    NEP_CHECK_LAUNCH();
    return NEP_OK;
}

}  // namespace nep

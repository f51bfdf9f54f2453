// Left eigenvectors and the resolvent (Sec. 2 Eqs. (nep-left), (resolvent); Sec. 3.2.5 asks for
// both, and Sec. 4.5.4 applies the conjugate transpose of a factored operator with the same
// factorisation), on the band LU of the path.
//
// Left eigenvectors factor T(lambda)^* itself (assembled from the split's column view with the
// bandwidths swapped) and run the path's LU and substitution sweeps on it. The conjugate-transpose
// solve below serves callers that must reuse the factors of T.
//
// Conjugate-transpose solve T^* w = b from the factors of T. The LU applies, at step c, the
// interchange P_c of rows c and ipiv[c], then the elementary L_c = I + l_c e_c^T (l_c: the
// stored multipliers of column c), so T = P_0 L_0 P_1 L_1 ... P_{n-1} L_{n-1} U and
//   w = P_0 L_0^{-*} P_1 L_1^{-*} ... P_{n-1} L_{n-1}^{-*} U^{-*} b.
// U^* is lower triangular with the rows of U (as stored) for its columns: a forward pass
// z_c = b_c / conj U(c,c), b_{c+t} -= conj U(c,c+t) z_c for t <= kl+ku. Then for c = n-1 .. 0:
// z_c -= l_c^* z(c+1 .. c+kl) (a dot product) and z_c <-> z_{ipiv[c]}.
// An exactly zero pivot (the factor of an exactly singular matrix, info != 0) stands for a
// tiny one, the inverse-iteration convention: the solution is then dominated by the null
// direction instead of being infinite.
//
// Bands whose staged chunks fit in 200 KB of shared memory (kl+ku up to ~190 for complex128,
// ~380 for complex64): one CTA per (point, right-hand side), a compute warp and a producer
// warp. The producer stages the next chunk of 32 steps (U rows, or L columns and pivots) in
// shared memory with cp.async while the compute warp runs the current one; the live entries of
// the solution sit in a shared ring of R slots, refilled from global memory 32 steps ahead.
// One warp barrier per step, one CTA barrier per chunk. Wider bands: one warp per (point,
// right-hand side), in place in global memory.
#include <algorithm>
#include <vector>

#include "band_util.cuh"

namespace nep {

template <typename T>
__device__ __forceinline__ cx<T> recip_conj_or_tiny(cx<T> u) {
    // 1 / conj(u); a zero pivot stands for a tiny one
    if (u.re == T(0) && u.im == T(0)) return mk<T>(sizeof(T) == 4 ? T(1e20) : T(1e100), T(0));
    return conj(pivot_recip(u));
}

// ------------------------------------------------------------------ wide bands
template <typename T>
__global__ void __launch_bounds__(32) band_solve_adjoint_glb_kernel(int n, int kl, int ku, int ldab,
                                                                    const cx<T>* __restrict__ ab_all,
                                                                    const int* __restrict__ ipiv_all, int L,
                                                                    cx<T>* __restrict__ B_all,
                                                                    const int* __restrict__ active) {
    const int j = blockIdx.x, col = blockIdx.y, lane = threadIdx.x;
    if (active && !active[j]) return;
    const int kv = kl + ku;
    const cx<T>* ab = ab_all + (int64_t)j * n * ldab;
    const int* ipiv = ipiv_all + (int64_t)j * n;
    cx<T>* b = B_all + ((int64_t)j * L + col) * n;
    for (int c = 0; c < n; ++c) {
        const cx<T>* urow = ab + (int64_t)c * ldab;  // U(c, c+t) = urow[t]
        const cx<T> zc = b[c] * recip_conj_or_tiny(urow[0]);
        __syncwarp();
        for (int t = 1 + lane; t <= kv && c + t < n; t += 32) b[c + t] = fms(b[c + t], conj(urow[t]), zc);
        if (lane == 0) b[c] = zc;
        __syncwarp();
    }
    for (int c = n - 1; c >= 0; --c) {
        const cx<T>* lcol = ab + (int64_t)c * ldab + kv + 1;  // L(c+1+i, c) = lcol[i]
        cx<T> acc = mk<T>(0, 0);
        for (int i = lane; i < kl && c + 1 + i < n; i += 32) acc = fmac(acc, lcol[i], b[c + 1 + i]);
        for (int o = 16; o > 0; o >>= 1) {
            acc.re += __shfl_xor_sync(0xffffffffu, acc.re, o);
            acc.im += __shfl_xor_sync(0xffffffffu, acc.im, o);
        }
        if (lane == 0) {
            const cx<T> zc = b[c] - acc;
            int p = ipiv[c];
            if (p < c || p > c + kl || p >= n) p = c;  // a pivot outside the window is ignored
            if (p != c) b[c] = b[p];
            b[p] = zc;
        }
        __syncwarp();
    }
}

// ------------------------------------------------------------------ narrow bands
constexpr int kAdjCH = 32;  // steps per staged chunk (and per ring refill)

template <typename T>
__global__ void __launch_bounds__(64) band_solve_adjoint_kernel(int n, int kl, int ku, int ldab,
                                                                const cx<T>* __restrict__ ab_all,
                                                                const int* __restrict__ ipiv_all, int L,
                                                                cx<T>* __restrict__ B_all,
                                                                const int* __restrict__ active, int R) {
    const int j = blockIdx.x, col = blockIdx.y;
    if (active && !active[j]) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool producer = warp == 1;
    const int kv = kl + ku, W = kv + 1, M = R - 1;
    const cx<T>* ab = ab_all + (int64_t)j * n * ldab;
    const int* ipiv = ipiv_all + (int64_t)j * n;
    cx<T>* b = B_all + ((int64_t)j * L + col) * n;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // layout: ring[R] | stage[2][CH*W] | pst[2][CH]
    cx<T>* ring = reinterpret_cast<cx<T>*>(smem_raw);
    cx<T>* stage0 = ring + R;
    int* pst0 = reinterpret_cast<int*>(stage0 + 2 * kAdjCH * W);

    // ---- U^* z = b, forward; entry c in ring slot c & M
    auto issue_u = [&](int c0, int bsel) {
        const int cn = min(kAdjCH, n - c0);
        cx<T>* st = stage0 + bsel * kAdjCH * W;
        for (int e = lane; e < cn * W; e += 32) {
            const int cc = e / W, t = e - cc * W;
            if (c0 + cc + t < n) cp_async_cx(&st[e], ab + (int64_t)(c0 + cc) * ldab + t);
            else st[e] = mk<T>(0, 0);
        }
        cp_async_commit();
    };
    if (!producer)
        for (int t = lane; t < R && t < n; t += 32) ring[t] = b[t];
    cx<T> pend = mk<T>(0, 0);
    if (producer) issue_u(0, 0);
    for (int c0 = 0, chunk = 0; c0 < n; c0 += kAdjCH, ++chunk) {
        const int bsel = chunk & 1;
        if (producer) cp_async_wait_group<0>();
        __syncthreads();
        if (producer) {
            if (c0 + kAdjCH < n) issue_u(c0 + kAdjCH, bsel ^ 1);
            continue;
        }
        const int cn = min(kAdjCH, n - c0);
        const cx<T>* st = stage0 + bsel * kAdjCH * W;
        // refill: entry c0-32+lane+R enters the slot that entry c0-32+lane (done) left
        if (c0 >= kAdjCH && c0 - kAdjCH + lane + R < n) ring[(c0 - kAdjCH + lane) & M] = pend;
        if (c0 + lane + R < n) pend = b[c0 + lane + R];
        const cx<T> rd = lane < cn ? recip_conj_or_tiny(st[lane * W]) : mk<T>(0, 0);
        __syncwarp();
        for (int cc = 0; cc < cn; ++cc) {
            const int c = c0 + cc;
            const cx<T> zc = ring[c & M] * shfl_cx(rd, cc);
            const cx<T>* u = st + cc * W;
            for (int t = 1 + lane; t <= kv; t += 32)
                if (c + t < n) ring[(c + t) & M] = fms(ring[(c + t) & M], conj(u[t]), zc);
            if (lane == 0) b[c] = zc;
            __syncwarp();
        }
    }
    __syncthreads();
    if (kl == 0) return;  // no L and no interchanges: z is final

    // ---- L_c^{-*} and P_c for c = n-1 .. 0; entry c in ring slot (n-1-c) & M
    auto slot = [&](int c) { return (n - 1 - c) & M; };
    auto issue_l = [&](int chunk, int bsel) {
        const int chi = n - 1 - chunk * kAdjCH;  // largest c of the chunk
        const int cn = min(kAdjCH, chi + 1);
        cx<T>* st = stage0 + bsel * kAdjCH * W;
        for (int e = lane; e < cn * kl; e += 32) {
            const int cc = e / kl, i = e - cc * kl;
            const int c = chi - cc;
            if (c + 1 + i < n) cp_async_cx(&st[e], ab + (int64_t)c * ldab + kv + 1 + i);
            else st[e] = mk<T>(0, 0);
        }
        for (int e = lane; e < cn; e += 32) cp_async_i32(&pst0[bsel * kAdjCH + e], ipiv + chi - e);
        cp_async_commit();
    };
    if (!producer)
        for (int t = lane; t < R && t < n; t += 32) ring[t] = b[n - 1 - t];
    if (producer) issue_l(0, 0);
    for (int chunk = 0; chunk * kAdjCH < n; ++chunk) {
        const int bsel = chunk & 1;
        const int j0 = chunk * kAdjCH, chi = n - 1 - j0, cn = min(kAdjCH, chi + 1);
        if (producer) cp_async_wait_group<0>();
        __syncthreads();
        if (producer) {
            if (j0 + kAdjCH < n) issue_l(chunk + 1, bsel ^ 1);
            continue;
        }
        const cx<T>* st = stage0 + bsel * kAdjCH * W;
        const int* pst = pst0 + bsel * kAdjCH;
        // refill, in reversed order (entry j = n-1-c at slot j & M): entry j is live from step j
        // to step j+kl, so at this chunk entries jo = j0-32-kl+lane (done in the last chunk) hand
        // their slots to jo+R, loaded now and stored at the next chunk
        {
            const int jw = j0 - 2 * kAdjCH - kl + lane, jl = j0 - kAdjCH - kl + lane;
            if (jw >= 0 && jw + R < n) ring[jw & M] = pend;
            if (jl >= 0 && jl + R < n) pend = b[n - 1 - (jl + R)];
        }
        __syncwarp();
        for (int cc = 0; cc < cn; ++cc) {
            const int c = chi - cc;
            const cx<T>* l = st + cc * kl;
            cx<T> acc = mk<T>(0, 0);
            for (int i = lane; i < kl; i += 32)
                if (c + 1 + i < n) acc = fmac(acc, l[i], ring[slot(c + 1 + i)]);
            for (int o = 16; o > 0; o >>= 1) {
                acc.re += __shfl_xor_sync(0xffffffffu, acc.re, o);
                acc.im += __shfl_xor_sync(0xffffffffu, acc.im, o);
            }
            if (lane == 0) {
                const cx<T> zc = ring[slot(c)] - acc;
                int p = pst[cc];
                if (p < c || p > c + kl || p >= n) p = c;  // a pivot outside the window is ignored
                if (p != c) ring[slot(c)] = ring[slot(p)];
                ring[slot(p)] = zc;
                if (c + kl < n) b[c + kl] = ring[slot(c + kl)];  // final: no later step reaches it
            }
            __syncwarp();
        }
    }
    if (!producer)
        for (int c = lane; c < kl && c < n; c += 32) b[c] = ring[slot(c)];
}

template <typename T>
int launch_band_solve_adjoint(const SplitDev& s, int npts, const cx<T>* ab, const int* ipiv, int L, cx<T>* B,
                              const int* active, cudaStream_t st) {
    if (npts <= 0 || L <= 0) return NEP_OK;
    const int kv = s.kl + s.ku;
    // ring: the forward pass needs R >= kv + 33 (an entry refilled 32 steps before its first
    // update), the backward pass R >= kl + 64 (an entry stays live kl steps after its own)
    int R = 64;
    while (R < kv + kAdjCH + 1 || R < s.kl + 2 * kAdjCH) R <<= 1;
    const size_t smem = sizeof(cx<T>) * ((size_t)R + 2 * kAdjCH * (kv + 1)) + sizeof(int) * 2 * kAdjCH;
    if (smem <= 200 * 1024) {
        NEP_CUDA(allow_max_dynamic_smem(band_solve_adjoint_kernel<T>));
        band_solve_adjoint_kernel<T><<<dim3(npts, L), 64, smem, st>>>(s.n, s.kl, s.ku, s.ldab, ab, ipiv, L, B,
                                                                       active, R);
    } else {
        band_solve_adjoint_glb_kernel<T><<<dim3(npts, L), 32, 0, st>>>(s.n, s.kl, s.ku, s.ldab, ab, ipiv, L, B,
                                                                        active);
    }
    NEP_CHECK_LAUNCH();
    return NEP_OK;
}
template int launch_band_solve_adjoint<float>(const SplitDev&, int, const cx<float>*, const int*, int, cx<float>*,
                                              const int*, cudaStream_t);
template int launch_band_solve_adjoint<double>(const SplitDev&, int, const cx<double>*, const int*, int,
                                               cx<double>*, const int*, cudaStream_t);

// ------------------------------------------------------------------ left eigenvectors
// Band storage of T(z_p)^* for P points (left eigenvectors are right eigenvectors of T^*,
// Sec. 2): row r of T^* is the conjugate of column r of T, read through the split's column view;
// T^* has lower bandwidth ku and upper bandwidth kl, so entry (r, c) goes to slot c - r + ku of a
// row of ldab2 = 2 ku + kl + 1 slots. One warp per (point, row).
template <typename T>
__global__ void __launch_bounds__(256) assemble_adjoint_kernel(SplitDev s, int npts, const zd* __restrict__ F,
                                                               cx<T>* __restrict__ ab, int ldab2) {
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (gw >= (int64_t)npts * s.n) return;
    const int j = (int)(gw / s.n), r = (int)(gw % s.n);
    cx<T>* row = ab + ((int64_t)j * s.n + r) * ldab2;
    for (int t = lane; t < ldab2; t += 32) row[t] = mk<T>(0, 0);
    __syncwarp();
    for (int64_t k = s.colptr[r] + lane; k < s.colptr[r + 1]; k += 32) {
        const int64_t e = s.cidx[k];
        zd v = mk(0.0, 0.0);
        for (int i = 0; i < s.nterms; ++i)
            v = fma_(v, F[i + (int64_t)s.nterms * j],
                     mk(s.val[(int64_t)i * s.nnz + e], s.val_im ? s.val_im[(int64_t)i * s.nnz + e] : 0.0));
        row[s.crow[k] - r + s.ku] = cvt<T>(conj(v));
    }
}

// an exactly zero pivot of the factors stands for eps |U|_max of its point (the inverse-iteration
// convention, eps of the factor precision): with a zero pivot the LU left that column's
// multipliers at zero, so the factors become those of the matrix plus a tiny e_c e_c^T. One CTA
// per point.
template <typename T>
__global__ void __launch_bounds__(256) fix_zero_pivots_kernel(int n, int ldab, int kv, cx<T>* __restrict__ ab_all) {
    cx<T>* ab = ab_all + (int64_t)blockIdx.x * n * ldab;
    __shared__ T part[8];
    __shared__ T tiny;
    T mx = T(0);
    for (int64_t e = threadIdx.x; e < (int64_t)n * (kv + 1); e += blockDim.x) {
        const int c = (int)(e / (kv + 1)), t = (int)(e % (kv + 1));
        if (c + t < n) mx = fmax(mx, abs1(ab[(int64_t)c * ldab + t]));
    }
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        T m = T(0);
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) m = fmax(m, part[q]);
        const T eps = sizeof(T) == 4 ? T(5.96e-8) : T(1.11e-16);
        tiny = eps * (m > T(0) && isfinite(m) ? m : T(1));
    }
    __syncthreads();
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
        cx<T>* d = ab + (int64_t)c * ldab;
        if (d->re == T(0) && d->im == T(0)) *d = mk<T>(tiny, T(0));
    }
}

// F[i + nterms p] = f_i(lam_p), Fd likewise with f_i'
__global__ void left_coeffs_kernel(SplitDev s, int P, const zd* __restrict__ lam, zd* __restrict__ F,
                                   zd* __restrict__ Fd) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= P * s.nterms) return;
    const int i = t % s.nterms, p = t / s.nterms;
    const FnEval e = fn_eval(s.fn_nodes, s.fn_coef, s.fn_root[i], lam[p]);
    F[t] = e.f;
    Fd[t] = e.df;
}

__global__ void left_init_kernel(int P, int* __restrict__ active, int* __restrict__ its, double* __restrict__ eta) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    active[p] = 1;
    its[p] = 0;
    eta[p] = INFINITY;
}

// right-hand side of pair p in the solve precision: y_p (first step) or r_p = T(lambda_p)^* y_p
template <typename T>
__global__ void left_rhs_kernel(int64_t total, int n, const zd* __restrict__ src, cx<T>* __restrict__ B,
                                const int* __restrict__ active) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total || !active[t / n]) return;
    B[t] = cvt<T>(src[t]);
}

// y_p <- w (first step) or y_p - w, then unit 2-norm (scaled by the largest entry first: inverse
// iteration at an eigenvalue makes w huge); one CTA per pair
template <typename T>
__global__ void __launch_bounds__(256) left_update_kernel(int n, int first, zd* __restrict__ Y,
                                                          const cx<T>* __restrict__ B,
                                                          const int* __restrict__ active) {
    const int p = blockIdx.x;
    if (!active[p]) return;
    zd* y = Y + (int64_t)p * n;
    const cx<T>* w = B + (int64_t)p * n;
    __shared__ double part[8];
    __shared__ double scale;
    double mx = 0.0;
    for (int r = threadIdx.x; r < n; r += blockDim.x) {
        const zd v = first ? cvt<double>(w[r]) : y[r] - cvt<double>(w[r]);
        y[r] = v;
        mx = fmax(mx, abs1(v));
    }
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t = fmax(t, part[q]);
        scale = t > 0.0 && t <= 1.7e308 ? 1.0 / t : 0.0;
    }
    __syncthreads();
    const double inv = scale;
    double ss = 0.0;
    for (int r = threadIdx.x; r < n; r += blockDim.x) ss += norm2(inv * y[r]);
    for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = ss;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += part[q];
        scale = t > 0.0 ? inv / sqrt(t) : 0.0;
    }
    __syncthreads();
    for (int r = threadIdx.x; r < n; r += blockDim.x) y[r] = scale * y[r];
}

// R_p = T(lambda_p)^* y_p in FP64: (T^* y)_c = sum_r conj(T(r, c)) y_r over column c of the
// pattern, T(r, c) = sum_i F_i a_i(r, c). One thread per (p, c), rows in ascending order.
__global__ void left_apply_kernel(SplitDev s, int P, const zd* __restrict__ F, const zd* __restrict__ Y,
                                  zd* __restrict__ R, const int* __restrict__ active) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)P * s.n) return;
    const int p = (int)(t / s.n), c = (int)(t % s.n);
    if (!active[p]) return;
    const zd* y = Y + (int64_t)p * s.n;
    const zd* f = F + (int64_t)p * s.nterms;
    zd acc = mk(0.0, 0.0);
    for (int64_t k = s.colptr[c]; k < s.colptr[c + 1]; ++k) {
        const int64_t e = s.cidx[k];
        zd v = mk(0.0, 0.0);
        for (int i = 0; i < s.nterms; ++i)
            v = fma_(v, f[i], mk(s.val[(int64_t)i * s.nnz + e], s.val_im ? s.val_im[(int64_t)i * s.nnz + e] : 0.0));
        acc = fmac(acc, v, y[s.crow[k]]);
    }
    R[t] = acc;
}

// eta_L of pair p (Sec. 2 Eq. (sressplit) for T^*, whose terms have ||A_i^*||_inf = ||A_i||_1).
// The pair stops once eta_L < tol, or when a correction step gained less than a factor 2 (the
// floor that the eigenvalue's own error sets). A correction step that did not lower eta_L is
// undone (y <- Yprev): with factors exact to rounding, y - T^{-*} T^* y can cancel to nothing.
// One CTA per pair.
__global__ void __launch_bounds__(256) left_eta_kernel(SplitDev s, const zd* __restrict__ F,
                                                       zd* __restrict__ Y, const zd* __restrict__ Yprev,
                                                       const zd* __restrict__ R, double tol, int step, int last,
                                                       double* __restrict__ eta, int* __restrict__ active,
                                                       int* __restrict__ its) {
    const int p = blockIdx.x;
    if (!active[p]) return;
    __shared__ double part[2][8];
    __shared__ int restore;
    double rr = 0.0, yy = 0.0;
    for (int r = threadIdx.x; r < s.n; r += blockDim.x) {
        rr += norm2(R[(int64_t)p * s.n + r]);
        yy += norm2(Y[(int64_t)p * s.n + r]);
    }
    for (int o = 16; o > 0; o >>= 1) {
        rr += __shfl_xor_sync(0xffffffffu, rr, o);
        yy += __shfl_xor_sync(0xffffffffu, yy, o);
    }
    if ((threadIdx.x & 31) == 0) {
        part[0][threadIdx.x >> 5] = rr;
        part[1][threadIdx.x >> 5] = yy;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0, den = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            a += part[0][w];
            b += part[1][w];
        }
        for (int i = 0; i < s.nterms; ++i) den += cabs_(F[(int64_t)p * s.nterms + i]) * s.norms1[i];
        const double e = (den > 0.0 && b > 0.0) ? sqrt(a) / (den * sqrt(b)) : INFINITY;
        const double prev = eta[p];
        restore = step >= 1 && !(e < prev);
        if (restore) {
            active[p] = 0;
        } else {
            eta[p] = e;
            its[p] = step + 1;
            if (!(e >= tol) || last || (step >= 1 && e > 0.5 * prev)) active[p] = 0;
        }
    }
    __syncthreads();
    if (restore)
        for (int r = threadIdx.x; r < s.n; r += blockDim.x) Y[(int64_t)p * s.n + r] = Yprev[(int64_t)p * s.n + r];
}

__global__ void left_count_kernel(int P, const int* __restrict__ active, int* __restrict__ out) {
    int cnt = 0;
    for (int p = threadIdx.x; p < P; p += blockDim.x) cnt += active[p];
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if (threadIdx.x == 0) *out = cnt;
}

// y_p <- y_p / conj(y_p^* T'(lambda_p) x_p) (AX: nterms x P x n products A_i x_p); a pair with
// y^* T' x = 0 keeps its unit vector and gets eta = +inf. One CTA per pair.
__global__ void __launch_bounds__(256) left_keldysh_kernel(int n, int nt, int P, const zd* __restrict__ Fd,
                                                           const zd* __restrict__ AX, zd* __restrict__ Y,
                                                           double* __restrict__ eta) {
    const int p = blockIdx.x;
    zd* y = Y + (int64_t)p * n;
    zd acc = mk(0.0, 0.0);
    for (int r = threadIdx.x; r < n; r += blockDim.x) {
        zd tx = mk(0.0, 0.0);
        for (int i = 0; i < nt; ++i) tx = fma_(tx, Fd[(int64_t)p * nt + i], AX[((int64_t)i * P + p) * n + r]);
        acc = fmac(acc, y[r], tx);
    }
    __shared__ zd part[8];
    __shared__ zd scale;
    for (int o = 16; o > 0; o >>= 1) {
        acc.re += __shfl_xor_sync(0xffffffffu, acc.re, o);
        acc.im += __shfl_xor_sync(0xffffffffu, acc.im, o);
    }
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        zd sum = mk(0.0, 0.0);
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) sum = sum + part[w];
        if (sum.re == 0.0 && sum.im == 0.0) {
            scale = mk(1.0, 0.0);
            eta[p] = INFINITY;
        } else {
            scale = cdiv(mk(1.0, 0.0), conj(sum));
        }
    }
    __syncthreads();
    for (int r = threadIdx.x; r < n; r += blockDim.x) y[r] = scale * y[r];
}


// counts the pairs whose y or eta is not finite
__global__ void left_nonfinite_kernel(int64_t total, int n, const zd* __restrict__ Y, const double* __restrict__ eta,
                                      int* __restrict__ cnt) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    const zd v = Y[t];
    const bool bad = !isfinite(v.re) || !isfinite(v.im) || (t % n == 0 && isnan(eta[t / n]));
    if (bad) atomicAdd(cnt, 1);
}

// One route of the left iteration. adjoint = false: T(lambda)^* assembled and factored itself,
// solved by the path's substitution sweeps. adjoint = true: T(lambda) factored, solved with the
// conjugate-transpose kernel (the order of the two triangular solves reversed): the fallback for
// a pair whose null vector spans more orders of magnitude than the first route's back
// substitution can hold in complex64 (its entries grow from the last row up).
template <typename T>
static int left_route(const SplitDev& s, bool adjoint, int P, const zd* lam, const zd* X, zd* Y, double* eta, int* its,
                      double tol, int max_it, int* steps_host, int* nonfinite, cudaStream_t st) {
    const int n = s.n, nt = s.nterms;
    StreamScratch w(st);
    zd *F = nullptr, *Fd = nullptr, *AX = nullptr, *R = nullptr, *Yprev = nullptr;
    cx<T>*ab = nullptr, *ut = nullptr, *B = nullptr;
    // the factored band: T(lambda)^* (bandwidths swapped) or T(lambda)
    SplitDev sh = s;
    if (!adjoint) {
        sh.kl = s.ku;
        sh.ku = s.kl;
        sh.ldab = 2 * sh.kl + sh.ku + 1;
    }
    int *ipiv = nullptr, *info = nullptr, *active = nullptr, *cnt = nullptr;
    NEP_TRY(w.get(&F, (size_t)nt * P));
    NEP_TRY(w.get(&Fd, (size_t)nt * P));
    NEP_TRY(w.get(&ab, (size_t)P * n * sh.ldab));
    if (!adjoint && band_sweeps_fit(sh.kl, sh.ku)) NEP_TRY(w.get(&ut, (size_t)P * n * (sh.kl + sh.ku + 1)));
    NEP_TRY(w.get(&ipiv, (size_t)P * n));
    NEP_TRY(w.get(&info, (size_t)P));
    NEP_TRY(w.get(&B, (size_t)P * n));
    NEP_TRY(w.get(&R, (size_t)P * n));
    NEP_TRY(w.get(&Yprev, (size_t)P * n));
    NEP_TRY(w.get(&AX, (size_t)nt * n * P));
    NEP_TRY(w.get(&active, (size_t)P));
    NEP_TRY(w.get(&cnt, 1));
    left_coeffs_kernel<<<ceil_div(P * nt, 128), 128, 0, st>>>(s, P, lam, F, Fd);
    NEP_CHECK_LAUNCH();
    if (adjoint) {
        // T(lambda_p) factored once; the conjugate-transpose kernel takes care of a zero pivot
        NEP_TRY(launch_assemble<T>(s, P, F, ab, nullptr, nullptr, st));
        NEP_TRY(launch_band_lu<T>(s, P, ab, ipiv, info, nullptr, st));
    } else {
        // T(lambda_p)^* factored once with the path's LU; the substitution sweeps then solve with it
        assemble_adjoint_kernel<T><<<ceil_div((int64_t)P * n * 32, 256), 256, 0, st>>>(s, P, F, ab, sh.ldab);
        NEP_CHECK_LAUNCH();
        NEP_TRY(launch_band_lu<T>(sh, P, ab, ipiv, info, nullptr, st));
        fix_zero_pivots_kernel<T><<<P, 256, 0, st>>>(n, sh.ldab, sh.kl + sh.ku, ab);
        NEP_CHECK_LAUNCH();
        if (ut) NEP_TRY(band_transpose_u<T>(sh, P, ab, ut, st));
    }
    left_init_kernel<<<ceil_div(P, 128), 128, 0, st>>>(P, active, its, eta);
    NEP_CHECK_LAUNCH();
    NEP_CUDA(cudaMemcpyAsync(Y, X, sizeof(zd) * (size_t)n * P, cudaMemcpyDeviceToDevice, st));
    int* host = nullptr;
    host = pinned_slot_get();
    if (!host) { set_error("no pinned host memory"); return NEP_ERR_NOMEM; }
    int rc = NEP_OK, k = 0;
    const int64_t total = (int64_t)P * n;
    for (; k < max_it; ++k) {
        // step 0: inverse iteration y <- T^{-*} y; later steps: y <- y - T^{-*} (T^* y) with the
        // residual in FP64, which removes the factors' rounding from y
        left_rhs_kernel<T><<<ceil_div(total, 256), 256, 0, st>>>(total, n, k == 0 ? Y : R, B, active);
        count_launch();
        if (k > 0 && cudaMemcpyAsync(Yprev, Y, sizeof(zd) * (size_t)total, cudaMemcpyDeviceToDevice, st) != cudaSuccess) {
            rc = NEP_ERR_CUDA;
            break;
        }
        if ((rc = adjoint ? launch_band_solve_adjoint<T>(s, P, ab, ipiv, 1, B, active, st)
                          : launch_band_solve<T>(sh, P, ab, ut, ipiv, 1, B, active, st)))
            break;
        left_update_kernel<T><<<P, 256, 0, st>>>(n, k == 0, Y, B, active);
        count_launch();
        left_apply_kernel<<<ceil_div(total, 256), 256, 0, st>>>(s, P, F, Y, R, active);
        count_launch();
        left_eta_kernel<<<P, 256, 0, st>>>(s, F, Y, Yprev, R, tol, k, k == max_it - 1, eta, active, its);
        count_launch();
        left_count_kernel<<<1, 32, 0, st>>>(P, active, cnt);
        count_launch();
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) { rc = cuda_fail(e, "left eigenvector kernels", __FILE__, __LINE__); break; }
        if (cudaMemcpyAsync(host, cnt, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            rc = NEP_ERR_CUDA;
            break;
        }
        if (*host == 0) {
            ++k;
            break;
        }
    }
    if (!rc) {
        if (steps_host) *steps_host = std::min(k, max_it);
        rc = launch_term_spmm(s, P, X, AX, st);
    }
    if (!rc) {
        left_keldysh_kernel<<<P, 256, 0, st>>>(n, nt, P, Fd, AX, Y, eta);
        count_launch();
        if (cudaMemsetAsync(cnt, 0, sizeof(int), st) != cudaSuccess) rc = NEP_ERR_CUDA;
    }
    if (!rc) {
        left_nonfinite_kernel<<<ceil_div(total, 256), 256, 0, st>>>(total, n, Y, eta, cnt);
        count_launch();
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) rc = cuda_fail(e, "left eigenvector kernels", __FILE__, __LINE__);
    }
    if (!rc && (cudaMemcpyAsync(host, cnt, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess))
        rc = NEP_ERR_CUDA;
    if (!rc) *nonfinite = *host;
    pinned_slot_put(host);
    return rc;
}

template <typename T>
int left_eigvecs(const SplitDev& s, int P, const zd* lam, const zd* X, zd* Y, double* eta, int* its, double tol,
                 int max_it, int* steps_host, cudaStream_t st) {
    if (steps_host) *steps_host = 0;
    if (P <= 0) return NEP_OK;
    int bad = 0;
    NEP_TRY(left_route<T>(s, false, P, lam, X, Y, eta, its, tol, max_it, steps_host, &bad, st));
    if (bad) NEP_TRY(left_route<T>(s, true, P, lam, X, Y, eta, its, tol, max_it, steps_host, &bad, st));
    return NEP_OK;
}
template int left_eigvecs<float>(const SplitDev&, int, const zd*, const zd*, zd*, double*, int*, double, int, int*,
                                 cudaStream_t);
template int left_eigvecs<double>(const SplitDev&, int, const zd*, const zd*, zd*, double*, int*, double, int,
                                  int*, cudaStream_t);

// ------------------------------------------------------------------ resolvent
// Wt[i + P (j nv + k)] = D[i + P k] / (z_j - lam_i)
__global__ void resolvent_weights_kernel(int P, int nz, int nv, const zd* __restrict__ lam, const zd* __restrict__ z,
                                         const zd* __restrict__ D, zd* __restrict__ Wt) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)P * nz * nv) return;
    const int i = (int)(t % P);
    const int64_t q = t / P;  // j nv + k
    const int k = (int)(q % nv), j = (int)(q / nv);
    Wt[t] = cdiv(D[i + (int64_t)P * k], z[j] - lam[i]);
}

int apply_resolvent(int n, int P, const zd* lam, const zd* X, const zd* Y, int nz, const zd* z, int nv, const zd* V,
                    zd* out, cudaStream_t st) {
    if (n <= 0 || nz <= 0 || nv <= 0) return NEP_OK;
    if (P <= 0) {
        NEP_CUDA(cudaMemsetAsync(out, 0, sizeof(zd) * (size_t)n * nz * nv, st));
        return NEP_OK;
    }
    StreamScratch w(st);
    zd *D = nullptr, *Wt = nullptr, *part = nullptr;
    const size_t part_elems = (size_t)P * nv * std::min(64, std::max(1, n / 32));
    NEP_TRY(w.get(&D, (size_t)P * nv));
    NEP_TRY(w.get(&Wt, (size_t)P * nz * nv));
    NEP_TRY(w.get(&part, part_elems));
    // D = Y^* V (P x nv), then out = X Wt (n x nz nv): two FP64 products on the path's GEMM
    NEP_TRY(zgemm(P, nv, n, 1, Y, n, V, n, D, P, part, part_elems, st));
    resolvent_weights_kernel<<<ceil_div((int64_t)P * nz * nv, 256), 256, 0, st>>>(P, nz, nv, lam, z, D, Wt);
    NEP_CHECK_LAUNCH();
    NEP_TRY(zgemm(n, nz * nv, P, 0, X, n, Wt, P, out, n, nullptr, 0, st));
    return NEP_OK;
}

}  // namespace nep

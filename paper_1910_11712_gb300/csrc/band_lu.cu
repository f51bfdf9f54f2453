// Kernel (b): batched complex banded LU with partial pivoting and the banded solves.
//
// The contour method needs one factorisation of T(z_j) per quadrature point (the
// factorisations that dominate the cost of every solver in Sec. 4, cf. Table 2's "PC build").
// All points are independent, so one CTA factors one point and the whole batch runs in
// one launch.
//
// Band layout (row-oriented, in place). Before the LU, row r of a point holds
// A(r, r-kl+t) at ab[r*ldab + t], t in [0, kl+ku]. The LU writes, for every row c,
//   ab[c*ldab + t]            = U(c, c+t),       t in [0, kv]   (kv = kl + ku)
//   ab[c*ldab + kv + 1 + i]   = L(c+1+i, c),     i in [0, kl)
// which only reuses slots of rows that have already entered the elimination window.
//
// Elimination order (right-looking, unblocked, partial pivoting): at step c the active
// window is rows c..c+kl by columns c..c+kv; the pivot is the first row maximising
// |Re|+|Im| in column c; rows c and p swap across the window; the multipliers
// l = a(:,c)/a(c,c) form column c of L; rows c+1..c+kl receive the rank-1 update
// a(r,k) -= l(r) u(k) with u the pivot row. Row c+kl enters the window at step c (its
// first nonzero is column c) and column c+kv enters empty (fill-in only).
//
// Three implementations share this elimination and its stored factors: lu_col.cu (register
// window, kl <= 64 and kl + ku <= 128), lu_wide.cu (blocked, wider bands) and lu_glb_kernel
// below, which keeps the window in a global (L2-resident) scratch array for bands beyond both.
#include <cstdlib>
#include "band_util.cuh"

namespace nep {

// First index of the maximum of |Re|+|Im| over pcol[0..cnt-1], computed by one warp.
// Ties resolve to the smallest index (the same rule as LAPACK's izamax).
template <typename T>
__device__ __forceinline__ int warp_pivot(const cx<T>* pcol, int cnt, int lane) {
    T best = T(-1);
    int bi = 0x7fffffff;
    for (int i = lane; i < cnt; i += 32) {
        T m = abs1(pcol[i]);
        if (m > best) { best = m; bi = i; }
    }
    if constexpr (sizeof(T) == 4) {
        // non-negative floats order like their bit patterns: max magnitude, then the smallest
        // index among the lanes holding it (two warp reductions)
        const unsigned mb = best < 0 ? 0u : __float_as_uint(best);
        const unsigned mx = __reduce_max_sync(0xffffffffu, mb);
        const int p = (int)__reduce_min_sync(0xffffffffu, mb == mx ? (unsigned)bi : 0xffffffffu);
        return p < cnt ? p : 0;  // a column of NaNs matches no row: keep the diagonal
    } else {
        for (int o = 16; o > 0; o >>= 1) {
            T ob = __shfl_xor_sync(0xffffffffu, best, o);
            int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        return bi < cnt ? bi : 0;
    }
}

// Pivot step by warp 0: chooses the pivot among pcol[0..cnt-1], swaps it to pcol[0],
// writes U(c,c), the multipliers (shared lvec and global L column) and ipiv.
template <typename T>
__device__ __forceinline__ void pivot_step(cx<T>* pcol, cx<T>* lvec, int* piv_s, int* info_s, int c, int n, int kl,
                                           int kv, int ldab, cx<T>* ab, int* ipiv, int lane) {
    const int cnt = min(kl, n - 1 - c) + 1;
    int p = warp_pivot(pcol, cnt, lane);
    cx<T> pv = pcol[p];
    const bool zero = (pv.re == T(0) && pv.im == T(0));
    if (zero) p = 0;
    __syncwarp();
    if (lane == 0 && p != 0) {
        cx<T> t = pcol[0];
        pcol[0] = pcol[p];
        pcol[p] = t;
    }
    __syncwarp();
    cx<T>* out = ab + (int64_t)c * ldab;
    const cx<T> rpv = zero ? mk<T>(0, 0) : pivot_recip(pv);
    for (int i = lane; i < kl; i += 32) {
        cx<T> l = mk<T>(0, 0);
        if (!zero && c + 1 + i < n) l = pcol[i + 1] * rpv;
        lvec[i] = l;
        out[kv + 1 + i] = l;
    }
    if (lane == 0) {
        out[0] = zero ? mk<T>(0, 0) : pv;
        ipiv[c] = c + p;
        *piv_s = p;
        if (zero && *info_s == 0) *info_s = c + 1;
    }
}

// Same elimination with the window W[cs*kl + rs] (row slot r mod kl, column slot k mod kv)
// in a per-point global scratch array. For kl = 0 the band is upper triangular and no
// elimination happens besides copying U.
template <typename T>
__global__ void __launch_bounds__(1024, 1)
    lu_glb_kernel(int n, int kl, int ku, int ldab, cx<T>* __restrict__ ab_all, int* __restrict__ ipiv_all,
                  int* __restrict__ info_all, const int* __restrict__ active, cx<T>* __restrict__ win_all) {
    const int j = blockIdx.x;
    if (active && !active[j]) return;
    const int kv = kl + ku;
    const int RS = max(kl, 1), CS = max(kv, 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    cx<T>* ab = ab_all + (int64_t)j * n * ldab;
    int* ipiv = ipiv_all + (int64_t)j * n;
    cx<T>* W = win_all + (int64_t)j * RS * CS;

    extern __shared__ unsigned char smem_raw[];
    cx<T>* nrow = reinterpret_cast<cx<T>*>(smem_raw);  // 2 x (kv+1)
    cx<T>* pcol = nrow + 2 * (kv + 1);                  // kl+1
    cx<T>* lvec = pcol + (kl + 1);                      // kl
    cx<T>* uvec = lvec + max(kl, 1);                    // kv
    __shared__ int piv_s, info_s;
    if (threadIdx.x == 0) info_s = 0;
    // initial window rows 0..kl-1, columns 0..kv-1
    for (int64_t e = threadIdx.x; e < (int64_t)RS * CS; e += blockDim.x) {
        const int cs = (int)(e / RS), rs = (int)(e % RS);
        const int r = rs, k = cs, t = k - r + kl;
        cx<T> v = mk<T>(0, 0);
        if (r < kl && k < kv && r < n && k < n && t >= 0 && t <= kv) v = ab[(int64_t)r * ldab + t];
        W[e] = v;
    }
    for (int t = threadIdx.x; t <= kv; t += blockDim.x) {
        cx<T> v = mk<T>(0, 0);
        if (kl < n && t < n) v = ab[(int64_t)kl * ldab + t];
        nrow[t] = v;
    }
    __syncthreads();
    for (int c = 0; c < n; ++c) {
        cx<T>* nr = nrow + (c & 1) * (kv + 1);
        for (int i = threadIdx.x; i < kl; i += blockDim.x) pcol[i] = W[(int64_t)(c % CS) * RS + (c + i) % RS];
        if (threadIdx.x == 0) pcol[kl] = nr[0];
        cp_async_wait_all();
        __syncthreads();  // S1
        {
            const int r = c + 1 + kl;
            cx<T>* nx = nrow + ((c + 1) & 1) * (kv + 1);
            for (int t = threadIdx.x - 32; t <= kv; t += blockDim.x - 32) {
                if (t < 0) continue;
                if (r < n && c + 1 + t < n) cp_async_cx(nx + t, ab + (int64_t)r * ldab + t);
                else nx[t] = mk<T>(0, 0);
            }
        }
        if (warp == 0) pivot_step(pcol, lvec, &piv_s, &info_s, c, n, kl, kv, ldab, ab, ipiv, lane);
        __syncthreads();  // S2
        const int prel = piv_s;
        cx<T>* urow = ab + (int64_t)c * ldab;
        // column pass: swap rows c and c+prel, broadcast vector u, insert row c+kl
        for (int t = threadIdx.x; t < kv; t += blockDim.x) {
            const int k = c + 1 + t;
            cx<T> u = mk<T>(0, 0);
            if (k < n) {
                const int64_t col = (int64_t)(k % CS) * RS;
                const bool fresh = (k == c + kv);  // column entering the window: no stored values yet
                cx<T> vc = (fresh || kl == 0) ? mk<T>(0, 0) : W[col + c % RS];
                cx<T> vnew = nr[k - c];
                cx<T> newval;
                if (prel == kl) {
                    u = vnew;
                    newval = vc;
                } else {
                    newval = vnew;
                    if (prel != 0) {
                        const int64_t ip = col + (c + prel) % RS;
                        u = fresh ? mk<T>(0, 0) : W[ip];
                        W[ip] = vc;
                    } else {
                        u = vc;
                    }
                }
                urow[1 + t] = u;
                if (kl > 0) W[col + (c + kl) % RS] = newval;  // slot of row c (RS == kl)
                if (fresh) {
                    for (int i = 1; i < kl; ++i)
                        if (i != prel) W[col + (c + i) % RS] = mk<T>(0, 0);
                }
            }
            uvec[t] = u;
        }
        __syncthreads();  // S3
        // rank-1 update of rows c+1..c+kl, columns c+1..c+kv
        const int nrows = min(kl, n - 1 - c), ncols = min(kv, n - 1 - c);
        if (nrows > 0 && ncols > 0) {
            const int64_t tot = (int64_t)nrows * ncols;
            for (int64_t e = threadIdx.x; e < tot; e += blockDim.x) {
                const int t = (int)(e / nrows), i = (int)(e % nrows);
                const int k = c + 1 + t, r = c + 1 + i;
                cx<T>* w = W + (int64_t)(k % CS) * RS + r % RS;
                *w = fms(*w, lvec[i], uvec[t]);
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) info_all[j] = info_s;
}

// ------------------------------------------------------------------ dispatch
template <typename T>
int launch_band_lu(const SplitDev& s, int npts, cx<T>* ab, int* ipiv, int* info, const int* active, cudaStream_t st,
                   int lu_kernel) {
    if (npts <= 0) return NEP_OK;
    const int kv = s.kl + s.ku;
    // complex64, the tensor-core kernel asked for by name on a band the register window also takes
    if constexpr (sizeof(T) == 4)
        if ((lu_kernel == LU_TC3 || lu_kernel == LU_TC1) && band_lu_col_fits(s.kl, s.ku) && band_lu_tc_can(s.kl))
            return launch_band_lu_tc(s, npts, ab, ipiv, info, active, st, lu_kernel == LU_TC1 ? 1 : 3);
    // register window, one barrier per step (lu_col.cu): kl <= 64, kv <= 128
    if (band_lu_col_fits(s.kl, s.ku)) return launch_band_lu_col<T>(s, npts, ab, ipiv, info, active, st);
    // wide bands in complex64: trailing updates on the tensor core
    if constexpr (sizeof(T) == 4)
        if (lu_kernel != LU_SIMT && (lu_kernel != LU_AUTO || lu_tc_enabled()) && band_lu_tc_fits(s.kl))
            return launch_band_lu_tc(s, npts, ab, ipiv, info, active, st, lu_kernel == LU_TC1 ? 1 : 3);
    // wide bands: blocked LU with the trailing window in global memory
    if (s.kl >= 1 && band_lu_wide_fits(s.kl, (int)sizeof(cx<T>)))
        return launch_band_lu_wide<T>(s, npts, ab, ipiv, info, active, st);
    // global-window path: per-point scratch of max(kl,1) x max(kv,1) elements
    const int RS = s.kl > 1 ? s.kl : 1, CS = kv > 1 ? kv : 1;
    const size_t win_bytes = sizeof(cx<T>) * (size_t)RS * CS * npts;
    cx<T>* win = nullptr;
    NEP_CUDA(cudaMallocAsync((void**)&win, win_bytes, st));
    const size_t smem = sizeof(cx<T>) * (size_t)(2 * (kv + 1) + (s.kl + 1) + (s.kl > 1 ? s.kl : 1) + CS);
    if (smem > 48 * 1024)
        NEP_CUDA(allow_max_dynamic_smem(lu_glb_kernel<T>));
    lu_glb_kernel<T><<<npts, 1024, smem, st>>>(s.n, s.kl, s.ku, s.ldab, ab, ipiv, info, active, win);
    count_launch();
    cudaError_t e = cudaGetLastError();
    cudaFreeAsync(win, st);
    if (e != cudaSuccess) return cuda_fail(e, "lu_glb_kernel", __FILE__, __LINE__);
    return NEP_OK;
}

template int launch_band_lu<float>(const SplitDev&, int, cx<float>*, int*, int*, const int*, cudaStream_t, int);
template int launch_band_lu<double>(const SplitDev&, int, cx<double>*, int*, int*, const int*, cudaStream_t, int);

// ------------------------------------------------------------------ banded solves
// One warp per right-hand side column, one CTA per (point, group of columns). Forward
// sweep: the (kl+1)-row window of the current right-hand side lives in shared memory
// (slot r mod (kl+1)); at step c rows c and ipiv[c] swap, x_c is final, rows c+1..c+kl
// take x_c times the L column and row c+kl+1 enters the freed slot. Backward sweep
// (columns n-1..0): x_c = w_c / U(c,c) and rows c-kv..c-1 take x_c times U column c;
// window of kv+1 rows. L columns (contiguous) and U columns (gathered from U rows,
// coalesced by rows) are staged in shared memory in chunks of CH steps shared by all warps.
template <typename T>
__device__ __forceinline__ void cp_async_int(int* smem, const int* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}

template <typename T, int RH>
__global__ void __launch_bounds__(512)
    band_solve_kernel(int n, int kl, int ku, int ldab, const cx<T>* __restrict__ ab_all,
                      const int* __restrict__ ipiv_all, int L, cx<T>* __restrict__ B_all,
                      const int* __restrict__ active, int CH) {
    const int j = blockIdx.x;
    if (active && !active[j]) return;
    const int kv = kl + ku;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nwarps = blockDim.x >> 5;
    const int col0 = (blockIdx.y * nwarps + warp) * RH;  // first right-hand side of this warp
    const int nrh = max(0, min(RH, L - col0));
    const bool has_col = nrh > 0;
    const cx<T>* ab = ab_all + (int64_t)j * n * ldab;
    const int* ipiv = ipiv_all + (int64_t)j * n;
    cx<T>* bbase = B_all + ((int64_t)j * L + (has_col ? col0 : 0)) * n;  // column r at bbase + r*n

    extern __shared__ unsigned char smem_raw[];
    const int RF = kl + 1, RB = kv + 1;
    const int WIN = RF > RB ? RF : RB;
    const int wide = kv > kl ? kv : (kl > 0 ? kl : 1);
    // layout: win[nwarps][WIN*RH] | nb[2][nwarps][CH*RH] | stage[2][CH*wide] | diag[2][CH] | pst[2][CH]
    cx<T>* win = reinterpret_cast<cx<T>*>(smem_raw) + (int64_t)warp * WIN * RH;
    cx<T>* nb0 = reinterpret_cast<cx<T>*>(smem_raw) + (int64_t)nwarps * WIN * RH;
    cx<T>* stage0 = nb0 + 2 * (int64_t)nwarps * CH * RH;
    cx<T>* diag0 = stage0 + 2 * (int64_t)CH * wide;
    int* pst0 = reinterpret_cast<int*>(diag0 + 2 * CH);
    auto nbuf = [&](int bsel) { return nb0 + ((int64_t)bsel * nwarps + warp) * CH * RH; };
    auto sbuf = [&](int bsel) { return stage0 + (int64_t)bsel * CH * wide; };

    // ---- forward: row interchanges and unit lower L. Row r of right-hand side q lives at
    //      win[(r mod RF)*RH + q].
    auto issue_fwd = [&](int c0, int bsel) {
        const int cn = min(CH, n - c0);
        cx<T>* st = sbuf(bsel);
        for (int e = threadIdx.x; e < cn * kl; e += blockDim.x) {
            const int cc = e / kl, i = e - cc * kl;
            cp_async_cx(&st[e], ab + (int64_t)(c0 + cc) * ldab + kv + 1 + i);
        }
        for (int e = threadIdx.x; e < cn; e += blockDim.x) cp_async_int<T>(&pst0[bsel * CH + e], ipiv + c0 + e);
        if (has_col) {
            cx<T>* nb = nbuf(bsel);
            for (int e = lane; e < cn * RH; e += 32) {
                const int cc = e / RH, q = e - cc * RH;
                const int rn = c0 + cc + kl + 1;
                if (rn < n && q < nrh) cp_async_cx(&nb[e], bbase + (int64_t)q * n + rn);
                else nb[e] = mk<T>(0, 0);
            }
        }
        cp_async_commit();
    };
    for (int e = lane; e < RF * RH; e += 32) {
        const int i = e / RH, q = e - i * RH;
        win[e] = (q < nrh && i < n) ? bbase[(int64_t)q * n + i] : mk<T>(0, 0);
    }
    int sc = 0;
    issue_fwd(0, 0);
    for (int c0 = 0, chunk = 0; c0 < n; c0 += CH, ++chunk) {
        const int cn = min(CH, n - c0);
        const int bsel = chunk & 1;
        cp_async_wait_group<0>();
        __syncthreads();
        if (c0 + CH < n) issue_fwd(c0 + CH, bsel ^ 1);
        if (has_col) {
            const cx<T>* st = sbuf(bsel);
            const int* pst = pst0 + bsel * CH;
            const cx<T>* nb = nbuf(bsel);
            for (int cc = 0; cc < cn; ++cc) {
                const int c = c0 + cc;
                const int p = pst[cc] - c;
                if (p != 0 && lane < RH) {
                    int s1 = sc + p;
                    if (s1 >= RF) s1 -= RF;
                    const cx<T> t = win[sc * RH + lane];
                    win[sc * RH + lane] = win[s1 * RH + lane];
                    win[s1 * RH + lane] = t;
                }
                __syncwarp();
                const cx<T>* lc = st + cc * kl;
                const int lim = min(kl, n - 1 - c) * RH;
                for (int e = lane; e < lim; e += 32) {
                    const int i = e / RH, q = e - i * RH;
                    int s = sc + 1 + i;
                    if (s >= RF) s -= RF;
                    win[s * RH + q] = fms(win[s * RH + q], lc[i], win[sc * RH + q]);
                }
                __syncwarp();
                if (lane < nrh) {
                    bbase[(int64_t)lane * n + c] = win[sc * RH + lane];
                    win[sc * RH + lane] = nb[cc * RH + lane];
                } else if (lane < RH) {
                    win[sc * RH + lane] = nb[cc * RH + lane];
                }
                if (++sc == RF) sc = 0;
                __syncwarp();
            }
        }
    }
    // ---- backward: U with bandwidth kv; row r of right-hand side q at win[(r mod RB)*RH + q]
    cp_async_wait_group<0>();
    __syncthreads();
    auto issue_bwd = [&](int c1, int bsel) {
        const int cn = min(CH, c1 + 1);
        const int cbase = c1 - cn + 1;
        cx<T>* st = sbuf(bsel);
        cx<T>* dg = diag0 + bsel * CH;
        const int rlo = cbase - kv, rhi = c1 - 1;
        const int nr = rhi - rlo + 1;
        for (int e = threadIdx.x; e < nr * cn; e += blockDim.x) {
            const int ri = e / cn, cc = e - ri * cn;
            const int r = rlo + ri, c = cbase + cc, t = c - r;
            if (r >= 0 && t >= 1 && t <= kv) cp_async_cx(&st[cc * kv + (t - 1)], ab + (int64_t)r * ldab + t);
        }
        for (int e = threadIdx.x; e < cn; e += blockDim.x) cp_async_cx(&dg[e], ab + (int64_t)(cbase + e) * ldab);
        if (has_col) {
            cx<T>* nb = nbuf(bsel);
            for (int e = lane; e < cn * RH; e += 32) {
                const int cc = e / RH, q = e - cc * RH;
                const int rn = cbase + cc - kv - 1;
                if (rn >= 0 && q < nrh) cp_async_cx(&nb[e], bbase + (int64_t)q * n + rn);
                else nb[e] = mk<T>(0, 0);
            }
        }
        cp_async_commit();
    };
    for (int e = lane; e < RB * RH; e += 32) {
        const int i = e / RH, q = e - i * RH;
        const int r = n - 1 - i;
        if (r >= 0) win[(r % RB) * RH + q] = q < nrh ? bbase[(int64_t)q * n + r] : mk<T>(0, 0);
    }
    sc = (n - 1) % RB;
    issue_bwd(n - 1, 0);
    for (int c1 = n - 1, chunk = 0; c1 >= 0; c1 -= CH, ++chunk) {
        const int cn = min(CH, c1 + 1);
        const int cbase = c1 - cn + 1;
        const int bsel = chunk & 1;
        cp_async_wait_group<0>();
        __syncthreads();
        if (c1 - CH >= 0) issue_bwd(c1 - CH, bsel ^ 1);
        if (has_col) {
            const cx<T>* st = sbuf(bsel);
            const cx<T>* dg = diag0 + bsel * CH;
            const cx<T>* nb = nbuf(bsel);
            const cx<T> rd = lane < cn ? cdiv(mk<T>(1, 0), dg[lane]) : mk<T>(0, 0);
            for (int cc = cn - 1; cc >= 0; --cc) {
                const int c = cbase + cc;
                cx<T> r;
                r.re = __shfl_sync(0xffffffffu, rd.re, cc);
                r.im = __shfl_sync(0xffffffffu, rd.im, cc);
                if (lane < RH) win[sc * RH + lane] = win[sc * RH + lane] * r;
                __syncwarp();
                const cx<T>* uc = st + cc * kv;
                const int lim = min(kv, c) * RH;
                for (int e = lane; e < lim; e += 32) {
                    const int i = e / RH, q = e - i * RH;
                    int s = sc - 1 - i;
                    if (s < 0) s += RB;
                    win[s * RH + q] = fms(win[s * RH + q], uc[i], win[sc * RH + q]);
                }
                __syncwarp();
                if (lane < nrh) {
                    bbase[(int64_t)lane * n + c] = win[sc * RH + lane];
                    win[sc * RH + lane] = nb[cc * RH + lane];
                } else if (lane < RH) {
                    win[sc * RH + lane] = nb[cc * RH + lane];
                }
                if (--sc < 0) sc = RB - 1;
                __syncwarp();
            }
        }
    }
}

template <typename T>
int launch_band_solve(const SplitDev& s, int npts, const cx<T>* ab, const cx<T>* ut, const int* ipiv, int L, cx<T>* B,
                      const int* active, cudaStream_t st, int rh_force) {
    if (npts <= 0 || L <= 0) return NEP_OK;
    const int kv = s.kl + s.ku;
    // register windows for narrow bands (kl+1 <= 288 and kv+1 <= 288 rows): two sweeps with
    // slot-ordered coefficients
    if (band_sweeps_fit(s.kl, s.ku)) return band_sweeps<T>(s, npts, ab, ut, ipiv, L, B, active, st, rh_force);
    // complex64 factors: blocked substitution (NEP_SOLVE_UNBLOCKED=1 keeps the per-step sweeps below)
    if constexpr (sizeof(T) == 4) {
        static const bool unblocked = [] {
            const char* e = std::getenv("NEP_SOLVE_UNBLOCKED");
            return e && e[0] == '1';
        }();
        if (!unblocked) {
            const int rc = launch_band_solve_blocked(s, npts, ab, ipiv, L, B, active, st);
            if (rc != NEP_ERR_UNSUPPORTED) return rc;
        }
    }
    // general path: shared-memory windows, one right-hand side per warp, four warps per CTA
    constexpr int RH = 1;
    const int warps_total = L;
    const int wpb = warps_total < 4 ? warps_total : 4;
    const int gy = (warps_total + wpb - 1) / wpb;
    const int WIN = (s.kl + 1) > (kv + 1) ? (s.kl + 1) : (kv + 1);
    const int wide = kv > s.kl ? kv : (s.kl > 0 ? s.kl : 1);
    const size_t budget = 200 * 1024;
    int CH = 32;
    auto bytes = [&](int ch) {
        return sizeof(cx<T>) * ((size_t)wpb * WIN * RH + 2 * (size_t)wpb * ch * RH + 2 * (size_t)ch * wide + 2 * ch) +
               sizeof(int) * 2 * ch;
    };
    while (CH > 1 && bytes(CH) > budget) CH >>= 1;
    const size_t smem = bytes(CH);
    if (smem > 227 * 1024) return NEP_ERR_UNSUPPORTED;
    NEP_CUDA(allow_max_dynamic_smem(band_solve_kernel<T, RH>));
    dim3 grid(npts, gy);
    band_solve_kernel<T, RH><<<grid, wpb * 32, smem, st>>>(s.n, s.kl, s.ku, s.ldab, ab, ipiv, L, B, active, CH);
    NEP_CHECK_LAUNCH();
    return NEP_OK;
}

template int launch_band_solve<float>(const SplitDev&, int, const cx<float>*, const cx<float>*, const int*, int,
                                      cx<float>*, const int*, cudaStream_t, int);
template int launch_band_solve<double>(const SplitDev&, int, const cx<double>*, const cx<double>*, const int*, int,
                                       cx<double>*, const int*, cudaStream_t, int);

}  // namespace nep

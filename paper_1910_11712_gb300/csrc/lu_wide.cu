// Kernel (b) for wide bands: blocked batched complex banded LU with partial pivoting, one CTA
// per quadrature point. Used where the register windows of band_lu.cu do not fit (kl > 64):
// there every column step of the unblocked elimination touches a kl x (kl+ku) window, and
// doing those updates a panel at a time turns them into a matrix product.
//
// Same elimination and the same stored factors as band_lu.cu: the pivot of column c is the
// first row maximising |Re|+|Im| among rows c..c+kl, rows c and p swap, l = a(:,c)/a(c,c) is
// stored as column c of L (later interchanges are not applied to it), U(c, c..c+kv) as row c.
// Per panel [p0, p0+NB):
//   1. the panel columns (rows p0 .. p0+NB-1+kl) are copied to shared memory and factored
//      column by column; interchanges are applied across the panel, so the panel's copy of the
//      multipliers (L~) carries the later interchanges, while the output copy is written when
//      each column is computed;
//   2. for the trailing columns, in chunks: the panel's interchanges (composed once into one
//      permutation of the rows involved), then U12 = L~11^{-1} A12 by forward substitution
//      (k ascending; a warp per column, lanes over its rows), written to the output rows;
//   3. A22 -= L~21 U12 (k ascending) on the chunk.
// Applying the panel's interchanges first and its eliminations after changes neither the
// operations nor their order on any element of the trailing columns (a value ending in row r
// received the update of step k with the multiplier then in its row, which the interchanges
// carried to row r of L~), so the factors equal the unblocked ones up to the order of the
// real products inside each complex product.
//
// The trailing part lives in a per-point window in global memory (L2-resident when the batch's
// windows fit): rows [p0, p0+kl+NB) x columns [p0, p0+kv+NB), circular (row r in slot
// r mod RWp, column c in slot c mod CWp, column-major). After a panel its rows are final, the
// next NB rows of the band enter the freed row slots, and NB new columns enter as zeros.
#include "band_util.cuh"

namespace nep {

template <typename T, int NB>
__global__ void __launch_bounds__(512, 1)
    lu_wide_kernel(int n, int kl, int ku, int ldab, cx<T>* __restrict__ ab_all, int* __restrict__ ipiv_all,
                   int* __restrict__ info_all, const int* __restrict__ active, cx<T>* __restrict__ win_all, int RWp,
                   int CWp, int CHW) {
    const int j = blockIdx.x;
    if (active && !active[j]) return;
    const int kv = kl + ku;
    const int RW = kl + NB, CW = kv + NB;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nthr = blockDim.x, nwarp = nthr >> 5;
    cx<T>* ab = ab_all + (int64_t)j * n * ldab;
    int* ipiv = ipiv_all + (int64_t)j * n;
    cx<T>* W = win_all + (int64_t)j * RWp * CWp;
    auto wi = [&](int r, int c) -> int64_t { return (int64_t)(r % RWp) + (int64_t)RWp * (c % CWp); };

    extern __shared__ unsigned char smem_raw[];
    cx<T>* Ps = reinterpret_cast<cx<T>*>(smem_raw);  // RW x NB panel, column-major (local rows)
    cx<T>* Us = Ps + (int64_t)RW * NB;               // NB x CHW: U12 chunk, column jc at Us[NB*jc]
    int* src = reinterpret_cast<int*>(Us + (int64_t)NB * CHW);  // RW: row permutation of the panel
    int* plist = src + RW;                                      // partner rows (local, >= nbc)
    __shared__ int piv_sh[NB];
    __shared__ int info_s, npart_s;
    if (tid == 0) info_s = 0;

    // window: zero, then rows 0 .. RW-1 of the band
    auto load_rows = [&](int r0, int r1) {
        for (int r = r0 + warp; r < r1; r += nwarp) {
            const cx<T>* srow = ab + (int64_t)r * ldab - (r - kl);  // srow[c] = A(r, c)
            const int clo = max(r - kl, 0), chi = min(r + ku, n - 1);
            for (int c = clo + lane; c <= chi; c += 32) W[wi(r, c)] = srow[c];
        }
    };
    for (int64_t e = tid; e < (int64_t)RWp * CWp; e += nthr) W[e] = mk<T>(0, 0);
    __syncthreads();
    load_rows(0, min(RW, n));
    __syncthreads();

    for (int p0 = 0; p0 < n; p0 += NB) {
        const int nbc = min(NB, n - p0);
        const int pr = min(RW, n - p0);  // panel rows (local 0 .. pr-1)

        // ---- 0. panel columns to shared memory (warps over columns, lanes over rows)
        for (int q = warp; q < nbc; q += nwarp)
            for (int i = lane; i < RW; i += 32) Ps[i + (int64_t)RW * q] = i < pr ? W[wi(p0 + i, p0 + q)] : mk<T>(0, 0);
        __syncthreads();

        // ---- 1. panel factorisation
        for (int k = 0; k < nbc; ++k) {
            const int c = p0 + k;
            const int last = min(k + kl, pr - 1), cnt = last - k + 1;  // candidate rows k .. last
            cx<T>* colk = Ps + (int64_t)RW * k;
            if (warp == 0) {
                T best = T(-1);
                int bi = 0x7fffffff;
                for (int i = lane; i < cnt; i += 32) {
                    const T m = abs1(colk[k + i]);
                    if (m > best) { best = m; bi = i; }
                }
                int p;
                if constexpr (sizeof(T) == 4) {
                    const unsigned mb = best < 0 ? 0u : __float_as_uint(best);
                    const unsigned mx = __reduce_max_sync(0xffffffffu, mb);
                    p = (int)__reduce_min_sync(0xffffffffu, mb == mx ? (unsigned)bi : 0xffffffffu);
                } else {
                    for (int o = 16; o > 0; o >>= 1) {
                        const T ob = __shfl_xor_sync(0xffffffffu, best, o);
                        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
                    }
                    p = bi;
                }
                if (p >= cnt) p = 0;  // a column of NaNs matches no row: keep the diagonal
                const cx<T> pv = colk[k + p];
                const bool zero = pv.re == T(0) && pv.im == T(0);
                if (zero) p = 0;
                if (p != 0)
                    for (int q = lane; q < nbc; q += 32) {
                        cx<T>* pq = Ps + (int64_t)RW * q;
                        const cx<T> t = pq[k];
                        pq[k] = pq[k + p];
                        pq[k + p] = t;
                    }
                if (lane == 0) {
                    ipiv[c] = c + p;
                    piv_sh[k] = c + p;
                    if (zero && info_s == 0) info_s = c + 1;
                    Ps[(int64_t)RW * NB + 0] = zero ? mk<T>(0, 0) : cdiv(mk<T>(1, 0), pv);  // scratch: 1/pivot in Us[0]
                }
            }
            __syncthreads();
            // multipliers of rows k+1 .. last (all threads); their output copy is final now
            {
                const cx<T> rpv = Us[0];
                cx<T>* out = ab + (int64_t)c * ldab + kv + 1;
                for (int i = tid; i < kl; i += nthr) {
                    cx<T> l = mk<T>(0, 0);
                    if (k + 1 + i <= last) {
                        l = colk[k + 1 + i] * rpv;
                        colk[k + 1 + i] = l;
                    }
                    out[i] = l;
                }
            }
            __syncthreads();
            // rank-1 update of the panel columns right of k (warps over columns, lanes over rows)
            for (int q = k + 1 + warp; q < nbc; q += nwarp) {
                cx<T>* pq = Ps + (int64_t)RW * q;
                const cx<T> u = pq[k];
                for (int i = k + 1 + lane; i <= last; i += 32) pq[i] = fms(pq[i], colk[i], u);
            }
            __syncthreads();
        }

        // ---- the panel's interchanges as one permutation: row (local) l receives old row src[l]
        for (int l = tid; l < RW; l += nthr) src[l] = l;
        __syncthreads();
        if (tid == 0) {
            int np = 0;
            for (int k = 0; k < nbc; ++k) {
                const int b = piv_sh[k] - p0;
                if (b != k) {
                    const int t = src[k];
                    src[k] = src[b];
                    src[b] = t;
                    if (b >= nbc) {
                        bool seen = false;
                        for (int q = 0; q < np; ++q) seen |= plist[q] == b;
                        if (!seen) plist[np++] = b;
                    }
                }
            }
            npart_s = np;
        }
        __syncthreads();
        const int npart = npart_s;

        // ---- 2, 3. trailing columns [p0+nbc, cend) in chunks, rows [p0+nbc, rend)
        const int cend = min(p0 + nbc + kv, n), rend = min(p0 + nbc + kl, n);
        const int mr = rend - (p0 + nbc);
        for (int c0 = p0 + nbc; c0 < cend; c0 += CHW) {
            const int cw = min(CHW, cend - c0);
            // interchanges and U12, one warp per column with lane k on row p0 + k (NB <= 32):
            // u_i -= l_ik u_k for k ascending, the substitution's order of operations
            for (int jc = warp; jc < cw; jc += nwarp) {
                const int q = c0 + jc;
                const cx<T> u0 = lane < nbc ? W[wi(p0 + src[lane], q)] : mk<T>(0, 0);
                const cx<T> x = lane < npart ? W[wi(p0 + src[plist[lane]], q)] : mk<T>(0, 0);
                __syncwarp();
                if (lane < npart) W[wi(p0 + plist[lane], q)] = x;
                cx<T> u = u0;
                for (int k = 0; k + 1 < nbc; ++k) {
                    const cx<T> uk = shfl_cx(u, k);
                    if (lane > k && lane < nbc) u = fms(u, Ps[lane + (int64_t)RW * k], uk);
                }
                if (lane < nbc) {
                    Us[(int64_t)NB * jc + lane] = u;
                    const int r = p0 + lane;
                    if (q - r <= kv) ab[(int64_t)r * ldab + (q - r)] = u;
                }
            }
            __syncthreads();
            // A22 -= L~21 U12: 4 x 4 tiles, rows tr + RT*ii (consecutive threads, consecutive rows)
            if (mr > 0) {
                const int RT = (mr + 3) >> 2, CT = (cw + 3) >> 2;
                for (int e = tid; e < RT * CT; e += nthr) {
                    const int tr = e % RT, tc = e / RT;
                    int64_t wr[4], wc[4];
                    int li[4];
                    bool rok[4], cok[4];
#pragma unroll
                    for (int ii = 0; ii < 4; ++ii) {
                        const int lr = nbc + tr + RT * ii;  // local panel row
                        rok[ii] = tr + RT * ii < mr;
                        li[ii] = rok[ii] ? lr : nbc;
                        wr[ii] = (int64_t)((p0 + li[ii]) % RWp);
                    }
#pragma unroll
                    for (int jj = 0; jj < 4; ++jj) {
                        cok[jj] = 4 * tc + jj < cw;
                        wc[jj] = (int64_t)RWp * ((c0 + (cok[jj] ? 4 * tc + jj : 0)) % CWp);
                    }
                    cx<T> acc[4][4];
#pragma unroll
                    for (int ii = 0; ii < 4; ++ii)
#pragma unroll
                        for (int jj = 0; jj < 4; ++jj) acc[ii][jj] = W[wr[ii] + wc[jj]];
                    for (int k = 0; k < nbc; ++k) {
                        const cx<T>* lk = Ps + (int64_t)RW * k;
                        cx<T> l[4], uu[4];
#pragma unroll
                        for (int ii = 0; ii < 4; ++ii) l[ii] = lk[li[ii]];
#pragma unroll
                        for (int jj = 0; jj < 4; ++jj) uu[jj] = Us[(int64_t)NB * (cok[jj] ? 4 * tc + jj : 0) + k];
#pragma unroll
                        for (int ii = 0; ii < 4; ++ii)
#pragma unroll
                            for (int jj = 0; jj < 4; ++jj) acc[ii][jj] = fms(acc[ii][jj], l[ii], uu[jj]);
                    }
#pragma unroll
                    for (int ii = 0; ii < 4; ++ii)
#pragma unroll
                        for (int jj = 0; jj < 4; ++jj)
                            if (rok[ii] && cok[jj]) W[wr[ii] + wc[jj]] = acc[ii][jj];
                }
            }
            __syncthreads();
        }

        // ---- 4. the panel part of the finished rows: U(r, r .. p0+nbc-1)
        for (int k = warp; k < nbc; k += nwarp) {
            const int r = p0 + k;
            cx<T>* out = ab + (int64_t)r * ldab;
            for (int q = k + lane; q < nbc; q += 32) out[q - k] = Ps[k + (int64_t)RW * q];
            // entries of row r beyond the band of the trailing columns are zero
            for (int t = (cend - r) + lane; t <= kv; t += 32)
                if (t >= 0) out[t] = mk<T>(0, 0);
        }
        // ---- 5. next window: rows [p0+RW, p0+RW+NB) and columns [p0+CW, p0+CW+NB) enter as zeros
        if (p0 + NB < n) {
            const int rn0 = p0 + RW;
            for (int e = tid; e < NB * CWp; e += nthr) {
                const int ir = e / CWp, jc = e - ir * CWp;
                W[(int64_t)((rn0 + ir) % RWp) + (int64_t)RWp * jc] = mk<T>(0, 0);
            }
            for (int e = tid; e < NB * RWp; e += nthr) {
                const int jc = e / RWp, i = e - jc * RWp;
                W[(int64_t)i + (int64_t)RWp * ((p0 + CW + jc) % CWp)] = mk<T>(0, 0);
            }
            __syncthreads();
            if (rn0 < n) load_rows(rn0, min(rn0 + NB, n));
        }
        __syncthreads();
    }
    if (tid == 0) info_all[j] = info_s;
}

// Shared memory of lu_wide_kernel for a band and panel width.
static size_t wide_smem(int kl, int nb, int chw, size_t esz) {
    const size_t rw = (size_t)kl + nb;
    return esz * (rw * nb + (size_t)nb * chw) + sizeof(int) * (rw + nb);
}

template <typename T, int NB>
static int run_wide(const SplitDev& s, int npts, cx<T>* ab, int* ipiv, int* info, const int* active, cudaStream_t st,
                    int chw) {
    const int kv = s.kl + s.ku;
    const int rwp = (s.kl + NB + NB - 1) / NB * NB, cwp = (kv + NB + NB - 1) / NB * NB;
    const size_t smem = wide_smem(s.kl, NB, chw, sizeof(cx<T>));
    cx<T>* win = nullptr;
    NEP_CUDA(cudaMallocAsync((void**)&win, sizeof(cx<T>) * (size_t)rwp * cwp * npts, st));
    cudaError_t e = allow_max_dynamic_smem(lu_wide_kernel<T, NB>);
    if (e == cudaSuccess) {
        lu_wide_kernel<T, NB><<<npts, 512, smem, st>>>(s.n, s.kl, s.ku, s.ldab, ab, ipiv, info, active, win, rwp, cwp,
                                                      chw);
        count_launch();
        e = cudaGetLastError();
    }
    cudaFreeAsync(win, st);
    if (e != cudaSuccess) return cuda_fail(e, "lu_wide_kernel", __FILE__, __LINE__);
    return NEP_OK;
}

bool band_lu_wide_fits(int kl, int elem_bytes) {
    for (int nb : {32, 16, 8})
        if (wide_smem(kl, nb, 64, (size_t)elem_bytes) <= 200 * 1024) return true;
    return false;
}

template <typename T>
int launch_band_lu_wide(const SplitDev& s, int npts, cx<T>* ab, int* ipiv, int* info, const int* active,
                        cudaStream_t st) {
    if (npts <= 0) return NEP_OK;
    const size_t esz = sizeof(cx<T>);
    // widest panel (and then the widest column chunk) whose shared memory fits
    for (int chw : {128, 64}) {
        if (wide_smem(s.kl, 32, chw, esz) <= 200 * 1024) return run_wide<T, 32>(s, npts, ab, ipiv, info, active, st, chw);
        if (wide_smem(s.kl, 16, chw, esz) <= 200 * 1024) return run_wide<T, 16>(s, npts, ab, ipiv, info, active, st, chw);
    }
    if (wide_smem(s.kl, 8, 64, esz) <= 200 * 1024) return run_wide<T, 8>(s, npts, ab, ipiv, info, active, st, 64);
    return NEP_ERR_UNSUPPORTED;
}

template int launch_band_lu_wide<float>(const SplitDev&, int, cx<float>*, int*, int*, const int*, cudaStream_t);
template int launch_band_lu_wide<double>(const SplitDev&, int, cx<double>*, int*, int*, const int*, cudaStream_t);

}  // namespace nep

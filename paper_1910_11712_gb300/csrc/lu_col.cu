// Kernel (b), narrow bands (kl <= 64, kl + ku <= 128): batched complex banded LU with partial
// pivoting, one CTA of 16 warps per quadrature point and one CTA barrier per column step.
//
// The elimination and the stored factors are those of band_lu.cu: at step c the pivot is the
// first row maximising |Re|+|Im| among rows c..c+kl, rows c and p swap across the window,
// l = a(:,c)/a(c,c) is column c of L, rows c+1..c+kl receive a(r,k) -= l(r) u(k) with u the
// pivot row. Every element receives the same operations in the same order, so the factors are
// the same bit for bit.
//
// Register window with rows across lanes and columns across warps. Row slot s (lane s % 32,
// register s / 32, s < kl) holds one window row and carries its row index as a label;
// column slot s (warp s / CPW, register s % CPW, s < CS = 16 CPW >= kl+ku) holds column k with
// k mod CS = s, also labelled. An interchange moves no data: the pivot row leaves the window
// as row c of U, the entering row c+kl takes over its slot, and the slot of row c takes the
// pivot row's label. The slot column c+1 leaves after step c+1's pivot takes column c+1+CS,
// zero in every window row (beyond the band, or the band's next column when CS = kl+ku).
// A column is held by one warp, so
//   * the pivot row of a warp's columns passes through a per-warp shared buffer (no CTA
//     barrier), and
//   * the warp holding column c+1 computes that column's update first and chooses pivot c+1
//     from it (warp reductions) while the other warps run step c (look-ahead); multipliers and
//     pivot go to a double-buffered shared slot that the barrier ending the step publishes.
// Rows entering the window are fetched PF steps ahead with cp.async by the other warps.
#include "band_util.cuh"

namespace nep {

// First (smallest) index among the lanes' maxima: best/bi are a lane's own maximum and index
// (best < 0 and a large bi where the lane has no candidate).
template <typename T>
__device__ __forceinline__ int warp_argmax_first(T best, int bi) {
    if constexpr (sizeof(T) == 4) {
        // non-negative floats order like their bit patterns
        const unsigned mb = best < 0 ? 0u : __float_as_uint(best);
        const unsigned mx = __reduce_max_sync(0xffffffffu, mb);
        return (int)__reduce_min_sync(0xffffffffu, mb == mx ? (unsigned)bi : 0x7fffffffu);
    } else {
        for (int o = 16; o > 0; o >>= 1) {
            const T ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ob > best || (ob == best && oi < bi)) {
                best = ob;
                bi = oi;
            }
        }
        return bi;
    }
}

// acc - l u, the operations of fms(): for complex float as two packed f32x2 fused multiply-adds
// over (re, im), (acc.re, acc.im) + (-l.re, -l.re)(u.re, u.im) then + (l.im, -l.im)(u.im, u.re),
// lane for lane the same roundings as the scalar form.
struct LPack {
    unsigned long long nre, imm;  // (-l.re, -l.re), (l.im, -l.im)
};
__device__ __forceinline__ unsigned long long pack2(float lo, float hi) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ LPack lpack(cx<float> l) { return LPack{pack2(-l.re, -l.re), pack2(l.im, -l.im)}; }
__device__ __forceinline__ cx<float> fms_packed(cx<float> acc, const LPack& l, unsigned long long u,
                                                unsigned long long us) {
    unsigned long long a = pack2(acc.re, acc.im);
    asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(a) : "l"(l.nre), "l"(u));
    asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(a) : "l"(l.imm), "l"(us));
    cx<float> r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.re), "=f"(r.im) : "l"(a));
    return r;
}

template <typename T, int RPL, int CPW>
__global__ void __launch_bounds__(512, 1)
    lu_col_kernel(int n, int kl, int ku, int ldab, cx<T>* __restrict__ ab_all, int* __restrict__ ipiv_all,
                  int* __restrict__ info_all, const int* __restrict__ active) {
    constexpr int NW = 16, PF = 8, CS = NW * CPW;
    constexpr bool PACKED = sizeof(T) == 4;
    const int j = blockIdx.x;
    if (active && !active[j]) return;
    const int kv = kl + ku;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    cx<T>* ab = ab_all + (int64_t)j * n * ldab;
    int* ipiv = ipiv_all + (int64_t)j * n;

    // row c+kl at [c % (PF+1)]: columns c .. c+CS (zero beyond c+kv)
    __shared__ cx<T> nrow[PF + 1][CS + 1];
    __shared__ cx<T> lvec[2][32 * RPL];  // multipliers of pivot step c by row slot, at [c & 1]
    __shared__ cx<T> xrow[NW][CPW];      // per warp: the pivot row on its columns
    __shared__ int piv_s[2], info_s;
    if (threadIdx.x == 0) info_s = 0;

    bool vr[RPL];
    int lab[RPL], colk[CPW];
    cx<T> a[RPL][CPW];
#pragma unroll
    for (int q = 0; q < RPL; ++q) {
        vr[q] = lane + 32 * q < kl;
        lab[q] = vr[q] ? lane + 32 * q : 0x40000000;
    }
#pragma unroll
    for (int p = 0; p < CPW; ++p) colk[p] = warp * CPW + p;
    // rows 0..kl-1, columns 0..CS-1
#pragma unroll
    for (int q = 0; q < RPL; ++q)
#pragma unroll
        for (int p = 0; p < CPW; ++p) {
            const int r = lane + 32 * q, k = colk[p], t = k - r + kl;
            cx<T> v = mk<T>(0, 0);
            if (vr[q] && r < n && k < n && t >= 0 && t <= kv) v = ab[(int64_t)r * ldab + t];
            a[q][p] = v;
        }
    if (CS > kv)
        for (int e = threadIdx.x; e < (PF + 1) * (CS - kv); e += blockDim.x)
            nrow[e / (CS - kv)][kv + 1 + e % (CS - kv)] = mk<T>(0, 0);
    // rows kl .. kl+PF-1 (steps 0 .. PF-1): one commit group per row
    for (int d = 0; d < PF; ++d) {
        const int r = kl + d;
        for (int t = threadIdx.x; t <= kv; t += blockDim.x) {
            if (r < n && d + t < n) cp_async_cx(&nrow[d][t], ab + (int64_t)r * ldab + t);
            else nrow[d][t] = mk<T>(0, 0);
        }
        cp_async_commit();
    }

    // Pivot of column c1 by the warp holding it: col[q] is the column's value in row slot q
    // (row lab[q], in c1 .. c1+kl-1); row c1+kl enters from nrow. Writes the multipliers by row
    // slot as they stand after the interchange (and to L), U(c1,c1), ipiv and the pivot row.
    auto pivot = [&](int c1, const cx<T>(&col)[RPL]) {
        const int nb = c1 & 1, re = c1 + kl;
        const cx<T> ve = nrow[c1 % (PF + 1)][0];
        T best = T(-1);
        int bi = 0x7fffffff;
#pragma unroll
        for (int q = 0; q < RPL; ++q)
            if (vr[q] && lab[q] < n) {
                const T m = abs1(col[q]);
                if (m > best || (m == best && lab[q] < bi)) {
                    best = m;
                    bi = lab[q];
                }
            }
        if (lane == 0 && re < n) {
            const T m = abs1(ve);
            if (m > best) {  // the entering row has the largest index: ties stay in the window
                best = m;
                bi = re;
            }
        }
        int P = warp_argmax_first(best, bi);
        if (P >= n) P = c1;  // a column of NaNs matches no row: keep the diagonal
        // value of row P (P == re: the entering row), from the lane holding it
        cx<T> mP = col[0];
        bool hasP = vr[0] && lab[0] == P;
#pragma unroll
        for (int q = 1; q < RPL; ++q)
            if (vr[q] && lab[q] == P) {
                mP = col[q];
                hasP = true;
            }
        const int lP = __ffs(__ballot_sync(0xffffffffu, hasP)) - 1;
        const cx<T> vP = shfl_cx(mP, lP < 0 ? 0 : lP);
        const cx<T> pv = P == re ? ve : vP;
        const bool zero = pv.re == T(0) && pv.im == T(0);
        if (zero) P = c1;
        const cx<T> rpv = zero ? mk<T>(0, 0) : pivot_recip(pv);
        cx<T>* out = ab + (int64_t)c1 * ldab;
#pragma unroll
        for (int q = 0; q < RPL; ++q) {
            if (!vr[q]) continue;
            // after the interchange: the pivot's slot holds row re, row c1's slot row P
            int nl = lab[q];
            cx<T> val = col[q];
            if (P != re && lab[q] == P) {
                nl = re;
                val = ve;
            } else if (lab[q] == c1) {
                nl = P;
            }
            const cx<T> l = (!zero && nl < n) ? val * rpv : mk<T>(0, 0);
            lvec[nb][lane + 32 * q] = l;
            out[kv + nl - c1] = l;  // L(nl, c1) at kv + 1 + (nl - c1 - 1)
        }
        if (lane == 0) {
            out[0] = zero ? mk<T>(0, 0) : pv;
            ipiv[c1] = P;
            piv_s[nb] = P;
            if (zero && info_s == 0) info_s = c1 + 1;
        }
    };

    cp_async_wait_group<PF - 1>();  // row kl
    __syncthreads();
    if (warp == 0) {
        cx<T> col[RPL];
#pragma unroll
        for (int q = 0; q < RPL; ++q) col[q] = a[q][0];
        pivot(0, col);
    }
    // column 0 leaves: its slot holds column CS, zero in rows < kl
    if (warp == 0) {
#pragma unroll
        for (int q = 0; q < RPL; ++q) a[q][0] = mk<T>(0, 0);
        colk[0] += CS;
    }
    cp_async_wait_group<PF - 2>();  // row kl+1, for the look-ahead of step 0
    __syncthreads();

    int s1 = 1 % CS;  // column slot of column c+1
    for (int c = 0; c < n; ++c) {
        const int cb = c & 1, re = c + kl;
        const int P = piv_s[cb];
        const bool in_win = P != re;
        const cx<T>* nr = nrow[c % (PF + 1)];
        // the pivot row's slot takes the entering row; publish the pivot row on this warp's columns
        bool isp[RPL];
#pragma unroll
        for (int q = 0; q < RPL; ++q) {
            isp[q] = in_win && lab[q] == P;
            if (isp[q])
#pragma unroll
                for (int p = 0; p < CPW; ++p) xrow[warp][p] = a[q][p];
        }
        if (!in_win && lane == 0)
#pragma unroll
            for (int p = 0; p < CPW; ++p) xrow[warp][p] = nr[colk[p] - c];
        // labels after the interchange
#pragma unroll
        for (int q = 0; q < RPL; ++q) lab[q] = isp[q] ? re : (lab[q] == c ? P : lab[q]);
        cx<T> lq[RPL];
#pragma unroll
        for (int q = 0; q < RPL; ++q) lq[q] = vr[q] ? lvec[cb][lane + 32 * q] : mk<T>(0, 0);
        __syncwarp();
        cx<T>* urow = ab + (int64_t)c * ldab;
        const int w1 = s1 / CPW, p1 = s1 % CPW;
        const bool look = warp == w1 && c + 1 < n;
        if (look) {
            // column c+1 after step c, for the pivot of step c+1
            const cx<T> u1 = xrow[warp][p1], vn1 = nr[1];
            cx<T> col[RPL];
#pragma unroll
            for (int p = 0; p < CPW; ++p)
                if (p == p1)
#pragma unroll
                    for (int q = 0; q < RPL; ++q) col[q] = fms(isp[q] ? vn1 : a[q][p], lq[q], u1);
            pivot(c + 1, col);
        }
        // step c on every column of this warp (interchange, entering row, U(c, k), rank-1)
        if constexpr (PACKED) {
            LPack lp[RPL];
#pragma unroll
            for (int q = 0; q < RPL; ++q) lp[q] = lpack(reinterpret_cast<const cx<float>&>(lq[q]));
#pragma unroll
            for (int p = 0; p < CPW; ++p) {
                const int t = colk[p] - c;
                const cx<T> u = xrow[warp][p], vn = nr[t];
                if (lane == p && t <= kv && colk[p] < n) urow[t] = u;
                const unsigned long long u2 = pack2(u.re, u.im), us2 = pack2(u.im, u.re);
#pragma unroll
                for (int q = 0; q < RPL; ++q) {
                    const cx<T> x = isp[q] ? vn : a[q][p];
                    a[q][p] = fms_packed(x, lp[q], u2, us2);
                }
            }
        } else {
#pragma unroll
            for (int p = 0; p < CPW; ++p) {
                const int t = colk[p] - c;
                const cx<T> u = xrow[warp][p], vn = nr[t];
                if (lane == p && t <= kv && colk[p] < n) urow[t] = u;
#pragma unroll
                for (int q = 0; q < RPL; ++q) a[q][p] = fms(isp[q] ? vn : a[q][p], lq[q], u);
            }
        }
        // column c+1 leaves at step c+1: its slot holds column c+1+CS, zero in the window rows
#pragma unroll
        for (int p = 0; p < CPW; ++p)
            if (colk[p] == c + 1) {
#pragma unroll
                for (int q = 0; q < RPL; ++q) a[q][p] = mk<T>(0, 0);
                colk[p] += CS;
            }
        // row c+kl+PF (columns c+PF .. c+PF+kv) into the ring slot step c-1 freed, by the warps
        // after the look-ahead warp
        {
            const int idx = ((warp - w1 - 1 + NW) % NW) * 32 + lane;
            const int r = c + kl + PF;
            cx<T>* dst = nrow[(c + PF) % (PF + 1)];
            if (idx < (NW - 1) * 32 && idx <= kv) {
                if (r < n && c + PF + idx < n) cp_async_cx(&dst[idx], ab + (int64_t)r * ldab + idx);
                else dst[idx] = mk<T>(0, 0);
            }
            cp_async_commit();
        }
        s1 = s1 + 1 == CS ? 0 : s1 + 1;
        cp_async_wait_group<PF - 2>();  // row c+2+kl, for the look-ahead of step c+1
        __syncthreads();                // pivot c+1 published; xrow and lvec[cb] free
    }
    if (threadIdx.x == 0) info_all[j] = info_s;
}

bool band_lu_col_fits(int kl, int ku) { return kl >= 1 && kl <= 64 && ku >= 0 && kl + ku <= 128; }

template <typename T, int RPL, int CPW>
static int run_col(const SplitDev& s, int npts, cx<T>* ab, int* ipiv, int* info, const int* active, cudaStream_t st) {
    lu_col_kernel<T, RPL, CPW><<<npts, 512, 0, st>>>(s.n, s.kl, s.ku, s.ldab, ab, ipiv, info, active);
    NEP_CHECK_LAUNCH();
    return NEP_OK;
}

template <typename T, int RPL>
static int col_cpw(const SplitDev& s, int npts, cx<T>* ab, int* ipiv, int* info, const int* active, cudaStream_t st) {
    // 16 warps x CPW column slots >= kl + ku, CPW even
    const int cpw = ((s.kl + s.ku + 15) / 16 + 1) & ~1;
    switch (cpw) {
        case 2: return run_col<T, RPL, 2>(s, npts, ab, ipiv, info, active, st);
        case 4: return run_col<T, RPL, 4>(s, npts, ab, ipiv, info, active, st);
        case 6: return run_col<T, RPL, 6>(s, npts, ab, ipiv, info, active, st);
        case 8: return run_col<T, RPL, 8>(s, npts, ab, ipiv, info, active, st);
    }
    return NEP_ERR_INTERNAL;
}

template <typename T>
int launch_band_lu_col(const SplitDev& s, int npts, cx<T>* ab, int* ipiv, int* info, const int* active,
                       cudaStream_t st) {
    if (npts <= 0) return NEP_OK;
    if (!band_lu_col_fits(s.kl, s.ku)) return NEP_ERR_INTERNAL;
    return s.kl <= 32 ? col_cpw<T, 1>(s, npts, ab, ipiv, info, active, st)
                      : col_cpw<T, 2>(s, npts, ab, ipiv, info, active, st);
}

template int launch_band_lu_col<float>(const SplitDev&, int, cx<float>*, int*, int*, const int*, cudaStream_t);
template int launch_band_lu_col<double>(const SplitDev&, int, cx<double>*, int*, int*, const int*, cudaStream_t);

}  // namespace nep

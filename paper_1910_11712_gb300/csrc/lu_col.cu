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
// column slot s (warp s % 16, register s / 16, s < CS = 16 CPW >= kl+ku, a power of two) holds
// column k with k mod CS = s. An interchange moves no data: the pivot row leaves the window
// as row c of U, the entering row c+kl takes over its slot, and the slot of row c takes the
// pivot row's label. The slot column c+1 leaves after step c+1's pivot takes column c+1+CS,
// zero in every window row (beyond the band, or the band's next column when CS = kl+ku).
// A column is held by one warp, so
//   * the pivot row of a warp's columns passes through a per-warp shared buffer (no CTA
//     barrier), and
//   * the warp holding column c+1 computes that column's update and chooses pivot c+1 from it
//     (warp reductions) while the other warps run step c (look-ahead); multipliers and pivot go
//     to a double-buffered shared slot that the barrier ending the step publishes. That warp
//     runs its own part of step c at the start of step c+1, when the look-ahead has moved to the
//     next warp (consecutive columns sit in consecutive warps), so the chain between two
//     barriers is one column update and one pivot choice.
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

// Packed pairs of floats for fma.rn.f32x2 (sm_100 and later): every lane is an ordinary fused
// multiply-add with one rounding.
__device__ __forceinline__ unsigned long long pack2(float lo, float hi) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void unpack2(unsigned long long v, float& lo, float& hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ unsigned long long fma2(unsigned long long a, unsigned long long b, unsigned long long c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// v, or +0 when z (by bit mask)
template <typename T>
__device__ __forceinline__ cx<T> mask_cx(cx<T> v, bool z) {
    if constexpr (sizeof(T) == 8) {
        const long long keep = z ? 0ll : -1ll;
        return mk<T>(__longlong_as_double(__double_as_longlong(v.re) & keep),
                     __longlong_as_double(__double_as_longlong(v.im) & keep));
    } else {
        const int keep = z ? 0 : -1;
        return mk<T>(__int_as_float(__float_as_int(v.re) & keep), __int_as_float(__float_as_int(v.im) & keep));
    }
}

template <typename T, int RPL, int CPW>
__global__ void __launch_bounds__(512, 1)
    lu_col_kernel(int n, int kl, int ku, int ldab, cx<T>* __restrict__ ab_all, int* __restrict__ ipiv_all,
                  int* __restrict__ info_all, const int* __restrict__ active, const PointDesc* __restrict__ pd) {
    constexpr int NW = 16, PF = 8, RING = PF + 2, CS = NW * CPW;  // CS a power of two
    // complex float: the column registers pair up, (2h, 2h+1), one 64-bit register for the two
    // real parts of a row and one for the imaginary parts. With u = (u0, u1) the pivot row on the
    // pair and l the row's multiplier, a pair's update is four f32x2 fused multiply-adds,
    // re -= l.re u.re, re += l.im u.im, im -= l.re u.im, im -= l.im u.re: the operations of fms()
    // lane for lane. The pivot row's registers are the broadcast format as they stand.
    constexpr bool PAIRED = sizeof(T) == 4 && CPW % 2 == 0;
    constexpr int CPH = PAIRED ? CPW / 2 : 1;
    static_assert((CS & (CS - 1)) == 0, "column slots must be a power of two");
    int j = blockIdx.x;
    if (pd) {  // a point of one of several problems sharing the launch
        const PointDesc d = pd[blockIdx.x];
        n = d.n, kl = d.kl, ku = d.ku, ldab = d.ldab;
        ab_all = static_cast<cx<T>*>(d.ab), ipiv_all = d.ipiv, info_all = d.info, active = d.active;
        j = 0;
    }
    if (active && !active[j]) return;
    const int kv = kl + ku;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    cx<T>* ab = ab_all + (int64_t)j * n * ldab;
    int* ipiv = ipiv_all + (int64_t)j * n;

    // Row c+kl enters at step c from ring entry c % RING (RING = PF + 2 keeps row c-1+kl readable
    // during step c): its value in column c in n0, and columns c+1 .. c+CS (zero beyond c+kv) in
    // column-slot order, so that a warp's part is where its registers want it: per warp and
    // register pair (re 2h, re 2h+1, im 2h, im 2h+1) when PAIRED, per warp and register otherwise.
    __shared__ ulonglong2 nsp[PAIRED ? RING : 1][PAIRED ? NW : 1][CPH];
    __shared__ cx<T> nsg[PAIRED ? 1 : RING][PAIRED ? 1 : NW][CPW];
    __shared__ cx<T> n0[RING];
    // multipliers of pivot step c by row slot at [c % 3] (three buffers: the warp that runs step c
    // late reads them during step c+1, while pivot c+2 is written); when PAIRED also as the packed
    // operands (-l.re, -l.re), (l.im, l.im), (-l.im, -l.im)
    __shared__ cx<T> lvec[3][32 * RPL];
    __shared__ unsigned long long lvp[PAIRED ? 3 : 1][3][32 * RPL];
    // per warp: the pivot row on its columns; when PAIRED, (re 2h, re 2h+1, im 2h, im 2h+1)
    __shared__ ulonglong2 xrow2[PAIRED ? NW : 1][CPH];
    __shared__ cx<T> xrow[PAIRED ? 1 : NW][PAIRED ? 1 : CPW];
    __shared__ int piv_s[3], info_s;
    if (threadIdx.x == 0) info_s = 0;

    cx<T> a[PAIRED ? 1 : RPL][CPW] = {};
    unsigned long long are[PAIRED ? RPL : 1][CPH] = {}, aim[PAIRED ? RPL : 1][CPH] = {};
    auto get = [&](int q, int p) __attribute__((always_inline)) -> cx<T> {
        if constexpr (PAIRED) {
            float r0, r1, i0, i1;
            unpack2(are[q][p >> 1], r0, r1);
            unpack2(aim[q][p >> 1], i0, i1);
            return (p & 1) ? mk<T>(r1, i1) : mk<T>(r0, i0);
        } else {
            return a[q][p];
        }
    };
    auto set = [&](int q, int p, cx<T> v) __attribute__((always_inline)) {
        if constexpr (PAIRED) {
            float r0, r1, i0, i1;
            unpack2(are[q][p >> 1], r0, r1);
            unpack2(aim[q][p >> 1], i0, i1);
            if (p & 1) {
                r1 = v.re;
                i1 = v.im;
            } else {
                r0 = v.re;
                i0 = v.im;
            }
            are[q][p >> 1] = pack2(r0, r1);
            aim[q][p >> 1] = pack2(i0, i1);
        } else {
            a[q][p] = v;
        }
    };
    // the broadcast pivot row: element p of this warp's columns
    auto get_u = [&](int p) __attribute__((always_inline)) -> cx<T> {
        if constexpr (PAIRED) {
            const float* f = reinterpret_cast<const float*>(&xrow2[warp][p >> 1]);
            return mk<T>(f[p & 1], f[2 + (p & 1)]);
        } else {
            return xrow[warp][p];
        }
    };
    // column slots interleave over the warps: slot s = p*NW + warp. Before step c the slot holds
    // column k = c+1+((s-c-1) mod CS); toff is k - c
    auto toff = [&](int p, int c) __attribute__((always_inline)) { return 1 + ((p * NW + warp - c - 1) & (CS - 1)); };

    bool vr[RPL];
    int lab[RPL];
#pragma unroll
    for (int q = 0; q < RPL; ++q) {
        vr[q] = lane + 32 * q < kl;
        lab[q] = vr[q] ? lane + 32 * q : 0x40000000;
    }
    // rows 0..kl-1, columns 0..CS-1 (slot s holds column s until pivot 0 has used column 0)
#pragma unroll
    for (int p = 0; p < CPW; ++p) {
#pragma unroll
        for (int q = 0; q < RPL; ++q) {
            const int r = lane + 32 * q, k = p * NW + warp, t = k - r + kl;
            cx<T> v = mk<T>(0, 0);
            if (vr[q] && r < n && k < n && t >= 0 && t <= kv) v = ab[(int64_t)r * ldab + t];
            set(q, p, v);
        }
    }
    // element t (0 .. CS) of row r = c0 + kl, the row entering at step c0, into ring entry e
    auto fetch = [&](int e, int c0, int t) __attribute__((always_inline)) {
        const int r = c0 + kl, k = c0 + t;
        const bool in = r < n && k < n && t <= kv;
        const cx<T>* src = ab + (int64_t)r * ldab + t;
        if (t == 0) {
            if (in) cp_async_cx(&n0[e], src);
            else n0[e] = mk<T>(0, 0);
            return;
        }
        const int sl = k & (CS - 1), w = sl & (NW - 1), p = sl / NW;
        if constexpr (PAIRED) {
            float* f = reinterpret_cast<float*>(&nsp[e][w][p >> 1]);
            if (in) {
                cp_async_f32(f + (p & 1), reinterpret_cast<const float*>(src));
                cp_async_f32(f + 2 + (p & 1), reinterpret_cast<const float*>(src) + 1);
            } else {
                f[p & 1] = 0.f;
                f[2 + (p & 1)] = 0.f;
            }
        } else {
            if (in) cp_async_cx(&nsg[e][w][p], src);
            else nsg[e][w][p] = mk<T>(0, 0);
        }
    };
    // rows kl .. kl+PF-1 (steps 0 .. PF-1): one commit group per row
    for (int d = 0; d < PF; ++d) {
        for (int t = threadIdx.x; t <= CS; t += blockDim.x) fetch(d, d, t);
        cp_async_commit();
    }

    // Pivot of column c1 by the warp holding it: col[q] is the column's value in row slot q
    // (row lab[q], in c1 .. c1+kl-1); row c1+kl enters from the ring. Writes the multipliers by row
    // slot as they stand after the interchange (and to L), U(c1,c1), ipiv and the pivot row.
    auto pivot = [&](int c1, const cx<T>(&col)[RPL]) __attribute__((always_inline)) {
        const int nb = c1 % 3, re = c1 + kl;
        const cx<T> ve = n0[c1 % RING];
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
            if constexpr (PAIRED) {
                lvp[nb][0][lane + 32 * q] = pack2(-l.re, -l.re);
                lvp[nb][1][lane + 32 * q] = pack2(l.im, l.im);
                lvp[nb][2][lane + 32 * q] = pack2(-l.im, -l.im);
            }
            out[kv + nl - c1] = l;  // L(nl, c1) at kv + 1 + (nl - c1 - 1)
        }
        if (lane == 0) {
            out[0] = zero ? mk<T>(0, 0) : pv;
            ipiv[c1] = P;
            piv_s[nb] = P;
            if (zero && info_s == 0) info_s = c1 + 1;
        }
    };

    // Step cc on this warp's columns: publish the pivot row (row Pc; the entering row when
    // Pc = cc+kl), the pivot's slot takes the entering row, a(r, k) -= l(r) u(k), U(cc, k) to
    // the band, and the slot of column cc+1 (if this warp holds it) empties for column cc+1+CS.
    auto run_step = [&](int cc, int Pc, const bool(&ispc)[RPL]) __attribute__((always_inline)) {
        const int e = cc % RING, lb = cc % 3;
        // the pivot row's lane publishes its registers, then takes the entering row into them
#pragma unroll
        for (int q = 0; q < RPL; ++q)
            if (ispc[q]) {
                if constexpr (PAIRED) {
#pragma unroll
                    for (int h = 0; h < CPH; ++h) {
                        xrow2[warp][h] = make_ulonglong2(are[q][h], aim[q][h]);
                        const ulonglong2 v = nsp[e][warp][h];
                        are[q][h] = v.x;
                        aim[q][h] = v.y;
                    }
                } else {
#pragma unroll
                    for (int p = 0; p < CPW; ++p) {
                        xrow[warp][p] = a[q][p];
                        a[q][p] = nsg[e][warp][p];
                    }
                }
            }
        if (Pc == cc + kl && lane == 0) {  // the pivot is the entering row itself
            if constexpr (PAIRED) {
#pragma unroll
                for (int h = 0; h < CPH; ++h) xrow2[warp][h] = nsp[e][warp][h];
            } else {
#pragma unroll
                for (int p = 0; p < CPW; ++p) xrow[warp][p] = nsg[e][warp][p];
            }
        }
        __syncwarp();
        if constexpr (PAIRED) {
            unsigned long long nlre[RPL], lim[RPL], nlim[RPL];
#pragma unroll
            for (int q = 0; q < RPL; ++q) {
                nlre[q] = vr[q] ? lvp[lb][0][lane + 32 * q] : 0ull;
                lim[q] = vr[q] ? lvp[lb][1][lane + 32 * q] : 0ull;
                nlim[q] = vr[q] ? lvp[lb][2][lane + 32 * q] : 0ull;
            }
#pragma unroll
            for (int h = 0; h < CPH; ++h) {
                const ulonglong2 u = xrow2[warp][h];  // (re pair, im pair)
#pragma unroll
                for (int q = 0; q < RPL; ++q) {
                    are[q][h] = fma2(nlre[q], u.x, are[q][h]);
                    are[q][h] = fma2(lim[q], u.y, are[q][h]);
                    aim[q][h] = fma2(nlre[q], u.y, aim[q][h]);
                    aim[q][h] = fma2(nlim[q], u.x, aim[q][h]);
                }
            }
        } else {
            cx<T> lqc[RPL];
#pragma unroll
            for (int q = 0; q < RPL; ++q) lqc[q] = vr[q] ? lvec[lb][lane + 32 * q] : mk<T>(0, 0);
#pragma unroll
            for (int p = 0; p < CPW; ++p) {
                const cx<T> u = xrow[warp][p];
#pragma unroll
                for (int q = 0; q < RPL; ++q) a[q][p] = fms(a[q][p], lqc[q], u);
            }
        }
        if (lane < CPW) {
            const int t = toff(lane, cc);
            if (t <= kv && cc + t < n) ab[(int64_t)cc * ldab + t] = get_u(lane);
        }
        // the slot of column cc+1 empties for column cc+1+CS (in the warp holding it; a bit
        // mask on every register rather than a store to one chosen at run time, which would
        // move the window out of registers)
        const int s1 = (cc + 1) & (CS - 1);
        if ((s1 & (NW - 1)) == warp) {
            const int pz = s1 / NW;
            if constexpr (PAIRED) {
                const unsigned long long keep = (pz & 1) ? 0x00000000ffffffffull : 0xffffffff00000000ull;
#pragma unroll
                for (int h = 0; h < CPH; ++h) {
                    const unsigned long long m = h == (pz >> 1) ? keep : ~0ull;
#pragma unroll
                    for (int q = 0; q < RPL; ++q) {
                        are[q][h] &= m;
                        aim[q][h] &= m;
                    }
                }
            } else {
#pragma unroll
                for (int p = 0; p < CPW; ++p)
#pragma unroll
                    for (int q = 0; q < RPL; ++q) a[q][p] = mask_cx(a[q][p], p == pz);
            }
        }
        __syncwarp();  // the buffer is read before the next step publishes into it
    };

    cp_async_wait_group<PF - 1>();  // row kl
    __syncthreads();
    if (warp == 0) {
        cx<T> col[RPL];
#pragma unroll
        for (int q = 0; q < RPL; ++q) col[q] = get(q, 0);
        pivot(0, col);
        // column 0 leaves: its slot holds column CS, zero in rows < kl
#pragma unroll
        for (int q = 0; q < RPL; ++q) set(q, 0, mk<T>(0, 0));
    }
    cp_async_wait_group<PF - 2>();  // row kl+1, for the look-ahead of step 0
    __syncthreads();

    // the warp that chose pivot c+1 during step c runs its own step c at the start of step c+1
    bool deferred = false;
    int Pd = 0;
    bool ispd[RPL];
#pragma unroll
    for (int q = 0; q < RPL; ++q) ispd[q] = false;
    for (int c = 0; c < n; ++c) {
        if (deferred) {
            run_step(c - 1, Pd, ispd);
            deferred = false;
        }
        const int cb = c % 3, re = c + kl;
        const int P = piv_s[cb];
        bool isp[RPL];
#pragma unroll
        for (int q = 0; q < RPL; ++q) {
            isp[q] = P != re && lab[q] == P;
            lab[q] = isp[q] ? re : (lab[q] == c ? P : lab[q]);  // labels after the interchange
        }
        const int s1 = (c + 1) & (CS - 1), w1 = s1 & (NW - 1), p1 = s1 / NW;
        if (warp == w1 && c + 1 < n) {
            // column c+1 after step c, for the pivot of step c+1 (look-ahead); the rest of step
            // c on this warp's columns waits for the next step
            cx<T> lq[RPL], mine[RPL];
#pragma unroll
            for (int q = 0; q < RPL; ++q) lq[q] = vr[q] ? lvec[cb][lane + 32 * q] : mk<T>(0, 0);
#pragma unroll
            for (int q = 0; q < RPL; ++q) mine[q] = mk<T>(0, 0);
#pragma unroll
            for (int p = 0; p < CPW; ++p)
                if (p == p1)
#pragma unroll
                    for (int q = 0; q < RPL; ++q) mine[q] = get(q, p);
            cx<T> up = mine[0];
            bool has = isp[0];
#pragma unroll
            for (int q = 1; q < RPL; ++q)
                if (isp[q]) {
                    up = mine[q];
                    has = true;
                }
            const int lp = __ffs(__ballot_sync(0xffffffffu, has)) - 1;
            cx<T> vn1;  // the entering row in column c+1
            if constexpr (PAIRED) {
                const float* f = reinterpret_cast<const float*>(&nsp[c % RING][warp][p1 >> 1]);
                vn1 = mk<T>(f[p1 & 1], f[2 + (p1 & 1)]);
            } else {
                vn1 = nsg[c % RING][warp][p1];
            }
            const cx<T> u1 = P == re ? vn1 : shfl_cx(up, lp < 0 ? 0 : lp);
            cx<T> col[RPL];
#pragma unroll
            for (int q = 0; q < RPL; ++q) col[q] = fms(isp[q] ? vn1 : mine[q], lq[q], u1);
            pivot(c + 1, col);
            deferred = true;
            Pd = P;
#pragma unroll
            for (int q = 0; q < RPL; ++q) ispd[q] = isp[q];
        } else {
            run_step(c, P, isp);
        }
        // row c+kl+PF into ring entry (c+PF) % RING, by the warps after the look-ahead warp (the
        // one behind it runs two steps' updates in this step)
        {
            const int idx = ((warp - w1 - 1) & (NW - 1)) * 32 + lane;
            if (idx < (NW - 2) * 32 && idx <= CS) fetch((c + PF) % RING, c + PF, idx);
            cp_async_commit();
        }
        cp_async_wait_group<PF - 2>();  // row c+2+kl, for the look-ahead of step c+1
        __syncthreads();                // pivot c+1 published
    }
    if (threadIdx.x == 0) info_all[j] = info_s;
}

bool band_lu_col_fits(int kl, int ku) { return kl >= 1 && kl <= 64 && ku >= 0 && kl + ku <= 128; }

template <typename T, int RPL, int CPW>
static int run_col(const SplitDev& s, int npts, cx<T>* ab, int* ipiv, int* info, const int* active, cudaStream_t st,
                   const PointDesc* pd = nullptr) {
    lu_col_kernel<T, RPL, CPW><<<npts, 512, 0, st>>>(s.n, s.kl, s.ku, s.ldab, ab, ipiv, info, active, pd);
    NEP_CHECK_LAUNCH();
    return NEP_OK;
}

template <typename T, int RPL>
static int col_cpw(int kv, const SplitDev& s, int npts, cx<T>* ab, int* ipiv, int* info, const int* active,
                   cudaStream_t st, const PointDesc* pd) {
    // 16 warps x CPW column slots >= kl + ku, CPW a power of two
    if (kv <= 16) return run_col<T, RPL, 1>(s, npts, ab, ipiv, info, active, st, pd);
    if (kv <= 32) return run_col<T, RPL, 2>(s, npts, ab, ipiv, info, active, st, pd);
    if (kv <= 64) return run_col<T, RPL, 4>(s, npts, ab, ipiv, info, active, st, pd);
    return run_col<T, RPL, 8>(s, npts, ab, ipiv, info, active, st, pd);
}

template <typename T>
int launch_band_lu_col(const SplitDev& s, int npts, cx<T>* ab, int* ipiv, int* info, const int* active,
                       cudaStream_t st) {
    if (npts <= 0) return NEP_OK;
    if (!band_lu_col_fits(s.kl, s.ku)) return NEP_ERR_INTERNAL;
    return s.kl <= 32 ? col_cpw<T, 1>(s.kl + s.ku, s, npts, ab, ipiv, info, active, st, nullptr)
                      : col_cpw<T, 2>(s.kl + s.ku, s, npts, ab, ipiv, info, active, st, nullptr);
}

int lu_col_instance(int kl, int ku) {
    const int kv = kl + ku;
    return (kl <= 32 ? 0 : 4) + (kv <= 16 ? 0 : kv <= 32 ? 1 : kv <= 64 ? 2 : 3);
}

template <typename T>
int launch_band_lu_col_batch(int instance, int count, const PointDesc* pd_dev, cudaStream_t st) {
    if (count <= 0) return NEP_OK;
    SplitDev s{};  // sizes and buffers come from the descriptors
    const int kv = (instance & 3) == 0 ? 16 : (instance & 3) == 1 ? 32 : (instance & 3) == 2 ? 64 : 128;
    return instance < 4 ? col_cpw<T, 1>(kv, s, count, nullptr, nullptr, nullptr, nullptr, st, pd_dev)
                        : col_cpw<T, 2>(kv, s, count, nullptr, nullptr, nullptr, nullptr, st, pd_dev);
}
template int launch_band_lu_col_batch<float>(int, int, const PointDesc*, cudaStream_t);
template int launch_band_lu_col_batch<double>(int, int, const PointDesc*, cudaStream_t);

template int launch_band_lu_col<float>(const SplitDev&, int, cx<float>*, int*, int*, const int*, cudaStream_t);
template int launch_band_lu_col<double>(const SplitDev&, int, cx<double>*, int*, int*, const int*, cudaStream_t);

}  // namespace nep

// Blocked substitution with complex64 band factors too wide for the register-window sweeps (the
// bandwidth-576 square-root problem): the same forward (row interchanges and unit lower L) and
// backward (upper U, bandwidth kl + ku) sweeps as LAPACK's banded solve, regrouped into blocks of
// NB = 16 steps so that most of the work becomes a small matrix product.
//
// Forward, block of steps c0 .. c0+nb-1, on the window of rows [c0, c0 + nb + kl):
//   * the stored L columns (each taken before the later interchanges of its factorisation) are
//     brought to the block's "panel form": column k takes the interchanges k+1 .. nb-1 of the block
//     (one thread per column). Then M_{nb-1} P_{nb-1} ... M_0 P_0 = M~_{nb-1} ... M~_0 P_{nb-1} ... P_0
//     with M~_k = I - (P_{nb-1} ... P_{k+1} l_k) e_k^T, as no later interchange touches row k;
//   * the block's interchanges are applied to the right-hand sides at once (one thread per column);
//   * the unit lower nb x nb triangle of the panel form gives x (one warp per right-hand side,
//     lane i holding row c0 + i);
//   * the rows below, [c0 + nb, c0 + nb + kl), take w -= L~21 x: a kl x nb by nb x R product, one
//     thread per row with the R right-hand sides in registers.
// Backward, block of rows top .. c1 from the bottom, on the window [top - kl - ku, c1]:
//   * the upper nb x nb triangle gives x (one warp per right-hand side);
//   * the rows above take w -= U(rows, top .. c1) x, U read straight from the band rows.
// The windows are rings of rows in shared memory; rows enter by asynchronous copies into the slots
// the finished block frees, and the next block's L columns and pivots are copied while the current
// block runs. Results equal the sweeps' up to the order of the FP32 roundings.
#include <algorithm>
#include <cstdlib>

#include "band_util.cuh"

namespace nep {

namespace {

constexpr int kBlkNB = 16;     // steps per block
constexpr int kBlkRMax = 16;   // right-hand sides per CTA (register accumulators)
constexpr int kBlkThreads = 512;
constexpr int kBlkChunk = kBlkThreads / 2;  // backward: U rows staged per chunk (two threads a row)
constexpr int kBlkUS = kBlkNB + 1;          // staged U row stride (odd: rows fall on distinct banks)

// RT right-hand-side columns per CTA (a multiple of 4; columns beyond the point's L stay zero).
// Shared memory: X (NB x RT, rows 16-byte aligned for paired loads) first, then the window ring
// (odd row stride RT + 1), then the forward's two L panels and pivots, or the backward's two U
// triangles and two staged chunks of U rows.
__host__ __device__ inline size_t blk_smem_fwd(int kl, int RT) {
    const size_t PF = kBlkNB + kl;
    return sizeof(zf) * ((size_t)kBlkNB * RT + PF * (RT + 1) + 2 * (size_t)kBlkNB * PF) + sizeof(int) * 2 * kBlkNB;
}
__host__ __device__ inline size_t blk_smem_bwd(int kv, int RT) {
    const size_t PB = kBlkNB + kv;
    return sizeof(zf) * ((size_t)kBlkNB * RT + PB * (RT + 1) + 2 * (size_t)kBlkNB * (kBlkNB + 1) +
                         2 * (size_t)kBlkChunk * kBlkUS);
}

// acc[q] -= a * x[q] for the H values x (16-byte aligned), read two at a time
template <int H>
__device__ __forceinline__ void axpy_row(zf (&acc)[H], zf a, const zf* x) {
    const float4* x2 = reinterpret_cast<const float4*>(x);
#pragma unroll
    for (int h = 0; h < H / 2; ++h) {
        const float4 v = x2[h];
        acc[2 * h] = fms(acc[2 * h], a, mk(v.x, v.y));
        acc[2 * h + 1] = fms(acc[2 * h + 1], a, mk(v.z, v.w));
    }
}

// w[q] (q in one half of the RT columns, row stride of w: 1) -= sum_k a[k] X[k][q]
template <int RT>
__device__ __forceinline__ void update_half(zf* w, const zf (&a)[kBlkNB], const zf* X1, int half) {
    constexpr int H = RT / 2;
    zf acc[H];
#pragma unroll
    for (int q = 0; q < H; ++q) acc[q] = w[q];
#pragma unroll
    for (int k = 0; k < kBlkNB; ++k) axpy_row<H>(acc, a[k], X1 + k * RT + half * H);
#pragma unroll
    for (int q = 0; q < H; ++q) w[q] = acc[q];
}

template <int RT>
__global__ void __launch_bounds__(kBlkThreads, 1)
    band_solve_blocked_kernel(int n, int kl, int ku, int ldab, const zf* __restrict__ ab_all,
                              const int* __restrict__ ipiv_all, int L, zf* __restrict__ B_all,
                              const int* __restrict__ active) {
    const int j = blockIdx.x;
    if (active && !active[j]) return;
    const int q0 = blockIdx.y * RT;
    const int nr = min(RT, L - q0);
    if (nr <= 0) return;
    constexpr int NB = kBlkNB, RS = RT + 1, H = RT / 2;
    const int kv = kl + ku;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nthr = blockDim.x, nwarp = nthr >> 5;
    const zf* ab = ab_all + (int64_t)j * n * ldab;
    const int* ipiv = ipiv_all + (int64_t)j * n;
    zf* B = B_all + ((int64_t)j * L + q0) * n;  // right-hand side q at B + q n
    extern __shared__ __align__(16) unsigned char smem_raw[];
    zf* X1 = reinterpret_cast<zf*>(smem_raw);  // NB x RT: the block's solution rows (zero padded)
    zf* sm = X1 + NB * RT;
    const zf zero = mk(0.0f, 0.0f);
    for (int e = tid; e < NB * RT; e += nthr) X1[e] = zero;

    // ===================================================================== forward
    {
        const int PF = NB + kl;
        zf* W = sm;                                 // PF x RS: row r at slot r mod PF
        zf* Lp0 = W + (size_t)PF * RS;              // 2 x (NB columns of PF local rows)
        int* pv0 = reinterpret_cast<int*>(Lp0 + 2 * (size_t)NB * PF);  // 2 x NB pivots
        auto Lp = [&](int b) { return Lp0 + (size_t)b * NB * PF; };
        for (int e = tid; e < 2 * NB * PF; e += nthr) Lp0[e] = zero;
        for (int q = 0; q < RT; ++q)
            for (int r = tid; r < PF; r += nthr) W[r * RS + q] = (r < n && q < nr) ? B[(int64_t)q * n + r] : zero;
        __syncthreads();
        // column k of the panel at c0: local rows k+1 .. k+kl from the stored L column c0+k, rows
        // beyond k+kl zero (an earlier block's interchanges may have left values there); rows 0 .. k
        // are never written
        auto issue_panel = [&](int c0, int b) {
            const int nbc = min(NB, n - c0);
            zf* P = Lp(b);
            for (int k = 0; k < nbc; ++k) {
                const zf* src = ab + (int64_t)(c0 + k) * ldab + kv + 1;
                zf* dst = P + (size_t)k * PF + k + 1;
                for (int i = tid; i < kl; i += nthr) cp_async_cx(dst + i, src + i);
            }
            if (tid < NB * NB) {
                const int k = tid / NB, i = tid - k * NB;
                if (i < NB - 1 - k) P[(size_t)k * PF + k + kl + 1 + i] = zero;
            }
            if (tid < nbc) cp_async_i32(&pv0[b * NB + tid], ipiv + c0 + tid);
            cp_async_commit();
        };
        issue_panel(0, 0);
        int sbase = 0;  // slot of row c0
        for (int c0 = 0, blk = 0; c0 < n; c0 += NB, ++blk) {
            const int nbc = min(NB, n - c0);
            const int b = blk & 1;
            cp_async_wait_group<0>();
            __syncthreads();
            if (c0 + NB < n) issue_panel(c0 + NB, b ^ 1);
            zf* P = Lp(b);
            const int* pv = pv0 + b * NB;
            if (tid < nbc) {  // panel form of column k
                zf* col = P + (size_t)tid * PF;
                for (int kp = tid + 1; kp < nbc; ++kp) {
                    const int p = pv[kp] - c0;
                    if (p != kp) {
                        const zf t = col[kp];
                        col[kp] = col[p];
                        col[p] = t;
                    }
                }
            } else if (tid >= 32 && tid < 32 + nr) {  // the block's interchanges, in order
                const int q = tid - 32;
                for (int k = 0; k < nbc; ++k) {
                    const int p = pv[k] - c0;
                    if (p != k) {
                        int s1 = sbase + k, s2 = sbase + p;
                        if (s1 >= PF) s1 -= PF;
                        if (s2 >= PF) s2 -= PF;
                        const zf t = W[s1 * RS + q];
                        W[s1 * RS + q] = W[s2 * RS + q];
                        W[s2 * RS + q] = t;
                    }
                }
            }
            __syncthreads();
            for (int q = warp; q < nr; q += nwarp) {  // unit lower triangle of the panel form
                int s = sbase + lane;
                if (s >= PF) s -= PF;
                zf w = lane < nbc ? W[s * RS + q] : zero;
                for (int k = 0; k + 1 < nbc; ++k) {
                    const zf xk = shfl_cx(w, k);
                    if (lane > k && lane < nbc) w = fms(w, P[(size_t)k * PF + lane], xk);
                }
                if (lane < NB) X1[lane * RT + q] = w;  // zero beyond the block's nbc rows
                if (lane < nbc) B[(int64_t)q * n + c0 + lane] = w;
            }
            __syncthreads();
            // rows c0 + PF + i enter the slots of the finished rows c0 + i
            for (int e = tid; e < nbc * nr; e += nthr) {
                const int i = e % nbc, q = e / nbc;
                const int r = c0 + PF + i;
                int s = sbase + i;
                if (s >= PF) s -= PF;
                if (r < n) cp_async_cx(&W[s * RS + q], B + (int64_t)q * n + r);
                else W[s * RS + q] = zero;
            }
            cp_async_commit();
            // rows below the block: w -= L~21 x, two threads a row (one half of the columns each);
            // columns of P beyond nbc meet zero rows of X1
            const int rows = min(kl, n - c0 - nbc);
            for (int t = tid; t < 2 * rows; t += nthr) {
                const int lr = nbc + (t >> 1), half = t & 1;
                int s = sbase + lr;
                if (s >= PF) s -= PF;
                zf a[NB];
#pragma unroll
                for (int k = 0; k < NB; ++k) a[k] = P[(size_t)k * PF + lr];
                update_half<RT>(W + s * RS + half * H, a, X1, half);
            }
            sbase += nbc;
            if (sbase >= PF) sbase -= PF;
        }
        cp_async_wait_group<0>();
        __syncthreads();
    }

    // ===================================================================== backward
    {
        const int PB = NB + kv;
        zf* W = sm;                                  // PB x RS: row r at slot r mod PB
        zf* U0 = W + (size_t)PB * RS;                // 2 x NB x (NB+1): U(top+i, top+k) at i (NB+1) + k
        zf* S0 = U0 + 2 * (size_t)NB * (NB + 1);     // 2 x kBlkChunk x kBlkUS staged U rows
        auto issue_u11 = [&](int c1, int b) {
            const int top = max(0, c1 - NB + 1), nbc = c1 - top + 1;
            zf* Ub = U0 + (size_t)b * NB * (NB + 1);
            if (tid < NB * NB) {
                const int i = tid / NB, k = tid - i * NB;
                if (i < nbc && k < nbc && k >= i) {
                    if (k - i <= kv) cp_async_cx(&Ub[i * (NB + 1) + k], ab + (int64_t)(top + i) * ldab + (k - i));
                    else Ub[i * (NB + 1) + k] = zero;  // beyond the band (kl + ku < NB - 1)
                }
            }
            cp_async_commit();
        };
        // chunk ch of the block ending at row c1: rows top - kv + ch kBlkChunk + l, their entries
        // U(r, top .. top + NB - 1) (zero beyond the band and beyond the block)
        const int nch = (kv + kBlkChunk - 1) / kBlkChunk;
        auto issue_chunk = [&](int c1, int ch, int b) {
            const int top = max(0, c1 - NB + 1), nbc = c1 - top + 1;
            zf* S = S0 + (size_t)b * kBlkChunk * kBlkUS;
            for (int e = tid; e < kBlkChunk * NB; e += nthr) {
                const int l = e >> 4, k = e & (NB - 1);
                const int t = ch * kBlkChunk + l;
                const int r = top - kv + t;
                const int off = top - r;
                zf* dst = S + l * kBlkUS + k;
                if (t < kv && r >= 0 && k < nbc && off + k <= kv) cp_async_cx(dst, ab + (int64_t)r * ldab + off + k);
                else *dst = zero;
            }
            cp_async_commit();
        };
        for (int q = 0; q < RT; ++q)
            for (int r = max(0, n - PB) + tid; r < n; r += nthr) W[(r % PB) * RS + q] = q < nr ? B[(int64_t)q * n + r] : zero;
        for (int e = tid; e < NB * RT; e += nthr) X1[e] = zero;
        issue_u11(n - 1, 0);
        issue_chunk(n - 1, 0, 0);
        int sb = 0;  // staging buffer of the next chunk to compute
        for (int c1 = n - 1, blk = 0; c1 >= 0; c1 -= NB, ++blk) {
            const int top = max(0, c1 - NB + 1), nbc = c1 - top + 1;
            const int b = blk & 1;
            cp_async_wait_group<0>();
            __syncthreads();
            if (top > 0) issue_u11(top - 1, b ^ 1);
            const zf* Ub = U0 + (size_t)b * NB * (NB + 1);
            for (int q = warp; q < nr; q += nwarp) {  // upper triangle, bottom row first
                const zf rd = lane < nbc ? pivot_recip(Ub[lane * (NB + 1) + lane]) : zero;
                zf w = lane < nbc ? W[((top + lane) % PB) * RS + q] : zero;
                for (int k = nbc - 1; k >= 0; --k) {
                    const zf xk = shfl_cx(w, k) * shfl_cx(rd, k);
                    if (lane == k) w = xk;
                    else if (lane < k) w = fms(w, Ub[lane * (NB + 1) + k], xk);
                }
                if (lane < NB) X1[lane * RT + q] = lane < nbc ? w : zero;
                if (lane < nbc) B[(int64_t)q * n + top + lane] = w;
            }
            __syncthreads();
            // rows top - PB + i enter the slots of the finished rows top + i
            for (int e = tid; e < nbc * nr; e += nthr) {
                const int i = e % nbc, q = e / nbc;
                const int r = top - PB + i;
                if (r >= 0) cp_async_cx(&W[((top + i) % PB) * RS + q], B + (int64_t)q * n + r);
            }
            cp_async_commit();
            // rows above the block, a chunk of staged U rows at a time: w -= U(r, top .. c1) x
            for (int ch = 0; ch < nch; ++ch) {
                if (ch > 0) {
                    cp_async_wait_group<0>();
                    __syncthreads();
                }
                if (ch + 1 < nch) issue_chunk(c1, ch + 1, sb ^ 1);
                else if (top > 0) issue_chunk(top - 1, 0, sb ^ 1);
                const zf* S = S0 + (size_t)sb * kBlkChunk * kBlkUS;
                const int l = tid >> 1, half = tid & 1;
                const int t = ch * kBlkChunk + l;
                const int r = top - kv + t;
                if (t < kv && r >= 0) {
                    zf a[NB];
#pragma unroll
                    for (int k = 0; k < NB; ++k) a[k] = S[l * kBlkUS + k];
                    update_half<RT>(W + (r % PB) * RS + half * H, a, X1, half);
                }
                sb ^= 1;
            }
        }
        cp_async_wait_group<0>();
    }
}

}  // namespace

// Right-hand sides per CTA: the fewest CTAs per point with at most kBlkRMax columns each (rounded
// up to a multiple of 4) whose windows fit in shared memory; 0 if none does
int band_solve_blocked_rhs(int kl, int ku, int L) {
    const int kv = kl + ku;
    for (int groups = (L + kBlkRMax - 1) / kBlkRMax; groups <= L; ++groups) {
        const int RT = (((L + groups - 1) / groups) + 3) / 4 * 4;
        const size_t bytes = std::max(blk_smem_fwd(kl, RT), blk_smem_bwd(kv, RT));
        if (bytes <= 220 * 1024) return RT;
        if (RT == 4) break;
    }
    return 0;
}

template <int RT>
static int launch_blocked(const SplitDev& s, int npts, const zf* ab, const int* ipiv, int L, zf* B, const int* active,
                          cudaStream_t st) {
    const int kv = s.kl + s.ku;
    const size_t smem = std::max(blk_smem_fwd(s.kl, RT), blk_smem_bwd(kv, RT));
    NEP_CUDA(allow_max_dynamic_smem(band_solve_blocked_kernel<RT>));
    dim3 grid(npts, (L + RT - 1) / RT);
    band_solve_blocked_kernel<RT><<<grid, kBlkThreads, smem, st>>>(s.n, s.kl, s.ku, s.ldab, ab, ipiv, L, B, active);
    NEP_CHECK_LAUNCH();
    return NEP_OK;
}

int launch_band_solve_blocked(const SplitDev& s, int npts, const zf* ab, const int* ipiv, int L, zf* B,
                              const int* active, cudaStream_t st) {
    if (npts <= 0 || L <= 0) return NEP_OK;
    switch (band_solve_blocked_rhs(s.kl, s.ku, L)) {
        case 4: return launch_blocked<4>(s, npts, ab, ipiv, L, B, active, st);
        case 8: return launch_blocked<8>(s, npts, ab, ipiv, L, B, active, st);
        case 12: return launch_blocked<12>(s, npts, ab, ipiv, L, B, active, st);
        case 16: return launch_blocked<16>(s, npts, ab, ipiv, L, B, active, st);
        default: return NEP_ERR_UNSUPPORTED;
    }
}

}  // namespace nep

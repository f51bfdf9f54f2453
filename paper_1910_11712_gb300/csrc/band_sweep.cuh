// Banded forward/backward substitution sweeps for narrow bands (kernel (b), solve part).
// Instantiated once per element type (band_sweep_f.cu, band_sweep_d.cu) so the two compile in
// parallel.
#pragma once
#include <algorithm>
#include <cstdlib>
#include <type_traits>

#include "band_util.cuh"

namespace nep {

// One substitution sweep (forward with L and the row interchanges, or backward with U) for
// narrow bands; each warp carries RH right-hand sides. Step k handles row c = k (forward) or
// c = n-1-k (backward); the row with step index k' lives in window slot s = k' mod RS,
// RS = 32*RPL, held by lane s / RPL in register s % RPL. Consecutive steps therefore cycle
// through the registers in a fixed order, so with the step loop unrolled by RPL every
// register index is a compile-time constant. The row leaving the window at step k (row c
// itself) is replaced in the same register by the row with step index k + RS, which needs
// its first update only later (RS > window width).
//
// The coefficients of step k form one contiguous column col(k)[d], d in [1, W]:
//   forward  (W = kl):    col(k)[d] = ab[c*ldab + kv + d] = L(c+d, c)
//   backward (W = kl+ku): col(k)[d] = ut[c*(kv+1) + d]  = U(c-d, c), col(k)[0] = U(c,c)
// (ut: the U factor stored by columns, band_transpose_u). Per chunk of CH steps the CTA
// stages every step's column in slot order (zero outside the window), so each lane reads its
// RPL coefficients at fixed offsets, shares them across its RH right-hand sides and updates
// all its registers without predicates:  w(row of slot) -= col(k)[d] * x_c, with x_c the row's
// value after the interchange with row ipiv[c] (forward) or the row's value times 1/U(c,c)
// (backward). Interchanges are rare in practice, so a chunk without any runs a loop without
// the interchange test. A lane's RPL coefficients sit RPLP = RPL | 1 (odd) elements after the
// previous lane's, so the 8-byte loads of a warp step fall in distinct bank pairs (an even stride
// conflicts: RPL = 4 took 2.8x the shared-load wavefronts); steps are RSP = 32 RPLP + 1 apart.
// The second half of the CTA's warps are producers: they stage chunk c+1 into the other buffer
// while the compute warps (one or more right-hand sides each) run chunk c, so the staging's index
// work and copy issue stay off the compute warps' dependency chains. One CTA barrier per chunk:
// each producer arrives once its copies have landed, the compute warps once the chunk is done.
template <typename T, int RPL, bool BWD, int RH>
__global__ void __launch_bounds__(256)
    band_sweep_kernel(int n, int kl, int ku, int ldab, const cx<T>* __restrict__ ab_all,
                      const cx<T>* __restrict__ ut_all, const int* __restrict__ ipiv_all, int L,
                      cx<T>* __restrict__ B_all, const int* __restrict__ active, int CH,
                      const PointDesc* __restrict__ pd) {
    int j = blockIdx.x;
    if (pd) {  // a point of one of several problems sharing the launch (the grid covers the largest L)
        const PointDesc d = pd[blockIdx.x];
        n = d.n, kl = d.kl, ku = d.ku, ldab = d.ldab, L = d.L;
        ab_all = static_cast<const cx<T>*>(d.ab), ut_all = static_cast<const cx<T>*>(d.ut), ipiv_all = d.ipiv;
        B_all = static_cast<cx<T>*>(d.B), active = d.active;
        j = 0;
        if ((int)blockIdx.y * ((blockDim.x >> 5) / 2) * RH >= L) return;  // no right-hand side of this point here
    }
    if (active && !active[j]) return;
    constexpr int RS = 32 * RPL, RPLP = RPL | 1, RSP = 32 * RPLP + 1;
    const int kv = kl + ku;
    const int W = BWD ? kv : kl;  // window width: rows updated per step
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nwarps = (blockDim.x >> 5) / 2;  // compute warps; warps nwarps .. 2 nwarps-1 produce
    const bool producer = warp >= nwarps;
    const int pw = warp - nwarps;  // producer index
    const int col0 = (blockIdx.y * nwarps + warp) * RH;
    const int64_t cstride = BWD ? kv + 1 : ldab;
    const cx<T>* colbase = BWD ? ut_all + (int64_t)j * n * (kv + 1) : ab_all + (int64_t)j * n * ldab + kv;
    const int* ipiv = ipiv_all + (int64_t)j * n;
    bool has[RH];
    cx<T>* bh[RH];
#pragma unroll
    for (int h = 0; h < RH; ++h) {
        has[h] = !producer && col0 + h < L;
        bh[h] = B_all + ((int64_t)j * L + (has[h] ? col0 + h : 0)) * n;
    }
    const bool any = has[0];
    auto row_of = [&](int k) { return BWD ? n - 1 - k : k; };

    // layout: coef[2][CH*RSP] | dg[2][CH] (U(c,c)) | nb[2][nwarps][RH*CH] | ob[nwarps][RH*CH] | piv[2][CH]
    extern __shared__ unsigned char smem_raw[];
    cx<T>* coef0 = reinterpret_cast<cx<T>*>(smem_raw);
    cx<T>* dg0 = coef0 + 2 * (int64_t)CH * RSP;
    cx<T>* nb0 = dg0 + 2 * CH;
    cx<T>* ob0 = nb0 + 2 * (int64_t)nwarps * RH * CH;
    cx<T>* ob = ob0 + (int64_t)warp * RH * CH;
    int* piv0 = reinterpret_cast<int*>(ob0 + (int64_t)nwarps * RH * CH);

    // run by the producer warps, which split the steps and the entering rows
    auto issue = [&](int k0, int bsel) {
        const int cn = min(CH, n - k0);
        cx<T>* cf = coef0 + (int64_t)bsel * CH * RSP;
        // every slot of every step has exactly one writer: the window rows d in [1, W] copy their
        // coefficient (zero past the matrix), the other RS - W slots (d = 0 and d > W) zero
        for (int cc = pw; cc < cn; cc += nwarps) {
            const int k = k0 + cc, km = k % RS;
            cx<T>* dst = cf + cc * RSP;
            const cx<T>* src = colbase + (BWD ? n - 1 - k : k) * cstride;
            for (int d = 1 + lane; d <= RS; d += 32) {
                int sl = km + (d == RS ? 0 : d);
                if (sl >= RS) sl -= RS;
                const int at = (sl / RPL) * RPLP + sl % RPL;  // lane sl / RPL, register sl % RPL
                if (d <= W && k + d < n) cp_async_cx(dst + at, src + d);
                else dst[at] = mk<T>(0, 0);
            }
        }
        if (pw == 0 && lane < cn) {
            const int k = k0 + lane;
            if (!BWD) cp_async_i32(&piv0[bsel * CH + lane], ipiv + k);
            else cp_async_cx(&dg0[bsel * CH + lane], colbase + (n - 1 - k) * cstride);
        }
        // the rows entering the window of compute warp pw during the chunk
        for (int w = pw; w < nwarps; w += nwarps) {
            cx<T>* nb = nb0 + ((int64_t)bsel * nwarps + w) * RH * CH;
#pragma unroll
            for (int h = 0; h < RH; ++h) {
                const int col = (blockIdx.y * nwarps + w) * RH + h;
                const cx<T>* bw = B_all + ((int64_t)j * L + (col < L ? col : 0)) * n;
                for (int cc = lane; cc < cn; cc += 32) {
                    const int k = k0 + cc + RS;
                    if (col < L && k < n) cp_async_cx(&nb[h * CH + cc], bw + row_of(k));
                    else nb[h * CH + cc] = mk<T>(0, 0);
                }
            }
        }
        cp_async_commit();
    };

    cx<T> a[RH][RPL];
#pragma unroll
    for (int h = 0; h < RH; ++h)
#pragma unroll
        for (int q = 0; q < RPL; ++q) {
            const int k = lane * RPL + q;
            a[h][q] = (has[h] && k < n) ? bh[h][row_of(k)] : mk<T>(0, 0);
        }
    int lane_k = 0;  // lane holding the current step's row

    // one chunk of steps; SWAPS: some step of the chunk interchanges rows (forward only)
    auto run_chunk = [&](auto swaps_tag, int k0, int cn, const cx<T>* cf, const int* pv, cx<T> rdl,
                         const cx<T>* nb) {
        constexpr bool SWAPS = decltype(swaps_tag)::value;
        for (int g = 0; g < cn; g += RPL) {
#pragma unroll
            for (int u = 0; u < RPL; ++u) {
                const int cc = g + u;
                if (cc < cn) {
                    cx<T> x[RH];
#pragma unroll
                    for (int h = 0; h < RH; ++h) x[h] = shfl_cx(a[h][u], lane_k);
                    if constexpr (SWAPS) {
                        const int p = pv[cc] - (k0 + cc);
                        if (p != 0) {
                            // interchange rows c and c+p: slot of c+p is (lane_k*RPL + u + p) mod RS
                            int sp = lane_k * RPL + u + p;
                            if (sp >= RS) sp -= RS;
                            const int lp = sp / RPL, qp = sp - lp * RPL;
#pragma unroll
                            for (int h = 0; h < RH; ++h) {
                                const cx<T> vp = shfl_cx(sel_reg(a[h], qp), lp);
                                if (lane == lp) set_reg(a[h], qp, x[h]);
                                x[h] = vp;
                            }
                        }
                    }
                    if constexpr (BWD) {
                        const cx<T> rd = shfl_cx(rdl, cc);
#pragma unroll
                        for (int h = 0; h < RH; ++h) x[h] = x[h] * rd;
                    }
                    const cx<T>* c1 = cf + (int64_t)cc * RSP;
#pragma unroll
                    for (int q = 0; q < RPL; ++q) {
                        const cx<T> cq = c1[q];
#pragma unroll
                        for (int h = 0; h < RH; ++h) a[h][q] = fms(a[h][q], cq, x[h]);
                    }
                    if (lane == lane_k) {
#pragma unroll
                        for (int h = 0; h < RH; ++h) a[h][u] = nb[h * CH + cc];
                    }
                    if (lane == 0) {
#pragma unroll
                        for (int h = 0; h < RH; ++h) ob[h * CH + cc] = x[h];
                    }
                }
                if (u == RPL - 1) lane_k = lane_k == 31 ? 0 : lane_k + 1;
            }
        }
    };

    if (producer) issue(0, 0);
    for (int k0 = 0, chunk = 0; k0 < n; k0 += CH, ++chunk) {
        const int cn = min(CH, n - k0);
        const int bsel = chunk & 1;
        cp_async_wait_group<0>();  // the producer's copies of this chunk (a no-op elsewhere)
        __syncthreads();           // chunk staged; the other buffer's chunk finished
        if (producer) {
            if (k0 + CH < n) issue(k0 + CH, bsel ^ 1);
            continue;
        }
        if (any) {
            const cx<T>* cf = coef0 + (int64_t)bsel * CH * RSP + lane * RPLP;
            const int* pv = piv0 + bsel * CH;
            const cx<T>* nb = nb0 + ((int64_t)bsel * nwarps + warp) * RH * CH;
            cx<T> rdl = mk<T>(0, 0);
            bool swaps = false;
            if constexpr (BWD) {
                if (lane < cn) rdl = cdiv(mk<T>(1, 0), dg0[bsel * CH + lane]);
            } else {
                swaps = __any_sync(0xffffffffu, lane < cn && pv[lane] != k0 + lane);
            }
            if (swaps) run_chunk(std::true_type{}, k0, cn, cf, pv, rdl, nb);
            else run_chunk(std::false_type{}, k0, cn, cf, pv, rdl, nb);
            __syncwarp();
#pragma unroll
            for (int h = 0; h < RH; ++h)
                if (has[h])
                    for (int cc = lane; cc < cn; cc += 32) bh[h][row_of(k0 + cc)] = ob[h * CH + cc];
            __syncwarp();
        }
    }
}

// ut[j][c*(kv+1) + d] = U(c-d, c) for d in [0, kv] (zero where c-d < 0): the U factor of the
// band layout stored by columns, so the backward sweep stages each step's column contiguously.
// One thread per output element; the reads of a column are strided but the rows they touch
// are reused by the neighbouring columns from L1/L2, and the writes are coalesced.
template <typename T>
__global__ void band_transpose_u_kernel(int n, int kv, int ldab, const cx<T>* __restrict__ ab_all,
                                        cx<T>* __restrict__ ut_all) {
    const int j = blockIdx.y;
    const int64_t per = (int64_t)n * (kv + 1);
    const cx<T>* ab = ab_all + (int64_t)j * n * ldab;
    cx<T>* ut = ut_all + (int64_t)j * per;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < per; e += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(e / (kv + 1)), d = (int)(e - (int64_t)c * (kv + 1));
        ut[e] = c - d >= 0 ? ab[(int64_t)(c - d) * ldab + d] : mk<T>(0, 0);
    }
}

template <typename T, int RPL, bool BWD, int RH>
static int run_sweep(const SplitDev& s, int npts, const cx<T>* ab, const cx<T>* ut, const int* ipiv, int L,
                     cx<T>* B, const int* active, cudaStream_t st) {
    constexpr int RSP = 32 * (RPL | 1) + 1;
    const int warps = (L + RH - 1) / RH;
    // four compute warps per CTA (those beyond the right-hand sides idle), and as many producer
    // warps: with fewer right-hand sides the staging of a chunk fell on one producer warp and the
    // compute warp waited for it at every chunk barrier (single right-hand side: 1.7x slower)
    const int wpb = 4;
    const int gy = (warps + wpb - 1) / wpb;
    auto bytes = [&](int ch) {
        return sizeof(cx<T>) * (2 * (size_t)ch * RSP + 2 * (size_t)ch + 3 * (size_t)wpb * RH * ch) +
               sizeof(int) * 2 * ch;
    };
    int CH = 32 - 32 % RPL;
    while (CH > RPL && bytes(CH) > 200 * 1024) CH -= RPL;
    const size_t smem = bytes(CH);
    if (smem > 227 * 1024) return NEP_ERR_UNSUPPORTED;
    NEP_CUDA(allow_max_dynamic_smem(band_sweep_kernel<T, RPL, BWD, RH>));
    band_sweep_kernel<T, RPL, BWD, RH><<<dim3(npts, gy), 2 * wpb * 32, smem, st>>>(s.n, s.kl, s.ku, s.ldab, ab, ut,
                                                                             ipiv, L, B, active, CH, nullptr);
    NEP_CHECK_LAUNCH();
    return NEP_OK;
}

// The same sweep over points of several problems (descriptors pd_dev[count]; maxL the most
// right-hand sides of any of them): the launch shape of run_sweep, per-point arithmetic unchanged.
template <typename T, int RPL, bool BWD, int RH>
static int run_sweep_batch(int count, int maxL, const PointDesc* pd_dev, cudaStream_t st) {
    constexpr int RSP = 32 * (RPL | 1) + 1;
    const int warps = (maxL + RH - 1) / RH;
    const int wpb = 4;
    const int gy = (warps + wpb - 1) / wpb;
    auto bytes = [&](int ch) {
        return sizeof(cx<T>) * (2 * (size_t)ch * RSP + 2 * (size_t)ch + 3 * (size_t)wpb * RH * ch) +
               sizeof(int) * 2 * ch;
    };
    int CH = 32 - 32 % RPL;
    while (CH > RPL && bytes(CH) > 200 * 1024) CH -= RPL;
    const size_t smem = bytes(CH);
    if (smem > 227 * 1024) return NEP_ERR_UNSUPPORTED;
    NEP_CUDA(allow_max_dynamic_smem(band_sweep_kernel<T, RPL, BWD, RH>));
    band_sweep_kernel<T, RPL, BWD, RH><<<dim3(count, gy), 2 * wpb * 32, smem, st>>>(0, 0, 0, 0, nullptr, nullptr,
                                                                              nullptr, maxL, nullptr, nullptr, CH,
                                                                              pd_dev);
    NEP_CHECK_LAUNCH();
    return NEP_OK;
}

template <typename T, bool BWD, int RH>
static int sweep_batch_rpl(int rpl, int count, int maxL, const PointDesc* pd, cudaStream_t st) {
    switch (rpl) {
        case 1: return run_sweep_batch<T, 1, BWD, RH>(count, maxL, pd, st);
        case 2: return run_sweep_batch<T, 2, BWD, RH>(count, maxL, pd, st);
        case 3: return run_sweep_batch<T, 3, BWD, RH>(count, maxL, pd, st);
        case 4: return run_sweep_batch<T, 4, BWD, RH>(count, maxL, pd, st);
        case 5: return run_sweep_batch<T, 5, BWD, RH>(count, maxL, pd, st);
        case 6: return run_sweep_batch<T, 6, BWD, RH>(count, maxL, pd, st);
        case 7: return run_sweep_batch<T, 7, BWD, RH>(count, maxL, pd, st);
        case 8: return run_sweep_batch<T, 8, BWD, RH>(count, maxL, pd, st);
        case 9: return run_sweep_batch<T, 9, BWD, RH>(count, maxL, pd, st);
    }
    return NEP_ERR_UNSUPPORTED;
}

template <typename T, bool BWD>
static int sweep_batch_dispatch(int rpl, int rh, int count, int maxL, const PointDesc* pd, cudaStream_t st) {
    switch (rh) {
        case 1: return sweep_batch_rpl<T, BWD, 1>(rpl, count, maxL, pd, st);
        case 4: return sweep_batch_rpl<T, BWD, 4>(rpl, count, maxL, pd, st);
        default: return sweep_batch_rpl<T, BWD, 2>(rpl, count, maxL, pd, st);
    }
}

// Right-hand sides per warp of the substitution sweeps. One warp per right-hand side keeps the
// most chains in flight when there are few (N x L below 1.5 per SM sub-partition); with more,
// two or four per warp share the coefficient loads and the step bookkeeping. Measured with the
// producer warps: bandwidth 64 with 1024 chains (1.7 per sub-partition) takes 0.823 ms per
// solve with two against 0.849 with one, and eight concurrent passes run 7 % faster; four give
// another 1.6 % of throughput but 1.32 ms per solve. Bandwidth 128 with 4096 chains gains 2x from
// four over one, and 10 % over two (70 against 76 ms of solves per pass). NEP_SOLVE_RH = 1, 2 or 4 overrides the choice: a tuning knob only, the results are identical.
template <typename T>
static int sweep_rh(int chains) {
    static const int forced = [] {
        const char* e = std::getenv("NEP_SOLVE_RH");
        const int v = e ? std::atoi(e) : 0;
        return (v == 1 || v == 2 || v == 4) ? v : 0;
    }();
    if (forced) return forced;
    static const int smsp = [] {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        return 4 * (sms > 0 ? sms : 152);
    }();
    // about one or two warps per sub-partition; complex FP64 (FP64-throughput-bound) takes at least two
    const int rh = chains >= 6 * smsp ? 4 : 2 * chains >= 3 * smsp ? 2 : 1;
    return sizeof(T) == 4 ? rh : (rh < 2 ? 2 : rh);
}

template <typename T, bool BWD, int RH>
static int sweep_rpl(int rpl, const SplitDev& s, int npts, const cx<T>* ab, const cx<T>* ut, const int* ipiv, int L,
                     cx<T>* B, const int* active, cudaStream_t st) {
    switch (rpl) {
        case 1: return run_sweep<T, 1, BWD, RH>(s, npts, ab, ut, ipiv, L, B, active, st);
        case 2: return run_sweep<T, 2, BWD, RH>(s, npts, ab, ut, ipiv, L, B, active, st);
        case 3: return run_sweep<T, 3, BWD, RH>(s, npts, ab, ut, ipiv, L, B, active, st);
        case 4: return run_sweep<T, 4, BWD, RH>(s, npts, ab, ut, ipiv, L, B, active, st);
        case 5: return run_sweep<T, 5, BWD, RH>(s, npts, ab, ut, ipiv, L, B, active, st);
        case 6: return run_sweep<T, 6, BWD, RH>(s, npts, ab, ut, ipiv, L, B, active, st);
        case 7: return run_sweep<T, 7, BWD, RH>(s, npts, ab, ut, ipiv, L, B, active, st);
        case 8: return run_sweep<T, 8, BWD, RH>(s, npts, ab, ut, ipiv, L, B, active, st);
        case 9: return run_sweep<T, 9, BWD, RH>(s, npts, ab, ut, ipiv, L, B, active, st);
    }
    return NEP_ERR_UNSUPPORTED;
}

template <typename T, bool BWD>
static int sweep_dispatch(int rpl, const SplitDev& s, int npts, const cx<T>* ab, const cx<T>* ut, const int* ipiv,
                          int L, cx<T>* B, const int* active, cudaStream_t st, int rh_force) {
    switch (rh_force == 1 || rh_force == 2 || rh_force == 4 ? rh_force : sweep_rh<T>(npts * L)) {
        case 1: return sweep_rpl<T, BWD, 1>(rpl, s, npts, ab, ut, ipiv, L, B, active, st);
        case 4: return sweep_rpl<T, BWD, 4>(rpl, s, npts, ab, ut, ipiv, L, B, active, st);
        default: return sweep_rpl<T, BWD, 2>(rpl, s, npts, ab, ut, ipiv, L, B, active, st);
    }
}

// Registers per lane of a sweep's window for window width W: RS = 32 RPL > W. (A variant with
// RS = W, the entering row moved ahead of the step's update, executed fewer instructions on
// bandwidth 64 but ran no faster: 0.349 + 0.506 ms per solve against 0.345 + 0.476; each step is
// bound by its dependency chain rather than by issue.)
inline int sweep_rpl_of(int W) { return (W + 1 + 31) / 32; }

// Sweep launch shape of a problem: rows per lane of the forward and backward windows and right-hand
// sides per warp (from the problem's own chain count N L). Points of problems with equal keys share
// batched launches.
template <typename T>
void sweep_key(int kl, int ku, int npts, int L, int* rplf, int* rplb, int* rh, int rh_force) {
    *rplf = sweep_rpl_of(kl);
    *rplb = sweep_rpl_of(kl + ku);
    *rh = rh_force == 1 || rh_force == 2 || rh_force == 4 ? rh_force : sweep_rh<T>(npts * L);
}

template <typename T>
int band_sweeps_batch(int rplf, int rplb, int rh, int count, int maxL, const PointDesc* pd, cudaStream_t st) {
    if (count <= 0 || maxL <= 0) return NEP_OK;
    const int rc = sweep_batch_dispatch<T, false>(rplf, rh, count, maxL, pd, st);
    if (rc != NEP_OK) return rc;
    return sweep_batch_dispatch<T, true>(rplb, rh, count, maxL, pd, st);
}

template <typename T>
int band_sweeps(const SplitDev& s, int npts, const cx<T>* ab, const cx<T>* ut, const int* ipiv, int L, cx<T>* B,
                const int* active, cudaStream_t st, int rh_force) {
    if (npts <= 0 || L <= 0) return NEP_OK;
    if (!band_sweeps_fit(s.kl, s.ku) || !ut) return NEP_ERR_UNSUPPORTED;
    const int rplf = sweep_rpl_of(s.kl), rplb = sweep_rpl_of(s.kl + s.ku);
    const int rc = sweep_dispatch<T, false>(rplf, s, npts, ab, ut, ipiv, L, B, active, st, rh_force);
    if (rc != NEP_OK) return rc;
    return sweep_dispatch<T, true>(rplb, s, npts, ab, ut, ipiv, L, B, active, st, rh_force);
}

template <typename T>
int band_transpose_u(const SplitDev& s, int npts, const cx<T>* ab, cx<T>* ut, cudaStream_t st) {
    if (npts <= 0) return NEP_OK;
    const int64_t per = (int64_t)s.n * (s.kl + s.ku + 1);
    const int bx = (int)std::min<int64_t>((per + 255) / 256, 1024);
    band_transpose_u_kernel<T><<<dim3(bx, npts), 256, 0, st>>>(s.n, s.kl + s.ku, s.ldab, ab, ut);
    NEP_CHECK_LAUNCH();
    return NEP_OK;
}

}  // namespace nep

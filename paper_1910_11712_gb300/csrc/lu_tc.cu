// Kernel (b) for wide bands in complex64: the blocked banded LU of lu_wide.cu with its trailing
// update A22 -= L~21 U12 on the fifth-generation tensor core. One CTA per quadrature point.
//
// Elimination, pivot rule and stored factors are those of lu_wide.cu (the unblocked LU's order of
// operations per element); only the trailing product changes arithmetic: it runs as TF32 tensor-
// core products with FP32 accumulation, each FP32 operand split as hi + lo (hi = TF32 rounding,
// lo = TF32 rounding of the rest) and the three products hi*hi + hi*lo + lo*hi summed (~2^-22
// relative error per product, close to FP32; the refinement of the solves removes the rest).
//
// The complex product is one real product (the 4M form): with L~21 = Lr + i Li, U12 = Ur + i Ui,
//   row 2i   of A = [ Lr(i,:)  -Li(i,:) ],  row 2i+1 of A = [ Li(i,:)  Lr(i,:) ],
//   column j of B = [ Ur(:,j) ; Ui(:,j) ],
// so (A B)(2i, j) = Re (L~21 U12)(i, j) and (A B)(2i+1, j) = Im: K = 2 NB = 64, and the real and
// imaginary parts of one complex row sit in adjacent accumulator lanes.
//
// Per panel [p0, p0 + NB):
//   0-1. panel columns to shared memory and factored column by column (as lu_wide.cu);
//   2.   the panel's interchanges on the trailing columns, U12 by forward substitution (a warp per
//        column, lanes over its rows), written back into the window rows p0 .. p0+NB-1 and from
//        there to the output rows;
//   3.   A (from L~21) written to a per-point global operand image in the tensor core's
//        shared-memory layout, 64 complex rows (128 MMA rows) per tile, hi part then lo part;
//   4.   per tile of 128 trailing columns: B (from U12) written to shared memory by the threads;
//        per tile of 64 trailing rows: its A tile staged by a TMA tensor copy (double-buffered),
//        24 MMAs (M = 128, N = 128, K = 8) into one of two tensor-memory accumulators, and the
//        accumulator drained by all 16 warps (tcgen05.ld), which subtract it from the window.
// The shared memory of steps 0-3 (the panel) and of step 4 (B, two A buffers) is shared.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstdlib>
#include <mutex>

#include "band_util.cuh"
#include "tc_ptx.cuh"

namespace nep {

namespace {
constexpr int NB = 32;                          // panel width: complex columns per panel
constexpr int MT = 64;                          // complex rows per A tile (128 MMA rows)
constexpr int NT = 128;                         // complex columns per B tile (MMA N)
constexpr int KR = 2 * NB;                      // real K of the 4M product
constexpr int PART = 128 * KR;                  // floats in one TF32 part (hi or lo) of a tile
constexpr int TILE_BYTES = 2 * PART * 4;        // hi + lo: 64 KB
constexpr uint32_t LBO = 128 * 16;              // bytes between core matrices adjacent along K
constexpr uint32_t SBO = 128;                   // bytes between 8-row groups
constexpr uint32_t TMEM_COLS = 2 * NT;          // two FP32 accumulators of 128 x 128
constexpr long long WAIT_CYCLES = 4000000000ll; // bounded waits: about two seconds

// (row, k) of a tile -> float offset in one part: core matrices of 8 rows x 4 floats (128 B),
// 16 row groups at SBO, K chunks of 4 at LBO. Inverse: f -> (row, k).
__device__ __forceinline__ void tile_rk(int f, int& r, int& k) {
    const int k4 = f >> 9, rem = f & 511;
    r = (rem >> 5) * 8 + ((rem >> 2) & 7);
    k = k4 * 4 + (rem & 3);
}
}  // namespace

size_t lu_tc_smem(int kl) {
    const size_t rw = (size_t)kl + NB;
    const size_t early = 8 * rw * NB;
    const size_t late = 3 * (size_t)TILE_BYTES;
    return 1024 + (early > late ? early : late) + sizeof(int) * (rw + NB);
}

__global__ void __launch_bounds__(512, 1)
    lu_tc_kernel(int n, int kl, int ku, int ldab, zf* __restrict__ ab_all, int* __restrict__ ipiv_all,
                 int* __restrict__ info_all, const int* __restrict__ active, zf* __restrict__ win_all, int RWp,
                 int CWp, float* __restrict__ aimg_all, int nmt_max, const __grid_constant__ CUtensorMap tmap,
                 int* __restrict__ err, const PointDesc* __restrict__ pd, int passes) {
    const int j = blockIdx.x;  // also the point's operand image and its TMA coordinate
    zf* ab = ab_all + (int64_t)j * n * ldab;
    int* ipiv = ipiv_all + (int64_t)j * n;
    int* info_out = info_all + j;
    zf* W = win_all + (int64_t)j * RWp * CWp;
    if (pd) {  // a point of one of several problems sharing the launch
        const PointDesc d = pd[j];
        n = d.n, kl = d.kl, ku = d.ku, ldab = d.ldab, RWp = d.RWp, CWp = d.CWp;
        ab = static_cast<zf*>(d.ab), ipiv = d.ipiv, info_out = d.info, W = static_cast<zf*>(d.win);
        active = d.active;
        if (active && !active[0]) return;
    } else if (active && !active[j]) {
        return;
    }
    const int kv = kl + ku;
    const int RW = kl + NB;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nthr = blockDim.x, nwarp = nthr >> 5;
    float* aimg = aimg_all + (int64_t)j * nmt_max * (TILE_BYTES / 4);
    auto wi = [&](int r, int c) -> int64_t { return (int64_t)(r % RWp) + (int64_t)RWp * (c % CWp); };

    extern __shared__ unsigned char smem_raw[];
    unsigned char* R = smem_raw + ((1024 - (tc::smem_u32(smem_raw) & 1023)) & 1023);
    zf* Ps = reinterpret_cast<zf*>(R);        // RW x NB panel (steps 0-3)
    float* Bimg = reinterpret_cast<float*>(R);                           // step 4: B (hi, lo)
    float* Abuf0 = reinterpret_cast<float*>(R + TILE_BYTES);             // step 4: A tiles
    float* Abuf1 = reinterpret_cast<float*>(R + 2 * TILE_BYTES);
    const size_t early = 8 * (size_t)RW * NB;
    const size_t region = early > 3 * (size_t)TILE_BYTES ? early : 3 * (size_t)TILE_BYTES;
    int* src = reinterpret_cast<int*>(R + region);
    int* plist = src + RW;
    __shared__ int piv_sh[NB];
    __shared__ int info_s, npart_s, abort_s;
    __shared__ zf rpv_s;
    __shared__ uint32_t tmem_s;
    __shared__ __align__(8) uint64_t full_b[2], done_b[2], free_b[2];

    if (tid == 0) {
        info_s = 0;
        abort_s = 0;
        for (int b = 0; b < 2; ++b) {
            tc::mbar_init(&full_b[b], 1);
            tc::mbar_init(&done_b[b], 1);
            tc::mbar_init(&free_b[b], 16);  // one arrival per warp
        }
        tc::mbar_init_fence();
        tc::tma_prefetch_desc(&tmap);
    }
    if (warp == 0) {
        tc::tmem_alloc(&tmem_s, TMEM_COLS);
        tc::tmem_relinquish();
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = tmem_s;
    volatile int* abort_v = &abort_s;
    // bounded wait; a timeout (or an earlier one) sets the error and stops later waits
    auto wait = [&](uint64_t* bar, uint32_t parity) -> bool {
        if (*abort_v) return false;
        const long long t0 = clock64();
        while (!tc::mbar_try_wait(bar, parity)) {
            if (*abort_v) return false;
            if (clock64() - t0 > WAIT_CYCLES) {
                *abort_v = 1;
                atomicExch(err, 1);
                return false;
            }
        }
        return true;
    };
    // TMA loads issued into each A buffer and awaited by the MMA issuer (thread 0 only)
    int tma_issued[2] = {0, 0}, tma_seen[2] = {0, 0};
    long long g = 0;  // tiles processed so far: accumulator / A buffer g & 1, phase (g >> 1) & 1
    const uint32_t idesc = tc::idesc_tf32(128, NT);

    auto load_rows = [&](int r0, int r1) {
        for (int r = r0 + warp; r < r1; r += nwarp) {
            const zf* srow = ab + (int64_t)r * ldab - (r - kl);  // srow[c] = A(r, c)
            const int clo = max(r - kl, 0), chi = min(r + ku, n - 1);
            for (int c = clo + lane; c <= chi; c += 32) W[wi(r, c)] = srow[c];
        }
    };
    for (int64_t e = tid; e < (int64_t)RWp * CWp; e += nthr) W[e] = mk(0.0f, 0.0f);
    __syncthreads();
    load_rows(0, min(RW, n));
    __syncthreads();

    for (int p0 = 0; p0 < n; p0 += NB) {
        const int nbc = min(NB, n - p0);
        const int pr = min(RW, n - p0);

        // ---- 0. panel columns to shared memory (eight independent loads per lane, then the stores)
        for (int q = warp; q < nbc; q += nwarp) {
            const zf* wc = W + (int64_t)RWp * ((p0 + q) % CWp);
            for (int i0 = 0; i0 < RW; i0 += 256) {
                zf v[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int i = i0 + lane + 32 * u;
                    v[u] = i < pr ? wc[(p0 + i) % RWp] : mk(0.0f, 0.0f);
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int i = i0 + lane + 32 * u;
                    if (i < RW) Ps[i + (int64_t)RW * q] = v[u];
                }
            }
        }
        __syncthreads();

        // ---- 1. panel factorisation (pivot: first row maximising |Re|+|Im| among rows k .. k+kl)
        for (int k = 0; k < nbc; ++k) {
            const int c = p0 + k;
            const int last = min(k + kl, pr - 1), cnt = last - k + 1;
            zf* colk = Ps + (int64_t)RW * k;
            if (warp == 0) {
                float best = -1.0f;
                int bi = 0x7fffffff;
                for (int i = lane; i < cnt; i += 32) {
                    const float m = abs1(colk[k + i]);
                    if (m > best) { best = m; bi = i; }
                }
                const unsigned mb = best < 0 ? 0u : __float_as_uint(best);
                const unsigned mx = __reduce_max_sync(0xffffffffu, mb);
                int p = (int)__reduce_min_sync(0xffffffffu, mb == mx ? (unsigned)bi : 0xffffffffu);
                if (p >= cnt) p = 0;  // a column of NaNs matches no row: keep the diagonal
                const zf pv = colk[k + p];
                const bool zero = pv.re == 0.0f && pv.im == 0.0f;
                if (zero) p = 0;
                if (p != 0)
                    for (int q = lane; q < nbc; q += 32) {
                        zf* pq = Ps + (int64_t)RW * q;
                        const zf t = pq[k];
                        pq[k] = pq[k + p];
                        pq[k + p] = t;
                    }
                if (lane == 0) {
                    ipiv[c] = c + p;
                    piv_sh[k] = c + p;
                    if (zero && info_s == 0) info_s = c + 1;
                    rpv_s = zero ? mk(0.0f, 0.0f) : cdiv(mk(1.0f, 0.0f), pv);
                }
            }
            __syncthreads();
            {
                const zf rpv = rpv_s;
                zf* out = ab + (int64_t)c * ldab + kv + 1;
                for (int i = tid; i < kl; i += nthr) {
                    zf l = mk(0.0f, 0.0f);
                    if (k + 1 + i <= last) {
                        l = colk[k + 1 + i] * rpv;
                        colk[k + 1 + i] = l;
                    }
                    out[i] = l;
                }
            }
            __syncthreads();
            for (int q = k + 1 + warp; q < nbc; q += nwarp) {
                zf* pq = Ps + (int64_t)RW * q;
                const zf u = pq[k];
                for (int i = k + 1 + lane; i <= last; i += 32) pq[i] = fms(pq[i], colk[i], u);
            }
            __syncthreads();
        }

        // ---- the panel's interchanges as one permutation: local row l receives old row src[l]
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
        const int cend = min(p0 + nbc + kv, n), rend = min(p0 + nbc + kl, n);
        const int mr = rend - (p0 + nbc);

        // ---- 2. interchanges and U12 = L~11^{-1} A12, one warp per trailing column with lane k on
        // row p0 + k: u_i -= l_ik u_k for k ascending (the substitution's order of operations), the
        // result back into the window rows p0 .. p0+nbc-1 (they retire after this panel)
        // (four columns per warp at a time: four independent substitution chains)
        {
            const int srow = lane < nbc ? src[lane] : 0;
            const int prow = lane < npart ? src[plist[lane]] : 0;
            const int dst = lane < npart ? plist[lane] : 0;
            const zf* lrow = Ps + lane;
            for (int q0 = p0 + nbc + 4 * warp; q0 < cend; q0 += 4 * nwarp) {
                zf u[4], x[4];
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    const int q = q0 + m;
                    u[m] = q < cend && lane < nbc ? W[wi(p0 + srow, q)] : mk(0.0f, 0.0f);
                    x[m] = q < cend && lane < npart ? W[wi(p0 + prow, q)] : mk(0.0f, 0.0f);
                }
                __syncwarp();
#pragma unroll
                for (int m = 0; m < 4; ++m)
                    if (q0 + m < cend && lane < npart) W[wi(p0 + dst, q0 + m)] = x[m];
                for (int k = 0; k + 1 < nbc; ++k) {
                    const zf l = lrow[(int64_t)RW * k];
                    const bool act = lane > k && lane < nbc;
#pragma unroll
                    for (int m = 0; m < 4; ++m) {
                        const zf uk = shfl_cx(u[m], k);
                        if (act) u[m] = fms(u[m], l, uk);
                    }
                }
#pragma unroll
                for (int m = 0; m < 4; ++m)
                    if (q0 + m < cend && lane < nbc) W[wi(p0 + lane, q0 + m)] = u[m];
            }
        }
        __syncthreads();
        // U12 rows to the output band (warps over rows, lanes over columns)
        for (int k = warp; k < nbc; k += nwarp) {
            const int r = p0 + k;
            for (int q = p0 + nbc + lane; q < cend; q += 32)
                if (q - r <= kv) ab[(int64_t)r * ldab + (q - r)] = W[wi(r, q)];
        }

        // ---- the panel part of the finished rows: U(r, r .. p0+nbc-1), zeros beyond the band
        for (int k = warp; k < nbc; k += nwarp) {
            const int r = p0 + k;
            zf* out = ab + (int64_t)r * ldab;
            for (int q = k + lane; q < nbc; q += 32) out[q - k] = Ps[k + (int64_t)RW * q];
            for (int t = (cend - r) + lane; t <= kv; t += 32)
                if (t >= 0) out[t] = mk(0.0f, 0.0f);
        }

        // ---- 3. A operand image of L~21 (global, the tensor core's layout), tiles of 64 rows
        const int nmt = mr > 0 ? (mr + MT - 1) / MT : 0;
        const int ntn = (cend > p0 + nbc && mr > 0) ? (cend - (p0 + nbc) + NT - 1) / NT : 0;
        if (ntn > 0) {
            for (int e = tid; e < nmt * PART; e += nthr) {
                const int mt = e / PART, f = e - mt * PART;
                int r, k;
                tile_rk(f, r, k);
                const int i = mt * MT + (r >> 1), cc = k & (NB - 1);
                float v = 0.0f;
                if (i < mr && cc < nbc) {
                    const zf l = Ps[nbc + i + (int64_t)RW * cc];
                    const bool imrow = (r & 1) != 0, second = k >= NB;
                    v = imrow ? (second ? l.re : l.im) : (second ? -l.im : l.re);
                }
                float hi, lo;
                tc::split_tf32(v, hi, lo);
                float* t = aimg + (int64_t)mt * 2 * PART;
                t[f] = hi;
                t[PART + f] = lo;
            }
            tc::fence_async_global();
        }
        __syncthreads();

        // ---- 4. A22 -= L~21 U12 on the tensor core
        for (int nt = 0; nt < ntn; ++nt) {
            const int c0 = p0 + nbc + nt * NT;
            const int ncol = min(NT, cend - c0);
            if (tid == 0 && !*abort_v)
                for (int q = 0; q < min(2, nmt); ++q) {
                    const int b = (int)((g + q) & 1);
                    float* dst = b ? Abuf1 : Abuf0;
                    tc::mbar_arrive_expect_tx(&full_b[b], TILE_BYTES);
                    tc::tma_load_3d(dst, &tmap, &full_b[b], 0, q * 256, j);
                    ++tma_issued[b];
                }
            // the C rows of the first A tile towards L2 while B is built (lane q: column q of its group)
            if ((warp >> 2) * 32 + lane < ncol && 16 * (warp & 3) < mr)
                tc::prefetch_l2(W + (int64_t)((p0 + nbc + 16 * (warp & 3)) % RWp) +
                                (int64_t)RWp * ((c0 + (warp >> 2) * 32 + lane) % CWp));
            // B: row rn of the operand = complex column c0 + rn of U12, K = [Ur ; Ui]; lanes over the
            // 32 rows of U12 (contiguous in the window), eight independent loads, then the stores
            for (int e0 = 0; e0 < NB * NT; e0 += 8 * nthr) {
                zf u[8];
#pragma unroll
                for (int s = 0; s < 8; ++s) {
                    const int e = e0 + tid + s * nthr, kk = e & (NB - 1), rn = e >> 5;
                    u[s] = rn < ncol && kk < nbc ? W[wi(p0 + kk, c0 + rn)] : mk(0.0f, 0.0f);
                }
#pragma unroll
                for (int s = 0; s < 8; ++s) {
                    const int e = e0 + tid + s * nthr, kk = e & (NB - 1), rn = e >> 5;
                    const int fr = (kk >> 2) * 512 + (rn >> 3) * 32 + (rn & 7) * 4 + (kk & 3);  // k = kk
                    const int fi = fr + (NB >> 2) * 512;                                        // k = kk + NB
                    float hi, lo;
                    tc::split_tf32(u[s].re, hi, lo);
                    Bimg[fr] = hi;
                    Bimg[PART + fr] = lo;
                    tc::split_tf32(u[s].im, hi, lo);
                    Bimg[fi] = hi;
                    Bimg[PART + fi] = lo;
                }
            }
            tc::fence_async_shared();
            __syncthreads();

            // MMA issue for tile t of this column tile (thread 0)
            auto issue = [&](int t) {
                const long long gt = g + t;
                const int b = (int)(gt & 1);
                if (!wait(&full_b[b], (uint32_t)((gt >> 1) & 1))) return;
                ++tma_seen[b];
                if (gt >= 2 && !wait(&free_b[b], (uint32_t)(((gt >> 1) - 1) & 1))) return;
                tc::tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(b * NT);
                const uint32_t abase = tc::smem_u32(b ? Abuf1 : Abuf0), bbase = tc::smem_u32(Bimg);
                const int pa[3] = {0, 0, 1}, pb[3] = {0, 1, 0};  // hi*hi, hi*lo, lo*hi
                // passes = 3: hi*hi + hi*lo + lo*hi (~FP32); passes = 1: hi*hi alone (TF32 operands)
                for (int ps = 0; ps < passes; ++ps)
#pragma unroll
                    for (int s = 0; s < KR / 8; ++s) {
                        const uint64_t ad = tc::smem_desc(abase + (uint32_t)(pa[ps] * PART * 4) + s * 2 * LBO, LBO, SBO);
                        const uint64_t bd = tc::smem_desc(bbase + (uint32_t)(pb[ps] * PART * 4) + s * 2 * LBO, LBO, SBO);
                        tc::mma_tf32(d, ad, bd, idesc, (ps | s) != 0);
                    }
                tc::mma_commit(&done_b[b]);
            };
            for (int t = 0; t < nmt; ++t) {
                const long long gt = g + t;
                const int b = (int)(gt & 1);
                const uint32_t ph = (uint32_t)((gt >> 1) & 1);
                const int cb = (warp >> 2) * 32;  // this warp's 32 columns of the tile
                // the C rows of tile t + 1 towards L2: lane q takes column cb + q, one line (16 rows)
                if (t + 1 < nmt && cb + lane < ncol) {
                    const int i = (t + 1) * MT + 16 * (warp & 3);
                    if (i < mr)
                        tc::prefetch_l2(W + (int64_t)((p0 + nbc + i) % RWp) + (int64_t)RWp * ((c0 + cb + lane) % CWp));
                }
                if (tid == 0) {
                    if (t == 0) issue(0);
                    if (t + 1 < nmt) issue(t + 1);
                }
                __syncwarp();
                const bool ok = __all_sync(0xffffffffu, wait(&done_b[b], ph));
                // MMA t is done: its A buffer takes tile t + 2 (the copy runs during this epilogue)
                if (tid == 0 && ok && t + 2 < nmt) {
                    float* dst = b ? Abuf1 : Abuf0;
                    tc::mbar_arrive_expect_tx(&full_b[b], TILE_BYTES);
                    tc::tma_load_3d(dst, &tmap, &full_b[b], 0, (t + 2) * 256, j);
                    ++tma_issued[b];
                }
                __syncwarp();
                if (ok) {
                    tc::tc_fence_after();
                    float v[32];
                    const uint32_t taddr = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(b * NT + cb);
                    tc::tmem_ld_32x32b_x32(taddr, v);
                    tc::tc_fence_before();
                    __syncwarp();
                    if (lane == 0) tc::mbar_arrive(&free_b[b]);
                    // lanes 2m and 2m+1 hold the real and imaginary rows of complex row m: they trade
                    // halves, the even lane then updating columns 0..15 and the odd one 16..31 as
                    // complex (8-byte) read-modify-writes
                    const bool odd = (lane & 1) != 0;
                    float re[16], im[16];
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        const float send = odd ? v[q] : v[16 + q];
                        const float recv = __shfl_xor_sync(0xffffffffu, send, 1);
                        re[q] = odd ? recv : v[q];
                        im[q] = odd ? v[16 + q] : recv;
                    }
                    const int rr = (warp & 3) * 32 + lane;
                    const int i = t * MT + (rr >> 1);
                    if (i < mr) {
                        zf* wrow = W + (int64_t)((p0 + nbc + i) % RWp);
                        const int h = odd ? 16 : 0;
                        const int cs = (c0 + cb + h) % CWp;
                        zf cur[16];
#pragma unroll
                        for (int q = 0; q < 16; ++q) {
                            const int sl = cs + q < CWp ? cs + q : cs + q - CWp;
                            cur[q] = cb + h + q < ncol ? wrow[(int64_t)RWp * sl] : mk(0.0f, 0.0f);
                        }
#pragma unroll
                        for (int q = 0; q < 16; ++q) {
                            const int sl = cs + q < CWp ? cs + q : cs + q - CWp;
                            if (cb + h + q < ncol) wrow[(int64_t)RWp * sl] = mk(cur[q].re - re[q], cur[q].im - im[q]);
                        }
                    }
                }
            }
            g += nmt;
            __syncthreads();
        }
        if (*abort_v) break;

        // ---- 5. next window: rows [p0+RW, p0+RW+NB) and columns [p0+RW.., ) enter
        if (p0 + NB < n) {
            const int CW = kv + NB;
            const int rn0 = p0 + RW;
            for (int e = tid; e < NB * RWp; e += nthr) {
                const int jc = e / RWp, i = e - jc * RWp;
                W[(int64_t)i + (int64_t)RWp * ((p0 + CW + jc) % CWp)] = mk(0.0f, 0.0f);
            }
            __syncthreads();
            // column slot s holds the column c in [p0 + NB, p0 + NB + CWp) with c = s (mod CWp)
            const int r = rn0 + lane;
            const int per = (CWp + nwarp - 1) / nwarp;
            const int cbase = p0 + NB;
            for (int s0 = warp * per; s0 < min(CWp, (warp + 1) * per); s0 += 8) {
                zf v[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int s = s0 + u;
                    const int c = cbase + posmod(s - cbase, CWp);
                    v[u] = (s < min(CWp, (warp + 1) * per) && lane < NB && r < n && c >= r - kl && c <= r + ku && c < n)
                               ? ab[(int64_t)r * ldab + (c - r + kl)]
                               : mk(0.0f, 0.0f);
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int s = s0 + u;
                    if (s < min(CWp, (warp + 1) * per)) W[(int64_t)(r % RWp) + (int64_t)RWp * s] = v[u];
                }
            }
        }
        __syncthreads();
    }
    // wind down: copies and products in flight finish (bounded) before the memory is released
    if (tid == 0) {
        for (int b = 0; b < 2; ++b)
            for (int u = tma_seen[b]; u < tma_issued[b]; ++u) {
                const long long t0 = clock64();
                while (!tc::mbar_try_wait(&full_b[b], (uint32_t)(u & 1)) && clock64() - t0 < WAIT_CYCLES) {
                }
            }
        if (g > 0) {
            const long long last = g - 1;
            const long long t0 = clock64();
            while (!tc::mbar_try_wait(&done_b[last & 1], (uint32_t)((last >> 1) & 1)) && clock64() - t0 < WAIT_CYCLES) {
            }
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, TMEM_COLS);
    }
    if (tid == 0) *info_out = *abort_v ? n + 1 : info_s;
}

// ------------------------------------------------------------------ host side
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

bool lu_tc_enabled() {
    static const bool on = [] {
        const char* e = getenv("NEP_LU_TC");
        return !(e && e[0] == '0');
    }();
    return on;
}

bool band_lu_tc_can(int kl) { return kl >= NB && lu_tc_smem(kl) <= 227 * 1024; }

bool band_lu_tc_fits(int kl) { return kl > 64 && band_lu_tc_can(kl); }

int launch_band_lu_tc(const SplitDev& s, int npts, zf* ab, int* ipiv, int* info, const int* active, cudaStream_t st,
                      int passes) {
    if (npts <= 0) return NEP_OK;
    if (!band_lu_tc_can(s.kl)) return NEP_ERR_UNSUPPORTED;
    auto encode = encode_fn();
    if (!encode) {
        set_error("cuTensorMapEncodeTiled is not available from the driver");
        return NEP_ERR_CUDA;
    }
    const int kv = s.kl + s.ku;
    const int rwp = (s.kl + NB + NB - 1) / NB * NB, cwp = (kv + NB + NB - 1) / NB * NB;
    const size_t smem = lu_tc_smem(s.kl);
    const int nmt_max = (s.kl + MT - 1) / MT;
    zf* win = nullptr;
    float* aimg = nullptr;
    int* err = nullptr;
    NEP_CUDA(cudaMallocAsync((void**)&win, sizeof(zf) * (size_t)rwp * cwp * npts, st));
    cudaError_t e = cudaMallocAsync((void**)&aimg, (size_t)TILE_BYTES * nmt_max * npts, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&err, sizeof(int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), st);
    CUtensorMap tmap;
    if (e == cudaSuccess) {
        // the operand images as a 3-D array of floats: 64 per image row (256 B), 256 image rows per
        // tile, nmt_max tiles per point, npts points; one box = one tile (64 KB)
        const cuuint64_t dims[3] = {64, (cuuint64_t)nmt_max * 256, (cuuint64_t)npts};
        const cuuint64_t strides[2] = {256, (cuuint64_t)nmt_max * TILE_BYTES};
        const cuuint32_t box[3] = {64, 256, 1};
        const cuuint32_t estr[3] = {1, 1, 1};
        const CUresult r = encode(&tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, aimg, dims, strides, box, estr,
                                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) {
            cudaFreeAsync(win, st);
            cudaFreeAsync(aimg, st);
            cudaFreeAsync(err, st);
            set_error("cuTensorMapEncodeTiled failed (%d)", (int)r);
            return NEP_ERR_CUDA;
        }
    }
    if (e == cudaSuccess) e = allow_max_dynamic_smem(lu_tc_kernel);
    if (e == cudaSuccess) {
        lu_tc_kernel<<<npts, 512, smem, st>>>(s.n, s.kl, s.ku, s.ldab, ab, ipiv, info, active, win, rwp, cwp, aimg,
                                              nmt_max, tmap, err, nullptr, passes);
        count_launch();
        e = cudaGetLastError();
    }
    int herr = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (win) cudaFreeAsync(win, st);
    if (aimg) cudaFreeAsync(aimg, st);
    if (err) cudaFreeAsync(err, st);
    if (e != cudaSuccess) return cuda_fail(e, "lu_tc_kernel", __FILE__, __LINE__);
    if (herr) {
        set_error("lu_tc_kernel: a bounded wait on the tensor-core pipeline expired");
        return NEP_ERR_INTERNAL;
    }
    return NEP_OK;
}

// The tensor-core LU over points of several complex64 problems (each with kl > 64 and within the
// shared-memory budget): windows per point, one operand-image array and tensor map for the batch.
int launch_band_lu_tc_batch(const std::vector<PointDesc>& items_in, cudaStream_t st, int passes) {
    const int count = (int)items_in.size();
    if (count <= 0) return NEP_OK;
    auto encode = encode_fn();
    if (!encode) {
        set_error("cuTensorMapEncodeTiled is not available from the driver");
        return NEP_ERR_CUDA;
    }
    std::vector<PointDesc> items(items_in);
    size_t smem = 0, win_elems = 0;
    int nmt_max = 1;
    for (auto& d : items) {
        if (!band_lu_tc_can(d.kl)) return NEP_ERR_UNSUPPORTED;
        const int kv = d.kl + d.ku;
        d.RWp = (d.kl + NB + NB - 1) / NB * NB;
        d.CWp = (kv + NB + NB - 1) / NB * NB;
        win_elems += (size_t)d.RWp * d.CWp;
        smem = std::max(smem, lu_tc_smem(d.kl));
        nmt_max = std::max(nmt_max, (d.kl + MT - 1) / MT);
    }
    zf* win = nullptr;
    float* aimg = nullptr;
    int* err = nullptr;
    PointDesc* pd = nullptr;
    NEP_CUDA(cudaMallocAsync((void**)&win, sizeof(zf) * win_elems, st));
    cudaError_t e = cudaMallocAsync((void**)&aimg, (size_t)TILE_BYTES * nmt_max * count, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&err, sizeof(int), st);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&pd, sizeof(PointDesc) * count, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), st);
    size_t off = 0;
    for (auto& d : items) {
        d.win = win + off;
        off += (size_t)d.RWp * d.CWp;
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(pd, items.data(), sizeof(PointDesc) * count, cudaMemcpyHostToDevice, st);
    CUtensorMap tmap;
    if (e == cudaSuccess) {
        const cuuint64_t dims[3] = {64, (cuuint64_t)nmt_max * 256, (cuuint64_t)count};
        const cuuint64_t strides[2] = {256, (cuuint64_t)nmt_max * TILE_BYTES};
        const cuuint32_t box[3] = {64, 256, 1};
        const cuuint32_t estr[3] = {1, 1, 1};
        if (encode(&tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, aimg, dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            e = cudaErrorInvalidValue;
    }
    if (e == cudaSuccess) e = allow_max_dynamic_smem(lu_tc_kernel);
    if (e == cudaSuccess) {
        lu_tc_kernel<<<count, 512, smem, st>>>(0, 0, 0, 0, nullptr, nullptr, nullptr, nullptr, nullptr, 0, 0, aimg,
                                               nmt_max, tmap, err, pd, passes);
        count_launch();
        e = cudaGetLastError();
    }
    int herr = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (win) cudaFreeAsync(win, st);
    if (aimg) cudaFreeAsync(aimg, st);
    if (err) cudaFreeAsync(err, st);
    if (pd) cudaFreeAsync(pd, st);
    if (e != cudaSuccess) return cuda_fail(e, "lu_tc_kernel (batch)", __FILE__, __LINE__);
    if (herr) {
        set_error("lu_tc_kernel: a bounded wait on the tensor-core pipeline expired");
        return NEP_ERR_INTERNAL;
    }
    return NEP_OK;
}

}  // namespace nep

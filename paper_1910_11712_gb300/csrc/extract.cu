// Extraction of the eigenpairs from the contour moments (all on the device, FP64 unless noted):
//   * zgemm_kernel      dense complex products (column-major, op(A) in {A, A^H}), split-K
//                       with a fixed-order reduction so results never depend on scheduling;
//   * jacobi_kernel     one-sided (Hestenes) Jacobi SVD, cooperative across CTAs: round-robin
//                       pairings, one warp per column pair, a bounded grid barrier per round
//                       (FP64 throughput per SM is low on this part, so the pairs of a round
//                       are spread over many SMs);
//   * schur_eig_kernel  complex Hessenberg reduction + single-shift QR + triangular
//                       eigenvectors, one warp, used in FP32 for the reduced Hankel matrix
//                       (its eigenvalues only seed FP64 Newton, its eigenvectors only fix a
//                       basis of an already determined span);
//   * newton_kernel     Newton's method (Sec. 4.1 Eq. (newton)) on the projected split form
//                       sum_i f_i(lambda) B_i y = 0 (Sec. 4.2 Eq. (narnoldi-split)), bordered
//                       by the normalisation u^H y = 1, one CTA per candidate;
//   * residual/select   scaled residual eta (Sec. 2 Eq. (sressplit), infinity norms of the A_i
//                       as in Sec. 6), inside test, duplicate removal and ordering.
#include <cooperative_groups.h>
#include <cstdlib>

#include "nep_common.cuh"

namespace nep {

// ------------------------------------------------------------------ dense products
// C = op(A) B (column-major, op in {A, A^H}). A CTA computes a BM x BN tile with (BM/TM) x (BN/TN)
// threads of TM x TN outputs, K in steps of GK through shared memory; long K splits over CTAs
// into a workspace reduced in a fixed order, so results never depend on scheduling. FP64
// arithmetic is the bound on this part (about two FP64 FMAs per clock per SM), so the launcher
// picks the tile shape and the split that waste the least of it: padding beyond M and N (the
// reduced dimensions here are rarely multiples of 32) and SMs left idle or doubly loaded.
constexpr int GK = 8;
template <int BM, int BN, int TM, int TN>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
    zgemm_kernel(int M, int N, int K, int opA, const zd* __restrict__ A, int lda, const zd* __restrict__ B, int ldb,
                 zd* __restrict__ C, int ldc, int kchunk, int64_t part_stride) {
    constexpr int TX = BM / TM, TY = BN / TN, NT = TX * TY;
    __shared__ zd As[GK][BM + 1];
    __shared__ zd Bs[GK][BN + 1];
    const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
    const int kb = blockIdx.z * kchunk, ke = min(K, kb + kchunk);
    zd acc[TM][TN];
#pragma unroll
    for (int a = 0; a < TM; ++a)
#pragma unroll
        for (int b = 0; b < TN; ++b) acc[a][b] = mk(0.0, 0.0);
    for (int k0 = kb; k0 < ke; k0 += GK) {
        // loads run along the contiguous index of each operand
        for (int t = threadIdx.x; t < GK * BM; t += NT) {
            const int kk = opA == 0 ? t / BM : t % GK, mm = opA == 0 ? t % BM : t / GK;
            const int gm = m0 + mm, gk = k0 + kk;
            zd v = mk(0.0, 0.0);
            if (gm < M && gk < ke) v = opA == 0 ? A[gm + (int64_t)lda * gk] : conj(A[gk + (int64_t)lda * gm]);
            As[kk][mm] = v;
        }
        for (int t = threadIdx.x; t < GK * BN; t += NT) {
            const int kk = t % GK, nn = t / GK;
            const int gn = n0 + nn, gk = k0 + kk;
            Bs[kk][nn] = (gn < N && gk < ke) ? B[gk + (int64_t)ldb * gn] : mk(0.0, 0.0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GK; ++kk) {
            zd av[TM], bv[TN];
#pragma unroll
            for (int a = 0; a < TM; ++a) av[a] = As[kk][tx + TX * a];
#pragma unroll
            for (int b = 0; b < TN; ++b) bv[b] = Bs[kk][ty + TY * b];
#pragma unroll
            for (int a = 0; a < TM; ++a)
#pragma unroll
                for (int b = 0; b < TN; ++b) acc[a][b] = fma_(acc[a][b], av[a], bv[b]);
        }
        __syncthreads();
    }
    zd* Cz = C + (int64_t)blockIdx.z * part_stride;
#pragma unroll
    for (int a = 0; a < TM; ++a)
#pragma unroll
        for (int b = 0; b < TN; ++b) {
            const int gm = m0 + tx + TX * a, gn = n0 + ty + TY * b;
            if (gm < M && gn < N) Cz[gm + (int64_t)ldc * gn] = acc[a][b];
        }
}

__global__ void zgemm_reduce_kernel(int M, int N, int splits, const zd* __restrict__ part, zd* __restrict__ C, int ldc) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)M * N) return;
    const int m = (int)(t % M), n = (int)(t / M);
    zd acc = mk(0.0, 0.0);
    for (int z = 0; z < splits; ++z) acc = acc + part[(int64_t)z * M * N + t];
    C[m + (int64_t)ldc * n] = acc;
}

namespace {
struct GemmShape {
    int bm, bn;
};
constexpr GemmShape kGemmShapes[] = {{64, 32}, {64, 24}, {32, 32}, {32, 24}, {24, 24}, {32, 16}, {24, 16}};

template <int BM, int BN, int TM, int TN>
void zgemm_launch(dim3 grid, int M, int N, int K, int opA, const zd* A, int lda, const zd* B, int ldb, zd* C, int ldc,
                  int kchunk, int64_t part_stride, cudaStream_t st) {
    zgemm_kernel<BM, BN, TM, TN><<<grid, (BM / TM) * (BN / TN), 0, st>>>(M, N, K, opA, A, lda, B, ldb, C, ldc, kchunk,
                                                                       part_stride);
}
}  // namespace

// C = op(A) B. part: workspace of splits*M*N elements when K is long (nullptr => no split).
int zgemm(int M, int N, int K, int opA, const zd* A, int lda, const zd* B, int ldb, zd* C, int ldc, zd* part,
          size_t part_elems, cudaStream_t st) {
    if (M <= 0 || N <= 0) return NEP_OK;
    static const int sms = [] {
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        return v > 0 ? v : 152;
    }();
    // score = useful fraction of the padded tiles x SM load balance (mean over max CTAs per SM),
    // a split costing a little for its partial sums and their reduction
    int best = 0, best_splits = 1;
    double best_score = -1.0;
    for (int c = 0; c < (int)(sizeof(kGemmShapes) / sizeof(kGemmShapes[0])); ++c) {
        const int bm = kGemmShapes[c].bm, bn = kGemmShapes[c].bn;
        const int64_t tiles = (int64_t)ceil_div(M, bm) * ceil_div(N, bn);
        const double pad = (double)M * N / ((double)ceil_div(M, bm) * bm * ceil_div(N, bn) * bn);
        const int max_splits = part ? std::max(1, std::min<int>(K / 32, (int)std::min<size_t>(64, part_elems / ((size_t)M * N)))) : 1;
        for (int sp = 1; sp <= max_splits; ++sp) {
            const double ctas = (double)tiles * sp;
            const double waves = std::ceil(ctas / sms);
            const double score = pad * (ctas / sms) / waves * (sp > 1 ? 0.97 : 1.0);
            if (score > best_score + 1e-9) {
                best_score = score;
                best = c;
                best_splits = sp;
            }
        }
    }
    const int bm = kGemmShapes[best].bm, bn = kGemmShapes[best].bn;
    const int kchunk = ceil_div(ceil_div(K, best_splits), GK) * GK;
    const int splits = std::max(1, ceil_div(K, kchunk));
    dim3 grid(ceil_div(M, bm), ceil_div(N, bn), splits);
    zd* out = splits == 1 ? C : part;
    const int ldo = splits == 1 ? ldc : M;
    const int64_t ps = splits == 1 ? 0 : (int64_t)M * N;
    switch (best) {
        case 0: zgemm_launch<64, 32, 4, 2>(grid, M, N, K, opA, A, lda, B, ldb, out, ldo, kchunk, ps, st); break;
        case 1: zgemm_launch<64, 24, 4, 2>(grid, M, N, K, opA, A, lda, B, ldb, out, ldo, kchunk, ps, st); break;
        case 2: zgemm_launch<32, 32, 2, 2>(grid, M, N, K, opA, A, lda, B, ldb, out, ldo, kchunk, ps, st); break;
        case 3: zgemm_launch<32, 24, 2, 2>(grid, M, N, K, opA, A, lda, B, ldb, out, ldo, kchunk, ps, st); break;
        case 4: zgemm_launch<24, 24, 2, 2>(grid, M, N, K, opA, A, lda, B, ldb, out, ldo, kchunk, ps, st); break;
        case 5: zgemm_launch<32, 16, 2, 1>(grid, M, N, K, opA, A, lda, B, ldb, out, ldo, kchunk, ps, st); break;
        default: zgemm_launch<24, 16, 2, 1>(grid, M, N, K, opA, A, lda, B, ldb, out, ldo, kchunk, ps, st); break;
    }
    NEP_CHECK_LAUNCH();
    if (splits > 1) {
        zgemm_reduce_kernel<<<ceil_div((int64_t)M * N, 256), 256, 0, st>>>(M, N, splits, part, C, ldc);
        NEP_CHECK_LAUNCH();
    }
    return NEP_OK;
}

// ------------------------------------------------------------------ grid barrier
// Barrier for a cooperative launch (all CTAs co-resident) on a monotonically increasing
// arrival counter: barrier number e completes once the counter reaches e * gridDim.x, so it
// needs one atomic per CTA and no reset. Every wait is bounded: after `limit` polls (2^24 by
// default: seconds) the CTA records an error and continues, and once an error is recorded no
// barrier waits any more. The kernels using it have data-independent loop bounds, so a wait that
// gave up leaves wrong values but no out-of-range access; the host returns NEP_ERR_INTERNAL.
struct GridBar {
    unsigned int* count;
    unsigned int* gen;  // unused by this barrier, kept for the work layout
    int* err;
    long long limit;
};

__device__ __forceinline__ void grid_barrier(GridBar b, unsigned int& epoch) {
    __syncthreads();
    ++epoch;
    if (threadIdx.x == 0) {
        const unsigned int target = epoch * gridDim.x;
        __threadfence();
        atomicAdd(b.count, 1u);
        volatile unsigned int* vc = b.count;
        volatile int* ve = b.err;
        long long spins = 0;
        while (*vc < target) {
            if (*ve) break;  // another wait already timed out: do not add seconds per barrier
            if (++spins > b.limit) {
                atomicExch(b.err, 1);
                break;
            }
        }
        __threadfence();
    }
    __syncthreads();
}

// Loads of data that other CTAs of the same (cooperative) launch write: L2 only (ld.global.cg),
// never a possibly stale L1 line.
__device__ __forceinline__ zd ldcg(const zd* p) {
    const double2 v = __ldcg(reinterpret_cast<const double2*>(p));
    return mk(v.x, v.y);
}
__device__ __forceinline__ double ldcg(const double* p) { return __ldcg(p); }

// ------------------------------------------------------------------ one-sided Jacobi SVD
// A (rows x cols, column-major) is rotated in place until its columns are mutually
// orthogonal: A V = U Sigma. Rotation of columns (p, q) with alpha = |a_p|^2,
// beta = |a_q|^2, gamma = a_p^H a_q = |gamma| e^{i phi}: the angle with
// tan(theta) = t = sgn(zeta)/(|zeta| + sqrt(1 + zeta^2)), zeta = (beta - alpha)/(2|gamma|), zeroes
// the new a_p^H a_q; with c = cos(theta), s = sin(theta)
//   a_p <- c a_p - s e^{-i phi} a_q,   a_q <- s e^{i phi} a_p + c a_q   (same on V).
// Pairs per round follow the circle method over P = cols rounded up to even.

// c and s e^{i phi} = sr + i si of the rotation above, or false when the pair already counts as
// orthogonal (|gamma| <= tol sqrt(alpha beta)) or a column is zero. Multiplying t through by
// 2|gamma| gives, with D = beta - alpha and q = |D| + sqrt(D^2 + 4|gamma|^2),
//   c = q / sqrt(q^2 + 4|gamma|^2),   s e^{i phi} = 2 sgn(D) gamma / sqrt(q^2 + 4|gamma|^2):
// one square root and one reciprocal square root and no division (FP64 issue slots are the scarce
// resource here). c^2 + |s|^2 = 1 holds to the rounding of the reciprocal square root whatever the
// rounding of q, which only moves the angle. Outside the range where q^2 + 4|gamma|^2 is a normal
// number far from overflow, the zeta form (scaled by |gamma|) is used instead.
__device__ __forceinline__ bool jacobi_rotation(double al, double be, double gr, double gi, double tol, double& c,
                                                double& sr, double& si) {
    const double g2 = fma(gr, gr, gi * gi);
    if (!(g2 > (tol * tol) * (al * be)) || al == 0.0 || be == 0.0) return false;
    const double D = be - al, g4 = 4.0 * g2;
    const double q = fabs(D) + sqrt(fma(D, D, g4));
    const double h = fma(q, q, g4);
    if (h >= 1e-280 && h <= 1e280) {
        const double r = rsqrt(h);
        const double f = (D >= 0.0 ? 2.0 : -2.0) * r;
        c = q * r;
        sr = f * gr;
        si = f * gi;
        return true;
    }
    const double g = hypot(gr, gi);
    const double zeta = D / (2.0 * g);
    const double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
    c = 1.0 / sqrt(1.0 + t * t);
    const double sn = c * t / g;
    sr = sn * gr;
    si = sn * gi;
    return true;
}

// x <- c x - conj(s e) y,  y <- (s e) x + c y  with s e = sr + i si: twelve FP64 operations.
__device__ __forceinline__ void jacobi_apply(double c, double sr, double si, zd& x, zd& y) {
    const zd xo = mk(fma(c, x.re, -fma(sr, y.re, si * y.im)), fma(c, x.im, fma(-sr, y.im, si * y.re)));
    const zd yo = mk(fma(sr, x.re, fma(-si, x.im, c * y.re)), fma(sr, x.im, fma(si, x.re, c * y.im)));
    x = xo;
    y = yo;
}

// Sum of four per-lane values over the warp as a reduce-scatter: after the call lane l holds the
// warp total of value (l >> 3) & 3. Six FP64 additions where four butterflies take twenty.
__device__ __forceinline__ double warp_reduce_scatter4(double v0, double v1, double v2, double v3, int lane) {
    const bool h16 = (lane & 16) != 0, h8 = (lane & 8) != 0;
    double k0 = h16 ? v2 : v0, k1 = h16 ? v3 : v1;
    k0 += __shfl_xor_sync(0xffffffffu, h16 ? v0 : v2, 16);
    k1 += __shfl_xor_sync(0xffffffffu, h16 ? v1 : v3, 16);
    double k = h8 ? k1 : k0;
    k += __shfl_xor_sync(0xffffffffu, h8 ? k0 : k1, 8);
    for (int o = 4; o > 0; o >>= 1) k += __shfl_xor_sync(0xffffffffu, k, o);
    return k;
}

__global__ void __launch_bounds__(256) jacobi_kernel(int rows, int cols, zd* __restrict__ A, zd* __restrict__ Vm,
                                                     int max_sweeps, double tol, int* __restrict__ flags,
                                                     int* __restrict__ sweeps_out, GridBar bar) {
    const int lane = threadIdx.x & 31;
    // nsub warps per CTA (4 or 8): with several, the CTA works on one pair at a time (warps split
    // rows, one warp per SM sub-partition so the pair gets the whole SM's FP64 rate); with one,
    // each warp takes its own pair
    const int nsub = blockDim.x >> 5;
    const int gwarp = nsub > 1 ? (int)blockIdx.x : (int)(blockIdx.x * nsub + (threadIdx.x >> 5));
    const int nwarps = nsub > 1 ? (int)gridDim.x : (int)(gridDim.x * nsub);
    // per-warp partial sums, double-buffered: a warp writes buffer b of pair k + 2 only after the
    // barrier of pair k + 1, which every warp reaches after reading buffer b of pair k
    __shared__ double red4[2][8][4];
    int buf = 0;
    const int P = cols + (cols & 1);
    // V = I
    unsigned int epoch = 0;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < (int64_t)cols * cols;
         t += (int64_t)gridDim.x * blockDim.x)
        Vm[t] = mk((t % cols) == (t / cols) ? 1.0 : 0.0, 0.0);
    grid_barrier(bar, epoch);
    int sweep = 0;
    for (; sweep < max_sweeps; ++sweep) {
        if (blockIdx.x == 0 && threadIdx.x == 0) flags[(sweep + 1) & 1] = 0;
        for (int round = 0; round < P - 1; ++round) {
            for (int pi = gwarp; pi < P / 2; pi += nwarps) {
                int p, q;
                {
                    auto pos = [&](int k) { return k == 0 ? 0 : ((k - 1 + round) % (P - 1)) + 1; };
                    p = pos(pi);
                    q = pos(P - 1 - pi);
                }
                if (p >= cols || q >= cols) continue;
                if (p > q) { const int t = p; p = q; q = t; }
                zd* ap = A + (int64_t)p * rows;
                zd* aq = A + (int64_t)q * rows;
                zd* vp = Vm + (int64_t)p * cols;
                zd* vq = Vm + (int64_t)q * cols;
                if (rows <= 256 && cols <= 256 && nsub > 1) {
                    // the CTA's warps split the rows: one register element per lane per column
                    // (rows <= 32 * nsub * 2); partial dot products meet in shared memory
                    const int tid = threadIdx.x, nthr = blockDim.x;
                    const bool two = rows > nthr || cols > nthr;  // second element per thread needed
                    zd xa[2], ya[2], xv[2], yv[2];
#pragma unroll
                    for (int t = 0; t < 2; ++t) {
                        const int i = tid + nthr * t;
                        const bool ua = (t == 0 || two) && i < rows, uv = (t == 0 || two) && i < cols;
                        xa[t] = ua ? ldcg(ap + i) : mk(0.0, 0.0);
                        ya[t] = ua ? ldcg(aq + i) : mk(0.0, 0.0);
                        xv[t] = uv ? ldcg(vp + i) : mk(0.0, 0.0);
                        yv[t] = uv ? ldcg(vq + i) : mk(0.0, 0.0);
                    }
                    double al = norm2(xa[0]), be = norm2(ya[0]);
                    zd ga = fmac(mk(0.0, 0.0), xa[0], ya[0]);
                    if (two) {
                        al += norm2(xa[1]);
                        be += norm2(ya[1]);
                        ga = fmac(ga, xa[1], ya[1]);
                    }
                    const double ws = warp_reduce_scatter4(al, be, ga.re, ga.im, lane);
                    const int w = tid >> 5;
                    if ((lane & 7) == 0) red4[buf][w][lane >> 3] = ws;
                    __syncthreads();
                    // every warp adds the nsub partials itself, in the same order, so all warps
                    // hold bit-identical rotation scalars without another barrier: lane l takes
                    // value l & 3 of warp l >> 2
                    double x = (lane >> 2) < nsub ? red4[buf][lane >> 2][lane & 3] : 0.0;
                    buf ^= 1;
                    for (int o = 4; o < 4 * nsub; o <<= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
                    al = __shfl_sync(0xffffffffu, x, 0);
                    be = __shfl_sync(0xffffffffu, x, 1);
                    const double gr = __shfl_sync(0xffffffffu, x, 2), gi = __shfl_sync(0xffffffffu, x, 3);
                    double c, sr, si;
                    if (!jacobi_rotation(al, be, gr, gi, tol, c, sr, si)) continue;
#pragma unroll
                    for (int u = 0; u < 2; ++u) {
                        const int i = tid + nthr * u;
                        if (u == 1 && !two) break;
                        if (i < rows) {
                            jacobi_apply(c, sr, si, xa[u], ya[u]);
                            ap[i] = xa[u];
                            aq[i] = ya[u];
                        }
                        if (i < cols) {
                            jacobi_apply(c, sr, si, xv[u], yv[u]);
                            vp[i] = xv[u];
                            vq[i] = yv[u];
                        }
                    }
                    if (tid == 0) atomicOr(&flags[sweep & 1], 1);
                    continue;
                }
                double al = 0.0, be = 0.0;
                zd ga = mk(0.0, 0.0);
                for (int i = lane; i < rows; i += 32) {
                    const zd x = ldcg(ap + i), y = ldcg(aq + i);
                    al += norm2(x);
                    be += norm2(y);
                    ga = fmac(ga, x, y);
                }
                const double ws = warp_reduce_scatter4(al, be, ga.re, ga.im, lane);
                al = __shfl_sync(0xffffffffu, ws, 0);
                be = __shfl_sync(0xffffffffu, ws, 8);
                const double gr = __shfl_sync(0xffffffffu, ws, 16), gi = __shfl_sync(0xffffffffu, ws, 24);
                double c, sr, si;
                if (!jacobi_rotation(al, be, gr, gi, tol, c, sr, si)) continue;
                for (int i = lane; i < rows; i += 32) {
                    zd x = ldcg(ap + i), y = ldcg(aq + i);
                    jacobi_apply(c, sr, si, x, y);
                    ap[i] = x;
                    aq[i] = y;
                }
                for (int i = lane; i < cols; i += 32) {
                    zd x = ldcg(vp + i), y = ldcg(vq + i);
                    jacobi_apply(c, sr, si, x, y);
                    vp[i] = x;
                    vq[i] = y;
                }
                if (lane == 0) atomicOr(&flags[sweep & 1], 1);
            }
            grid_barrier(bar, epoch);
        }
        const int any = *((volatile int*)&flags[sweep & 1]);
        if (!any) break;
        grid_barrier(bar, epoch);  // everyone has read the flag before it is cleared again
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *sweeps_out = sweep + 1;
}

// sigma_i = |a_i|, descending order; U(:, r) = a_(i)/sigma, W(:, r) = V(:, i) for rank r of i.
__global__ void svd_finish_kernel(int rows, int cols, const zd* __restrict__ A, const zd* __restrict__ Vm,
                                  zd* __restrict__ U, zd* __restrict__ W, double* __restrict__ sigma) {
    extern __shared__ double nrm[];
    int* rk = reinterpret_cast<int*>(nrm + cols);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int i = w; i < cols; i += nw) {
        double s = 0.0;
        const zd* a = A + (int64_t)i * rows;
        for (int r = lane; r < rows; r += 32) s += norm2(a[r]);
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) nrm[i] = sqrt(s);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < cols; i += blockDim.x) {
        int rank = 0;
        for (int k = 0; k < cols; ++k) rank += (nrm[k] > nrm[i]) || (nrm[k] == nrm[i] && k < i);
        rk[i] = rank;
        sigma[rank] = nrm[i];
    }
    __syncthreads();
    if (U)
        for (int64_t e = threadIdx.x; e < (int64_t)rows * cols; e += blockDim.x) {
            const int i = (int)(e / rows), r = (int)(e - (int64_t)i * rows);
            const double inv = nrm[i] > 0 ? 1.0 / nrm[i] : 0.0;
            U[(int64_t)rk[i] * rows + r] = inv * A[e];
        }
    for (int64_t e = threadIdx.x; e < (int64_t)cols * cols; e += blockDim.x) {
        const int i = (int)(e / cols), r = (int)(e - (int64_t)i * cols);
        W[(int64_t)rk[i] * cols + r] = Vm[e];
    }
}

// The same Jacobi SVD on one thread-block cluster of CS CTAs (CS = 16 where the GPU allows it):
// CTA r keeps the columns j = r (mod CS) of A and of V in shared memory for the whole run, and each
// warp of the cluster takes one column pair per round (pair pi on warp pi mod (CS x warps per CTA)),
// reading and writing the pair's columns where they live through distributed shared memory. The
// pairs of a round are disjoint, so a round needs no barrier inside it; the cluster's hardware
// barrier between rounds replaces the grid barrier. The rotations, their order and the stopping
// rule are those of jacobi_kernel with one warp per pair (its lane order for the dot products).
// A sweep that rotated nothing ends the run: each CTA records a rotation in its own flag (one per
// sweep parity), every CTA reads all flags after the last round and so all take the same decision,
// and a cluster barrier follows the reads, so no CTA leaves while another still reads its flag.
namespace cgj = cooperative_groups;
// Sum of R values by pairwise halving (R a power of two): independent additions instead of one chain.
template <int R, typename V>
__device__ __forceinline__ V tree_sum(V (&v)[R]) {
#pragma unroll
    for (int h = R / 2; h > 0; h /= 2)
#pragma unroll
        for (int u = 0; u < h; ++u) v[u] = v[u] + v[u + h];
    return v[0];
}

// R: elements per lane of a column of A and of V (rows, cols <= 32 R); each warp holds its pair's
// four columns in registers for the round: one load and one store of every element.
template <int R>
__global__ void __launch_bounds__(256) jacobi_cluster_kernel(int rows, int cols, zd* __restrict__ A,
                                                             zd* __restrict__ Vm, int max_sweeps, double tol,
                                                             int* __restrict__ sweeps_out) {
    cgj::cluster_group cluster = cgj::this_cluster();
    const int CS = (int)cluster.num_blocks();
    const int rank = (int)cluster.block_rank();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const int ncl = (cols + CS - 1) / CS;  // column slots of this CTA: global j = c CS + rank
    extern __shared__ __align__(16) unsigned char sraw[];
    zd* acol = reinterpret_cast<zd*>(sraw);  // ncl x rows
    zd* vcol = acol + (size_t)ncl * rows;    // ncl x cols
    __shared__ int rotated[2];
    for (int c = 0; c < ncl; ++c) {
        const int j = c * CS + rank;
        for (int i = tid; i < rows; i += blockDim.x) acol[(size_t)c * rows + i] = j < cols ? A[(int64_t)j * rows + i] : mk(0.0, 0.0);
        for (int i = tid; i < cols; i += blockDim.x) vcol[(size_t)c * cols + i] = mk(i == j ? 1.0 : 0.0, 0.0);
    }
    if (tid == 0) rotated[0] = rotated[1] = 0;
    cluster.sync();
    auto acol_of = [&](int j) { return cluster.map_shared_rank(acol + (size_t)(j / CS) * rows, j % CS); };
    auto vcol_of = [&](int j) { return cluster.map_shared_rank(vcol + (size_t)(j / CS) * cols, j % CS); };
    const int P = cols + (cols & 1);
    const int gwarp = rank * nw + warp, nwarps = CS * nw;
    int sweep = 0;
    for (; sweep < max_sweeps; ++sweep) {
        const int par = sweep & 1;
        // this flag was last read before the barrier that closed sweep - 2; the rounds of sweep - 1
        // have passed cluster barriers since
        if (tid == 0) rotated[par] = 0;
        __syncthreads();
        for (int round = 0; round < P - 1; ++round) {
            for (int pi = gwarp; pi < P / 2; pi += nwarps) {
                auto pos = [&](int k) { return k == 0 ? 0 : ((k - 1 + round) % (P - 1)) + 1; };
                int p = pos(pi), q = pos(P - 1 - pi);
                if (p >= cols || q >= cols) continue;
                if (p > q) { const int t = p; p = q; q = t; }
                zd* ap = acol_of(p);
                zd* aq = acol_of(q);
                zd* vp = vcol_of(p);
                zd* vq = vcol_of(q);
                zd x[R], y[R], vx[R], vy[R];
#pragma unroll
                for (int u = 0; u < R; ++u) {
                    const int i = lane + 32 * u;
                    x[u] = i < rows ? ap[i] : mk(0.0, 0.0);
                    y[u] = i < rows ? aq[i] : mk(0.0, 0.0);
                }
#pragma unroll
                for (int u = 0; u < R; ++u) {  // in flight while the rotation is computed
                    const int i = lane + 32 * u;
                    vx[u] = i < cols ? vp[i] : mk(0.0, 0.0);
                    vy[u] = i < cols ? vq[i] : mk(0.0, 0.0);
                }
                double pa[R], pb[R];
                zd pg[R];
#pragma unroll
                for (int u = 0; u < R; ++u) {
                    pa[u] = norm2(x[u]);
                    pb[u] = norm2(y[u]);
                    pg[u] = fmac(mk(0.0, 0.0), x[u], y[u]);
                }
                double al = tree_sum<R>(pa), be = tree_sum<R>(pb);
                const zd ga = tree_sum<R>(pg);
                const double ws = warp_reduce_scatter4(al, be, ga.re, ga.im, lane);
                al = __shfl_sync(0xffffffffu, ws, 0);
                be = __shfl_sync(0xffffffffu, ws, 8);
                const double gr = __shfl_sync(0xffffffffu, ws, 16), gi = __shfl_sync(0xffffffffu, ws, 24);
                double c, sr, si;
                if (!jacobi_rotation(al, be, gr, gi, tol, c, sr, si)) continue;
#pragma unroll
                for (int u = 0; u < R; ++u) {
                    const int i = lane + 32 * u;
                    if (i < rows) {
                        jacobi_apply(c, sr, si, x[u], y[u]);
                        ap[i] = x[u];
                        aq[i] = y[u];
                    }
                    if (i < cols) {
                        jacobi_apply(c, sr, si, vx[u], vy[u]);
                        vp[i] = vx[u];
                        vq[i] = vy[u];
                    }
                }
                if (lane == 0) rotated[par] = 1;
            }
            cluster.sync();
        }
        int any = 0;
        for (int r = 0; r < CS; ++r) any |= *cluster.map_shared_rank(&rotated[par], r);
        cluster.sync();
        if (!any) break;
    }
    for (int c = 0; c < ncl; ++c) {
        const int j = c * CS + rank;
        if (j >= cols) break;
        for (int i = tid; i < rows; i += blockDim.x) A[(int64_t)j * rows + i] = acol[(size_t)c * rows + i];
        for (int i = tid; i < cols; i += blockDim.x) Vm[(int64_t)j * cols + i] = vcol[(size_t)c * cols + i];
    }
    if (rank == 0 && tid == 0) *sweeps_out = sweep + 1;
}

// Launches jacobi_cluster_kernel<R> (R the smallest of 1, 2, 4, 8 with rows, cols <= 32 R) on the
// largest cluster the GPU takes (16 or 8 CTAs) whose column slots fit in shared memory, when
// NEP_JACOBI_CLUSTER=1 asks for it (read at every call); false otherwise, or when no cluster fits or
// rows or cols exceed 256, and the caller runs jacobi_kernel. The cooperative grid kernel is the
// default: a round there has one SM per column pair, where the cluster gives a pair one SM
// sub-partition, and on this part's FP64 rate a pass alone is about 10 % faster with the grid
// kernel. The cluster kernel needs no co-resident grid and gives concurrent passes about 3 % more
// throughput.
template <int R>
static bool launch_jacobi_cluster_r(int rows, int cols, zd* A, zd* Vm, int max_sweeps, double tol, int* sweeps_out,
                                    cudaStream_t st) {
    // 16 if non-portable cluster sizes are accepted, else 8 (set once, thread-safe), and the dynamic
    // shared memory limit raised once to the opt-in maximum: a per-call limit races between host
    // threads launching different sizes
    static const int allowed = [] {
        const int a = cudaFuncSetAttribute(jacobi_cluster_kernel<R>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess
                          ? 16
                          : 8;
        cudaGetLastError();
        return a;
    }();
    if (allow_max_dynamic_smem(jacobi_cluster_kernel<R>) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    const int P = cols + (cols & 1);
    for (int CS = allowed; CS >= 8; CS /= 2) {
        const int ncl = (cols + CS - 1) / CS;
        const size_t smem = sizeof(zd) * (size_t)ncl * ((size_t)rows + cols);
        if (smem > 200 * 1024) continue;
        // one pair per warp and round where the pairs allow it, at most eight warps per CTA
        const int nw = std::max(1, std::min(8, (P / 2 + CS - 1) / CS));
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(CS);
        cfg.blockDim = dim3(32 * nw);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = CS;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int nclusters = 0;
        if (cudaOccupancyMaxActiveClusters(&nclusters, jacobi_cluster_kernel<R>, &cfg) != cudaSuccess || nclusters < 1) {
            cudaGetLastError();
            continue;
        }
        if (cudaLaunchKernelEx(&cfg, jacobi_cluster_kernel<R>, rows, cols, A, Vm, max_sweeps, tol, sweeps_out) !=
            cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        count_launch();
        return true;
    }
    return false;
}

static bool launch_jacobi_cluster(int rows, int cols, zd* A, zd* Vm, int max_sweeps, double tol, int* sweeps_out,
                                  cudaStream_t st) {
    const char* e = std::getenv("NEP_JACOBI_CLUSTER");
    if (!e || e[0] != '1') return false;
    const int need = (std::max(rows, cols) + 31) / 32;
    if (need <= 1) return launch_jacobi_cluster_r<1>(rows, cols, A, Vm, max_sweeps, tol, sweeps_out, st);
    if (need <= 2) return launch_jacobi_cluster_r<2>(rows, cols, A, Vm, max_sweeps, tol, sweeps_out, st);
    if (need <= 4) return launch_jacobi_cluster_r<4>(rows, cols, A, Vm, max_sweeps, tol, sweeps_out, st);
    if (need <= 8) return launch_jacobi_cluster_r<8>(rows, cols, A, Vm, max_sweeps, tol, sweeps_out, st);
    return false;
}

// A is destroyed; U (rows x cols) may be nullptr; W (cols x cols); sigma (cols).
int jacobi_svd(int rows, int cols, zd* A, zd* U, zd* W, double* sigma, JacobiWork w, cudaStream_t st) {
    if (cols <= 0) return NEP_OK;
    NEP_CUDA(cudaMemsetAsync(w.flags, 0, 2 * sizeof(int), st));
    NEP_CUDA(cudaMemsetAsync(w.bar, 0, 2 * sizeof(unsigned), st));
    const int P = cols + (cols & 1);
    int dev = 0, sms = 0;
    NEP_CUDA(cudaGetDevice(&dev));
    NEP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    // one column pair per CTA of four warps (one per SM sub-partition) for matrices up to 256
    // rows, so that each pair gets the whole SM's FP64 rate; one pair per warp beyond that
    const int tpb = (rows <= 256 && cols <= 256) ? 128 : 32;
    int per_sm = 0;
    NEP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, jacobi_kernel, tpb, 0));
    int blocks = std::max(1, std::min(P / 2, sms * std::max(per_sm, 1)));
    GridBar gb{w.bar, w.bar + 1, w.err, wait_limit()};
    int max_sweeps = 40;
    // columns count as orthogonal once |a_p^H a_q| <= rows * eps * |a_p| |a_q|: below that the
    // rotation angle is rounding noise
    double tol = std::max(rows, 1) * 2.220446049250313e-16;
    // the cooperative grid, or one cluster with distributed shared memory where asked for and it fits
    if (!launch_jacobi_cluster(rows, cols, A, w.Vm, max_sweeps, tol, w.sweeps, st)) {
        void* args[] = {&rows, &cols, &A, &w.Vm, &max_sweeps, &tol, &w.flags, &w.sweeps, &gb};
        NEP_CUDA(cudaLaunchCooperativeKernel((const void*)jacobi_kernel, dim3(blocks), dim3(tpb), args, 0, st));
        count_launch();
    }
    svd_finish_kernel<<<1, 256, (sizeof(double) + sizeof(int)) * cols, st>>>(rows, cols, A, w.Vm, U, W, sigma);
    NEP_CHECK_LAUNCH();
    return NEP_OK;
}

// ------------------------------------------------------------------ QR with column pivoting
// Householder QR with column pivoting, FP64, cooperative across CTAs (one warp per CTA, warp w
// owns columns j = w mod gridDim.x). Step k: every CTA finds the same pivot p (largest remaining
// squared column norm, first index on ties); the owner of column k swaps columns k and p and
// builds the reflector H_k = I - tau v v^H (v_0 = 1) with H_k^H [alpha; x] = [beta; 0]
// (barrier); every owner applies H_k^H to its columns j > k and recomputes their remaining
// norms (barrier). On exit A holds R in its upper triangle and v below it, perm the column
// order (A P = Q R, Q = H_0 H_1 ... H_{n-1}). Used to precondition one-sided Jacobi: on the
// graded block Hankel matrices of the contour method, Jacobi on R^H needs several times fewer
// sweeps than on A itself.
__global__ void __launch_bounds__(32) qrcp_kernel(int rows, int cols, zd* __restrict__ A, zd* __restrict__ tau,
                                                  int* __restrict__ perm, double* __restrict__ nrm2, double stop2,
                                                  int* __restrict__ steps_out, GridBar bar) {
    const int lane = threadIdx.x;
    const int G = gridDim.x;
    unsigned int epoch = 0;
    for (int j = blockIdx.x; j < cols; j += G) {
        const zd* a = A + (int64_t)j * rows;
        double s = 0.0;
        for (int i = lane; i < rows; i += 32) s += norm2(a[i]);
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) {
            nrm2[j] = s;
            perm[j] = j;
        }
    }
    grid_barrier(bar, epoch);
    const int steps = min(rows, cols);
    double first = 0.0;  // |R_00|^2
    int done = steps;
    for (int k = 0; k < steps; ++k) {
        // pivot: first index of the largest remaining norm among columns k..cols-1 (every CTA
        // finds the same one, so all agree on stopping)
        double best = -1.0, rest = 0.0;
        int bi = cols;
        for (int j = k + lane; j < cols; j += 32) {
            const double v = ldcg(nrm2 + j);
            rest += v;
            if (v > best) { best = v; bi = j; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
            rest += __shfl_xor_sync(0xffffffffu, rest, o);
        }
        if (bi >= cols) bi = k;  // NaN norms match no column
        if (k == 0) first = best;
        // ||R_22||_F^2 (the sum of the remaining squared column norms) <= stop2 |R_00|^2: dropping
        // the trailing block moves no singular value by more than sqrt(stop2) |R_00|
        if (rest <= stop2 * first) {
            done = k;
            break;
        }
        const int owner = k % G;
        if ((int)blockIdx.x == owner) {
            const int p = bi;
            zd* ak = A + (int64_t)k * rows;
            if (p != k) {
                zd* ap = A + (int64_t)p * rows;
                for (int i = lane; i < rows; i += 32) {
                    const zd t = ldcg(ak + i);
                    ak[i] = ldcg(ap + i);
                    ap[i] = t;
                }
                // nrm2 is not swapped: the other CTAs may still be searching it, and every
                // column j > k gets its remaining norm recomputed after the barrier anyway
                if (lane == 0) {
                    const int tp = __ldcg(perm + k);
                    perm[k] = __ldcg(perm + p);
                    perm[p] = tp;
                }
            }
            __syncwarp();
            // reflector of ak[k..rows-1]
            double xs = 0.0;
            for (int i = k + 1 + lane; i < rows; i += 32) xs += norm2(ldcg(ak + i));
            for (int o = 16; o > 0; o >>= 1) xs += __shfl_xor_sync(0xffffffffu, xs, o);
            const zd alpha = ldcg(ak + k);
            zd t = mk(0.0, 0.0);
            if (xs > 0.0 || alpha.im != 0.0) {
                const double an = hypot(alpha.re, alpha.im);
                const double bnorm = sqrt(an * an + xs);
                const double beta = alpha.re >= 0 ? -bnorm : bnorm;  // beta real, sign opposite Re(alpha)
                t = mk((beta - alpha.re) / beta, -alpha.im / beta);
                const zd scale = cdiv(mk(1.0, 0.0), alpha - mk(beta, 0.0));
                __syncwarp();
                for (int i = k + 1 + lane; i < rows; i += 32) ak[i] = ldcg(ak + i) * scale;
                __syncwarp();
                if (lane == 0) ak[k] = mk(beta, 0.0);
            }
            if (lane == 0) tau[k] = t;
            __threadfence();
        }
        grid_barrier(bar, epoch);
        // apply H_k^H = I - conj(tau) v v^H to the owned columns j > k
        const zd tk = ldcg(tau + k);
        const zd* v = A + (int64_t)k * rows;
        for (int j = blockIdx.x; j < cols; j += G) {
            if (j <= k) continue;
            zd* a = A + (int64_t)j * rows;
            zd s = lane == 0 ? ldcg(a + k) : mk(0.0, 0.0);
            for (int i = k + 1 + lane; i < rows; i += 32) s = fmac(s, ldcg(v + i), ldcg(a + i));
            for (int o = 16; o > 0; o >>= 1) {
                s.re += __shfl_xor_sync(0xffffffffu, s.re, o);
                s.im += __shfl_xor_sync(0xffffffffu, s.im, o);
            }
            const zd f = conj(tk) * s;
            double rest = 0.0;
            if (lane == 0) a[k] = ldcg(a + k) - f;
            for (int i = k + 1 + lane; i < rows; i += 32) {
                a[i] = fms(ldcg(a + i), ldcg(v + i), f);
                rest += norm2(a[i]);
            }
            for (int o = 16; o > 0; o >>= 1) rest += __shfl_xor_sync(0xffffffffu, rest, o);
            if (lane == 0) nrm2[j] = rest;
        }
        grid_barrier(bar, epoch);
    }
    if (blockIdx.x == 0) {
        for (int k = done + lane; k < steps; k += 32) tau[k] = mk(0.0, 0.0);  // H_k = I beyond the stop
        if (lane == 0) *steps_out = done;
    }
}

// The same QR with column pivoting on one thread-block cluster of CS CTAs (CS = 16 where the
// GPU allows it): CTA r keeps the columns j = r (mod CS) in shared memory, and the cluster's
// barriers (hardware, about a microsecond less than a grid barrier each) and distributed shared
// memory replace the grid barrier and the global column traffic. Per step k: every CTA publishes
// the largest remaining norm of its columns (first index on ties) and their sum, and all read the
// CTA results in the same order, so they agree on the pivot and on the stop; the owners of columns
// k and p exchange them through their swap buffers; the owner of column k builds the reflector;
// every CTA copies it and applies H_k^H to its columns j > k, one warp per column with the lane
// order of qrcp_kernel, and recomputes their remaining norms. On exit A, tau, perm and the step
// count are as qrcp_kernel leaves them.
constexpr int kQrcpClusterThreads = 128;
namespace cg = cooperative_groups;
__global__ void __launch_bounds__(kQrcpClusterThreads) qrcp_cluster_kernel(int rows, int cols, zd* __restrict__ A,
                                                                           zd* __restrict__ tau,
                                                                           int* __restrict__ perm, double stop2,
                                                                           int* __restrict__ steps_out) {
    cg::cluster_group cluster = cg::this_cluster();
    const int CS = (int)cluster.num_blocks();
    const int rank = (int)cluster.block_rank();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const int ncl = (cols + CS - 1) / CS;  // column slots of this CTA: global j = c CS + rank
    extern __shared__ __align__(16) unsigned char sraw[];
    zd* colm = reinterpret_cast<zd*>(sraw);      // ncl x rows
    zd* vloc = colm + (size_t)ncl * rows;        // rows: the current reflector
    zd* swp = vloc + rows;                       // rows: swap buffer
    double* lnorm = reinterpret_cast<double*>(swp + rows);  // ncl
    int* lperm = reinterpret_cast<int*>(lnorm + ncl);       // ncl
    __shared__ double slot_best, slot_rest, b_first;
    __shared__ int slot_idx, swp_perm, b_p, b_stop;
    __shared__ zd tau_s, tau_b;
    auto col = [&](int c) { return colm + (size_t)c * rows; };
    for (int c = 0; c < ncl; ++c) {
        const int j = c * CS + rank;
        for (int i = tid; i < rows; i += blockDim.x) col(c)[i] = j < cols ? A[(int64_t)j * rows + i] : mk(0.0, 0.0);
    }
    __syncthreads();
    for (int c = warp; c < ncl; c += nw) {
        const int j = c * CS + rank;
        double s = 0.0;
        for (int i = lane; i < rows; i += 32) s += norm2(col(c)[i]);
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) {
            lnorm[c] = j < cols ? s : -1.0;
            lperm[c] = j;
        }
    }
    const int steps = min(rows, cols);
    int done = steps;
    for (int k = 0; k < steps; ++k) {
        __syncthreads();
        if (warp == 0) {  // this CTA's best remaining column and the sum of its remaining norms
            double best = -1.0, rest = 0.0;
            int bi = cols;
            for (int c = lane; c < ncl; c += 32) {
                const int j = c * CS + rank;
                if (j >= k && j < cols) {
                    const double v = lnorm[c];
                    rest += v;
                    if (v > best) { best = v; bi = j; }
                }
            }
            for (int o = 16; o > 0; o >>= 1) {
                const double ob = __shfl_xor_sync(0xffffffffu, best, o);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
                rest += __shfl_xor_sync(0xffffffffu, rest, o);
            }
            if (lane == 0) {
                slot_best = best;
                slot_idx = bi;
                slot_rest = rest;
            }
        }
        cluster.sync();
        if (warp == 0) {  // the cluster's pivot and remaining mass, the same in every CTA
            double best = -1.0, rest = 0.0;
            int bi = cols;
            if (lane < CS) {
                best = *cluster.map_shared_rank(&slot_best, lane);
                bi = *cluster.map_shared_rank(&slot_idx, lane);
                rest = *cluster.map_shared_rank(&slot_rest, lane);
            }
            for (int o = 16; o > 0; o >>= 1) {
                const double ob = __shfl_xor_sync(0xffffffffu, best, o);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
                rest += __shfl_xor_sync(0xffffffffu, rest, o);
            }
            if (lane == 0) {
                if (bi >= cols) bi = k;  // NaN norms match no column
                if (k == 0) b_first = best;
                b_p = bi;
                b_stop = rest <= stop2 * b_first;
            }
        }
        cluster.sync();  // every CTA has read the slots before they are written again
        if (b_stop) {
            done = k;
            break;
        }
        const int p = b_p;
        const int ok = k % CS, op = p % CS, ck = k / CS, cp = p / CS;
        if (p != k) {
            if (ok == op) {
                if (rank == ok) {
                    for (int i = tid; i < rows; i += blockDim.x) {
                        const zd t = col(ck)[i];
                        col(ck)[i] = col(cp)[i];
                        col(cp)[i] = t;
                    }
                    if (tid == 0) {
                        const int t = lperm[ck];
                        lperm[ck] = lperm[cp];
                        lperm[cp] = t;
                    }
                }
            } else {
                if (rank == ok || rank == op) {
                    const int c = rank == ok ? ck : cp;
                    for (int i = tid; i < rows; i += blockDim.x) swp[i] = col(c)[i];
                    if (tid == 0) swp_perm = lperm[c];
                }
                cluster.sync();
                if (rank == ok || rank == op) {
                    const int c = rank == ok ? ck : cp, other = rank == ok ? op : ok;
                    const zd* rs = cluster.map_shared_rank(swp, other);
                    for (int i = tid; i < rows; i += blockDim.x) col(c)[i] = rs[i];
                    if (tid == 0) lperm[c] = *cluster.map_shared_rank(&swp_perm, other);
                }
            }
        }
        __syncthreads();
        if (rank == ok && warp == 0) {  // reflector of column k, rows k .. rows-1
            zd* ak = col(ck);
            double xs = 0.0;
            for (int i = k + 1 + lane; i < rows; i += 32) xs += norm2(ak[i]);
            for (int o = 16; o > 0; o >>= 1) xs += __shfl_xor_sync(0xffffffffu, xs, o);
            const zd alpha = ak[k];
            zd t = mk(0.0, 0.0);
            if (xs > 0.0 || alpha.im != 0.0) {
                const double an = hypot(alpha.re, alpha.im);
                const double bnorm = sqrt(an * an + xs);
                const double beta = alpha.re >= 0 ? -bnorm : bnorm;  // beta real, sign opposite Re(alpha)
                t = mk((beta - alpha.re) / beta, -alpha.im / beta);
                const zd scale = cdiv(mk(1.0, 0.0), alpha - mk(beta, 0.0));
                __syncwarp();
                for (int i = k + 1 + lane; i < rows; i += 32) ak[i] = ak[i] * scale;
                __syncwarp();
                if (lane == 0) ak[k] = mk(beta, 0.0);
            }
            if (lane == 0) {
                tau_s = t;
                tau[k] = t;
            }
        }
        cluster.sync();  // the reflector is published; the swap buffers have been read
        {
            const zd* rv = cluster.map_shared_rank(colm + (size_t)ck * rows, ok);
            for (int i = k + 1 + tid; i < rows; i += blockDim.x) vloc[i] = rv[i];
            if (tid == 0) tau_b = *cluster.map_shared_rank(&tau_s, ok);
        }
        __syncthreads();
        const zd tk = tau_b;
        for (int c = warp; c < ncl; c += nw) {  // apply H_k^H = I - conj(tau) v v^H to columns j > k
            const int j = c * CS + rank;
            if (j <= k || j >= cols) continue;
            zd* a = col(c);
            zd sm = lane == 0 ? a[k] : mk(0.0, 0.0);
            for (int i = k + 1 + lane; i < rows; i += 32) sm = fmac(sm, vloc[i], a[i]);
            for (int o = 16; o > 0; o >>= 1) {
                sm.re += __shfl_xor_sync(0xffffffffu, sm.re, o);
                sm.im += __shfl_xor_sync(0xffffffffu, sm.im, o);
            }
            const zd f = conj(tk) * sm;
            double rest = 0.0;
            __syncwarp();
            if (lane == 0) a[k] = a[k] - f;
            for (int i = k + 1 + lane; i < rows; i += 32) {
                a[i] = fms(a[i], vloc[i], f);
                rest += norm2(a[i]);
            }
            for (int o = 16; o > 0; o >>= 1) rest += __shfl_xor_sync(0xffffffffu, rest, o);
            if (lane == 0) lnorm[c] = rest;
        }
    }
    __syncthreads();
    for (int c = 0; c < ncl; ++c) {
        const int j = c * CS + rank;
        if (j >= cols) continue;
        for (int i = tid; i < rows; i += blockDim.x) A[(int64_t)j * rows + i] = col(c)[i];
        if (tid == 0) perm[j] = lperm[c];
    }
    if (rank == 0) {
        for (int k = done + tid; k < steps; k += blockDim.x) tau[k] = mk(0.0, 0.0);  // H_k = I beyond the stop
        if (tid == 0) *steps_out = done;
    }
    cluster.sync();  // no CTA leaves while another may still read its shared memory
}

// Launches qrcp_cluster_kernel on the largest cluster the GPU takes (16 or 8 CTAs) whose columns
// fit in shared memory; returns false (nothing launched) when none does.
static bool launch_qrcp_cluster(int rows, int cols, zd* A, zd* tau, int* perm, double stop2, int* steps_dev,
                                cudaStream_t st) {
    // 16 if non-portable cluster sizes are accepted, else 8 (set once, thread-safe), and the dynamic
    // shared memory limit raised once to the opt-in maximum: a per-call limit races between host
    // threads launching different sizes
    static const int allowed = [] {
        const int a = cudaFuncSetAttribute(qrcp_cluster_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess
                          ? 16
                          : 8;
        cudaGetLastError();
        return a;
    }();
    if (allow_max_dynamic_smem(qrcp_cluster_kernel) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    for (int CS = allowed; CS >= 8; CS /= 2) {
        const int ncl = (cols + CS - 1) / CS;
        if (ncl > 32) continue;
        const size_t smem = sizeof(zd) * ((size_t)ncl * rows + 2 * (size_t)rows) + (sizeof(double) + sizeof(int)) * ncl;
        if (smem > 200 * 1024) continue;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(CS);
        cfg.blockDim = dim3(kQrcpClusterThreads);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = CS;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int nclusters = 0;
        if (cudaOccupancyMaxActiveClusters(&nclusters, qrcp_cluster_kernel, &cfg) != cudaSuccess || nclusters < 1) {
            cudaGetLastError();
            continue;
        }
        if (cudaLaunchKernelEx(&cfg, qrcp_cluster_kernel, rows, cols, A, tau, perm, stop2, steps_dev) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        count_launch();
        return true;
    }
    return false;
}

// R^H of the upper triangle of A (n x n): Rh(i, j) = conj(A(j, i)) for i >= j, 0 above.
__global__ void rh_from_qr_kernel(int n, int ncols, const zd* __restrict__ A, zd* __restrict__ Rh) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)n * ncols) return;
    const int i = (int)(t % n), j = (int)(t / n);
    Rh[t] = i >= j ? conj(A[j + (int64_t)n * i]) : mk(0.0, 0.0);
}

// U(:, c) = [Wj(:, c); 0] for c < mq (Wj: mq x mq), zero columns c >= mq of U and W, sigma[c] = 0
// for c >= mq: the singular triplets of the dropped trailing block are reported as zero.
__global__ void qr_pad_kernel(int n, int mq, const zd* __restrict__ Wj, zd* __restrict__ U, zd* __restrict__ W,
                              double* __restrict__ sigma) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)n * n) return;
    const int i = (int)(t % n), c = (int)(t / n);
    if (c < mq) {
        U[t] = i < mq ? Wj[i + (int64_t)mq * c] : mk(0.0, 0.0);
    } else {
        U[t] = mk(0.0, 0.0);
        W[t] = mk(0.0, 0.0);
        if (i == 0) sigma[c] = 0.0;
    }
}

// X <- Q X with Q = H_0 H_1 ... H_{n-1} from qrcp_kernel (reflectors below the diagonal of A):
// one warp per column of X, reflectors applied from the last to the first.
__global__ void apply_q_kernel(int rows, int nref, const zd* __restrict__ A, const zd* __restrict__ tau,
                               int ncols, zd* __restrict__ X) {
    const int lane = threadIdx.x & 31;
    const int c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (c >= ncols) return;
    zd* x = X + (int64_t)c * rows;
    for (int k = nref - 1; k >= 0; --k) {
        const zd* v = A + (int64_t)k * rows;
        zd s = lane == 0 ? x[k] : mk(0.0, 0.0);
        for (int i = k + 1 + lane; i < rows; i += 32) s = fmac(s, v[i], x[i]);
        for (int o = 16; o > 0; o >>= 1) {
            s.re += __shfl_xor_sync(0xffffffffu, s.re, o);
            s.im += __shfl_xor_sync(0xffffffffu, s.im, o);
        }
        const zd f = tau[k] * s;
        __syncwarp();
        if (lane == 0) x[k] = x[k] - f;
        for (int i = k + 1 + lane; i < rows; i += 32) x[i] = fms(x[i], v[i], f);
        __syncwarp();
    }
}

// Q (rows x r) = the first r columns of the identity
__global__ void eye_cols_kernel(int rows, int r, zd* __restrict__ Q) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)rows * r) return;
    const int i = (int)(t % rows), c = (int)(t / rows);
    Q[t] = mk(i == c ? 1.0 : 0.0, 0.0);
}

// W(perm[i], c) = Uj(i, c)
__global__ void permute_rows_kernel(int n, int ncols, const int* __restrict__ perm, const zd* __restrict__ Uj,
                                    zd* __restrict__ W) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)n * ncols) return;
    const int i = (int)(t % n), c = (int)(t / n);
    W[perm[i] + (int64_t)n * c] = Uj[t];
}

// SVD of a square n x n matrix A (destroyed) preconditioned by QR with column pivoting:
// A P = Q R, one-sided Jacobi on R^H = Uj Sigma Wj^H, then A = (Q Wj) Sigma (P Uj)^H. The QR stops
// at the first step mq where the trailing block R_22 (rows and columns mq..n-1) has Frobenius
// norm <= trunc |R_00|: its rows of R are dropped, which moves every singular value by at most
// ||R_22||_2 <= trunc |R_00| <= trunc sigma_1 (Weyl), and Jacobi runs on the n x mq matrix
// R(0:mq, :)^H only. Singular values and vectors beyond mq are returned as zero.
int qrcp_jacobi_svd(int n, zd* A, zd* U, zd* W, double* sigma, zd* work1, zd* work2, zd* work3, zd* tau, int* perm,
                    double* nrm2, int* steps_dev, int* steps_host, double trunc, JacobiWork w, cudaStream_t st) {
    if (n <= 0) return NEP_OK;
    NEP_CUDA(cudaMemsetAsync(w.bar, 0, 2 * sizeof(unsigned), st));
    int dev = 0, sms = 0;
    NEP_CUDA(cudaGetDevice(&dev));
    NEP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    int per_sm = 0;
    NEP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, qrcp_kernel, 32, 0));
    int blocks = std::max(1, std::min(n, sms * std::max(per_sm, 1)));
    GridBar gb{w.bar, w.bar + 1, w.err, wait_limit()};
    int rows = n, cols = n;
    double stop2 = trunc * trunc;
    // one cluster with distributed shared memory where it fits, else the cooperative grid
    if (!launch_qrcp_cluster(rows, cols, A, tau, perm, stop2, steps_dev, st)) {
        void* args[] = {&rows, &cols, &A, &tau, &perm, &nrm2, &stop2, &steps_dev, &gb};
        NEP_CUDA(cudaLaunchCooperativeKernel((const void*)qrcp_kernel, dim3(blocks), dim3(32), args, 0, st));
        count_launch();
    }
    NEP_CUDA(cudaMemcpyAsync(steps_host, steps_dev, sizeof(int), cudaMemcpyDeviceToHost, st));
    NEP_CUDA(cudaStreamSynchronize(st));
    const int mq = std::max(0, std::min(n, *steps_host));
    if (mq > 0) {
        rh_from_qr_kernel<<<ceil_div((int64_t)n * mq, 256), 256, 0, st>>>(n, mq, A, work1);
        NEP_CHECK_LAUNCH();
        // Jacobi on R(0:mq, :)^H: work1 -> Uj (work2, n x mq), Wj (work3, mq x mq)
        NEP_TRY(jacobi_svd(n, mq, work1, work2, work3, sigma, w, st));
    }
    qr_pad_kernel<<<ceil_div((int64_t)n * n, 256), 256, 0, st>>>(n, mq, work3, U, W, sigma);
    NEP_CHECK_LAUNCH();
    if (mq > 0) {
        apply_q_kernel<<<ceil_div(mq, 4), 128, 0, st>>>(n, mq, A, tau, mq, U);
        NEP_CHECK_LAUNCH();
        permute_rows_kernel<<<ceil_div((int64_t)n * mq, 256), 256, 0, st>>>(n, mq, perm, work2, W);
        NEP_CHECK_LAUNCH();
    }
    return NEP_OK;
}

// An orthonormal basis of the range of A (rows x cols, column-major, overwritten): Householder QR
// with column pivoting (qrcp_kernel), stopped once the remaining columns' squared Frobenius mass is
// at most trunc^2 |R_00|^2; r = min(its steps, rmax) (at least 1) and Q (rows x r) = H_0 ... H_{r-1}
// applied to the first r columns of the identity. tau: min(rows, cols); perm, nrm2: cols.
int qr_range_basis(int rows, int cols, zd* A, zd* Q, int rmax, double trunc, zd* tau, int* perm, double* nrm2,
                   int* steps_dev, unsigned* bar, int* err, int* r_out, cudaStream_t st) {
    *r_out = 0;
    if (rows <= 0 || cols <= 0) return NEP_OK;
    NEP_CUDA(cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), st));
    NEP_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
    int dev = 0, sms = 0;
    NEP_CUDA(cudaGetDevice(&dev));
    NEP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    int per_sm = 0;
    NEP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, qrcp_kernel, 32, 0));
    int blocks = std::max(1, std::min(cols, sms * std::max(per_sm, 1)));
    GridBar gb{bar, bar + 1, err, wait_limit()};
    double stop2 = trunc * trunc;
    void* args[] = {&rows, &cols, &A, &tau, &perm, &nrm2, &stop2, &steps_dev, &gb};
    NEP_CUDA(cudaLaunchCooperativeKernel((const void*)qrcp_kernel, dim3(blocks), dim3(32), args, 0, st));
    count_launch();
    int steps = 0, e = 0;
    NEP_CUDA(cudaMemcpyAsync(&steps, steps_dev, sizeof(int), cudaMemcpyDeviceToHost, st));
    NEP_CUDA(cudaMemcpyAsync(&e, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    NEP_CUDA(cudaStreamSynchronize(st));
    if (e) {
        set_error("qr_range_basis: a bounded grid barrier timed out");
        return NEP_ERR_INTERNAL;
    }
    const int r = std::max(1, std::min(std::min(steps, rmax), std::min(rows, cols)));
    eye_cols_kernel<<<ceil_div((int64_t)rows * r, 256), 256, 0, st>>>(rows, r, Q);
    NEP_CHECK_LAUNCH();
    apply_q_kernel<<<ceil_div(r, 4), 128, 0, st>>>(rows, r, A, tau, r, Q);
    NEP_CHECK_LAUNCH();
    *r_out = r;
    return NEP_OK;
}

// ------------------------------------------------------------------ basis of a column block
// Pivoted Cholesky of the Gram matrix G = X^H X (m x m, Hermitian positive semidefinite), one
// CTA, FP64: at step k the column with the largest remaining squared norm d_p (the diagonal of
// the updated Gram matrix) is taken; the factorisation stops when d_p <= tol2 * max_i G_ii,
// i.e. when every remaining column lies within sqrt(tol2) (relative) of the span of the chosen
// ones. With P the pivoting and R the k' x k' factor, X P(:, 1:k') R^{-1} has orthonormal
// columns spanning the chosen columns; Z = P(:, 1:k') R^{-1} (m x k') is written so that the
// basis is the product X Z.
__global__ void __launch_bounds__(256) pchol_kernel(int m, const zd* __restrict__ G, double tol2, int* __restrict__ rank_out,
                                                    zd* __restrict__ Z, zd* __restrict__ gwork, int use_smem) {
    extern __shared__ unsigned char sraw[];
    zd* A = use_smem ? reinterpret_cast<zd*>(sraw) : gwork;  // m x m, column-major
    double* d = reinterpret_cast<double*>(A + (int64_t)m * m);
    int* perm = reinterpret_cast<int*>(d + m);
    __shared__ int piv_s, rank_s;
    __shared__ double dmax0;
    const int tid = threadIdx.x;
    for (int e = tid; e < m * m; e += blockDim.x) A[e] = G[e];
    for (int i = tid; i < m; i += blockDim.x) perm[i] = i;
    __syncthreads();
    for (int i = tid; i < m; i += blockDim.x) d[i] = A[i + (int64_t)m * i].re;
    __syncthreads();
    if (tid == 0) {
        double mx = 0;
        for (int i = 0; i < m; ++i) mx = fmax(mx, d[i]);
        dmax0 = mx;
        rank_s = m;
    }
    __syncthreads();
    for (int k = 0; k < m; ++k) {
        if (tid == 0) {
            int p = k;
            for (int i = k + 1; i < m; ++i)
                if (d[i] > d[p]) p = i;
            piv_s = (d[p] > tol2 * dmax0 && d[p] > 0) ? p : -1;
            if (piv_s < 0) rank_s = k;
        }
        __syncthreads();
        const int p = piv_s;
        if (p < 0) break;
        if (p != k) {
            // symmetric interchange of rows and columns k and p
            for (int i = tid; i < m; i += blockDim.x) {
                const zd t = A[i + (int64_t)m * k];
                A[i + (int64_t)m * k] = A[i + (int64_t)m * p];
                A[i + (int64_t)m * p] = t;
            }
            __syncthreads();
            for (int j = tid; j < m; j += blockDim.x) {
                const zd t = A[k + (int64_t)m * j];
                A[k + (int64_t)m * j] = A[p + (int64_t)m * j];
                A[p + (int64_t)m * j] = t;
            }
            if (tid == 0) {
                const double td = d[k];
                d[k] = d[p];
                d[p] = td;
                const int tp = perm[k];
                perm[k] = perm[p];
                perm[p] = tp;
            }
            __syncthreads();
        }
        const double rkk = sqrt(A[k + (int64_t)m * k].re);
        // row k of R (stored in place): R(k, j) = A(k, j) / R(k, k), j > k
        for (int j = k + 1 + tid; j < m; j += blockDim.x) A[k + (int64_t)m * j] = (1.0 / rkk) * A[k + (int64_t)m * j];
        __syncthreads();
        // R(k, k) replaces A(k, k) only now, after every thread has read A(k, k) above; the
        // trailing update below does not read it
        if (tid == 0) A[k + (int64_t)m * k] = mk(rkk, 0.0);
        // trailing update A(i, j) -= conj(R(k, i)) R(k, j), i, j > k
        const int nr = m - k - 1;
        for (int e = tid; e < nr * nr; e += blockDim.x) {
            const int i = k + 1 + e % nr, j = k + 1 + e / nr;
            A[i + (int64_t)m * j] = A[i + (int64_t)m * j] - conj(A[k + (int64_t)m * i]) * A[k + (int64_t)m * j];
        }
        __syncthreads();
        for (int i = k + 1 + tid; i < m; i += blockDim.x) d[i] = A[i + (int64_t)m * i].re;
        __syncthreads();
    }
    const int kr = rank_s;
    // Z = P(:, 1:kr) R^{-1}: column c of R^{-1} by back substitution (one thread per column)
    for (int e = tid; e < m * kr; e += blockDim.x) Z[e] = mk(0.0, 0.0);
    __syncthreads();
    for (int c = tid; c < kr; c += blockDim.x) {
        // solve R x = e_c (upper triangular); x_i = 0 for i > c
        for (int i = c; i >= 0; --i) {
            zd s = mk(i == c ? 1.0 : 0.0, 0.0);
            for (int t = i + 1; t <= c; ++t) s = fms(s, A[i + (int64_t)m * t], Z[perm[t] + (int64_t)m * c]);
            Z[perm[i] + (int64_t)m * c] = cdiv(s, A[i + (int64_t)m * i]);
        }
    }
    if (tid == 0) *rank_out = kr;
}

int launch_pchol(int m, const zd* G, double tol2, int* rank_out, zd* Z, zd* gwork, cudaStream_t st) {
    if (m <= 0) return NEP_OK;
    const size_t bytes = sizeof(zd) * (size_t)m * m + sizeof(double) * m + sizeof(int) * m + 64;
    const int use_smem = bytes <= 200 * 1024;
    if (use_smem)
        NEP_CUDA(allow_max_dynamic_smem(pchol_kernel));
    else if (!gwork)
        return NEP_ERR_INTERNAL;
    pchol_kernel<<<1, 256, use_smem ? bytes : 0, st>>>(m, G, tol2, rank_out, Z, gwork, use_smem);
    NEP_CHECK_LAUNCH();
    return NEP_OK;
}

// ------------------------------------------------------------------ small complex eigenproblem
// One warp. H (m x m, leading dimension ld) and Z live in shared or global memory. Steps:
// Householder reduction to Hessenberg form (Z accumulates the reflectors), single-shift QR
// sweeps with Wilkinson shifts and deflation on |h(k,k-1)| <= eps (|h(k,k)| + |h(k-1,k-1)|),
// then eigenvectors of the triangular Schur factor by back substitution, mapped by Z.
template <typename T>
__device__ void givens(cx<T> x, cx<T> y, T* c, cx<T>* s) {
    // [c s; -conj(s) c] [x; y] = [r; 0]
    const T ax = hypot(x.re, x.im), ay = hypot(y.re, y.im);
    if (ay == T(0)) { *c = T(1); *s = mk<T>(0, 0); return; }
    if (ax == T(0)) { *c = T(0); *s = conj(cdiv(y, mk<T>(ay, 0))); return; }
    const T nrm = hypot(ax, ay);
    *c = ax / nrm;
    const cx<T> ph = mk<T>(x.re / ax, x.im / ax);
    *s = (T(1) / nrm) * (ph * conj(y));
}

// The Schur form of the m x m matrix in H (one CTA of blockDim.x threads, a multiple of 32;
// leading dimension ld): H <- Z^H H Z upper triangular, Z accumulating the transformations (Z must
// hold I, or a unitary to be updated, on entry); v is m scratch elements, red blockDim.x / 32
// (unused with one warp). Returns 1 if the QR iteration hit its sweep limit. With several warps
// the rotations' row, column and Z updates spread over them (FP64 issues slowly on one warp).
template <typename T>
__device__ int schur_form(int m, cx<T>* H, cx<T>* Z, cx<T>* v, int ld, T* red) {
    const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, nw = nthr >> 5;
    const int tz = (tid + nthr / 2) % nthr;  // Z rows go to the other half of the threads
    const T eps = sizeof(T) == 4 ? T(6e-8) : T(1.2e-16);
    // the bulge's next x, y after step k, double-buffered by step parity (as in hqr_eigvals_kernel)
    __shared__ cx<T> xy[2][2];
    auto h = [&](int i, int j) -> cx<T>& { return H[i + (int64_t)ld * j]; };
    auto z = [&](int i, int j) -> cx<T>& { return Z[i + (int64_t)ld * j]; };
    auto sync = [&]() {
        if (nw > 1) __syncthreads();
        else __syncwarp();
    };
    auto bsum = [&](T x) -> T {
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (nw == 1) return x;
        if (lane == 0) red[tid >> 5] = x;
        __syncthreads();
        T t = 0;
        for (int w = 0; w < nw; ++w) t += red[w];
        __syncthreads();
        return t;
    };
    // Hessenberg reduction
    for (int k = 0; k + 2 < m; ++k) {
        T nx = 0;
        for (int i = k + 1 + tid; i < m; i += nthr) nx += norm2(h(i, k));
        nx = sqrt(bsum(nx));
        if (nx == T(0)) continue;
        const cx<T> x0 = h(k + 1, k);
        const T a0 = hypot(x0.re, x0.im);
        const cx<T> ph = a0 > 0 ? mk<T>(x0.re / a0, x0.im / a0) : mk<T>(1, 0);
        // v = x + ph*|x| e1, reflector I - 2 v v^H / (v^H v)
        for (int i = k + 1 + tid; i < m; i += nthr) v[i] = h(i, k);
        sync();
        if (tid == 0) v[k + 1] = v[k + 1] + nx * ph;
        sync();
        T vv = 0;
        for (int i = k + 1 + tid; i < m; i += nthr) vv += norm2(v[i]);
        const T sc = T(2) / bsum(vv);
        // left: rows k+1.., columns k..m-1 (threads over columns)
        for (int j = k + tid; j < m; j += nthr) {
            cx<T> s = mk<T>(0, 0);
            for (int i = k + 1; i < m; ++i) s = fmac(s, v[i], h(i, j));
            s = sc * s;
            for (int i = k + 1; i < m; ++i) h(i, j) = fms(h(i, j), v[i], s);
        }
        sync();
        // right: columns k+1.., all rows (threads over rows), and Z
        for (int i = tid; i < m; i += nthr) {
            cx<T> s = mk<T>(0, 0);
            for (int j = k + 1; j < m; ++j) s = fma_(s, h(i, j), v[j]);
            s = sc * s;
            for (int j = k + 1; j < m; ++j) h(i, j) = fms(h(i, j), s, conj(v[j]));
        }
        for (int i = tz; i < m; i += nthr) {
            cx<T> sz = mk<T>(0, 0);
            for (int j = k + 1; j < m; ++j) sz = fma_(sz, z(i, j), v[j]);
            sz = sc * sz;
            for (int j = k + 1; j < m; ++j) z(i, j) = fms(z(i, j), sz, conj(v[j]));
        }
        sync();
        for (int i = k + 2 + tid; i < m; i += nthr) h(i, k) = mk<T>(0, 0);
        sync();
    }
    // shifted QR
    int ihi = m - 1, iter = 0, since = 0, fail = 0;
    const int maxit = 60 * m + 100;
    while (ihi > 0) {
        if (iter++ > maxit) { fail = 1; break; }
        int l = ihi;
        while (l > 0) {
            const cx<T> sub = h(l, l - 1);
            const T ref = abs1(h(l, l)) + abs1(h(l - 1, l - 1));
            if (abs1(sub) <= eps * (ref > 0 ? ref : T(1))) break;
            --l;
        }
        sync();
        if (l > 0) {
            if (tid == 0) h(l, l - 1) = mk<T>(0, 0);
            sync();
        }
        if (l == ihi) {
            --ihi;
            since = 0;
            continue;
        }
        ++since;
        // Wilkinson shift from the trailing 2x2 of the active block
        const cx<T> a = h(ihi - 1, ihi - 1), b = h(ihi - 1, ihi), c2 = h(ihi, ihi - 1), d = h(ihi, ihi);
        cx<T> mu;
        if (since % 11 == 10) {
            mu = d + mk<T>(T(0.75) * abs1(c2), T(0));  // exceptional shift
        } else {
            const cx<T> tr = a + d, det = a * d - b * c2;
            const cx<T> disc = csqrt_(tr * tr - T(4) * det);
            const cx<T> r1 = T(0.5) * (tr + disc), r2 = T(0.5) * (tr - disc);
            mu = norm2(r1 - d) < norm2(r2 - d) ? r1 : r2;
        }
        cx<T> x = h(l, l) - mu, y = h(l + 1, l);
        sync();  // every thread has read the shift and x, y before the first rotation rewrites them
        for (int k = l; k < ihi; ++k) {
            T cs;
            cx<T> sn;
            givens(x, y, &cs, &sn);
            // rows k, k+1 from column max(l, k-1) to m-1
            for (int j = max(l, k - 1) + tid; j < m; j += nthr) {
                const cx<T> p = h(k, j), q = h(k + 1, j);
                h(k, j) = cs * p + sn * q;
                h(k + 1, j) = cs * q - conj(sn) * p;
            }
            sync();
            // columns k, k+1 for rows 0..min(k+2, ihi); Z all rows
            const int rlim = min(k + 2, ihi);
            for (int i = tid; i <= rlim; i += nthr) {
                const cx<T> p = h(i, k), q = h(i, k + 1);
                const cx<T> nk = cs * p + conj(sn) * q;
                h(i, k) = nk;
                h(i, k + 1) = cs * q - sn * p;
                if (i == k + 1 || i == k + 2) xy[k & 1][i - k - 1] = nk;
            }
            for (int i = tz; i < m; i += nthr) {
                const cx<T> p = z(i, k), q = z(i, k + 1);
                z(i, k) = cs * p + conj(sn) * q;
                z(i, k + 1) = cs * q - sn * p;
            }
            sync();
            if (k + 1 < ihi) {  // from the copy: the next row rotation rewrites h(k+1, k), h(k+2, k)
                x = xy[k & 1][0];
                y = xy[k & 1][1];
            }
        }
    }
    sync();
    return fail;
}

template <typename T>
__global__ void schur_eig_kernel(int m, const zd* __restrict__ Ain, zd* __restrict__ eval, zd* __restrict__ evec,
                                 int* __restrict__ status, cx<T>* gbuf, int use_smem) {
    extern __shared__ unsigned char sraw[];
    const int ld = m + 1;
    cx<T>* H = use_smem ? reinterpret_cast<cx<T>*>(sraw) : gbuf;
    cx<T>* Z = H + (int64_t)m * ld;
    cx<T>* v = Z + (int64_t)m * ld;  // m
    const int lane = threadIdx.x;
    const T eps = sizeof(T) == 4 ? T(6e-8) : T(1.2e-16);
    auto h = [&](int i, int j) -> cx<T>& { return H[i + (int64_t)ld * j]; };
    auto z = [&](int i, int j) -> cx<T>& { return Z[i + (int64_t)ld * j]; };
    for (int t = lane; t < m * m; t += 32) {
        const int i = t % m, j = t / m;
        h(i, j) = cvt<T>(Ain[i + (int64_t)m * j]);
        z(i, j) = mk<T>(i == j ? T(1) : T(0), T(0));
    }
    __syncwarp();
    const int fail = schur_form<T>(m, H, Z, v, ld, (T*)nullptr);
    __syncwarp();
    for (int i = lane; i < m; i += 32) eval[i] = cvt<double>(h(i, i));
    if (lane == 0 && status) *status = fail;
    if (!evec) return;
    // eigenvectors of the upper triangular Schur factor, then x = Z v
    T hn = 0;
    for (int t = lane; t < m * m; t += 32) {
        const int i = t % m, j = t / m;
        if (i <= j) hn = fmax(hn, abs1(h(i, j)));
    }
    for (int o = 16; o > 0; o >>= 1) hn = fmax(hn, __shfl_xor_sync(0xffffffffu, hn, o));
    const T small = eps * (hn > 0 ? hn : T(1));
    for (int e = 0; e < m; ++e) {
        const cx<T> lam = h(e, e);
        for (int i = lane; i < m; i += 32) v[i] = i < e ? -h(i, e) : (i == e ? mk<T>(1, 0) : mk<T>(0, 0));
        __syncwarp();
        for (int k = e - 1; k >= 0; --k) {
            cx<T> den = h(k, k) - lam;
            if (abs1(den) < small) den = mk<T>(small, 0);
            const cx<T> vk = cdiv(v[k], den);
            __syncwarp();
            if (lane == 0) v[k] = vk;
            for (int i = lane; i < k; i += 32) v[i] = fms(v[i], h(i, k), vk);
            __syncwarp();
        }
        for (int i = lane; i < m; i += 32) {
            cx<T> s = mk<T>(0, 0);
            for (int k = 0; k <= e; ++k) s = fma_(s, z(i, k), v[k]);
            evec[i + (int64_t)m * e] = cvt<double>(s);
        }
        __syncwarp();
    }
}

template <typename T>
int small_eig(int m, const zd* A, zd* eval, zd* evec, int* status, void* gbuf, cudaStream_t st) {
    if (m <= 0) return NEP_OK;
    const size_t bytes = sizeof(cx<T>) * ((size_t)2 * m * (m + 1) + m);
    const int use_smem = bytes <= 200 * 1024;
    if (use_smem)
        NEP_CUDA(allow_max_dynamic_smem(schur_eig_kernel<T>));
    else if (!gbuf)
        return NEP_ERR_INTERNAL;
    schur_eig_kernel<T><<<1, 32, use_smem ? bytes : 0, st>>>(m, A, eval, evec, status, (cx<T>*)gbuf, use_smem);
    NEP_CHECK_LAUNCH();
    return NEP_OK;
}
template int small_eig<float>(int, const zd*, zd*, zd*, int*, void*, cudaStream_t);
template int small_eig<double>(int, const zd*, zd*, zd*, int*, void*, cudaStream_t);

// ------------------------------------------------------------------ Krylov-Schur restart
// The FP64 Schur form H = Z T Z^H of an m x m matrix (one CTA of kKsSchurThreads): eval = diag(T),
// T (upper triangular) and Z written with leading dimension m. gbuf (2 m (m+1) + m complex128) is
// used when shared memory is too small.
constexpr int kKsSchurThreads = 128;
__global__ void __launch_bounds__(kKsSchurThreads) ks_schur_kernel(int m, const zd* __restrict__ A, zd* __restrict__ eval,
                                                                  zd* __restrict__ Tout, zd* __restrict__ Zout,
                                                                  int* __restrict__ status, zd* gbuf, int use_smem) {
    extern __shared__ unsigned char sraw[];
    __shared__ double red[kKsSchurThreads / 32];
    const int ld = m + 1, tid = threadIdx.x, nthr = blockDim.x;
    zd* H = use_smem ? reinterpret_cast<zd*>(sraw) : gbuf;
    zd* Z = H + (int64_t)m * ld;
    zd* v = Z + (int64_t)m * ld;
    for (int t = tid; t < m * m; t += nthr) {
        const int i = t % m, j = t / m;
        H[i + (int64_t)ld * j] = A[t];
        Z[i + (int64_t)ld * j] = mk(i == j ? 1.0 : 0.0, 0.0);
    }
    __syncthreads();
    const int fail = schur_form<double>(m, H, Z, v, ld, red);
    for (int t = tid; t < m * m; t += nthr) {
        const int i = t % m, j = t / m;
        Tout[t] = i <= j ? H[i + (int64_t)ld * j] : mk(0.0, 0.0);
        Zout[t] = Z[i + (int64_t)ld * j];
    }
    for (int i = tid; i < m; i += nthr) eval[i] = H[i + (int64_t)ld * i];
    if (tid == 0 && status) *status = fail;
}

// Reorders the Schur form (T, Z, leading dimension m) so that the diagonal entries that stood at
// positions sel[0 .. p) come first, in that order: each is moved up by swaps of adjacent diagonal
// entries, the swap at k by the rotation G with G [T(k,k+1); T(k+1,k+1) - T(k,k)] = [r; 0] (that
// vector is the eigenvector of the 2 x 2 block for T(k+1,k+1)): rows k, k+1 of T <- G (rows),
// columns k, k+1 of T and of Z <- (columns) G^H, then T(k+1,k) = 0 and the two diagonal entries
// exchanged exactly. One warp.
__global__ void ks_reorder_kernel(int m, int p, const int* __restrict__ sel, zd* __restrict__ T, zd* __restrict__ Z) {
    extern __shared__ int posbuf[];  // pos[m]: current position of original index q; at[m]: inverse
    int* pos = posbuf;
    int* at = posbuf + m;
    const int lane = threadIdx.x;
    for (int q = lane; q < m; q += 32) {
        pos[q] = q;
        at[q] = q;
    }
    __syncwarp();
    auto t = [&](int i, int j) -> zd& { return T[i + (int64_t)m * j]; };
    for (int dst = 0; dst < p; ++dst) {
        const int q = sel[dst];
        for (int j = pos[q]; j > dst; --j) {
            const int k = j - 1;
            const zd a = t(k, k), b = t(k + 1, k + 1);
            double cs;
            zd sn;
            givens(t(k, k + 1), b - a, &cs, &sn);
            __syncwarp();
            for (int c = k + lane; c < m; c += 32) {
                const zd x = t(k, c), y = t(k + 1, c);
                t(k, c) = cs * x + sn * y;
                t(k + 1, c) = cs * y - conj(sn) * x;
            }
            __syncwarp();
            for (int r = lane; r <= k + 1; r += 32) {
                const zd x = t(r, k), y = t(r, k + 1);
                t(r, k) = cs * x + conj(sn) * y;
                t(r, k + 1) = cs * y - sn * x;
            }
            for (int r = lane; r < m; r += 32) {
                const zd x = Z[r + (int64_t)m * k], y = Z[r + (int64_t)m * (k + 1)];
                Z[r + (int64_t)m * k] = cs * x + conj(sn) * y;
                Z[r + (int64_t)m * (k + 1)] = cs * y - sn * x;
            }
            __syncwarp();
            if (lane == 0) {
                t(k + 1, k) = mk(0.0, 0.0);
                t(k, k) = b;
                t(k + 1, k + 1) = a;
                const int qa = at[k], qb = at[k + 1];
                at[k] = qb;
                at[k + 1] = qa;
                pos[qb] = k;
                pos[qa] = k + 1;
            }
            __syncwarp();
        }
    }
}

int launch_ks_schur(int m, const zd* A, zd* eval, zd* T, zd* Z, int* status, zd* gbuf, cudaStream_t st) {
    if (m <= 0) return NEP_OK;
    const size_t bytes = sizeof(zd) * ((size_t)2 * m * (m + 1) + m);
    const int use_smem = bytes <= 200 * 1024;
    if (use_smem) NEP_CUDA(allow_max_dynamic_smem(ks_schur_kernel));
    else if (!gbuf) return NEP_ERR_INTERNAL;
    ks_schur_kernel<<<1, kKsSchurThreads, use_smem ? bytes : 0, st>>>(m, A, eval, T, Z, status, gbuf, use_smem);
    NEP_CHECK_LAUNCH();
    return NEP_OK;
}

int launch_ks_reorder(int m, int p, const int* sel, zd* T, zd* Z, cudaStream_t st) {
    if (m <= 0 || p <= 0) return NEP_OK;
    ks_reorder_kernel<<<1, 32, sizeof(int) * 2 * m, st>>>(m, p, sel, T, Z);
    NEP_CHECK_LAUNCH();
    return NEP_OK;
}

// The rotation of givens() from one reciprocal square root: c and s do not change when x and y are
// scaled by a common positive factor, so after scaling by 1 / max(|Re|, |Im|) (no overflow or
// underflow in the squares), with n^2 = |x|^2 + |y|^2,
//   c = |x| / n = |x|^2 r,   s = (x / |x|) conj(y) / n = x conj(y) r,   r = 1 / sqrt(|x|^2 n^2).
template <typename T>
__device__ __forceinline__ void givens_rsqrt(cx<T> x, cx<T> y, T* c, cx<T>* s) {
    const T mx = fmax(abs1(x), abs1(y));
    if (!(mx > T(0))) {
        *c = T(1);
        *s = mk<T>(0, 0);
        return;
    }
    T k;
    if constexpr (sizeof(T) == 4) k = __frcp_rn(mx);
    else k = __drcp_rn(mx);
    x = k * x;
    y = k * y;
    const T ax2 = norm2(x), ay2 = norm2(y);
    auto rs = [](T v) -> T {
        if constexpr (sizeof(T) == 4) return rsqrtf(v);
        else return rsqrt(v);
    };
    if (ay2 == T(0)) {
        *c = T(1);
        *s = mk<T>(0, 0);
        return;
    }
    if (ax2 == T(0)) {
        *c = T(0);
        *s = rs(ay2) * conj(y);
        return;
    }
    const T r = rs(ax2 * (ax2 + ay2));
    *c = ax2 * r;
    *s = r * (x * conj(y));
}

// ------------------------------------------------------------------ eigenvalues, then inverse iteration
// Faster variant for the reduced Hankel matrix: (1) one CTA (one warp below m = 64, four from
// there, the rotations' row and column updates spread over them) reduces to Hessenberg form and
// runs the shifted QR iteration updating only the active block (eigenvalues only, no Schur
// vectors); (2) one warp per eigenvalue solves (A - theta I) v = v twice by Gaussian
// elimination with partial pivoting (inverse iteration) for the eigenvector.
template <typename T>
__global__ void hqr_eigvals_kernel(int m, const zd* __restrict__ Ain, zd* __restrict__ eval, int* __restrict__ status,
                                   cx<T>* gbuf, int use_smem) {
    extern __shared__ unsigned char sraw[];
    __shared__ T red[32];
    // the bulge's next x, y (h(k+1, k), h(k+2, k) after step k), double-buffered by step parity: all
    // threads read them after the step's last barrier while step k+1's row rotation, which no
    // barrier separates from those reads, rewrites the entries in h
    __shared__ cx<T> xy[2][2];
    const int ld = m + 1;
    cx<T>* H = use_smem ? reinterpret_cast<cx<T>*>(sraw) : gbuf;
    cx<T>* v = H + (int64_t)m * ld;
    const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, nw = nthr >> 5;
    const T eps = sizeof(T) == 4 ? T(6e-8) : T(1.2e-16);
    auto h = [&](int i, int j) -> cx<T>& { return H[i + (int64_t)ld * j]; };
    auto sync = [&]() {
        if (nw > 1) __syncthreads();
        else __syncwarp();
    };
    auto bsum = [&](T x) -> T {
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (nw == 1) return x;
        if (lane == 0) red[tid >> 5] = x;
        __syncthreads();
        T t = 0;
        for (int w = 0; w < nw; ++w) t += red[w];
        __syncthreads();
        return t;
    };
    for (int t = tid; t < m * m; t += nthr) h(t % m, t / m) = cvt<T>(Ain[t]);
    sync();
    for (int k = 0; k + 2 < m; ++k) {
        T nx = 0;
        for (int i = k + 1 + tid; i < m; i += nthr) nx += norm2(h(i, k));
        nx = sqrt(bsum(nx));
        if (nx == T(0)) continue;
        const cx<T> x0 = h(k + 1, k);
        const T a0 = hypot(x0.re, x0.im);
        const cx<T> ph = a0 > 0 ? mk<T>(x0.re / a0, x0.im / a0) : mk<T>(1, 0);
        for (int i = k + 1 + tid; i < m; i += nthr) v[i] = h(i, k);
        sync();
        if (tid == 0) v[k + 1] = v[k + 1] + nx * ph;
        sync();
        T vv = 0;
        for (int i = k + 1 + tid; i < m; i += nthr) vv += norm2(v[i]);
        const T sc = T(2) / bsum(vv);
        for (int j = k + tid; j < m; j += nthr) {
            cx<T> sm = mk<T>(0, 0);
            for (int i = k + 1; i < m; ++i) sm = fmac(sm, v[i], h(i, j));
            sm = sc * sm;
            for (int i = k + 1; i < m; ++i) h(i, j) = fms(h(i, j), v[i], sm);
        }
        sync();
        for (int i = tid; i < m; i += nthr) {
            cx<T> sm = mk<T>(0, 0);
            for (int j = k + 1; j < m; ++j) sm = fma_(sm, h(i, j), v[j]);
            sm = sc * sm;
            for (int j = k + 1; j < m; ++j) h(i, j) = fms(h(i, j), sm, conj(v[j]));
        }
        sync();
        for (int i = k + 2 + tid; i < m; i += nthr) h(i, k) = mk<T>(0, 0);
        sync();
    }
    int ihi = m - 1, iter = 0, since = 0, fail = 0;
    const int maxit = 60 * m + 100;
    while (ihi > 0) {
        if (iter++ > maxit) { fail = 1; break; }
        // the largest l <= ihi with a negligible h(l, l-1) (0 if none), 32 subdiagonals per ballot;
        // every warp finds the same l
        int l = 0;
        for (int base = ihi; base > 0; base -= 32) {
            const int li = base - lane;
            bool small = false;
            if (li > 0) {
                const T ref = abs1(h(li, li)) + abs1(h(li - 1, li - 1));
                small = abs1(h(li, li - 1)) <= eps * (ref > 0 ? ref : T(1));
            }
            const unsigned bal = __ballot_sync(0xffffffffu, small);
            if (bal) {
                l = base - (__ffs(bal) - 1);
                break;
            }
        }
        sync();
        if (l > 0 && tid == 0) h(l, l - 1) = mk<T>(0, 0);
        sync();
        if (l == ihi) { --ihi; since = 0; continue; }
        ++since;
        const cx<T> a = h(ihi - 1, ihi - 1), b = h(ihi - 1, ihi), c2 = h(ihi, ihi - 1), d = h(ihi, ihi);
        cx<T> mu;
        if (since % 11 == 10) {
            mu = d + mk<T>(T(0.75) * abs1(c2), T(0));
        } else {
            const cx<T> tr = a + d, det = a * d - b * c2;
            const cx<T> disc = csqrt_(tr * tr - T(4) * det);
            const cx<T> r1 = T(0.5) * (tr + disc), r2 = T(0.5) * (tr - disc);
            mu = norm2(r1 - d) < norm2(r2 - d) ? r1 : r2;
        }
        cx<T> x = h(l, l) - mu, y = h(l + 1, l);
        sync();  // every thread has read the shift and x, y before the first rotation rewrites them
        for (int k = l; k < ihi; ++k) {
            T cs;
            cx<T> sn;
            givens_rsqrt(x, y, &cs, &sn);
            // active block only: rows k, k+1 over columns max(l, k-1)..ihi; columns k, k+1 over rows l..min(k+2, ihi)
            for (int j = max(l, k - 1) + tid; j <= ihi; j += nthr) {
                const cx<T> p = h(k, j), q = h(k + 1, j);
                h(k, j) = cs * p + sn * q;
                h(k + 1, j) = cs * q - conj(sn) * p;
            }
            sync();
            const int rlim = min(k + 2, ihi);
            for (int i = l + tid; i <= rlim; i += nthr) {
                const cx<T> p = h(i, k), q = h(i, k + 1);
                const cx<T> nk = cs * p + conj(sn) * q;
                h(i, k) = nk;
                h(i, k + 1) = cs * q - sn * p;
                if (i == k + 1 || i == k + 2) xy[k & 1][i - k - 1] = nk;
            }
            sync();
            if (k + 1 < ihi) {  // from the copy: the next row rotation rewrites h(k+1, k), h(k+2, k)
                x = xy[k & 1][0];
                y = xy[k & 1][1];
            }
        }
    }
    sync();
    for (int i = tid; i < m; i += nthr) eval[i] = cvt<double>(h(i, i));
    if (tid == 0 && status) *status = fail;
}

template <typename T>
__global__ void inverse_iteration_kernel(int m, const zd* __restrict__ Ain, const zd* __restrict__ eval,
                                         zd* __restrict__ evec, cx<T>* gbuf, int use_smem) {
    extern __shared__ unsigned char sraw[];
    const int e = blockIdx.x;
    const int ld = m + 1;
    cx<T>* A = use_smem ? reinterpret_cast<cx<T>*>(sraw) : gbuf + (int64_t)e * ((int64_t)m * ld + 2 * m);
    cx<T>* x = A + (int64_t)m * ld;
    int* piv = reinterpret_cast<int*>(x + m);
    const int lane = threadIdx.x;
    const T eps = sizeof(T) == 4 ? T(6e-8) : T(1.2e-16);
    const cx<T> th = cvt<T>(eval[e]);
    T anorm = 0;
    for (int t = lane; t < m * m; t += 32) {
        const int i = t % m, j = t / m;
        cx<T> a = cvt<T>(Ain[t]);
        if (i == j) a = a - th;
        A[i + (int64_t)ld * j] = a;
        anorm = fmax(anorm, abs1(a));
    }
    for (int o = 16; o > 0; o >>= 1) anorm = fmax(anorm, __shfl_xor_sync(0xffffffffu, anorm, o));
    const T tiny = eps * (anorm > 0 ? anorm : T(1));
    __syncwarp();
    // LU with partial pivoting (row interchanges recorded in piv)
    for (int k = 0; k < m; ++k) {
        T best = T(-1);
        int bi = k;
        for (int i = k + lane; i < m; i += 32) {
            const T a = abs1(A[i + (int64_t)ld * k]);
            if (a > best) { best = a; bi = i; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const T ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        if (lane == 0) piv[k] = bi;
        if (bi != k)
            for (int j = lane; j < m; j += 32) {
                const cx<T> t = A[k + (int64_t)ld * j];
                A[k + (int64_t)ld * j] = A[bi + (int64_t)ld * j];
                A[bi + (int64_t)ld * j] = t;
            }
        __syncwarp();
        cx<T> pv = A[k + (int64_t)ld * k];
        if (abs1(pv) < tiny) pv = mk<T>(tiny, 0);  // singular to working precision: perturb the pivot
        const cx<T> rp = cdiv(mk<T>(1, 0), pv);
        __syncwarp();
        if (lane == 0) A[k + (int64_t)ld * k] = pv;
        for (int i = k + 1 + lane; i < m; i += 32) A[i + (int64_t)ld * k] = A[i + (int64_t)ld * k] * rp;
        __syncwarp();
        for (int i = k + 1 + lane; i < m; i += 32) {
            const cx<T> l = A[i + (int64_t)ld * k];
            for (int j = k + 1; j < m; ++j) A[i + (int64_t)ld * j] = fms(A[i + (int64_t)ld * j], l, A[k + (int64_t)ld * j]);
        }
        __syncwarp();
    }
    for (int i = lane; i < m; i += 32) x[i] = mk<T>(T(1), T(0));
    __syncwarp();
    for (int it = 0; it < 2; ++it) {
        for (int k = 0; k < m; ++k) {
            const int p = piv[k];
            if (p != k && lane == 0) { const cx<T> t = x[k]; x[k] = x[p]; x[p] = t; }
            __syncwarp();
            const cx<T> xk = x[k];
            for (int i = k + 1 + lane; i < m; i += 32) x[i] = fms(x[i], A[i + (int64_t)ld * k], xk);
            __syncwarp();
        }
        for (int k = m - 1; k >= 0; --k) {
            const cx<T> xk = cdiv(x[k], A[k + (int64_t)ld * k]);
            __syncwarp();
            if (lane == 0) x[k] = xk;
            for (int i = lane; i < k; i += 32) x[i] = fms(x[i], A[i + (int64_t)ld * k], xk);
            __syncwarp();
        }
        T nrm = 0;
        for (int i = lane; i < m; i += 32) nrm += norm2(x[i]);
        for (int o = 16; o > 0; o >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
        const T inv = nrm > 0 ? T(1) / sqrt(nrm) : T(0);
        __syncwarp();
        for (int i = lane; i < m; i += 32) x[i] = inv * x[i];
        __syncwarp();
    }
    for (int i = lane; i < m; i += 32) evec[i + (int64_t)m * e] = cvt<double>(x[i]);
}

// Eigenvalues (and eigenvectors by inverse iteration) of a small complex matrix, precision T.
// gbuf: m * ((m+1)*m + 2m) elements of cx<T>, used when shared memory is too small.
template <typename T>
int small_eig_fast(int m, const zd* A, zd* eval, zd* evec, int* status, void* gbuf, cudaStream_t st) {
    if (m <= 0) return NEP_OK;
    const size_t b1 = sizeof(cx<T>) * ((size_t)m * (m + 1) + m);
    const int s1 = b1 <= 200 * 1024;
    if (s1) NEP_CUDA(allow_max_dynamic_smem(hqr_eigvals_kernel<T>));
    else if (!gbuf) return NEP_ERR_INTERNAL;
    // four warps once the matrix is large enough for the rotations' row and column updates to spread
    hqr_eigvals_kernel<T><<<1, m >= 64 ? 128 : 32, s1 ? b1 : 0, st>>>(m, A, eval, status, (cx<T>*)gbuf, s1);
    NEP_CHECK_LAUNCH();
    if (!evec) return NEP_OK;
    const size_t b2 = sizeof(cx<T>) * ((size_t)m * (m + 1) + m) + sizeof(int) * m + 16;
    const int s2 = b2 <= 200 * 1024;
    if (s2)
        NEP_CUDA(allow_max_dynamic_smem(inverse_iteration_kernel<T>));
    else if (!gbuf) return NEP_ERR_INTERNAL;
    inverse_iteration_kernel<T><<<m, 32, s2 ? b2 : 0, st>>>(m, A, eval, evec, (cx<T>*)gbuf, s2);
    NEP_CHECK_LAUNCH();
    return NEP_OK;
}
template int small_eig_fast<float>(int, const zd*, zd*, zd*, int*, void*, cudaStream_t);
template int small_eig_fast<double>(int, const zd*, zd*, zd*, int*, void*, cudaStream_t);

// ------------------------------------------------------------------ helpers
// Scale column c of X (rows x cols) by 1/|x_c|_2 (optionally fixing the phase so the first
// entry of largest modulus is real positive); nrm_out[c] = |x_c|_2 before scaling.
__global__ void __launch_bounds__(256) normalize_columns_kernel(int rows, zd* __restrict__ X, int fix_phase,
                                                                double* __restrict__ nrm_out) {
    __shared__ double red[32];
    __shared__ int redi[32];
    __shared__ double rmax[32];
    const int c = blockIdx.x;
    zd* x = X + (int64_t)c * rows;
    double s = 0.0, best = -1.0;
    int bi = 0x7fffffff;
    for (int i = threadIdx.x; i < rows; i += blockDim.x) {
        const double a = norm2(x[i]);
        s += a;
        if (a > best) { best = a; bi = i; }
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if (lane == 0) { red[w] = s; rmax[w] = best; redi[w] = bi; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ts = 0.0, tb = -1.0;
        int ti = 0x7fffffff;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
            ts += red[k];
            if (rmax[k] > tb || (rmax[k] == tb && redi[k] < ti)) { tb = rmax[k]; ti = redi[k]; }
        }
        red[0] = ts;
        redi[0] = ti < rows ? ti : 0;  // NaN entries match no index
    }
    __syncthreads();
    const double nrm = sqrt(red[0]);
    if (nrm_out && threadIdx.x == 0) nrm_out[c] = nrm;
    if (nrm == 0.0) return;
    zd f = mk(1.0 / nrm, 0.0);
    if (fix_phase) {
        const zd p = x[redi[0]];
        const double ap = hypot(p.re, p.im);
        f = mk(p.re / (ap * nrm), -p.im / (ap * nrm));
    }
    __syncthreads();
    for (int i = threadIdx.x; i < rows; i += blockDim.x) x[i] = x[i] * f;
}

// out_i = A_i Q for every term i (Q: n x k), out: nterms x n x k
__global__ void term_spmm_kernel(SplitDev s, int k, const zd* __restrict__ Q, zd* __restrict__ out) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nk = (int64_t)s.n * k;
    if (t >= nk * s.nterms) return;
    const int i = (int)(t / nk);
    const int64_t rc = t % nk;
    const int r = (int)(rc % s.n), c = (int)(rc / s.n);
    zd acc = mk(0.0, 0.0);
    for (int64_t e = s.rowptr[r]; e < s.rowptr[r + 1]; ++e) {
        const zd a = mk(s.val[(int64_t)i * s.nnz + e], s.val_im ? s.val_im[(int64_t)i * s.nnz + e] : 0.0);
        acc = fma_(acc, a, Q[(int64_t)c * s.n + s.col[e]]);
    }
    out[t] = acc;
}

// ------------------------------------------------------------------ Newton on the projected NEP
// One CTA per candidate. Each step evaluates f_i, f_i' at l, forms the residual B(l) y and
// B'(l) y from the products v_i = B_i y, builds the bordered Jacobian
// J = [[B(l), B'(l) y], [y^H, 0]] in complex64 and solves J [dy; dl] = -[B(l) y; 0] by Gaussian
// elimination with partial pivoting in FP32 (rows are never moved: the pivot row of each
// column is recorded and later columns skip it; one CTA barrier per column, the next pivot
// found by the warp that updated that column). While the step is large, the residual is formed
// in FP32 from the complex64 copies of the B_i: the iterate is then far from the FP64 fixed
// point anyway. Once |dl| <= 1e-5 max(1, |l|), or the FP32 steps stop shrinking below 1e-3, the
// residual is formed in FP64 from the FP64 B_i and y, so the iteration converges to the FP64
// solution (the FP32 Jacobian only makes that final convergence linear, rate ~ kappa(J) 6e-8).
// The stopping test |dl| <= tol max(1, |l|) is applied to FP64 steps only.
__device__ __forceinline__ zf shfl_cx32(zf v, int src) {
    return mk(__shfl_sync(0xffffffffu, v.re, src), __shfl_sync(0xffffffffu, v.im, src));
}
struct NewtonLayout {
    size_t J, rhs, rpv, y32, B32, y, fv, vb, prow, used, total;
};
__host__ __device__ inline NewtonLayout newton_layout(int k, int nterms) {
    const size_t K1 = (size_t)k + 1;
    NewtonLayout L{};
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o += (bytes + 15) / 16 * 16;
        return at;
    };
    L.J = take(sizeof(zf) * K1 * K1);
    L.rhs = take(sizeof(zf) * K1);
    L.rpv = take(sizeof(zf) * K1);
    L.y32 = take(sizeof(zf) * K1);
    L.B32 = take(sizeof(zf) * (size_t)nterms * k * k);
    L.y = take(sizeof(zd) * K1);
    L.fv = take(sizeof(zd) * 2 * (size_t)nterms);
    L.vb = take(sizeof(zd) * (size_t)nterms * k);
    L.prow = take(sizeof(int) * K1);
    L.used = take(sizeof(int) * K1);
    L.total = o;
    return L;
}
size_t newton_scratch_bytes(int k, int nterms) { return newton_layout(k, nterms).total; }

__global__ void convert_c64_kernel(int64_t count, const zd* __restrict__ in, zf* __restrict__ out) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < count) out[t] = cvt<float>(in[t]);
}

template <int MB>  // rows per lane in the elimination: K1 <= 32 MB
__global__ void __launch_bounds__(256, 1) newton_kernel(SplitDev s, int k, const zd* __restrict__ Bs,
                                                     const zf* __restrict__ Bs32, const zd* __restrict__ lam0,
                                                     const zd* __restrict__ Y0, int ldy0, zd c, double rad, double ea,
                                                     double eb, int maxit, int abandon,
                                                     double tol, zd* __restrict__ lam_out, zd* __restrict__ Yout,
                                                     int* __restrict__ ok_out, int* __restrict__ its_out,
                                                     unsigned char* __restrict__ gscratch, int use_smem,
                                                     const zd* __restrict__ fv_ext, double* __restrict__ nstate,
                                                     int steps) {
    extern __shared__ unsigned char sraw[];
    const int cand = blockIdx.x;
    const int K1 = k + 1, nt = s.nterms;
    const NewtonLayout lay = newton_layout(k, nt);
    unsigned char* base = use_smem ? sraw : gscratch + (int64_t)cand * lay.total;
    zf* J = reinterpret_cast<zf*>(base + lay.J);      // K1 x K1, column-major
    zf* rhs = reinterpret_cast<zf*>(base + lay.rhs);  // K1
    zf* rpv = reinterpret_cast<zf*>(base + lay.rpv);  // 1 / pivot of each column
    zf* y32 = reinterpret_cast<zf*>(base + lay.y32);  // complex64 copy of y
    zf* B32 = reinterpret_cast<zf*>(base + lay.B32);  // nt x k x k
    zd* y = reinterpret_cast<zd*>(base + lay.y);      // FP64 iterate
    zd* fv = reinterpret_cast<zd*>(base + lay.fv);    // f_i, f_i'
    zd* vb = reinterpret_cast<zd*>(base + lay.vb);    // v_i = B_i y, nt x k
    int* prow = reinterpret_cast<int*>(base + lay.prow);
    int* used = reinterpret_cast<int*>(base + lay.used);
    __shared__ double redd[32];
    __shared__ zf f32s[32];
    __shared__ int stop_s, fp64_s, sing_s;
    __shared__ zd lam_s;
    __shared__ double dprev_s;
    const int tid = threadIdx.x;
    const int lane = tid & 31, w = tid >> 5, nw = blockDim.x >> 5;
    // step mode (host-supplied functions): nstate[4 cand ..] = steps done, finished, FP64 phase,
    // last |dlambda|; the iterate stays in this candidate's global work area between launches, and
    // each launch runs `steps` steps with f_i, f_i' at the current iterate from fv_ext
    double* stc = nstate ? nstate + 4 * (int64_t)cand : nullptr;
    const int it0 = stc ? (int)stc[0] : 0;
    if (stc && stc[1] != 0.0) return;

    for (int64_t e = tid; e < (int64_t)nt * k * k; e += blockDim.x) B32[e] = Bs32[e];
    if (it0 > 0) {
        // resume: the iterate y (and its complex64 copy) is still in the work area
        if (tid == 0) {
            lam_s = lam_out[cand];
            stop_s = 0;
            fp64_s = stc[2] != 0.0;
            dprev_s = stc[3];
        }
        __syncthreads();
    }
    double ss = 0.0;
    int ok = 1, it = 0;
    if (it0 == 0) {
        for (int i = tid; i < k; i += blockDim.x) {
            y[i] = Y0[(int64_t)cand * ldy0 + i];
            ss += norm2(y[i]);
        }
        for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
        if (lane == 0) redd[w] = ss;
        __syncthreads();
        if (tid == 0) {
            double t = 0;
            for (int q = 0; q < nw; ++q) t += redd[q];
            redd[0] = t;
            lam_s = lam0[cand];
            stop_s = 0;
            fp64_s = 0;
            dprev_s = 0.0;
        }
        __syncthreads();
        {
            const double inv = redd[0] > 0 ? 1.0 / sqrt(redd[0]) : 0.0;
            for (int i = tid; i < k; i += blockDim.x) {
                y[i] = inv * y[i];
                y32[i] = cvt<float>(y[i]);
            }
        }
        ok = redd[0] > 0;
    } else {
        ok = ok_out[cand];
    }
    const int itend = stc ? min(maxit, it0 + steps) : maxit;
    bool finished = false;  // stopped (converged, failed, left) rather than out of steps
    __syncthreads();
    for (it = it0 + 1; it <= itend && ok; ++it) {
        const bool fp64 = fp64_s != 0;
        if (tid < nt) {
            if (fv_ext) {
                fv[tid] = fv_ext[(int64_t)cand * 2 * nt + tid];
                fv[nt + tid] = fv_ext[(int64_t)cand * 2 * nt + nt + tid];
            } else {
                const FnEval fe = fn_eval(s.fn_nodes, s.fn_coef, s.fn_root[tid], lam_s);
                fv[tid] = fe.f;
                fv[nt + tid] = fe.df;
            }
        }
        for (int r = tid; r < K1; r += blockDim.x) used[r] = 0;
        // v_i = B_i y, one (row, term) per thread: FP64 near the solution, FP32 before
        for (int e = tid; e < nt * k; e += blockDim.x) {
            const int i = e / k, r = e - i * k;
            zd v;
            if (fp64) {
                const zd* Bi = Bs + (int64_t)i * k * k + r;
                zd v0 = mk(0.0, 0.0), v1 = mk(0.0, 0.0);
                int q = 0;
#pragma unroll 4
                for (; q + 1 < k; q += 2) {
                    v0 = fma_(v0, Bi[(int64_t)k * q], y[q]);
                    v1 = fma_(v1, Bi[(int64_t)k * (q + 1)], y[q + 1]);
                }
                if (q < k) v0 = fma_(v0, Bi[(int64_t)k * q], y[q]);
                v = v0 + v1;
            } else {
                const zf* Bi = B32 + (int64_t)i * k * k + r;
                zf v0 = mk(0.0f, 0.0f), v1 = mk(0.0f, 0.0f);
                int q = 0;
#pragma unroll 4
                for (; q + 1 < k; q += 2) {
                    v0 = fma_(v0, Bi[(int64_t)k * q], y32[q]);
                    v1 = fma_(v1, Bi[(int64_t)k * (q + 1)], y32[q + 1]);
                }
                if (q < k) v0 = fma_(v0, Bi[(int64_t)k * q], y32[q]);
                v = cvt<double>(v0 + v1);
            }
            vb[(int64_t)i * k + r] = v;
        }
        if (tid < nt) f32s[tid] = cvt<float>(fv[tid]);
        __syncthreads();
        // J(0:k, 0:k) = B(l) in FP32 (warps over columns, lanes over rows); J(0:k, k) = B'(l) y,
        // rhs = -B(l) y; the border row y^H
        for (int q = w; q < k; q += nw)
            for (int r = lane; r < k; r += 32) {
                zf b = mk(0.0f, 0.0f);
                for (int i = 0; i < nt; ++i) b = fma_(b, f32s[i], B32[(int64_t)i * k * k + r + (int64_t)k * q]);
                J[r + (int64_t)K1 * q] = b;
            }
        for (int r = tid; r < k; r += blockDim.x) {
            zd bd = mk(0.0, 0.0), gd = mk(0.0, 0.0);
            for (int i = 0; i < nt; ++i) {
                const zd v = vb[(int64_t)i * k + r];
                bd = fma_(bd, fv[i], v);
                gd = fma_(gd, fv[nt + i], v);
            }
            rhs[r] = cvt<float>(-bd);
            J[r + (int64_t)K1 * k] = cvt<float>(gd);
        }
        for (int q = tid; q < k; q += blockDim.x) J[k + (int64_t)K1 * q] = cvt<float>(conj(y[q]));
        if (tid == 0) {
            J[k + (int64_t)K1 * k] = mk(0.0f, 0.0f);
            rhs[k] = mk(0.0f, 0.0f);
            sing_s = 0;
        }
        __syncthreads();
        // Gaussian elimination with row indirection. A lane keeps its rows r = lane + 32 b
        // (b < nb) in registers while it sweeps the columns of its warp; the multipliers of a
        // column are formed once per lane. Warp 0 takes column col+1 first and finds its pivot
        // (the first row maximising |Re|+|Im| among the rows that are not pivots yet) from the
        // values it has just computed.
        const int nb = (K1 + 31) >> 5;  // <= MB
        // value of row r from the lane that holds it (all lanes call)
        auto v_at = [&](const zf (&v)[MB], int r) {
            const int br = r >> 5;
            zf own = v[0];
#pragma unroll
            for (int b2 = 1; b2 < MB; ++b2)
                if (b2 == br) own = v[b2];
            return shfl_cx32(own, r & 31);
        };
        auto pick = [&](const zf (&v)[MB], const bool (&act)[MB], int col) {
            float best = -1.0f;
            int bi = K1;
#pragma unroll
            for (int b2 = 0; b2 < MB; ++b2)
                if (b2 < nb && act[b2]) {
                    const float a = abs1(v[b2]);
                    if (a > best) { best = a; bi = lane + 32 * b2; }
                }
            for (int o = 16; o > 0; o >>= 1) {
                const float ob = __shfl_xor_sync(0xffffffffu, best, o);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
            }
            const bool okp = best > 0.0f && bi < K1;  // the same in every lane after the butterfly
            const zf pv = v_at(v, okp ? bi : 0);
            if (lane == 0) {
                prow[col] = okp ? bi : -1;
                if (okp) rpv[col] = cdiv(mk(1.0f, 0.0f), pv);
            }
        };
        if (w == 0) {
            zf v[MB];
            bool act[MB];
#pragma unroll
            for (int b2 = 0; b2 < MB; ++b2) {
                const int r = lane + 32 * b2;
                act[b2] = b2 < nb && r < K1;
                v[b2] = act[b2] ? J[r] : mk(0.0f, 0.0f);
            }
            pick(v, act, 0);
        }
        __syncthreads();
        for (int col = 0; col < K1; ++col) {
            const int p = prow[col];
            if (p < 0) break;  // uniform: every thread reads the same value after the barrier
            const zf rp = rpv[col];
            // rows that are not pivots yet (row p is excluded explicitly: its used flag is set
            // during this phase) and their multipliers
            bool act[MB];
            zf g[MB];
#pragma unroll
            for (int b2 = 0; b2 < MB; ++b2) {
                const int r = lane + 32 * b2;
                act[b2] = b2 < nb && r < K1 && r != p && !used[r];
                g[b2] = act[b2] ? J[r + (int64_t)K1 * col] * rp : mk(0.0f, 0.0f);
            }
            for (int q = col + 1 + w; q <= K1; q += nw) {
                zf* jq = q < K1 ? J + (int64_t)K1 * q : rhs;
                const zf u = jq[p];
                zf v[MB];
#pragma unroll
                for (int b2 = 0; b2 < MB; ++b2)
                    if (act[b2]) v[b2] = jq[lane + 32 * b2];
#pragma unroll
                for (int b2 = 0; b2 < MB; ++b2)
                    if (act[b2]) {
                        v[b2] = fms(v[b2], g[b2], u);
                        jq[lane + 32 * b2] = v[b2];
                    }
                if (w == 0 && q == col + 1 && q < K1) pick(v, act, q);
            }
            if (tid == 0) used[p] = 1;
            __syncthreads();
        }
        // singular bordered system (some column had no nonzero pivot)
        if (tid == 0) {
            int sg = 0;
            for (int col = 0; col < K1; ++col) sg |= prow[col] < 0;
            sing_s = sg;
        }
        __syncthreads();
        if (sing_s) { ok = 0; finished = true; break; }
        // back substitution in pivot order (warp 0): lane holds the transformed right-hand sides of
        // the pivots i = lane + 32 b; x_col = rhs(col) / U(col, col), then every earlier pivot row
        // drops x_col times its entry in column col. The solution goes to y32 (rebuilt below).
        if (w == 0) {
            zf rv[MB];
            int pr[MB];
#pragma unroll
            for (int b2 = 0; b2 < MB; ++b2) {
                const int i = lane + 32 * b2;
                pr[b2] = (b2 < nb && i < K1) ? prow[i] : 0;
                rv[b2] = (b2 < nb && i < K1) ? rhs[pr[b2]] : mk(0.0f, 0.0f);
            }
            for (int col = K1 - 1; col >= 0; --col) {
                const int bc = col >> 5, lc = col & 31;
                zf own = rv[0];
#pragma unroll
                for (int b2 = 1; b2 < MB; ++b2)
                    if (b2 == bc) own = rv[b2];
                const zf x = shfl_cx32(own, lc) * rpv[col];
                if (lane == lc) y32[col] = x;
#pragma unroll
                for (int b2 = 0; b2 < MB; ++b2) {
                    const int i = lane + 32 * b2;
                    if (b2 < nb && i < col) rv[b2] = fms(rv[b2], J[pr[b2] + (int64_t)K1 * col], x);
                }
            }
        }
        __syncthreads();
        double s2 = 0.0;
        for (int i = tid; i < k; i += blockDim.x) {
            y[i] = y[i] + cvt<double>(y32[i]);
            s2 += norm2(y[i]);
        }
        for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        __syncthreads();
        if (lane == 0) redd[w] = s2;
        __syncthreads();
        if (tid == 0) {
            double t = 0;
            for (int q = 0; q < nw; ++q) t += redd[q];
            redd[0] = t;
            const zd dl = cvt<double>(y32[k]);
            const zd nl = lam_s + dl;
            lam_s = nl;
            const double al = hypot(nl.re, nl.im), ad = hypot(dl.re, dl.im);
            // st: 1 converged, 2 failed (not finite, zero iterate), 3 left the region (beyond the
            // disc |l - c| <= rad, or unconverged after `abandon` steps and outside Gamma by 10%:
            // a shortcut for candidates whose iterates end outside, where acceptance drops them;
            // abandon = 0 turns it off)
            int st = 0;
            if (!isfinite(nl.re) || !isfinite(nl.im) || !(t > 0)) st = 2;
            else if (hypot(nl.re - c.re, nl.im - c.im) > rad) st = 3;
            else if (fp64 && ad <= tol * fmax(1.0, al)) st = 1;
            if (st == 0 && abandon > 0 && it >= abandon) {
                const double qx = (nl.re - c.re) / ea, qy = (nl.im - c.im) / eb;
                if (qx * qx + qy * qy > 1.21) st = 3;
            }
            if (!fp64 && (ad <= 1e-5 * fmax(1.0, al) || (it > 2 && ad > 0.5 * dprev_s && ad <= 1e-3 * fmax(1.0, al))))
                fp64_s = 1;
            dprev_s = ad;
            stop_s = st;
        }
        __syncthreads();
        const double inv = redd[0] > 0 ? 1.0 / sqrt(redd[0]) : 0.0;
        for (int i = tid; i < k; i += blockDim.x) {
            y[i] = inv * y[i];
            y32[i] = cvt<float>(y[i]);
        }
        __syncthreads();
        if (stop_s == 2) { ok = 0; finished = true; break; }
        if (stop_s == 3) { ok = 2; finished = true; break; }
        if (stop_s == 1) { finished = true; break; }
    }
    if (!ok) finished = true;
    const int done_its = finished ? it : it - 1;  // steps taken so far
    for (int i = tid; i < k; i += blockDim.x) Yout[(int64_t)cand * k + i] = y[i];
    if (tid == 0) {
        lam_out[cand] = lam_s;
        ok_out[cand] = ok;
        its_out[cand] = min(done_its, maxit);
        if (stc) {
            stc[0] = done_its;
            stc[1] = (finished || done_its >= maxit) ? 1.0 : 0.0;
            stc[2] = fp64_s ? 1.0 : 0.0;
            stc[3] = dprev_s;
        }
    }
}

int launch_newton(const SplitDev& s, int k, int ncand, const zd* Bs, zf* Bs32, const zd* lam0, const zd* Y0, int ldy0,
                  zd c, double rad, double ea, double eb, int maxit, int abandon, double tol, zd* lam_out, zd* Yout, int* ok,
                  int* its, unsigned char* gscratch, cudaStream_t st, const zd* fv_ext, double* nstate, int steps) {
    if (ncand <= 0) return NEP_OK;
    const int64_t nb = (int64_t)s.nterms * k * k;
    convert_c64_kernel<<<(int)((nb + 255) / 256), 256, 0, st>>>(nb, Bs, Bs32);
    NEP_CHECK_LAUNCH();
    const size_t bytes = newton_scratch_bytes(k, s.nterms);
    const int use_smem = bytes <= 200 * 1024 && !nstate;  // step mode keeps the iterate in global memory
    if (!use_smem && !gscratch) return NEP_ERR_INTERNAL;
    auto run = [&](auto kern) -> int {
        if (use_smem) NEP_CUDA(allow_max_dynamic_smem(kern));
        kern<<<ncand, 256, use_smem ? bytes : 0, st>>>(s, k, Bs, Bs32, lam0, Y0, ldy0, c, rad, ea, eb, maxit, abandon, tol,
                                                       lam_out, Yout, ok, its, gscratch, use_smem, fv_ext,
                                                       nstate, steps);
        NEP_CHECK_LAUNCH();
        return NEP_OK;
    };
    const int K1 = k + 1;
    if (K1 <= 64) return run(newton_kernel<2>);
    if (K1 <= 96) return run(newton_kernel<3>);
    if (K1 <= 160) return run(newton_kernel<5>);
    if (K1 <= 288) return run(newton_kernel<9>);
    set_error("projected Newton: basis of %d vectors exceeds 287", k);
    return NEP_ERR_UNSUPPORTED;
}

// ------------------------------------------------------------------ residuals and selection
// eta_c = |sum_i f_i(l_c) A_i x_c|_2 / (sum_i |f_i(l_c)| |A_i|_inf |x_c|_2), one CTA per pair.
// fv_ext (or nullptr): f_i(l_c) from the host, at fv_ext[c * 2 nterms + i], for host-supplied functions.
__global__ void __launch_bounds__(256) eta_kernel(SplitDev s, const zd* __restrict__ lam, const zd* __restrict__ X,
                                                  double* __restrict__ eta, const zd* __restrict__ fv_ext) {
    __shared__ zd fv[32];
    __shared__ double red[2][32];
    const int cnd = blockIdx.x;
    if (threadIdx.x < s.nterms)
        fv[threadIdx.x] = fv_ext ? fv_ext[(int64_t)cnd * 2 * s.nterms + threadIdx.x]
                                 : fn_eval(s.fn_nodes, s.fn_coef, s.fn_root[threadIdx.x], lam[cnd]).f;
    __syncthreads();
    const zd* x = X + (int64_t)cnd * s.n;
    double rr = 0.0, xx = 0.0;
    for (int r = threadIdx.x; r < s.n; r += blockDim.x) {
        zd acc = mk(0.0, 0.0);
        for (int64_t e = s.rowptr[r]; e < s.rowptr[r + 1]; ++e) {
            zd t = mk(0.0, 0.0);
            for (int i = 0; i < s.nterms; ++i) {
                const zd a = mk(s.val[(int64_t)i * s.nnz + e], s.val_im ? s.val_im[(int64_t)i * s.nnz + e] : 0.0);
                t = fma_(t, fv[i], a);
            }
            acc = fma_(acc, t, x[s.col[e]]);
        }
        rr += norm2(acc);
        xx += norm2(x[r]);
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        rr += __shfl_xor_sync(0xffffffffu, rr, o);
        xx += __shfl_xor_sync(0xffffffffu, xx, o);
    }
    if (lane == 0) { red[0][w] = rr; red[1][w] = xx; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0, b = 0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) { a += red[0][q]; b += red[1][q]; }
        double den = 0;
        for (int i = 0; i < s.nterms; ++i) den += hypot(fv[i].re, fv[i].im) * s.norms[i];
        eta[cnd] = (den > 0 && b > 0) ? sqrt(a) / (den * sqrt(b)) : INFINITY;
    }
}

// Keep candidates inside the ellipse with eta <= eig_tol and a Newton run that neither failed nor
// left the region (ok == 1); drop
// duplicates (|dl| <= 1e-10 max(1,|l|) and |x_a^H x_b| >= 1 - 1e-8; keep the smaller eta);
// order by (Re, Im). order_out[0] = count, then the selected candidate indices.
__global__ void select_kernel(int ncand, const zd* __restrict__ lam, const double* __restrict__ eta,
                              const int* __restrict__ ok, const zd* __restrict__ G, zd c, double ea, double eb,
                              double eig_tol, int* __restrict__ order_out) {
    extern __shared__ int sidx[];
    int* keep = sidx;            // ncand
    int* byeta = sidx + ncand;   // ncand
    if (threadIdx.x != 0) return;
    int nk = 0;
    for (int a = 0; a < ncand; ++a) {
        const zd d = lam[a] - c;
        const double q = (d.re / ea) * (d.re / ea) + (d.im / eb) * (d.im / eb);
        if (ok[a] == 1 && q < 1.0 && eta[a] <= eig_tol) byeta[nk++] = a;
    }
    // insertion sort by eta (stable)
    for (int i = 1; i < nk; ++i) {
        const int v = byeta[i];
        int p = i - 1;
        while (p >= 0 && eta[byeta[p]] > eta[v]) { byeta[p + 1] = byeta[p]; --p; }
        byeta[p + 1] = v;
    }
    int na = 0;
    for (int i = 0; i < nk; ++i) {
        const int a = byeta[i];
        bool dup = false;
        for (int q = 0; q < na && !dup; ++q) {
            const int b = keep[q];
            const zd d = lam[a] - lam[b];
            const double la = hypot(lam[a].re, lam[a].im);
            const zd ip = G[a + (int64_t)ncand * b];
            if (hypot(d.re, d.im) <= 1e-10 * fmax(1.0, la) && hypot(ip.re, ip.im) >= 1.0 - 1e-8) dup = true;
        }
        if (!dup) keep[na++] = a;
    }
    // order by (Re, Im)
    for (int i = 1; i < na; ++i) {
        const int v = keep[i];
        int p = i - 1;
        while (p >= 0 && (lam[keep[p]].re > lam[v].re || (lam[keep[p]].re == lam[v].re && lam[keep[p]].im > lam[v].im))) {
            keep[p + 1] = keep[p];
            --p;
        }
        keep[p + 1] = v;
    }
    order_out[0] = na;
    for (int i = 0; i < na; ++i) order_out[1 + i] = keep[i];
}

}  // namespace nep

namespace nep {

// ------------------------------------------------------------------ small helpers and launchers
__global__ void scale_cols_kernel(int rows, int cols, zd* __restrict__ X, int ld, const double* __restrict__ s,
                                  int mode) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)rows * cols) return;
    const int r = (int)(t % rows), c = (int)(t / rows);
    const double v = s[c];
    const double f = mode == 0 ? (v > 0 ? 1.0 / v : 0.0) : (v > 0 ? 1.0 / sqrt(v) : 0.0);
    X[r + (int64_t)ld * c] = f * X[r + (int64_t)ld * c];
}

__global__ void scale_rows_kernel(int rows, int cols, zd* __restrict__ X, int ld, const double* __restrict__ s) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)rows * cols) return;
    const int r = (int)(t % rows), c = (int)(t / rows);
    const double v = s[r];
    X[r + (int64_t)ld * c] = (v > 0 ? 1.0 / v : 0.0) * X[r + (int64_t)ld * c];
}

__global__ void candidates_kernel(int m, const zd* __restrict__ theta, zd c, double a, zd* __restrict__ lam) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < m) lam[t] = c + a * theta[t];
}

__global__ void fill_int_kernel(int n, int* __restrict__ p, int v) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) p[t] = v;
}

// count of sigma_i > tol * sigma_0 (sigma descending)
__global__ void rank_kernel(int n, const double* __restrict__ sigma, double tol, int* __restrict__ out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int m = 0;
    if (n > 0 && sigma[0] > 0)
        for (int i = 0; i < n; ++i) m += sigma[i] > tol * sigma[0];
    *out = m;
}

int launch_scale_cols(int rows, int cols, zd* X, int ld, const double* s, int mode, cudaStream_t st) {
    if (rows <= 0 || cols <= 0) return NEP_OK;
    scale_cols_kernel<<<ceil_div((int64_t)rows * cols, 256), 256, 0, st>>>(rows, cols, X, ld, s, mode);
    NEP_CHECK_LAUNCH();
    return NEP_OK;
}
int launch_scale_rows(int rows, int cols, zd* X, int ld, const double* s, cudaStream_t st) {
    if (rows <= 0 || cols <= 0) return NEP_OK;
    scale_rows_kernel<<<ceil_div((int64_t)rows * cols, 256), 256, 0, st>>>(rows, cols, X, ld, s);
    NEP_CHECK_LAUNCH();
    return NEP_OK;
}
int launch_candidates(int m, const zd* theta, zd c, double a, zd* lam, cudaStream_t st) {
    if (m <= 0) return NEP_OK;
    candidates_kernel<<<ceil_div(m, 128), 128, 0, st>>>(m, theta, c, a, lam);
    NEP_CHECK_LAUNCH();
    return NEP_OK;
}
int launch_fill_int(int n, int* p, int v, cudaStream_t st) {
    if (n <= 0) return NEP_OK;
    fill_int_kernel<<<ceil_div(n, 256), 256, 0, st>>>(n, p, v);
    NEP_CHECK_LAUNCH();
    return NEP_OK;
}
int launch_rank(int n, const double* sigma, double tol, int* out, cudaStream_t st) {
    rank_kernel<<<1, 32, 0, st>>>(n, sigma, tol, out);
    NEP_CHECK_LAUNCH();
    return NEP_OK;
}
int launch_normalize_columns(int rows, int cols, zd* X, int fix_phase, double* nrm, cudaStream_t st) {
    if (cols <= 0) return NEP_OK;
    normalize_columns_kernel<<<cols, 256, 0, st>>>(rows, X, fix_phase, nrm);
    NEP_CHECK_LAUNCH();
    return NEP_OK;
}
int launch_term_spmm(const SplitDev& s, int k, const zd* Q, zd* out, cudaStream_t st) {
    if (k <= 0) return NEP_OK;
    const int64_t tot = (int64_t)s.n * k * s.nterms;
    term_spmm_kernel<<<ceil_div(tot, 256), 256, 0, st>>>(s, k, Q, out);
    NEP_CHECK_LAUNCH();
    return NEP_OK;
}
int launch_eta(const SplitDev& s, int ncand, const zd* lam, const zd* X, double* eta, cudaStream_t st,
               const zd* fv_ext) {
    if (ncand <= 0) return NEP_OK;
    eta_kernel<<<ncand, 256, 0, st>>>(s, lam, X, eta, fv_ext);
    NEP_CHECK_LAUNCH();
    return NEP_OK;
}
int launch_select(int ncand, const zd* lam, const double* eta, const int* ok, const zd* G, zd c, double ea, double eb,
                  double eig_tol, int* order, cudaStream_t st) {
    select_kernel<<<1, 32, sizeof(int) * 2 * (ncand > 0 ? ncand : 1), st>>>(ncand, lam, eta, ok, G, c, ea, eb, eig_tol,
                                                                            order);
    NEP_CHECK_LAUNCH();
    return NEP_OK;
}

}  // namespace nep

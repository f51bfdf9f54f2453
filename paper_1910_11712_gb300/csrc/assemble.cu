// Kernel (a): split-form assembly of the shifted matrices T(z_j) = sum_i f_i(z_j) A_i
// (Sec. 2 Eq. (split); Sec. 3.2.2 builds T(lambda) from the f_i values and l-1 sparse
// axpys) for every quadrature point at once, written straight into the row-oriented band
// storage that the banded LU consumes.
//
// One warp per (point, row): the warp zero-fills the row's ldab slots with coalesced
// stores, then scatters the union-pattern entries sum_i F[i,j] a_i(r,k) (FP64 sum, one
// rounding to the storage type) to slot k - r + kl. The FP64 row sums of |t_rk| give
// ||T(z_j)||_inf for the refinement's backward error; the FP64 values of T(z_j) on the
// union pattern (tval) feed the FP64 residual of the refinement. Bound: HBM writes (n*ldab elements
// per point).
#include "nep_common.cuh"

namespace nep {

__device__ __forceinline__ void atomic_max_nonneg(double* addr, double v) {
    // non-negative doubles order like their bit patterns
    atomicMax(reinterpret_cast<unsigned long long*>(addr), (unsigned long long)__double_as_longlong(v));
}

template <typename T>
__global__ void __launch_bounds__(256) assemble_band_kernel(SplitDev s, int npts, const zd* __restrict__ F,
                                                            cx<T>* __restrict__ ab, double* __restrict__ tnorm,
                                                            zd* __restrict__ tval) {
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t total = (int64_t)npts * s.n;
    if (gw >= total) return;
    const int j = (int)(gw / s.n);
    const int r = (int)(gw - (int64_t)j * s.n);
    cx<T>* row = ab ? ab + ((int64_t)j * s.n + r) * s.ldab : nullptr;
    if (row)
        for (int t = lane; t < s.ldab; t += 32) row[t] = mk<T>(0, 0);
    __syncwarp();
    const int64_t e0 = s.rowptr[r], e1 = s.rowptr[r + 1];
    double rowsum = 0.0;
    for (int64_t e = e0 + lane; e < e1; e += 32) {
        zd v = mk(0.0, 0.0);
        for (int i = 0; i < s.nterms; ++i) {
            zd f = F[i + (int64_t)s.nterms * j];
            zd a = mk(s.val[(int64_t)i * s.nnz + e], s.val_im ? s.val_im[(int64_t)i * s.nnz + e] : 0.0);
            v = fma_(v, f, a);
        }
        const int k = s.col[e];
        if (row) row[k - r + s.kl] = cvt<T>(v);
        if (tval) tval[(int64_t)j * s.nnz + e] = v;
        rowsum += hypot(v.re, v.im);
    }
    for (int o = 16; o > 0; o >>= 1) rowsum += __shfl_xor_sync(0xffffffffu, rowsum, o);
    if (lane == 0 && tnorm) atomic_max_nonneg(tnorm + j, rowsum);
}

template <typename T>
int launch_assemble(const SplitDev& s, int npts, const zd* F, cx<T>* ab, double* tnorm, zd* tval, cudaStream_t st) {
    if (npts <= 0) return NEP_OK;
    if (tnorm) NEP_CUDA(cudaMemsetAsync(tnorm, 0, sizeof(double) * npts, st));
    const int64_t warps = (int64_t)npts * s.n;
    const int blocks = ceil_div(warps * 32, 256);
    assemble_band_kernel<T><<<blocks, 256, 0, st>>>(s, npts, F, ab, tnorm, tval);
    NEP_CHECK_LAUNCH();
    return NEP_OK;
}

template int launch_assemble<float>(const SplitDev&, int, const zd*, cx<float>*, double*, zd*, cudaStream_t);
template int launch_assemble<double>(const SplitDev&, int, const zd*, cx<double>*, double*, zd*, cudaStream_t);

}  // namespace nep

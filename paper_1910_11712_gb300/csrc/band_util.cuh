// Device helpers shared by the banded LU and the banded substitution kernels.
#pragma once
#include "nep_common.cuh"

namespace nep {

template <typename T>
__device__ __forceinline__ cx<T> shfl_cx(cx<T> v, int src) {
    cx<T> r;
    r.re = __shfl_sync(0xffffffffu, v.re, src);
    r.im = __shfl_sync(0xffffffffu, v.im, src);
    return r;
}

__device__ __forceinline__ int posmod(int a, int m) {
    int r = a % m;
    return r < 0 ? r + m : r;
}


// Asynchronous global->shared copy of one complex element (8 or 16 bytes); completion is
// awaited with cp_async_wait_all() before the barrier that publishes the data.
template <typename T>
__device__ __forceinline__ void cp_async_cx(cx<T>* smem, const cx<T>* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    if constexpr (sizeof(cx<T>) == 16) {
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
    } else {
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
    }
}
__device__ __forceinline__ void cp_async_f32(float* smem, const float* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_i32(int* smem, const int* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait_group() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// 1/v for a nonzero pivot: conj(v) / |v|^2 with one correctly rounded reciprocal, where |v|^2 is
// safely inside the normal range (the common case); Smith's scaled division otherwise.
template <typename T>
__device__ __forceinline__ cx<T> pivot_recip(cx<T> v) {
    const T m = fmax(fabs(v.re), fabs(v.im));
    const T lo = sizeof(T) == 4 ? T(1e-15) : T(1e-150), hi = sizeof(T) == 4 ? T(1e15) : T(1e150);
    if (m >= lo && m <= hi) {
        const T d = v.re * v.re + v.im * v.im;
        T r;
        if constexpr (sizeof(T) == 4) r = __frcp_rn(d);
        else r = __drcp_rn(d);
        return mk<T>(v.re * r, -v.im * r);
    }
    return cdiv(mk<T>(1, 0), v);
}

template <typename T, int RPL>
__device__ __forceinline__ cx<T> sel_reg(const cx<T> (&a)[RPL], int q) {
    cx<T> v = a[0];
#pragma unroll
    for (int t = 1; t < RPL; ++t)
        if (t == q) v = a[t];
    return v;
}
template <typename T, int RPL>
__device__ __forceinline__ void set_reg(cx<T> (&a)[RPL], int q, cx<T> v) {
#pragma unroll
    for (int t = 0; t < RPL; ++t)
        if (t == q) a[t] = v;
}

}  // namespace nep

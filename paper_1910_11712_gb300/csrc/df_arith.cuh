// Double-float arithmetic on FP32 pairs: a value is the unevaluated sum hi + lo (about 48
// significant bits). Error-free transformations: Knuth's two-sum, and the product error by fma.
// These run on the FP32 pipe, which issues about 68 times faster than FP64 on this part. The
// products and sums use the _rn intrinsics, which the compiler never fuses into an fma: a fused
// multiply-add inside a two-sum would break its error-free property.
#pragma once

namespace nep {

__device__ __forceinline__ void df_two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void df_quick_two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}
// (h, l) -= (ah, al) (bh, bl)
__device__ __forceinline__ void df_fms(float& h, float& l, float ah, float al, float bh, float bl) {
    const float p = __fmul_rn(ah, bh);
    float pe = fmaf(ah, bh, -p);
    pe = fmaf(ah, bl, fmaf(al, bh, pe));
    float s, e;
    df_two_sum(h, -p, s, e);
    e += l - pe;
    df_quick_two_sum(s, e, h, l);
}
// (h, l) += d
__device__ __forceinline__ void df_add1(float& h, float& l, float d) {
    float s, e;
    df_two_sum(h, d, s, e);
    e += l;
    df_quick_two_sum(s, e, h, l);
}

// (h, l) += (ah, al) (bh, bl)
__device__ __forceinline__ void df_fma(float& h, float& l, float ah, float al, float bh, float bl) {
    const float p = __fmul_rn(ah, bh);
    float pe = fmaf(ah, bh, -p);
    pe = fmaf(ah, bl, fmaf(al, bh, pe));
    float s, e;
    df_two_sum(h, p, s, e);
    e += l + pe;
    df_quick_two_sum(s, e, h, l);
}

}  // namespace nep

// Double-float arithmetic on the float32 pipe: a value is the unevaluated sum
// h + l of two float32 numbers (|l| <= ulp(h) / 2), about 48 significant bits.
// Products are exact through fmaf (two_prod), sums through the two-sum of Knuth
// (two_sum); no float64 instruction is issued.  GB300 runs float64 at 1/64 of
// the float32 rate, so the float32-storage kernels that need more than float32
// accuracy (the pulse geometry, the focal-plane sums) use these instead.
//
// The compiler keeps IEEE semantics here (no reassociation without fast-math;
// the only contractions are the explicit fmaf calls).
#pragma once

#include <cuda_runtime.h>

namespace psatd {

struct FF {
    float h, l;
};

__host__ __device__ __forceinline__ FF ff_from(double v) {
    FF f;
    f.h = (float)v;
    f.l = (float)(v - (double)f.h);
    return f;
}
__device__ __forceinline__ FF two_sum(float a, float b) {
    const float s = a + b, bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ FF quick_two_sum(float a, float b) {   // |a| >= |b|
    const float s = a + b;
    return {s, b - (s - a)};
}
__device__ __forceinline__ FF two_prod(float a, float b) {
    const float p = a * b;
    return {p, fmaf(a, b, -p)};
}
__device__ __forceinline__ FF ff_add(FF a, FF b) {
    const FF s = two_sum(a.h, b.h);
    return quick_two_sum(s.h, s.l + (a.l + b.l));
}
__device__ __forceinline__ FF ff_sub(FF a, FF b) { return ff_add(a, {-b.h, -b.l}); }
__device__ __forceinline__ FF ff_neg(FF a) { return {-a.h, -a.l}; }
__device__ __forceinline__ FF ff_mul(FF a, FF b) {
    const FF p = two_prod(a.h, b.h);
    return quick_two_sum(p.h, fmaf(a.h, b.l, fmaf(a.l, b.h, p.l)));
}
__device__ __forceinline__ FF ff_mul_f(FF a, float b) {
    const FF p = two_prod(a.h, b);
    return quick_two_sum(p.h, fmaf(a.l, b, p.l));
}
__device__ __forceinline__ FF ff_sqr(FF a) {
    const FF p = two_prod(a.h, a.h);
    return quick_two_sum(p.h, fmaf(2.f * a.h, a.l, p.l));
}
__device__ __forceinline__ float ff_float(FF a) { return a.h + a.l; }

// complex double-float, stored as float4 {re.h, re.l, im.h, im.l}
struct CFF {
    FF re, im;
};
__device__ __forceinline__ CFF cff_load(const float4& v) { return {{v.x, v.y}, {v.z, v.w}}; }
__device__ __forceinline__ float4 cff_store(const CFF& c) { return make_float4(c.re.h, c.re.l, c.im.h, c.im.l); }
__host__ __device__ __forceinline__ float4 cff_from(double re, double im) {
    const FF r = ff_from(re), i = ff_from(im);
    return make_float4(r.h, r.l, i.h, i.l);
}
// acc += w v for a float32 complex v
__device__ __forceinline__ void cff_mac(CFF& acc, const CFF& w, float2 v) {
    acc.re = ff_add(acc.re, ff_sub(ff_mul_f(w.re, v.x), ff_mul_f(w.im, v.y)));
    acc.im = ff_add(acc.im, ff_add(ff_mul_f(w.re, v.y), ff_mul_f(w.im, v.x)));
}
// acc += w v for a real float32 v
__device__ __forceinline__ void cff_mac_real(CFF& acc, const CFF& w, float v) {
    acc.re = ff_add(acc.re, ff_mul_f(w.re, v));
    acc.im = ff_add(acc.im, ff_mul_f(w.im, v));
}
// acc += w v for a double-float complex v
__device__ __forceinline__ void cff_mac_cff(CFF& acc, const CFF& w, const CFF& v) {
    acc.re = ff_add(acc.re, ff_sub(ff_mul(w.re, v.re), ff_mul(w.im, v.im)));
    acc.im = ff_add(acc.im, ff_add(ff_mul(w.re, v.im), ff_mul(w.im, v.re)));
}
__device__ __forceinline__ CFF cff_add(const CFF& a, const CFF& b) { return {ff_add(a.re, b.re), ff_add(a.im, b.im)}; }
// sum over the 32 lanes of a warp (every lane gets the total)
__device__ __forceinline__ CFF cff_warp_sum(CFF a) {
    for (int o = 16; o > 0; o >>= 1) {
        CFF b;
        b.re.h = __shfl_xor_sync(0xffffffffu, a.re.h, o);
        b.re.l = __shfl_xor_sync(0xffffffffu, a.re.l, o);
        b.im.h = __shfl_xor_sync(0xffffffffu, a.im.h, o);
        b.im.l = __shfl_xor_sync(0xffffffffu, a.im.l, o);
        a = cff_add(a, b);
    }
    return a;
}

}  // namespace psatd

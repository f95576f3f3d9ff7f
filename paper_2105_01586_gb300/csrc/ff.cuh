// ff.cuh -- float-float ("double-single") arithmetic on the FP32 pipes.
//
// GB300 executes about 2 FP64 FMAs per clock per SM against 128 FP32 FMAs,
// so per-pixel and per-row work that needs more than FP32 precision is done
// in float-float: a value is the unevaluated sum hi + lo of two floats with
// |lo| <= ulp(hi)/2, about 48 significant bits.  The building blocks are the
// classical error-free transformations: Knuth's TwoSum (the rounding error
// of a float sum is a float and can be recovered with six additions), the
// FMA-based TwoProd (the rounding error of a float product is
// fma(a, b, -a*b)), and renormalisation by Dekker's FastTwoSum.  The code
// relies on IEEE single precision without reassociation (nvcc's default).
#pragma once

namespace fem {

struct ff {
    float hi, lo;
};

__device__ __forceinline__ ff ff_make(float a) { return ff{a, 0.0f}; }

// exact split of a double into hi + lo (lo holds the next 24 bits)
__device__ __forceinline__ ff ff_from_double(double v) {
    float hi = (float)v;
    float lo = (float)(v - (double)hi);
    return ff{hi, lo};
}

__device__ __forceinline__ double ff_to_double(ff a) { return (double)a.hi + (double)a.lo; }

// s + e == a + b exactly (any a, b)
__device__ __forceinline__ ff two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return ff{s, e};
}

// s + e == a + b exactly when |a| >= |b| (or a == 0)
__device__ __forceinline__ ff fast_two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float e = __fsub_rn(b, __fsub_rn(s, a));
    return ff{s, e};
}

// p + e == a * b exactly
__device__ __forceinline__ ff two_prod(float a, float b) {
    float p = __fmul_rn(a, b);
    float e = __fmaf_rn(a, b, -p);
    return ff{p, e};
}

__device__ __forceinline__ ff ff_add(ff a, ff b) {
    ff s = two_sum(a.hi, b.hi);
    float e = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
    return fast_two_sum(s.hi, e);
}

__device__ __forceinline__ ff ff_add_f(ff a, float b) {
    ff s = two_sum(a.hi, b);
    float e = __fadd_rn(s.lo, a.lo);
    return fast_two_sum(s.hi, e);
}

__device__ __forceinline__ ff ff_neg(ff a) { return ff{-a.hi, -a.lo}; }

__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff_neg(b)); }

// a * b for a float b
__device__ __forceinline__ ff ff_mul_f(ff a, float b) {
    ff p = two_prod(a.hi, b);
    float e = __fmaf_rn(a.lo, b, p.lo);
    return fast_two_sum(p.hi, e);
}

__device__ __forceinline__ ff ff_mul(ff a, ff b) {
    ff p = two_prod(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo));
    return fast_two_sum(p.hi, e);
}

__device__ __forceinline__ ff ff_sqr(ff a) {
    ff p = two_prod(a.hi, a.hi);
    float e = __fmaf_rn(__fadd_rn(a.hi, a.hi), a.lo, p.lo);
    return fast_two_sum(p.hi, e);
}

// multiplication by a power of two is exact on both parts
__device__ __forceinline__ ff ff_scale_pow2(ff a, float s) { return ff{a.hi * s, a.lo * s}; }

__device__ __forceinline__ ff ff_shfl_xor(ff a, int o) {
    return ff{__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)};
}

__device__ __forceinline__ ff ff_warp_sum(ff a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a = ff_add(a, ff_shfl_xor(a, o));
    return a;
}

}  // namespace fem

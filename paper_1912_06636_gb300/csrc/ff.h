// Float-float ("double-float") arithmetic on the FP32 pipe: a value is the unevaluated sum
// h + l of two FP32 numbers with |l| <= ulp(h) / 2 (after renormalisation), about 48 bits of
// significand. The building blocks are the error-free transformations of Dekker (T. J. Dekker,
// "A floating-point technique for extending the available precision", Numer. Math. 18 (1971)):
//   two_sum(a, b):  s = fl(a + b) and e with s + e = a + b exactly (Knuth's branch-free form),
//   quick(a, b):    the same when |a| >= |b| (three operations),
//   two_prod(a, b): p = fl(a b) and e = fma(a, b, -p) with p + e = a b exactly.
// On this GPU the FP64 pipe runs at about 1/60 of the FP32 rate, so a float-float operation
// (7 to 15 FP32 instructions) costs a fraction of one FP64 instruction.
//
// Error bounds (u = 2^-24): mul and fma drop the product l_a l_b and round three FMAs, a
// relative error of a few u^2 of |a b|; add rounds the sum of the low parts, an error of a few u^2
// of |a| + |b| (not of |a + b|: under cancellation the relative error of the result grows, but
// it stays bounded by the magnitudes that entered, which is the scale every tolerance of this
// project is measured against).
//
// Every operation uses the _rn intrinsics: the compiler never contracts them into FMAs, which
// would break the exactness of the transformations.
#pragma once

#ifdef __CUDACC__
#include <cuda_runtime.h>

namespace ffa {

struct F {
    float h, l;
};

__device__ __forceinline__ F make(float h, float l) { return F{h, l}; }

// Nearest float-float of an FP64 value (two conversions and one FP64 subtraction; the pair
// holds the double's 53 bits to 48 of them).
__device__ __forceinline__ F from_double(double x) {
    const float h = __double2float_rn(x);
    return F{h, __double2float_rn(__dsub_rn(x, (double)h))};
}

__device__ __forceinline__ double to_double(F x) { return __dadd_rn((double)x.h, (double)x.l); }

// s + e = a + b exactly, for |a| >= |b| (or a = 0)
__device__ __forceinline__ F quick(float a, float b) {
    const float s = __fadd_rn(a, b);
    return F{s, __fsub_rn(b, __fsub_rn(s, a))};
}

// s + e = a + b exactly, any order
__device__ __forceinline__ F two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return F{s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}

__device__ __forceinline__ F neg(F x) { return F{-x.h, -x.l}; }

// 2 x, exactly
__device__ __forceinline__ F twice(F x) { return F{__fadd_rn(x.h, x.h), __fadd_rn(x.l, x.l)}; }

// x y
__device__ __forceinline__ F mul(F x, F y) {
    const float p = __fmul_rn(x.h, y.h);
    float e = __fmaf_rn(x.h, y.h, -p);
    e = __fmaf_rn(x.h, y.l, __fmaf_rn(x.l, y.h, e));
    return quick(p, e);
}

// x b, b an FP32 number
__device__ __forceinline__ F mulf(F x, float b) {
    const float p = __fmul_rn(x.h, b);
    const float e = __fmaf_rn(x.l, b, __fmaf_rn(x.h, b, -p));
    return quick(p, e);
}

// x + y
__device__ __forceinline__ F add(F x, F y) {
    const F s = two_sum(x.h, y.h);
    return quick(s.h, __fadd_rn(s.l, __fadd_rn(x.l, y.l)));
}

__device__ __forceinline__ F sub(F x, F y) { return add(x, neg(y)); }

// a b + c with one renormalisation
__device__ __forceinline__ F fma(F a, F b, F c) {
    const float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, e));
    const F s = two_sum(p, c.h);
    return quick(s.h, __fadd_rn(s.l, __fadd_rn(e, c.l)));
}

// a b + c d with one renormalisation
__device__ __forceinline__ F dot2(F a, F b, F c, F d) {
    const float p = __fmul_rn(a.h, b.h), q = __fmul_rn(c.h, d.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, e));
    float f = __fmaf_rn(c.h, d.h, -q);
    f = __fmaf_rn(c.h, d.l, __fmaf_rn(c.l, d.h, f));
    const F s = two_sum(p, q);
    return quick(s.h, __fadd_rn(s.l, __fadd_rn(e, f)));
}

}  // namespace ffa

// A float-float value in memory (8 bytes, like the FP64 it replaces): the split path's
// evaluated basis functions. Built from an FP64 (the near-nucleus points, evaluated in FP64) or
// from a float-float result; read back as FP64 where an FP64 consumer needs it.
struct __align__(8) FF2 {
    float h, l;
    FF2() = default;
    __device__ explicit FF2(double x) {
        const ffa::F f = ffa::from_double(x);
        h = f.h;
        l = f.l;
    }
    __device__ explicit FF2(ffa::F f) : h(f.h), l(f.l) {}
    __device__ explicit operator double() const { return ffa::to_double(ffa::F{h, l}); }
    __device__ ffa::F f() const { return ffa::F{h, l}; }
};
#endif
